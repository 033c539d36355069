"""Thin ctypes binding of ``include/lbm.h`` (liblbm.so): the same names, argument
marshalling only.  Every step of the method runs in the library's CUDA kernels;
there is no CPU fallback, and loading fails loudly if the library is missing.

PyTorch provides device memory (through the ``dev_alloc``/``dev_free`` hook,
backed by its caching allocator) and streams when a caller asks for it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LBM_OK, LBM_EINVAL, LBM_EUNSUPPORTED, LBM_ENOMEM = 0, -1, -2, -3
LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ENOTCONVERGED, LBM_EIO = -4, -5, -6, -7, -8
LBM_D2Q9, LBM_D3Q19, LBM_D2Q13, LBM_D2Q25 = 0, 1, 2, 3
LBM_STENCIL_LATTICE, LBM_ISO4, LBM_ISO6, LBM_ISO8, LBM_ISO10 = 0, 4, 6, 8, 10
LBM_PSI_EXP, LBM_PSI_PENG_ROBINSON = 0, 1
LBM_BGK, LBM_MRT, LBM_BGK_EDM = 0, 1, 2
LBM_FP64, LBM_FP32_SHIFTED = 0, 1
LBM_PATH_AUTO, LBM_PATH_TWO_PASS, LBM_PATH_ONE_PASS = 0, 1, 2

Q_OF = {LBM_D2Q9: 9, LBM_D3Q19: 19, LBM_D2Q13: 13, LBM_D2Q25: 25}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lattice", ctypes.c_int), ("stencil", ctypes.c_int), ("psi", ctypes.c_int),
        ("T_over_Tc", ctypes.c_double), ("G", ctypes.c_double), ("tau", ctypes.c_double),
        ("collision", ctypes.c_int),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("precision", ctypes.c_int), ("path", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
        ("wall_rows", ctypes.c_int), ("rho_w", ctypes.c_double),
    ]


class lbm_obs(ctypes.Structure):
    _fields_ = [
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double), ("dp", ctypes.c_double),
        ("max_u", ctypes.c_double), ("mean_u", ctypes.c_double), ("mass", ctypes.c_double),
        ("mom", ctypes.c_double * 3), ("thickness", ctypes.c_double), ("step", ctypes.c_int64),
    ]

    def as_dict(self):
        return {"rho_l": self.rho_l, "rho_g": self.rho_g, "dp": self.dp, "max_u": self.max_u,
                "mean_u": self.mean_u, "mass": self.mass, "mom_x": self.mom[0],
                "mom_y": self.mom[1], "mom_z": self.mom[2], "thickness": self.thickness,
                "step": self.step}


class LbmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.lbm_strerror(code).decode() if _lib else str(code)
        detail = _lib.lbm_last_error().decode() if _lib else ""
        super().__init__(f"{where}: {msg} ({code}): {detail}")


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); identical to include/lbm.h
_SIGNATURES = {
    "lbm_params_default": (_I, [ctypes.POINTER(lbm_params)]),
    "lbm_create": (_I, [ctypes.POINTER(lbm_params), ctypes.POINTER(_P)]),
    "lbm_destroy": (_I, [_P]),
    "lbm_init_droplet": (_I, [_P, _D, _D, _D, _D]),
    "lbm_init_flat": (_I, [_P, _D, _D, _D, _I]),
    "lbm_init_from_rho": (_I, [_P, _dp]),
    "lbm_get_populations": (_I, [_P, _dp]),
    "lbm_set_populations": (_I, [_P, _dp]),
    "lbm_step": (_I, [_P, _L]),
    "lbm_step_timed": (_I, [_P, _L, _dp, _I, ctypes.POINTER(_I)]),
    "lbm_step_kernel_name": (ctypes.c_char_p, [_P, _I]),
    "lbm_schedule_report": (_I, [_P, ctypes.c_char_p, _I]),
    "lbm_set_schedule": (_I, [_P, ctypes.c_char_p]),
    "lbm_run_to_steady": (_I, [_P, _D, _L, _L, ctypes.POINTER(_L)]),
    "lbm_observables": (_I, [_P, ctypes.POINTER(lbm_obs)]),
    "lbm_get_fields": (_I, [_P, _dp, _dp]),
    "lbm_device_state": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_L),
                              ctypes.POINTER(_I)]),
    "lbm_save": (_I, [_P, ctypes.c_char_p]),
    "lbm_load": (_I, [_P, ctypes.c_char_p]),
    "lbm_bytes_per_update": (_D, [_P]),
    "lbm_moments_noalloc": (_I, [_P, _I, _I, _I, _I, _I, _D, _P, _dp]),
    "lbm_batch_create": (_I, [ctypes.POINTER(lbm_params), _dp, _I, ctypes.POINTER(_P)]),
    "lbm_batch_destroy": (_I, [_P]),
    "lbm_batch_step": (_I, [_P, _L]),
    "lbm_batch_run_to_steady": (_I, [_P, _D, _L, _L, ctypes.POINTER(_L), ctypes.POINTER(lbm_obs)]),
    "lbm_batch_observables": (_I, [_P, ctypes.POINTER(lbm_obs)]),
    "lbm_batch_get_populations": (_I, [_P, _I, _dp]),
    "lbm_batch_set_populations": (_I, [_P, _I, _dp]),
    "lbm_batch_schedule_report": (_I, [_P, ctypes.c_char_p, _I]),
    "lbm_batch_set_schedule": (_I, [_P, ctypes.c_char_p]),
    "lbm_mlp_create": (_I, [ctypes.POINTER(_P), ctypes.c_uint64]),
    "lbm_mlp_destroy": (_I, [_P]),
    "lbm_mlp_num_params": (_I, []),
    "lbm_mlp_get_params": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "lbm_mlp_set_params": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "lbm_mlp_features": (_I, [_dp, _L, ctypes.POINTER(ctypes.c_float)]),
    "lbm_mlp_predict": (_I, [_P, ctypes.POINTER(ctypes.c_float), _L, ctypes.POINTER(ctypes.c_float)]),
    "lbm_mlp_loss_grad": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _I,
                               ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_float)]),
    "lbm_mlp_train": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _L, _I, _D, _I,
                           ctypes.POINTER(_D)]),
    "lbm_mlp_save": (_I, [_P, ctypes.c_char_p]),
    "lbm_mlp_load": (_I, [ctypes.POINTER(_P), ctypes.c_char_p]),
    "lbm_init_droplet_learned": (_I, [_P, _P, _D, _D, _D, _D, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "lbm_reference_density": (_I, [_P, ctypes.POINTER(_D)]),
    "lbm_diag_wait_timeout": (_I, [_P]),
    "lbm_strerror": (ctypes.c_char_p, [_I]),
    "lbm_last_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it in-tree first if asked); raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(code, where):
    if code != LBM_OK:
        raise LbmError(code, where)
    return code


def _dptr(a):
    return a.ctypes.data_as(_dp)


# ---- the C calls under their own names ---------------------------------------------
def lbm_params_default() -> lbm_params:
    p = lbm_params()
    _check(load().lbm_params_default(ctypes.byref(p)), "lbm_params_default")
    return p


def lbm_create(params: lbm_params) -> int:
    h = _P()
    _check(load().lbm_create(ctypes.byref(params), ctypes.byref(h)), "lbm_create")
    return h.value


def lbm_destroy(ctx) -> None:
    _check(load().lbm_destroy(ctx), "lbm_destroy")


def lbm_init_droplet(ctx, rho_l, rho_g, R, width) -> None:
    _check(load().lbm_init_droplet(ctx, rho_l, rho_g, R, width), "lbm_init_droplet")


def lbm_init_flat(ctx, rho_l, rho_g, width, axis=0) -> None:
    _check(load().lbm_init_flat(ctx, rho_l, rho_g, width, axis), "lbm_init_flat")


def lbm_init_from_rho(ctx, rho: np.ndarray) -> None:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    _check(load().lbm_init_from_rho(ctx, _dptr(rho)), "lbm_init_from_rho")


def lbm_get_populations(ctx, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(load().lbm_get_populations(ctx, _dptr(out)), "lbm_get_populations")
    return out


def lbm_set_populations(ctx, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().lbm_set_populations(ctx, _dptr(f)), "lbm_set_populations")


def lbm_step(ctx, n: int) -> None:
    _check(load().lbm_step(ctx, int(n)), "lbm_step")


def lbm_step_timed(ctx, n: int):
    """n steps with CUDA events around every kernel; returns {kernel name: mean ms}."""
    ms = (ctypes.c_double * 8)()
    k = _I()
    _check(load().lbm_step_timed(ctx, int(n), ms, 8, ctypes.byref(k)), "lbm_step_timed")
    return {load().lbm_step_kernel_name(ctx, i).decode(): ms[i] for i in range(k.value)}


def lbm_step_kernel_name(ctx, i: int) -> str:
    return load().lbm_step_kernel_name(ctx, i).decode()


def lbm_schedule_report(ctx) -> dict:
    """{'chosen': name, name: ms per step, ...} of the step-schedule autotuner."""
    buf = ctypes.create_string_buffer(4096)
    _check(load().lbm_schedule_report(ctx, buf, 4096), "lbm_schedule_report")
    out = {}
    for item in buf.value.decode().split(";"):
        k, v = item.split("=")
        out[k] = v if k == "chosen" else float(v)
    return out


def lbm_set_schedule(ctx, name: str) -> None:
    _check(load().lbm_set_schedule(ctx, name.encode()), "lbm_set_schedule")


def lbm_run_to_steady(ctx, tol, max_steps, check_every=1):
    taken = _L()
    code = load().lbm_run_to_steady(ctx, tol, int(max_steps), int(check_every), ctypes.byref(taken))
    if code not in (LBM_OK, LBM_ENOTCONVERGED):
        raise LbmError(code, "lbm_run_to_steady")
    return taken.value, code == LBM_OK


def lbm_observables(ctx) -> dict:
    o = lbm_obs()
    _check(load().lbm_observables(ctx, ctypes.byref(o)), "lbm_observables")
    return o.as_dict()


def lbm_get_fields(ctx, rho_out=None, u_out=None) -> None:
    _check(load().lbm_get_fields(ctx, _dptr(rho_out) if rho_out is not None else None,
                                 _dptr(u_out) if u_out is not None else None), "lbm_get_fields")


def lbm_device_state(ctx):
    ptr, q, n, e = _P(), _I(), _L(), _I()
    _check(load().lbm_device_state(ctx, ctypes.byref(ptr), ctypes.byref(q), ctypes.byref(n),
                                   ctypes.byref(e)), "lbm_device_state")
    return ptr.value, q.value, n.value, e.value


def lbm_save(ctx, path: str) -> None:
    _check(load().lbm_save(ctx, path.encode()), "lbm_save")


def lbm_load(ctx, path: str) -> None:
    _check(load().lbm_load(ctx, path.encode()), "lbm_load")


def lbm_bytes_per_update(ctx) -> float:
    return load().lbm_bytes_per_update(ctx)


def lbm_moments_noalloc(f_dev, lattice, precision, nx, ny, nz, rho_bar=0.0, stream=None):
    """Mass and momentum (4 doubles) of a device population buffer; allocates nothing."""
    out = np.empty(4)
    _check(load().lbm_moments_noalloc(f_dev, lattice, precision, nx, ny, nz, rho_bar, stream,
                                      _dptr(out)), "lbm_moments_noalloc")
    return out


def lbm_batch_create(params_list, init) -> int:
    n = len(params_list)
    arr = (lbm_params * n)(*params_list)
    init = np.ascontiguousarray(init, dtype=np.float64).reshape(-1)
    assert init.size == 4 * n
    h = _P()
    _check(load().lbm_batch_create(arr, _dptr(init), n, ctypes.byref(h)), "lbm_batch_create")
    return h.value


def lbm_batch_destroy(b) -> None:
    _check(load().lbm_batch_destroy(b), "lbm_batch_destroy")


def lbm_batch_step(b, n: int) -> None:
    _check(load().lbm_batch_step(b, int(n)), "lbm_batch_step")


def lbm_batch_run_to_steady(b, n_domains, tol, max_steps, check_every=100):
    steps = (_L * n_domains)()
    obs = (lbm_obs * n_domains)()
    code = load().lbm_batch_run_to_steady(b, tol, int(max_steps), int(check_every), steps, obs)
    if code not in (LBM_OK, LBM_ENOTCONVERGED):
        raise LbmError(code, "lbm_batch_run_to_steady")
    return list(steps), [o.as_dict() for o in obs], code == LBM_OK


def lbm_batch_observables(b, n_domains):
    obs = (lbm_obs * n_domains)()
    _check(load().lbm_batch_observables(b, obs), "lbm_batch_observables")
    return [o.as_dict() for o in obs]


def lbm_batch_get_populations(b, d, nx, ny):
    out = np.empty(9 * nx * ny)
    _check(load().lbm_batch_get_populations(b, int(d), _dptr(out)), "lbm_batch_get_populations")
    return out.reshape(9, 1, ny, nx)


def lbm_batch_set_populations(b, d, f) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    _check(load().lbm_batch_set_populations(b, int(d), _dptr(f)), "lbm_batch_set_populations")


def lbm_batch_schedule_report(b) -> dict:
    """{'chosen': name, name: ms per step, ...} of the batch tile-shape autotuner."""
    buf = ctypes.create_string_buffer(4096)
    _check(load().lbm_batch_schedule_report(b, buf, 4096), "lbm_batch_schedule_report")
    out = {}
    for item in buf.value.decode().split(";"):
        k, v = item.split("=")
        out[k] = v if k == "chosen" else float(v)
    return out


def lbm_batch_set_schedule(b, name: str) -> None:
    _check(load().lbm_batch_set_schedule(b, name.encode()), "lbm_batch_set_schedule")


class Batch:
    """Owner of one lbm_batch: domains = list of dicts with nx, ny, G, tau,
    stencil, rho_l, rho_g, R, width."""

    def __init__(self, domains, precision=LBM_FP32_SHIFTED, stream=None, torch_alloc=False):
        self._alloc = None
        plist = []
        init = []
        for d in domains:
            p = lbm_params_default()
            p.nx, p.ny, p.nz = d["nx"], d["ny"], 1
            p.G, p.tau, p.stencil = d["G"], d["tau"], d.get("stencil", 4)
            p.precision = precision
            plist.append(p)
            init += [d["rho_l"], d["rho_g"], d["R"], d["width"]]
        if stream is not None:
            plist[0].stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        if torch_alloc:
            self._alloc = TorchAllocator(stream=stream)
            plist[0].dev_alloc = self._alloc.alloc_fn
            plist[0].dev_free = self._alloc.free_fn
        self.domains = list(domains)
        self.n = len(domains)
        self.h = lbm_batch_create(plist, init)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n):
        lbm_batch_step(self.h, n)

    def run_to_steady(self, tol, max_steps, check_every=100):
        return lbm_batch_run_to_steady(self.h, self.n, tol, max_steps, check_every)

    def observables(self):
        return lbm_batch_observables(self.h, self.n)

    def get_f(self, d):
        dd = self.domains[d]
        return lbm_batch_get_populations(self.h, d, dd["nx"], dd["ny"])

    def set_f(self, d, f):
        lbm_batch_set_populations(self.h, d, f)

    def schedule_report(self):
        return lbm_batch_schedule_report(self.h)

    def set_schedule(self, name):
        lbm_batch_set_schedule(self.h, name)


_fptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))  # noqa: E731


class MLP:
    """The warm-start network (lbm_mlp_*): parameters on the GPU, training and
    inference by the library's kernels."""

    def __init__(self, seed=1906, handle=None):
        if handle is None:
            h = _P()
            _check(load().lbm_mlp_create(ctypes.byref(h), int(seed)), "lbm_mlp_create")
            handle = h.value
        self.h = handle

    @classmethod
    def load_file(cls, path):
        h = _P()
        _check(load().lbm_mlp_load(ctypes.byref(h), path.encode()), "lbm_mlp_load")
        return cls(handle=h.value)

    def close(self):
        if getattr(self, "h", None):
            load().lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def num_params():
        return load().lbm_mlp_num_params()

    @staticmethod
    def features(raw):
        raw = np.ascontiguousarray(raw, dtype=np.float64).reshape(-1, 5)
        out = np.empty(raw.shape, dtype=np.float32)
        _check(load().lbm_mlp_features(_dptr(raw), len(raw), _fptr(out)), "lbm_mlp_features")
        return out

    def get_params(self):
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(load().lbm_mlp_get_params(self.h, _fptr(out)), "lbm_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().lbm_mlp_set_params(self.h, _fptr(p)), "lbm_mlp_set_params")

    def predict(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 5)
        y = np.empty(len(X), dtype=np.float32)
        _check(load().lbm_mlp_predict(self.h, _fptr(X), len(X), _fptr(y)), "lbm_mlp_predict")
        return y

    def loss_grad(self, X, t):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 5)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = _D()
        g = np.empty(self.num_params(), dtype=np.float32)
        _check(load().lbm_mlp_loss_grad(self.h, _fptr(X), _fptr(t), len(X), ctypes.byref(loss), _fptr(g)),
               "lbm_mlp_loss_grad")
        return loss.value, g

    def train(self, X, t, epochs, lr=1e-3, batch=4096):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 5)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = _D()
        _check(load().lbm_mlp_train(self.h, _fptr(X), _fptr(t), len(X), int(epochs), float(lr), int(batch),
                                    ctypes.byref(loss)), "lbm_mlp_train")
        return loss.value

    def save(self, path):
        _check(load().lbm_mlp_save(self.h, path.encode()), "lbm_mlp_save")


def lbm_init_droplet_learned(ctx, mlp, R, rho_l, rho_g, width):
    """Returns (used_fallback, R_eff)."""
    fb = _I()
    reff = _D()
    _check(load().lbm_init_droplet_learned(ctx, mlp.h, R, rho_l, rho_g, width, ctypes.byref(fb),
                                           ctypes.byref(reff)), "lbm_init_droplet_learned")
    return bool(fb.value), reff.value


def lbm_reference_density(ctx) -> float:
    v = _D()
    _check(load().lbm_reference_density(ctx, ctypes.byref(v)), "lbm_reference_density")
    return v.value


def lbm_diag_wait_timeout(ctx) -> int:
    """Runs the bounded-wait probe; returns the library's code (LBM_ETIMEOUT expected)."""
    return int(_lib.lbm_diag_wait_timeout(ctx))


def lbm_strerror(code: int) -> str:
    return load().lbm_strerror(code).decode()


# ---- PyTorch plumbing: caching-allocator hook and streams ------------------------------
class TorchAllocator:
    """dev_alloc / dev_free callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, device=None, stream=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)
        self.live = 0
        self.calls = 0

    def _alloc(self, nbytes, _ctx):
        try:
            p = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None
        self.live += 1
        self.calls += 1
        return p

    def _free(self, ptr, _ctx):
        if ptr:
            self._torch.cuda.caching_allocator_delete(ptr)
            self.live -= 1


class Domain:
    """Convenience owner of one lbm_ctx; numpy in, numpy out."""

    def __init__(self, nx, ny, nz=1, lattice=LBM_D2Q9, stencil=LBM_STENCIL_LATTICE, psi=LBM_PSI_EXP,
                 T_over_Tc=0.0, G=-5.0, tau=1.0, collision=LBM_BGK, s_e=1.64, s_eps=1.54, s_q=1.9,
                 precision=LBM_FP64, path=LBM_PATH_AUTO, stream=None, torch_alloc=False, wall_rows=0, rho_w=1.0):
        p = lbm_params_default()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.lattice, p.stencil, p.psi = lattice, stencil, psi
        p.T_over_Tc, p.G, p.tau = T_over_Tc, G, tau
        p.collision, p.s_e, p.s_eps, p.s_q = collision, s_e, s_eps, s_q
        p.precision, p.path = precision, path
        p.wall_rows, p.rho_w = wall_rows, rho_w
        self._alloc = None
        if stream is not None:
            p.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        if torch_alloc:
            self._alloc = TorchAllocator(stream=stream)
            p.dev_alloc = self._alloc.alloc_fn
            p.dev_free = self._alloc.free_fn
        self.params = p
        self.Q = Q_OF[lattice]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.ctx = lbm_create(p)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_droplet(self, rho_l, rho_g, R, width):
        lbm_init_droplet(self.ctx, rho_l, rho_g, R, width)

    def init_flat(self, rho_l, rho_g, width, axis=0):
        lbm_init_flat(self.ctx, rho_l, rho_g, width, axis)

    def init_from_rho(self, rho):
        lbm_init_from_rho(self.ctx, np.asarray(rho, dtype=np.float64).reshape(-1))

    def init_droplet_learned(self, mlp, R, rho_l, rho_g, width):
        return lbm_init_droplet_learned(self.ctx, mlp, R, rho_l, rho_g, width)

    def get_f(self):
        out = np.empty(self.Q * self.N)
        lbm_get_populations(self.ctx, out)
        return out.reshape((self.Q,) + self.shape)

    def set_f(self, f):
        lbm_set_populations(self.ctx, np.asarray(f, dtype=np.float64).reshape(-1))

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def schedule_report(self):
        return lbm_schedule_report(self.ctx)

    def set_schedule(self, name):
        lbm_set_schedule(self.ctx, name)

    def step_timed(self, n=1):
        return lbm_step_timed(self.ctx, n)

    def run_to_steady(self, tol, max_steps, check_every=1):
        return lbm_run_to_steady(self.ctx, tol, max_steps, check_every)

    def observables(self):
        return lbm_observables(self.ctx)

    def fields(self):
        rho = np.empty(self.N)
        u = np.empty(3 * self.N)
        lbm_get_fields(self.ctx, rho, u)
        return {"rho": rho.reshape(self.shape), "u": u.reshape(self.shape + (3,))}

    def save(self, path):
        lbm_save(self.ctx, path)

    def load(self, path):
        lbm_load(self.ctx, path)

    def bytes_per_update(self):
        return lbm_bytes_per_update(self.ctx)
