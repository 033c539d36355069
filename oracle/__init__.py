"""Plain FP64 CPU oracle of the Shan-Chen pseudo-potential LB step (arXiv:1906.11027).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library
(``paper_1906_11027_gb300``) never imports it, and this package imports nothing
from the GPU library: the two share no code, tables or constants.

The arithmetic lives in ``lbm_oracle.c`` (plain C loops in double precision,
compiled with ``-ffp-contract=off``); this module only compiles it and marshals
numpy arrays through ctypes.

Parity pins (all in ``tests/test_oracle_*.py``): Table 1 and the isotropy
identities of every lattice and force stencil (Sec. 2-3, Eq. 2), monomial moments
and plane-wave Taylor series of the force (Eqs. 1-2), the closed-form one-step
update at u = 0 and tau = 1 (Eqs. 5-6), moments of feq and of Guo's source
(Eq. 4), streaming as a permutation (Eq. 3), MRT = BGK at uniform rates,
shear-wave viscosity c_s^2 (tau - 1/2) (Sec. 3, tau = 11/12 and 19/24),
the wall of Fig. 6 (the one-sided force of a virtual wall density in closed
form, no-slip shear-wave decay in a bounce-back channel),
conservation of mass and momentum, the Peng-Robinson critical point and
density-ratio range (Sec. 3), flat-interface coexistence from mechanical
stability and Laplace's law.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19, D2Q13, D2Q25 = 0, 1, 2, 3
PSI_EXP, PSI_PR = 0, 1
BGK, MRT, EDM = 0, 1, 2

_dptr = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_iptr = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over cells, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # LBM_ORACLE_LIB: a separately compiled copy (the mutation tests plant
        # mistakes in one and check that the pins catch them)
        lib = ctypes.CDLL(os.environ.get("LBM_ORACLE_LIB") or build())
        V, I, D, P, L = None, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
        sig = {
            "or_create": (P, [I, I, I, I, I, I, D, D, D, I, D, D, D]),
            "or_destroy": (V, [P]),
            "or_lattice_table": (I, [I, _iptr, _dptr, ctypes.POINTER(D)]),
            "or_stencil_table": (I, [I, I, _iptr, _dptr]),
            "or_Q": (I, [P]), "or_N": (I, [P]), "or_cs2": (D, [P]), "or_cs2p": (D, [P]),
            "or_step_count": (L, [P]),
            "or_mrt_matrix": (I, [P, _dptr, _dptr]),
            "or_psi_of_rho": (D, [P, D]),
            "or_pressure": (D, [P, D]),
            "or_force_field": (V, [P, _dptr, _dptr]),
            "or_collide_cell": (V, [P, _dptr, _dptr, _dptr, P, P]),
            "or_step": (V, [P, L]),
            "or_init_from_rho": (V, [P, _dptr]),
            "or_init_droplet": (V, [P, D, D, D, D]),
            "or_init_flat": (V, [P, D, D, D, I]),
            "or_set_f": (V, [P, _dptr]),
            "or_get_f": (V, [P, _dptr]),
            "or_fields": (V, [P, P, P, P, P]),
            "or_observables": (V, [P, _dptr]),
            "or_pr_critical_T": (D, []),
            "or_pr_alpha": (D, [D]),
            "or_pr_pressure": (D, [D, D, D]),
            "or_set_wall": (I, [P, I, D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def lattice_table(lattice: int):
    """(c [Q,3] int, w [Q], cs2) of the oracle's velocity set."""
    lib = _load()
    c = np.zeros(75, dtype=np.int32)
    w = np.zeros(25)
    cs2 = ctypes.c_double()
    q = lib.or_lattice_table(lattice, c, w, ctypes.byref(cs2))
    return c[: 3 * q].reshape(q, 3).copy(), w[:q].copy(), cs2.value


def stencil_table(dim: int, order: int):
    """(e [n,3] int, unit weights [n]) of the oracle's force stencil."""
    lib = _load()
    e = np.zeros(192, dtype=np.int32)
    w = np.zeros(64)
    n = lib.or_stencil_table(dim, order, e, w)
    if n == 0:
        raise ValueError(f"no {dim}-D stencil of order {order}")
    return e[: 3 * n].reshape(n, 3).copy(), w[:n].copy()


_tc_cache = []


def pr_critical_T() -> float:
    if not _tc_cache:
        _tc_cache.append(_load().or_pr_critical_T())
    return _tc_cache[0]


def pr_pressure(rho: float, T_over_Tc: float) -> float:
    return _load().or_pr_pressure(float(rho), T_over_Tc, pr_critical_T())


class Sim:
    """One periodic domain of the oracle.  Arrays are numpy float64, x fastest,
    populations as f[b, z, y, x] (SoA), vectors as [..., 3]."""

    OBS_KEYS = ("rho_l", "rho_g", "dp", "max_u", "mean_u", "mass",
                "mom_x", "mom_y", "mom_z", "thickness", "step")

    def __init__(self, lattice=D2Q9, nx=64, ny=64, nz=1, stencil=4, psi=PSI_EXP,
                 T_over_Tc=0.0, G=-5.0, tau=1.0, coll=BGK,
                 s_e=1.64, s_eps=1.54, s_q=1.9):
        self._lib = _load()
        self._h = self._lib.or_create(lattice, nx, ny, nz, stencil, psi, T_over_Tc, G, tau,
                                      coll, s_e, s_eps, s_q)
        if not self._h:
            raise ValueError("oracle: unsupported parameter combination")
        self.lattice = lattice
        self.Q = self._lib.or_Q(self._h)
        self.N = self._lib.or_N(self._h)
        self.dim = 3 if lattice == D3Q19 else 2
        self.shape = (nz if self.dim == 3 else 1, ny, nx)
        self.cs2 = self._lib.or_cs2(self._h)
        self.cs2p = self._lib.or_cs2p(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    def set_wall(self, rows, rho_w):
        """Solid band y < rows with virtual wall density rho_w (Sec. 3, Fig. 6)."""
        if not self._lib.or_set_wall(self._h, int(rows), float(rho_w)):
            raise ValueError("oracle: wall band thinner than the lattice reach or force radius, or bad rho_w")
        self.wall_rows = int(rows)

    # -- initial conditions
    def init_droplet(self, rho_l, rho_g, R, width):
        self._lib.or_init_droplet(self._h, rho_l, rho_g, R, width)

    def init_flat(self, rho_l, rho_g, width, axis=0):
        self._lib.or_init_flat(self._h, rho_l, rho_g, width, axis)

    def init_from_rho(self, rho):
        self._lib.or_init_from_rho(self._h, np.ascontiguousarray(rho, dtype=np.float64).ravel())

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        assert f.size == self.Q * self.N
        self._lib.or_set_f(self._h, f)

    def get_f(self):
        f = np.empty(self.Q * self.N)
        self._lib.or_get_f(self._h, f)
        return f.reshape((self.Q,) + self.shape)

    # -- time stepping
    def step(self, n=1):
        self._lib.or_step(self._h, int(n))

    @property
    def step_count(self):
        return self._lib.or_step_count(self._h)

    # -- fields and observables
    def fields(self):
        """dict rho, psi (shape), F, u (shape + (3,)) of the current state."""
        rho = np.empty(self.N); psi = np.empty(self.N)
        F = np.empty(3 * self.N); u = np.empty(3 * self.N)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self._lib.or_fields(self._h, p(rho), p(psi), p(F), p(u))
        return {"rho": rho.reshape(self.shape), "psi": psi.reshape(self.shape),
                "F": F.reshape(self.shape + (3,)), "u": u.reshape(self.shape + (3,))}

    def observables(self):
        out = np.empty(11)
        self._lib.or_observables(self._h, out)
        return dict(zip(self.OBS_KEYS, out.tolist()))

    # -- pieces of the method, for closed-form checks
    def psi_of_rho(self, rho):
        return self._lib.or_psi_of_rho(self._h, float(rho))

    def pressure(self, rho):
        return self._lib.or_pressure(self._h, float(rho))

    def force_field(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.float64).ravel()
        assert psi.size == self.N
        F = np.empty(3 * self.N)
        self._lib.or_force_field(self._h, psi, F)
        return F.reshape(self.shape + (3,))

    def collide_cell(self, fin, F):
        fin = np.ascontiguousarray(fin, dtype=np.float64)
        Fv = np.zeros(3); Fv[: len(F)] = F
        fout = np.empty(self.Q)
        rho = ctypes.c_double(); u = np.zeros(3)
        self._lib.or_collide_cell(self._h, fin, Fv, fout, ctypes.addressof(rho),
                                  u.ctypes.data_as(ctypes.c_void_p))
        return fout, rho.value, u

    def mrt_matrix(self):
        M = np.empty(self.Q * self.Q); Minv = np.empty(self.Q * self.Q)
        self._lib.or_mrt_matrix(self._h, M, Minv)
        return M.reshape(self.Q, self.Q), Minv.reshape(self.Q, self.Q)
