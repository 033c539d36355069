"""Failure detection on the GPU path, made on the host or through bounded waits,
never by faulting the GPU.

- LBM_ENOMEM: a device allocator hook that refuses its k-th request, for every
  k that lbm_create and lbm_batch_create reach.  Each failing call returns
  LBM_ENOMEM, hands back everything it had already taken (the hook's count of
  live blocks returns to zero), and a context made afterwards works.  A
  context's scratch allocation (lbm_init_droplet) fails the same way and
  leaves the context usable.
- LBM_ENONFINITE from the Peng-Robinson potential (reading R6): above the
  density where p_EOS - c_s^2 rho changes sign, the square-root argument of
  psi = sqrt(2 (p_EOS - c_s^2 rho) / (G c_s^2)) is negative; the kernel flags
  it and the next readback reports it.
- LBM_ETIMEOUT: the library's bounded-wait probe waits on a barrier that
  nothing completes; the wait gives up, the call reports LBM_ETIMEOUT through
  the device error word, and the context keeps stepping correctly.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


class RefusingAllocator:
    """Wraps the library's torch-backed hook; refuses request number `fail_at`
    (1-based) and every request while `refuse_all` is set."""

    def __init__(self, lbm, fail_at=0):
        self.inner = lbm.TorchAllocator()
        self.fail_at = fail_at
        self.refuse_all = False
        self.requests = 0
        self.alloc_fn = lbm.ALLOC_FN(self._alloc)
        self.free_fn = lbm.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        self.requests += 1
        if self.refuse_all or self.requests == self.fail_at:
            return None
        return self.inner._alloc(nbytes, ctx)

    def _free(self, ptr, ctx):
        self.inner._free(ptr, ctx)

    @property
    def live(self):
        return self.inner.live


def params(lbm, alloc, **kw):
    p = lbm.lbm_params_default()
    p.nx, p.ny, p.nz = kw.get("nx", 40), kw.get("ny", 30), kw.get("nz", 1)
    p.lattice = kw.get("lattice", lbm.LBM_D2Q9)
    p.precision = kw.get("precision", lbm.LBM_FP64)
    p.G, p.tau, p.stencil = -5.0, 1.0, 4
    p.dev_alloc, p.dev_free = alloc.alloc_fn, alloc.free_fn
    return p


@pytest.mark.parametrize("lattice,nz,precision", [(0, 1, 0), (1, 12, 1)])
def test_create_reports_enomem_for_every_refused_request(lbm, lattice, nz, precision):
    probe = RefusingAllocator(lbm)
    ctx = lbm.lbm_create(params(lbm, probe, lattice=lattice, nz=nz, precision=precision))
    n_requests = probe.requests
    lbm.lbm_destroy(ctx)
    assert n_requests >= 6 and probe.live == 0
    for k in range(1, n_requests + 1):
        a = RefusingAllocator(lbm, fail_at=k)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(params(lbm, a, lattice=lattice, nz=nz, precision=precision))
        assert e.value.code == lbm.LBM_ENOMEM, k
        assert a.live == 0, f"request {k}: {a.live} blocks not handed back"
    # the library is still usable
    ok = RefusingAllocator(lbm)
    ctx = lbm.lbm_create(params(lbm, ok, lattice=lattice, nz=nz, precision=precision))
    lbm.lbm_init_droplet(ctx, 2.0, 0.15, 6.0, 2.0)
    lbm.lbm_step(ctx, 3)
    assert np.isfinite(lbm.lbm_observables(ctx)["mass"])
    lbm.lbm_destroy(ctx)
    assert ok.live == 0


def test_batch_create_reports_enomem_for_every_refused_request(lbm):
    doms = [dict(nx=64, ny=64, G=-5.0, tau=1.0, stencil=4, rho_l=2.0, rho_g=0.15, R=12.0, width=2.0),
            dict(nx=96, ny=64, G=-4.8, tau=0.8, stencil=8, rho_l=1.8, rho_g=0.2, R=15.0, width=2.0)]

    def plist(alloc):
        out, init = [], []
        for d in doms:
            p = lbm.lbm_params_default()
            p.nx, p.ny, p.nz = d["nx"], d["ny"], 1
            p.G, p.tau, p.stencil, p.precision = d["G"], d["tau"], d["stencil"], lbm.LBM_FP32_SHIFTED
            out.append(p)
            init += [d["rho_l"], d["rho_g"], d["R"], d["width"]]
        out[0].dev_alloc, out[0].dev_free = alloc.alloc_fn, alloc.free_fn
        return out, init

    probe = RefusingAllocator(lbm)
    b = lbm.lbm_batch_create(*plist(probe))
    n_requests = probe.requests
    lbm.lbm_batch_destroy(b)
    assert n_requests >= 10 and probe.live == 0
    for k in range(1, n_requests + 1):
        a = RefusingAllocator(lbm, fail_at=k)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_batch_create(*plist(a))
        assert e.value.code == lbm.LBM_ENOMEM, k
        assert a.live == 0, f"request {k}: {a.live} blocks not handed back"


def test_scratch_refusal_leaves_the_context_usable(lbm):
    a = RefusingAllocator(lbm)
    ctx = lbm.lbm_create(params(lbm, a))
    lbm.lbm_init_droplet(ctx, 2.0, 0.15, 8.0, 2.0)
    lbm.lbm_step(ctx, 5)
    before = lbm.lbm_observables(ctx)
    a.refuse_all = True
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_init_droplet(ctx, 1.9, 0.2, 9.0, 2.0)
    assert e.value.code == lbm.LBM_ENOMEM
    a.refuse_all = False
    assert lbm.lbm_observables(ctx) == before  # the failed call changed nothing
    lbm.lbm_step(ctx, 5)
    assert lbm.lbm_observables(ctx)["mass"] == pytest.approx(before["mass"], rel=1e-13)
    lbm.lbm_destroy(ctx)
    assert a.live == 0


def pr_psi_argument(rho, T_over_Tc):
    """p_EOS - c_s^2 rho for D2Q9 (c_s^2 = 1/3), written out for this check."""
    import oracle
    return oracle.pr_pressure(rho, T_over_Tc) - rho / 3.0


def test_negative_peng_robinson_argument_reported(lbm):
    T = 0.9
    assert pr_psi_argument(9.8, T) > 0 > pr_psi_argument(5.0, T)  # 9.8 is past the sign change
    dom = lbm.Domain(16, 16, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=T, G=-1.0, tau=1.0)
    rho = np.full(256, 5.0)
    rho[100] = 9.8
    dom.init_from_rho(rho)
    dom.step(1)
    with pytest.raises(lbm.LbmError) as e:
        dom.observables()
    assert e.value.code == lbm.LBM_ENONFINITE
    assert "Peng-Robinson" in str(e.value)


def test_bounded_wait_reports_timeout_and_context_survives(lbm):
    dom = lbm.Domain(48, 40, precision=lbm.LBM_FP32_SHIFTED)
    ref = lbm.Domain(48, 40, precision=lbm.LBM_FP32_SHIFTED)
    for d in (dom, ref):
        d.init_droplet(2.0, 0.15, 10.0, 2.0)
        d.step(7)
    rc = lbm.lbm_diag_wait_timeout(dom.ctx)
    assert rc == lbm.LBM_ETIMEOUT, lbm.lbm_strerror(rc)
    assert "wait" in lbm.load().lbm_last_error().decode()
    # the error word was cleared and the context steps on as if nothing happened
    dom.step(9)
    ref.step(9)
    assert np.array_equal(dom.get_f(), ref.get_f())
    assert dom.observables() == ref.observables()
