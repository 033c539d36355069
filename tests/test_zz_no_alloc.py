"""lbm_moments_noalloc: the allocation-free mass/momentum reduction.

Some callers cannot allocate device memory when they need the totals (their
device memory is reserved up front by another framework's pool, or cudaMalloc is
off limits on their latency-critical path).  This entry point takes the
population buffer and a host array and keeps its block partials in a static
device array.  The test calls it twice in a row through the C ABI and compares
both results with lbm_observables (which uses the context's allocated scratch):
the mass at the FP64 parity tolerance of the other tests, 1e-12 relative, and
the momentum at 1e-12 in FP64 storage.  With FP32 storage the observables take
each cell's force in FP32, so the half-force sum they add, zero in exact
arithmetic, is zero only up to that round-off, bounded from the cells' own
forces.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


C9 = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]], dtype=float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def moving_state(rho, u0):
    """D2Q9 populations w_b rho (1 + c_b . u0 / c_s^2): sum f = rho and
    sum f c = rho u0, so the total momentum is large and known."""
    cu = (C9 @ np.asarray(u0, dtype=float))[:, None, None, None]
    return W9[:, None, None, None] * rho[None] * (1.0 + 3.0 * cu)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_observables_twice(lbm, precision):
    nx, ny = 96, 80
    dom = lbm.Domain(nx, ny, precision=precision)
    dom.init_droplet(2.0, 0.15, 20.0, 2.0)
    f0 = moving_state(dom.fields()["rho"], (0.01, -0.02))
    dom.set_f(f0)
    # FP32 storage keeps f - w_b rho_bar with rho_bar the mean density of the
    # state it was set from
    rho_bar = float(f0.sum(axis=0).mean()) if precision == 1 else 0.0
    dom.step(37)
    ptr, Q, ncells, elem = lbm.lbm_device_state(dom.ctx)
    assert (Q, ncells, elem) == (9, nx * ny, 8 if precision == 0 else 4)
    obs = dom.observables()
    first = lbm.lbm_moments_noalloc(ptr, lbm.LBM_D2Q9, precision, nx, ny, 1, rho_bar)
    second = lbm.lbm_moments_noalloc(ptr, lbm.LBM_D2Q9, precision, nx, ny, 1, rho_bar)
    assert np.array_equal(first, second)
    ref = np.array([obs["mass"], obs["mom_x"], obs["mom_y"], obs["mom_z"]])
    assert first[0] == pytest.approx(ref[0], rel=1e-12)
    # the observables' momentum adds sum_x F / 2, which is zero up to round-off
    scale = np.abs(ref[1:3]).max()
    assert scale > 1.0
    bound = 1e-12 * scale
    if precision == 1:
        # FP32 storage: each cell's force is taken in FP32 (a few operations,
        # well inside 2^-21 of |F|); F = 2 (rho u - j) from the FP64 fields
        fld, f = dom.fields(), dom.get_f()[:, 0]
        j = np.einsum("bi,byx->iyx", C9, f)
        F = 2.0 * (fld["rho"][0][None] * np.moveaxis(fld["u"][0][..., :2], -1, 0) - j)
        bound += 0.5 * 2.0 ** -21 * np.abs(F).sum()
    assert np.abs(first[1:] - ref[1:]).max() <= bound


def test_noalloc_rejects_oversized_domain(lbm):
    dom = lbm.Domain(16, 16)
    dom.init_droplet(2.0, 0.15, 4.0, 2.0)
    ptr, _, _, _ = lbm.lbm_device_state(dom.ctx)
    with pytest.raises(lbm.LbmError) as e:
        # 4096^2 * 2 cells > 16,777,216: rejected on the host before any launch
        lbm.lbm_moments_noalloc(ptr, lbm.LBM_D2Q9, 0, 8192, 4096, 1)
    assert e.value.code == lbm.LBM_EINVAL
    assert "static scratch" in lbm.load().lbm_last_error().decode()
