"""lbm_moments_noalloc: the allocation-free mass/momentum reduction.

Some callers cannot allocate device memory when they need the totals (their
device memory is reserved up front by another framework's pool, or cudaMalloc is
off limits on their latency-critical path).  This entry point takes the
population buffer and a host array and keeps its block partials in a static
device array.

The tests call it twice in a row through the C ABI and check both results:
- against lbm_observables (which uses the context's allocated scratch): the
  mass at the FP64 parity tolerance of the other tests, 1e-12 relative, and the
  momentum at 1e-12 in FP64 storage.  With FP32 storage the observables take
  each cell's force in FP32, so the half-force sum they add, zero in exact
  arithmetic, is zero only up to that round-off, bounded from the cells' own
  forces;
- against values that do not come from the library: the mass of the FP64
  oracle run from the same populations, and the total momentum the state was
  built with, sum_x rho u0, which every step conserves because the forces of
  Eq. 1 sum to zero over the periodic box;
- on D3Q19 and on a D2Q9 box with a wall, where the momentum covers the solid
  band as well (compared with a host sum of the populations).
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ORACLE_LAT = {0: oracle.D2Q9, 1: oracle.D3Q19}


def moving_state(lattice, rho, u0):
    """Populations w_b rho (1 + c_b . u0 / c_s^2): sum f = rho and sum f c = rho u0,
    so the total momentum is large and known."""
    c, w, cs2 = oracle.lattice_table(ORACLE_LAT[lattice])
    cu = (c.astype(float) @ np.asarray(u0, dtype=float))[:, None, None, None]
    return w[:, None, None, None] * rho[None] * (1.0 + cu / cs2)


def noalloc_twice(lbm, dom, lattice, precision, shape):
    import torch
    nz, ny, nx = shape
    # the context steps on its own non-blocking stream and the reduction runs on
    # the legacy stream: wait for the steps before reading their buffer
    torch.cuda.synchronize()
    ptr, Q, ncells, elem = lbm.lbm_device_state(dom.ctx)
    assert (ncells, elem) == (nx * ny * nz, 8 if precision == 0 else 4)
    rho_bar = lbm.lbm_reference_density(dom.ctx)
    assert (rho_bar == 0.0) == (precision == 0)
    first = lbm.lbm_moments_noalloc(ptr, lattice, precision, nx, ny, nz, rho_bar)
    second = lbm.lbm_moments_noalloc(ptr, lattice, precision, nx, ny, nz, rho_bar)
    assert np.array_equal(first, second)
    return first


@pytest.mark.parametrize("lattice,shape,precision", [
    (0, (1, 80, 96), 0),
    (0, (1, 80, 96), 1),
    (1, (20, 24, 28), 0),
    (1, (20, 24, 28), 1),
])
def test_noalloc_matches_observables_oracle_and_momentum_twice(lbm, lattice, shape, precision):
    nz, ny, nx = shape
    steps = 37
    u0 = (0.01, -0.02, 0.015)[: 3 if lattice == 1 else 2] + ((0.0,) if lattice == 0 else ())
    dom = lbm.Domain(nx, ny, nz, lattice=lattice, stencil=4, precision=precision)
    dom.init_droplet(2.0, 0.15, min(nx, ny) / 4, 2.0)
    f0 = moving_state(lattice, dom.fields()["rho"], u0)
    dom.set_f(f0)
    dom.step(steps)
    obs = dom.observables()
    got = noalloc_twice(lbm, dom, lattice, precision, shape)

    # 1. the library's own observables
    ref = np.array([obs["mass"], obs["mom_x"], obs["mom_y"], obs["mom_z"]])
    assert got[0] == pytest.approx(ref[0], rel=1e-12)
    scale = np.abs(ref[1:]).max()
    assert scale > 1.0
    bound = 1e-12 * scale
    if precision == 1:
        # FP32 storage: each cell's force is taken in FP32 (a few operations,
        # well inside 2^-21 of |F|); F = 2 (rho u - j) from the FP64 fields
        c, _, _ = oracle.lattice_table(ORACLE_LAT[lattice])
        fld, f = dom.fields(), dom.get_f()
        j = np.einsum("bi,b...->i...", c.astype(float), f)
        F = 2.0 * (fld["rho"][None] * np.moveaxis(fld["u"], -1, 0) - j)
        bound += 0.5 * 2.0 ** -21 * np.abs(F).sum()
    assert np.abs(got[1:] - ref[1:]).max() <= bound

    # 2. independent of the library: the oracle's mass after the same steps, and
    #    the momentum the state was built with (sum_x F = 0 keeps it)
    sim = oracle.Sim(ORACLE_LAT[lattice], nx, ny, nz, stencil=4, G=-5.0, tau=1.0)
    sim.set_f(f0)
    sim.step(steps)
    mass_oracle = sim.observables()["mass"]
    mom0 = f0.sum(axis=0).sum() * np.asarray(u0)
    tol = 1e-12 if precision == 0 else 2e-6
    assert got[0] == pytest.approx(mass_oracle, rel=tol)
    assert np.abs(got[1:] - mom0).max() <= tol * np.abs(mom0).max()


def test_noalloc_with_a_wall_sums_every_cell(lbm):
    nx, ny = 64, 48
    dom = lbm.Domain(nx, ny, stencil=4, wall_rows=2, rho_w=1.0)
    dom.init_droplet(2.0, 0.15, 10.0, 2.0)
    dom.step(25)
    got = noalloc_twice(lbm, dom, 0, 0, (1, ny, nx))
    assert got[0] == pytest.approx(dom.observables()["mass"], rel=1e-12)
    c, _, _ = oracle.lattice_table(oracle.D2Q9)
    f = dom.get_f()
    mom = c.astype(float).T @ f.reshape(9, -1).sum(axis=1)  # every cell, the solid band too
    assert np.abs(got[1:] - mom).max() <= 1e-12 * max(np.abs(f).sum() / 9, 1.0)


def test_noalloc_rejects_oversized_domain(lbm):
    dom = lbm.Domain(16, 16)
    dom.init_droplet(2.0, 0.15, 4.0, 2.0)
    ptr, _, _, _ = lbm.lbm_device_state(dom.ctx)
    with pytest.raises(lbm.LbmError) as e:
        # 4096^2 * 2 cells > 16,777,216: rejected on the host before any launch
        lbm.lbm_moments_noalloc(ptr, lbm.LBM_D2Q9, 0, 8192, 4096, 1)
    assert e.value.code == lbm.LBM_EINVAL
    assert "static scratch" in lbm.load().lbm_last_error().decode()
