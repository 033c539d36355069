"""GPU parity of the wall (Sec. 3, Fig. 6): the solid band y < wall_rows with
standard bounce-back and the virtual wall density rho_w, through the C ABI,
against the FP64 oracle element by element on the same sessile-droplet start.

FP64 bar: 1e-12 relative (max norm) on the populations after 300 steps; the
observables (taken at the wall's probe nodes, velocity statistics over the
fluid) to the same bar.  FP32 deviation storage: the 2e-4 budget of the
droplet parity tests (about 40 float operations per population and step at
unit round-off 6e-8, accumulated over 300 steps).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

LAT = {0: oracle.D2Q9, 2: oracle.D2Q13, 3: oracle.D2Q25}


def sessile_rho(nx, ny, rows, rho_l, rho_g, r0, width=3.0):
    """Half-disc of liquid sitting on the band's top row, centred at x = nx/2;
    each solid row starts with the density of the fluid row above the band."""
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    r = np.hypot(x - nx // 2, y - rows)
    rho = 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - r0) / width)
    rho[:rows] = rho[rows]
    return rho


def wall_pair(lbm, lattice, nx, ny, rows, rho_w, *, stencil=0, coll=0, psi=0, T=0.0, G=-5.0, tau=1.0,
              precision=0):
    dom = lbm.Domain(nx, ny, lattice=lattice, stencil=stencil, collision=coll, psi=psi, T_over_Tc=T, G=G,
                     tau=tau, precision=precision, wall_rows=rows, rho_w=rho_w)
    ref = oracle.Sim(LAT[lattice], nx, ny, 1, stencil=stencil, psi=psi, T_over_Tc=T, G=G, tau=tau, coll=coll)
    ref.set_wall(rows, rho_w)
    return dom, ref


def rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


CASES = [  # lattice, stencil, collision, psi, ragged (nx, ny), rows, rho_w
    (0, 4, 0, 0, (45, 37), 1, 0.8),
    (0, 8, 0, 0, (45, 37), 2, 1.6),
    (0, 4, 1, 0, (40, 33), 1, 1.2),   # MRT
    (0, 4, 2, 0, (45, 37), 1, 0.8),   # exact-difference forcing
    (2, 0, 0, 0, (41, 35), 2, 1.0),   # D2Q13
    (3, 0, 2, 0, (41, 35), 2, 1.0),   # D2Q25, exact-difference
]


@pytest.mark.parametrize("lattice,stencil,coll,psi,shape,rows,rho_w", CASES)
def test_wall_matches_oracle(lbm, lattice, stencil, coll, psi, shape, rows, rho_w):
    nx, ny = shape
    dom, ref = wall_pair(lbm, lattice, nx, ny, rows, rho_w, stencil=stencil, coll=coll, psi=psi)
    rho0 = sessile_rho(nx, ny, rows, 2.0, 0.15, 10.0)
    dom.init_from_rho(rho0)
    ref.init_from_rho(rho0)
    dom.step(300)
    ref.step(300)
    assert rel_max(dom.get_f(), ref.get_f()) <= 1e-12
    og, oo = dom.observables(), ref.observables()
    for k in ("rho_l", "rho_g", "mass", "dp"):
        assert og[k] == pytest.approx(oo[k], rel=1e-12, abs=1e-13)
    for k in ("max_u", "mean_u"):
        assert og[k] == pytest.approx(oo[k], rel=1e-10)
    # the momenta are sums of nx*ny terms rho u that cancel (a symmetric drop):
    # the bar is the per-cell 1e-12 times the number of cells and the largest term
    mom_bar = 1e-12 * nx * ny * 2.0 * oo["max_u"]
    for k in ("mom_x", "mom_y"):
        assert abs(og[k] - oo[k]) <= mom_bar
    fg, fo = dom.fields(), ref.fields()
    assert np.all(fg["u"][0, :rows] == 0.0)
    np.testing.assert_allclose(fg["u"][0, rows:, :, :2], fo["u"][0, rows:, :, :2], rtol=0, atol=1e-12)


@pytest.mark.parametrize("T,rho_w", [(0.9, 1.5), (0.9, 4.5)])
def test_peng_robinson_wall_matches_oracle(lbm, T, rho_w):
    """The configuration of Fig. 6: P-R at T/Tc = 0.9, exact-difference forcing,
    D2Q25, wall densities 1.5 and 4.5."""
    from theory import maxwell
    rv, rl = maxwell(T)
    nx, ny, rows = 48, 36, 2
    dom, ref = wall_pair(lbm, 3, nx, ny, rows, rho_w, coll=2, psi=1, T=T, G=-1.0, tau=19 / 24)
    rho0 = sessile_rho(nx, ny, rows, rl, rv, 12.0)
    dom.init_from_rho(rho0)
    ref.init_from_rho(rho0)
    dom.step(300)
    ref.step(300)
    assert rel_max(dom.get_f(), ref.get_f()) <= 1e-12


def test_wall_fp32_within_budget(lbm):
    nx, ny, rows = 64, 48, 2
    dom, ref = wall_pair(lbm, 0, nx, ny, rows, 1.2, stencil=8, precision=1)
    rho0 = sessile_rho(nx, ny, rows, 2.0, 0.15, 14.0)
    dom.init_from_rho(rho0)
    ref.init_from_rho(rho0)
    dom.step(300)
    ref.step(300)
    assert rel_max(dom.get_f(), ref.get_f()) <= 2e-4
    og, oo = dom.observables(), ref.observables()
    assert og["mass"] == pytest.approx(oo["mass"], rel=1e-6)
    assert og["rho_l"] == pytest.approx(oo["rho_l"], rel=2e-4)


def test_wall_conserves_mass_over_a_long_run(lbm):
    """Bounce-back moves mass between the band and the fluid but never loses
    it: the sum over every node stays at its start to FP64 round-off."""
    nx, ny, rows = 96, 64, 2
    dom = lbm.Domain(nx, ny, stencil=8, G=-5.0, tau=1.0, wall_rows=rows, rho_w=1.0)
    dom.init_from_rho(sessile_rho(nx, ny, rows, 2.0, 0.15, 20.0))
    m0 = dom.observables()["mass"]
    dom.step(5000)
    assert dom.observables()["mass"] == pytest.approx(m0, rel=1e-12)


def test_wall_rejects_a_density_without_psi(lbm):
    """P-R psi of rho_w = 10 (near the co-volume limit 1/b = 10.5) has a
    negative argument: refused at creation."""
    with pytest.raises(lbm.LbmError) as e:
        lbm.Domain(32, 32, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=0.9, G=-1.0, wall_rows=1, rho_w=10.0)
    assert e.value.code == lbm.LBM_EINVAL


def test_wall_density_sets_wettability(lbm):
    """Fig. 6: tuning the wall's virtual density tunes the wettability.  A P-R
    droplet at T/Tc = 0.9 (exact-difference forcing, D2Q9 E4) on a wall whose
    rho_w = 1.5 sits near the vapour density (0.58) stands as a non-wetting cap
    (contact angle above 90 degrees); with rho_w = 4.5, near the liquid density
    (5.9), it spreads (below 90 degrees)."""
    from theory import maxwell
    from paper_1906_11027_gb300.experiments import fit_contact_angle
    rv, rl = maxwell(0.9)
    rows, nx, ny = 2, 160, 82
    theta = {}
    for rho_w in (1.5, 4.5):
        dom = lbm.Domain(nx, ny, stencil=4, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=0.9, G=-1.0,
                         collision=lbm.LBM_BGK_EDM, wall_rows=rows, rho_w=rho_w)
        dom.init_from_rho(sessile_rho(nx, ny, rows, rl, rv, 25.0))
        _, ok = dom.run_to_steady(1e-10, 200000, 100)
        assert ok
        dom.step(20000)
        rho = dom.fields()["rho"][0]
        dom.close()
        r_l, r_v = rho[rows + 2:, nx // 2].max(), np.median(rho[rows + 2:, 0])
        theta[rho_w] = fit_contact_angle(rho, rows, 0.5 * (r_l + r_v))[0]
    print("contact angle by rho_w:", theta)
    assert theta[1.5] > 90.0 > theta[4.5]
