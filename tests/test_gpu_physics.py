"""Steady states of the library at the sizes of the paper's parameter study
(Sec. 3): D2Q9 MRT droplets on 256^2, a flat interface on a 512 x 64 strip, and
a 512^2 domain, checked against what theory fixes at any size:

- a static droplet obeys Laplace's law, dp linear in 1/R with a small intercept;
- a flat interface reaches the coexistence densities of the mechanical-stability
  condition with eps = 0 (the nearest-neighbour force's discrete pressure
  tensor), and equal bulk pressures;
- FP32 deviation storage reaches the FP64 steady state within stated tolerances
  on rho_l, rho_g, dp and max|u|;
- the 8th-order force stencil lowers the spurious currents of the 4th-order one
  (Shan's remedy, the paper's Fig. 3 claim);
- at 512^2 the MRT step agrees with the FP64 oracle to 1e-12 step by step;
- the paper's own runs (exact-difference forcing, Peng-Robinson, 60 x 60
  droplet and a flat strip): the consistent lattices lower the spurious
  currents by about an order of magnitude below the 8th-order stencil, the
  8th-order stencil helps less at low temperature, and the interface widens
  from D2Q9 to D2Q13 to D2Q25.
"""
import numpy as np
import pytest

import oracle
from theory import mechanical_stability

pytestmark = pytest.mark.gpu

MRT = dict(collision=1, s_e=1.64, s_eps=1.54, s_q=1.9)


def steady(lbm, dom, tol=1e-10, max_steps=400000, require=True):
    steps, ok = dom.run_to_steady(tol, max_steps, 100)
    assert ok or not require, "no steady state within max_steps"
    return steps, dom.observables()


def test_laplace_law_d2q9_mrt_256(lbm):
    rg, rl = mechanical_stability(-5.0, 0.0)
    radii = np.array([20.0, 40.0, 80.0])
    dps = []
    for R in radii:
        dom = lbm.Domain(256, 256, G=-5.0, tau=1.0, stencil=4, **MRT)
        dom.init_droplet(rl, rg, R, 3.0)
        _, o = steady(lbm, dom)
        dps.append(o["dp"])
        dom.close()
    dps = np.array(dps)
    A = np.vstack([np.ones_like(radii), 1.0 / radii]).T
    (intercept, sigma), *_ = np.linalg.lstsq(A, dps, rcond=None)
    pred = A @ np.array([intercept, sigma])
    r2 = 1.0 - ((dps - pred) ** 2).sum() / ((dps - dps.mean()) ** 2).sum()
    print(f"Laplace fit: sigma {sigma:.5f}, intercept {intercept:.2e}, R^2 {r2:.6f}, dp {dps}")
    assert sigma > 0
    assert r2 > 0.999
    assert abs(intercept) < 0.05 * dps.min()


@pytest.mark.parametrize("G,tol_l,tol_g,settles", [(-4.5, 5e-4, 5e-3, True), (-5.0, 5e-4, 5e-3, True),
                                                  (-5.5, 5e-3, 2e-2, False)])
def test_flat_strip_512x64_coexistence(lbm, G, tol_l, tol_g, settles):
    """The gas density carries the lattice's discretisation error, which grows as
    the interface sharpens with |G|; eps = 1 would give 0.156 at G = -5 and 0.105
    at G = -5.5.  A flat interface keeps a small residual current (the discrete
    force is not an exact gradient, Eq. 7): at G = -4.5 and -5 the bulk pressures
    agree to a few 1e-6 and max|u| stays at the 1e-6 level.  At G = -5.5 the
    64-cell-wide strip keeps a current near 1e-3 that has not settled after
    200,000 steps (with MRT and with BGK alike; a 4-cell-wide strip settles), so
    there only the densities are pinned."""
    rg, rl = mechanical_stability(G, 0.0)
    dom = lbm.Domain(512, 64, G=G, tau=1.0, stencil=4, **MRT)
    dom.init_flat(rl, rg, 4.0, 0)
    steps, o = steady(lbm, dom, max_steps=200000, require=settles)
    print(f"G {G}: rho_l {o['rho_l']:.6f} (theory {rl:.6f}), rho_g {o['rho_g']:.6f} (theory {rg:.6f}), "
          f"dp {o['dp']:.2e}, max_u {o['max_u']:.2e}, steps {steps}")
    assert o["rho_l"] == pytest.approx(rl, rel=tol_l)
    assert o["rho_g"] == pytest.approx(rg, rel=tol_g)
    if settles:
        assert abs(o["dp"]) < 2e-5
        assert o["max_u"] < 2e-5


def test_fp32_steady_state_against_fp64_256(lbm):
    """The stated FP32 tolerances at a steady droplet: rho_l and rho_g within
    1e-4 relative, dp within 1e-3 relative, max|u| within 5%."""
    rg, rl = mechanical_stability(-5.0, 0.0)
    res = {}
    for prec in (0, 1):
        dom = lbm.Domain(256, 256, G=-5.0, tau=1.0, stencil=4, precision=prec, **MRT)
        dom.init_droplet(rl, rg, 40.0, 3.0)
        _, res[prec] = steady(lbm, dom)
        dom.close()
    a, b = res[1], res[0]
    print("FP32 vs FP64 steady droplet: rho_l %.2e rho_g %.2e dp %.2e max_u %.2e" % (
        a["rho_l"] / b["rho_l"] - 1, a["rho_g"] / b["rho_g"] - 1, a["dp"] / b["dp"] - 1, a["max_u"] / b["max_u"] - 1))
    assert a["rho_l"] == pytest.approx(b["rho_l"], rel=1e-4)
    assert a["rho_g"] == pytest.approx(b["rho_g"], rel=1e-4)
    assert a["dp"] == pytest.approx(b["dp"], rel=1e-3)
    assert a["max_u"] == pytest.approx(b["max_u"], rel=0.05)


def test_higher_isotropy_lowers_spurious_currents_256(lbm):
    rg, rl = mechanical_stability(-5.0, 0.0)
    umax = {}
    for order in (4, 8):
        dom = lbm.Domain(256, 256, G=-5.0, tau=1.0, stencil=order)
        dom.init_droplet(rl, rg, 40.0, 3.0)
        _, o = steady(lbm, dom)
        umax[order] = o["max_u"]
        dom.close()
    print("steady max|u|:", umax)
    assert umax[4] > umax[8]


def test_d2q9_mrt_512_fp64_against_oracle(lbm):
    rg, rl = mechanical_stability(-5.0, 0.0)
    dom = lbm.Domain(512, 512, G=-5.0, tau=0.8, stencil=4, **MRT)
    ref = oracle.Sim(oracle.D2Q9, 512, 512, stencil=4, G=-5.0, tau=0.8, coll=oracle.MRT,
                     s_e=1.64, s_eps=1.54, s_q=1.9)
    for d in (dom, ref):
        d.init_droplet(rl, rg, 80.0, 3.0)
    dom.step(30)
    ref.step(30)
    f, fr = dom.get_f(), ref.get_f()
    assert np.abs(f - fr).max() <= 1e-12 * np.abs(fr).max()
    o, oo = dom.observables(), ref.observables()
    for k in ("rho_l", "rho_g", "dp"):
        assert o[k] == pytest.approx(oo[k], rel=1e-12, abs=1e-14)
    # a sum of 262,144 densities in another order: rounding ~ sqrt(N) eps .. N eps
    assert o["mass"] == pytest.approx(oo["mass"], rel=1e-11)


def test_consistent_lattice_lowers_spurious_currents_pr_128(lbm):
    """The paper's central claim (Sec. 3, Figs. 2-3) at a larger size and at
    steady state: a Peng-Robinson droplet at T/Tc = 0.9 has spurious currents
    that fall from D2Q9 with the 4th-order force stencil to D2Q9 with the
    8th-order one (Shan's remedy) and much further with the consistent D2Q25
    model (lattice = force stencil)."""
    from theory import maxwell
    rv, rl = maxwell(0.9)
    umax = {}
    for name, lat, st in (("iso4", lbm.LBM_D2Q9, 4), ("iso8", lbm.LBM_D2Q9, 8), ("q25", lbm.LBM_D2Q25, 0)):
        dom = lbm.Domain(128, 128, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=0.9,
                         G=-1.0, tau=1.0)
        dom.init_droplet(rl, rv, 32.0, 3.0)
        steps, o = steady(lbm, dom, max_steps=200000, require=False)
        umax[name] = o["max_u"]
        dom.close()
    print("steady max|u| (P-R, T/Tc = 0.9):", umax, "iso8/q25 = %.1f" % (umax["iso8"] / umax["q25"]))
    assert umax["iso4"] > umax["iso8"] > umax["q25"]
    assert umax["iso8"] / umax["q25"] > 3.0


def _pr_droplet_edm(lbm, lat, st, tau, T, rv, rl):
    dom = lbm.Domain(60, 60, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=T,
                     G=-1.0, tau=tau, collision=lbm.LBM_BGK_EDM)
    dom.init_droplet(rl, rv, 15.0, 3.0)
    steady(lbm, dom, max_steps=100000)
    dom.step(20000)
    o = dom.observables()
    dom.close()
    return o


def test_consistent_lattices_lower_spurious_currents_edm_60(lbm):
    """The paper's droplet test as it ran it (Sec. 3, Fig. 3): 60 x 60, r0 = 15,
    Peng-Robinson at T/Tc = 0.8 with the exact-difference forcing, D2Q13 and
    D2Q25 at the equal-viscosity relaxation times.  Max and mean |u| fall from
    4th- to 8th-order isotropy (Shan's remedy) and by about another order of
    magnitude with the consistent lattices."""
    from theory import maxwell
    rv, rl = maxwell(0.8)
    o = {name: _pr_droplet_edm(lbm, lat, st, tau, 0.8, rv, rl)
         for name, lat, st, tau in (("iso4", lbm.LBM_D2Q9, 4, 1.0), ("iso8", lbm.LBM_D2Q9, 8, 1.0),
                                    ("q13", lbm.LBM_D2Q13, 0, 11.0 / 12.0), ("q25", lbm.LBM_D2Q25, 0, 19.0 / 24.0))}
    for k in ("max_u", "mean_u"):
        print(k, {n: "%.3e" % v[k] for n, v in o.items()})
        assert o["iso4"][k] > o["iso8"][k] > o["q13"][k] > o["q25"][k]
    assert o["iso8"]["max_u"] / o["q25"]["max_u"] > 8.0
    assert o["iso8"]["mean_u"] / o["q25"]["mean_u"] > 20.0


def test_shan_remedy_fades_at_low_temperature_edm_60(lbm):
    """Sec. 3 observes that the higher-order force stencil helps less as the
    temperature falls: the E4/E8 ratio of the spurious currents at T/Tc = 0.7
    is well below the one at 0.9."""
    from theory import maxwell
    ratio = {}
    for T in (0.7, 0.9):
        rv, rl = maxwell(T)
        u4 = _pr_droplet_edm(lbm, lbm.LBM_D2Q9, 4, 1.0, T, rv, rl)["max_u"]
        u8 = _pr_droplet_edm(lbm, lbm.LBM_D2Q9, 8, 1.0, T, rv, rl)["max_u"]
        ratio[T] = u4 / u8
    print("E4/E8 max|u| ratio:", ratio)
    assert ratio[0.9] > 2.0
    assert ratio[0.7] < 0.6 * ratio[0.9]


def test_flat_interface_edm_coexistence_and_thickness(lbm):
    """The flat-interface test of Sec. 3 (Figs. 4-5) at T/Tc = 0.75 with the
    exact-difference forcing on a 200 x 8 strip: every model keeps the liquid
    density within 0.5% of the Maxwell value, the vapour density falls short of
    it (the thermodynamic inconsistency the paper leaves alone), the 8th-order
    stencil falls shortest and the consistent lattices are no worse than
    E4, and the interface (1.05 rho_v <= rho <= 0.95 rho_l) widens from D2Q9 E4
    to D2Q13 to D2Q25."""
    from theory import maxwell
    from paper_1906_11027_gb300.experiments import interface_thickness
    rv, rl = maxwell(0.75)
    res = {}
    for name, lat, st, tau in (("iso4", lbm.LBM_D2Q9, 4, 1.0), ("iso8", lbm.LBM_D2Q9, 8, 1.0),
                               ("q13", lbm.LBM_D2Q13, 0, 1.0), ("q25", lbm.LBM_D2Q25, 0, 1.0)):
        dom = lbm.Domain(200, 8, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=0.75,
                         G=-1.0, tau=tau, collision=lbm.LBM_BGK_EDM)
        dom.init_flat(rl, rv, 3.0, 0)
        steady(lbm, dom, max_steps=200000)
        dom.step(20000)
        line = dom.fields()["rho"][0, 4, :]
        dom.close()
        r_l, r_v = float(line[100]), float(line[0])
        _, width = interface_thickness(line, r_v, r_l)
        res[name] = (r_v, r_l, width)
    print("flat interface (rho_v, rho_l, thickness), Maxwell %.4f / %.4f:" % (rv, rl), res)
    for r_v, r_l, _ in res.values():
        assert abs(r_l / rl - 1.0) < 5e-3
        assert r_v < rv
    assert res["iso8"][0] < res["iso4"][0] <= res["q13"][0]
    assert res["iso8"][0] < res["q25"][0]
    assert res["iso4"][2] < res["q13"][2] < res["q25"][2]
