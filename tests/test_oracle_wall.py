"""Pins of the oracle's wall (Sec. 3, Fig. 6): standard bounce-back at the
solid nodes of a band y < rows, and the wall's virtual density rho_w in Eq. 1.

- The force that a uniform fluid feels near the wall has a one-sided closed
  form: each stencil vector that reaches from a fluid node into the band
  contributes psi_w instead of psi_f, so, with the pairs (e, -e),
  F_y(k rows above the band) = -G psi_f (psi_f - psi_w) * sum over e_y > k of w~ e_y,
  mirrored under the band's periodic image, and zero deeper in the fluid.
- A shear wave u_x = U sin(pi (y - y_w) / H) in the channel decays as
  exp(-nu (pi/H)^2 t) with nu = c_s^2 (tau - 1/2) and no-slip walls half-way
  between the last solid row and the first fluid row (H = fluid rows).
  Full-way bounce-back places the wall there to within the O(1/H) slip of
  the scheme, hence the 2% bound at H = 32.
- The scheme conserves the mass of all nodes (solid nodes hold the reflected
  populations for one step).
"""
import numpy as np
import pytest

import oracle

CASES = [(oracle.D2Q9, 4), (oracle.D2Q9, 8), (oracle.D2Q13, 0), (oracle.D2Q25, 0)]
ORDER_OF_LATTICE = {oracle.D2Q9: 4, oracle.D2Q13: 6, oracle.D2Q25: 8}


def band_rows(lattice, stencil):
    c, _, _ = oracle.lattice_table(lattice)
    e, _ = oracle.stencil_table(2, stencil or ORDER_OF_LATTICE[lattice])
    return int(max(np.abs(c).max(), np.abs(e).max()))


@pytest.mark.parametrize("lattice,stencil", CASES)
@pytest.mark.parametrize("psi,G,T,rho_f,rho_w", [(oracle.PSI_EXP, -5.0, 0.0, 2.0, 0.7),
                                                 (oracle.PSI_PR, -1.0, 0.9, 5.0, 1.5)])
def test_wall_force_is_one_sided(lattice, stencil, psi, G, T, rho_f, rho_w):
    rows = band_rows(lattice, stencil)
    nx, ny = 8, 24
    sim = oracle.Sim(lattice, nx, ny, 1, stencil=stencil, psi=psi, T_over_Tc=T, G=G)
    sim.set_wall(rows, rho_w)
    sim.init_from_rho(np.full((ny, nx), rho_f))
    F = sim.fields()["F"][0]
    _, _, cs2 = oracle.lattice_table(lattice)
    e, wu = oracle.stencil_table(2, stencil or ORDER_OF_LATTICE[lattice])
    pf, pw = sim.psi_of_rho(rho_f), sim.psi_of_rho(rho_w)
    radius = int(np.abs(e).max())
    scale = max(abs(G * pf * (pf - pw)), 1e-300)
    for y in range(ny):
        if y < rows:
            expect = 0.0  # solid nodes carry no force
        else:
            k_lo, k_hi = y - rows, ny - 1 - y  # fluid rows between y and the band, below and above
            s_lo = sum(cs2 * w * ev[1] for ev, w in zip(e, wu) if ev[1] > k_lo)
            s_hi = sum(cs2 * w * ev[1] for ev, w in zip(e, wu) if ev[1] > k_hi)
            expect = -G * pf * (pf - pw) * (s_lo - s_hi)
        np.testing.assert_allclose(F[y, :, 1], expect, rtol=1e-12, atol=1e-14 * scale)
        np.testing.assert_allclose(F[y, :, 0], 0.0, atol=1e-14 * scale)
    # deeper than the stencil radius from the band the fluid feels nothing
    assert np.abs(F[rows + radius: ny - radius, :, 1]).max() <= 1e-14 * scale
    # a wall less wettable than the fluid (psi_w < psi_f, G < 0) pushes it away
    assert F[rows, 0, 1] > 0.0 and F[ny - 1, 0, 1] < 0.0


def _feq(c, w, cs2, rho, u):
    cu = np.einsum("bi,i...->b...", c[:, :2].astype(float), u)
    uu = (u ** 2).sum(0)
    return w[:, None, None] * rho * (1.0 + cu / cs2 + cu ** 2 / (2 * cs2 ** 2) - uu / (2 * cs2))


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D2Q13, oracle.D2Q25])
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_wall_channel_shear_wave_decays_with_no_slip(lattice, tau):
    rows = 2
    H, nx = 32, 8
    ny = H + rows
    sim = oracle.Sim(lattice, nx, ny, 1, stencil=0, G=0.0, tau=tau)
    sim.set_wall(rows, 1.0)
    c, w, cs2 = oracle.lattice_table(lattice)
    y = np.arange(ny)
    fluid = y >= rows
    mode = np.where(fluid, np.sin(np.pi * (y - rows + 0.5) / H), 0.0)
    U = 1e-4
    u = np.zeros((2, ny, nx))
    u[0] = U * mode[:, None]
    sim.set_f(_feq(c, w, cs2, np.ones((ny, nx)), u)[:, None])
    nu, k = cs2 * (tau - 0.5), np.pi / H
    t = int(round(0.5 / (nu * k * k)))
    sim.step(t)
    ux = sim.fields()["u"][0, :, :, 0]
    expect = U * mode * np.exp(-nu * k * k * t)
    assert np.abs(ux - expect[:, None]).max() <= 0.02 * U * np.exp(-nu * k * k * t)
    assert np.all(ux[~fluid] == 0.0)


def test_wall_conserves_mass_and_reads_observables_at_the_wall():
    lattice, stencil, rows = oracle.D2Q9, 8, 2
    nx, ny = 40, 32
    sim = oracle.Sim(lattice, nx, ny, 1, stencil=stencil, G=-5.0, tau=1.0)
    sim.set_wall(rows, 1.2)
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    r = np.hypot(x - nx / 2, y - rows)
    rho0 = 0.5 * (2.0 + 0.15) - 0.5 * (2.0 - 0.15) * np.tanh(2.0 * (r - 10.0) / 3.0)
    rho0[:rows] = rho0[rows]  # solid rows start like the fluid row above them
    sim.init_from_rho(rho0)
    m0 = sim.observables()["mass"]
    sim.step(300)
    o = sim.observables()
    f = sim.fields()
    assert o["mass"] == pytest.approx(m0, rel=1e-13)
    assert o["rho_l"] == f["rho"][0, rows, nx // 2]
    assert o["rho_g"] == f["rho"][0, ny - 1, 0]
    speed = np.linalg.norm(f["u"][0], axis=-1)
    assert np.all(speed[:rows] == 0.0)
    assert o["max_u"] == speed.max()
    assert o["mean_u"] == pytest.approx(speed[rows:].mean(), rel=1e-12)


def test_wall_band_rules():
    sim = oracle.Sim(oracle.D2Q25, 16, 16, 1, stencil=0, G=-5.0)
    with pytest.raises(ValueError):
        sim.set_wall(1, 1.0)  # thinner than the lattice's reach of 2
    with pytest.raises(ValueError):
        sim.set_wall(16, 1.0)  # no fluid left
    sim.set_wall(2, 1.0)
