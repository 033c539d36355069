"""Pins of the oracle's collision and streaming (Eqs. 3-6) and of its invariants.

- feq (Eq. 4) through its defining moments: sum feq = rho, sum feq c = rho u,
  sum feq c c = rho c_s^2 I + rho u u.
- Guo's source (Eq. 4) through the moments of the post-collision state: mass
  kept, momentum gains exactly F, and the second moment relaxes with the
  (1 - 1/(2 tau))(u F + F u) source of a second-order forcing scheme.
- Eqs. 5-6: at u = 0 and tau = 1 the density after one step is
  sum_b w_b [rho(x - c_b) + c_b . F(x - c_b) / (2 c_s^2)], and the first line of
  Eq. 7 gives the streamed momentum the same way.
- Streaming (Eq. 3) as the permutation f_b(x + c_b) <- f*_b(x), brute force.
- MRT with every rate 1/tau is BGK; mass and momentum are conserved; a centred
  droplet stays mirror-symmetric.
- Exact-difference forcing (the paper's runs, Sec. 3) through its moments: mass
  kept, momentum gains exactly F, and the second moment is the BGK relaxation
  towards feq at u' = j/rho plus rho (v v - u' u') with v = u' + F/rho; at
  tau = 1 the result is the equilibrium at v.
"""
import numpy as np
import pytest

import oracle

LATS = [(oracle.D2Q9, 4), (oracle.D2Q13, 6), (oracle.D2Q25, 8), (oracle.D3Q19, 4)]


def lattice(lat):
    c, w, cs2 = oracle.lattice_table(lat)
    return c.astype(float), w, cs2


@pytest.mark.parametrize("lat,order", LATS)
def test_feq_moments(lat, order):
    rng = np.random.default_rng(7)
    c, w, cs2 = lattice(lat)
    sim = oracle.Sim(lat, 4, 4, 4 if lat == oracle.D3Q19 else 1, stencil=order, tau=1.0)
    for _ in range(5):
        fin = w * rng.uniform(0.5, 2.0, size=len(w))
        feq, rho, u = sim.collide_cell(fin, [0.0, 0.0, 0.0])  # tau = 1, F = 0 -> feq
        assert rho == pytest.approx(fin.sum(), rel=1e-15)
        np.testing.assert_allclose(u, (fin @ c) / rho, rtol=1e-13, atol=1e-16)
        assert feq.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(feq @ c, rho * u, atol=1e-14)
        P = np.einsum("b,bi,bj->ij", feq, c, c)
        np.testing.assert_allclose(P, rho * cs2 * np.eye(3) * (np.abs(c).sum(0) > 0) + rho * np.outer(u, u),
                                   atol=1e-14)


@pytest.mark.parametrize("lat,order", LATS)
@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_guo_forcing_moments(lat, order, tau):
    rng = np.random.default_rng(11)
    c, w, cs2 = lattice(lat)
    dim = 3 if lat == oracle.D3Q19 else 2
    sim = oracle.Sim(lat, 4, 4, 4 if dim == 3 else 1, stencil=order, tau=tau)
    for _ in range(5):
        fin = w * rng.uniform(0.5, 2.0, size=len(w))
        F = np.zeros(3)
        F[:dim] = rng.normal(scale=0.01, size=dim)
        fout, rho, u = sim.collide_cell(fin, F)
        j = fin @ c
        np.testing.assert_allclose(u, (j + F / 2) / rho, rtol=1e-13, atol=1e-16)
        assert fout.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(fout @ c, j + F, atol=1e-14)
        mask = np.outer(np.abs(c).sum(0) > 0, np.abs(c).sum(0) > 0)
        Pin = np.einsum("b,bi,bj->ij", fin, c, c)
        Peq = rho * cs2 * np.eye(3) + rho * np.outer(u, u)
        Pout = np.einsum("b,bi,bj->ij", fout, c, c)
        expect = Pin - (Pin - Peq) / tau + (1 - 1 / (2 * tau)) * (np.outer(u, F) + np.outer(F, u))
        np.testing.assert_allclose(Pout[mask], expect[mask], atol=1e-13)


def shift(a, d):
    """a(x - d) on a periodic [z, y, x] array."""
    return np.roll(a, shift=(int(d[2]), int(d[1]), int(d[0])), axis=(0, 1, 2))


@pytest.mark.parametrize("lat,order", LATS)
def test_one_step_at_zero_velocity_tau1(lat, order):
    """Eqs. 5-6 (and Eq. 7, first line) at tau = 1 with u = 0 at time t."""
    rng = np.random.default_rng(3)
    c, w, cs2 = lattice(lat)
    dim = 3 if lat == oracle.D3Q19 else 2
    shape = (6, 7, 8) if dim == 3 else (1, 11, 13)
    sim = oracle.Sim(lat, shape[2], shape[1], shape[0], stencil=order, G=-5.0, tau=1.0)
    rho = rng.uniform(0.3, 1.8, size=shape)
    psi = -np.expm1(-rho)
    F = sim.force_field(psi)
    # populations with sum f = rho and sum f c = -F/2, so that u = 0 exactly
    f = np.stack([w[b] * (rho - (F @ c[b]) / (2 * cs2)) for b in range(len(w))])
    sim.set_f(f)
    sim.step(1)
    f1 = sim.get_f()
    rho1 = f1.sum(axis=0)
    expect = sum(w[b] * shift(rho + (F @ c[b]) / (2 * cs2), c[b]) for b in range(len(w)))
    np.testing.assert_allclose(rho1, expect, rtol=1e-13)
    j1 = np.einsum("bzyx,bi->zyxi", f1, c)
    expect_j = sum(w[b] * shift(rho + (F @ c[b]) / (2 * cs2), c[b])[..., None] * c[b] for b in range(len(w)))
    np.testing.assert_allclose(j1, expect_j, atol=1e-13)


@pytest.mark.parametrize("lat,order", LATS)
def test_streaming_is_the_shift_permutation(lat, order):
    """G = 0 and f = w rho: u = 0 and F = 0, so the collision is the identity and
    one step must give f_b(x) = w_b rho(x - c_b) up to the rounding of the
    identity collision (4x3 and 3x2x4 boxes; a wrong shift is an O(1) error)."""
    rng = np.random.default_rng(5)
    c, w, _ = lattice(lat)
    dim = 3 if lat == oracle.D3Q19 else 2
    shape = (4, 2, 3) if dim == 3 else (1, 3, 4)
    sim = oracle.Sim(lat, shape[2], shape[1], shape[0], stencil=order, G=0.0, tau=0.9)
    rho = rng.uniform(0.5, 1.5, size=shape)
    sim.init_from_rho(rho)
    sim.step(1)
    f1 = sim.get_f()
    for b in range(len(w)):
        np.testing.assert_allclose(f1[b], w[b] * shift(rho, c[b]), rtol=1e-14, atol=0)


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 32, 32)), (oracle.D3Q19, (12, 12, 12))])
def test_mrt_with_uniform_rates_is_bgk(lat, shape):
    tau = 0.8
    nz, ny, nx = shape
    a = oracle.Sim(lat, nx, ny, nz, G=-5.0, tau=tau, coll=oracle.BGK)
    b = oracle.Sim(lat, nx, ny, nz, G=-5.0, tau=tau, coll=oracle.MRT,
                   s_e=1 / tau, s_eps=1 / tau, s_q=1 / tau)
    for s in (a, b):
        s.init_droplet(2.0, 0.15, nx / 4, 2.0)
        s.step(40)
    fa, fb = a.get_f(), b.get_f()
    assert np.abs(fa - fb).max() <= 1e-13 * np.abs(fa).max()


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_mrt_basis_rows_orthogonal(lat):
    s = oracle.Sim(lat, 4, 4, 4 if lat == oracle.D3Q19 else 1, coll=oracle.MRT)
    M, Minv = s.mrt_matrix()
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    np.testing.assert_allclose(M @ Minv, np.eye(s.Q), atol=1e-13)


@pytest.mark.parametrize("lat,order,coll,shape", [
    (oracle.D2Q9, 4, oracle.BGK, (1, 40, 48)),
    (oracle.D2Q9, 10, oracle.MRT, (1, 40, 48)),
    (oracle.D2Q25, 8, oracle.BGK, (1, 40, 40)),
    (oracle.D3Q19, 6, oracle.BGK, (16, 16, 16)),
])
def test_mass_and_momentum_conserved(lat, order, coll, shape):
    nz, ny, nx = shape
    s = oracle.Sim(lat, nx, ny, nz, stencil=order, G=-5.0, tau=0.9, coll=coll)
    s.init_droplet(2.0, 0.15, min(nx, ny) / 4, 2.0)
    o0 = s.observables()
    s.step(200)
    o1 = s.observables()
    assert abs(o1["mass"] - o0["mass"]) <= 1e-13 * o0["mass"]
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(o1[k] - o0[k]) <= 1e-12 * o0["mass"]


def test_centred_droplet_stays_symmetric():
    s = oracle.Sim(oracle.D2Q9, 48, 48, stencil=8, G=-5.0, tau=1.0)
    s.init_droplet(2.0, 0.15, 12, 2.0)
    s.step(300)
    rho = s.fields()["rho"][0]
    mirror_x = np.roll(rho[:, ::-1], 1, axis=1)  # x -> nx - x (mod nx)
    assert np.abs(rho - mirror_x).max() < 1e-12
    assert np.abs(rho - rho.T).max() < 1e-12


@pytest.mark.parametrize("lat,order", LATS)
@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_exact_difference_forcing_moments(lat, order, tau):
    rng = np.random.default_rng(13)
    c, w, cs2 = lattice(lat)
    dim = 3 if lat == oracle.D3Q19 else 2
    sim = oracle.Sim(lat, 4, 4, 4 if dim == 3 else 1, stencil=order, tau=tau, coll=oracle.EDM)
    iso = np.eye(3) * (np.abs(c).sum(0) > 0)
    for _ in range(5):
        fin = w * rng.uniform(0.5, 2.0, size=len(w))
        F = np.zeros(3)
        F[:dim] = rng.normal(scale=0.01, size=dim)
        fout, rho, u = sim.collide_cell(fin, F)
        j = fin @ c
        up = j / rho
        v = up + F / rho
        np.testing.assert_allclose(u, (j + F / 2) / rho, rtol=1e-13, atol=1e-16)
        assert fout.sum() == pytest.approx(fin.sum(), rel=1e-14)
        np.testing.assert_allclose(fout @ c, j + F, atol=1e-14)
        P_in = np.einsum("b,bi,bj->ij", fin, c, c)
        P_eq = rho * cs2 * iso + rho * np.outer(up, up)
        P_out = np.einsum("b,bi,bj->ij", fout, c, c)
        expect = (1 - 1 / tau) * P_in + P_eq / tau + rho * (np.outer(v, v) - np.outer(up, up))
        np.testing.assert_allclose(P_out, expect, atol=1e-13)
        if tau == 1.0:
            np.testing.assert_allclose(P_out, rho * cs2 * iso + rho * np.outer(v, v), atol=1e-13)


def test_exact_difference_forcing_differs_from_guo():
    """The two schemes share mass and momentum but not the second moment: at
    tau = 0.6 with a finite force they must not coincide."""
    c, w, cs2 = lattice(oracle.D2Q9)
    fin = w * np.linspace(0.8, 1.2, len(w))
    F = np.array([0.02, -0.01, 0.0])
    a = oracle.Sim(oracle.D2Q9, 4, 4, tau=0.6, coll=oracle.EDM).collide_cell(fin, F)[0]
    b = oracle.Sim(oracle.D2Q9, 4, 4, tau=0.6, coll=oracle.BGK).collide_cell(fin, F)[0]
    assert np.abs(a - b).max() > 1e-6
