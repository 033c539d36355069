"""Pins of the oracle's MRT collision moment by moment (reading R7; the paper
names MRT only through its references).

R7 fixes an orthogonal moment basis and one relaxation rate per moment:
- D2Q9 (Lallemand & Luo): 1, e = 3|c|^2 - 4, eps = (9|c|^4 - 21|c|^2 + 8)/2,
  j_x, q_x = (3|c|^2 - 5) c_x, j_y, q_y, p_xx = c_x^2 - c_y^2, p_xy = c_x c_y;
  rates 1/tau on the conserved and stress moments, s_e on e, s_eps on eps,
  s_q on q_x, q_y.
- D3Q19 (d'Humieres et al.): 1, e = 19|c|^2 - 30, eps = (21|c|^4 - 53|c|^2 + 24)/2,
  j and q = (5|c|^2 - 9) c per axis, 3p_xx = 3c_x^2 - |c|^2,
  pi_xx = (3|c|^2 - 5)(3c_x^2 - |c|^2), p_ww = c_y^2 - c_z^2,
  pi_ww = (3|c|^2 - 5)(c_y^2 - c_z^2), p_xy, p_yz, p_xz, and the third-order
  m_x = (c_y^2 - c_z^2) c_x, m_y = (c_z^2 - c_x^2) c_y, m_z = (c_x^2 - c_y^2) c_z;
  rates 1/tau on the conserved and stress moments, s_e on e, s_eps on eps and
  both pi, s_q on q and m.

The basis is written out here as the polynomials above, evaluated on the
velocity set, so nothing is taken from the oracle's own matrix.

1. A state at rest in equilibrium plus a small perturbation along one
   non-conserved moment's polynomial keeps rho and j, and one force-free
   collision scales that perturbation by (1 - s_k) and leaves every other
   moment alone.
2. With a force, every moment follows its own definition
   m*_k = m_k - s_k (m_k - m_eq,k) + (1 - s_k/2) m_src,k, with m_eq and m_src
   the moments of Eq. 4's equilibrium and Guo source.
The rates are all different, so a swapped or misplaced rate fails.
"""
import numpy as np
import pytest

import oracle

TAU = 0.8
RATES = dict(s_e=1.1, s_eps=1.3, s_q=1.7)


def d2q9_basis(c):
    x, y = c[:, 0], c[:, 1]
    c2 = x * x + y * y
    rows = [
        ("rho", np.ones_like(x), "cons"),
        ("e", 3 * c2 - 4, "s_e"),
        ("eps", (9 * c2 * c2 - 21 * c2 + 8) / 2, "s_eps"),
        ("jx", x, "cons"),
        ("qx", (3 * c2 - 5) * x, "s_q"),
        ("jy", y, "cons"),
        ("qy", (3 * c2 - 5) * y, "s_q"),
        ("pxx", x * x - y * y, "stress"),
        ("pxy", x * y, "stress"),
    ]
    return rows


def d3q19_basis(c):
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    c2 = x * x + y * y + z * z
    rows = [
        ("rho", np.ones_like(x), "cons"),
        ("e", 19 * c2 - 30, "s_e"),
        ("eps", (21 * c2 * c2 - 53 * c2 + 24) / 2, "s_eps"),
        ("jx", x, "cons"), ("qx", (5 * c2 - 9) * x, "s_q"),
        ("jy", y, "cons"), ("qy", (5 * c2 - 9) * y, "s_q"),
        ("jz", z, "cons"), ("qz", (5 * c2 - 9) * z, "s_q"),
        ("3pxx", 3 * x * x - c2, "stress"),
        ("3pixx", (3 * c2 - 5) * (3 * x * x - c2), "s_eps"),
        ("pww", y * y - z * z, "stress"),
        ("piww", (3 * c2 - 5) * (y * y - z * z), "s_eps"),
        ("pxy", x * y, "stress"), ("pyz", y * z, "stress"), ("pxz", x * z, "stress"),
        ("mx", (y * y - z * z) * x, "s_q"),
        ("my", (z * z - x * x) * y, "s_q"),
        ("mz", (x * x - y * y) * z, "s_q"),
    ]
    return rows


CASES = [(oracle.D2Q9, d2q9_basis), (oracle.D3Q19, d3q19_basis)]


def setup(lat, basis_fn):
    c, w, cs2 = oracle.lattice_table(lat)
    c = c.astype(float)
    rows = basis_fn(c)
    M = np.array([r[1] for r in rows], dtype=float)
    rate = {"cons": 1 / TAU, "stress": 1 / TAU, **RATES}
    S = np.array([rate[r[2]] for r in rows])
    dim = 3 if lat == oracle.D3Q19 else 2
    sim = oracle.Sim(lat, 4, 4, 4 if dim == 3 else 1, tau=TAU, coll=oracle.MRT, **RATES)
    return c, w, cs2, rows, M, S, sim, dim


@pytest.mark.parametrize("lat,basis_fn", CASES, ids=["D2Q9", "D3Q19"])
def test_basis_is_orthogonal(lat, basis_fn):
    """The written-out basis is orthogonal and complete on the velocity set."""
    c, w, cs2, rows, M, S, sim, dim = setup(lat, basis_fn)
    G = M @ M.T
    assert np.allclose(G - np.diag(np.diag(G)), 0.0)
    assert np.linalg.matrix_rank(M) == len(w)


@pytest.mark.parametrize("lat,basis_fn", CASES, ids=["D2Q9", "D3Q19"])
def test_each_moment_relaxes_at_its_own_rate(lat, basis_fn):
    c, w, cs2, rows, M, S, sim, dim = setup(lat, basis_fn)
    rho, eps = 1.3, 1e-3
    base = rho * w  # equilibrium at rest
    for k, (name, phi, cls) in enumerate(rows):
        if cls == "cons":
            continue
        fin = base + eps * phi
        assert fin.sum() == pytest.approx(rho, rel=1e-15)
        assert np.allclose(fin @ c, 0.0, atol=1e-15)
        fout, r, u = sim.collide_cell(fin, [0.0, 0.0, 0.0])
        assert np.allclose(u, 0.0, atol=1e-15)
        dm = M @ (fout - base)
        expect = np.zeros(len(w))
        expect[k] = (1 - S[k]) * (phi @ phi) * eps
        np.testing.assert_allclose(dm, expect, atol=1e-12, err_msg=f"moment {name}")


@pytest.mark.parametrize("lat,basis_fn", CASES, ids=["D2Q9", "D3Q19"])
def test_forced_collision_follows_the_moment_definition(lat, basis_fn):
    c, w, cs2, rows, M, S, sim, dim = setup(lat, basis_fn)
    rng = np.random.default_rng(5)
    for _ in range(6):
        fin = w * rng.uniform(0.6, 1.8, size=len(w))
        F = np.zeros(3)
        F[:dim] = rng.normal(scale=0.02, size=dim)
        fout, rho, u = sim.collide_cell(fin, F)
        # Eq. 4: equilibrium and Guo source at u = (j + F/2)/rho
        u_ = (fin @ c + 0.5 * F) / fin.sum()
        cu = c @ u_
        feq = fin.sum() * w * (1 + cu / cs2 + cu ** 2 / (2 * cs2 ** 2) - (u_ @ u_) / (2 * cs2))
        src = w * (((c - u_) @ F) / cs2 + cu * (c @ F) / cs2 ** 2)
        m, meq, msrc = M @ fin, M @ feq, M @ src
        expect = m - S * (m - meq) + (1 - S / 2) * msrc
        np.testing.assert_allclose(M @ fout, expect, rtol=1e-12, atol=1e-14)
