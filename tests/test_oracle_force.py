"""Pins of the oracle's interaction force, Eq. 1, through its Taylor series, Eq. 2.

(1) Monomial fields psi = 1 + X^a Y^b (Z^c) around a node turn the stencil sum into
    the moment tensors sum_a w_a e_ai e_a^(abc): the oracle's force at that node
    must equal -G c_s^2 e_n (isotropic coefficient) for every rank n up to the
    stencil's order (this fixes weights, shells, sign, the factor G and the
    c_s^2 scaling of the weights).
(2) A plane wave psi = psi0 + eps sin(k.x + phi) gives the exact stencil sum
    eps cos(k.x + phi) S(k); the isotropic Taylor series of S truncated at the
    stencil's order must approach the oracle's force as |k|^(order) (relative).
"""
import itertools
import math
import numpy as np
import pytest

import oracle
from tests.test_oracle_tables import derive_stencil, dfact, even_multi_indices, STENCILS

LAT = {2: oracle.D2Q9, 3: oracle.D3Q19}


@pytest.mark.parametrize("dim,order,shells", STENCILS)
def test_force_on_monomials_gives_isotropic_moments(dim, order, shells):
    G = -1.0
    L = 12
    sim = oracle.Sim(LAT[dim], L, L, L if dim == 3 else 1, stencil=order, G=G)
    cs2 = sim.cs2
    _, e_coef = derive_stencil(dim, shells, order)
    grids = np.meshgrid(*[np.arange(L) - L // 2] * dim, indexing="ij")
    # oracle arrays are [z, y, x]; build coordinates in that layout
    if dim == 2:
        X = grids[0].T[None, :, :]  # y rows, x columns
        Y = grids[1].T[None, :, :]
        coords = (X, Y)
    else:
        Z, Y, X = np.meshgrid(*[np.arange(L) - L // 2] * 3, indexing="ij")
        coords = (X, Y, Z)
    centre = (L // 2,) * 3 if dim == 3 else (0, L // 2, L // 2)
    for n in range(2, order + 3):
        for idx in itertools.product(range(n), repeat=dim):
            if sum(idx) != n - 1:
                continue
            field = np.ones_like(coords[0], dtype=float)
            for comp, p in zip(coords, idx):
                field = field * comp.astype(float) ** p
            F = sim.force_field(1.0 + field)[centre]
            for i in range(dim):
                full = list(idx)
                full[i] += 1
                if any(p % 2 for p in full):
                    expected = 0.0  # odd moments vanish by symmetry
                elif n <= order:
                    expected = -G * cs2 * float(e_coef[n]) * np.prod([dfact(p - 1) for p in full])
                else:
                    continue  # beyond the stencil's order: not isotropic
                assert F[i] == pytest.approx(expected, rel=1e-13, abs=1e-13)


def taylor_S(kvec, e_coef, order):
    """Isotropic Taylor series of S(k) = sum_a w e_a sin(k.e_a), unit weights:
    k sum_m (-1)^m e_(2m+2) |k|^(2m) / (2^m m!) for 2m + 2 <= order."""
    k2 = float(np.dot(kvec, kvec))
    s = 0.0
    for m in range(order // 2):
        s += (-1) ** m * float(e_coef[2 * m + 2]) * k2 ** m / (2 ** m * math.factorial(m))
    return kvec * s


def plane_wave_error(dim, order, L, mode, G=-1.0):
    sim = oracle.Sim(LAT[dim], L, L, L if dim == 3 else 1, stencil=order, G=G)
    shells = dict((o, s) for d, o, s in STENCILS if d == dim)[order]
    _, e_coef = derive_stencil(dim, shells, order)
    k = 2 * np.pi * np.array(mode, dtype=float) / L
    psi0, eps, phase = 0.7, 0.05, 0.3
    if dim == 2:
        Y, X = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
        theta = (k[0] * X + k[1] * Y + phase)[None]
    else:
        Z, Y, X = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
        theta = k[0] * X + k[1] * Y + k[2] * Z + phase
    psi = psi0 + eps * np.sin(theta)
    F = sim.force_field(psi)[..., :dim]
    S = sim.cs2 * taylor_S(k, e_coef, order)
    F_series = (-G) * psi[..., None] * eps * np.cos(theta)[..., None] * S
    scale = np.abs(F_series).max()
    return np.abs(F - F_series).max() / scale


@pytest.mark.parametrize("dim,order,mode,L1", [
    (2, 4, (1, 2), 32), (2, 6, (1, 2), 32), (2, 8, (1, 2), 32), (2, 10, (1, 2), 24),
    (3, 4, (1, 2, 3), 24), (3, 6, (1, 2, 3), 24),
])
def test_force_plane_wave_matches_taylor_series_to_order(dim, order, mode, L1):
    e1 = plane_wave_error(dim, order, L1, mode)
    e2 = plane_wave_error(dim, order, 2 * L1, mode)
    slope = np.log2(e1 / e2)
    # truncation after the |k|^(order-2) term of S: relative error ~ |k|^order
    assert slope == pytest.approx(order, abs=0.35), (e1, e2, slope)
    assert e1 < 0.2


def test_force_sum_over_domain_vanishes():
    """sum_x F(x) = 0: the pair (x, x+e) and (x+e, x) cancel (Eq. 1, +-e symmetry)."""
    rng = np.random.default_rng(1906)
    for lat, order, shape in ((oracle.D2Q9, 10, (1, 23, 29)), (oracle.D3Q19, 6, (9, 10, 11))):
        nz, ny, nx = shape
        sim = oracle.Sim(lat, nx, ny, nz, stencil=order, G=-5.0)
        psi = rng.uniform(0.1, 0.9, size=shape)
        F = sim.force_field(psi)
        assert np.abs(F.sum(axis=(0, 1, 2))).max() < 1e-12 * np.abs(F).sum()
