"""Pins of the oracle's initial state and of its interface-thickness count.

- Initial state (Sec. 3 droplet test, readings R3 and R15): the density is the
  tanh profile rho0 = (rho_l + rho_g)/2 - (rho_l - rho_g)/2 tanh(2 (r - R) / W),
  r the minimum-image distance to the centre node (n/2 on every axis, integer
  division), and the populations are feq(rho0, u = 0) = w_b rho0.  The flat
  slab uses the same profile with r the distance to the middle node along the
  normal axis and R = L/4.  The expected values here are computed from that
  statement alone: the images are searched explicitly, and the weights come
  from Table 1 (tests/golden/table1_lattices.json).  Odd and even sizes put
  the centre node on both sides of the geometric middle.
- Thickness (Sec. 3, Fig. 5): the number of nodes on the x line through the
  centre whose density lies in [1.05 rho_g, 0.95 rho_l], with rho_l read at the
  centre node and rho_g at node 0.  On a freshly initialised slab or droplet
  the densities are the closed-form profile, so the count follows by direct
  enumeration.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NAMES = {oracle.D2Q9: "D2Q9", oracle.D2Q13: "D2Q13", oracle.D2Q25: "D2Q25"}


def table1_weights(lat):
    """Velocities and weights of Table 1 (2-D lattices) or of the standard D3Q19
    set, as {velocity: weight}."""
    if lat == oracle.D3Q19:
        out = {(0, 0, 0): 1 / 3}
        for v in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            for s in (1, -1):
                out[tuple(s * np.array(v))] = 1 / 18
        for i, j in ((0, 1), (0, 2), (1, 2)):
            for si in (1, -1):
                for sj in (1, -1):
                    v = [0, 0, 0]
                    v[i], v[j] = si, sj
                    out[tuple(v)] = 1 / 36
        return out
    with open(os.path.join(GOLD, "table1_lattices.json")) as fh:
        shells = json.load(fh)[NAMES[lat]]["w"]
    out = {}
    for c2, w in shells.items():
        for x in range(-3, 4):
            for y in range(-3, 4):
                if x * x + y * y == int(c2):
                    out[(x, y, 0)] = float(Fraction(w))
    return out


def min_image_dist(i, n):
    """|i - n//2| over the periodic images, searched explicitly."""
    d = np.asarray(i, dtype=float) - (n // 2)
    return np.min(np.abs(np.stack([d, d - n, d + n])), axis=0)


def tanh_profile(r, rho_l, rho_g, R, W):
    return 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - R) / W)


def expected_populations(lat, rho0):
    sim_c, _, _ = oracle.lattice_table(lat)
    weights = table1_weights(lat)
    w = np.array([weights[tuple(int(v) for v in c)] for c in sim_c])
    return w[:, None, None, None] * rho0[None]


@pytest.mark.parametrize("lat,shape,R,W", [
    (oracle.D2Q9, (1, 29, 37), 9.0, 2.0),
    (oracle.D2Q9, (1, 64, 64), 16.0, 2.0),
    (oracle.D2Q25, (1, 30, 31), 7.5, 3.0),
    (oracle.D3Q19, (11, 20, 15), 4.0, 2.0),
    (oracle.D3Q19, (16, 16, 16), 5.0, 4.0),
])
def test_droplet_initial_state_is_the_tanh_profile(lat, shape, R, W):
    nz, ny, nx = shape
    sim = oracle.Sim(lat, nx, ny, nz)
    sim.init_droplet(2.0, 0.15, R, W)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = min_image_dist(x, nx) ** 2 + min_image_dist(y, ny) ** 2
    if lat == oracle.D3Q19:
        r2 = r2 + min_image_dist(z, nz) ** 2
    rho0 = tanh_profile(np.sqrt(r2), 2.0, 0.15, R, W)
    np.testing.assert_allclose(sim.get_f(), expected_populations(lat, rho0), rtol=1e-14, atol=0)
    # the centre node (n/2 on each axis) carries the liquid side of the profile
    rc = tanh_profile(0.0, 2.0, 0.15, R, W)
    assert sim.get_f().sum(axis=0)[nz // 2 if lat == oracle.D3Q19 else 0, ny // 2, nx // 2] == pytest.approx(rc)


@pytest.mark.parametrize("lat,shape,axis,W", [
    (oracle.D2Q9, (1, 6, 41), 0, 2.0),
    (oracle.D2Q9, (1, 40, 5), 1, 3.0),
    (oracle.D2Q13, (1, 4, 64), 0, 4.0),
    (oracle.D3Q19, (21, 4, 6), 2, 2.0),
])
def test_flat_initial_state_is_the_tanh_slab(lat, shape, axis, W):
    nz, ny, nx = shape
    sim = oracle.Sim(lat, nx, ny, nz)
    sim.init_flat(1.9, 0.12, W, axis=axis)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, L = ((x, nx), (y, ny), (z, nz))[axis]
    rho0 = tanh_profile(min_image_dist(i, L), 1.9, 0.12, 0.25 * L, W)
    np.testing.assert_allclose(sim.get_f(), expected_populations(lat, rho0), rtol=1e-14, atol=0)


def band_count(line, rho_l, rho_g):
    lo, hi = 1.05 * rho_g, 0.95 * rho_l
    # no node sits so close to an edge of the band that rounding could move it
    assert np.min(np.abs(line - lo)) > 1e-9 and np.min(np.abs(line - hi)) > 1e-9
    return int(np.count_nonzero((line >= lo) & (line <= hi)))


@pytest.mark.parametrize("nx,ny,W", [(64, 6, 6.0), (81, 5, 3.0), (50, 8, 10.0)])
def test_thickness_counts_band_nodes_of_a_flat_slab(nx, ny, W):
    sim = oracle.Sim(oracle.D2Q9, nx, ny)
    sim.init_flat(1.9, 0.12, W, axis=0)
    line = tanh_profile(min_image_dist(np.arange(nx), nx), 1.9, 0.12, 0.25 * nx, W)
    expect = band_count(line, line[nx // 2], line[0])
    assert expect >= 4  # both interfaces contribute several nodes
    assert sim.observables()["thickness"] == expect


def test_thickness_counts_band_nodes_through_a_droplet_centre():
    nx, ny, R, W = 48, 36, 10.0, 5.0
    sim = oracle.Sim(oracle.D2Q9, nx, ny)
    sim.init_droplet(1.9, 0.12, R, W)
    # the x line through the centre row: r = |x - nx/2| (the row is y = ny/2)
    line = tanh_profile(min_image_dist(np.arange(nx), nx), 1.9, 0.12, R, W)
    corner = tanh_profile(np.hypot(nx // 2, ny // 2), 1.9, 0.12, R, W)
    expect = band_count(line, line[nx // 2], corner)
    assert expect >= 4
    assert sim.observables()["thickness"] == expect
