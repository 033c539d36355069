"""Host-side analysis of the Sec. 3 temperature sweeps: the interface-thickness
measure (the region 1.05 rho_v <= rho <= 0.95 rho_l of a flat interface) and
the Peng-Robinson helpers of the experiment module, checked against closed
forms and against the independent forms in tests/theory.py."""
import numpy as np
import pytest

from paper_1906_11027_gb300 import experiments as ex
from theory import maxwell, pr_critical_T


def _tanh_slab(n, rv, rl, w, x1, x2):
    x = np.arange(n, dtype=float)
    return rv + (rl - rv) * 0.5 * (np.tanh((x - x1) / w) - np.tanh((x - x2) / w))


@pytest.mark.parametrize("w", [1.5, 3.0, 6.0])
def test_thickness_of_a_tanh_slab_matches_the_closed_form(w):
    n, rv, rl = 400, 0.05, 7.0
    line = _tanh_slab(n, rv, rl, w, 100.3, 300.3)
    counts, width = ex.interface_thickness(line, line[0], line[n // 2])
    # one tanh interface crosses rho = rv + (rl - rv) (1 + tanh(s/w)) / 2 at
    # s = w artanh(2 (rho - rv) / (rl - rv) - 1)
    lo, hi = 1.05 * line[0], 0.95 * line[n // 2]
    s = [w * np.arctanh(2.0 * (v - line[0]) / (line[n // 2] - line[0]) - 1.0) for v in (lo, hi)]
    exact = s[1] - s[0]
    assert width == pytest.approx(exact, rel=0.03)
    # the node count brackets the continuous width
    for c in counts:
        assert exact - 1.0 <= c <= exact + 1.0


def test_thickness_of_a_step_profile():
    # no node lies inside the band; the interpolated profile is a one-node ramp,
    # so the crossings are (hi - lo) / (rl - rv) apart
    line = np.full(64, 0.1)
    line[16:48] = 5.0
    counts, width = ex.interface_thickness(line, 0.1, 5.0)
    assert counts == (0, 0)
    assert width == pytest.approx((0.95 * 5.0 - 1.05 * 0.1) / (5.0 - 0.1), rel=1e-12)


def test_critical_temperature_matches_the_symbolic_solution():
    assert ex.critical_T() == pytest.approx(pr_critical_T(), rel=1e-10)


@pytest.mark.parametrize("t", [0.6, 0.8, 0.95])
def test_maxwell_densities_match_the_independent_construction(t):
    rv, rl = ex.maxwell(t, ex.critical_T())
    rv2, rl2 = maxwell(t)
    assert rv == pytest.approx(rv2, rel=1e-6)
    assert rl == pytest.approx(rl2, rel=1e-6)


@pytest.mark.parametrize("theta_deg", [50.0, 90.0, 130.0])
def test_contact_angle_of_a_synthetic_cap(theta_deg):
    """A circular cap of known contact angle, drawn as a smooth density field on
    a grid above a two-row band (the wall surface half-way below the first fluid
    row), is recovered by the circle fit to within 2 degrees."""
    rows, nx, ny, R = 2, 160, 90, 30.0
    ys = rows - 0.5
    yc = ys - R * np.cos(np.radians(theta_deg))  # centre height for this angle
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    d = np.hypot(x - 80.0, y - yc) - R
    rho = 0.5 * (6.0 + 0.6) - 0.5 * (6.0 - 0.6) * np.tanh(2.0 * d / 4.0)
    rho[y < ys] = 3.0
    theta, base, height, radius = ex.fit_contact_angle(rho, rows, 3.3)
    assert theta == pytest.approx(theta_deg, abs=2.0)
    assert radius == pytest.approx(R, rel=0.02)
    assert height == pytest.approx(R * (1.0 - np.cos(np.radians(theta_deg))), abs=1.0)
