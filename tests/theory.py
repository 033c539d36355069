"""Closed-form predictions the tests compare against (no oracle, no library).

mechanical_stability: coexistence densities (rho_g, rho_l) of a flat interface
for psi = 1 - exp(-rho) and p = c_s^2 rho + (G c_s^2 / 2) psi^2, from equal
bulk pressures and  int_{rho_g}^{rho_l} (p0 - p) psi' / psi^(1 + eps) drho = 0;
eps = 0 is the published value for the nearest-neighbour force with Guo
forcing: Shan, Phys. Rev. E 77, 066702 (2008) derives the force's pressure
tensor, whose gradient part has no (grad psi)^2 term, and Li, Luo & Li,
Phys. Rev. E 86, 016709 (2012) give eps = -2 alpha / beta for Guo's scheme,
alpha and beta the coefficients of (grad psi)^2 and psi lap(psi) in it.
"""
import numpy as np
from scipy.integrate import quad
from scipy.optimize import fsolve


def mechanical_stability(G, eps, cs2=1 / 3):
    psi = lambda r: -np.expm1(-r)
    dpsi = lambda r: np.exp(-r)
    p = lambda r: cs2 * r + 0.5 * G * cs2 * psi(r) ** 2

    def eqs(v):
        rg, rl = v
        p0 = p(rl)
        integral = quad(lambda r: (p0 - p(r)) * dpsi(r) / psi(r) ** (1 + eps), rg, rl,
                        epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        return [p(rg) - p(rl), integral]
    # start from the spinodal pair (dp/drho = 0) widened outwards, which keeps
    # fsolve off the trivial rho_g = rho_l root near the critical coupling
    r = np.linspace(1e-3, 4.0, 40001)
    dp = np.gradient(p(r), r)
    neg = np.where(dp < 0)[0]
    guess = [0.5 * r[neg[0]], 1.5 * r[neg[-1]]] if len(neg) else [0.12, 1.9]
    rg, rl = fsolve(eqs, guess, xtol=1e-13)
    assert rl - rg > 1e-3, "no phase separation at this G"
    return np.array([rg, rl])


# Peng-Robinson EOS of the paper's Sec. 3 (a = 2/49, b = 2/21, R = 1, omega = 0.344)
PR_A, PR_B, PR_OMEGA = 2.0 / 49.0, 2.0 / 21.0, 0.344


def _pr_p(rho, T, alpha):
    return rho * T / (1.0 - PR_B * rho) - PR_A * alpha * rho ** 2 / (1.0 + 2.0 * PR_B * rho - (PR_B * rho) ** 2)


_TC = []


def pr_critical_T():
    """Critical temperature of the EOS with alpha = 1: dp/drho = d2p/drho2 = 0,
    with exact (symbolic) derivatives."""
    if not _TC:
        import sympy as sp
        rho, T = sp.symbols("rho T", positive=True)
        a, b = sp.Rational(2, 49), sp.Rational(2, 21)
        p = rho * T / (1 - b * rho) - a * rho ** 2 / (1 + 2 * b * rho - (b * rho) ** 2)
        sol = sp.nsolve([sp.diff(p, rho), sp.diff(p, rho, 2)], [rho, T], [2.6, 0.073], prec=30)
        _TC.append(float(sol[1]))
    return _TC[0]


def pr_pressure(rho, T_over_Tc, Tc=None):
    Tc = pr_critical_T() if Tc is None else Tc
    k = 0.37464 + 1.54226 * PR_OMEGA - 0.26992 * PR_OMEGA ** 2
    alpha = (1.0 + k * (1.0 - np.sqrt(T_over_Tc))) ** 2
    return _pr_p(rho, T_over_Tc * Tc, alpha)


def maxwell(T_over_Tc):
    """Equal-area coexistence of the P-R isotherm: p(rv) = p(rl) = p0 and
    int_{rv}^{rl} (p - p0) / rho^2 drho = 0."""
    from scipy.optimize import brentq
    Tc = pr_critical_T()
    p = lambda r: pr_pressure(r, T_over_Tc, Tc)
    rho = np.linspace(1e-3, 10.0, 40001)
    dp = np.gradient(p(rho), rho)
    spin = rho[np.where(np.diff(np.sign(dp)) != 0)[0]]
    r_max, r_min = spin[0], spin[1]

    def area(p0):
        rv = brentq(lambda r: p(r) - p0, 1e-12, r_max)
        rl = brentq(lambda r: p(r) - p0, r_min, 9.9)
        return quad(lambda r: (p(r) - p0) / r ** 2, rv, rl, limit=400)[0], rv, rl

    lo, hi = max(p(r_min), p(1e-6)), p(r_max)
    p0 = brentq(lambda q: area(q)[0], lo + 1e-14, hi - 1e-14, xtol=1e-15)
    _, rv, rl = area(p0)
    return rv, rl
