"""Closed-form predictions the tests compare against (no oracle, no library).

mechanical_stability: coexistence densities (rho_g, rho_l) of a flat interface
for psi = 1 - exp(-rho) and p = c_s^2 rho + (G c_s^2 / 2) psi^2, from equal
bulk pressures and  int_{rho_g}^{rho_l} (p0 - p) psi' / psi^(1 + eps) drho = 0;
eps = 0 is the value the discrete pressure tensor of the nearest-neighbour
force gives with Guo forcing.
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
