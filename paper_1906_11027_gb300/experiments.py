"""Spurious currents against temperature, the comparison of the paper's Sec. 3
(Figs. 2-3): a static Peng-Robinson droplet on a 60 x 60 periodic box,
r0 = 15, for D2Q9 with force stencils of 4th/6th/8th-order isotropy and for the
consistent D2Q13 / D2Q25 models (lattice = force stencil), at the paper's
equal-viscosity relaxation times (tau = 1, 11/12, 19/24).  Each run goes to
steady state; the line reports max|u|, the coexistence densities and steps.

    python -m paper_1906_11027_gb300.experiments [--temps 0.6,0.7,0.8,0.9,0.95] [--forcing edm]

--forcing guo (the default) uses Guo's scheme with BGK; --forcing edm uses the
exact-difference method the paper's own runs use.  The figures' data are not
available, so the numbers show the trend, not the paper's curves.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1906_11027_gb300 import lbm  # noqa: E402

# Peng-Robinson of Sec. 3: a = 2/49, b = 2/21, R = 1, omega = 0.344
A, B, OMEGA = 2.0 / 49.0, 2.0 / 21.0, 0.344
MODELS = (("D2Q9 E4", lbm.LBM_D2Q9, 4, 1.0), ("D2Q9 E6", lbm.LBM_D2Q9, 6, 1.0),
          ("D2Q9 E8", lbm.LBM_D2Q9, 8, 1.0), ("D2Q13", lbm.LBM_D2Q13, 0, 11.0 / 12.0),
          ("D2Q25", lbm.LBM_D2Q25, 0, 19.0 / 24.0))


def _p(rho, T, alpha):
    return rho * T / (1.0 - B * rho) - A * alpha * rho ** 2 / (1.0 + 2.0 * B * rho - (B * rho) ** 2)


def critical_T():
    from scipy.optimize import fsolve

    def eqs(v):  # dp/drho = d2p/drho2 = 0 with alpha = 1, analytic derivatives
        r, T = v
        u = 1.0 + 2.0 * B * r - (B * r) ** 2
        du = 2.0 * B - 2.0 * B * B * r
        d1 = T / (1.0 - B * r) ** 2 - A * (2.0 * r * u - r * r * du) / u ** 2
        num = 2.0 * r * u - r * r * du
        dnum = 2.0 * u + 2.0 * r * du - 2.0 * r * du - r * r * (-2.0 * B * B)
        d2 = 2.0 * B * T / (1.0 - B * r) ** 3 - A * (dnum * u * u - num * 2.0 * u * du) / u ** 4
        return [d1, d2]
    return float(fsolve(eqs, [2.6, 0.073], xtol=1e-12)[1])


def maxwell(T_over_Tc, Tc):
    """Equal-area coexistence densities (rho_v, rho_l) of the isotherm."""
    from scipy.integrate import quad
    from scipy.optimize import brentq
    k = 0.37464 + 1.54226 * OMEGA - 0.26992 * OMEGA ** 2
    alpha = (1.0 + k * (1.0 - np.sqrt(T_over_Tc))) ** 2
    p = lambda r: _p(r, T_over_Tc * Tc, alpha)  # noqa: E731
    rho = np.linspace(1e-3, 10.0, 40001)
    dp = np.gradient(p(rho), rho)
    spin = rho[np.where(np.diff(np.sign(dp)) != 0)[0]]
    r_max, r_min = spin[0], spin[1]

    def area(p0):
        rv = brentq(lambda r: p(r) - p0, 1e-12, r_max)
        rl = brentq(lambda r: p(r) - p0, r_min, 9.9)
        return quad(lambda r: (p(r) - p0) / r ** 2, rv, rl, limit=400)[0], rv, rl

    p0 = brentq(lambda q: area(q)[0], max(p(r_min), p(1e-6)) + 1e-14, p(r_max) - 1e-14, xtol=1e-15)
    _, rv, rl = area(p0)
    return rv, rl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--temps", default="0.6,0.7,0.8,0.85,0.9,0.95")
    ap.add_argument("--n", type=int, default=60)
    ap.add_argument("--r0", type=float, default=15.0)
    ap.add_argument("--max-steps", type=int, default=200000)
    ap.add_argument("--forcing", choices=["guo", "edm"], default="guo")
    a = ap.parse_args()
    lbm.load()
    Tc = critical_T()
    rows = []
    for T in [float(t) for t in a.temps.split(",")]:
        rv, rl = maxwell(T, Tc)
        for name, lat, st, tau in MODELS:
            coll = lbm.LBM_BGK_EDM if a.forcing == "edm" else lbm.LBM_BGK
            dom = lbm.Domain(a.n, a.n, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=T,
                             G=-1.0, tau=tau, collision=coll)
            dom.init_droplet(rl, rv, a.r0, 3.0)
            try:
                steps, ok = dom.run_to_steady(1e-10, a.max_steps, 100)
                o = dom.observables()
                row = dict(T_over_Tc=T, model=name, forcing=a.forcing, tau=round(tau, 4), steps=steps, steady=ok,
                           max_u=o["max_u"], mean_u=o["mean_u"], rho_l=o["rho_l"], rho_v=o["rho_g"],
                           maxwell_rho_l=rl, maxwell_rho_v=rv)
            except lbm.LbmError as e:
                row = dict(T_over_Tc=T, model=name, forcing=a.forcing, tau=round(tau, 4), error=str(e))
            dom.close()
            rows.append(row)
            print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
