"""The temperature sweeps of the paper's Sec. 3, for D2Q9 with force stencils
of 4th/6th/8th-order isotropy and for the consistent D2Q13 / D2Q25 models
(lattice = force stencil).  D2Q13 and D2Q25 run at tau = 1 ("T") and at the
equal-viscosity tau = 11/12 and 19/24 ("V"), as in Fig. 3.

--case droplet (Figs. 2-3): a static Peng-Robinson droplet on a 60 x 60
periodic box, r0 = 15, run to steady state and then --extra steps
further (the line gives the relative drift over those); it reports max|u| and
mean|u| (the spurious currents) with the centre and far-corner densities.

--case flat (Figs. 4-5): a liquid slab between two flat interfaces normal to x
on a periodic 200 x 8 strip, started from the Maxwell densities; the line
reports the coexistence densities against the Maxwell construction and the
interface thickness, i.e. the width of the region 1.05 rho_v <= rho <=
0.95 rho_l with the run's own bulk densities: the node count per interface and
the distance between the linearly interpolated crossings of the two levels.

--case wall (Fig. 6): a droplet on a flat wall at T/Tc = 0.9 (--temps), on a
160 x 80 fluid region above a two-row solid band with standard bounce-back,
for wall densities rho_w = 1.5 and 4.5 (--rho-w) and D2Q9 E4 / E8 and D2Q25;
the line reports the contact angle of a circle fitted to the interface, the
droplet's base and height, and the spurious currents.

    python -m paper_1906_11027_gb300.experiments [--case flat|wall] [--forcing edm] [--temps 0.7,0.8,0.9]

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
          ("D2Q9 E8", lbm.LBM_D2Q9, 8, 1.0), ("D2Q13T", lbm.LBM_D2Q13, 0, 1.0),
          ("D2Q13V", lbm.LBM_D2Q13, 0, 11.0 / 12.0), ("D2Q25T", lbm.LBM_D2Q25, 0, 1.0),
          ("D2Q25V", lbm.LBM_D2Q25, 0, 19.0 / 24.0))


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


def interface_thickness(line, rho_v, rho_l):
    """Width of the rising interface of a periodic line profile (vapour at the
    ends, liquid in the middle) between the levels 1.05 rho_v and 0.95 rho_l:
    (nodes inside the band on each of the two interfaces, the mean of both, and
    the mean distance between the interpolated level crossings)."""
    lo, hi = 1.05 * rho_v, 0.95 * rho_l
    n = len(line)
    half = n // 2
    inside = (line >= lo) & (line <= hi)
    counts = (int(inside[:half].sum()), int(inside[half:].sum()))

    def crossing(seg, level):
        # first index i with seg[i] < level <= seg[i+1], interpolated linearly
        for i in range(len(seg) - 1):
            if seg[i] < level <= seg[i + 1]:
                return i + (level - seg[i]) / (seg[i + 1] - seg[i])
        return float("nan")
    rise = line[:half + 1]
    fall = line[half:][::-1]  # the falling interface read from the far side
    widths = [crossing(seg, hi) - crossing(seg, lo) for seg in (rise, fall)]
    return counts, float(np.mean(widths))


def fit_contact_angle(rho, rows, level):
    """Contact angle (degrees, through the liquid) of a sessile droplet: a
    least-squares circle x^2 + y^2 + D x + E y + F = 0 through the interface
    points (rho = level, linear interpolation along rows and columns, away
    from the two rows next to the wall), measured against the wall surface
    half-way between the last solid row and the first fluid row.  Returns
    (angle, base width at the surface, height above it, radius)."""
    ny, nx = rho.shape
    pts = []
    for y in range(rows + 2, ny):
        line = rho[y]
        if line.max() < level:
            continue
        i = int(np.argmax(line >= level))
        if 0 < i:
            pts.append((i - 1 + (level - line[i - 1]) / (line[i] - line[i - 1]), y))
        j = nx - 1 - int(np.argmax(line[::-1] >= level))
        if j < nx - 1:
            pts.append((j + (line[j] - level) / (line[j] - line[j + 1]), y))
    for x in range(nx):
        col = rho[rows + 2:, x]
        if col.max() < level:
            continue
        k = len(col) - 1 - int(np.argmax(col[::-1] >= level))
        if k < len(col) - 1:
            pts.append((x, rows + 2 + k + (col[k] - level) / (col[k] - col[k + 1])))
    if len(pts) < 6:
        raise ValueError(f"only {len(pts)} interface points at level {level:.4g}")
    P = np.array(pts)
    Am = np.column_stack([P[:, 0], P[:, 1], np.ones(len(P))])
    D, E, F = np.linalg.lstsq(Am, -(P ** 2).sum(1), rcond=None)[0]
    xc, yc = -D / 2.0, -E / 2.0
    R = float(np.sqrt(xc * xc + yc * yc - F))
    ys = rows - 0.5
    h = yc - ys
    cos_t = float(np.clip(-h / R, -1.0, 1.0))
    base = 2.0 * float(np.sqrt(max(R * R - h * h, 0.0)))
    return float(np.degrees(np.arccos(cos_t))), base, h + R, R


def run_wall(a, T, Tc, rv, rl, name, lat, st, tau, coll, rho_w):
    rows, nx, ny = 2, a.wall_nx, a.wall_ny + 2
    dom = lbm.Domain(nx, ny, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=T,
                     G=-1.0, tau=tau, collision=coll, wall_rows=rows, rho_w=rho_w)
    try:
        x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
        r = np.hypot(x - nx // 2, y - rows)
        rho0 = 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2.0 * (r - a.wall_r0) / 3.0)
        rho0[:rows] = rho0[rows]
        dom.init_from_rho(rho0)
        steps, ok = dom.run_to_steady(1e-10, a.max_steps, 100)
        u1 = dom.observables()["max_u"]
        dom.step(a.extra)
        o = dom.observables()
        rho = dom.fields()["rho"][0]
        r_l = float(rho[rows + 2:, nx // 2].max())
        r_v = float(np.median(rho[rows + 2:, 0]))
        row = dict(T_over_Tc=T, model=name, forcing=a.forcing, tau=round(tau, 4), rho_w=rho_w, steps=steps,
                   steady=ok, rho_l=r_l, rho_v=r_v, rho_min=float(rho[rows:].min()),
                   rho_max=float(rho[rows:].max()), max_u=o["max_u"], mean_u=o["mean_u"], extra_steps=a.extra,
                   max_u_drift=abs(o["max_u"] / u1 - 1.0))
        try:
            theta, base, height, R = fit_contact_angle(rho, rows, 0.5 * (r_l + r_v))
            row.update(contact_angle_deg=theta, base=base, height=height, radius=R)
        except ValueError as e:
            row.update(fit_error=str(e))
        return row
    finally:
        dom.close()


def run_droplet(a, T, Tc, rv, rl, name, lat, st, tau, coll):
    dom = lbm.Domain(a.n, a.n, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=T,
                     G=-1.0, tau=tau, collision=coll)
    try:
        dom.init_droplet(rl, rv, a.r0, 3.0)
        steps, ok = dom.run_to_steady(1e-10, a.max_steps, 100)
        o1 = dom.observables()
        dom.step(a.extra)
        o = dom.observables()
        return dict(T_over_Tc=T, model=name, forcing=a.forcing, tau=round(tau, 4), steps=steps, steady=ok,
                    max_u=o["max_u"], mean_u=o["mean_u"], rho_l=o["rho_l"], rho_v=o["rho_g"],
                    maxwell_rho_l=rl, maxwell_rho_v=rv, extra_steps=a.extra,
                    max_u_drift=abs(o["max_u"] / o1["max_u"] - 1.0))
    finally:
        dom.close()


def run_flat(a, T, Tc, rv, rl, name, lat, st, tau, coll):
    dom = lbm.Domain(a.flat_nx, 8, lattice=lat, stencil=st, psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=T,
                     G=-1.0, tau=tau, collision=coll)
    try:
        dom.init_flat(rl, rv, 3.0, 0)
        steps, ok = dom.run_to_steady(1e-10, a.max_steps, 100)
        rho_v1 = dom.observables()["rho_g"]
        dom.step(a.extra)
        o = dom.observables()
        line = dom.fields()["rho"][0, 4, :]
        rho_l, rho_v = float(line[a.flat_nx // 2]), float(line[0])
        counts, width = interface_thickness(line, rho_v, rho_l)
        return dict(T_over_Tc=T, model=name, forcing=a.forcing, tau=round(tau, 4), steps=steps, steady=ok,
                    rho_l=rho_l, rho_v=rho_v, maxwell_rho_l=rl, maxwell_rho_v=rv,
                    rho_l_rel_dev=rho_l / rl - 1.0, rho_v_rel_dev=rho_v / rv - 1.0,
                    thickness_nodes=counts, thickness=width, max_u=o["max_u"], extra_steps=a.extra,
                    rho_v_drift=abs(rho_v / rho_v1 - 1.0))
    finally:
        dom.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--temps", default="0.6,0.7,0.8,0.85,0.9,0.95")
    ap.add_argument("--n", type=int, default=60)
    ap.add_argument("--r0", type=float, default=15.0)
    ap.add_argument("--max-steps", type=int, default=200000)
    ap.add_argument("--forcing", choices=["guo", "edm"], default="guo")
    ap.add_argument("--case", choices=["droplet", "flat", "wall"], default="droplet")
    ap.add_argument("--rho-w", default="1.5,4.5", help="wall densities of --case wall")
    ap.add_argument("--wall-nx", type=int, default=160)
    ap.add_argument("--wall-ny", type=int, default=80)
    ap.add_argument("--wall-r0", type=float, default=25.0)
    ap.add_argument("--flat-nx", type=int, default=200)
    ap.add_argument("--extra", type=int, default=20000,
                    help="steps run after the steady test passes; the values reported are taken after them, "
                         "with their drift over those steps")
    ap.add_argument("--models", default="", help="comma-separated subset of: " + ", ".join(m[0] for m in MODELS))
    a = ap.parse_args()
    wanted = a.models or ("D2Q9 E4,D2Q9 E8,D2Q25V" if a.case == "wall" else "")
    models = [m for m in MODELS if not wanted or m[0] in wanted.split(",")]
    run = {"droplet": run_droplet, "flat": run_flat, "wall": run_wall}[a.case]
    wall_densities = [float(v) for v in a.rho_w.split(",")] if a.case == "wall" else [None]
    coll = lbm.LBM_BGK_EDM if a.forcing == "edm" else lbm.LBM_BGK
    lbm.load()
    Tc = critical_T()
    for T in [float(t) for t in a.temps.split(",")]:
        rv, rl = maxwell(T, Tc)
        for name, lat, st, tau in models:
            for rho_w in wall_densities:
                extra = (rho_w,) if a.case == "wall" else ()
                try:
                    row = run(a, T, Tc, rv, rl, name, lat, st, tau, coll, *extra)
                except lbm.LbmError as e:
                    row = dict(T_over_Tc=T, model=name, forcing=a.forcing, tau=round(tau, 4), case=a.case,
                               rho_w=rho_w, error=str(e))
                print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
