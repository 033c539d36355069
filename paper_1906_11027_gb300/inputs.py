"""Seeded synthetic workloads.  Random draws only: no step of the method is
computed here, so tests, the benchmark and the oracle can share these inputs.

sweep_domains: the parameter sweep of independent periodic D2Q9 droplets -- side L
uniform in {64, 96, 128, 192, 256}, G ~ U[-5.5, -4.3], tau in {0.6, 0.8, 1.0},
R ~ U[8, 0.35 L], force-stencil order in {4, 6, 8, 10}; every droplet starts from
the tanh profile with rho_l = 2.0, rho_g = 0.15, width 2.  Seed 11027.
"""
from __future__ import annotations

import numpy as np

SWEEP_SEED = 11027
SWEEP_SIZES = (64, 96, 128, 192, 256)


def sweep_domains(n: int = 512, seed: int = SWEEP_SEED, sizes=SWEEP_SIZES):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = int(rng.choice(sizes))
        out.append(dict(nx=L, ny=L,
                        G=float(rng.uniform(-5.5, -4.3)),
                        tau=float(rng.choice([0.6, 0.8, 1.0])),
                        R=float(rng.uniform(8.0, 0.35 * L)),
                        stencil=int(rng.choice([4, 6, 8, 10])),
                        rho_l=2.0, rho_g=0.15, width=2.0))
    return out
