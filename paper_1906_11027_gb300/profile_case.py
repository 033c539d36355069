"""Small profiling driver: one domain, a few directly launched steps, so that a
profiler can capture individual kernels.

    python -m paper_1906_11027_gb300.profile_case --lattice d3q19 --n 128 [--nz 32] --steps 6 \
        [--precision fp32|fp64] [--stencil 4] [--coll bgk|mrt] [--path auto|two|one] [--schedule NAME]
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1906_11027_gb300 import lbm  # noqa: E402

LATTICES = {"d2q9": lbm.LBM_D2Q9, "d3q19": lbm.LBM_D3Q19, "d2q13": lbm.LBM_D2Q13, "d2q25": lbm.LBM_D2Q25}
COLLS = {"bgk": lbm.LBM_BGK, "mrt": lbm.LBM_MRT}
PATHS = {"auto": lbm.LBM_PATH_AUTO, "two": lbm.LBM_PATH_TWO_PASS, "one": lbm.LBM_PATH_ONE_PASS}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", choices=sorted(LATTICES), default="d3q19")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--nz", type=int, default=0, help="3-D: number of z planes (default n)")
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--stencil", type=int, default=0)
    ap.add_argument("--coll", choices=sorted(COLLS), default="bgk")
    ap.add_argument("--path", choices=sorted(PATHS), default="auto")
    ap.add_argument("--schedule", default=None, help="pin a schedule by name (lbm_schedule_report)")
    a = ap.parse_args()
    lat = LATTICES[a.lattice]
    nz = (a.nz or a.n) if lat == lbm.LBM_D3Q19 else 1
    dom = lbm.Domain(a.n, a.n, nz, lattice=lat, stencil=a.stencil,
                     precision=lbm.LBM_FP32_SHIFTED if a.precision == "fp32" else lbm.LBM_FP64,
                     collision=COLLS[a.coll], path=PATHS[a.path])
    if a.schedule:
        dom.set_schedule(a.schedule)
    dom.init_droplet(2.0, 0.15, 0.15 * a.n, 2.0)
    for _ in range(a.steps):  # one call per step: no graph replay
        dom.step(1)
    print("mass", dom.observables()["mass"])


if __name__ == "__main__":
    main()
