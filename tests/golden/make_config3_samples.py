"""Writes tests/golden/config3_oracle_samples.txt: the FP64 oracle's iterates
of the full-size 3D workload (depth 5, 243^3 cells, k = 8 pi, exterior
scaling layer of 10% per side with theta = pi/6, centred Gaussian of width
0.05) after one and two BPX cycles (omega = 0.6 on every level, Appendix A
Algorithm 4 with the BPX transfer), started from the seeded random iterate
1e-3 * random_complex(3, 5, 7).  Stored: 1024 seeded sample vertices (flat
index into the (3^5 + 1)^3 vertex array, x fastest) with both iterates'
values there, and the oracle's residual norms |b - H u| of the start and of
both iterates.  A GPU test repeats the two cycles and compares the samples
and the norms.  Calls only the oracle; about five minutes and 3 GB on one
host core.

    python tests/golden/make_config3_samples.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1508_03954_gb300 import workloads as W  # noqa: E402

DEPTH, SAMPLES, CYCLES, OMEGA = 5, 1024, 2, 0.6
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_oracle_samples.txt")


def main():
    c = W.config3(DEPTH)
    n = 3 ** DEPTH
    o = O.Hierarchy(3, DEPTH, c["k2"], c["theta"], c["layer_width"])
    o.set_rhs_nodal(c["f"])
    u0 = W.random_complex(3, DEPTH, 7) * 1e-3
    o.set_solution(u0)
    norms = [float(np.linalg.norm(o.residual()))]
    rng = np.random.default_rng(11)
    ijk = rng.integers(1, n, size=(SAMPLES, 3))  # interior vertices (z, y, x)
    flat = (ijk[:, 0] * (n + 1) + ijk[:, 1]) * (n + 1) + ijk[:, 2]
    its = []
    for _ in range(CYCLES):
        o.cycle(np.full(DEPTH, OMEGA), O.ADD, O.HIERARCHICAL)
        its.append(np.ravel(o.u)[flat].copy())
        norms.append(float(np.linalg.norm(o.residual())))
    with open(OUT, "w") as fh:
        fh.write("# " + json.dumps({"depth": DEPTH, "variant": "BPX (ADD + HIERARCHICAL)", "omega": OMEGA,
                                    "u0": "1e-3 * random_complex(3, 5, 7)", "cycles": CYCLES,
                                    "residual_norms": norms}) + "\n")
        fh.write("# flat_index re(u_1) im(u_1) re(u_2) im(u_2)\n")
        for k in range(SAMPLES):
            fh.write(f"{flat[k]} {its[0][k].real:.17e} {its[0][k].imag:.17e} "
                     f"{its[1][k].real:.17e} {its[1][k].imag:.17e}\n")


if __name__ == "__main__":
    main()
