"""Writes tests/golden/config3_oracle_samples.txt: the FP64 oracle's iterates
of the full-size 3D workload (depth 5, 243^3 cells, k = 8 pi, exterior
scaling layer of 10% per side with theta = pi/6, centred Gaussian of width
0.05) after one and two cycles (omega = 0.6 on every level, Appendix A
Algorithm 4) of each variant -- additive, hierarchical basis, BPX, and the
hierarchical basis with the hierarchical transfer -- each started from the
seeded random iterate 1e-3 * random_complex(3, 5, 7).  Stored per variant: a
header line with the residual norms |b - H u| of the start and of both
iterates, then 512 seeded sample vertices (flat index into the (3^5 + 1)^3
vertex array, x fastest, the same for every variant) with both iterates'
values there.  A GPU test repeats the cycles and compares the samples and
the norms.  Calls only the oracle; about five minutes and 3 GB per variant
on one host core.

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

DEPTH, SAMPLES, CYCLES, OMEGA = 5, 512, 2, 0.6
VARIANTS = {"add": (O.ADD, O.DLINEAR), "hb": (O.HB, O.DLINEAR), "bpx": (O.ADD, O.HIERARCHICAL),
            "hb-hier": (O.HB, O.HIERARCHICAL)}
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_oracle_samples.txt")


def main():
    c = W.config3(DEPTH)
    n = 3 ** DEPTH
    rng = np.random.default_rng(11)
    ijk = rng.integers(1, n, size=(SAMPLES, 3))  # interior vertices (z, y, x)
    flat = (ijk[:, 0] * (n + 1) + ijk[:, 1]) * (n + 1) + ijk[:, 2]
    u0 = W.random_complex(3, DEPTH, 7) * 1e-3
    o = O.Hierarchy(3, DEPTH, c["k2"], c["theta"], c["layer_width"])
    o.set_rhs_nodal(c["f"])
    with open(OUT, "w") as fh:
        for name, (var, tr) in VARIANTS.items():
            o.set_solution(u0)
            norms = [float(np.linalg.norm(o.residual()))]
            its = []
            for _ in range(CYCLES):
                o.cycle(np.full(DEPTH, OMEGA), var, tr)
                its.append(np.ravel(o.u)[flat].copy())
                norms.append(float(np.linalg.norm(o.residual())))
            fh.write("# " + json.dumps({"variant": name, "depth": DEPTH, "omega": OMEGA,
                                        "u0": "1e-3 * random_complex(3, 5, 7)", "cycles": CYCLES,
                                        "residual_norms": norms, "samples": SAMPLES}) + "\n")
            fh.write("# flat_index re(u_1) im(u_1) re(u_2) im(u_2)\n")
            for k in range(SAMPLES):
                fh.write(f"{flat[k]} {its[0][k].real:.17e} {its[0][k].imag:.17e} "
                         f"{its[1][k].real:.17e} {its[1][k].imag:.17e}\n")
            fh.flush()


if __name__ == "__main__":
    main()
