"""Writes tests/golden/table2_adaptive_oracle.txt: the FP64 oracle's runs of
the channel problem of Section 7.4 on dynamically refined grids (Table 2,
adaptive column set-up): from the regular grid of h = 1/27 with cells down to
h = 1/2187 (depth 7), 50 iterations of one cycle and one step of
feature-based refinement (Section 5.3: 10% refined, 2% erased, 20 bins,
absolute residual veto 1e-2), the solvers of the table with the factors
looked up by succ(v).  Per run: the fine-grid vertices after the last step
and max|r_50| / max|r_0|.  These are the oracle's values, not the paper's
(the printed column is not reproduced by either reading of the veto); they
pin the GPU's dynamic path at the size the bench measures.  Calls only the
oracle; about 13 minutes per run on one host core.

    python tests/golden/make_table2_adaptive.py THETA_DEG SOLVER [...]  # appends one line per run
    python tests/golden/make_table2_adaptive.py --header               # puts the header on top
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from oracle.adaptive import AdaptiveHierarchy  # noqa: E402
from paper_1508_03954_gb300 import workloads as W  # noqa: E402

DEPTH, MIN_LEVEL, ITERS = 7, 3, 50
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "table2_adaptive_oracle.txt")


def run(deg, solver):
    c = W.channel(deg, DEPTH)
    ref = {lev: np.full((3 ** lev,) * 2, lev < MIN_LEVEL) for lev in range(1, DEPTH)}
    o = AdaptiveHierarchy(2, DEPTH, c["k2"], c["theta"], c["layer_width"], ref, c["theta_interior"])
    o.set_rhs_nodal(c["f"])
    r0 = o.residual_max()
    for it in range(1, ITERS + 1):
        if solver == "jacobi":
            w = (W.CHANNEL_OMEGA1 if it % 2 else W.CHANNEL_OMEGA2) if deg == 0 else 0.4
            o.cycle(O.omega_scheme(O.JACOBI, w, DEPTH), O.ADD, O.DLINEAR)
        elif solver == "transition":
            o.cycle(O.omega_scheme(O.TRANSITION, 0.4, DEPTH, it), O.ADD, O.DLINEAR)
        else:
            o.cycle(O.omega_scheme(O.UCG, 0.4, DEPTH), O.ADD, O.HIERARCHICAL)
        o.adapt(MIN_LEVEL, 0.1, 0.02, 20, 1e-2)
    return {"theta_deg": deg, "solver": solver, "fine_vertices": o.fine_vertex_count(),
            "reduction_max_norm": o.residual_max() / r0}


HEADER = """# The FP64 oracle's runs of the channel problem of Section 7.4 (Eq. 08-gaussian)
# on dynamically refined grids, the set-up of Table 2's adaptive column: h = 1/27
# start grid, cells down to h = 1/2187 (depth 7), 50 iterations of one cycle and
# one feature-based refinement step (Section 5.3; absolute residual veto 1e-2).
# Oracle values, not the printed ones.  Written by make_table2_adaptive.py.
"""


def put_header():
    rows = [ln for ln in open(OUT) if ln.strip() and not ln.startswith("#")] if os.path.exists(OUT) else []
    with open(OUT, "w") as fh:
        fh.write(HEADER)
        fh.writelines(rows)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args == ["--header"]:
        put_header()
        sys.exit(0)
    for deg, solver in zip(args[0::2], args[1::2]):
        line = json.dumps(run(float(deg), solver))
        with open(OUT, "a") as fh:
            fh.write(line + "\n")
        print(line, flush=True)
