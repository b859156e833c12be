"""Per-stage timeline of one 2D complex128 cycle from the device trace.

With tracing on (mg_set_trace), every tile of the persistent fine sweep and
every item of the persistent coarse chain records {taken, dependencies met,
done, SM} in device globaltimer nanoseconds.  This module groups the chain
items into their stages (the sweeps of levels s-1 .. 1, then the correction
stages), mirroring how the library lays the chain out, and prints when each
stage's dependencies were met and when its items finished, relative to the
start of the fine sweep.

    python -m paper_1508_03954_gb300.trace            # the bench workload

Only the layout rules are repeated here; every time comes from the device.
"""
from __future__ import annotations

import math

import numpy as np


def chain_stages(n_fine: int):
    """(name, items) of the chain stages of a 2D cycle whose finest level has
    n_fine cells per axis (the library's tiling rules: 4-cell tiles where a
    level has at least 60 coarse vertices per axis, 1-cell tiles where the
    tiles of one cell still fit one per SM, 2-cell tiles otherwise; the two
    correction stages use chunks of 64..256 vertices, about two per SM)."""
    s = int(round(math.log(n_fine, 3)))
    out = []
    for lev in range(s - 1, 0, -1):
        n = 3 ** lev
        ncv = n // 3 + 1
        tc = 4 if ncv >= 60 else (1 if ncv * ncv <= 152 else 2)
        tiles = (n // 3 + tc) // tc
        out.append((f"sweep level {lev}", tiles * tiles))

    def corr(lev):
        nv = (3 ** lev + 1) ** 2
        chunk = min(256, max(64, (nv // 304 + 63) // 64 * 64))
        return (nv + chunk - 1) // chunk

    top = s - 1
    if top >= 3:
        out.append((f"corr_{top - 1} from levels 1..{top - 1}", corr(top - 1)))
        out.append((f"corr_{top} = t_{top} + P corr_{top - 1}", corr(top)))
    elif top == 2:
        out.append(("corr_2 from levels 1..2", corr(2)))
    return out


def fine_tiles(n_fine: int) -> int:
    tl = (n_fine // 3 + 8) // 8
    return tl * tl


def timeline(solver, variant, omega, transfer, warm=3):
    """Runs warm + 1 traced cycles and returns (fine summary, stage rows)."""
    n = solver.n
    stages = chain_stages(n)
    nchain = sum(k for _, k in stages)
    nfine = fine_tiles(n)
    solver.set_trace(True)
    for _ in range(warm + 1):
        solver.cycle(variant, omega, transfer)
    fine, chain = solver.get_trace(nfine, nchain)
    solver.set_trace(False)
    fine = fine.astype(np.int64)
    chain = chain.astype(np.int64)
    t0 = fine[:, 0].min()
    fsum = {"tiles": nfine, "start": 0.0, "end": (fine[:, 2].max() - t0) / 1e3,
            "last_taken": (fine[:, 0].max() - t0) / 1e3,
            "tile_mean": float(np.mean(fine[:, 2] - fine[:, 0])) / 1e3}
    rows, i = [], 0
    for name, k in stages:
        seg = chain[i:i + k]
        i += k
        rows.append({"stage": name, "items": k,
                     "ready_first": (seg[:, 1].min() - t0) / 1e3, "ready_last": (seg[:, 1].max() - t0) / 1e3,
                     "done_first": (seg[:, 2].min() - t0) / 1e3, "done_last": (seg[:, 2].max() - t0) / 1e3,
                     "work_mean": float(np.mean(seg[:, 2] - seg[:, 1])) / 1e3})
    return fsum, rows


def main():
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1508_03954_gb300 import build as B
    from paper_1508_03954_gb300 import mg
    from paper_1508_03954_gb300 import workloads as W
    B.build()
    mg.load()
    c = W.config2()
    s = mg.Solver(2, c["depth"], c["k2"], c["theta"], c["layer_width"])
    s.set_rhs(c["f"])
    om = np.full(c["depth"], 0.6)
    fsum, rows = timeline(s, mg.MG_BPX, om, mg.MG_HIERARCHICAL)
    print(f"fine sweep: {fsum['tiles']} tiles, 0.0 .. {fsum['end']:.1f} us "
          f"(last tile taken at {fsum['last_taken']:.1f} us, tile mean {fsum['tile_mean']:.1f} us)")
    print("| stage | items | dependencies met (us) | items done (us) | mean item (us) |")
    print("|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['stage']} | {r['items']} | {r['ready_first']:.1f} .. {r['ready_last']:.1f} | "
              f"{r['done_first']:.1f} .. {r['done_last']:.1f} | {r['work_mean']:.2f} |")
    s.close()


if __name__ == "__main__":
    main()
