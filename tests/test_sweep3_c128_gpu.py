"""Parity of the separable complex128 3D sweep (finest levels with 27 or more
cells per axis, coarse levels with 81 or more) with the FP64 oracle, through
the C ABI.

Per-iterate relative L2 against the oracle within 1e-12 (the complex128
contract) over several cycles, every variant and transfer, at depths 3 and 4
(the finest level runs the separable kernel: one tile of 9 coarse cells at
depth 3, three per axis at depth 4, the last one owning the boundary coarse
column), with layers that make some, none or all axis rows complex, real
and complex relaxation factors.  At the full 3D size (depth 5, 14.5 M
vertices; level 4 runs the separable kernel as a coarse level) the oracle's
two iterates of every variant are stored at 512 seeded sample vertices
(written by tests/golden/make_config3_samples.py, which calls only the
oracle).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1508_03954_gb300 import build as B
from paper_1508_03954_gb300 import mg
from paper_1508_03954_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
TH = math.pi / 6
VARIANTS = [  # (library variant, library transfer, oracle variant, oracle transfer)
    (mg.MG_ADD, mg.MG_DLINEAR, O.ADD, O.DLINEAR),
    (mg.MG_HB, mg.MG_DLINEAR, O.HB, O.DLINEAR),
    (mg.MG_BPX, mg.MG_HIERARCHICAL, O.ADD, O.HIERARCHICAL),
    (mg.MG_HB, mg.MG_HIERARCHICAL, O.HB, O.HIERARCHICAL),
]
IDS = ["add", "hb", "bpx", "hb-hier"]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_oracle_samples.txt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    mg.load()


def rel_l2(a, b):
    den = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (den if den > 0 else 1.0)


def run(depth, w, k2, var, omega, cycles, seed):
    f = W.random_complex(3, depth, seed)
    u0 = W.random_complex(3, depth, seed + 1)
    g = mg.Solver(3, depth, W.constant_k2(3, depth, k2), TH, w)
    o = O.Hierarchy(3, depth, W.constant_k2(3, depth, k2), TH, w)
    g.set_rhs(f)
    o.set_rhs_nodal(f)
    g.set_solution(u0)
    o.set_solution(u0)
    worst = 0.0
    for n in range(cycles):
        g.cycle(var[0], omega, var[1])
        o.cycle(omega, var[2], var[3])
        e = rel_l2(g.get_solution(), o.u)
        worst = max(worst, e)
        assert e <= TOL, f"iterate {n + 1}: rel L2 {e:.3e}"
        # the fused norm of the iterate that entered this cycle
    a_g, _ = g.residual_norm()
    a_o, _ = o.residual_norm()
    assert abs(a_g - a_o) <= 1e-12 * a_o
    g.close()
    return worst


@pytest.mark.parametrize("var", VARIANTS, ids=IDS)
@pytest.mark.parametrize("w", [0.1, 0.5, 0.0], ids=["layer", "all-scaled", "no-layer"])
def test_depth3_iterates(var, w):
    run(3, w, -30.0 if w == 0.0 else 40.0, var, np.array([0.5, 0.6 + 0.05j, 0.7]), 4, 100)


@pytest.mark.parametrize("var", VARIANTS, ids=IDS)
@pytest.mark.parametrize("omega", [np.array([0.55, 0.6, 0.6, 0.65]),
                                   np.array([0.5 - 0.02j, 0.6, 0.6 + 0.03j, 0.65 - 0.01j])], ids=["real", "complex"])
def test_depth4_iterates(var, omega):
    run(4, 0.1, 25.0, var, omega, 2, 200)


def _golden_blocks():
    blocks, cur = {}, None
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("# {"):
                cur = json.loads(line[2:])
                cur["rows"] = []
                blocks[cur["variant"]] = cur
            elif not line.startswith("#") and line.strip():
                cur["rows"].append([float(x) for x in line.split()])
    return blocks


@pytest.mark.parametrize("var", VARIANTS, ids=IDS)
def test_config3_full_size_iterates_match_stored_oracle_samples(var):
    """Full-size 3D workload (the finest level and level 4 run the separable
    kernel): two cycles from the stored seeded start; the iterates at the
    oracle's sample vertices and the residual norms."""
    head = _golden_blocks()[IDS[VARIANTS.index(var)]]
    rows = np.array(head["rows"])
    flat = rows[:, 0].astype(np.int64)
    u1 = rows[:, 1] + 1j * rows[:, 2]
    u2 = rows[:, 3] + 1j * rows[:, 4]
    c = W.config3(head["depth"])
    g = mg.Solver(3, head["depth"], c["k2"], c["theta"], c["layer_width"])
    g.set_rhs(c["f"])
    g.set_solution(W.random_complex(3, head["depth"], 7) * 1e-3)
    a0, _ = g.residual_norm()
    norms = head["residual_norms"]
    assert abs(a0 - norms[0]) <= 1e-12 * norms[0]
    om = np.full(head["depth"], head["omega"])
    for k, ref in enumerate((u1, u2)):
        g.cycle(var[0], om, var[1])
        u = np.ravel(g.get_solution())[flat]
        assert rel_l2(u, ref) <= TOL, (k, rel_l2(u, ref))
        a, _ = g.residual_norm()
        assert abs(a - norms[k + 1]) <= 1e-12 * norms[k + 1], (k, a, norms[k + 1])
    g.close()


def test_largest_3d_grid_keeps_the_symmetries_of_a_symmetric_problem():
    """3D depth 6 (729^3 cells, 389 M vertices, 6.2 GB per complex128 array;
    the largest 3D grid here, beyond any oracle run): constant k^2, a layer on
    every face, a centred Gaussian and a zero start are invariant under the 48
    symmetries of the cube, so after two BPX cycles the iterate must be too,
    to rounding -- the separable sweep's tiles, ranges and halo indexing treat
    x, y and z differently, and a transposed or shifted index breaks this.
    The fused residual norm of the cycle also equals the standalone one."""
    depth = 6
    n = 3 ** depth
    k2 = W.constant_k2(3, depth, 40.0)
    f = W.gaussian(3, depth, (0.5, 0.5, 0.5), 0.05).astype(np.complex128)
    g = mg.Solver(3, depth, k2, TH, 0.1)
    g.set_rhs(f)
    om = np.full(depth, 0.6)
    g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
    a_ref, _ = g.residual_norm()
    g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
    a_fused, _ = g.last_cycle_norm()
    assert abs(a_fused - a_ref) <= 1e-12 * a_ref, (a_fused, a_ref)
    u = g.get_solution()
    g.close()
    scale = np.abs(u).max()
    assert scale > 0
    for t in [u.transpose(1, 0, 2), u.transpose(2, 1, 0), u.transpose(0, 2, 1), u[::-1, :, :], u[:, ::-1, :],
              u[:, :, ::-1], u.transpose(1, 2, 0)[::-1, :, ::-1]]:
        assert np.abs(t - u).max() <= 1e-12 * scale
    assert u.shape == (n + 1,) * 3


@pytest.mark.parametrize("var", [VARIANTS[0], VARIANTS[2]], ids=["add", "bpx"])
def test_fmg_start_in_3d_matches_oracle(var):
    """FMG grid unfolding in 3D (depth 4): the stages up to level 3 run the
    separable sweep as their finest level (with BPX: du and I du stored, P I du
    taken through the pending correction), so the interpolated start checks
    that the pending correction is complete at every stage."""
    depth = 4
    k2 = W.constant_k2(3, depth, 30.0)
    f = W.random_complex(3, depth, 41)
    g = mg.Solver(3, depth, k2, TH, 0.1)
    g.set_rhs(f)
    om = np.array([0.6, 0.55, 0.6, 0.65])
    g.fmg(var[0], om, var[1], 3)
    ho = O.fmg_start(3, depth, k2, TH, 0.1, f, om, var[2], var[3], 3)
    assert rel_l2(g.get_solution(), ho.u) <= TOL
    g.close()
