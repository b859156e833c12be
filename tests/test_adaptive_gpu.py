"""Parity of the adaptive-grid path (mg_create_adaptive) with the adaptive
oracle (oracle/adaptive.py, pinned in tests/test_oracle_adaptive.py to the
regular oracle and to the conforming finite-element solution): every
level's values and the fine-grid function after each cycle to 1e-12, the
residual norms, a converged solve, and full refinement against the regular
library path."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle.adaptive import AdaptiveHierarchy
from paper_1508_03954_gb300 import build as B
from paper_1508_03954_gb300 import mg
from paper_1508_03954_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
TH = math.pi / 6
VARIANTS = [
    (mg.MG_ADD, mg.MG_DLINEAR, O.ADD, O.DLINEAR),
    (mg.MG_HB, mg.MG_DLINEAR, O.HB, O.DLINEAR),
    (mg.MG_BPX, mg.MG_HIERARCHICAL, O.ADD, O.HIERARCHICAL),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    mg.load()


def rel_l2(a, b):
    den = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (den if den > 0 else 1.0)


def corner_refinement(d, depth):
    """Refines the level-1 cells touching the origin except the far corner
    (an L in 2D), then on every level the children nearest the origin plus a
    short strip -- hanging vertices on every level, re-entrant corners."""
    ref = {}
    r1 = np.zeros((3,) * d, dtype=bool)
    r1[(0,) * d] = True
    for ax in range(d):
        idx = [0] * d
        idx[ax] = 1
        r1[tuple(idx)] = True
    ref[1] = r1
    for lev in range(2, depth):
        n = 3 ** lev
        r = np.zeros((n,) * d, dtype=bool)
        r[(slice(0, n // 3),) * d] = True
        strip = [slice(0, n // 9 + 1)] * d
        strip[-1] = slice(n // 3, n // 3 + 2)
        r[tuple(strip)] = True
        ref[lev] = r
    return ref


def pair(d, depth, k2, theta, w, refine, f, u0):
    g = mg.Solver.adaptive(d, depth, k2, theta, w, refine)
    o = AdaptiveHierarchy(d, depth, k2, theta, w, refine)
    g.set_rhs(f)
    o.set_rhs_nodal(f)
    g.set_solution(u0)
    u0z = np.array(u0, dtype=np.complex128)
    O.zero_boundary(u0z)
    lv = {depth: u0z}
    for lev in range(depth - 1, 0, -1):
        lv[lev] = O.inject(lv[lev + 1])
    o.set_solution_levels(lv)
    return g, o


def check_state(g, o, depth, what):
    """Every level's values at the vertices of its existing cells (values
    elsewhere are never read), and the fine-grid function."""
    for lev in range(1, depth + 1):
        m = o.exists[lev]
        e = rel_l2(g.get_level(lev, 0)[m], o.u[lev][m])
        assert e <= TOL, f"{what}: level {lev} rel L2 {e:.3e}"
    e = rel_l2(g.get_solution(), o.composite_on_fine())
    assert e <= TOL, f"{what}: fine-grid function rel L2 {e:.3e}"


@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx"])
@pytest.mark.parametrize("depth,w", [(3, 0.2), (4, 0.2), (3, 0.5)])
def test_adaptive_iterates_2d(var, depth, w):
    d = 2
    k2 = W.constant_k2(d, depth, 30.0)
    g, o = pair(d, depth, k2, TH, w, corner_refinement(d, depth), W.random_complex(d, depth, 3),
                W.random_complex(d, depth, 4))
    check_state(g, o, depth, "start")
    om = np.array([0.6 - 0.02j * l for l in range(depth)])
    for k in range(3):
        g.cycle(var[0], om, var[1])
        o.cycle(om, var[2], var[3])
        check_state(g, o, depth, f"cycle {k + 1}")
    a, _ = g.residual_norm()
    b, _ = o.residual_norm()
    assert abs(a - b) <= 1e-12 * b
    g.close()


def test_adaptive_varying_shift_and_3d():
    """A per-cell shift (mean of vertex k^2) in 2D, and a 3D corner refinement."""
    rng = np.random.default_rng(9)
    for d, depth in [(2, 3), (3, 2)]:
        n = 3 ** depth
        k2 = rng.uniform(-20.0, 60.0, size=(n + 1,) * d) if d == 2 else W.constant_k2(d, depth, 25.0)
        g, o = pair(d, depth, k2, TH, 0.2, corner_refinement(d, depth), W.random_complex(d, depth, 5),
                    W.random_complex(d, depth, 6))
        om = np.full(depth, 0.55)
        for k in range(2):
            g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
            o.cycle(om, O.ADD, O.HIERARCHICAL)
            check_state(g, o, depth, f"d={d} cycle {k + 1}")
        g.close()


def test_full_refinement_matches_the_regular_library_path():
    """Every cell refined: the adaptive path and the regular cycle agree
    (uniform scaling, constant shift: Lemma 2)."""
    d, depth = 2, 4
    k2 = W.constant_k2(d, depth, 40.0)
    ref = {lev: np.ones((3 ** lev,) * d, dtype=bool) for lev in range(1, depth)}
    f, u0 = W.random_complex(d, depth, 7), W.random_complex(d, depth, 8)
    g = mg.Solver.adaptive(d, depth, k2, TH, 0.5, ref)
    r = mg.Solver(d, depth, k2, TH, 0.5)
    for s in (g, r):
        s.set_rhs(f)
        s.set_solution(u0)
    om = np.array([0.5, 0.55, 0.6, 0.65])
    for _ in range(3):
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        r.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
    assert rel_l2(g.get_solution(), r.get_solution()) <= TOL
    g.close()
    r.close()


def test_adaptive_solve_reaches_the_oracle_fixed_point():
    """A definite problem on the corner refinement: mg_solve converges to
    1e-10 and lands on the oracle's fixed point (the conforming finite-element
    solution of the adaptive mesh)."""
    d, depth, k2v = 2, 3, -20.0
    n = 3 ** depth
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)
    f = (1.0 + X + 2.0 * Y + 3.0 * X * Y).astype(np.complex128)
    k2 = W.constant_k2(d, depth, k2v)
    ref = corner_refinement(d, depth)
    g = mg.Solver.adaptive(d, depth, k2, 0.0, 0.0, ref)
    g.set_rhs(f)
    om = mg.omega_scheme(mg.MG_OMEGA_UCG, 0.6, depth)
    st, cycles, rel = g.solve(mg.MG_BPX, om, mg.MG_HIERARCHICAL, 1e-10, 1000)
    assert st == mg.MG_OK and rel <= 1e-10, (st, cycles, rel)
    o = AdaptiveHierarchy(d, depth, k2, 0.0, 0.0, ref)
    o.set_rhs_nodal(f)
    for _ in range(cycles + 50):
        o.cycle(om, O.ADD, O.HIERARCHICAL)
    assert rel_l2(g.get_solution(), o.composite_on_fine()) <= 1e-9
    g.close()


def test_adaptive_rejects_what_it_does_not_run():
    d, depth = 2, 2
    k2 = W.constant_k2(d, depth, 1.0)
    ref = {1: np.ones((3, 3), dtype=bool)}
    g = mg.Solver.adaptive(d, depth, k2, 0.0, 0.0, ref)
    with pytest.raises(mg.MgError):
        g.set_precision(mg.MG_C64_REFINE, 4)
    with pytest.raises(mg.MgError):
        g.fmg(mg.MG_BPX, np.full(depth, 0.6), mg.MG_HIERARCHICAL, 3)
    g.close()
    with pytest.raises(mg.MgError):
        mg.Solver.adaptive(4, 1, W.constant_k2(4, 1, 1.0), 0.0, 0.0, {})


def test_residual_max_matches_the_oracle():
    d, depth = 2, 4
    k2 = W.constant_k2(d, depth, 30.0)
    g, o = pair(d, depth, k2, TH, 0.2, corner_refinement(d, depth), W.random_complex(d, depth, 21),
                W.random_complex(d, depth, 22))
    om = np.full(depth, 0.6)
    for _ in range(2):
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        o.cycle(om, O.ADD, O.HIERARCHICAL)
    a, b = g.residual_max(), o.residual_max()
    assert abs(a - b) <= 1e-12 * b
    g.close()


def decision_margins(o, bins, veto, relative=False):
    """How far the oracle's state is from flipping a decision: the distance
    of every fine-grid vertex's scaled indicator to the interior bin edges,
    and of |r / diag| to the veto (relative).  The parity of the flags
    below needs both well above the rounding difference of the two sides."""
    s = o.refinement_indicator()
    r = o.level_residuals()
    vals = np.concatenate([s[lev][o.fine_grid(lev)] for lev in range(1, o.L + 1)])
    lo, hi = vals.min(), vals.max()
    mb = mv = np.inf
    for lev in range(1, o.L + 1):
        f = o.fine_grid(lev)
        q = ((s[lev][f] - lo) / (hi - lo)) * bins
        mb = min(mb, np.abs(q - np.clip(np.round(q), 1, bins - 1)).min(initial=np.inf))
        ratio = np.abs(r[lev][f] / o.levels[lev].diag[f])
        bound = veto * np.abs(o.u[lev][f]) if relative else veto
        mv = min(mv, (np.abs(ratio - bound) / bound).min(initial=np.inf))
    return mb, mv


def check_flags_and_state(g, o, depth, what):
    got = g.refinement()
    for lev in range(1, depth):
        np.testing.assert_array_equal(got[lev], o.refined[lev], err_msg=f"{what}: refine flags of level {lev}")
    check_state(g, o, depth, what)


@pytest.mark.parametrize("d,depth,steps,relative,veto", [(2, 5, 6, False, 1e-2), (3, 3, 3, False, 1e-2),
                                                         (2, 5, 6, True, 0.3)])
def test_dynamic_refinement_matches_the_oracle(d, depth, steps, relative, veto):
    """Feature-based refinement (Section 5.3) from the regular level-2 grid:
    cycle, then mg_adapt, repeatedly (erasing a large fraction every other
    step).  Every step selects the same vertices, yields the same refine
    flags and fine-grid vertex count, and the values of every level and the
    fine-grid function match the oracle to 1e-12."""
    k2 = W.constant_k2(d, depth, 25.0)
    ref = {1: np.ones((3,) * d, dtype=bool)}
    for lev in range(2, depth):
        ref[lev] = np.zeros((3 ** lev,) * d, dtype=bool)
    f = W.gaussian(d, depth, (0.3, 0.6, 0.45)[:d], 0.05)
    g, o = pair(d, depth, k2, TH, 0.2, ref, f, np.zeros((3 ** depth + 1,) * d, complex))
    om = np.full(depth, 0.6)
    erased = 0
    for k in range(steps):
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        o.cycle(om, O.ADD, O.HIERARCHICAL)
        mb, mv = decision_margins(o, 20, veto, relative)
        assert mb > 1e-9 and mv > 1e-9, (mb, mv)
        ef = 0.3 if k % 2 else 0.02
        st = g.adapt(2, 0.1, ef, 20, veto, veto_relative=relative)
        ost = o.adapt(2, 0.1, ef, 20, veto, veto_relative=relative)
        assert st[:3] == ost, (k, st, ost)
        assert st[3] == max(lev for lev in range(1, depth + 1) if o.cells[lev].any())
        erased += st[1]
        check_flags_and_state(g, o, depth, f"step {k + 1}")
    assert erased > 0
    # cycles on the final grid still agree
    for k in range(2):
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        o.cycle(om, O.ADD, O.HIERARCHICAL)
    check_state(g, o, depth, "after the last step")
    a, b = g.residual_max(), o.residual_max()
    assert abs(a - b) <= 1e-12 * b
    g.close()


def test_adapt_arguments_and_refinement_roundtrip():
    d, depth = 2, 3
    k2 = W.constant_k2(d, depth, 1.0)
    ref = corner_refinement(d, depth)
    g = mg.Solver.adaptive(d, depth, k2, 0.0, 0.0, ref)
    o = AdaptiveHierarchy(d, depth, k2, 0.0, 0.0, ref)
    got = g.refinement()
    for lev in range(1, depth):
        np.testing.assert_array_equal(got[lev], o.refined[lev])
    for bad in [dict(min_level=0), dict(min_level=2, bins=0), dict(min_level=2, bins=65),
                dict(min_level=2, refine_frac=1.5), dict(min_level=2, veto=0.0)]:
        with pytest.raises(mg.MgError):
            g.adapt(**bad)
    g.close()
    r = mg.Solver(d, depth, k2, 0.0, 0.0)
    with pytest.raises(mg.MgError):
        r.adapt(1)
    r.close()


GOLDEN_T2A = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2_adaptive_oracle.txt")


def test_table2_adaptive_runs_match_the_stored_oracle_runs():
    """The dynamic path at the size the bench measures (depth 7: 50 cycles and
    50 refinement steps per run, the schedule of forms.channel_table2_adaptive):
    every stored oracle run (tests/golden/table2_adaptive_oracle.txt, written
    by make_table2_adaptive.py) ends on the same grid and with the same
    max-norm reduction."""
    rows = [json.loads(ln) for ln in open(GOLDEN_T2A) if ln.strip() and not ln.startswith("#")]
    assert rows
    depth, min_level = 7, 3
    for row in rows:
        deg, solver = row["theta_deg"], row["solver"]
        c = W.channel(deg, depth)
        ref = {lev: np.full((3 ** lev,) * 2, lev < min_level) for lev in range(1, depth)}
        s = mg.Solver.adaptive(2, depth, c["k2"], c["theta"], c["layer_width"], ref, c["theta_interior"])
        s.set_rhs(c["f"])
        s.set_solution(np.zeros(s.shape, complex))
        r0 = s.residual_max()
        st = None
        for it in range(1, 51):
            if solver == "jacobi":
                w = (W.CHANNEL_OMEGA1 if it % 2 else W.CHANNEL_OMEGA2) if deg == 0 else 0.4
                s.cycle(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_JACOBI, w, depth), mg.MG_DLINEAR)
            elif solver == "transition":
                s.cycle(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_TRANSITION, 0.4, depth, it), mg.MG_DLINEAR)
            else:
                s.cycle(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_UCG, 0.4, depth), mg.MG_HIERARCHICAL)
            st = s.adapt(min_level, 0.1, 0.02, 20, 1e-2)
        red = s.residual_max() / r0
        s.close()
        assert st[2] == row["fine_vertices"], (deg, solver, st, row)
        assert abs(red - row["reduction_max_norm"]) <= 1e-10 * abs(row["reduction_max_norm"]), (deg, solver, red)
