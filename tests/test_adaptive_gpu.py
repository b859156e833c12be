"""Parity of the adaptive-grid path (mg_create_adaptive) with the adaptive
oracle (oracle/adaptive.py, pinned in tests/test_oracle_adaptive.py to the
regular oracle and to the conforming finite-element solution): every
level's values and the fine-grid function after each cycle to 1e-12, the
residual norms, a converged solve, and full refinement against the regular
library path."""
import math

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
        g.residual_max()
    g.close()
    with pytest.raises(mg.MgError):
        mg.Solver.adaptive(4, 1, W.constant_k2(4, 1, 1.0), 0.0, 0.0, {})
