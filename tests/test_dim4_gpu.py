"""Parity of the four-dimensional path (p = 4 of Section 7.1) with the FP64
oracle, through the C ABI.

complex128 iterates must match the oracle's to 1e-12 relative L2 for every
variant, with and without a scaling layer, a one-sided layer with a rotated
interior, and on depths 1-3 (the oracle is generic in d and pinned in four
dimensions in the CPU suite).  At the full size (depth 4, 82^4 vertices) the
oracle is too slow; there the checks are properties: the analytic discrete
Poisson solution of Section 7.1 has a zero residual, and the cycle (complex128
and the complex64 refinement form) converges to it.
"""
import math

import numpy as np
import pytest

import oracle as O
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


def pair(depth, k2, theta, layer, theta_i, f, u0):
    kf = W.constant_k2(4, depth, k2)
    g = mg.Solver(4, depth, kf, theta, layer, theta_i)
    o = O.Hierarchy(4, depth, kf, theta, layer, theta_i)
    g.set_rhs(f)
    o.set_rhs_nodal(f)
    g.set_solution(u0)
    o.set_solution(u0)
    return g, o


@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx"])
@pytest.mark.parametrize("depth,layer,thi", [(1, 0.2, 0.0), (2, 0.2, 0.0), (2, 0.5, 0.0), (2, (0.0, 1 / 3), 0.3),
                                             (2, 0.0, 0.0)])
def test_cycle_iterates_4d(var, depth, layer, thi):
    f = W.gaussian(4, depth, (0.4, 0.5, 0.6, 0.45), 0.15)
    g, o = pair(depth, 15.0, TH, layer, thi, f, W.random_complex(4, depth, 40 + depth))
    om = np.array([0.6 - 0.02j * l for l in range(depth)])
    for k in range(3):
        g.cycle(var[0], om, var[1])
        o.cycle(om, var[2], var[3])
        e = rel_l2(g.get_solution(), o.u)
        assert e <= TOL, f"cycle {k + 1}: rel L2 {e:.3e}"
    g.close()


def test_cycle_iterates_4d_depth3():
    """28^4 vertices: every pass spans many blocks, two cycles of BPX."""
    depth = 3
    f = W.gaussian(4, depth, (0.5, 0.5, 0.5, 0.5), 0.2)
    g, o = pair(depth, 25.0, TH, 1 / 3, 0.0, f, W.random_complex(4, depth, 7))
    om = np.full(depth, 0.7)
    for k in range(2):
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        o.cycle(om, O.ADD, O.HIERARCHICAL)
        e = rel_l2(g.get_solution(), o.u)
        assert e <= TOL, f"cycle {k + 1}: rel L2 {e:.3e}"
    g.close()


def test_levels_norms_and_rhs_4d():
    """b_L = M f, the restricted right-hand sides, the injected copies, the
    residual norms (Euclidean and max) and the fused cycle norm."""
    depth = 2
    f = W.random_complex(4, depth, 3)
    g, o = pair(depth, 12.0, TH, 0.2, 0.0, f, W.random_complex(4, depth, 4))
    assert rel_l2(g.get_level(depth, 1), o.b) <= 1e-13
    a, r = g.residual_norm()
    oa, _ = o.residual_norm()
    assert abs(a - oa) <= 1e-12 * oa and r == 1.0
    assert abs(g.residual_max() - o.residual_max()) <= 1e-12 * o.residual_max()
    u0 = g.get_solution()
    tr = {}
    om = np.full(depth, 0.6)
    g.cycle(mg.MG_ADD, om, mg.MG_DLINEAR)
    o.cycle(om, O.ADD, O.DLINEAR, trace=tr)
    a_cycle, _ = g.last_cycle_norm()
    assert abs(a_cycle - oa) <= 1e-12 * oa  # residual of the iterate entering the cycle
    assert rel_l2(g.get_level(1, 1), tr["b"][1]) <= 1e-12
    np.testing.assert_array_equal(g.get_level(1, 0), O.inject(u0))
    a, _ = g.residual_norm()
    oa, _ = o.residual_norm()
    assert abs(a - oa) <= 1e-12 * oa
    g.close()


def test_solve_4d_reports_status():
    """A definite problem converges under mg_solve; the indefinite one with
    undamped unit factors diverges and is reported, not raised."""
    depth = 2
    f = W.gaussian(4, depth, (0.5, 0.5, 0.5, 0.5), 0.2)
    g = mg.Solver(4, depth, W.constant_k2(4, depth, -40.0), 0.0, 0.0)
    g.set_rhs(f)
    st, n, rel = g.solve(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_EXP, 0.8, depth), mg.MG_DLINEAR, 1e-9, 500)
    assert st == mg.MG_OK and rel <= 1e-9
    o = O.Hierarchy(4, depth, W.constant_k2(4, depth, -40.0), 0.0, 0.0)
    o.set_rhs_nodal(f)
    r = o.residual(g.get_solution())
    assert np.linalg.norm(r) <= 1.01e-9 * np.linalg.norm(o.b)
    g.close()
    g = mg.Solver(4, depth, W.constant_k2(4, depth, 400.0), 0.0, 0.0)
    g.set_rhs(f)
    st, n, rel = g.solve(mg.MG_ADD, np.full(depth, 1.0), mg.MG_DLINEAR, 1e-9, 500)
    assert st == mg.MG_DIVERGED
    g.close()


def test_poisson_4d_full_size():
    """Depth 4 (82^4 = 45 M vertices): the discrete solution
    pi^2 (mu/kappa) prod sin(pi x_i) of rhs 4 pi^2 prod sin(pi x_i) (Section
    7.1) has a residual at rounding level, and the cycle (exponential damping,
    omega = 0.8) converges to it."""
    depth, d = 4, 4
    n = 3 ** depth
    h = 1.0 / n
    s1 = np.sin(math.pi * np.arange(n + 1) / n)
    s = s1[:, None, None, None] * s1[None, :, None, None] * s1[None, None, :, None] * s1[None, None, None, :]
    kap = (2 / h) * (1 - math.cos(math.pi * h))
    mu = (h / 3) * (2 + math.cos(math.pi * h))
    exact = (math.pi ** 2 * (mu / kap) * s).astype(np.complex128)
    g = mg.Solver(d, depth, W.constant_k2(d, depth, 0.0), 0.0, 0.0)
    g.set_rhs((d * math.pi ** 2 * s).astype(np.complex128))
    b_norm, _ = g.residual_norm()  # u = 0
    g.set_solution(exact)
    r_exact, _ = g.residual_norm()
    # rounding level: 81 terms per row, each about h^2 |u| while the row sums
    # to about 4 pi^2 h^4 |u|, so 81 x 2^-53 x 1/(4 pi^2 h^2) ~ 1.5e-12
    assert r_exact <= 2e-12 * b_norm
    g.set_solution(np.zeros_like(exact))
    g.residual_norm()
    om = mg.omega_scheme(mg.MG_OMEGA_EXP, 0.8, depth)
    st, cycles, rel = g.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 400)
    assert st == mg.MG_OK, (st, cycles, rel)
    err = np.abs(g.get_solution() - exact).max() / np.abs(exact).max()
    assert err <= 1e-6, err
    g.close()


@pytest.mark.parametrize("depth,m,var", [(2, 3, VARIANTS[0]), (2, 3, VARIANTS[1]), (2, 3, VARIANTS[2]),
                                         (3, 1, VARIANTS[2])])
def test_c64_outer_step_4d(depth, m, var):
    """One outer step of the refinement form in four dimensions: the complex64
    correction e of m inner cycles on H e = r0 against the oracle's m FP64
    cycles on the same inner problem, to the complex64 bound of the 2D/3D
    test (2e-5 up to depth 4)."""
    kf = W.constant_k2(4, depth, 18.0)
    f = W.random_complex(4, depth, 100)
    u0 = W.random_complex(4, depth, 200)
    g = mg.Solver(4, depth, kf, TH, 0.2)
    o = O.Hierarchy(4, depth, kf, TH, 0.2)
    g.set_rhs(f)
    o.set_rhs_nodal(f)
    g.set_solution(u0)
    o.set_solution(u0)
    omega = np.array([0.6 - 0.03j * l for l in range(depth)])
    g.set_precision(mg.MG_C64_REFINE, m)
    st, n, _ = g.solve(var[0], omega, var[1], 1e-30, m)
    assert st == mg.MG_NOT_CONVERGED and n == m
    oi = O.Hierarchy(4, depth, kf, TH, 0.2)
    oi.b = o.residual()
    O.zero_boundary(oi.b)
    for _ in range(m):
        oi.cycle(omega, var[2], var[3])
    err = rel_l2(g.get_solution() - o.u, oi.u)
    assert err <= 2e-5, f"relative L2 of e: {err:.3e}"
    g.close()


def test_c64_refinement_4d_full_size():
    """Depth 4: the refinement form reaches 1e-8 (FP64 residual, checked
    again by mg_residual_norm) on the Section 7.1 Poisson problem and lands on
    the discrete solution."""
    depth, d = 4, 4
    n = 3 ** depth
    h = 1.0 / n
    s1 = np.sin(math.pi * np.arange(n + 1) / n)
    s = s1[:, None, None, None] * s1[None, :, None, None] * s1[None, None, :, None] * s1[None, None, None, :]
    kap = (2 / h) * (1 - math.cos(math.pi * h))
    mu = (h / 3) * (2 + math.cos(math.pi * h))
    exact = math.pi ** 2 * (mu / kap) * s
    g = mg.Solver(d, depth, W.constant_k2(d, depth, 0.0), 0.0, 0.0)
    g.set_rhs((d * math.pi ** 2 * s).astype(np.complex128))
    g.set_precision(mg.MG_C64_REFINE, 16)
    st, cycles, rel = g.solve(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_EXP, 0.8, depth), mg.MG_DLINEAR, 1e-8, 1000)
    assert st == mg.MG_OK and rel <= 1e-8, (st, cycles, rel)
    _, rel2 = g.residual_norm()
    assert abs(rel2 - rel) <= 1e-6 * rel
    err = np.abs(g.get_solution() - exact).max() / np.abs(exact).max()
    assert err <= 1e-6, err
    g.close()


def test_4d_rejects_what_it_does_not_run():
    k2 = W.constant_k2(4, 1, 1.0)
    k2v = k2.copy()
    k2v[1, 1, 1, 1] = 2.0
    with pytest.raises(mg.MgError):
        mg.Solver(4, 1, k2v, 0.0, 0.0)  # varying shift
    g = mg.Solver(4, 1, k2, 0.0, 0.0)
    with pytest.raises(mg.MgError):
        g.fmg(mg.MG_BPX, np.full(1, 0.6), mg.MG_HIERARCHICAL, 3)
    g.close()
