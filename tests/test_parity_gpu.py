"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

complex128 cycles must match the oracle's per-cycle iterates to 1e-12
relative L2 (the target the solver is specified against); the complex64
refinement form must reach its FP64 residual tolerance as checked by the
oracle's own residual.  Inputs are seeded and shared; nothing expected comes
from the CUDA path.
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
VARIANTS = [  # (library variant, library transfer, oracle variant, oracle transfer)
    (mg.MG_ADD, mg.MG_DLINEAR, O.ADD, O.DLINEAR),
    (mg.MG_HB, mg.MG_DLINEAR, O.HB, O.DLINEAR),
    (mg.MG_BPX, mg.MG_HIERARCHICAL, O.ADD, O.HIERARCHICAL),
    (mg.MG_HB, mg.MG_HIERARCHICAL, O.HB, O.HIERARCHICAL),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    mg.load()


def rel_l2(a, b):
    den = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (den if den > 0 else 1.0)


def pair(d, depth, k2, theta, w, f, u0=None):
    g = mg.Solver(d, depth, k2, theta, w)
    o = O.Hierarchy(d, depth, k2, theta, w)
    g.set_rhs(f)
    o.set_rhs_nodal(f)
    if u0 is not None:
        g.set_solution(u0)
        o.set_solution(u0)
    return g, o


def run_iterates(g, o, var, omega, ncyc, tol=TOL):
    worst = 0.0
    for n in range(ncyc):
        g.cycle(var[0], omega, var[1])
        o.cycle(omega, var[2], var[3])
        e = rel_l2(g.get_solution(), o.u)
        worst = max(worst, e)
        assert e <= tol, f"iterate {n + 1}: rel L2 {e:.3e}"
    return worst


# ------------------------------------------------------------------ cycles
@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx", "hb-hier"])
@pytest.mark.parametrize("depth,w", [(1, 0.1), (2, 4 / 27), (3, 4 / 27), (4, 0.1), (4, 0.5), (3, 0.0)])
def test_cycle_iterates_2d(var, depth, w):
    k2 = W.constant_k2(2, depth, 30.0 + 5 * depth)
    f = W.random_complex(2, depth, 10 + depth)
    u0 = W.random_complex(2, depth, 20 + depth)
    g, o = pair(2, depth, k2, TH, w, f, u0)
    omega = np.array([0.6 + 0.05j * l for l in range(depth)])
    run_iterates(g, o, var, omega, 4)


@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx", "hb-hier"])
@pytest.mark.parametrize("depth,w", [(1, 0.2), (2, 0.1), (3, 0.1)])
def test_cycle_iterates_3d(var, depth, w):
    k2 = W.constant_k2(3, depth, 20.0)
    f = W.random_complex(3, depth, 30 + depth)
    u0 = W.random_complex(3, depth, 40 + depth)
    g, o = pair(3, depth, k2, TH, w, f, u0)
    omega = np.array([0.5, 0.55, 0.6][:depth])
    run_iterates(g, o, var, omega, 3)


@pytest.mark.parametrize("d,depth", [(2, 3), (2, 4), (3, 2)])
def test_cycle_iterates_varying_shift(d, depth):
    """Per-cell shift (mean of vertex k^2), as in k^2 = E - V(x)."""
    rng = np.random.default_rng(5)
    k2 = rng.uniform(-50.0, 400.0, size=(3 ** depth + 1,) * d)
    f = W.random_complex(d, depth, 50)
    g, o = pair(d, depth, k2, TH, 0.1, f)
    omega = np.full(depth, 0.6)
    for var in VARIANTS[::2]:
        run_iterates(g, o, var, omega, 3)


def test_config1_thirty_cycles():
    """2D depth 3, k = 4 pi, 4-cell layer, additive MG omega = 0.6, 30
    cycles: the configured problem (it diverges slowly; parity holds per
    iterate)."""
    c = W.config1()
    g, o = pair(c["d"], c["depth"], c["k2"], c["theta"], c["layer_width"], c["f"])
    omega = np.full(3, c["omega_s"])
    run_iterates(g, o, VARIANTS[0], omega, c["cycles"])
    _, rel = g.residual_norm()
    _, orel = o.residual_norm()
    assert abs(rel - orel) <= 1e-10 * orel


def test_config2_full_size_iterates():
    """Depth 6 (729^2 cells), the launch configuration the benchmark times."""
    c = W.config2()
    g, o = pair(c["d"], c["depth"], c["k2"], c["theta"], c["layer_width"], c["f"])
    omega = np.full(6, 0.6)
    run_iterates(g, o, VARIANTS[2], omega, 2)
    run_iterates(g, o, VARIANTS[0], omega, 1)


# ------------------------------------------------------------------ pieces
@pytest.mark.parametrize("d,depth", [(2, 4), (3, 3), (3, 4)])
def test_rhs_and_restricted_rhs_and_injection(d, depth):
    # 3D: b_L = M f by separable mass passes; b_l of the coarse levels from the
    # level sweeps and from the point kernels' restriction of the stored residual
    k2 = W.constant_k2(d, depth, 50.0)
    f = W.random_complex(d, depth, 3)
    u0 = W.random_complex(d, depth, 4)
    g, o = pair(d, depth, k2, TH, 0.1, f, u0)
    assert rel_l2(g.get_level(depth, 1), o.b) <= 1e-13
    tr = {}
    g.cycle(mg.MG_ADD, np.full(depth, 0.6), mg.MG_DLINEAR)
    o.cycle(np.full(depth, 0.6), O.ADD, O.DLINEAR, trace=tr)
    for lev in range(1, depth):
        assert rel_l2(g.get_level(lev, 1), tr["b"][lev]) <= 1e-12, lev
        # Lemma 1: the coarse copy is the injection of the iterate entering the cycle
        inj = u0.copy()
        O.zero_boundary(inj)
        for _ in range(depth - lev):
            inj = O.inject(inj)
        np.testing.assert_array_equal(g.get_level(lev, 0), inj)


def test_residual_norm():
    depth = 4
    k2 = W.constant_k2(2, depth, 70.0)
    g, o = pair(2, depth, k2, TH, 0.1, W.random_complex(2, depth, 8), W.random_complex(2, depth, 9))
    a, r = g.residual_norm()
    oa, orl = o.residual_norm()
    assert abs(a - oa) <= 1e-12 * oa and r == 1.0
    g.cycle(mg.MG_BPX, np.full(depth, 0.6), mg.MG_HIERARCHICAL)
    o.cycle(np.full(depth, 0.6), O.ADD, O.HIERARCHICAL)
    a, r = g.residual_norm()
    oa, orl = o.residual_norm()
    assert abs(r - orl) <= 1e-11 * orl


def test_fmg_start_matches_oracle():
    c = W.config2(depth=4)
    g, _ = pair(c["d"], c["depth"], c["k2"], c["theta"], c["layer_width"], c["f"])
    om = np.full(4, 0.6)
    g.fmg(mg.MG_BPX, om, mg.MG_HIERARCHICAL, 3)
    ho = O.fmg_start(2, 4, c["k2"], c["theta"], c["layer_width"], c["f"], om, O.ADD,
                     O.HIERARCHICAL, 3)
    assert rel_l2(g.get_solution(), ho.u) <= TOL


# ------------------------------------------------------------------ solves
def test_solve_converges_galerkin_and_matches_dense():
    """Aligned layer (w = 1/3) with a definite shift: Galerkin on every level,
    the cycle converges to the discrete solution (dense direct solve)."""
    depth = 3
    k2 = W.constant_k2(2, depth, -200.0)
    f = W.gaussian(2, depth, (0.5, 0.5), 0.1).astype(complex)
    g, o = pair(2, depth, k2, TH, 1 / 3, f)
    st, ncyc, rel = g.solve(mg.MG_BPX, np.full(depth, 0.6), mg.MG_HIERARCHICAL, 1e-10, 400)
    assert st == mg.MG_OK and rel <= 1e-10
    ost, oc, orel = o.solve(np.full(depth, 0.6), O.ADD, O.HIERARCHICAL, tol=1e-10, max_cycles=400)
    assert ost == 0 and abs(ncyc - oc) <= 8
    u = g.get_solution()
    r = o.residual(u)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(o.b)


def test_solve_reports_divergence():
    c = W.config1()
    g, o = pair(c["d"], c["depth"], c["k2"], c["theta"], c["layer_width"], c["f"])
    st, n, rel = g.solve(mg.MG_ADD, np.full(3, 0.6), mg.MG_DLINEAR, 1e-8, 400)
    assert st == mg.MG_DIVERGED and (rel > 1e6 or not np.isfinite(rel))


def test_precision_form_reaches_fp64_tolerance():
    """complex64 cycles inside FP64 defect correction on the definite
    companion of the 10%-layer problem: the plain cycle stalls at its
    FAS-perturbed fixed point, the refinement form reaches 1e-8 in FP64 as
    measured by the oracle."""
    c = W.definite(W.config2(depth=4))
    g, o = pair(c["d"], c["depth"], c["k2"], c["theta"], c["layer_width"], c["f"])
    om = O.omega_scheme(O.EXP, 0.6, 4)
    g.set_precision(mg.MG_C64_REFINE, 4)
    st, n, rel = g.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 400)
    assert st == mg.MG_OK and rel <= 1e-8
    r = o.residual(g.get_solution())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(o.b)


@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx", "hb-hier"])
def test_depth6_every_variant(var):
    """Full-size 2D level (the 12-coarse-cell tiles of the FP64 sweep), 4-cell
    layer (more Galerkin row classes), complex relaxation factors."""
    c = W.config2()
    g, o = pair(2, 6, c["k2"], c["theta"], 4 / 27, c["f"], W.random_complex(2, 6, 77))
    omega = np.array([0.6 - 0.02j * l for l in range(6)])
    run_iterates(g, o, var, omega, 1)


@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx", "hb-hier"])
def test_cycle_iterates_3d_depth4(var):
    """3D depth 4: the finest level runs the large-tile z-marching sweep with
    several z-chunks; coarse levels the small tiles."""
    depth = 4
    k2 = W.constant_k2(3, depth, 25.0)
    f = W.random_complex(3, depth, 61)
    u0 = W.random_complex(3, depth, 62)
    g, o = pair(3, depth, k2, TH, 0.1, f, u0)
    run_iterates(g, o, var, np.array([0.55, 0.6, 0.6, 0.65]), 1)


def test_config3_full_size_fused_norm_matches_standalone_residual():
    """3D depth 5 (243^3 cells, the bench's 3D size): the residual fused into
    the z-marching fine sweep equals the independent standalone residual of
    the same iterate (a property that holds at any size)."""
    c = W.config3()
    g = mg.Solver(3, 5, c["k2"], c["theta"], c["layer_width"])
    g.set_rhs(c["f"])
    g.set_solution(W.random_complex(3, 5, 7) * 1e-3)
    om = np.full(5, 0.6)
    for _ in range(2):
        a_ref, _ = g.residual_norm()  # standalone kernel on the iterate about to enter the cycle
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        a_fused, _ = g.last_cycle_norm()
        assert abs(a_fused - a_ref) <= 1e-12 * a_ref, (a_fused, a_ref)


@pytest.mark.parametrize("var", VARIANTS, ids=["add", "hb", "bpx", "hb-hier"])
@pytest.mark.parametrize("k,depth", [(5, 2), (15, 3), (45, 4)])
def test_csg_regime_iterates(var, k, depth):
    """The paper's complex-scaled-grid regime (Section 7.3): every cell rotated
    (layer width 0.5) by 35 degrees, kh = 5/9, omega = 0.8 on every level."""
    k2 = W.constant_k2(2, depth, float(k * k))
    f = W.gaussian(2, depth, (0.5, 0.5), 0.05)
    g, o = pair(2, depth, k2, math.radians(35.0), 0.5, f, W.random_complex(2, depth, 90 + depth))
    run_iterates(g, o, var, np.full(depth, 0.8), 3)


@pytest.mark.parametrize("d,depth", [(2, 4), (3, 3)])
def test_pinned_host_buffers_take_the_direct_path_and_match(d, depth):
    """Page-locked host buffers are read and written by kernels over the host
    link (mg_set_solution zeroes the ring on the way in, mg_get_solution
    writes U + P corr straight to host memory); results are bit-identical to
    the staged copies of pageable buffers and to the oracle's iterates."""
    import torch
    k2 = W.constant_k2(d, depth, 40.0)
    f = W.gaussian(d, depth, (0.4, 0.5, 0.6)[:d], 0.05)
    u0 = W.random_complex(d, depth, 31)
    u0[(0,) * d] = 5.0 + 1j  # a boundary value the ring zeroing must drop
    om = np.full(depth, 0.6)
    runs = []
    for pinned in (False, True):
        g = mg.Solver(d, depth, k2, TH, 0.2)
        if pinned:
            fh = torch.from_numpy(f.astype(np.complex128)).pin_memory()
            uh = torch.from_numpy(u0).pin_memory()
            out = torch.empty(g.shape, dtype=torch.complex128).pin_memory()
        else:
            fh, uh, out = f.astype(np.complex128), u0, np.empty(g.shape, dtype=np.complex128)
        g.set_rhs(fh)
        g.set_solution(uh)
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        g.get_solution(out)
        runs.append(out.numpy().copy() if pinned else out.copy())
        g.close()
    np.testing.assert_array_equal(runs[0], runs[1])
    o = O.Hierarchy(d, depth, k2, TH, 0.2)
    o.set_rhs_nodal(f)
    o.set_solution(u0)
    o.cycle(om, O.ADD, O.HIERARCHICAL)
    o.cycle(om, O.ADD, O.HIERARCHICAL)
    assert rel_l2(runs[1], o.u) <= TOL
