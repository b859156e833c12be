"""Pins of the adaptive-grid oracle (oracle/adaptive.py) against independent
routes: the regular oracle on a fully refined tree, and the conforming
finite-element solution on the adaptive mesh (hanging values constrained by
d-linear interpolation), computed as a dense Galerkin solve over the
hierarchical generating system sampled on the uniform finest grid."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from oracle.adaptive import AdaptiveHierarchy, child_cells

TH = math.pi / 6


def full_refinement(d, depth):
    return {lev: np.ones((3 ** lev,) * d, dtype=bool) for lev in range(1, depth)}


def l_shaped_refinement(depth):
    """2D: level 1 refines the three cells touching the lower-left corner
    cell (an L around the origin), level 2 the children nearest the origin,
    and so on -- a corner refinement with hanging vertices on every level."""
    ref = {}
    r1 = np.zeros((3, 3), dtype=bool)
    r1[0, 0] = r1[0, 1] = r1[1, 0] = True
    ref[1] = r1
    for lev in range(2, depth):
        n = 3 ** lev
        r = np.zeros((n, n), dtype=bool)
        r[: n // 3, : n // 3] = True
        r[: n // 9 + 1, n // 3: n // 3 + 2] = True
        ref[lev] = r
    return ref


def seeded(d, depth, seed):
    rng = np.random.default_rng(seed)
    n = 3 ** depth
    return rng.standard_normal((n + 1,) * d) + 1j * rng.standard_normal((n + 1,) * d)


@pytest.mark.parametrize("variant,transfer", [(O.ADD, O.DLINEAR), (O.HB, O.DLINEAR), (O.ADD, O.HIERARCHICAL)])
@pytest.mark.parametrize("theta,w", [(TH, 0.5), (0.0, 0.0)])
def test_full_refinement_equals_regular_oracle(variant, transfer, theta, w):
    """Every cell of levels 1..L-1 refined, invariant scaling and shift: the
    adaptive cycle is the regular one (Lemma 2), iterate by iterate."""
    d, depth, k2 = 2, 3, 40.0
    n = 3 ** depth
    kf = np.full((n + 1,) * d, k2)
    f = seeded(d, depth, 1)
    u0 = seeded(d, depth, 2)
    reg = O.Hierarchy(d, depth, kf, theta, w)
    reg.set_rhs_nodal(f)
    reg.set_solution(u0)
    ada = AdaptiveHierarchy(d, depth, kf, theta, w, full_refinement(d, depth))
    ada.set_rhs_nodal(f)
    u0z = u0.copy()
    O.zero_boundary(u0z)
    lv = {depth: u0z}
    for lev in range(depth - 1, 0, -1):
        lv[lev] = O.inject(lv[lev + 1])
    ada.set_solution_levels(lv)
    om = np.array([0.55 + 0.05j, 0.6, 0.65 - 0.02j])
    for _ in range(3):
        reg.cycle(om, variant, transfer)
        ada.cycle(om, variant, transfer)
        np.testing.assert_allclose(ada.u[depth], reg.u, rtol=0, atol=1e-12 * np.abs(reg.u).max())
    a, _ = ada.residual_norm()
    b, _ = reg.residual_norm()
    assert abs(a - b) <= 1e-12 * b


def test_refinement_structure_and_hanging_vertices():
    """The L-shaped corner refinement: cells of level l + 1 are the children of
    refined level-l cells; a vertex carries an unknown exactly when its 2^d
    cells exist; hanging vertices sit on the refinement boundary."""
    ada = AdaptiveHierarchy(2, 3, np.zeros((28, 28)), 0.0, 0.0, l_shaped_refinement(3))
    assert ada.cells[2].sum() == 3 * 9 and ada.cells[3].sum() == 13 * 9
    assert (ada.cells[2] == child_cells(ada.refined[1])).all()
    # level 2: the L of 3 level-1 cells is 6x6 minus the 3x3 top-right block
    assert ada.cells[2][:6, :6].sum() == 27 and not ada.cells[2][3:6, 3:6].any()
    # points inside the L carry unknowns; a vertex on the L's outer edge
    # (row 6) is hanging
    assert ada.unknown[2][2, 2] and ada.unknown[2][4, 2] and not ada.unknown[2][6, 2]
    assert ada.exists[2][6, 2] and not ada.unknown[2][6, 2]
    # the re-entrant corner (3, 3) of the L has 3 of its 4 cells: hanging
    assert ada.exists[2][3, 3] and not ada.unknown[2][3, 3]


def galerkin_composite_solution(ada, k2, f_fine):
    """The conforming finite-element solution on the adaptive mesh: u in the
    span G of the level basis functions of all unknowns, sampled on the
    uniform level-L grid, with G^T (b - H_L u) = 0 (b = M_L f, f d-linear on
    the coarsest grid so that every level samples the same function)."""
    d, L = ada.d, ada.L
    n = 3 ** L
    lev_L = O.Level(d, L, np.full((n + 1,) * d, k2), 0.0, 0.0)
    cols = []
    for lev in range(1, L + 1):
        for idx in zip(*np.nonzero(ada.unknown[lev])):
            e = np.zeros((3 ** lev + 1,) * d, dtype=np.complex128)
            e[idx] = 1.0
            for _ in range(L - lev):
                e = O.prolong(e)
            cols.append(e)
    G = np.stack([c[(slice(1, -1),) * d].ravel() for c in cols], axis=1)
    HG = np.stack([lev_L.apply(c)[(slice(1, -1),) * d].ravel() for c in cols], axis=1)
    b = lev_L.mass(f_fine)[(slice(1, -1),) * d].ravel()
    A = G.T @ HG  # G^T H G (G is real)
    rhs = G.T @ b
    y, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return G @ y


@pytest.mark.parametrize("variant,transfer", [(O.ADD, O.HIERARCHICAL), (O.ADD, O.DLINEAR)])
def test_fixed_point_is_the_composite_fe_solution(variant, transfer):
    """Corner refinement with hanging vertices on two levels, a definite
    problem: the cycle converges to the conforming finite-element solution of
    the adaptive mesh, computed independently by a dense Galerkin solve."""
    d, depth, k2 = 2, 3, -20.0
    n = 3 ** depth
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)
    f = (1.0 + X + 2.0 * Y + 3.0 * X * Y).astype(np.complex128)  # d-linear: sampled alike on all levels
    ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, k2), 0.0, 0.0, l_shaped_refinement(depth))
    ada.set_rhs_nodal(f)
    ref = galerkin_composite_solution(ada, k2, f)
    om = O.omega_scheme(O.UCG if transfer == O.HIERARCHICAL else O.EXP, 0.6, depth)
    ada.residual_norm()  # reference residual of u = 0
    for _ in range(400):
        ada.cycle(om, variant, transfer)
    _, rel = ada.residual_norm()
    got = ada.composite_on_fine()[(slice(1, -1),) * d].ravel()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert rel < 1e-9


def test_invariants_after_cycles():
    """Hanging values equal the interpolation from the coarser level and
    coarse values at vertices with a finer unknown equal the finer value."""
    d, depth = 2, 4
    n = 3 ** depth
    ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, 30.0), TH, 0.2, l_shaped_refinement(depth))
    ada.set_rhs_nodal(seeded(d, depth, 5))
    om = np.full(depth, 0.5)
    for _ in range(3):
        ada.cycle(om, O.ADD, O.HIERARCHICAL)
    for lev in range(2, depth + 1):
        hang = ada.exists[lev] & ~ada.unknown[lev]
        hang[(0, -1), :] = False
        hang[:, (0, -1)] = False
        p = O.prolong(ada.u[lev - 1])
        np.testing.assert_allclose(ada.u[lev][hang], p[hang], rtol=0, atol=1e-15)
    for lev in range(1, depth):
        fu = ada.unknown[lev + 1][::3, ::3]
        np.testing.assert_array_equal(ada.u[lev][fu], ada.u[lev + 1][::3, ::3][fu])


# ---------------------------------------------------------------------------
# succ(v) and the per-vertex relaxation factors (Section 5.1 table)

def succ_by_definition(ada):
    """succ(v) written out from its definition with plain loops: 0 unless all
    2^d cells of v's level around v are refined; else 1 + the minimum over
    the unknowns w of the next finer level that have a cell whose parent is
    a cell of v."""
    d, L = ada.d, ada.L
    memo = {}

    def cells_of(lev, v):
        out = []
        for e in itertools.product((0, 1), repeat=d):
            c = tuple(v[a] - 1 + e[a] for a in range(d))
            if all(0 <= c[a] < 3 ** lev for a in range(d)):
                out.append(c)
        return out

    def succ(lev, v):
        key = (lev, v)
        if key in memo:
            return memo[key]
        cs = cells_of(lev, v)
        refined_vertex = len(cs) == 2 ** d and all(ada.refined[lev][c] for c in cs)
        if not refined_vertex:
            memo[key] = 0
            return 0
        parents = set(cs)
        best = None
        n1 = 3 ** (lev + 1)
        for w in itertools.product(range(n1 + 1), repeat=d):
            if not ada.unknown[lev + 1][w]:
                continue
            if any(tuple(c[a] // 3 for a in range(d)) in parents for c in cells_of(lev + 1, w)):
                sw = succ(lev + 1, w)
                best = sw if best is None else min(best, sw)
        memo[key] = best + 1
        return best + 1

    return {lev: {v: succ(lev, v) for v in zip(*np.nonzero(ada.unknown[lev]))} for lev in range(1, L + 1)}


def test_succ_closed_form_on_regular_trees():
    """Fully refined trees: succ(v) = L - l at every unknown (the regular
    grid's level factors)."""
    for d, depth in [(2, 4), (3, 3)]:
        n = 3 ** depth
        ada = AdaptiveHierarchy(d, depth, np.zeros((n + 1,) * d), 0.0, 0.0, full_refinement(d, depth))
        for lev in range(1, depth + 1):
            assert (ada.succ[lev][ada.unknown[lev]] == depth - lev).all()


def corner_refinement_3d(depth):
    ref = {1: np.zeros((3, 3, 3), dtype=bool)}
    ref[1][0, 0, 0] = ref[1][0, 0, 1] = ref[1][0, 1, 0] = True
    for lev in range(2, depth):
        n = 3 ** lev
        r = np.zeros((n,) * 3, dtype=bool)
        r[: n // 3, : n // 3, : n // 9 + 1] = True
        ref[lev] = r
    return ref


@pytest.mark.parametrize("d,depth", [(2, 4), (3, 3)])
def test_succ_matches_its_definition_on_corner_refinements(d, depth):
    n = 3 ** depth
    ref = l_shaped_refinement(depth) if d == 2 else corner_refinement_3d(depth)
    ada = AdaptiveHierarchy(d, depth, np.zeros((n + 1,) * d), 0.0, 0.0, ref)
    want = succ_by_definition(ada)
    seen = set()
    for lev in range(1, depth + 1):
        for v, s in want[lev].items():
            assert ada.succ[lev][v] == s, (lev, v)
            seen.add(s)
    assert len(seen) >= (3 if d == 2 else 2)  # several succ values occur


def generating_system_cycle(ada, omega, transfer, f_fine, k2):
    """One cycle written densely on the uniform finest grid (invariant scaling
    and shift, so every level's diagonal is that of the prolongated basis
    function): du_(l,v) = omega[L-1-succ(v)] (G^T (b - H u))_(l,v) / (G^T H G)
    diagonal, T_l on each level's vector, and the prolongated sum added to
    the fine-grid function u.  succ comes from its definition.  With a
    constant shift and no scaling the operator is translation invariant, so
    the diagonal is formed once per level (from the level's first unknown;
    every unknown's hat lies inside the domain)."""
    d, L = ada.d, ada.L
    n = 3 ** L
    lev_L = O.Level(d, L, np.full((n + 1,) * d, k2), 0.0, 0.0)
    succ = succ_by_definition(ada)
    u = ada.composite_on_fine()
    res = lev_L.mass(f_fine) - lev_L.apply(u)
    corr = np.zeros_like(u)
    for lev in range(1, L + 1):
        t = np.zeros((3 ** lev + 1,) * d, dtype=np.complex128)
        a = None
        for v, s in succ[lev].items():
            e = np.zeros_like(t)
            e[v] = 1.0
            for _ in range(L - lev):
                e = O.prolong(e)
            g = np.vdot(e, res)  # e is real: e^T res
            if a is None:
                a = np.vdot(e, lev_L.apply(e))
            t[v] = omega[L - 1 - s] * g / a
        if transfer == O.HIERARCHICAL:
            t = t - O.prolong(O.inject(t))
        for _ in range(L - lev):
            t = O.prolong(t)
        corr += t
    out = u + corr
    O.zero_boundary(out)
    return out


@pytest.mark.parametrize("transfer", [O.DLINEAR, O.HIERARCHICAL])
def test_cycle_is_the_generating_system_correction_with_succ_factors(transfer):
    """Corner refinement, definite problem, distinct factors per succ: one
    cycle of the oracle equals the dense generating-system correction with
    factors looked up by succ(v) (so a coarse fine-grid vertex takes the
    finest level's factor)."""
    d, depth, k2 = 2, 3, -20.0
    n = 3 ** depth
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)
    f = (1.0 + X + 2.0 * Y + 3.0 * X * Y).astype(np.complex128)
    ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, k2), 0.0, 0.0, l_shaped_refinement(depth))
    ada.set_rhs_nodal(f)
    om = np.array([0.3, 0.45 + 0.05j, 0.6])
    for _ in range(2):
        ada.cycle(om, O.ADD, transfer)
    want = generating_system_cycle(ada, om, transfer, f, k2)
    ada.cycle(om, O.ADD, transfer)
    got = ada.composite_on_fine()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_cycle_is_the_generating_system_correction_in_3d():
    """The same dense check in three dimensions (depth 3, three refined
    level-1 cells and a level-2 block: hanging vertices on two levels),
    BPX transfer and distinct factors per succ."""
    d, depth, k2 = 3, 3, -15.0
    n = 3 ** depth
    x = np.arange(n + 1) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = (1.0 + X + 2.0 * Y - Z + 3.0 * X * Y * Z).astype(np.complex128)  # trilinear
    ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, k2), 0.0, 0.0, corner_refinement_3d(depth))
    ada.set_rhs_nodal(f)
    om = np.array([0.35, 0.5 - 0.05j, 0.65])
    ada.cycle(om, O.ADD, O.HIERARCHICAL)
    want = generating_system_cycle(ada, om, O.HIERARCHICAL, f, k2)
    ada.cycle(om, O.ADD, O.HIERARCHICAL)
    got = ada.composite_on_fine()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


# ---------------------------------------------------------------------------
# feature-based dynamic refinement (Section 5.3)

def set_levels_from(ada, fn):
    """u_l = fn sampled at every level's vertices (invariants restored)."""
    lv = {}
    for lev in range(1, ada.L + 1):
        m = 3 ** lev
        xs = np.meshgrid(*([np.arange(m + 1) / m] * ada.d), indexing="ij")
        lv[lev] = fn(*xs[::-1]).astype(np.complex128)  # x = last axis
    ada.set_solution_levels(lv)


def test_indicator_matches_plain_loops():
    d, depth = 2, 3
    ada = AdaptiveHierarchy(d, depth, np.zeros((28, 28)), TH, 0.2, l_shaped_refinement(depth))
    rng = np.random.default_rng(11)
    lv = {lev: rng.standard_normal((3 ** lev + 1,) * d) + 1j * rng.standard_normal((3 ** lev + 1,) * d)
          for lev in range(1, depth + 1)}
    ada.set_solution_levels(lv)
    s = ada.refinement_indicator()
    for lev in range(1, depth + 1):
        u = ada.u[lev]
        fine = ada.fine_grid(lev)
        for v in itertools.product(range(3 ** lev + 1), repeat=d):
            if not fine[v]:
                assert s[lev][v] == -1.0
                continue
            best = 0.0
            for ax in range(d):
                lo, hi = list(v), list(v)
                lo[ax] -= 1
                hi[ax] += 1
                best = max(best, abs(u[tuple(lo)] - 2 * u[v] + u[tuple(hi)]))
            assert abs(s[lev][v] - best) <= 1e-15 * max(best, 1.0), (lev, v)


def test_choose_bins():
    from oracle.adaptive import choose_bins
    assert choose_bins([3, 0, 0, 600], 67.6) == 1  # a skewed distribution takes the tail only
    assert choose_bins([10, 20, 30, 40], 30.0) == 2  # 10 + 20 = 30 exactly
    assert choose_bins([10, 20, 30, 40], 45.0) == 2  # |30-45| = 15 < |60-45| = 15 is a tie: the smaller k
    assert choose_bins([10, 20, 30, 40], 0.0) == 0
    assert choose_bins([5, 5], 100.0) == 2


def selection_by_hand(ada, min_level, refine_frac, erase_frac, bins):
    """Reading A6 with plain Python over the fine-grid vertices (no veto)."""
    s = ada.refinement_indicator()
    items = [(lev, v, s[lev][v]) for lev in range(1, ada.L + 1)
             for v in zip(*np.nonzero(ada.fine_grid(lev)))]
    vals = [x[2] for x in items]
    lo, hi = min(vals), max(vals)
    binof = {}
    for lev, v, sv in items:
        b = 0 if hi == lo else min(int(math.floor(((sv - lo) / (hi - lo)) * bins)), bins - 1)
        binof[(lev, v)] = b
    counts = [0] * bins
    for b in binof.values():
        counts[b] += 1
    from oracle.adaptive import choose_bins
    k_ref = choose_bins(counts[::-1], refine_frac * len(items))
    k_er = choose_bins(counts, erase_frac * len(items))
    ref = {key for key, b in binof.items() if b >= bins - k_ref}
    er = {key for key, b in binof.items() if b < k_er and key not in ref and key[0] >= min_level + 1}
    return ref, er


def bump(x, y):
    return x + 0.5 * y + 10.0 * np.exp(-((x - 0.8) ** 2 + (y - 0.75) ** 2) / 0.004)


def test_pure_refinement_refines_the_selected_vertices_and_keeps_the_function():
    d, depth = 2, 4
    n = 3 ** depth
    ref = {1: np.ones((3, 3), dtype=bool), 2: np.zeros((9, 9), dtype=bool), 3: np.zeros((27, 27), dtype=bool)}
    ref[2][5:8, 5:8] = True
    ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, -10.0), 0.0, 0.0, ref)
    set_levels_from(ada, bump)
    before = ada.composite_on_fine()
    sel, _ = selection_by_hand(ada, 2, 0.1, 0.0, 20)
    old = {lev: ada.refined[lev].copy() for lev in range(1, depth)}
    n_ref, n_er, nfine = ada.adapt(min_level=2, refine_frac=0.1, erase_frac=0.0, veto=np.inf)
    assert n_er == 0 and n_ref == sum(1 for lev, _ in sel if lev < depth) > 0
    expect = {lev: old[lev].copy() for lev in old}
    for lev, v in sel:
        if lev == depth:
            continue  # h_min
        for e in itertools.product((0, 1), repeat=d):
            expect[lev][tuple(v[a] - 1 + e[a] for a in range(d))] = True
    for lev in range(1, depth):
        np.testing.assert_array_equal(ada.refined[lev], expect[lev] & ada.cells[lev])
    assert any((ada.refined[lev] != old[lev]).any() for lev in old)
    np.testing.assert_allclose(ada.composite_on_fine(), before, rtol=0, atol=1e-14 * np.abs(before).max())
    assert nfine == ada.fine_vertex_count()


def test_erasing_coarsens_flat_refined_regions_only():
    """A refined patch where u is linear (s = 0) is coarsened when the bottom
    bin is erased; a patch at the bump is kept; level-1 cells (below
    min_level) are never coarsened; the fine-grid function is unchanged
    where the coarse interpolation reproduces it (linear u)."""
    d, depth = 2, 4
    n = 3 ** depth
    ref = {1: np.ones((3, 3), dtype=bool), 2: np.zeros((9, 9), dtype=bool), 3: np.zeros((27, 27), dtype=bool)}
    ref[2][1:3, 1:3] = True  # flat patch
    ref[2][6:8, 6:8] = True  # at the bump
    ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, -10.0), 0.0, 0.0, ref)
    set_levels_from(ada, bump)
    _, er = selection_by_hand(ada, 2, 0.0, 0.5, 20)
    assert er
    before = ada.composite_on_fine()
    ada.adapt(min_level=2, refine_frac=0.0, erase_frac=0.5, veto=np.inf)
    assert not ada.refined[2][1:3, 1:3].any()
    assert ada.refined[2][6:8, 6:8].all()
    assert ada.refined[1].all()
    # on the coarsened patch the function is the (linear) coarse interpolant
    sl = (slice(9, 27), slice(9, 27))
    np.testing.assert_allclose(ada.composite_on_fine()[sl], before[sl], rtol=0, atol=1e-13)


def test_vetoes():
    """A residual veto below every |r / diag| leaves the grid as it is; with
    no veto the same step refines."""
    d, depth = 2, 3
    n = 3 ** depth
    ref = {1: np.ones((3, 3), dtype=bool), 2: np.zeros((9, 9), dtype=bool)}
    ref[2][6:8, 6:8] = True
    for veto, changes in [(1e-300, False), (np.inf, True)]:
        ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, -10.0), 0.0, 0.0, ref)
        ada.set_rhs_nodal(np.ones((n + 1,) * d, dtype=np.complex128))
        set_levels_from(ada, bump)
        old = ada.refine_flags()
        ada.adapt(min_level=1, refine_frac=0.1, erase_frac=0.02, veto=veto)
        assert (ada.refine_flags() != old).any() == changes


def test_relative_veto():
    """Read relative to the vertex's value, the veto blocks the vertices whose
    Jacobi update |r / diag| exceeds veto |u(v)|: with veto 1e300 (an update
    never exceeds it) it selects what no veto selects; with a veto below
    every |r / diag| / |u| nothing changes; in between exactly the vertices
    above the bound are spared."""
    d, depth = 2, 3
    n = 3 ** depth
    ref = {1: np.ones((3, 3), dtype=bool), 2: np.zeros((9, 9), dtype=bool)}
    ref[2][6:8, 6:8] = True

    def make():
        ada = AdaptiveHierarchy(d, depth, np.full((n + 1,) * d, -10.0), 0.0, 0.0, ref)
        ada.set_rhs_nodal(np.ones((n + 1,) * d, dtype=np.complex128))
        set_levels_from(ada, bump)
        return ada

    free = make()
    free.adapt(min_level=1, refine_frac=0.1, erase_frac=0.02, veto=np.inf)
    loose = make()
    loose.adapt(min_level=1, refine_frac=0.1, erase_frac=0.02, veto=1e300, veto_relative=True)
    np.testing.assert_array_equal(loose.refine_flags(), free.refine_flags())
    tight = make()
    old = tight.refine_flags()
    tight.adapt(min_level=1, refine_frac=0.1, erase_frac=0.02, veto=1e-300, veto_relative=True)
    np.testing.assert_array_equal(tight.refine_flags(), old)
    # a bound between: the selected set shrinks to the vertices under the bound
    mid = make()
    r = mid.level_residuals()
    ratios = np.concatenate([np.abs(r[l] / mid.levels[l].diag)[mid.fine_grid(l)] /
                             np.abs(mid.u[l])[mid.fine_grid(l)] for l in range(1, depth + 1)])
    veto = float(np.median(ratios))
    n_ref_free = make().adapt(min_level=1, refine_frac=0.1, erase_frac=0.0, veto=np.inf)[0]
    n_ref_mid = mid.adapt(min_level=1, refine_frac=0.1, erase_frac=0.0, veto=veto, veto_relative=True)[0]
    assert 0 <= n_ref_mid < n_ref_free


def bump3(x, y, z):
    return x + 0.5 * y + 0.25 * z + 10.0 * np.exp(-((x - 0.8) ** 2 + (y - 0.75) ** 2 + (z - 0.7) ** 2) / 0.004)


def test_refining_and_erasing_in_three_dimensions():
    """The 3D counterparts of the two tests above (children, closures and
    corners over 3 axes): pure refinement refines exactly the cells around
    the hand-selected vertices and keeps the fine-grid function; erasing the
    bottom bins coarsens the refined patch where u is linear and keeps the
    one at the bump."""
    d, depth = 3, 3
    n = 3 ** depth
    ref = {1: np.ones((3, 3, 3), dtype=bool), 2: np.zeros((9, 9, 9), dtype=bool)}
    ref[2][1:3, 1:3, 1:3] = True  # flat patch (u linear there)
    ref[2][5:8, 6:8, 6:8] = True  # at the bump (z, y, x order: x = last axis)
    k2 = np.full((n + 1,) * d, -10.0)
    # pure refinement
    ada = AdaptiveHierarchy(d, depth, k2, 0.0, 0.0, ref)
    set_levels_from(ada, bump3)
    before = ada.composite_on_fine()
    sel, _ = selection_by_hand(ada, 2, 0.1, 0.0, 20)
    old = {lev: ada.refined[lev].copy() for lev in range(1, depth)}
    n_ref, n_er, _ = ada.adapt(min_level=2, refine_frac=0.1, erase_frac=0.0, veto=np.inf)
    assert n_er == 0 and n_ref == sum(1 for lev, _ in sel if lev < depth) > 0
    expect = {lev: old[lev].copy() for lev in old}
    for lev, v in sel:
        if lev == depth:
            continue
        for e in itertools.product((0, 1), repeat=d):
            expect[lev][tuple(v[a] - 1 + e[a] for a in range(d))] = True
    for lev in range(1, depth):
        np.testing.assert_array_equal(ada.refined[lev], expect[lev] & ada.cells[lev])
    np.testing.assert_allclose(ada.composite_on_fine(), before, rtol=0, atol=1e-14 * np.abs(before).max())
    # erasing
    ada = AdaptiveHierarchy(d, depth, k2, 0.0, 0.0, ref)
    set_levels_from(ada, bump3)
    _, er = selection_by_hand(ada, 2, 0.0, 0.5, 20)
    assert er
    before = ada.composite_on_fine()
    ada.adapt(min_level=2, refine_frac=0.0, erase_frac=0.5, veto=np.inf)
    assert not ada.refined[2][1:3, 1:3, 1:3].any()
    assert ada.refined[2][5:8, 6:8, 6:8].all()
    sl = (slice(3, 10), slice(3, 10), slice(3, 10))
    np.testing.assert_allclose(ada.composite_on_fine()[sl], before[sl], rtol=0, atol=1e-13)
