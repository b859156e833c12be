"""Pins of the adaptive-grid oracle (oracle/adaptive.py) against independent
routes: the regular oracle on a fully refined tree, and the conforming
finite-element solution on the adaptive mesh (hanging values constrained by
d-linear interpolation), computed as a dense Galerkin solve over the
hierarchical generating system sampled on the uniform finest grid."""
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
