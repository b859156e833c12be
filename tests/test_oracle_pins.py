"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent route to the same result -- closed-form stencils and eigenvalues
of the d-linear finite element operator, the Galerkin identity of nested
element spaces, the textbook additive correction scheme (Algorithm 1) built
from Kronecker products, dense direct solves, and the analytic Poisson
solution of Section 7.1, and the residual reductions that Table 2 prints for
the channel problem of Section 7.4.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O

TH = math.pi / 6


def dense_level(d, level, k2, theta, w, theta_interior=0.0):
    """Dense matrix of the oracle's level operator on interior unknowns,
    obtained by applying it to unit vectors."""
    lev = O.Level(d, level, k2, theta, w, theta_interior)
    n = 3 ** level
    inner = list(itertools.product(range(1, n), repeat=d))
    A = np.zeros((len(inner), len(inner)), dtype=np.complex128)
    for j, idx in enumerate(inner):
        e = np.zeros((n + 1,) * d, dtype=np.complex128)
        e[idx] = 1
        col = lev.apply(e)
        A[:, j] = [col[i] for i in inner]
    return A, inner, lev


# ---------------------------------------------------------------- 1D blocks
def tri_1d(hs):
    """Assembled 1D stiffness and mass on n cells of widths hs, interior rows
    and columns: the textbook tridiagonal matrices of linear elements."""
    n = len(hs)
    K = np.zeros((n - 1, n - 1), dtype=np.complex128)
    M = np.zeros((n - 1, n - 1), dtype=np.complex128)
    for i in range(1, n):  # vertex i between cells i-1 and i
        r = i - 1
        K[r, r] = 1 / hs[i - 1] + 1 / hs[i]
        M[r, r] = (hs[i - 1] + hs[i]) / 3
        if r > 0:
            K[r, r - 1] = -1 / hs[i - 1]
            M[r, r - 1] = hs[i - 1] / 6
        if r < n - 2:
            K[r, r + 1] = -1 / hs[i]
            M[r, r + 1] = hs[i] / 6
    return K, M


def kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def kron_operator(d, level, theta, w, k2):
    """H = sum_j (x)_k (K if k == j else M) - k2 (x)_k M for a constant shift:
    the separable form of the tensor-product element operator."""
    hs = O.axis_spacing(level, theta, w)  # same widths on every axis
    K, M = tri_1d(hs)
    H = -k2 * kron_all([M] * d)
    for j in range(d):
        H = H + kron_all([K if k == j else M for k in range(d)])
    return H


def interp_1d(nc):
    """Interior-to-interior tripartite linear interpolation in 1D."""
    P = np.zeros((3 * nc - 1, nc - 1))
    for c in range(1, nc):
        for o in range(-2, 3):
            f = 3 * c + o
            if 1 <= f <= 3 * nc - 1:
                P[f - 1, c - 1] = 1 - abs(o) / 3
    return P


# ---------------------------------------------------------------- element matrices
def test_element_matrix_2d_closed_form():
    h = 1 / 9
    kc, mc = O.element_matrices((h, h))
    # bilinear square element, local order (y, x): (0,0),(0,1),(1,0),(1,1)
    K = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6
    M = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) * h * h / 36
    np.testing.assert_allclose(kc, K, rtol=0, atol=1e-15)
    np.testing.assert_allclose(mc, M, rtol=0, atol=1e-18)


def _stencil(d, level, with_phi, k2=0.0, theta=0.0, w=0.0):
    n = 3 ** level
    lev = O.Level(d, level, np.full((n + 1,) * d, k2), theta, w)
    e = np.zeros((n + 1,) * d, dtype=np.complex128)
    c = (n // 2,) * d
    e[c] = 1
    col = lev.apply(e, with_phi=with_phi)
    sl = tuple(slice(i - 1, i + 2) for i in c)
    return col[sl]


def test_assembled_stencils_2d():
    h = 1 / 27
    K = _stencil(2, 3, True)
    np.testing.assert_allclose(K, np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]]) / 3,
                               rtol=0, atol=1e-14)
    M = _stencil(2, 3, False)
    np.testing.assert_allclose(M, np.array([[1, 4, 1], [4, 16, 4], [1, 4, 1]]) * h * h / 36,
                               rtol=1e-14, atol=0)


def test_assembled_stencils_3d():
    h = 1 / 9
    K = _stencil(3, 2, True)
    cls = np.zeros((3, 3, 3))
    for idx in itertools.product(range(3), repeat=3):
        nz = sum(1 for i in idx if i != 1)
        cls[idx] = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[nz]
    np.testing.assert_allclose(K, cls, rtol=0, atol=1e-15)
    M = _stencil(3, 2, False)
    w = np.array([1.0, 4.0, 1.0])
    ref = np.einsum("i,j,k->ijk", w, w, w) * h ** 3 / 216
    np.testing.assert_allclose(M, ref, rtol=1e-14, atol=0)


def test_diagonal_closed_form_and_dense():
    # uniform real interior: D = 8/3 - k^2 * 16 h^2/36
    h, k2 = 1 / 27, (4 * math.pi) ** 2
    n = 27
    lev = O.Level(2, 3, np.full((n + 1,) * 2, k2), 0.0, 0.0)
    np.testing.assert_allclose(lev.diag[5, 7], 8 / 3 - k2 * 16 * h * h / 36, rtol=1e-14)
    # with a layer and a varying shift: the diagonal of the dense operator
    rng = np.random.default_rng(0)
    k2f = rng.uniform(10, 50, size=(10, 10))
    A, inner, lev = dense_level(2, 2, k2f, TH, 0.2)
    np.testing.assert_allclose([lev.diag[i] for i in inner], np.diag(A), rtol=1e-14)


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("d,level", [(2, 3), (3, 2)])
def test_sine_mode_eigenvalues_uniform_complex_scaling(d, level):
    """Full complex scaled grid (w = 0.5): H s = lambda s for the Dirichlet
    sine modes with lambda = sum_j kappa_j prod_{k!=j} mu_k - k^2 prod mu."""
    n = 3 ** level
    k2 = (4 * math.pi) ** 2
    lev = O.Level(d, level, np.full((n + 1,) * d, k2), TH, 0.5)
    hc = (1 / n) * complex(math.cos(TH), math.sin(TH))
    x = np.arange(n + 1) / n
    for modes in [(1,) * d, (2, 3, 1)[:d], (n - 1,) + (4,) * (d - 1)]:
        s = np.ones((1,) * d)
        for ax, m in enumerate(modes):
            shape = [1] * d
            shape[ax] = n + 1
            s = s * np.sin(m * math.pi * x).reshape(shape)
        s = s.astype(np.complex128)
        kap = [(2 / hc) * (1 - math.cos(m * math.pi / n)) for m in modes]
        mu = [(hc / 3) * (2 + math.cos(m * math.pi / n)) for m in modes]
        lam = -k2 * np.prod(mu)
        for j in range(d):
            lam += kap[j] * np.prod([mu[k] for k in range(d) if k != j])
        Hs = lev.apply(s)
        inner = (slice(1, -1),) * d
        np.testing.assert_allclose(Hs[inner], lam * s[inner], rtol=1e-12,
                                   atol=1e-13 * abs(lam))


@pytest.mark.parametrize("d,level,w", [(2, 2, 0.2), (2, 3, 4 / 27), (3, 2, 0.1)])
def test_operator_equals_kronecker_of_1d_elements(d, level, w):
    """Coordinate-wise scaling with constant shift gives the separable operator
    sum_j (x)(K or M) - k^2 (x)M of 1D assembled matrices with per-cell widths."""
    n = 3 ** level
    k2 = 30.0
    A, _, _ = dense_level(d, level, np.full((n + 1,) * d, k2), TH, w)
    H = kron_operator(d, level, TH, w, k2)
    np.testing.assert_allclose(A, H, rtol=0, atol=1e-13 * np.abs(H).max())


def test_complex_symmetric_with_layer_and_varying_shift():
    rng = np.random.default_rng(1)
    k2 = rng.uniform(-20, 80, size=(10, 10))
    A, _, _ = dense_level(2, 2, k2, TH, 0.15)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    assert np.abs(A - A.conj().T).max() > 1e-3  # not Hermitian: complex h


def test_layer_membership_and_mass_rhs():
    """f = 1: b_v = sum over adjacent cells of prod_j h_j / 2^d, so a vertex
    whose cells are rotated along x only gets h e^{i th} * h (coordinate-wise
    scaling); the centre-of-cell rule puts exactly 4 cells per side in the
    layer of width 4/27 at depth 3."""
    n = 27
    rot = O.rotated_cells(3, 4 / 27)
    assert rot.sum() == 8 and rot[:4].all() and rot[-4:].all() and not rot[4:-4].any()
    assert O.rotated_cells(2, 4 / 27).sum() == 2 and O.rotated_cells(1, 4 / 27).sum() == 0
    assert O.rotated_cells(3, 0.5).all()
    h = 1 / n
    e = complex(math.cos(TH), math.sin(TH))
    H = O.Hierarchy(2, 3, np.zeros((n + 1, n + 1)), TH, 4 / 27)
    H.set_rhs_nodal(np.ones((n + 1, n + 1)))
    b = H.b
    np.testing.assert_allclose(b[13, 13], h * h, rtol=1e-14)          # interior
    np.testing.assert_allclose(b[13, 2], h * e * h, rtol=1e-14)       # x-layer only (axis 1 = x)
    np.testing.assert_allclose(b[2, 13], h * h * e, rtol=1e-14)       # y-layer only
    np.testing.assert_allclose(b[2, 2], h * h * e * e, rtol=1e-14)    # corner
    # vertex 4 lies between a rotated cell (3) and a plain one (4)
    np.testing.assert_allclose(b[13, 4], h * (h * e + h) / 2, rtol=1e-14)


# ---------------------------------------------------------------- transfers
@pytest.mark.parametrize("d,level", [(2, 2), (3, 2)])
def test_restriction_is_prolongation_transpose(d, level):
    nf, nc = 3 ** level, 3 ** (level - 1)
    Nc, Nf = (nc + 1) ** d, (nf + 1) ** d
    P = np.zeros((Nf, Nc))
    R = np.zeros((Nc, Nf))
    for j in range(Nc):
        e = np.zeros(Nc)
        e[j] = 1
        P[:, j] = O.prolong(e.reshape((nc + 1,) * d)).real.ravel()
    for j in range(Nf):
        e = np.zeros(Nf)
        e[j] = 1
        R[:, j] = O.restrict(e.reshape((nf + 1,) * d)).real.ravel()
    np.testing.assert_array_equal(R, P.T)
    # partition of unity and the 3^d column sum of interior coarse vertices
    np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    inner_c = [i for i, idx in enumerate(itertools.product(range(nc + 1), repeat=d))
               if all(0 < k < nc for k in idx)]
    np.testing.assert_allclose(R.sum(axis=1)[inner_c], 3.0 ** d, rtol=1e-15)
    # independent construction from 1D weights
    P1 = np.zeros((nf + 1, nc + 1))
    for c in range(nc + 1):
        for o in range(-2, 3):
            if 0 <= 3 * c + o <= nf:
                P1[3 * c + o, c] = 1 - abs(o) / 3
    np.testing.assert_allclose(P, kron_all([P1] * d), rtol=0, atol=2.5e-16)


def test_prolongation_reproduces_dlinear_functions():
    nc = 9
    xc = np.arange(nc + 1) / nc
    xf = np.arange(3 * nc + 1) / (3 * nc)
    f = lambda y, x: 2.0 - 3 * x + 0.5 * y + 7 * x * y
    Yc, Xc = np.meshgrid(xc, xc, indexing="ij")
    Yf, Xf = np.meshgrid(xf, xf, indexing="ij")
    np.testing.assert_allclose(O.prolong(f(Yc, Xc)).real, f(Yf, Xf), rtol=0, atol=1e-13)
    np.testing.assert_array_equal(O.inject(O.prolong(f(Yc, Xc))), f(Yc, Xc).astype(complex))


@pytest.mark.parametrize("d,level,k2", [(2, 2, 30.0), (2, 3, (4 * math.pi) ** 2), (3, 2, -40.0)])
def test_galerkin_identity_uniform_scaling(d, level, k2):
    """H_{l-1} = R H_l P for invariant scaling and shift (Section 4)."""
    nf, nc = 3 ** level, 3 ** (level - 1)
    Hf, _, _ = dense_level(d, level, np.full((nf + 1,) * d, k2), TH, 0.5)
    Hc, _, _ = dense_level(d, level - 1, np.full((nc + 1,) * d, k2), TH, 0.5)
    P = kron_all([interp_1d(nc)] * d)
    G = P.T @ Hf @ P
    np.testing.assert_allclose(G, Hc, rtol=0, atol=1e-13 * np.abs(Hc).max())


def test_galerkin_defect_at_unaligned_layer_edge():
    """With a layer edge that coarse cells straddle, rediscretisation deviates
    from R H P (Section 6, remark after Lemma 2) -- but only near the edge."""
    k2 = 30.0
    Hf, _, _ = dense_level(2, 3, np.full((28, 28), k2), TH, 4 / 27)
    Hc, inner, _ = dense_level(2, 2, np.full((10, 10), k2), TH, 4 / 27)
    P = kron_all([interp_1d(9)] * 2)
    E = np.abs(P.T @ Hf @ P - Hc).max(axis=1)
    assert E.max() > 1e-3
    far = [r for r, (y, x) in enumerate(inner) if 3 <= y <= 6 and 3 <= x <= 6]
    assert E[far].max() < 1e-12


# ---------------------------------------------------------------- cycle
def _problem(d, depth, k2, theta, w, seed=0):
    n = 3 ** depth
    rng = np.random.default_rng(seed)
    H = O.Hierarchy(d, depth, np.full((n + 1,) * d, k2), theta, w)
    f = rng.standard_normal((n + 1,) * d) + 1j * rng.standard_normal((n + 1,) * d)
    H.set_rhs_nodal(f)
    u0 = rng.standard_normal((n + 1,) * d) + 1j * rng.standard_normal((n + 1,) * d)
    H.set_solution(u0)
    return H


def test_single_level_cycle_is_damped_jacobi():
    H = _problem(2, 1, 20.0, TH, 0.2)
    A, inner, lev = dense_level(2, 1, np.full((4, 4), 20.0), TH, 0.2)
    u = np.array([H.u[i] for i in inner])
    b = np.array([H.b[i] for i in inner])
    w = 0.7 - 0.1j
    ref = u + w * (b - A @ u) / np.diag(A)
    H.cycle(np.array([w]))
    np.testing.assert_allclose([H.u[i] for i in inner], ref, rtol=1e-14)


@pytest.mark.parametrize("d,depth", [(2, 3), (3, 2)])
@pytest.mark.parametrize("variant,transfer", [(O.ADD, O.DLINEAR), (O.HB, O.DLINEAR),
                                              (O.ADD, O.HIERARCHICAL)])
def test_fas_cycle_equals_additive_correction_scheme(d, depth, variant, transfer):
    """Lemma 2 and Theorem 2: with invariant scaling and shift the FAS cycle
    is the textbook additive correction scheme (Algorithm 1 unrolled)
    u + sum_l P^{L-l} T_l omega_l D_l^{-1} R^{L-l} (b - H u),
    here assembled from Kronecker products of 1D matrices."""
    k2 = 25.0
    Hh = _problem(d, depth, k2, TH, 0.5)
    omega = np.array([0.55 + 0.05j, 0.6, 0.65 - 0.02j][:depth])
    Hs = {lev: kron_operator(d, lev, TH, 0.5, k2) for lev in range(1, depth + 1)}
    Ps = {lev: kron_all([interp_1d(3 ** (lev - 1))] * d) for lev in range(2, depth + 1)}
    n = 3 ** depth
    inner = list(itertools.product(range(1, n), repeat=d))
    u = np.array([Hh.u[i] for i in inner])
    b = np.array([Hh.b[i] for i in inner])
    r = b - Hs[depth] @ u
    corr = np.zeros_like(u)
    for lev in range(depth, 0, -1):
        rl = r
        for m in range(depth, lev, -1):
            rl = Ps[m].T @ rl
        du = omega[lev - 1] * rl / np.diag(Hs[lev])
        nl = 3 ** lev
        idx = list(itertools.product(range(1, nl), repeat=d))
        cp = np.array([all(i % 3 == 0 for i in t) for t in idx])
        if variant == O.HB:
            du = np.where(cp, 0, du)
        if transfer == O.HIERARCHICAL and lev > 1:
            du = du - Ps[lev] @ du[cp]       # P I du
        for m in range(lev + 1, depth + 1):
            du = Ps[m] @ du
        corr += du
    Hh.cycle(omega, variant, transfer)
    got = np.array([Hh.u[i] for i in inner])
    np.testing.assert_allclose(got, u + corr, rtol=0, atol=1e-12 * np.abs(u + corr).max())


def test_cycle_fixed_point_is_dense_solution_galerkin():
    """A convergent Galerkin setup (Poisson-like, phi < 0, theta = 0) converges
    to the dense direct solution of the 9x9-cell problem."""
    H = _problem(2, 2, -30.0, 0.0, 0.0, seed=3)
    H.set_solution(np.zeros((10, 10)))
    A, inner, _ = dense_level(2, 2, np.full((10, 10), -30.0), 0.0, 0.0)
    x = np.linalg.solve(A, np.array([H.b[i] for i in inner]))
    om = O.omega_scheme(O.UCG, 0.6, 2)
    for _ in range(200):
        H.cycle(om, O.ADD, O.HIERARCHICAL)
    np.testing.assert_allclose([H.u[i] for i in inner], x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_poisson_analytic_discrete_solution():
    """Section 7.1: rhs d pi^2 prod sin(pi x_i), phi = 0, theta = 0.  The mode
    (1,..,1) diagonalises K and M, so the discrete solution is
    pi^2 (mu/kappa) prod sin(pi x_i); the cycle converges to it and it is an
    O(h^2) approximation of prod sin(pi x_i)."""
    for d, depth in [(2, 3), (3, 2)]:
        n = 3 ** depth
        h = 1 / n
        x = np.arange(n + 1) / n
        s = np.ones((1,) * d)
        for ax in range(d):
            shape = [1] * d
            shape[ax] = n + 1
            s = s * np.sin(math.pi * x).reshape(shape)
        H = O.Hierarchy(d, depth, np.zeros((n + 1,) * d), 0.0, 0.0)
        H.set_rhs_nodal(d * math.pi ** 2 * s)
        kap = (2 / h) * (1 - math.cos(math.pi * h))
        mu = (h / 3) * (2 + math.cos(math.pi * h))
        exact = math.pi ** 2 * (mu / kap) * s
        np.testing.assert_allclose(H.residual(exact.astype(complex)), 0, atol=1e-12)
        om = O.omega_scheme(O.UCG, 0.8 if d == 2 else 0.6, depth)
        for _ in range(300):
            H.cycle(om, O.ADD, O.HIERARCHICAL)
        np.testing.assert_allclose(H.u.real, exact, rtol=0, atol=1e-9)
        assert np.abs(H.u.imag).max() < 1e-12
        err = np.abs(exact - s).max()
        assert err < 2.0 * (math.pi * h) ** 2 / 12 * d + 1e-12


def test_bpx_and_hb_cpoint_structure():
    """BPX: (id - P I) vanishes at c-points, so corr_l there equals P corr_{l-1}
    (Section 5.2); hb: the masked update leaves corr_l = P corr_{l-1} at
    c-points as well, while f-point updates pass unchanged."""
    for variant, transfer in [(O.ADD, O.HIERARCHICAL), (O.HB, O.DLINEAR)]:
        H = _problem(2, 3, 10.0, TH, 0.2)
        tr = {}
        H.cycle(np.array([0.6, 0.6, 0.6]), variant, transfer, trace=tr)
        for lev in (2, 3):
            cp = O.cpoint_mask(2, lev)
            pc = O.prolong(tr["corr"][lev - 1])
            np.testing.assert_allclose(tr["corr"][lev][cp], pc[cp], rtol=0, atol=1e-14)
            fp = ~cp
            fp[0, :] = fp[-1, :] = fp[:, 0] = fp[:, -1] = False
            assert np.abs(tr["corr"][lev][fp] - pc[fp]).max() > 1e-8


def test_omega_schemes():
    np.testing.assert_allclose(O.omega_scheme(O.JACOBI, 0.6, 3), [0, 0, 0.6])
    np.testing.assert_allclose(O.omega_scheme(O.UCG, 0.6, 3), [0.6, 0.6, 0.6])
    np.testing.assert_allclose(O.omega_scheme(O.LGRID, 0.6, 4, l_grid=1), [0, 0, 0.6, 0.6])
    np.testing.assert_allclose(O.omega_scheme(O.EXP, 0.5, 3), [0.125, 0.25, 0.5])
    np.testing.assert_allclose(O.omega_scheme(O.TRANSITION, 0.5, 3, iter_n=2),
                               [0.5 ** 1.5, 0.5, 0.5 ** 0.5])
    np.testing.assert_allclose(O.omega_scheme(O.TRANSITION, 0.5, 3, iter_n=1), [1, 1, 1])


# ---------------------------------------------------------------- general scaling (Section 7.4)
def test_one_sided_layer_membership():
    """Reading R1b: a layer within 1/3 of the high face holds the 27 cells of
    h = 1/81 whose centre exceeds 2/3; the low-face layer is its mirror image;
    a symmetric width w is the pair (w, w); layers covering the axis rotate
    every cell."""
    rot = O.rotated_cells(4, (0.0, 1 / 3))
    assert rot.sum() == 27 and rot[54:].all() and not rot[:54].any()
    assert (O.rotated_cells(4, (1 / 3, 0.0)) == rot[::-1]).all()
    for lev, w in [(3, 4 / 27), (2, 0.2), (3, 0.5), (1, 0.1)]:
        assert (O.rotated_cells(lev, w) == O.rotated_cells(lev, (w, w))).all()
    assert O.rotated_cells(3, (0.4, 0.6)).all()
    h = O.axis_spacing(2, math.radians(30), (0.0, 1 / 3), 0.25)
    np.testing.assert_allclose(h[:6], np.exp(0.25j) / 9, rtol=1e-15)
    np.testing.assert_allclose(h[6:], np.exp(1j * math.radians(30)) / 9, rtol=1e-15)


@pytest.mark.parametrize("d,level", [(2, 2), (2, 3), (3, 2)])
def test_operator_kronecker_general_scaling(d, level):
    """Layer at the high face plus a rotated interior with a constant shift:
    the oracle's operator equals the separable form built from textbook 1D
    element matrices whose widths are taken straight from the definition
    (centre above 2/3: h e^{i 30deg}, else h e^{i theta_I})."""
    n = 3 ** level
    th_l, th_i, k2 = math.radians(30), 0.4, 45.0
    hs = np.array([np.exp(1j * (th_l if (i + 0.5) / n > 2 / 3 else th_i)) / n for i in range(n)])
    K, M = tri_1d(hs)
    H = -k2 * kron_all([M] * d)
    for j in range(d):
        H = H + kron_all([K if k == j else M for k in range(d)])
    A, _, _ = dense_level(d, level, np.full((n + 1,) * d, k2), th_l, (0.0, 1 / 3), th_i)
    np.testing.assert_allclose(A, H, rtol=0, atol=1e-13 * np.abs(H).max())


@pytest.mark.parametrize("d,level", [(2, 3), (3, 2)])
def test_sine_mode_eigenvalues_rotated_interior(d, level):
    """No layer and an interior rotation theta: every cell has width
    h e^{i theta}, so the Dirichlet sine modes are eigenvectors with the
    closed-form eigenvalue of the uniformly scaled grid."""
    n = 3 ** level
    k2 = (3 * math.pi) ** 2
    lev = O.Level(d, level, np.full((n + 1,) * d, k2), 1.2, 0.0, TH)
    hc = (1 / n) * complex(math.cos(TH), math.sin(TH))
    x = np.arange(n + 1) / n
    for modes in [(1,) * d, (2, 5, 1)[:d]]:
        s = np.ones((1,) * d)
        for ax, m in enumerate(modes):
            shape = [1] * d
            shape[ax] = n + 1
            s = s * np.sin(m * math.pi * x).reshape(shape)
        kap = [(2 / hc) * (1 - math.cos(m * math.pi / n)) for m in modes]
        mu = [(hc / 3) * (2 + math.cos(m * math.pi / n)) for m in modes]
        lam = -k2 * np.prod(mu)
        for j in range(d):
            lam += kap[j] * np.prod([mu[k] for k in range(d) if k != j])
        Hs = lev.apply(s.astype(np.complex128))
        inner = (slice(1, -1),) * d
        np.testing.assert_allclose(Hs[inner], lam * s[inner], rtol=1e-12, atol=1e-13 * abs(lam))


def test_high_face_layer_is_mirror_of_low_face_layer():
    """Reflecting x -> 1 - x and y -> 1 - y maps the operator with layers at
    the high faces onto the one with layers at the low faces (varying shift
    reflected too)."""
    rng = np.random.default_rng(7)
    n = 27
    k2 = rng.uniform(-30, 90, size=(n + 1, n + 1))
    u = rng.standard_normal((n + 1, n + 1)) + 1j * rng.standard_normal((n + 1, n + 1))
    O.zero_boundary(u)
    hi = O.Level(2, 3, k2, math.radians(30), (0.0, 1 / 3), 0.3)
    lo = O.Level(2, 3, k2[::-1, ::-1], math.radians(30), (1 / 3, 0.0), 0.3)
    np.testing.assert_allclose(hi.apply(u), lo.apply(u[::-1, ::-1])[::-1, ::-1], rtol=0, atol=1e-12)
    assert np.abs(hi.apply(u) - lo.apply(u)).max() > 1e-3


def _table2_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_regular.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            rows[int(line[0])] = [None if v == "div" else float(v) for v in line[1:]]
    return rows


def channel_inputs(theta_deg, depth=4):
    """Eq. 08-gaussian sampled at the vertices of h = 3^-depth (written out
    here, independent of the input generator module)."""
    n = 3 ** depth
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)  # [y, x]
    phi = 45.0 ** 2 + 135.0 ** 2 * (np.exp(-(15 * X) ** 2) + np.exp(-(15 * Y) ** 2))
    chi = np.exp(-(125 * X) ** 2 - (125 * Y) ** 2)
    return phi, chi


def table2_reduction(theta_deg, solver, iters=50):
    """Max-norm residual reduction of one Table 2 run (readings R1b and R6:
    two-phase Jacobi at theta = 0, omega = 0.4 for every Jacobi with a
    rotated interior, transition damping from 0.4, BPX with undamped coarse
    corrections of 0.4)."""
    phi, chi = channel_inputs(theta_deg)
    H = O.Hierarchy(2, 4, phi, math.radians(30), (0.0, 1 / 3), math.radians(theta_deg))
    H.set_rhs_nodal(chi)
    r0 = H.residual_max()
    w1 = 0.01 * (math.sqrt(3) - 1j)
    for it in range(1, iters + 1):
        if solver == "jacobi":
            w = (w1 if it % 2 else -np.conj(w1)) if theta_deg == 0 else 0.4
            H.cycle(O.omega_scheme(O.JACOBI, w, 4), O.ADD, O.DLINEAR)
        elif solver == "transition":
            H.cycle(O.omega_scheme(O.TRANSITION, 0.4, 4, iter_n=it), O.ADD, O.DLINEAR)
        else:
            H.cycle(O.omega_scheme(O.UCG, 0.4, 4), O.ADD, O.HIERARCHICAL)
    return H.residual_max() / r0


@pytest.mark.parametrize("theta_deg", [0, 18, 25, 35, 45])
def test_table2_regular_column(theta_deg):
    """Table 2, regular grid: every printed reduction is matched within a
    factor of 2 and every divergence (bottom symbol) diverges here too.  The
    setup leaves details open (cell shift, norm scaling), so the pin is an
    order-of-magnitude one; a layer at the wrong faces or an interior that is
    not rotated moves the entries by orders of magnitude or to divergence."""
    paper = _table2_golden()[theta_deg]
    for solver, ref in zip(["jacobi", "transition", "bpx"], paper):
        got = table2_reduction(theta_deg, solver)
        if ref is None:
            assert not (got < 1.0), (solver, got)
        else:
            assert abs(math.log10(got / ref)) <= math.log10(2.0), (solver, got, ref)


# ---------------------------------------------------------------- four dimensions (Section 7.1, p = 4)
def _sparse_kron_all(mats):
    import scipy.sparse as sp
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


def _sparse_operator(d, level, theta, w, k2, theta_interior=0.0):
    hs = O.axis_spacing(level, theta, w, theta_interior)
    K, M = tri_1d(hs)
    H = -k2 * _sparse_kron_all([M] * d)
    for j in range(d):
        H = H + _sparse_kron_all([K if k == j else M for k in range(d)])
    return H


def _inner(x, d):
    return x[(slice(1, -1),) * d].reshape(-1)


@pytest.mark.parametrize("level,w", [(1, 0.2), (2, 0.2), (2, 0.5)])
def test_operator_4d_equals_kronecker_of_1d_elements(level, w):
    """d = 4: the oracle's cell-by-cell operator applied to random vectors
    equals the separable Kronecker form of textbook 1D element matrices."""
    n = 3 ** level
    k2 = 17.0
    lev = O.Level(4, level, np.full((n + 1,) * 4, k2), TH, w)
    H = _sparse_operator(4, level, TH, w, k2)
    rng = np.random.default_rng(level)
    for _ in range(2):
        u = rng.standard_normal((n + 1,) * 4) + 1j * rng.standard_normal((n + 1,) * 4)
        O.zero_boundary(u)
        ref = H @ _inner(u, 4)
        np.testing.assert_allclose(_inner(lev.apply(u), 4), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_sine_mode_eigenvalues_4d():
    """d = 4, every cell rotated: Dirichlet sine modes are eigenvectors with
    the closed-form eigenvalue sum_j kappa_j prod_{k != j} mu_k - k^2 prod mu."""
    n, d = 9, 4
    k2 = (2 * math.pi) ** 2
    lev = O.Level(d, 2, np.full((n + 1,) * d, k2), TH, 0.5)
    hc = (1 / n) * complex(math.cos(TH), math.sin(TH))
    x = np.arange(n + 1) / n
    for modes in [(1, 1, 1, 1), (2, 1, 3, 8)]:
        s = np.ones((1,) * d)
        for ax, m in enumerate(modes):
            shape = [1] * d
            shape[ax] = n + 1
            s = s * np.sin(m * math.pi * x).reshape(shape)
        kap = [(2 / hc) * (1 - math.cos(m * math.pi / n)) for m in modes]
        mu = [(hc / 3) * (2 + math.cos(m * math.pi / n)) for m in modes]
        lam = -k2 * np.prod(mu)
        for j in range(d):
            lam += kap[j] * np.prod([mu[k] for k in range(d) if k != j])
        Hs = lev.apply(s.astype(np.complex128))
        inner = (slice(1, -1),) * d
        np.testing.assert_allclose(Hs[inner], lam * s[inner], rtol=1e-12, atol=1e-13 * abs(lam))


@pytest.mark.parametrize("variant,transfer", [(O.ADD, O.DLINEAR), (O.HB, O.DLINEAR), (O.ADD, O.HIERARCHICAL)])
def test_fas_cycle_4d_equals_additive_correction_scheme(variant, transfer):
    """d = 4, depth 2: Lemma 2 / Theorem 2 with sparse Kronecker operators and
    interpolation, as in the 2D/3D pin."""
    d, depth, k2 = 4, 2, 25.0
    Hh = _problem(d, depth, k2, TH, 0.5)
    omega = np.array([0.55 + 0.05j, 0.6])
    Hs = {lev: _sparse_operator(d, lev, TH, 0.5, k2) for lev in (1, 2)}
    P = _sparse_kron_all([interp_1d(3)] * d)
    u = _inner(Hh.u, d)
    b = _inner(Hh.b, d)
    r = b - Hs[2] @ u
    corr = np.zeros_like(u)
    for lev in (2, 1):
        rl = r if lev == 2 else P.T @ r
        du = omega[lev - 1] * rl / Hs[lev].diagonal()
        idx = list(itertools.product(range(1, 3 ** lev), repeat=d))
        cp = np.array([all(i % 3 == 0 for i in t) for t in idx])
        if variant == O.HB:
            du = np.where(cp, 0, du)
        if transfer == O.HIERARCHICAL and lev > 1:
            du = du - P @ du[cp]
        if lev == 1:
            du = P @ du
        corr += du
    Hh.cycle(omega, variant, transfer)
    got = _inner(Hh.u, d)
    np.testing.assert_allclose(got, u + corr, rtol=0, atol=1e-12 * np.abs(u + corr).max())


def test_poisson_analytic_discrete_solution_4d():
    """Section 7.1 in four dimensions: rhs 4 pi^2 prod sin(pi x_i), phi = 0;
    the discrete solution pi^2 (mu/kappa) prod sin(pi x_i) makes the
    residual vanish and the cycle converges to it."""
    d, depth = 4, 2
    n = 3 ** depth
    h = 1 / n
    x = np.arange(n + 1) / n
    s = np.ones((1,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n + 1
        s = s * np.sin(math.pi * x).reshape(shape)
    H = O.Hierarchy(d, depth, np.zeros((n + 1,) * d), 0.0, 0.0)
    H.set_rhs_nodal(d * math.pi ** 2 * s)
    kap = (2 / h) * (1 - math.cos(math.pi * h))
    mu = (h / 3) * (2 + math.cos(math.pi * h))
    exact = math.pi ** 2 * (mu / kap) * s
    np.testing.assert_allclose(H.residual(exact.astype(complex)), 0, atol=1e-12)
    om = O.omega_scheme(O.EXP, 0.8, depth)
    for _ in range(60):
        H.cycle(om, O.ADD, O.DLINEAR)
    np.testing.assert_allclose(H.u.real, exact, rtol=0, atol=1e-8)


def _sine_mode(d, n):
    x = np.arange(n + 1) / n
    s = np.ones((1,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n + 1
        s = s * np.sin(math.pi * x).reshape(shape)
    return s


def test_fmg_start_first_stage_is_one_jacobi_step_with_the_finest_factor():
    """FMG (Section 5 remark, Section 7.1): with one cycle per stage on a
    depth-2 Poisson problem, stage 1 is a single level, i.e. one damped
    Jacobi step from zero with the factor the finest level of the full
    hierarchy has (reading 9: level l of stage s takes omega[l - 1 + L - s]);
    its rhs is the closed-form 2D Q1 mass stencil h^2/36 [1 4 1]^2 applied to
    f sampled at the level-1 vertices, its diagonal the Q1 stiffness centre
    8/3.  The stage-2 start is P of that step.  Distinct factors per level
    catch a wrong factor slice; f sampled anywhere but at every third fine
    vertex changes b_1."""
    d, depth = 2, 2
    n = 3 ** depth
    f = d * math.pi ** 2 * _sine_mode(d, n)
    om = np.array([0.3, 0.7])
    hs = O.fmg_start(d, depth, np.zeros((n + 1,) * d), 0.0, 0.0, f.astype(complex), om, O.ADD, O.DLINEAR,
                     cycles_per_stage=1)
    h = 1 / 3
    f1 = f[::3, ::3]
    w = np.array([1.0, 4.0, 1.0])
    b1 = np.zeros((4, 4))
    for i in (1, 2):
        for j in (1, 2):
            b1[i, j] = h * h / 36 * sum(w[a] * w[b] * f1[i - 1 + a, j - 1 + b] for a in range(3) for b in range(3))
    u1 = om[1] * b1 / (8.0 / 3.0)
    np.testing.assert_allclose(hs.u, O.prolong(u1.astype(complex)), rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,depth", [(2, 4), (3, 3)])
def test_fmg_start_is_the_prolongated_discrete_solution_of_the_coarser_stage(d, depth):
    """FMG with every stage solved (Poisson, Section 7.1 rhs, theta = 0,
    phi = 0): the start handed to the finest stage is P applied to the
    discrete solution of level L - 1, which is pi^2 (mu / kappa) prod sin(pi x)
    at h = 3^-(L - 1) in 2D (mode (1,..,1) diagonalises K and M; the 3D
    analogue divides by the sum over axes).  A wrong stage count, a wrong f
    sampling or a missing prolongation moves the start by far more than the
    tolerance."""
    n = 3 ** depth
    f = d * math.pi ** 2 * _sine_mode(d, n)
    om = O.omega_scheme(O.UCG, 0.8 if d == 2 else 0.6, depth)
    hs = O.fmg_start(d, depth, np.zeros((n + 1,) * d), 0.0, 0.0, f.astype(complex), om, O.ADD,
                     O.HIERARCHICAL, cycles_per_stage=250)
    m = 3 ** (depth - 1)
    h = 1 / m
    kap = (2 / h) * (1 - math.cos(math.pi * h))
    mu = (h / 3) * (2 + math.cos(math.pi * h))
    # H s = d kappa mu^(d-1) s and M s = mu^d s for the sine mode s
    exact = d * math.pi ** 2 * mu ** d / (d * kap * mu ** (d - 1)) * _sine_mode(d, m)
    np.testing.assert_allclose(hs.u, O.prolong(exact.astype(complex)), rtol=0, atol=1e-9)


@pytest.mark.parametrize("variant,transfer", [(O.ADD, O.DLINEAR), (O.HB, O.DLINEAR),
                                              (O.ADD, O.HIERARCHICAL), (O.HB, O.HIERARCHICAL)])
@pytest.mark.parametrize("d,depth,varying", [(2, 3, False), (2, 3, True), (3, 2, True)])
def test_fas_cycle_equals_dense_fas_restatement_without_galerkin(variant, transfer, d, depth, varying):
    """Where rediscretisation is not the Galerkin product -- a layer edge inside
    coarse cells (w = 0.1) and, optionally, a varying shift -- the FAS cycle is
    not the correction scheme (Lemma 2 needs Galerkin), so it is pinned against
    Algorithm 4 restated with dense matrices on the interior unknowns: each
    level's operator from unit vectors, P from Kronecker products of 1D
    tripartite interpolation, R = P^T, I as the c-point selection, two
    cycles."""
    n = 3 ** depth
    rng = np.random.default_rng(21)
    k2 = rng.uniform(-30, 90, size=(n + 1,) * d) if varying else np.full((n + 1,) * d, 40.0)
    w = 0.1
    H = O.Hierarchy(d, depth, k2, TH, w)
    f = rng.standard_normal((n + 1,) * d) + 1j * rng.standard_normal((n + 1,) * d)
    u0 = rng.standard_normal((n + 1,) * d) + 1j * rng.standard_normal((n + 1,) * d)
    H.set_rhs_nodal(f)
    H.set_solution(u0)
    omega = np.array([0.5 - 0.03j, 0.6, 0.65 + 0.02j][:depth])
    A, idx, dg = {}, {}, {}
    for lev in range(1, depth + 1):
        stride = 3 ** (depth - lev)
        k2l = k2[(slice(None, None, stride),) * d]  # coarse levels sample k^2 at their vertices
        A[lev], idx[lev], _ = dense_level(d, lev, k2l, TH, w)
        dg[lev] = np.diag(A[lev])
    Ps = {lev: kron_all([interp_1d(3 ** (lev - 1))] * d) for lev in range(2, depth + 1)}
    cps = {lev: np.array([all(i % 3 == 0 for i in t) for t in idx[lev]]) for lev in range(1, depth + 1)}
    u = np.array([H.u[i] for i in idx[depth]])
    b = np.array([H.b[i] for i in idx[depth]])
    for _ in range(2):
        ul, bl, du = {depth: u}, {depth: b}, {}
        for lev in range(depth, 0, -1):
            r = bl[lev] - A[lev] @ ul[lev]
            du[lev] = omega[lev - 1] * r / dg[lev]
            if lev > 1:
                ul[lev - 1] = ul[lev][cps[lev]]
                uh = ul[lev] - Ps[lev] @ ul[lev - 1]
                bl[lev - 1] = Ps[lev].T @ (bl[lev] - A[lev] @ uh)
        corr = None
        for lev in range(1, depth + 1):
            t = du[lev]
            if variant == O.HB:
                t = np.where(cps[lev], 0, t)
            if transfer == O.HIERARCHICAL and lev > 1:
                t = t - Ps[lev] @ t[cps[lev]]
            corr = t if lev == 1 else t + Ps[lev] @ corr
        u = u + corr
        H.cycle(omega, variant, transfer)
        got = np.array([H.u[i] for i in idx[depth]])
        np.testing.assert_allclose(got, u, rtol=0, atol=1e-12 * np.abs(u).max())
