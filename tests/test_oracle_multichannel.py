"""Pins of the coupled multichannel oracle (Section 7.5, readings M1-M3)
against routes independent of its own channel arithmetic:

* one channel, and uncoupled channels, reduce to the single-channel oracle
  (pinned on its own) run channel by channel;
* a real symmetric coupling matrix Phi = Q Lambda Q^T decouples: A = I (x) K
  - Phi (x) M is similar to I (x) K - Lambda (x) M, the block-Jacobi blocks
  transform the same way and the transfers act channel-wise, so the coupled
  cycle equals Q times independent single-channel cycles with shifts lambda_i
  on the rotated data;
* Dirichlet sine modes: A (x (x) s) = (kappa_s I - mu_s Phi) x (x) s with the
  closed-form K and M eigenvalues of the mode, for any complex Phi;
* the operator equals the dense Kronecker form built from textbook 1D
  element matrices, and a convergent setup's fixed point is the dense
  solution;
* one level: damped block Jacobi with the closed-form Q1 diagonal blocks.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.multichannel import MultiHierarchy, MultiLevel

TH = math.pi / 6


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _single(d, depth, phi, th, w, F_i, U_i):
    n = 3 ** depth
    h = O.Hierarchy(d, depth, np.full((n + 1,) * d, phi), th, w)
    h.set_rhs_nodal(F_i)
    h.set_solution(U_i)
    return h


VARS = [(O.ADD, O.DLINEAR), (O.HB, O.DLINEAR), (O.ADD, O.HIERARCHICAL), (O.HB, O.HIERARCHICAL)]


@pytest.mark.parametrize("var", VARS, ids=["add", "hb", "bpx", "hb-hier"])
@pytest.mark.parametrize("d,depth,w", [(2, 3, 0.2), (3, 2, 0.2)])
def test_uncoupled_channels_are_single_channel_cycles(var, d, depth, w):
    phis = np.array([-30.0, 12.0, 55.0])
    c = len(phis)
    n = 3 ** depth
    F = _rand((c,) + (n + 1,) * d, 1)
    U = _rand((c,) + (n + 1,) * d, 2)
    mh = MultiHierarchy(d, depth, np.diag(phis), TH, w)
    mh.set_rhs_nodal(F)
    mh.set_solution(U)
    singles = [_single(d, depth, phis[i], TH, w, F[i], U[i]) for i in range(c)]
    om = np.array([0.5, 0.6, 0.7][:depth])
    for _ in range(3):
        mh.cycle(om, *var)
        for i in range(c):
            singles[i].cycle(om, *var)
    for i in range(c):
        np.testing.assert_allclose(mh.u[i], singles[i].u, rtol=0, atol=1e-13 * np.abs(singles[i].u).max())


@pytest.mark.parametrize("var", VARS, ids=["add", "hb", "bpx", "hb-hier"])
@pytest.mark.parametrize("d,depth,w", [(2, 3, 0.2), (3, 2, 0.5)])
def test_symmetric_coupling_decouples_in_its_eigenbasis(var, d, depth, w):
    rng = np.random.default_rng(3)
    c = 4
    S = rng.uniform(-20, 20, size=(c, c))
    Phi = (S + S.T) / 2 + np.diag([-40.0, -10.0, 15.0, 35.0])
    lam, Q = np.linalg.eigh(Phi)
    n = 3 ** depth
    F = _rand((c,) + (n + 1,) * d, 4)
    U = _rand((c,) + (n + 1,) * d, 5)
    mh = MultiHierarchy(d, depth, Phi, TH, w)
    mh.set_rhs_nodal(F)
    mh.set_solution(U)
    Fr = np.einsum("ji,j...->i...", Q, F)  # Q^T F
    Ur = np.einsum("ji,j...->i...", Q, U)
    singles = [_single(d, depth, lam[i], TH, w, Fr[i], Ur[i]) for i in range(c)]
    om = np.array([0.55, 0.6 + 0.05j, 0.65][:depth])
    for _ in range(2):
        mh.cycle(om, *var)
        for i in range(c):
            singles[i].cycle(om, *var)
    back = np.einsum("ij,j...->i...", Q, np.array([s.u for s in singles]))
    np.testing.assert_allclose(mh.u, back, rtol=0, atol=1e-12 * np.abs(back).max())


@pytest.mark.parametrize("d,w", [(2, 0.0), (2, 0.5), (3, 0.5)])
def test_sine_modes_are_eigenvectors_of_the_coupled_operator(d, w):
    level = 2
    n = 3 ** level
    hc = (1.0 / n) * (complex(math.cos(TH), math.sin(TH)) if w >= 0.5 else 1.0)
    rng = np.random.default_rng(6)
    c = 3
    Phi = rng.standard_normal((c, c)) * 20 + 1j * rng.standard_normal((c, c)) * 5
    lev = MultiLevel(d, level, Phi, TH, w)
    x = rng.standard_normal(c) + 1j * rng.standard_normal(c)
    for modes in [(1,) * d, (2, 5, 3)[:d], (7, 1, 4)[:d]]:
        s = np.ones((1,) * d)
        kap, mu = [], []
        for ax, m in enumerate(modes):
            shape = [1] * d
            shape[ax] = n + 1
            s = s * np.sin(math.pi * m * np.arange(n + 1) / n).reshape(shape)
            kap.append((2 / hc) * (1 - math.cos(math.pi * m / n)))
            mu.append((hc / 3) * (2 + math.cos(math.pi * m / n)))
        lk = sum(kap[j] * np.prod([mu[a] for a in range(d) if a != j]) for j in range(d))
        lm = np.prod(mu)
        U = np.array([x[i] * s for i in range(c)])
        got = lev.apply(U)
        want = np.einsum("ij,j...->i...", lk * np.eye(c) - lm * Phi, U)
        inner = (slice(None),) + (slice(1, -1),) * d
        np.testing.assert_allclose(got[inner], want[inner], rtol=0, atol=1e-12 * np.abs(want).max())


def _tri_1d(hs):
    n = len(hs)
    K = np.zeros((n + 1, n + 1), dtype=np.complex128)
    M = np.zeros_like(K)
    for i, h in enumerate(hs):
        K[i:i + 2, i:i + 2] += np.array([[1, -1], [-1, 1]]) / h
        M[i:i + 2, i:i + 2] += np.array([[2, 1], [1, 2]]) * h / 6
    return K[1:-1, 1:-1], M[1:-1, 1:-1]


def _dense(d, level, Phi, th, w):
    """I (x) K - Phi (x) M on interior unknowns (channel slowest, x fastest),
    from textbook 1D element matrices with the per-cell widths."""
    K1, M1 = _tri_1d(O.axis_spacing(level, th, w))

    def kron_all(ms):
        out = ms[0]
        for m in ms[1:]:
            out = np.kron(out, m)
        return out
    K = sum(kron_all([K1 if k == j else M1 for k in range(d)]) for j in range(d))
    M = kron_all([M1] * d)
    c = Phi.shape[0]
    return np.kron(np.eye(c), K) - np.kron(Phi, M)


def _interior(U, d):
    return U[(slice(None),) + (slice(1, -1),) * d].reshape(U.shape[0], -1)


def test_operator_equals_dense_kronecker_form():
    d, level, w = 2, 2, 0.2
    rng = np.random.default_rng(7)
    c = 3
    Phi = rng.standard_normal((c, c)) * 10 + 1j * rng.standard_normal((c, c))
    lev = MultiLevel(d, level, Phi, TH, w)
    n = 3 ** level
    U = _rand((c,) + (n + 1,) * d, 8)
    for i in range(c):
        O.zero_boundary(U[i])
    A = _dense(d, level, Phi, TH, w)
    np.testing.assert_allclose(_interior(lev.apply(U), d).ravel(), A @ _interior(U, d).ravel(),
                               rtol=0, atol=1e-12 * np.abs(A).max())


def test_fixed_point_is_the_dense_solution():
    """No layer (theta = 0), a negative definite symmetric Phi: A is real
    symmetric positive definite and the BPX cycle converges to A^{-1} b."""
    d, depth = 2, 2
    Phi = -np.array([[40.0, 8.0, 2.0], [8.0, 30.0, 5.0], [2.0, 5.0, 60.0]])
    c = Phi.shape[0]
    n = 3 ** depth
    mh = MultiHierarchy(d, depth, Phi, 0.0, 0.0)
    F = _rand((c,) + (n + 1,) * d, 9)
    mh.set_rhs_nodal(F)
    A = _dense(d, depth, Phi, 0.0, 0.0)
    x = np.linalg.solve(A, _interior(mh.b, d).ravel())
    for _ in range(400):
        mh.cycle(np.array([0.6, 0.6]), O.ADD, O.HIERARCHICAL)
    np.testing.assert_allclose(_interior(mh.u, d).ravel(), x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_single_level_is_damped_block_jacobi_with_closed_form_blocks():
    """Level 1 alone (4 x 4 vertices, h = 1/3, no layer): D_v = (8/3) I -
    Phi (16 h^2 / 36) (the 2D Q1 stiffness and mass centres) at every
    interior vertex, and one cycle from zero gives omega D^{-1} b."""
    d, h = 2, 1 / 3
    Phi = np.array([[10.0, 3.0 + 1j], [3.0 - 2j, -5.0]])
    mh = MultiHierarchy(d, 1, Phi, 0.0, 0.0)
    F = _rand((2, 4, 4), 10)
    mh.set_rhs_nodal(F)
    om = 0.7 + 0.1j
    mh.cycle(np.array([om]), O.ADD, O.DLINEAR)
    D = (8 / 3) * np.eye(2) - Phi * (16 * h * h / 36)
    for v in [(1, 1), (1, 2), (2, 1), (2, 2)]:
        want = om * np.linalg.solve(D, mh.b[(slice(None),) + v])
        np.testing.assert_allclose(mh.u[(slice(None),) + v], want, rtol=1e-14, atol=0)
