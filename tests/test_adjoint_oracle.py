"""Pins of the oracle's dense adjoint: its gradients of J = |s|^2 equal
central finite differences of J computed with dense direct solves (the
definition of the derivative), for V and f, in 2D and 3D, including
vertices on the Dirichlet ring (they enter through cell shifts and the
mass rhs)."""
import math

import numpy as np
import pytest

import oracle.adjoint as A
import oracle as O
from paper_1508_03954_gb300 import workloads as W


def _setup(d, depth, seed):
    rng = np.random.default_rng(seed)
    n = 3 ** depth
    V = rng.uniform(0.0, 10.0, size=(n + 1,) * d)
    f = rng.uniform(-1.0, 1.0, size=(n + 1,) * d)
    if d == 2:
        xyz, g = W.circle_samples(64)
    else:
        xyz2, g = W.circle_samples(32)
        xyz = np.concatenate([xyz2, np.full((len(g), 1), 0.45)], axis=1)
    return V, f, xyz, g


@pytest.mark.parametrize("d,depth,E", [(2, 2, 30.0), (2, 2, -50.0), (3, 1, 20.0)])
def test_dense_adjoint_matches_central_differences(d, depth, E):
    V, f, xyz, g = _setup(d, depth, 3)
    th, w = math.pi / 6, 0.2
    G = A.adjoint_gradients(d, depth, E, V, th, w, f, xyz, g)
    rng = np.random.default_rng(9)
    n = 3 ** depth
    picks = [tuple(rng.integers(0, n + 1, size=d)) for _ in range(6)] + [(1,) * d, (0,) * d]
    for idx in picks:
        fdV = A.central_difference(d, depth, E, V, th, w, f, xyz, g, "V", idx, 1e-4)
        fdf = A.central_difference(d, depth, E, V, th, w, f, xyz, g, "f", idx, 1e-4)
        scale = max(abs(G["dJdV"]).max(), 1e-300)
        assert abs(G["dJdV"][idx] - fdV) <= 1e-6 * scale, (idx, G["dJdV"][idx], fdV)
        scale = max(abs(G["dJdf"]).max(), 1e-300)
        assert abs(G["dJdf"][idx] - fdf) <= 1e-6 * scale, (idx, G["dJdf"][idx], fdf)


def test_operator_is_complex_symmetric_so_adjoint_is_a_forward_solve():
    V, f, xyz, g = _setup(2, 2, 4)
    P = A.DenseProblem(2, 2, 30.0, V, math.pi / 6, 0.2)
    np.testing.assert_allclose(P.H, P.H.T, rtol=0, atol=1e-13 * abs(P.H).max())


def test_sample_vector_reproduces_interpolation_of_linear_fields():
    depth, d = 3, 2
    n = 3 ** depth
    x = np.arange(n + 1) / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    u = (2 * X - 3 * Y + 5 * X * Y).astype(complex)
    O.zero_boundary(u)
    xyz, g = W.circle_samples(40, radius=0.3)
    a = A.sample_vector(d, depth, xyz, g)
    exact = np.sum(g * (2 * xyz[:, 0] - 3 * xyz[:, 1] + 5 * xyz[:, 0] * xyz[:, 1]))
    assert abs(np.sum(a * u) - exact) <= 1e-12 * abs(exact)
