"""Dense FP64 adjoint of the far-field functional (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/helmholtz.py).

Forward problem: H(V) u = b with b = M f (consistent mass, reading R3),
k^2 = E - V per vertex (a cell uses the mean of its vertex values, reading
R2).  Functional: s = sum_q w_q u(x_q) with d-linear interpolation of the
fine vertex values, J = |s|^2.  The paper has no adjoint; this module
computes derivatives from the definition:
  * the adjoint lambda solves H^T lambda = a with the explicit transpose of
    the dense operator (no symmetry is assumed);
  * dH/dV_v is obtained from the oracle's own cell-wise assembly as the
    difference H(V + e_v) - H(V), which is exact because H is affine in V;
  * db/df_v is M e_v from the oracle's mass product.
Parity beyond the finite-difference pins in tests/ is not fixed by the
paper (its methods section has no adjoint).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .helmholtz import Level, cells_per_axis


def sample_vector(d, depth, xyz, w):
    """a with s = a . u: a_v = sum_q w_q psi_v(x_q) over the vertex array
    (numpy axis order, last axis = x), d-linear nodal basis psi_v."""
    n = cells_per_axis(depth)
    a = np.zeros((n + 1,) * d, dtype=np.complex128)
    for p in range(len(w)):
        x = xyz[p]
        idx, frac = [], []
        for ax in range(d):        # coordinate ax (x = 0) lives on numpy axis d-1-ax
            t = x[ax] * n
            k = min(max(int(math.floor(t)), 0), n - 1)
            idx.append(k)
            frac.append(t - k)
        for bits in itertools.product((0, 1), repeat=d):
            wt = 1.0
            pos = [0] * d
            for ax in range(d):
                wt *= frac[ax] if bits[ax] else 1.0 - frac[ax]
                pos[d - 1 - ax] = idx[ax] + bits[ax]
            a[tuple(pos)] += wt * w[p]
    inner = np.zeros_like(a)
    sl = (slice(1, -1),) * d
    inner[sl] = a[sl]          # Dirichlet vertices carry no unknowns
    return inner


class DenseProblem:
    """Dense interior operator H(V) and mass M of the fine level."""

    def __init__(self, d, depth, E, V, theta, layer_width):
        self.d, self.depth = d, depth
        self.E, self.theta, self.w = E, theta, layer_width
        self.V = np.asarray(V, dtype=np.float64)
        self.n = cells_per_axis(depth)
        self.inner = list(itertools.product(range(1, self.n), repeat=d))
        self.lev = Level(d, depth, E - self.V, theta, layer_width)
        self.H = self._dense(self.lev, with_phi=True)

    def _dense(self, lev, with_phi):
        n, d = self.n, self.d
        A = np.zeros((len(self.inner), len(self.inner)), dtype=np.complex128)
        for j, idx in enumerate(self.inner):
            e = np.zeros((n + 1,) * d, dtype=np.complex128)
            e[idx] = 1
            col = lev.apply(e, with_phi)
            A[:, j] = [col[i] for i in self.inner]
        return A

    def gather(self, x):
        return np.array([x[i] for i in self.inner])

    def scatter(self, v):
        out = np.zeros((self.n + 1,) * self.d, dtype=np.complex128)
        for k, i in enumerate(self.inner):
            out[i] = v[k]
        return out

    def solve(self, b_full):
        return self.scatter(np.linalg.solve(self.H, self.gather(b_full)))

    def rhs(self, f):
        return self.lev.mass(np.asarray(f, dtype=np.complex128))


def objective(d, depth, E, V, theta, w, f, xyz, g):
    """J = |s|^2 with dense solves; returns (J, s, u, b)."""
    P = DenseProblem(d, depth, E, V, theta, w)
    b = P.rhs(f)
    u = P.solve(b)
    a = sample_vector(d, depth, xyz, g)
    s = np.sum(a * u)
    return abs(s) ** 2, s, u, P


def adjoint_gradients(d, depth, E, V, theta, w, f, xyz, g):
    """dJ/dV and dJ/df at every fine vertex (real V, real f) by the dense
    adjoint: lambda = H^{-T} a; ds/dp = lambda^T (db/dp - (dH/dp) u)."""
    J, s, u, P = objective(d, depth, E, V, theta, w, f, xyz, g)
    a = sample_vector(d, depth, xyz, g)
    lam = P.scatter(np.linalg.solve(P.H.T, P.gather(a)))
    n = P.n
    shape = (n + 1,) * d
    dV = np.zeros(shape)
    df = np.zeros(shape)
    base_Hu = P.lev.apply(u)
    for idx in itertools.product(range(n + 1), repeat=d):
        e = np.zeros(shape)
        e[idx] = 1.0
        # H is affine in V: H(V + e_v) u - H(V) u = (dH/dV_v) u exactly
        dHu = Level(d, depth, E - (P.V + e), theta, w).apply(u) - base_Hu
        ds_dV = -np.sum(lam * dHu)
        dV[idx] = 2.0 * np.real(np.conj(s) * ds_dV)
        db = P.lev.mass(e.astype(np.complex128))
        ds_df = np.sum(lam * db)
        df[idx] = 2.0 * np.real(np.conj(s) * ds_df)
    return dict(J=J, s=s, u=u, lam=lam, dJdV=dV, dJdf=df)


def central_difference(d, depth, E, V, theta, w, f, xyz, g, which, idx, h):
    """(J(p + h e) - J(p - h e)) / (2h) for p = V or f at vertex idx."""
    V = np.asarray(V, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    e = np.zeros_like(V)
    e[idx] = 1.0
    if which == "V":
        jp = objective(d, depth, E, V + h * e, theta, w, f, xyz, g)[0]
        jm = objective(d, depth, E, V - h * e, theta, w, f, xyz, g)[0]
    else:
        jp = objective(d, depth, E, V, theta, w, f + h * e, xyz, g)[0]
        jm = objective(d, depth, E, V, theta, w, f - h * e, xyz, g)[0]
    return (jp - jm) / (2.0 * h)
