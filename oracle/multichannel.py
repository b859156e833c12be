"""Plain FP64 CPU oracle of the coupled multichannel cycle (Section 7.5).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or helper with the CUDA library.

Section 7.5 fuses c channels of Eq. coupledHelmholtz into one grid: every
vertex carries a C^c tuple, and the coupled multichannel variant keeps the
off-diagonal blocks A_ij inside a block of the operator (the matrix A-hat of
that section).  This file restates the additive cycle of helmholtz.py for such
tuples.  Readings (each is also listed in the design notes):

M1  Operator.  (A u)_i = H_ii u_i + sum_{j != i} A_ij u_j with
    H_ii = K - phi_i M (the single-channel operator of Section 4 with the
    channel's own constant shift) and A_ij = -kappa_ij M: the coupling blocks
    "contain potential terms", read as a constant coupling potential times
    the complex-scaled mass matrix.  Collected in a c x c matrix Phi
    (phi_i on the diagonal, kappa_ij off it): A = I (x) K - Phi (x) M.
    Phi is the same on every level (constant coefficients).
M2  Smoother.  Damped block Jacobi: du_v = omega_l D_v^{-1} r_v with
    D_v = K_vv I - Phi M_vv, the c x c diagonal block of A at vertex v.
M3  Cycle.  Appendix A Algorithm 4 with tuple unknowns: restriction,
    prolongation, injection, the hb mask and the BPX transfer act on every
    channel alike; the coarse right-hand side is R(b - A uhat).

K and M come from helmholtz.Level (the single-channel operator is pinned on
its own); everything channel-related is written out here.
"""
from __future__ import annotations

import numpy as np

from .helmholtz import (ADD, DLINEAR, HB, HIERARCHICAL, Level, _corners, _slab, cpoint_mask, inject,
                        prolong, restrict, zero_boundary)


class MultiLevel:
    """K, M and the c x c diagonal blocks of the coupled operator on one
    regular level."""

    def __init__(self, d, level, Phi, theta, layer_width):
        self.d, self.level = d, level
        self.n = 3 ** level
        self.Phi = np.asarray(Phi, dtype=np.complex128)
        self.c = self.Phi.shape[0]
        zero = np.zeros((self.n + 1,) * d)
        self.lev = Level(d, level, zero, theta, layer_width)  # zero shift: its operator is K
        self.kdiag = self.lev.diag
        mdiag = np.zeros((self.n + 1,) * d, dtype=np.complex128)
        for a in _corners(d):
            mdiag[_slab((self.n,) * d, a)] += self.lev.cell_entry(a, a, with_phi=False)
        self.mdiag = mdiag
        # D_v = K_vv I - Phi M_vv, as an array of c x c matrices over the vertices
        eye = np.eye(self.c, dtype=np.complex128)
        self.D = (self.kdiag[..., None, None] * eye - self.mdiag[..., None, None] * self.Phi)

    def K(self, x):
        return self.lev.apply(x)

    def M(self, x):
        return self.lev.mass(x)

    def apply(self, U):
        """(A U)_i = K U_i - sum_j Phi_ij M U_j; U has shape (c, N, .., N)."""
        KU = np.array([self.K(U[i]) for i in range(self.c)])
        MU = np.array([self.M(U[j]) for j in range(self.c)])
        return KU - np.einsum("ij,j...->i...", self.Phi, MU)

    def block_jacobi(self, R, omega):
        """omega D_v^{-1} r_v at every interior vertex (zero on the boundary)."""
        d = self.d
        out = np.zeros_like(R)
        inner = (slice(1, -1),) * d
        Dv = self.D[inner]                                   # (N-2, .., c, c)
        rv = np.moveaxis(R[(slice(None),) + inner], 0, -1)   # (N-2, .., c)
        sol = np.linalg.solve(Dv, rv[..., None])[..., 0]
        out[(slice(None),) + inner] = omega * np.moveaxis(sol, -1, 0)
        return out


def _each(f, U):
    return np.array([f(U[i]) for i in range(U.shape[0])])


class MultiHierarchy:
    """Regular levels 1..L of the coupled c-channel problem."""

    def __init__(self, d, depth, Phi, theta, layer_width):
        self.d, self.L = d, depth
        self.Phi = np.asarray(Phi, dtype=np.complex128)
        self.c = self.Phi.shape[0]
        self.levels = {lev: MultiLevel(d, lev, self.Phi, theta, layer_width) for lev in range(1, depth + 1)}
        shape = (self.c,) + (3 ** depth + 1,) * d
        self.u = np.zeros(shape, dtype=np.complex128)
        self.b = np.zeros_like(self.u)
        self.r0 = None

    def set_rhs_nodal(self, F):
        """b_L = M f channel by channel (F: (c, N, .., N) nodal values)."""
        F = np.asarray(F, dtype=np.complex128)
        self.b = _each(self.levels[self.L].M, F)
        self.r0 = None

    def set_solution(self, U):
        U = np.array(U, dtype=np.complex128)
        for i in range(self.c):
            zero_boundary(U[i])
        self.u = U
        self.r0 = None

    def residual(self, U=None):
        U = self.u if U is None else U
        R = self.b - self.levels[self.L].apply(U)
        for i in range(self.c):
            zero_boundary(R[i])
        return R

    def residual_norm(self):
        r = np.linalg.norm(self.residual().ravel())
        if self.r0 is None:
            self.r0 = r
        return r, (r / self.r0 if self.r0 > 0 else 0.0)

    def cycle(self, omega, variant=ADD, transfer=DLINEAR):
        """One additive FAS cycle (Algorithm 4) on c-channel tuples with the
        damped block-Jacobi smoother of reading M2."""
        L, d = self.L, self.d
        omega = np.asarray(omega, dtype=np.complex128)
        assert omega.shape == (L,)
        u = {L: self.u}
        b = {L: self.b}
        du = {}
        for lev in range(L, 0, -1):
            op = self.levels[lev]
            r = b[lev] - op.apply(u[lev])
            du[lev] = op.block_jacobi(r, omega[lev - 1])
            if lev > 1:
                u[lev - 1] = _each(inject, u[lev])
                uhat = u[lev] - _each(prolong, u[lev - 1])
                rhat = b[lev] - op.apply(uhat)
                b[lev - 1] = _each(lambda x: zero_boundary(restrict(x)), rhat)
        corr = None
        for lev in range(1, L + 1):
            t = du[lev]
            if variant == HB:
                t = np.where(cpoint_mask(d, lev)[None], 0, t)
            if transfer == HIERARCHICAL:
                t = t - _each(lambda x: prolong(inject(x)), t)
            corr = t if lev == 1 else t + _each(prolong, corr)
        self.u = self.u + corr
        for i in range(self.c):
            zero_boundary(self.u[i])
        return self.u
