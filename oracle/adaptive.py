"""FP64 CPU oracle of the additive multilevel cycle on an adaptive spacetree
(Reps & Weinzierl, Section 4.3 and the hanging-vertex treatment of
Section 3).

TEST INFRASTRUCTURE ONLY, like ``oracle.helmholtz``: nothing in the product
path may import it; it shares no code with the CUDA library.

Grid.  Level 1 has all 3^d cells.  A level-l cell may be refined into 3^d
level-(l+1) children (the ``refine`` flags); the cells of level l + 1 are the
children of refined level-l cells.  A vertex of level l is *hanging* when not
all of its 2^d level-l cells exist; its value is the d-linear interpolation
from level l - 1 (P).  The other interior vertices of existing cells carry
unknowns.  Cells that exist and are not refined are *leaves*; the fine grid
is the union of the leaves of all levels, the discrete space the conforming
d-linear space on it (hanging values constrained by P).

Readings (also listed in the design notes):

A1  The cycle on an adaptive grid is the additive correction scheme on the
    hierarchical generating system {phi_(l,v): v unknown on level l}, the form
    Lemma 2 and Theorem 2 prove the FAS cycle equal to:
        du_(l,v) = omega_l (f - H u, phi_(l,v)) / H_l[v, v]
    followed by u += sum_l sum_v du_(l,v) phi_(l,v) with the hb mask and the
    BPX transfer (id - P I) as on regular grids.  Where the rediscretised
    level operators equal the Galerkin ones (invariant scaling and shift)
    this is the paper's FAS cycle; on a regular grid (every cell of levels
    1..L-1 refined) it reduces to the regular oracle.
A2  The generating-system residual (f - H u, phi_(l,v)) is evaluated level by
    level: the cell-wise residual b_c - H_c u of the level-l leaves around v
    (level-l element matrices, f sampled at level-l vertices) plus R applied
    to the level-(l+1) residual, which includes the partial residuals of
    hanging vertices (only their existing cells contribute).  This is the
    generating-system form of "b_(l-1) = R rhat_l" (Eq. HTMG) with the PDE
    right-hand side on leaves.
A3  State: u_l on the vertices of every level holds the fine-grid function's
    values there.  After a cycle each level adds its correction
    corr_l = T_l du_l + P corr_(l-1); then coarse values at vertices that
    carry an unknown on the next finer level are injected from it (Eq.
    injection, finest first), and hanging values equal P u_(l-1).
"""
from __future__ import annotations

import numpy as np

from .helmholtz import (ADD, DLINEAR, HB, HIERARCHICAL, Level, _corners, _slab, cells_per_axis, cpoint_mask,
                        inject, prolong, restrict, zero_boundary)


def child_cells(mask):
    """Existence mask of the children of the cells flagged in ``mask``
    (each cell splits into 3^d children along every axis)."""
    out = mask
    for ax in range(mask.ndim):
        out = np.repeat(out, 3, axis=ax)
    return out


def adjacent_count(cells):
    """Per vertex of the level grid: how many of its 2^d cells exist."""
    d = cells.ndim
    n = cells.shape[0]
    cnt = np.zeros((n + 1,) * d, dtype=np.int64)
    for a in _corners(d):
        cnt[_slab((n,) * d, a)] += cells
    return cnt


class AdaptiveHierarchy:
    """Levels 1..L of an adaptive spacetree with the per-level state u_l.

    ``refine[l]`` (l = 1..L-1) flags the level-l cells to refine; flags of
    cells that do not exist are ignored.  k2 and f are given at the vertices
    of the uniform level-L grid and sampled (injection) on every level.
    """

    def __init__(self, d, depth, k2_fine, theta, layer_width, refine, theta_interior=0.0):
        self.d, self.L = d, depth
        k2 = np.asarray(k2_fine, dtype=np.float64)
        self.k2 = {depth: k2}
        for lev in range(depth - 1, 0, -1):
            self.k2[lev] = inject(self.k2[lev + 1])
        self.levels = {lev: Level(d, lev, self.k2[lev], theta, layer_width, theta_interior)
                       for lev in range(1, depth + 1)}
        self.cells = {1: np.ones((3,) * d, dtype=bool)}
        self.refined = {}
        for lev in range(1, depth):
            flags = np.asarray(refine[lev], dtype=bool) & self.cells[lev]
            self.refined[lev] = flags
            self.cells[lev + 1] = child_cells(flags)
        self.refined[depth] = np.zeros_like(self.cells[depth])
        self.leaf = {lev: self.cells[lev] & ~self.refined[lev] for lev in range(1, depth + 1)}
        self.unknown = {}
        self.exists = {}
        for lev in range(1, depth + 1):
            cnt = adjacent_count(self.cells[lev])
            inner = np.zeros_like(cnt, dtype=bool)
            inner[(slice(1, -1),) * d] = True
            self.exists[lev] = cnt > 0
            self.unknown[lev] = inner & (cnt == 2 ** d)
        n = cells_per_axis(depth)
        self.u = {lev: np.zeros((cells_per_axis(lev) + 1,) * d, dtype=np.complex128)
                  for lev in range(1, depth + 1)}
        self.f = {lev: np.zeros_like(self.u[lev]) for lev in self.u}
        self.r0 = None
        assert k2.shape == (n + 1,) * d

    # -- state
    def set_rhs_nodal(self, f):
        f = np.asarray(f, dtype=np.complex128)
        self.f = {self.L: f.copy()}
        for lev in range(self.L - 1, 0, -1):
            self.f[lev] = inject(self.f[lev + 1])
        self.r0 = None

    def set_solution_levels(self, u_by_level):
        """Sets u_l on every level and restores the invariants of A3."""
        for lev in range(1, self.L + 1):
            self.u[lev] = np.asarray(u_by_level[lev], dtype=np.complex128).copy()
            zero_boundary(self.u[lev])
        self._restore_invariants()
        self.r0 = None

    def _restore_invariants(self):
        # hanging values from the coarser level, coarse to fine
        for lev in range(2, self.L + 1):
            hang = self.exists[lev] & ~self.unknown[lev]
            p = prolong(self.u[lev - 1])
            self.u[lev][hang] = p[hang]
            zero_boundary(self.u[lev])
        # injection of values that carry an unknown on the finer level
        for lev in range(self.L - 1, 0, -1):
            fine_unknown = self.unknown[lev + 1][(slice(None, None, 3),) * self.d]
            self.u[lev][fine_unknown] = inject(self.u[lev + 1])[fine_unknown]

    # -- residuals
    def _leaf_residual(self, lev):
        """sum over the level-lev leaves around each vertex of b_c - H_c u
        (cell-wise element matrices, Section 3 / Appendix B)."""
        op = self.levels[lev]
        d, n = self.d, op.n
        cs = (n,) * d
        mask = self.leaf[lev].astype(np.float64)
        u, f = self.u[lev], self.f[lev]
        out = np.zeros((n + 1,) * d, dtype=np.complex128)
        for a in _corners(d):
            acc = np.zeros(cs, dtype=np.complex128)
            for b in _corners(d):
                acc += op.cell_entry(a, b, with_phi=False) * f[_slab(cs, b)]
                acc -= op.cell_entry(a, b) * u[_slab(cs, b)]
            out[_slab(cs, a)] += mask * acc
        return out

    def level_residuals(self):
        """Generating-system residuals r_l (reading A2), finest level first;
        entries outside the vertices of existing cells are zero."""
        r = {}
        below = None
        for lev in range(self.L, 0, -1):
            rl = self._leaf_residual(lev)
            if below is not None:
                rl = rl + restrict(below)
            rl = np.where(self.exists[lev], rl, 0)
            zero_boundary(rl)
            r[lev] = rl
            below = rl
        return r

    def residual_norm(self):
        """Euclidean norm of the residuals of all unknowns of the fine grid
        (the leaf-level unknowns: vertices carrying an unknown on their level
        but not on the next finer one) and its ratio to the starting one."""
        r = self.level_residuals()
        tot = 0.0
        for lev in range(1, self.L + 1):
            own = self.unknown[lev].copy()
            if lev < self.L:
                own &= ~self.unknown[lev + 1][(slice(None, None, 3),) * self.d]
            tot += float(np.sum(np.abs(r[lev][own]) ** 2))
        nrm = np.sqrt(tot)
        if self.r0 is None:
            self.r0 = nrm
        return nrm, (nrm / self.r0 if self.r0 > 0 else 0.0)

    # -- the cycle
    def cycle(self, omega, variant=ADD, transfer=DLINEAR):
        """One additive cycle (reading A1): residuals of every level (A2),
        damped Jacobi at the unknowns, the hb mask or BPX transfer, the
        corrections coarse to fine, and the update of every level (A3)."""
        L, d = self.L, self.d
        omega = np.asarray(omega, dtype=np.complex128)
        r = self.level_residuals()
        corr = None
        corrs = {}
        for lev in range(1, L + 1):
            op = self.levels[lev]
            t = np.zeros_like(r[lev])
            m = self.unknown[lev]
            t[m] = omega[lev - 1] * r[lev][m] / op.diag[m]
            if variant == HB:
                t = np.where(cpoint_mask(d, lev), 0, t)
            if transfer == HIERARCHICAL:
                t = t - prolong(inject(t))
            corr = t if lev == 1 else t + prolong(corr)
            corrs[lev] = corr
        for lev in range(1, L + 1):
            self.u[lev] = self.u[lev] + corrs[lev]
            zero_boundary(self.u[lev])
        self._restore_invariants()

    def composite_on_fine(self):
        """The fine-grid function sampled on the uniform level-L grid: on each
        leaf cell the d-linear interpolant of its level's corner values."""
        out = self.u[1].copy()
        for lev in range(2, self.L + 1):
            out = prolong(out)
            m = self.exists[lev]
            out[m] = self.u[lev][m]  # vertices of existing level-lev cells
        return out
