"""FP64 CPU oracle of the additive multilevel cycle on an adaptive spacetree
(Reps & Weinzierl: the adaptive Cartesian grids of Section 3, hanging
vertices and FAS injection of Section 4), with the per-vertex relaxation
factors of Section 5.1 and the feature-based dynamic refinement of Section
5.3.

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
A4  Relaxation factors are per vertex (the Section 5.1 table):
    omega(v) = omega[L - 1 - succ(v)], so the per-level array of the regular
    grid (indexed by the distance L - l to the finest level, which is
    succ(v) there) is read as a table over succ.  succ(v) = 0 unless all 2^d
    cells of v's level around v are refined (a refined vertex); then it is
    1 + the minimum over v's children: the vertices of the next finer level
    with a cell whose parent is one of v's cells (offsets -3..3 from 3v along
    every axis), counting those that carry an unknown (Dirichlet and hanging
    vertices hold no unknown and no succ).
A5  Refinement indicator: s(v) = max over the axes of the undivided second
    difference |u(v - e) - 2 u(v) + u(v + e)| on v's own level, at the
    fine-grid vertices (unknowns with no unknown at the same point on the
    next finer level: the unknowns of the fine grid).
A6  Selection: the span [min s, max s] over all fine-grid vertices is split
    into `bins` equal subranges (bin = floor((s - min) / (max - min) bins),
    the top value in the last bin).  Refinement takes the k top bins, k the
    smallest count whose vertex total is closest to refine_frac times the
    number of fine-grid vertices; erasing the k' bottom bins for erase_frac
    (a vertex in both sets is refined).  Both are vetoed where
    |r(v) / H_l[v, v]| > veto (r the generating-system residual of A2), or,
    read relative to the vertex's value, where |r(v) / H_l[v, v]| >
    veto |u(v)| (an update above that fraction of the value is a major one).
A7  Refining a vertex refines its 2^d cells (it becomes a refined vertex);
    vertices on the finest admissible level (h_min) are not refined.
    Erasing acts on the cells of the next coarser level: a refined
    level-(l-1) cell, l - 1 >= min_level (the h_max level), loses its
    children when they are leaves, none of them is being refined, and every
    fine-grid vertex of level l on the closed cell is erased -- one level of
    coarsening per step.
A8  New vertices start with zero hierarchical surplus: every vertex that
    exists after the step and did not carry an unknown both before and after
    it takes P u_(l-1) (coarse to fine), then the invariants of A3 are
    restored.  Pure refinement leaves the fine-grid function unchanged.
"""
from __future__ import annotations

import itertools

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
        self._set_structure({lev: np.asarray(refine[lev], dtype=bool) for lev in range(1, depth)})
        n = cells_per_axis(depth)
        self.u = {lev: np.zeros((cells_per_axis(lev) + 1,) * d, dtype=np.complex128)
                  for lev in range(1, depth + 1)}
        self.f = {lev: np.zeros_like(self.u[lev]) for lev in self.u}
        self.r0 = None
        assert k2.shape == (n + 1,) * d

    # -- structure
    def _set_structure(self, refine):
        """Cells, leaves, vertex classes and succ from the refine flags of
        levels 1..L-1 (flags of cells that do not exist are dropped)."""
        d, L = self.d, self.L
        self.cells = {1: np.ones((3,) * d, dtype=bool)}
        self.refined = {}
        for lev in range(1, L):
            flags = np.asarray(refine[lev], dtype=bool) & self.cells[lev]
            self.refined[lev] = flags
            self.cells[lev + 1] = child_cells(flags)
        self.refined[L] = np.zeros_like(self.cells[L])
        self.leaf = {lev: self.cells[lev] & ~self.refined[lev] for lev in range(1, L + 1)}
        self.unknown = {}
        self.exists = {}
        for lev in range(1, L + 1):
            cnt = adjacent_count(self.cells[lev])
            inner = np.zeros_like(cnt, dtype=bool)
            inner[(slice(1, -1),) * d] = True
            self.exists[lev] = cnt > 0
            self.unknown[lev] = inner & (cnt == 2 ** d)
        self.succ = self._succ()

    def _succ(self):
        """succ(v) at the unknowns of every level (reading A4), finest first."""
        d, L = self.d, self.L
        succ = {}
        big = np.iinfo(np.int64).max
        for lev in range(L, 0, -1):
            n = cells_per_axis(lev)
            s = np.zeros((n + 1,) * d, dtype=np.int64)
            refined_vertex = self.unknown[lev] & (adjacent_count(self.refined[lev]) == 2 ** d)
            if lev < L and refined_vertex.any():
                child = np.where(self.unknown[lev + 1], succ[lev + 1], big)
                m = np.full((n - 1,) * d, big, dtype=np.int64)
                for off in itertools.product(range(-3, 4), repeat=d):
                    # the children 3v + off of the inner vertices v = 1..n-1
                    m = np.minimum(m, child[tuple(slice(3 + o, 3 * (n - 1) + o + 1, 3) for o in off)])
                inner = (slice(1, -1),) * d
                s[inner] = np.where(refined_vertex[inner], m + 1, 0)
            succ[lev] = s
        return succ

    def fine_grid(self, lev):
        """The fine-grid vertices of a level: unknowns with no unknown at the
        same point on the next finer level."""
        own = self.unknown[lev].copy()
        if lev < self.L:
            own &= ~self.unknown[lev + 1][(slice(None, None, 3),) * self.d]
        return own

    def refine_flags(self):
        """The refine flags of levels 1..L-1, concatenated (x fastest), as
        the library takes and reports them."""
        return np.concatenate([self.refined[lev].ravel() for lev in range(1, self.L)]).astype(np.uint8)

    def fine_vertex_count(self):
        return int(sum(self.fine_grid(lev).sum() for lev in range(1, self.L + 1)))

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
        (cell-wise element matrices, Section 4 / Appendix B)."""
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
            tot += float(np.sum(np.abs(r[lev][self.fine_grid(lev)]) ** 2))
        nrm = np.sqrt(tot)
        if self.r0 is None:
            self.r0 = nrm
        return nrm, (nrm / self.r0 if self.r0 > 0 else 0.0)

    def residual_max(self):
        """Max norm of the residuals of the fine-grid vertices."""
        r = self.level_residuals()
        return max(float(np.abs(r[lev][self.fine_grid(lev)]).max(initial=0.0)) for lev in range(1, self.L + 1))

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
            om = omega[L - 1 - self.succ[lev]]  # reading A4
            t[m] = om[m] * r[lev][m] / op.diag[m]
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

    # -- feature-based dynamic refinement (Section 5.3)
    def refinement_indicator(self):
        """s(v) of reading A5 per level; -1 where v is not a fine-grid vertex."""
        d = self.d
        out = {}
        for lev in range(1, self.L + 1):
            u = self.u[lev]
            n = cells_per_axis(lev)
            inner = (slice(1, -1),) * d
            s = np.zeros((n - 1,) * d)
            for ax in range(d):
                lo = [slice(1, -1)] * d
                hi = [slice(1, -1)] * d
                lo[ax] = slice(0, -2)
                hi[ax] = slice(2, None)
                um, up, u0 = u[tuple(lo)], u[tuple(hi)], u[inner]
                sx = (um.real + up.real) - 2.0 * u0.real
                sy = (um.imag + up.imag) - 2.0 * u0.imag
                s = np.maximum(s, np.sqrt(sx * sx + sy * sy))
            full = np.full((n + 1,) * d, -1.0)
            full[inner] = s
            out[lev] = np.where(self.fine_grid(lev), full, -1.0)
        return out

    def adapt(self, min_level, refine_frac=0.1, erase_frac=0.02, bins=20, veto=1e-2, veto_relative=False):
        """One step of feature-based refinement and erasing (readings A5-A8).
        Returns (vertices selected for refinement, for erasing, fine-grid
        vertices after the step)."""
        d, L = self.d, self.L
        r = self.level_residuals()
        s = self.refinement_indicator()
        fine = {lev: self.fine_grid(lev) for lev in range(1, L + 1)}
        vals = np.concatenate([s[lev][fine[lev]] for lev in range(1, L + 1)])
        nfine = vals.size
        if nfine == 0:
            return 0, 0, 0  # no fine-grid vertex: nothing to select
        smin, smax = vals.min(), vals.max()
        binof = {}
        for lev in range(1, L + 1):
            if smax > smin:
                b = np.floor(((s[lev] - smin) / (smax - smin)) * bins).astype(np.int64)
                b = np.minimum(b, bins - 1)
            else:
                b = np.zeros(s[lev].shape, dtype=np.int64)
            binof[lev] = np.where(fine[lev], b, -1)
        counts = np.bincount(np.concatenate([binof[lev][fine[lev]] for lev in range(1, L + 1)]), minlength=bins)
        k_ref = choose_bins(counts[::-1], refine_frac * nfine)
        k_er = choose_bins(counts, erase_frac * nfine)
        refsel, ersel = {}, {}
        for lev in range(1, L + 1):
            bound = veto * np.abs(self.u[lev]) if veto_relative else veto
            vetoed = np.abs(r[lev] / self.levels[lev].diag) > bound
            top = fine[lev] & (binof[lev] >= bins - k_ref) & ~vetoed
            refsel[lev] = top & (lev < L)
            ersel[lev] = fine[lev] & (binof[lev] < k_er) & ~vetoed & ~top & (lev >= min_level + 1)
        # new refine flags, finest level first (reading A7)
        new = {}
        mark = {}
        for lev in range(L - 1, 0, -1):
            n = cells_per_axis(lev)
            cs = (n,) * d
            mk = np.zeros(cs, dtype=bool)
            for a in _corners(d):
                mk |= refsel[lev][_slab(cs, a)]  # cell c has the corner vertex c + a
            mark[lev] = mk
            old = self.refined[lev]
            coarsen = np.zeros(cs, dtype=bool)
            if lev >= min_level:
                kids_ref = np.zeros(cs, dtype=bool)
                kids_mark = np.zeros(cs, dtype=bool)
                for o in itertools.product(range(3), repeat=d):
                    sl = tuple(slice(oo, 3 * n, 3) for oo in o)
                    kids_ref |= self.refined[lev + 1][sl]
                    if lev + 1 < L:
                        kids_mark |= mark[lev + 1][sl]
                ok = np.ones(cs, dtype=bool)
                for o in itertools.product(range(4), repeat=d):
                    sl = tuple(slice(oo, oo + 3 * n - 2, 3) for oo in o)  # vertex 3c + o of level lev + 1
                    ok &= ~fine[lev + 1][sl] | ersel[lev + 1][sl]
                coarsen = old & ~kids_ref & ~kids_mark & ok
            new[lev] = self.cells[lev] & (mk | (old & ~coarsen))
        old_unknown = {lev: self.unknown[lev].copy() for lev in range(1, L + 1)}
        self._set_structure(new)
        # reading A8: zero surplus on new vertices, coarse to fine
        for lev in range(2, L + 1):
            take = self.exists[lev] & ~(self.unknown[lev] & old_unknown[lev])
            self.u[lev] = np.where(take, prolong(self.u[lev - 1]), self.u[lev])
            zero_boundary(self.u[lev])
        self._restore_invariants()
        n_ref = int(sum(refsel[lev].sum() for lev in range(1, L + 1)))
        n_er = int(sum(ersel[lev].sum() for lev in range(1, L + 1)))
        return n_ref, n_er, self.fine_vertex_count()

    def composite_on_fine(self):
        """The fine-grid function sampled on the uniform level-L grid: on each
        leaf cell the d-linear interpolant of its level's corner values."""
        out = self.u[1].copy()
        for lev in range(2, self.L + 1):
            out = prolong(out)
            m = self.exists[lev]
            out[m] = self.u[lev][m]  # vertices of existing level-lev cells
        return out


def choose_bins(counts, goal):
    """The number k of bins, taken from the front of ``counts``, whose vertex
    total is closest to ``goal``; the smallest such k (reading A6)."""
    best_k, best = 0, abs(goal)
    acc = 0
    for k in range(1, len(counts) + 1):
        acc += int(counts[k - 1])
        if abs(acc - goal) < best:
            best_k, best = k, abs(acc - goal)
    return best_k
