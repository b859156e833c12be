"""Plain FP64 CPU oracle of the complex additive multilevel cycle
(Reps & Weinzierl, "Complex additive geometric multilevel solvers for
Helmholtz equations on spacetrees").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or helper with the CUDA library; it never reads a value the
CUDA path produced.

Everything is complex128 (FP64), slow and literal:

* the operator is assembled cell by cell from 2^d x 2^d element matrices
  (Section 4 "Multigrid realisation" and Appendix B: every cell applies its
  local matrix to its 2^d vertex values and scatters into the residual and
  diagonal accumulators of its vertices);
* the cycle is the bottom-up FAS form of additive multigrid (Appendix A,
  Algorithm 4 ``buFAS``) with one relaxation factor per level (Section 5.1),
  the hierarchical-basis mask (Section 5.2, Eq. hb-omega) and the BPX
  prolongation of Appendix A (``P(u_{l-1} - I(u_l + du_l))``).

Grid conventions (regular levels of a tripartitioned spacetree, Section 3):
level l = 1..L has 3^l cells per axis, spacing 3^-l, (3^l + 1)^d vertices
including the Dirichlet ring, stored as numpy arrays whose LAST axis is x.
Level 0 carries no unknowns (l_min = 1).  Boundary entries are always zero.

Readings of the paper that this file fixes (each is also listed in the
design notes):

R1  Coordinate-wise exterior scaling: along axis j a cell's spacing is
    h*e^{i theta} when its centre c_j satisfies min(c_j, 1-c_j) < w, else h
    (Section 7.4 rotates the cells near the open faces; Section 7.3 scales
    the spacing along every axis).  w >= 0.5 rotates every cell (full complex
    scaled grid).  Membership uses the cell centre on every level.
R1b The channel problem of Section 7.4 puts the layer at two faces only (top
    and right, within 1/3 of the domain, 30 degrees) and rotates every other
    cell by theta, whatever the layer does: along each axis a
    cell with centre c is in the layer when c < w_lo or 1 - c < w_hi and has
    spacing h*e^{i theta}; every other cell has h*e^{i theta_interior}.
    ``layer_width`` is w (both faces, w_lo = w_hi = w) or the pair
    (w_lo, w_hi); the two layers covering the axis rotate every cell.
R2  The cell value of the shift is the mean of its 2^d vertex values of
    phi = k^2; coarse levels sample k^2 at their own vertices (injection).
R3  The fine right-hand side is the consistent mass product b = M f of nodal
    f (complex-scaled in layer cells).
R4  "Iterate n" is the fine solution after n cycles with every correction
    applied (the paper's pipelined traversal lags by half a sweep).
R5  R = P^T exactly (tripartite d-linear weights).
R6  The Section 7.4 table (used by the tests, not by this file's cycle):
    pure Jacobi is the cycle with zero factors below the finest level; on the
    unrotated problem (theta = 0) it alternates the two-phase factors
    0.01 (sqrt 3 - i) and its negated conjugate, and every Jacobi run with a
    rotated interior uses 0.4, the factor the text fixes for Jacobi smoothers
    that apply complex rotations.  The transition scheme and BPX use
    omega_S = 0.4.  Reductions are max norms, |r_50| / |r_0| from u = 0.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

ADD, HB = 0, 1               # variant: plain relaxation factors / c-points masked
DLINEAR, HIERARCHICAL = 0, 1  # transfer: T = id / T = (id - P I)


# ----------------------------------------------------------------------------
# Grid geometry
# ----------------------------------------------------------------------------
def cells_per_axis(level: int) -> int:
    """3^l cells per axis on level l (tripartition, Section 3)."""
    return 3 ** level


def layer_widths(layer_width):
    """(w_lo, w_hi) from a symmetric width w or a pair (readings R1, R1b)."""
    if np.ndim(layer_width) == 0:
        return float(layer_width), float(layer_width)
    lo, hi = layer_width
    return float(lo), float(hi)


def rotated_cells(level: int, layer_width) -> np.ndarray:
    """Readings R1/R1b: flag per cell index along one axis, True inside the
    layer.

    Cell i has centre c = (i + 1/2)/n; c < w_lo and 1 - c < w_hi are tested in
    the exact integer forms 2i + 1 < 2 w_lo n and 2n - 2i - 1 < 2 w_hi n.
    """
    n = cells_per_axis(level)
    lo, hi = layer_widths(layer_width)
    if lo + hi >= 1.0:
        return np.ones(n, dtype=bool)
    i = np.arange(n)
    return (2 * i + 1 < 2.0 * lo * n) | (2 * n - 2 * i - 1 < 2.0 * hi * n)


def axis_spacing(level: int, theta: float, layer_width, theta_interior: float = 0.0) -> np.ndarray:
    """Complex cell width per cell index along one axis: h e^{i theta} in the
    layer, h e^{i theta_interior} elsewhere (complex scaled grid, Section 2,
    Section 7.3 and Section 7.4)."""
    n = cells_per_axis(level)
    h = 1.0 / n
    out = np.full(n, h * complex(math.cos(theta_interior), math.sin(theta_interior)), dtype=np.complex128)
    out[rotated_cells(level, layer_width)] = h * complex(math.cos(theta), math.sin(theta))
    return out


# ----------------------------------------------------------------------------
# Element matrices (Section 4: Ritz-Galerkin p-linear elements; Appendix B)
# ----------------------------------------------------------------------------
def element_matrices_1d(h):
    """1D linear element on a cell of (complex) width h:
    stiffness (1/h)[[1,-1],[-1,1]] and mass (h/6)[[2,1],[1,2]]."""
    k = np.array([[1.0, -1.0], [-1.0, 1.0]], dtype=np.complex128) / h
    m = np.array([[2.0, 1.0], [1.0, 2.0]], dtype=np.complex128) * (h / 6.0)
    return k, m


def element_matrices(hs):
    """2^d x 2^d stiffness K_c and mass M_c of one d-linear cell with per-axis
    widths hs (numpy axis order, last = x).  Tensor products of the 1D
    matrices: M_c = M(h_0) x ... x M(h_{d-1}); K_c = sum_j of the same product
    with the j-th factor replaced by the stiffness.  Local vertex index is
    sum_k a_k 2^(d-1-k) (last axis fastest), matching np.kron."""
    ks, ms = zip(*(element_matrices_1d(h) for h in hs))
    d = len(hs)
    mc = ms[0]
    for k in range(1, d):
        mc = np.kron(mc, ms[k])
    kc = np.zeros_like(mc)
    for j in range(d):
        t = ks[0] if j == 0 else ms[0]
        for k in range(1, d):
            t = np.kron(t, ks[k] if k == j else ms[k])
        kc += t
    return kc, mc


def helmholtz_element(hs, phi):
    """H_c = K_c - phi M_c: the local matrix of -Laplace - phi (Eq. pHelmholtz)."""
    kc, mc = element_matrices(hs)
    return kc - phi * mc


# ----------------------------------------------------------------------------
# One level of the hierarchy
# ----------------------------------------------------------------------------
def _corners(d):
    return list(itertools.product((0, 1), repeat=d))


def _slab(shape_cells, offset):
    return tuple(slice(o, o + n) for o, n in zip(offset, shape_cells))


class Level:
    """Operator data of one regular level l: per-axis complex widths, cell
    shifts phi_c and the accumulated diagonal (Section 4: diag(H_l) is
    accumulated cell by cell, which complex layers and varying phi require)."""

    def __init__(self, d, level, k2_vertices, theta, layer_width, theta_interior=0.0):
        self.d, self.level = d, level
        self.n = cells_per_axis(level)
        self.h_axis = axis_spacing(level, theta, layer_width, theta_interior)
        k2 = np.asarray(k2_vertices, dtype=np.float64)
        assert k2.shape == (self.n + 1,) * d
        # R2: cell shift = mean of the 2^d vertex values
        acc = np.zeros((self.n,) * d)
        for a in _corners(d):
            acc += k2[_slab((self.n,) * d, a)]
        self.phi_cell = acc / (2 ** d)
        self.diag = self._assemble_diag()

    # per-cell entries of the 1D factors, broadcast along axis ``ax``
    def _factor(self, ax, kind, a, b):
        h = self.h_axis
        if kind == "K":
            v = (1.0 if a == b else -1.0) / h
        else:
            v = (2.0 if a == b else 1.0) * h / 6.0
        shape = [1] * self.d
        shape[ax] = self.n
        return v.reshape(shape)

    def cell_entry(self, a, b, with_phi=True):
        """Entry [a, b] of every cell's local matrix, as an n^d array:
        K_c[a,b] - phi_c M_c[a,b] (or M_c[a,b] alone when with_phi=False)."""
        d = self.d
        mprod = np.ones((1,) * d, dtype=np.complex128)
        for ax in range(d):
            mprod = mprod * self._factor(ax, "M", a[ax], b[ax])
        if not with_phi:
            return np.broadcast_to(mprod, (self.n,) * d)
        kent = np.zeros((1,) * d, dtype=np.complex128)
        for j in range(d):
            t = np.ones((1,) * d, dtype=np.complex128)
            for ax in range(d):
                t = t * self._factor(ax, "K" if ax == j else "M", a[ax], b[ax])
            kent = kent + t
        return kent - self.phi_cell * mprod

    def _assemble_diag(self):
        out = np.zeros((self.n + 1,) * self.d, dtype=np.complex128)
        for a in _corners(self.d):
            out[_slab((self.n,) * self.d, a)] += self.cell_entry(a, a)
        return out

    def apply(self, u, with_phi=True):
        """Element-wise matrix-free product (Appendix B): every cell applies
        its local matrix to its 2^d vertex values and adds the result to the
        accumulators of those vertices.  Rows of boundary vertices are
        dropped (Dirichlet vertices carry no unknowns)."""
        cs = (self.n,) * self.d
        out = np.zeros((self.n + 1,) * self.d, dtype=np.complex128)
        for a in _corners(self.d):
            acc = np.zeros(cs, dtype=np.complex128)
            for b in _corners(self.d):
                acc += self.cell_entry(a, b, with_phi) * u[_slab(cs, b)]
            out[_slab(cs, a)] += acc
        zero_boundary(out)
        return out

    def mass(self, f):
        """Consistent mass product M_l f (reading R3)."""
        return self.apply(f, with_phi=False)


def zero_boundary(x):
    """Homogeneous Dirichlet vertices (the outer ring) hold zero."""
    for ax in range(x.ndim):
        idx = [slice(None)] * x.ndim
        idx[ax] = 0
        x[tuple(idx)] = 0
        idx[ax] = -1
        x[tuple(idx)] = 0
    return x


# ----------------------------------------------------------------------------
# Grid transfer (Section 4: d-linear P, R = P^T, injection I)
# ----------------------------------------------------------------------------
def prolong(xc):
    """d-linear interpolation from level l-1 to level l on the tripartitioned
    grid: fine index 3c + o takes (1 - o/3) x[c] + (o/3) x[c+1] along each
    axis, applied axis by axis."""
    x = np.asarray(xc, dtype=np.complex128)
    for ax in range(x.ndim):
        x = np.moveaxis(x, ax, 0)
        nc = x.shape[0] - 1
        y = np.zeros((3 * nc + 1,) + x.shape[1:], dtype=np.complex128)
        y[0::3] = x
        y[1::3] = (2.0 / 3.0) * x[:-1] + (1.0 / 3.0) * x[1:]
        y[2::3] = (1.0 / 3.0) * x[:-1] + (2.0 / 3.0) * x[1:]
        x = np.moveaxis(y, 0, ax)
    return x


def restrict(xf):
    """R = P^T (reading R5): coarse c collects the fine values 3c + o,
    o = -2..2, with weights 1 - |o|/3 along each axis.  Written as the
    transpose of the interpolation weights, axis by axis."""
    x = np.asarray(xf, dtype=np.complex128)
    for ax in range(x.ndim):
        x = np.moveaxis(x, ax, 0)
        nc = (x.shape[0] - 1) // 3
        y = x[0::3].copy()
        y[:-1] += (2.0 / 3.0) * x[1::3] + (1.0 / 3.0) * x[2::3]
        y[1:] += (1.0 / 3.0) * x[1::3] + (2.0 / 3.0) * x[2::3]
        assert y.shape[0] == nc + 1
        x = np.moveaxis(y, 0, ax)
    return x


def inject(xf):
    """Injection I: the coarse vertex copies the fine vertex at the same
    position (Eq. injection, u_{l-1} = I u_l)."""
    return np.asarray(xf)[(slice(None, None, 3),) * np.asarray(xf).ndim].copy()


def cpoint_mask(d, level):
    """cPoint(v) (Section 5.1): the vertex coincides with a vertex of the next
    coarser level, i.e. all of its level-l indices are multiples of 3."""
    n = cells_per_axis(level)
    m = np.zeros((n + 1,) * d, dtype=bool)
    m[(slice(None, None, 3),) * d] = True
    return m


# ----------------------------------------------------------------------------
# Relaxation schemes (Section 5.1 table) on a regular grid: succ(v) = L - l
# ----------------------------------------------------------------------------
JACOBI, UCG, LGRID, EXP, TRANSITION = 0, 1, 2, 3, 4


def omega_scheme(scheme, omega_s, depth, iter_n=1, l_grid=0):
    """Per-level factors omega_l, index l-1, from the five schemes of the
    Section 5.1 table with succ = L - l on a regular grid:
    Jacobi only (succ = 0 gets omega_S, others 0), undamped coarse grid
    (omega_S everywhere), undamped L-grid (omega_S while succ <= L_g),
    exponential damping omega_S^(succ+1) and transition
    omega_S^((1 - 1/n)(succ+1)) at iteration n >= 1."""
    w = complex(omega_s)
    out = np.zeros(depth, dtype=np.complex128)
    for lev in range(1, depth + 1):
        succ = depth - lev
        if scheme == JACOBI:
            out[lev - 1] = w if succ == 0 else 0
        elif scheme == UCG:
            out[lev - 1] = w
        elif scheme == LGRID:
            out[lev - 1] = w if succ <= l_grid else 0
        elif scheme == EXP:
            out[lev - 1] = w ** (succ + 1)
        elif scheme == TRANSITION:
            out[lev - 1] = w ** ((1.0 - 1.0 / iter_n) * (succ + 1))
        else:
            raise ValueError("unknown scheme")
    return out


# ----------------------------------------------------------------------------
# The hierarchy and the cycle
# ----------------------------------------------------------------------------
class Hierarchy:
    """Levels 1..L of a regular tripartitioned spacetree with the fine-grid
    state (u_L, b_L).  Coarse solutions are never stored: they are the
    injections of u_L (Lemma 1, Eq. injection)."""

    def __init__(self, d, depth, k2_fine, theta, layer_width, theta_interior=0.0):
        self.d, self.L = d, depth
        self.theta, self.layer_width = theta, layer_width
        self.theta_interior = theta_interior
        k2 = np.asarray(k2_fine, dtype=np.float64)
        n = cells_per_axis(depth)
        assert k2.shape == (n + 1,) * d
        self.k2 = {depth: k2}
        for lev in range(depth - 1, 0, -1):
            self.k2[lev] = inject(self.k2[lev + 1])
        self.levels = {lev: Level(d, lev, self.k2[lev], theta, layer_width, theta_interior)
                       for lev in range(1, depth + 1)}
        self.u = np.zeros((n + 1,) * d, dtype=np.complex128)
        self.b = np.zeros_like(self.u)
        self.r0 = None

    def set_rhs_nodal(self, f):
        """b_L = M_L f for nodal f (reading R3); resets the reference residual."""
        f = np.asarray(f, dtype=np.complex128).copy()
        self.b = self.levels[self.L].mass(f)
        self.r0 = None

    def set_solution(self, u):
        u = np.asarray(u, dtype=np.complex128).copy()
        zero_boundary(u)
        self.u = u
        self.r0 = None

    def residual(self, u=None):
        u = self.u if u is None else u
        return self.b - self.levels[self.L].apply(u)

    def residual_max(self):
        """Maximum modulus of b - H u over the vertices (the max norm of the
        Section 7.4 table)."""
        return float(np.abs(self.residual()).max())

    def residual_norm(self):
        """Euclidean norm of b - H u over the fine vertices and the same norm
        relative to the residual of the starting solution (Section 7 norms;
        on a regular grid the h-weighted norm gives the same ratio)."""
        r = np.linalg.norm(self.residual().ravel())
        if self.r0 is None:
            self.r0 = r
        return r, (r / self.r0 if self.r0 > 0 else 0.0)

    def cycle(self, omega, variant=ADD, transfer=DLINEAR, trace=None):
        """One additive FAS cycle, Appendix A Algorithm 4 (buFAS) unrolled:

        fine to coarse, l = L..1:
            du_l   = omega_l diag(H_l)^{-1} (b_l - H_l u_l)       (Section 4 S)
            if l > 1:  u_{l-1} = I u_l
                       uhat_l  = u_l - P u_{l-1}                   (surplus)
                       rhat_l  = b_l - H_l uhat_l                  (Eq. HTMG)
                       b_{l-1} = R rhat_l
        coarse to fine, with the transfer T_l of the variant:
            corr_1 = T_1 du_1;  corr_l = T_l du_l + P corr_{l-1}
            u_L   <- u_L + corr_L
        T_l = id (additive), hb mask (Eq. hb-omega: du_l = 0 at c-points), or
        (id - P I) for BPX (Appendix A lemma: corr_l = du_l - P I du_l +
        P corr_{l-1}).  On level 1 the c-points are the Dirichlet corners.
        """
        L, d = self.L, self.d
        omega = np.asarray(omega, dtype=np.complex128)
        assert omega.shape == (L,)
        u = {L: self.u}
        b = {L: self.b}
        du = {}
        for lev in range(L, 0, -1):
            op = self.levels[lev]
            r = b[lev] - op.apply(u[lev])
            du[lev] = np.zeros_like(r)
            inner = (slice(1, -1),) * d
            du[lev][inner] = omega[lev - 1] * r[inner] / op.diag[inner]
            if trace is not None:
                trace.setdefault("r", {})[lev] = r
            if lev > 1:
                u[lev - 1] = inject(u[lev])
                uhat = u[lev] - prolong(u[lev - 1])
                rhat = b[lev] - op.apply(uhat)
                b[lev - 1] = zero_boundary(restrict(rhat))
        corr = None
        for lev in range(1, L + 1):
            t = du[lev]
            if variant == HB:
                t = np.where(cpoint_mask(d, lev), 0, t)
            if transfer == HIERARCHICAL:
                t = t - prolong(inject(t))
            corr = t if lev == 1 else t + prolong(corr)
            if trace is not None:
                trace.setdefault("corr", {})[lev] = corr
                trace.setdefault("du", {})[lev] = du[lev]
                trace.setdefault("b", {})[lev] = b[lev]
        self.u = self.u + corr
        zero_boundary(self.u)
        return self.u

    def solve(self, omega, variant=ADD, transfer=DLINEAR, tol=1e-8,
              max_cycles=100, diverge=1e6):
        """Cycles until the relative residual is <= tol.  Returns
        (status, cycles, rel): status 0 converged, 5 not converged,
        4 diverged (relative residual above ``diverge`` or not finite,
        the paper's bottom symbol in Tables 1-2)."""
        _, rel = self.residual_norm()
        n = 0
        while True:
            if not np.isfinite(rel) or rel > diverge:
                return 4, n, rel
            if rel <= tol:
                return 0, n, rel
            if n >= max_cycles:
                return 5, n, rel
            self.cycle(omega, variant, transfer)
            n += 1
            _, rel = self.residual_norm()


def fmg_start(d, depth, k2_fine, theta, layer_width, f_fine, omega,
              variant=ADD, transfer=DLINEAR, cycles_per_stage=3):
    """Grid unfolding (Remark on FMG, Section 5; Section 7.1): stage s = 1..L
    solves on levels 1..s with b_s = M_s f (f and k^2 sampled at level-s
    vertices), starts from P u_{s-1}, and runs ``cycles_per_stage`` cycles on
    every stage but the last.  Level l of stage s uses the factor that level
    l + (L - s) has in the full hierarchy (same distance to the finest level).
    Returns the depth-L hierarchy holding the interpolated start."""
    k2 = np.asarray(k2_fine, dtype=np.float64)
    f = np.asarray(f_fine, dtype=np.complex128)
    omega = np.asarray(omega, dtype=np.complex128)
    u_prev = None
    for s in range(1, depth + 1):
        stride = 3 ** (depth - s)
        sl = (slice(None, None, stride),) * d
        hs = Hierarchy(d, s, k2[sl], theta, layer_width)
        hs.set_rhs_nodal(f[sl])
        if u_prev is not None:
            hs.set_solution(prolong(u_prev))
        if s == depth:
            return hs
        w = omega[depth - s:]
        for _ in range(cycles_per_stage):
            hs.cycle(w, variant, transfer)
        u_prev = hs.u
    raise AssertionError("unreachable")
