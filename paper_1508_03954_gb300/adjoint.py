"""Differentiable far-field functional J(V, f) = |sum_q g_q u(x_q)|^2.

u solves H(V) u = M f with k^2 = E - V (per fine vertex).  The forward pass
runs the library's solver to a relative residual tolerance and keeps only the
converged u; the backward pass solves the adjoint system H^T lambda = a with
the same solver (the operator is complex-symmetric, H^T = H, so the adjoint
is another solve with right-hand side a_v = sum_q g_q psi_v(x_q)) and forms

    dJ/df_v = 2 Re(conj(s) (M lambda)_v),
    dJ/dV_v = 2 Re(conj(s) (-2^-d) sum_{cells c at v} lambda_c^T M_c u_c)

in the library (mg_adjoint_grad).  Every arithmetic step runs in the CUDA
library; this module only moves tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mg


class SolveOptions:
    def __init__(self, variant=mg.MG_ADD, transfer=mg.MG_DLINEAR, omega=None, tol=1e-10,
                 max_cycles=4000, precision=mg.MG_C64_REFINE, inner_cycles=16):
        self.variant, self.transfer, self.omega = variant, transfer, omega
        self.tol, self.max_cycles = tol, max_cycles
        self.precision, self.inner_cycles = precision, inner_cycles


def _solve(solver, opts):
    solver.set_precision(opts.precision, opts.inner_cycles)
    st, n, rel = solver.solve(opts.variant, opts.omega, opts.transfer, opts.tol, opts.max_cycles)
    if st != mg.MG_OK:
        raise mg.MgError(st, f"solve stopped at relative residual {rel:.3e} after {n} cycles")
    return n, rel


class FarField(torch.autograd.Function):
    """J = FarField.apply(V, f, solver, E, xyz, g, opts); V and f are real
    float64 CUDA tensors in the fine-vertex layout."""

    @staticmethod
    def forward(ctx, V, f, solver, E, xyz, g, opts):
        shape = solver.shape
        k2 = (E - V.detach()).to(torch.float64).contiguous().reshape(-1)
        solver.set_k2(k2)  # device tensor: no host round trip
        solver.set_rhs(f.detach().to(torch.complex128).contiguous().reshape(-1))
        solver.set_solution(np.zeros(shape, dtype=np.complex128))
        n_fwd, rel_fwd = _solve(solver, opts)
        u = torch.empty(solver.nv, dtype=torch.complex128, device=V.device)
        solver.get_solution(u)
        s = solver.sample(xyz, g)
        ctx.save_for_backward(u)  # only the converged forward solution
        ctx.solver, ctx.xyz, ctx.g, ctx.opts, ctx.s = solver, xyz, g, opts, s
        ctx.info = dict(forward_cycles=n_fwd, forward_rel=rel_fwd)
        return torch.tensor(abs(s) ** 2, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(ctx, gJ):
        (u,) = ctx.saved_tensors
        solver = ctx.solver
        solver.set_rhs_samples(ctx.xyz, ctx.g)
        solver.set_solution(np.zeros(solver.shape, dtype=np.complex128))
        _solve(solver, ctx.opts)
        lam = torch.empty(solver.nv, dtype=torch.complex128, device=u.device)
        solver.get_solution(lam)
        dV = torch.empty(solver.nv, dtype=torch.float64, device=u.device)
        df = torch.empty(solver.nv, dtype=torch.float64, device=u.device)
        solver.adjoint_grad(u, lam, ctx.s, dV, df)
        torch.cuda.current_stream().synchronize()
        return gJ * dV.reshape(solver.shape), gJ * df.reshape(solver.shape), None, None, None, None, None


def far_field(V, f, solver, E, xyz, g, opts):
    return FarField.apply(V, f, solver, E, xyz, g, opts)
