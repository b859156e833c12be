"""The allocation-free residual entry point, checked against the existing one.

mg_residual_noalloc serves callers that cannot allocate device memory when
they need a residual (frameworks that keep the whole device in their own
memory pool, time-critical loops that cannot take the synchronisation of an
allocation).  Its reduction scratch is a static device array inside the
library instead of memory from cudaMalloc.  Through the C ABI, two calls in a
row must reproduce the residual norm of the existing mg_residual_norm to the
1e-12 relative tolerance of the other parity tests, and grids above its
stated limit must be refused.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from paper_1508_03954_gb300 import build as B
from paper_1508_03954_gb300 import mg
from paper_1508_03954_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TH = math.pi / 6


def _zero_ring(u):
    u = u.copy()
    for ax in range(u.ndim):
        idx = [slice(None)] * u.ndim
        idx[ax] = 0
        u[tuple(idx)] = 0
        idx[ax] = -1
        u[tuple(idx)] = 0
    return u


@pytest.mark.parametrize("d,depth,varying", [(2, 4, False), (3, 3, False), (2, 3, True)])
def test_noalloc_residual_matches_existing_entry_point(d, depth, varying):
    import torch

    B.build()
    mg.load()
    n = 3 ** depth
    if varying:
        k2 = np.random.default_rng(7).uniform(-50.0, 300.0, size=(n + 1,) * d)
    else:
        k2 = W.constant_k2(d, depth, 45.0)
    s = mg.Solver(d, depth, k2, TH, 0.1)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    s.set_rhs(W.random_complex(d, depth, 11))
    b = torch.empty(s.nv, dtype=torch.complex128, device="cuda")
    s.get_level_device(depth, 1, b)
    r = torch.empty(s.nv, dtype=torch.complex128, device="cuda")
    norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (21, 22):  # two calls in a row, different solutions
        u0 = _zero_ring(W.random_complex(d, depth, seed))
        s.set_solution(u0)
        ref_abs, _ = s.residual_norm()
        u = torch.from_numpy(u0.reshape(-1)).cuda()
        s.residual_noalloc(u, b, r, norm2)
        torch.cuda.synchronize()
        got = math.sqrt(norm2.item())
        assert abs(got - ref_abs) <= 1e-12 * ref_abs, (got, ref_abs)
        assert abs(torch.linalg.vector_norm(r).item() - got) <= 1e-12 * got
    s.close()


def test_noalloc_residual_norm_only():
    """r = NULL: only the norm is formed, still equal to mg_residual_norm's."""
    import torch

    B.build()
    mg.load()
    d, depth = 2, 4
    s = mg.Solver(d, depth, W.constant_k2(d, depth, 45.0), TH, 0.1)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    s.set_rhs(W.random_complex(d, depth, 31))
    b = torch.empty(s.nv, dtype=torch.complex128, device="cuda")
    s.get_level_device(depth, 1, b)
    norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (32, 33):
        u0 = _zero_ring(W.random_complex(d, depth, seed))
        s.set_solution(u0)
        ref_abs, _ = s.residual_norm()
        s.residual_noalloc(torch.from_numpy(u0.reshape(-1)).cuda(), b, None, norm2)
        torch.cuda.synchronize()
        got = math.sqrt(norm2.item())
        assert abs(got - ref_abs) <= 1e-12 * ref_abs, (got, ref_abs)
    s.close()


def test_noalloc_residual_refuses_grids_above_its_limit():
    import torch

    B.build()
    mg.load()
    depth = 7  # 2188^2 = 4,787,344 vertices > 16384 * 256
    s = mg.Solver(2, depth, W.constant_k2(2, depth, 10.0), TH, 0.1)
    u = torch.zeros(s.nv, dtype=torch.complex128, device="cuda")
    norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgError) as ei:
        s.residual_noalloc(u, u, None, norm2)
    assert ei.value.code == mg.MG_ERR_INVALID and "4194304" in str(ei.value)
    s.close()
