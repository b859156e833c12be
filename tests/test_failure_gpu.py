"""Failure handling on the GPU without faulting it: a bounded device wait
that cannot be satisfied runs out, the kernel records it and finishes, the
host gets MG_ERR_TIMEOUT, and the context stays usable.  Divergence is
reported as a status (see test_parity_gpu)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1508_03954_gb300 import build as B
from paper_1508_03954_gb300 import mg
from paper_1508_03954_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    mg.load()


def test_unsatisfiable_wait_times_out_and_context_recovers():
    depth = 4
    k2 = W.constant_k2(2, depth, 40.0)
    f = W.random_complex(2, depth, 5)
    g = mg.Solver(2, depth, k2, math.pi / 6, 0.1)
    o = O.Hierarchy(2, depth, k2, math.pi / 6, 0.1)
    g.set_rhs(f)
    o.set_rhs_nodal(f)
    om = np.full(depth, 0.6)
    g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
    o.cycle(om, O.ADD, O.HIERARCHICAL)
    g.residual_norm()
    g.set_spin_limit(2000)
    g.debug_unsatisfiable_wait(True)
    with pytest.raises(mg.MgError) as ei:
        g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)  # the wait runs out on the device
        g.residual_norm()  # first synchronising call
    assert ei.value.code == mg.MG_ERR_TIMEOUT
    # recovery: switch the diagnostic off, restart from a known state, parity again
    g.debug_unsatisfiable_wait(False)
    g.set_spin_limit(1 << 22)
    u = o.u.copy()
    g.set_solution(u)
    g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
    o.cycle(om, O.ADD, O.HIERARCHICAL)
    got = g.get_solution()
    assert np.linalg.norm(got - o.u) <= 1e-12 * np.linalg.norm(o.u)
    g.close()


def test_invalid_calls_return_status_not_crash():
    g = mg.Solver(2, 2, W.constant_k2(2, 2, 1.0), 0.3, 0.1)
    with pytest.raises(mg.MgError) as ei:
        g.cycle(7, np.full(2, 0.6), mg.MG_DLINEAR)
    assert ei.value.code == mg.MG_ERR_INVALID
    with pytest.raises(mg.MgError):
        g.set_spin_limit(0)
    with pytest.raises(ValueError):
        g.set_rhs(np.zeros(5))
    g.close()
