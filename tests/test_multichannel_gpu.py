"""Parity of the coupled multichannel cycle (Section 7.5) on the GPU with its
FP64 oracle, through the C ABI: per-iterate relative L2 within 1e-12 over
three cycles of every variant and transfer, for general complex coupling
matrices (not symmetric), with a scaling layer, in 2D and 3D and for several
channel counts; the residual norm of the iterate within 1e-12."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.multichannel import MultiHierarchy
from paper_1508_03954_gb300 import build as B
from paper_1508_03954_gb300 import mg

pytestmark = pytest.mark.gpu

TOL = 1e-12
TH = math.pi / 6
VARIANTS = [(mg.MG_ADD, mg.MG_DLINEAR, O.ADD, O.DLINEAR), (mg.MG_HB, mg.MG_DLINEAR, O.HB, O.DLINEAR),
            (mg.MG_BPX, mg.MG_HIERARCHICAL, O.ADD, O.HIERARCHICAL), (mg.MG_HB, mg.MG_HIERARCHICAL, O.HB, O.HIERARCHICAL)]
IDS = ["add", "hb", "bpx", "hb-hier"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    mg.load()


def _phi(c, seed):
    rng = np.random.default_rng(seed)
    off = (rng.standard_normal((c, c)) * 8 + 1j * rng.standard_normal((c, c)) * 2) * (1 - np.eye(c))
    return np.diag(rng.uniform(-60, 60, size=c)) + off


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel_l2(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def run(d, depth, c, var, w, cycles=3, seed=0):
    Phi = _phi(c, seed)
    n = 3 ** depth
    F = _rand((c,) + (n + 1,) * d, seed + 1)
    U = _rand((c,) + (n + 1,) * d, seed + 2)
    o = MultiHierarchy(d, depth, Phi, TH, w)
    o.set_rhs_nodal(F)
    o.set_solution(U)
    g = mg.MultiChannel(d, depth, Phi, TH, w)
    g.set_rhs(np.moveaxis(F, 0, -1))
    g.set_solution(np.moveaxis(U, 0, -1))
    om = np.array([0.5 + 0.03j * l for l in range(depth)])
    a_g, _ = g.residual_norm()
    a_o, _ = o.residual_norm()
    assert abs(a_g - a_o) <= 1e-12 * a_o
    for k in range(cycles):
        g.cycle(var[0], om, var[1])
        o.cycle(om, var[2], var[3])
        e = rel_l2(np.moveaxis(g.get_solution(), -1, 0), o.u)
        assert e <= TOL, f"iterate {k + 1}: rel L2 {e:.3e}"
    a_g, _ = g.residual_norm()
    a_o, _ = o.residual_norm()
    assert abs(a_g - a_o) <= 1e-12 * a_o
    g.close()


@pytest.mark.parametrize("var", VARIANTS, ids=IDS)
@pytest.mark.parametrize("d,depth,c", [(2, 3, 1), (2, 3, 3), (2, 4, 2), (2, 3, 8), (3, 2, 4), (3, 3, 2)])
def test_iterates_match_oracle(var, d, depth, c):
    run(d, depth, c, var, 0.2, seed=10 * depth + c)


@pytest.mark.parametrize("w", [0.0, 0.5])
def test_no_layer_and_full_scaling(w):
    run(2, 3, 4, VARIANTS[2], w, seed=7)


def test_sixteen_channels():
    run(2, 2, 16, VARIANTS[0], 0.2, cycles=2, seed=5)
