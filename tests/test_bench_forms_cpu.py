"""The adaptive bench forms run end to end on the host against a stand-in for
the library and the CUDA events (no GPU, no numbers): their own Python --
workload set-up, the call sequence, the grid-structure counting and the
result layout -- is exercised on every CPU run, so a mistake there cannot
first show up in a GPU bench run."""
import types

import numpy as np

import bench


class _Event:
    def record(self, *args):
        pass

    def elapsed_time(self, other):
        return 1.0


class _Torch:
    class cuda:
        Event = staticmethod(lambda enable_timing=True: _Event())

        @staticmethod
        def synchronize():
            pass

        @staticmethod
        def current_stream():
            return types.SimpleNamespace(cuda_stream=0)


def _fake_mg(calls):
    class Solver:
        def __init__(self, d, depth, *args):
            self.shape = (3 ** depth + 1,) * d

        @classmethod
        def adaptive(cls, d, depth, k2, theta, layer, refine, theta_interior=0.0):
            assert set(refine) == set(range(1, depth))
            for lev in range(1, depth):
                assert refine[lev].shape == (3 ** lev,) * d
            calls.append("adaptive")
            return cls(d, depth)

        def set_stream(self, s):
            pass

        def set_rhs(self, f):
            assert f.shape == self.shape

        def set_solution(self, u):
            assert u.shape == self.shape

        def residual_max(self):
            return 1.0

        def cycle(self, variant, omega, transfer):
            calls.append("cycle")

        def adapt(self, min_level, refine_frac, erase_frac, bins, veto, veto_relative=False):
            calls.append("relative" if veto_relative else "absolute")
            return (1, 0, 100, 7)

        def solve(self, *args):
            return 0, 10, 1e-9

        def get_solution(self):
            return np.ones(self.shape, complex)

        def close(self):
            pass

    return types.SimpleNamespace(Solver=Solver, MG_ADD=0, MG_HB=1, MG_BPX=2, MG_DLINEAR=0, MG_HIERARCHICAL=1,
                                 MG_OMEGA_JACOBI=0, MG_OMEGA_UCG=1, MG_OMEGA_TRANSITION=4, MgError=RuntimeError,
                                 STATUS_NAMES={0: "MG_OK"}, omega_scheme=lambda *a: np.ones(a[2], complex))


def test_channel_table2_adaptive_form_layout():
    calls = []
    out = bench.channel_table2_adaptive(_fake_mg(calls), _Torch, iters=2, depth=5, min_level=3)
    runs = out["runs"]
    assert len(runs) == 5 * 3 * 2  # theta x solver x veto reading
    assert {r["veto"] for r in runs} == {"absolute", "relative"}
    assert calls.count("relative") == calls.count("absolute") == 5 * 3 * 2
    for r in runs:
        assert {"reduction_max_norm", "fine_vertices", "finest_level", "ms_cycle", "ms_adapt"} <= set(r)


def test_adaptive_form_counts_the_fine_grid_unknowns():
    """The form's own count of fine-grid unknowns (2D depth 6, the source
    refinement) is the figure quoted for it: 13,208 against 529,984."""
    calls = []
    out = bench.adaptive(_fake_mg(calls), _Torch, d=2, depth=6, cycles=2)
    assert out["adaptive"]["fine_unknowns"] == 13208
    assert out["regular"]["fine_unknowns"] == 529984
