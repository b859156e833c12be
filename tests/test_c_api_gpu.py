"""The library used from plain C through include/mg.h alone
(tests/c_api/solve_c.c): a definite 2D solve to 1e-10 (checked again by
mg_residual_norm inside the client), the same solve with complex64 cycles in
FP64 defect correction (solutions within 1e-7), a 3D cycle from a page-locked
host buffer, dynamic refinement of an adaptive grid, a batch of three
problems, the adjoint calls with a device k^2 field, and coupled two-channel
cycles."""
import os
import subprocess

import pytest

from paper_1508_03954_gb300 import build as B
from test_abi_cpu import build_c_client

pytestmark = pytest.mark.gpu


def test_plain_c_client_runs(root_dir, tmp_path):
    B.build()
    exe = build_c_client(root_dir, str(tmp_path / "solve_c"))
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.path.dirname(B.LIB) + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    p = subprocess.run([exe], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "status 0" in p.stdout, p.stdout
