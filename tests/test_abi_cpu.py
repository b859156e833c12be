"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/mg.h declares, validates arguments
before touching the device, and its host helper matches the relaxation
schemes of Section 5.1."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1508_03954_gb300 import build as B
from paper_1508_03954_gb300 import mg


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mg.load()


def declared_functions(root):
    names = set()
    inc = os.path.join(root, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mg_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib, root_dir):
    names = declared_functions(root_dir)
    assert {"mg_create", "mg_cycle", "mg_solve", "mg_residual_norm", "mg_set_rhs"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(mg.EXPORTS)


def test_argument_validation_before_device_work(lib):
    h = ctypes.c_void_p()
    k2 = np.zeros(100)
    kp = k2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for args in [(4, 2, kp, 0.5, 0.1), (2, 0, kp, 0.5, 0.1), (2, 2, None, 0.5, 0.1),
                 (2, 2, kp, 2.0, 0.1), (2, 2, kp, 0.5, 0.7), (2, 2, kp, -0.1, 0.1)]:
        assert lib.mg_create(*args, ctypes.byref(h)) == mg.MG_ERR_INVALID
        assert len(lib.mg_last_error(None)) > 0
    assert lib.mg_cycle(None, 0, None, 0) == mg.MG_ERR_INVALID
    assert lib.mg_solve(None, 0, None, 0, 1e-8, 1, None, None) == mg.MG_ERR_INVALID
    lib.mg_destroy(None)


@pytest.mark.parametrize("scheme,oscheme", [(mg.MG_OMEGA_JACOBI, O.JACOBI), (mg.MG_OMEGA_UCG, O.UCG),
                                            (mg.MG_OMEGA_LGRID, O.LGRID), (mg.MG_OMEGA_EXP, O.EXP),
                                            (mg.MG_OMEGA_TRANSITION, O.TRANSITION)])
def test_omega_scheme_helper(lib, scheme, oscheme):
    for it in (1, 2, 5):
        got = mg.omega_scheme(scheme, 0.6 + 0.1j, 5, iter_n=it, l_grid=2)
        ref = O.omega_scheme(oscheme, 0.6 + 0.1j, 5, iter_n=it, l_grid=2)
        np.testing.assert_allclose(got, ref, rtol=1e-14)


def test_trace_stage_layout_matches_chain_rules():
    """The trace helper's stage layout of the depth-6 chain (tiles of 4, 2, 1
    coarse cells by level size; correction chunks of about two per SM)."""
    from paper_1508_03954_gb300.trace import chain_stages, fine_tiles
    assert [k for _, k in chain_stages(729)] == [441, 196, 100, 16, 4, 106, 233]
    assert fine_tiles(729) == 961
    assert [k for _, k in chain_stages(243)] == [196, 100, 16, 4, 13, 106]


def build_c_client(root, out_path):
    """Compiles tests/c_api/solve_c.c against include/mg.h and links it with
    the in-tree libmg.so (no Python, no torch in the client)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-O2", "-I", os.path.join(root, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(root, "tests", "c_api", "solve_c.c"), "-o", out_path,
           "-L", os.path.dirname(B.LIB), "-lmg", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


def test_plain_c_client_compiles_and_links(lib, root_dir, tmp_path):
    exe = build_c_client(root_dir, str(tmp_path / "solve_c"))
    assert os.path.exists(exe)


def test_multichannel_argument_validation_before_device_work(lib):
    h = ctypes.c_void_p()
    phi = (mg.MgC128 * 4)()
    for args in [(4, 2, 2, phi, 0.5, 0.1), (2, 0, 2, phi, 0.5, 0.1), (2, 2, 5, phi, 0.5, 0.1),
                 (2, 2, 2, None, 0.5, 0.1), (2, 2, 2, phi, 2.0, 0.1), (2, 2, 2, phi, 0.5, 0.7),
                 (3, 7, 2, phi, 0.5, 0.1)]:
        assert lib.mg_mc_create(*args, ctypes.byref(h)) == mg.MG_ERR_INVALID
    assert lib.mg_mc_cycle(None, 0, None, 0) == mg.MG_ERR_INVALID
    assert lib.mg_mc_residual_norm(None, None, None) == mg.MG_ERR_INVALID
    lib.mg_mc_destroy(None)
