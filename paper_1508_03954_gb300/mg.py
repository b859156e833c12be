"""Thin ctypes binding of the C ABI in include/mg.h.

Argument marshalling only: every step of the solver runs in the CUDA library
``_lib/libmg.so``.  The library must be built (``build.build()``); when it is
missing every entry point raises ``RuntimeError`` -- there is no CPU
fallback.  Arrays are numpy arrays (host) or torch CUDA tensors (device),
complex128, C-contiguous, fine-vertex layout with x fastest.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MG_OK, MG_ERR_INVALID, MG_ERR_CUDA, MG_ERR_OOM, MG_DIVERGED, MG_NOT_CONVERGED, MG_ERR_TIMEOUT = range(7)
MG_ADD, MG_HB, MG_BPX = 0, 1, 2
MG_DLINEAR, MG_HIERARCHICAL = 0, 1
MG_C128, MG_C64_REFINE = 0, 1
MG_OMEGA_JACOBI, MG_OMEGA_UCG, MG_OMEGA_LGRID, MG_OMEGA_EXP, MG_OMEGA_TRANSITION = range(5)

STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID", 2: "MG_ERR_CUDA", 3: "MG_ERR_OOM",
                4: "MG_DIVERGED", 5: "MG_NOT_CONVERGED", 6: "MG_ERR_TIMEOUT"}

# every symbol include/mg.h declares
EXPORTS = ["mg_create", "mg_create_ecs", "mg_create_adaptive", "mg_adapt", "mg_get_refinement", "mg_destroy", "mg_set_stream", "mg_set_rhs", "mg_set_solution",
           "mg_get_solution", "mg_cycle", "mg_residual_norm", "mg_residual_max", "mg_last_cycle_norm", "mg_solve", "mg_set_precision",
           "mg_fmg", "mg_omega_scheme", "mg_get_level", "mg_set_timing", "mg_get_stats",
           "mg_set_trace", "mg_get_trace", "mg_set_spin_limit", "mg_debug_unsatisfiable_wait", "mg_set_k2", "mg_set_rhs_vector", "mg_sample",
           "mg_set_rhs_samples", "mg_adjoint_grad", "mg_residual_noalloc", "mg_batch_create",
           "mg_batch_destroy", "mg_batch_get_ctx", "mg_batch_set_stream", "mg_batch_solve",
           "mg_batch_autotune", "mg_batch_launches", "mg_batch_last_error", "mg_last_error",
           "mg_mc_create", "mg_mc_set_stream", "mg_mc_set_rhs", "mg_mc_set_solution", "mg_mc_get_solution",
           "mg_mc_cycle", "mg_mc_residual_norm", "mg_mc_last_error", "mg_mc_destroy"]


class MgC128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class MgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is not built; run "
                           "paper_1508_03954_gb300.build.build() (no CPU fallback exists)")
    L = ctypes.CDLL(p)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pc = ctypes.POINTER(MgC128)
    sig = {
        "mg_create": (ip, [ip, ip, ctypes.POINTER(dp), dp, dp, ctypes.POINTER(vp)]),
        "mg_create_ecs": (ip, [ip, ip, ctypes.POINTER(dp), dp, dp, dp, dp, ctypes.POINTER(vp)]),
        "mg_create_adaptive": (ip, [ip, ip, ctypes.POINTER(dp), dp, dp, dp, dp, ctypes.c_char_p, ctypes.POINTER(vp)]),
        "mg_adapt": (ip, [vp, dp, dp, ip, dp, ip, ip, ctypes.POINTER(ctypes.c_longlong)]),
        "mg_get_refinement": (ip, [vp, ctypes.c_char_p]),
        "mg_destroy": (None, [vp]),
        "mg_set_stream": (ip, [vp, vp]),
        "mg_set_rhs": (ip, [vp, vp, ip]),
        "mg_set_solution": (ip, [vp, vp, ip]),
        "mg_get_solution": (ip, [vp, vp, ip]),
        "mg_cycle": (ip, [vp, ip, pc, ip]),
        "mg_residual_norm": (ip, [vp, ctypes.POINTER(dp), ctypes.POINTER(dp)]),
        "mg_last_cycle_norm": (ip, [vp, ctypes.POINTER(dp), ctypes.POINTER(dp)]),
        "mg_residual_max": (ip, [vp, ctypes.POINTER(dp)]),
        "mg_solve": (ip, [vp, ip, pc, ip, dp, ip, ctypes.POINTER(ip), ctypes.POINTER(dp)]),
        "mg_set_precision": (ip, [vp, ip, ip]),
        "mg_fmg": (ip, [vp, ip, pc, ip, ip]),
        "mg_omega_scheme": (ip, [ip, MgC128, ip, ip, ip, pc]),
        "mg_get_level": (ip, [vp, ip, ip, vp, ip]),
        "mg_set_timing": (ip, [vp, ip]),
        "mg_get_stats": (ip, [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ip),
                              ctypes.POINTER(dp)]),
        "mg_residual_noalloc": (ip, [vp, vp, vp, vp, vp]),
        "mg_set_trace": (ip, [vp, ip]),
        "mg_set_spin_limit": (ip, [vp, ctypes.c_uint]),
        "mg_debug_unsatisfiable_wait": (ip, [vp, ip]),
        "mg_set_k2": (ip, [vp, ctypes.c_void_p, ctypes.c_int]),
        "mg_set_rhs_vector": (ip, [vp, vp, ip]),
        "mg_sample": (ip, [vp, ip, ctypes.POINTER(dp), pc, pc]),
        "mg_set_rhs_samples": (ip, [vp, ip, ctypes.POINTER(dp), pc]),
        "mg_adjoint_grad": (ip, [vp, vp, vp, MgC128, vp, vp]),
        "mg_get_trace": (ip, [vp, vp, ip, ip]),
        "mg_batch_create": (ip, [ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ctypes.POINTER(dp)),
                                 ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(vp)]),
        "mg_batch_destroy": (None, [vp]),
        "mg_batch_get_ctx": (ip, [vp, ip, ctypes.POINTER(vp)]),
        "mg_batch_set_stream": (ip, [vp, vp]),
        "mg_batch_solve": (ip, [vp, ip, ctypes.POINTER(pc), ip, dp, ip, ip, ctypes.POINTER(ip),
                                ctypes.POINTER(ip), ctypes.POINTER(dp)]),
        "mg_batch_autotune": (ip, [vp, ip, ctypes.POINTER(pc), ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                   ctypes.POINTER(dp)]),
        "mg_batch_launches": (ctypes.c_longlong, [vp]),
        "mg_batch_last_error": (ctypes.c_char_p, [vp]),
        "mg_last_error": (ctypes.c_char_p, [vp]),
        "mg_mc_create": (ip, [ip, ip, ip, pc, dp, dp, ctypes.POINTER(vp)]),
        "mg_mc_set_stream": (ip, [vp, vp]),
        "mg_mc_set_rhs": (ip, [vp, vp, ip]),
        "mg_mc_set_solution": (ip, [vp, vp, ip]),
        "mg_mc_get_solution": (ip, [vp, vp, ip]),
        "mg_mc_cycle": (ip, [vp, ip, pc, ip]),
        "mg_mc_residual_norm": (ip, [vp, ctypes.POINTER(dp), ctypes.POINTER(dp)]),
        "mg_mc_last_error": (ctypes.c_char_p, [vp]),
        "mg_mc_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _omega_array(omega, depth):
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.complex128).reshape(-1))
    if om.shape[0] != depth:
        raise ValueError(f"omega needs {depth} entries (one per level)")
    arr = (MgC128 * depth)()
    for i, w in enumerate(om):
        arr[i].re, arr[i].im = float(w.real), float(w.imag)
    return arr


def _ptr(x, nvals):
    """(pointer, on_device, keepalive) of a complex128 array of nvals values."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        import torch
        if x.dtype != torch.complex128 or not x.is_contiguous() or x.numel() != nvals:
            raise ValueError("device arrays must be contiguous complex128 tensors of the fine size")
        return ctypes.c_void_p(x.data_ptr()), (1 if x.is_cuda else 0), x
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    if a.size != nvals:
        raise ValueError(f"expected {nvals} values, got {a.size}")
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def omega_scheme(scheme, omega_s, depth, iter_n=1, l_grid=0):
    L = load()
    out = (MgC128 * depth)()
    w = MgC128(float(np.real(omega_s)), float(np.imag(omega_s)))
    rc = L.mg_omega_scheme(scheme, w, depth, iter_n, l_grid, out)
    if rc != MG_OK:
        raise MgError(rc, "mg_omega_scheme")
    return np.array([complex(o.re, o.im) for o in out])


class Solver:
    """One solver context (mg_create .. mg_destroy)."""

    @classmethod
    def wrap(cls, handle, d, depth, owner):
        """A view of a context owned by someone else (a batch)."""
        self = cls.__new__(cls)
        self.d, self.depth = d, depth
        self.n = 3 ** depth
        self.shape = (self.n + 1,) * d
        self.nv = (self.n + 1) ** d
        self._h = None  # never destroyed through this view
        self._view = handle
        self._owner = owner
        self._L = load()
        return self

    def __init__(self, d, depth, k2_field, theta, layer_width, theta_interior=0.0):
        """layer_width: w (a layer of width w at both faces of every axis,
        mg_create) or a pair (w_lo, w_hi) of one-sided widths; with a pair or
        a nonzero theta_interior the context comes from mg_create_ecs."""
        L = load()
        self.d, self.depth = d, depth
        self.n = 3 ** depth
        self.shape = (self.n + 1,) * d
        self.nv = (self.n + 1) ** d
        k2 = np.ascontiguousarray(np.asarray(k2_field, dtype=np.float64))
        if k2.size != self.nv:
            raise ValueError(f"k2_field needs {self.nv} values")
        h = ctypes.c_void_p()
        kp = k2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if np.ndim(layer_width) == 0 and theta_interior == 0.0:
            rc = L.mg_create(d, depth, kp, float(theta), float(layer_width), ctypes.byref(h))
        else:
            lo, hi = (layer_width, layer_width) if np.ndim(layer_width) == 0 else layer_width
            rc = L.mg_create_ecs(d, depth, kp, float(theta), float(theta_interior), float(lo), float(hi),
                                 ctypes.byref(h))
        if rc != MG_OK:
            raise MgError(rc, L.mg_last_error(None).decode())
        self._h = h
        self._view = h
        self._L = L

    @classmethod
    def adaptive(cls, d, depth, k2_field, theta, layer_width, refine, theta_interior=0.0):
        """A solver on an adaptive spacetree (mg_create_adaptive): refine maps
        level l = 1..depth-1 to a boolean array of its (3^l,)*d cells (numpy
        axis order, last axis = x); layer_width is w or a pair (w_lo, w_hi)
        as for the regular solver."""
        L = load()
        self = cls.__new__(cls)
        self.d, self.depth = d, depth
        self.n = 3 ** depth
        self.shape = (self.n + 1,) * d
        self.nv = (self.n + 1) ** d
        k2 = np.ascontiguousarray(np.asarray(k2_field, dtype=np.float64))
        if k2.size != self.nv:
            raise ValueError(f"k2_field needs {self.nv} values")
        flags = b"".join(np.ascontiguousarray(np.asarray(refine[lev], dtype=np.uint8)).tobytes()
                         for lev in range(1, depth))
        for lev in range(1, depth):
            if np.asarray(refine[lev]).size != 3 ** (lev * d):
                raise ValueError(f"refine[{lev}] needs {3 ** (lev * d)} flags")
        h = ctypes.c_void_p()
        lo, hi = (layer_width, layer_width) if np.ndim(layer_width) == 0 else layer_width
        rc = L.mg_create_adaptive(d, depth, k2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(theta),
                                  float(theta_interior), float(lo), float(hi), flags if flags else b"\0",
                                  ctypes.byref(h))
        if rc != MG_OK:
            raise MgError(rc, L.mg_last_error(None).decode())
        self._h = h
        self._view = h
        self._L = L
        return self

    # -- helpers
    def _check(self, rc, what):
        if rc not in (MG_OK,):
            raise MgError(rc, f"{what}: {self._L.mg_last_error(self._view).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.mg_destroy(self._h)
            self._h = None
            self._view = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def set_stream(self, stream_handle):
        self._check(self._L.mg_set_stream(self._view, ctypes.c_void_p(stream_handle)), "mg_set_stream")

    def set_rhs(self, f):
        p, dev, _keep = _ptr(f, self.nv)
        self._check(self._L.mg_set_rhs(self._view, p, dev), "mg_set_rhs")

    def set_solution(self, u):
        p, dev, _keep = _ptr(u, self.nv)
        self._check(self._L.mg_set_solution(self._view, p, dev), "mg_set_solution")

    def get_solution(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        p, dev, _keep = _ptr(out, self.nv)
        self._check(self._L.mg_get_solution(self._view, p, dev), "mg_get_solution")
        return out

    def get_level(self, level, which):
        n = 3 ** level
        out = np.empty(((n + 1),) * self.d, dtype=np.complex128)
        rc = self._L.mg_get_level(self._view, level, which, out.ctypes.data_as(ctypes.c_void_p), 0)
        self._check(rc, "mg_get_level")
        return out

    def cycle(self, variant, omega, transfer):
        self._check(self._L.mg_cycle(self._view, variant, _omega_array(omega, self.depth), transfer),
                    "mg_cycle")

    def residual_norm(self):
        a, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.mg_residual_norm(self._view, ctypes.byref(a), ctypes.byref(r)),
                    "mg_residual_norm")
        return a.value, r.value

    def adapt(self, min_level, refine_frac=0.1, erase_frac=0.02, bins=20, veto=1e-2, veto_relative=False):
        """One step of feature-based refinement (mg_adapt).  Returns (vertices
        selected for refining, for erasing, fine-grid vertices after the
        step, finest level with cells); raises MgError on MG_DIVERGED."""
        st = (ctypes.c_longlong * 4)()
        self._check(self._L.mg_adapt(self._view, float(refine_frac), float(erase_frac), int(bins), float(veto),
                                     1 if veto_relative else 0, int(min_level), st), "mg_adapt")
        return tuple(int(x) for x in st)

    def refinement(self):
        """The current refine flags {l: bool array of level l's cells}
        (mg_get_refinement), levels 1..depth-1."""
        sizes = [3 ** (lev * self.d) for lev in range(1, self.depth)]
        buf = ctypes.create_string_buffer(max(1, sum(sizes)))
        self._check(self._L.mg_get_refinement(self._view, buf), "mg_get_refinement")
        raw = np.frombuffer(buf.raw, dtype=np.uint8)
        out, off = {}, 0
        for lev, sz in zip(range(1, self.depth), sizes):
            out[lev] = raw[off:off + sz].reshape((3 ** lev,) * self.d).astype(bool)
            off += sz
        return out

    def residual_max(self):
        """Maximum modulus of the fine residual (mg_residual_max)."""
        a = ctypes.c_double()
        self._check(self._L.mg_residual_max(self._view, ctypes.byref(a)), "mg_residual_max")
        return a.value

    def last_cycle_norm(self):
        a, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.mg_last_cycle_norm(self._view, ctypes.byref(a), ctypes.byref(r)),
                    "mg_last_cycle_norm")
        return a.value, r.value

    def solve(self, variant, omega, transfer, tol, max_cycles):
        """Returns (status, cycles_done, rel_res); MG_DIVERGED and
        MG_NOT_CONVERGED are returned, not raised."""
        n, rel = ctypes.c_int(), ctypes.c_double()
        rc = self._L.mg_solve(self._view, variant, _omega_array(omega, self.depth), transfer,
                              float(tol), int(max_cycles), ctypes.byref(n), ctypes.byref(rel))
        if rc not in (MG_OK, MG_DIVERGED, MG_NOT_CONVERGED):
            self._check(rc, "mg_solve")
        return rc, n.value, rel.value

    def set_precision(self, precision, inner_cycles):
        self._check(self._L.mg_set_precision(self._view, precision, inner_cycles), "mg_set_precision")

    def set_timing(self, enable):
        self._check(self._L.mg_set_timing(self._view, 1 if enable else 0), "mg_set_timing")

    def get_stats(self):
        """(kernel launches, timed fine sweeps, their device ms) since the last call."""
        n, k, ms = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_double()
        self._check(self._L.mg_get_stats(self._view, ctypes.byref(n), ctypes.byref(k), ctypes.byref(ms)),
                    "mg_get_stats")
        return n.value, k.value, ms.value

    def set_k2(self, k2):
        """Fine k^2 field: a host array, or a contiguous float64 CUDA tensor
        (copied and turned into cell shifts on the solver's stream)."""
        if hasattr(k2, "data_ptr") and hasattr(k2, "is_cuda") and k2.is_cuda:
            import torch
            if k2.dtype != torch.float64 or not k2.is_contiguous() or k2.numel() != self.nv:
                raise ValueError(f"k2 on the device must be a contiguous float64 tensor of {self.nv} values")
            self._check(self._L.mg_set_k2(self._view, ctypes.c_void_p(k2.data_ptr()), 1), "mg_set_k2")
            return
        a = np.ascontiguousarray(np.asarray(k2, dtype=np.float64))
        if a.size != self.nv:
            raise ValueError(f"k2 needs {self.nv} values")
        self._check(self._L.mg_set_k2(self._view, a.ctypes.data_as(ctypes.c_void_p), 0), "mg_set_k2")

    def set_rhs_vector(self, b):
        p, dev, _keep = _ptr(b, self.nv)
        self._check(self._L.mg_set_rhs_vector(self._view, p, dev), "mg_set_rhs_vector")

    @staticmethod
    def _samples(xyz, w):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64))
        w = np.ascontiguousarray(np.asarray(w, dtype=np.complex128).reshape(-1))
        wa = (MgC128 * len(w))()
        for i, z in enumerate(w):
            wa[i].re, wa[i].im = float(z.real), float(z.imag)
        return xyz, wa, len(w)

    def sample(self, xyz, w):
        """s = sum_q w_q u(x_q); xyz shape (npts, d) with x first."""
        xyz, wa, m = self._samples(xyz, w)
        out = MgC128()
        self._check(self._L.mg_sample(self._view, m, xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), wa,
                                      ctypes.byref(out)), "mg_sample")
        return complex(out.re, out.im)

    def set_rhs_samples(self, xyz, w):
        xyz, wa, m = self._samples(xyz, w)
        self._check(self._L.mg_set_rhs_samples(self._view, m, xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               wa), "mg_set_rhs_samples")

    def adjoint_grad(self, u, lam, s, dJdV=None, dJdf=None):
        """Device tensors: u, lam complex128 (fine size); dJdV, dJdf float64 (fine size) or None."""
        for t in (u, lam):
            if not (t.is_cuda and t.is_contiguous() and t.numel() == self.nv):
                raise ValueError("u and lam must be contiguous CUDA tensors of the fine size")
        outs = []
        for t in (dJdV, dJdf):
            if t is None:
                outs.append(None)
            else:
                if not (t.is_cuda and t.is_contiguous() and t.numel() == self.nv):
                    raise ValueError("gradient outputs must be contiguous float64 CUDA tensors")
                outs.append(ctypes.c_void_p(t.data_ptr()))
        self._check(self._L.mg_adjoint_grad(self._view, ctypes.c_void_p(u.data_ptr()),
                                            ctypes.c_void_p(lam.data_ptr()),
                                            MgC128(float(np.real(s)), float(np.imag(s))), outs[0], outs[1]),
                    "mg_adjoint_grad")

    def set_spin_limit(self, polls):
        self._check(self._L.mg_set_spin_limit(self._view, int(polls)), "mg_set_spin_limit")

    def debug_unsatisfiable_wait(self, enable):
        self._check(self._L.mg_debug_unsatisfiable_wait(self._view, 1 if enable else 0),
                    "mg_debug_unsatisfiable_wait")

    def set_trace(self, enable):
        self._check(self._L.mg_set_trace(self._view, 1 if enable else 0), "mg_set_trace")

    def get_trace(self, fine_slots, chain_slots):
        """(fine, chain) uint64 arrays of shape (slots, 4): taken, ready, done (ns), SM."""
        out = np.zeros((fine_slots + chain_slots, 4), dtype=np.uint64)
        self._check(self._L.mg_get_trace(self._view, out.ctypes.data_as(ctypes.c_void_p), fine_slots,
                                         chain_slots), "mg_get_trace")
        return out[:fine_slots], out[fine_slots:]

    def residual_noalloc(self, u, b, r, norm2):
        """r = b - H_L u and |r|^2 into caller-owned device tensors, using
        the library's static scratch instead of any allocation.  u, b, r:
        complex128 CUDA tensors of the fine size (r may be None); norm2: a
        float64 CUDA tensor with at least one element."""
        import torch
        for t in (u, b):
            if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
                    and t.numel() == self.nv):
                raise ValueError("u and b must be contiguous complex128 CUDA tensors of the fine size")
        if r is not None and not (r.is_cuda and r.dtype == torch.complex128 and r.is_contiguous()
                                  and r.numel() == self.nv):
            raise ValueError("r must be a contiguous complex128 CUDA tensor of the fine size")
        if not (norm2.is_cuda and norm2.dtype == torch.float64 and norm2.numel() >= 1):
            raise ValueError("norm2 must be a float64 CUDA tensor")
        rp = ctypes.c_void_p(r.data_ptr()) if r is not None else None
        self._check(self._L.mg_residual_noalloc(self._view, ctypes.c_void_p(u.data_ptr()),
                                                ctypes.c_void_p(b.data_ptr()), rp,
                                                ctypes.c_void_p(norm2.data_ptr())),
                    "mg_residual_noalloc")

    def get_level_device(self, level, which, out):
        """Copies a per-level array into a caller-owned complex128 CUDA tensor."""
        rc = self._L.mg_get_level(self._view, level, which, ctypes.c_void_p(out.data_ptr()), 1)
        self._check(rc, "mg_get_level")
        return out

    def fmg(self, variant, omega, transfer, cycles_per_stage):
        self._check(self._L.mg_fmg(self._view, variant, _omega_array(omega, self.depth), transfer,
                                   cycles_per_stage), "mg_fmg")


# module-level names matching the C ABI
def mg_create(d, depth, k2_field, theta, layer_width):
    return Solver(d, depth, k2_field, theta, layer_width)


def mg_destroy(s):
    s.close()


def mg_set_stream(s, stream):
    s.set_stream(stream)


def mg_set_rhs(s, f):
    s.set_rhs(f)


def mg_set_solution(s, u):
    s.set_solution(u)


def mg_get_solution(s, out=None):
    return s.get_solution(out)


def mg_cycle(s, variant, omega, transfer):
    s.cycle(variant, omega, transfer)


def mg_residual_norm(s):
    return s.residual_norm()


def mg_solve(s, variant, omega, transfer, tol, max_cycles):
    return s.solve(variant, omega, transfer, tol, max_cycles)


def mg_set_precision(s, precision, inner_cycles):
    s.set_precision(precision, inner_cycles)


def mg_fmg(s, variant, omega, transfer, cycles_per_stage):
    s.fmg(variant, omega, transfer, cycles_per_stage)


def mg_omega_scheme(scheme, omega_s, depth, iter_n=1, l_grid=0):
    return omega_scheme(scheme, omega_s, depth, iter_n, l_grid)


class Batch:
    """Many 2D problems solved together (mg_batch_*)."""

    def __init__(self, specs):
        """specs: list of dicts with d, depth, k2 (constant field), theta, layer_width."""
        L = load()
        n = len(specs)
        self._keep = [np.ascontiguousarray(np.asarray(sp["k2"], dtype=np.float64)) for sp in specs]
        d = (ctypes.c_int * n)(*[sp["d"] for sp in specs])
        dep = (ctypes.c_int * n)(*[sp["depth"] for sp in specs])
        th = (ctypes.c_double * n)(*[sp["theta"] for sp in specs])
        lw = (ctypes.c_double * n)(*[sp["layer_width"] for sp in specs])
        kp = (ctypes.POINTER(ctypes.c_double) * n)(*[k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                                      for k in self._keep])
        h = ctypes.c_void_p()
        rc = L.mg_batch_create(n, d, dep, kp, th, lw, ctypes.byref(h))
        if rc != MG_OK:
            raise MgError(rc, L.mg_last_error(None).decode())
        self._h, self._L, self.n = h, L, n
        self.depths = [sp["depth"] for sp in specs]
        self.solvers = []
        for p in range(n):
            ch = ctypes.c_void_p()
            L.mg_batch_get_ctx(h, p, ctypes.byref(ch))
            self.solvers.append(Solver.wrap(ch, specs[p]["d"], specs[p]["depth"], self))

    def _om(self, omegas):
        arrs = [_omega_array(omegas[p], self.depths[p]) for p in range(self.n)]
        self._om_keep = arrs
        return (ctypes.POINTER(MgC128) * self.n)(*[ctypes.cast(a, ctypes.POINTER(MgC128)) for a in arrs])

    def _check(self, rc, what):
        if rc != MG_OK:
            raise MgError(rc, f"{what}: {self._L.mg_batch_last_error(self._h).decode()}")

    def set_stream(self, stream_handle):
        self._check(self._L.mg_batch_set_stream(self._h, ctypes.c_void_p(stream_handle)), "mg_batch_set_stream")

    def solve(self, variant, omegas, transfer, tol, max_outer, inner_cycles):
        """Returns (status[n], inner cycles[n], rel_res[n])."""
        st = (ctypes.c_int * self.n)()
        cy = (ctypes.c_int * self.n)()
        rl = (ctypes.c_double * self.n)()
        rc = self._L.mg_batch_solve(self._h, variant, self._om(omegas), transfer, float(tol), int(max_outer),
                                    int(inner_cycles), st, cy, rl)
        self._check(rc, "mg_batch_solve")
        return list(st), list(cy), list(rl)

    def autotune(self, variant, omegas, transfer, inner_cycles):
        tc, bp, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        rc = self._L.mg_batch_autotune(self._h, variant, self._om(omegas), transfer, int(inner_cycles),
                                       ctypes.byref(tc), ctypes.byref(bp), ctypes.byref(ms))
        self._check(rc, "mg_batch_autotune")
        return tc.value, bp.value, ms.value

    def launches(self):
        return self._L.mg_batch_launches(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.mg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiChannel:
    """Coupled multichannel context (mg_mc_create .. mg_mc_destroy): c channels
    per vertex, A = I (x) K - Phi (x) M.  Tuple arrays have shape
    (N, .., N, c) (channel fastest) or the same values flattened."""

    def __init__(self, d, depth, phi, theta, layer_width):
        self._L = load()
        phi = np.asarray(phi, dtype=np.complex128)
        if phi.ndim != 2 or phi.shape[0] != phi.shape[1]:
            raise ValueError("phi must be a square matrix")
        self.d, self.depth, self.c = d, depth, phi.shape[0]
        self.n = 3 ** depth
        self.nv = (self.n + 1) ** d
        self.shape = (self.n + 1,) * d + (self.c,)
        arr = (MgC128 * phi.size)()
        for k, z in enumerate(phi.reshape(-1)):
            arr[k].re, arr[k].im = float(z.real), float(z.imag)
        h = ctypes.c_void_p()
        rc = self._L.mg_mc_create(d, depth, self.c, arr, float(theta), float(layer_width), ctypes.byref(h))
        if rc != MG_OK:
            raise MgError(rc, "mg_mc_create")
        self._h = h

    def _check(self, rc, what):
        if rc != MG_OK:
            msg = self._L.mg_mc_last_error(self._h)
            raise MgError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.mg_mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self._L.mg_mc_set_stream(self._h, ctypes.c_void_p(stream)), "mg_mc_set_stream")

    def set_rhs(self, f):
        p, dev, _keep = _ptr(f, self.nv * self.c)
        self._check(self._L.mg_mc_set_rhs(self._h, p, dev), "mg_mc_set_rhs")

    def set_solution(self, u):
        p, dev, _keep = _ptr(u, self.nv * self.c)
        self._check(self._L.mg_mc_set_solution(self._h, p, dev), "mg_mc_set_solution")

    def get_solution(self, out=None):
        if out is None:
            a = np.empty(self.shape, dtype=np.complex128)
            self._check(self._L.mg_mc_get_solution(self._h, a.ctypes.data_as(ctypes.c_void_p), 0),
                        "mg_mc_get_solution")
            return a
        p, dev, _keep = _ptr(out, self.nv * self.c)
        self._check(self._L.mg_mc_get_solution(self._h, p, dev), "mg_mc_get_solution")
        return out

    def cycle(self, variant, omega, transfer):
        self._check(self._L.mg_mc_cycle(self._h, variant, _omega_array(omega, self.depth), transfer), "mg_mc_cycle")

    def residual_norm(self):
        a, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.mg_mc_residual_norm(self._h, ctypes.byref(a), ctypes.byref(r)), "mg_mc_residual_norm")
        return a.value, r.value
