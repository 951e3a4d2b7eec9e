"""Thin Python binding of libhs (include/hs.h): same names, argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory
(state tensors) and streams.  There is no CPU fallback: if the compiled
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HS_OK, HS_EINVAL, HS_ENOMEM, HS_ECUDA, HS_ETIMEOUT, HS_EDTYPE = 0, -1, -2, -3, -4, -5
HS_C64, HS_C128 = 1, 2
HS_METHOD_AUTO, HS_METHOD_PLAIN, HS_METHOD_FUSED, HS_METHOD_REG = 0, 1, 2, 3
HS_BUILD_DEFER_DIAGONALS = 1
HS_MAX_QUBITS = 30

_HERE = os.path.dirname(os.path.abspath(__file__))
# HS_DEBUG_BOUNDS=1 in the environment selects the index-checking build
# (_build.build(debug=True)); otherwise the ordinary one.
DEBUG_BOUNDS = os.environ.get("HS_DEBUG_BOUNDS", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "_build_debug" if DEBUG_BOUNDS else "_build", "libhs.so")

# Every symbol declared in include/hs.h and include/hs_dia.h.
EXPORTS = (
    "hs_build_factors", "hs_build_factors_masks", "hs_evolve", "hs_evolve_ex", "hs_apply_factor",
    "hs_fidelity", "hs_inner_device", "hs_factors_info", "hs_factor_get", "hs_free_factors", "hs_last_error",
    "hs_plan_factors", "hs_plan_schedule", "hs_evolve_plan", "hs_evolve_td_plan", "hs_inner_batch_noalloc", "hs_autotune",
    "hs_batch_create", "hs_batch_launch", "hs_batch_info", "hs_batch_free", "hs_free_factors_async",
    "hs_batch_free_async",
    "hs_dia_from_terms", "hs_dia_from_masks", "hs_dia_create", "hs_spgemm", "hs_spme", "hs_estimate_timesteps",
    "hs_spmv", "hs_dia_evolve", "hs_dia_convert", "hs_dia_info", "hs_dia_get", "hs_dia_free",
    "hs_kernel_launches", "hs_debug_bounds", "hs_expectation", "hs_build_factors_ex", "hs_build_factors_flags", "hs_factors_sequence",
    "hs_build_factors_td", "hs_evolve_td", "hs_factors_set_drive", "hs_dia_evolve_td",
    "hs_parse_terms", "hs_evolve_batch", "hs_batch_autotune",
)


class HSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libhs error {code}: {msg}")
        self.code = code


class BatchJob(ctypes.Structure):
    _fields_ = [("factors", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("n_rhs", ctypes.c_int),
                ("n_steps", ctypes.c_int)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int), ("low_bits", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("smem_kb", ctypes.c_int), ("no_tables", ctypes.c_int), ("tiles_per_cta", ctypes.c_int),
                ("method", ctypes.c_int), ("reg_bits", ctypes.c_int)]


class EvolveOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("tile_bits", ctypes.c_int), ("rhs_block", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("low_bits", ctypes.c_int), ("max_fuse", ctypes.c_int),
                ("smem_kb", ctypes.c_int), ("no_tables", ctypes.c_int), ("reg_bits", ctypes.c_int)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libhs.so (built by __graft_entry__.build()); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhs.so not found at {LIB_PATH}: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        L.hs_build_factors.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(d), sz, d, i, i, i, vp,
                                       ctypes.POINTER(vp)]
        L.hs_build_factors_masks.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(d), sz, i, d, i, i, i, vp, ctypes.POINTER(vp)]
        L.hs_evolve.argtypes = [vp, vp, i, i, vp]
        L.hs_evolve_ex.argtypes = [vp, vp, i, i, ctypes.POINTER(EvolveOpts), vp]
        L.hs_apply_factor.argtypes = [vp, i, vp, vp, i, vp]
        L.hs_fidelity.argtypes = [vp, vp, i, i, vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]
        L.hs_inner_device.argtypes = [vp, vp, i, i, vp, vp]
        L.hs_factors_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(ctypes.c_int64)]
        L.hs_factor_get.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(d)]
        ip, i64p = ctypes.POINTER(i), ctypes.POINTER(ctypes.c_int64)
        L.hs_plan_factors.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), sz, i, i, i,
                                      ip, ip, ip, ip, ip, i64p, i64p, i, i]
        L.hs_plan_schedule.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), sz, i, i, i,
                                       i, i, i, i, i, i, ip, ip, ip, ip, ip, i]
        L.hs_evolve_plan.argtypes = [vp, i, i, ctypes.POINTER(EvolveOpts), ip, ip, ip, ip]
        L.hs_evolve_td_plan.argtypes = [vp, i, i, ctypes.POINTER(EvolveOpts), ip, ip, ip, ip]
        L.hs_inner_batch_noalloc.argtypes = [vp, vp, i, i, i, vp, vp]
        L.hs_autotune.argtypes = [vp, vp, i, i, vp, ctypes.POINTER(EvolveOpts)]
        L.hs_batch_create.argtypes = [ctypes.POINTER(BatchJob), sz, ctypes.POINTER(BatchOpts), ctypes.POINTER(vp)]
        L.hs_batch_launch.argtypes = [vp, vp]
        L.hs_batch_info.argtypes = [vp, ip, i64p, i64p, ip]
        L.hs_batch_free.argtypes = [vp]
        L.hs_free_factors_async.argtypes = [vp, vp]
        L.hs_batch_free_async.argtypes = [vp, vp]
        L.hs_batch_free.restype = None
        L.hs_free_factors.argtypes = [vp]
        L.hs_free_factors.restype = None
        L.hs_last_error.restype = ctypes.c_char_p
        dp = ctypes.POINTER(d)
        L.hs_dia_from_terms.argtypes = [ctypes.POINTER(ctypes.c_char_p), dp, sz, vp, ctypes.POINTER(vp)]
        L.hs_dia_from_masks.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), dp, sz, i,
                                        vp, ctypes.POINTER(vp)]
        L.hs_dia_create.argtypes = [i, i64p, sz, dp, i, vp, ctypes.POINTER(vp)]
        L.hs_spgemm.argtypes = [vp, vp, vp, ctypes.POINTER(vp), dp]
        L.hs_spme.argtypes = [vp, d, d, i, vp, ctypes.POINTER(vp), ip, ip]
        L.hs_estimate_timesteps.argtypes = [vp, d, i, d, i, i, vp, ip]
        L.hs_spmv.argtypes = [vp, vp, vp, i, vp]
        L.hs_dia_evolve.argtypes = [vp, vp, i, i, vp]
        L.hs_dia_convert.argtypes = [vp, i, vp, ctypes.POINTER(vp)]
        L.hs_dia_info.argtypes = [vp, ip, ip, i64p, ip]
        L.hs_dia_get.argtypes = [vp, i64p, dp]
        L.hs_dia_free.argtypes = [vp]
        L.hs_dia_free.restype = None
        L.hs_expectation.argtypes = [vp, vp, i, vp, dp, dp]
        L.hs_build_factors_ex.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                          dp, sz, i, d, i, i, i, i, vp, ctypes.POINTER(vp)]
        L.hs_build_factors_flags.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                             dp, sz, i, d, i, i, i, i, i, vp, ctypes.POINTER(vp)]
        L.hs_factors_sequence.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), i, ctypes.POINTER(i)]
        L.hs_build_factors_td.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                          dp, dp, sz, i, d, i, i, i, i, vp, ctypes.POINTER(vp)]
        L.hs_evolve_td.argtypes = [vp, vp, i, dp, i, ctypes.POINTER(EvolveOpts), vp]
        L.hs_factors_set_drive.argtypes = [vp, d, vp]
        L.hs_dia_evolve_td.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), dp, dp, sz,
                                       i, d, dp, i, d, i, vp, i, i, vp]
        L.hs_parse_terms.argtypes = [ctypes.POINTER(ctypes.c_char_p), sz, ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i)]
        L.hs_evolve_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(i), sz,
                                      vp]
        L.hs_batch_autotune.argtypes = [ctypes.POINTER(BatchJob), sz, vp, ctypes.POINTER(BatchOpts)]
        L.hs_kernel_launches.argtypes = []
        L.hs_kernel_launches.restype = ctypes.c_uint64
        L.hs_debug_bounds.argtypes = [ctypes.POINTER(ctypes.c_uint64), i]
        for name in EXPORTS:
            if name not in ("hs_free_factors", "hs_last_error", "hs_batch_free", "hs_dia_free", "hs_kernel_launches"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def hs_debug_bounds(reset: bool = False):
    """Index-check record of the library: None for the ordinary build, else
    (failures, site, index, extent) of the first failure (zeros when none)."""
    w = (ctypes.c_uint64 * 4)()
    rc = lib().hs_debug_bounds(w, int(bool(reset)))
    if rc < 0:
        _check(rc)
    return None if rc == 0 else tuple(int(v) for v in w)


def hs_kernel_launches() -> int:
    """Kernels launched through libhs so far in this process."""
    return int(lib().hs_kernel_launches())


def _check(rc: int):
    if rc != HS_OK:
        raise HSError(rc, lib().hs_last_error().decode(errors="replace"))


def _dtype_code(dtype) -> int:
    import torch
    if dtype in ("c64", torch.complex64, HS_C64):
        return HS_C64
    if dtype in ("c128", torch.complex128, HS_C128):
        return HS_C128
    raise ValueError(f"unsupported dtype {dtype!r}")


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _state_args(psi):
    """(pointer, n_rhs, n_qubits, dtype code) of a CUDA state tensor (N,) or (R, N)."""
    import torch
    if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
        raise TypeError("state must be a CUDA tensor")
    if not psi.is_contiguous():
        raise ValueError("state must be contiguous")
    N = psi.shape[-1]
    n = int(N).bit_length() - 1
    if N != 1 << n:
        raise ValueError("state length must be a power of two")
    n_rhs = 1 if psi.dim() == 1 else int(np.prod(psi.shape[:-1]))
    return psi.data_ptr(), n_rhs, n, _dtype_code(psi.dtype)


class Factors:
    """Owner of an hs_factors handle (freed on close or garbage collection)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        nf, nq, ns, dt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        vb = ctypes.c_int64()
        _check(lib().hs_factors_info(self.handle, ctypes.byref(nf), ctypes.byref(nq), ctypes.byref(ns),
                                     ctypes.byref(dt), ctypes.byref(vb)))
        self.n_factors, self.n_qubits, self.n_steps, self.dtype_code = nf.value, nq.value, ns.value, dt.value
        order, ln = ctypes.c_int(), ctypes.c_int()
        _check(lib().hs_factors_sequence(self.handle, ctypes.byref(order), None, 0, ctypes.byref(ln)))
        seq = (ctypes.c_int * max(1, ln.value))()
        _check(lib().hs_factors_sequence(self.handle, None, seq, ln.value, ctypes.byref(ln)))
        self.order = order.value
        self.sequence = [int(seq[k]) for k in range(ln.value)]  # factors one step applies
        self.value_bytes = vb.value

    @property
    def dtype(self) -> str:
        return "c64" if self.dtype_code == HS_C64 else "c128"

    def factor(self, g: int, values: bool = True):
        """(term_first, term_last, offsets, values) of factor g; values as complex128 (the Eq. 6 view)."""
        tf, tl, nd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().hs_factor_get(self.handle, g, ctypes.byref(tf), ctypes.byref(tl), ctypes.byref(nd), None, None))
        offs = np.zeros(nd.value, dtype=np.int64)
        N = 1 << self.n_qubits
        _check(lib().hs_factor_get(self.handle, g, None, None, None,
                                   offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None))
        vals = None
        if values:
            S = int(np.sum(N - np.abs(offs)))
            buf = np.zeros(2 * S, dtype=np.float64)
            _check(lib().hs_factor_get(self.handle, g, None, None, None, None,
                                       buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
            vals = buf.view(np.complex128)
        return tf.value, tl.value, offs, vals

    def close(self, stream=None):
        """Free the factor set; with a stream, in stream order without synchronising."""
        if self.handle and self.handle.value:
            if _lib is not None:
                if stream is None:
                    _lib.hs_free_factors(self.handle)
                else:
                    _lib.hs_free_factors_async(self.handle, _stream(stream))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hs_parse_terms(labels: Sequence[str]):
    """(x, z, n_qubits) of Pauli labels, parsed by the library (rightmost
    character = qubit 0)."""
    n_terms = len(labels)
    arr = (ctypes.c_char_p * max(1, n_terms))(*[l.encode() for l in labels])
    x = np.zeros(max(1, n_terms), dtype=np.uint64)
    z = np.zeros(max(1, n_terms), dtype=np.uint64)
    nq = ctypes.c_int()
    _check(lib().hs_parse_terms(arr, n_terms, x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(nq)))
    return x[:n_terms], z[:n_terms], nq.value


def hs_build_factors(labels: Sequence[str], coeffs, t: float, n_steps: int, diag_budget: int, dtype="c64",
                     stream=None, order: int = 1, defer_diagonals: bool = False) -> Factors:
    """defer_diagonals: HS_BUILD_DEFER_DIAGONALS (the stored diagonals are built
    by the first call that reads them; register sweeps never do)."""
    if order != 1 or defer_diagonals:
        x, z, n = hs_parse_terms(labels)
        return hs_build_factors_masks(x, z, coeffs, n, t, n_steps, diag_budget, dtype, stream, order,
                                      defer_diagonals)
    arr = (ctypes.c_char_p * len(labels))(*[l.encode() for l in labels])
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if c.size != len(labels):
        raise ValueError("one coefficient per label")
    out = ctypes.c_void_p()
    _check(lib().hs_build_factors(arr, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(labels), float(t),
                                  int(n_steps), int(diag_budget), _dtype_code(dtype), _stream(stream),
                                  ctypes.byref(out)))
    return Factors(out.value)


def hs_build_factors_masks(x, z, coeffs, n_qubits: int, t: float, n_steps: int, diag_budget: int, dtype="c64",
                           stream=None, order: int = 1, defer_diagonals: bool = False) -> Factors:
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    za = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if not (xa.size == za.size == c.size):
        raise ValueError("x, z and coeffs differ in length")
    out = ctypes.c_void_p()
    _check(lib().hs_build_factors_flags(xa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                        za.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), xa.size, int(n_qubits),
                                        float(t), int(n_steps), int(diag_budget), int(order), _dtype_code(dtype),
                                        HS_BUILD_DEFER_DIAGONALS if defer_diagonals else 0, _stream(stream),
                                        ctypes.byref(out)))
    return Factors(out.value)


def hs_build_factors_td(x, z, coeffs0, coeffs1, n_qubits: int, t: float, n_steps: int, diag_budget: int,
                        dtype="c64", stream=None, order: int = 1) -> Factors:
    """Factor set of H(t) = H0 + f(t) H1 (term j: coeffs0[j] in H0, coeffs1[j]
    in H1), values built for f = 0; evolve it with hs_evolve_td."""
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    za = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    a = np.ascontiguousarray(np.asarray(coeffs0, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(coeffs1, dtype=np.float64))
    if not (xa.size == za.size == a.size == b.size):
        raise ValueError("x, z, coeffs0 and coeffs1 differ in length")
    out = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().hs_build_factors_td(xa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                     za.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                     a.ctypes.data_as(dp), b.ctypes.data_as(dp), xa.size, int(n_qubits), float(t),
                                     int(n_steps), int(diag_budget), int(order), _dtype_code(dtype),
                                     _stream(stream), ctypes.byref(out)))
    return Factors(out.value)


def _check_state(f: Factors, psi):
    ptr, n_rhs, n, code = _state_args(psi)
    if n != f.n_qubits:
        raise ValueError(f"state has {n} qubits, factors {f.n_qubits}")
    if code != f.dtype_code:
        raise HSError(HS_EDTYPE, "state dtype differs from the factors' dtype")
    return ptr, n_rhs


def hs_evolve(f: Factors, psi, n_steps: int, stream=None) -> None:
    ptr, n_rhs = _check_state(f, psi)
    _check(lib().hs_evolve(f.handle, ptr, n_rhs, int(n_steps), _stream(stream)))


def _opts(method, tile_bits, rhs_block, use_graph, low_bits, max_fuse, smem_kb, no_tables, reg_bits) -> EvolveOpts:
    return EvolveOpts(int(method), int(tile_bits), int(rhs_block), int(bool(use_graph)), int(low_bits), int(max_fuse),
                      int(smem_kb), int(bool(no_tables)), int(reg_bits))


def hs_evolve_ex(f: Factors, psi, n_steps: int, method: int = HS_METHOD_AUTO, tile_bits: int = 0,
                 rhs_block: int = 0, use_graph: bool = False, low_bits: int = 0, max_fuse: int = 0, smem_kb: int = 0,
                 no_tables: bool = False, reg_bits: int = 0, stream=None) -> None:
    ptr, n_rhs = _check_state(f, psi)
    o = _opts(method, tile_bits, rhs_block, use_graph, low_bits, max_fuse, smem_kb, no_tables, reg_bits)
    _check(lib().hs_evolve_ex(f.handle, ptr, n_rhs, int(n_steps), ctypes.byref(o), _stream(stream)))


def hs_evolve_td(f: Factors, psi, drive, method: int = HS_METHOD_AUTO, tile_bits: int = 0, rhs_block: int = 0,
                 use_graph: bool = False, low_bits: int = 0, max_fuse: int = 0, smem_kb: int = 0,
                 no_tables: bool = False, reg_bits: int = 0, stream=None) -> None:
    """One step per entry of `drive` (the frozen value of f for that step)."""
    ptr, n_rhs = _check_state(f, psi)
    fv = np.ascontiguousarray(np.asarray(drive, dtype=np.float64).ravel())
    o = _opts(method, tile_bits, rhs_block, use_graph, low_bits, max_fuse, smem_kb, no_tables, reg_bits)
    _check(lib().hs_evolve_td(f.handle, ptr, n_rhs, fv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), fv.size,
                              ctypes.byref(o), _stream(stream)))


def hs_factors_set_drive(f: Factors, drive: float, stream=None) -> None:
    _check(lib().hs_factors_set_drive(f.handle, float(drive), _stream(stream)))


def hs_evolve_plan(f: Factors, n_rhs: int, n_steps: int, method: int = HS_METHOD_AUTO, tile_bits: int = 0,
                   rhs_block: int = 0, use_graph: bool = False, low_bits: int = 0, max_fuse: int = 0,
                   smem_kb: int = 0, no_tables: bool = False, reg_bits: int = 0):
    """(n_sweep_launches, n_plain_launches, tile_bits, rhs_block) hs_evolve_ex would use."""
    o = _opts(method, tile_bits, rhs_block, use_graph, low_bits, max_fuse, smem_kb, no_tables, reg_bits)
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().hs_evolve_plan(f.handle, int(n_rhs), int(n_steps), ctypes.byref(o), ctypes.byref(a), ctypes.byref(b),
                                ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def hs_evolve_td_plan(f: Factors, n_rhs: int, n_steps: int, method: int = HS_METHOD_AUTO, tile_bits: int = 0,
                      rhs_block: int = 0, use_graph: bool = False, low_bits: int = 0, max_fuse: int = 0,
                      smem_kb: int = 0, no_tables: bool = False, reg_bits: int = 0):
    """(n_sweep_launches, n_plain_launches, tile_bits, rhs_block) of a whole hs_evolve_td
    of n_steps steps."""
    o = _opts(method, tile_bits, rhs_block, use_graph, low_bits, max_fuse, smem_kb, no_tables, reg_bits)
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().hs_evolve_td_plan(f.handle, int(n_rhs), int(n_steps), ctypes.byref(o), ctypes.byref(a),
                                   ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def hs_autotune(f: Factors, psi, n_steps: int, stream=None) -> dict:
    """Time candidate launch parameters on a copy of psi; the winner is used by later
    default-option evolutions of the same shape.  Returns it as a dict."""
    ptr, n_rhs = _check_state(f, psi)
    o = EvolveOpts()
    _check(lib().hs_autotune(f.handle, ptr, n_rhs, int(n_steps), _stream(stream), ctypes.byref(o)))
    return dict(method=o.method, tile_bits=o.tile_bits, rhs_block=o.rhs_block, low_bits=o.low_bits,
                max_fuse=o.max_fuse, smem_kb=o.smem_kb, reg_bits=o.reg_bits)


def hs_apply_factor(f: Factors, g: int, x, y, stream=None) -> None:
    px, n_rhs = _check_state(f, x)
    py, n_rhs2 = _check_state(f, y)
    if n_rhs != n_rhs2:
        raise ValueError("x and y differ in shape")
    _check(lib().hs_apply_factor(f.handle, int(g), px, py, n_rhs, _stream(stream)))


def hs_fidelity(a, b, stream=None) -> Tuple[float, float, float]:
    """(|<a|b>|^2 / (|a|^2 |b|^2), |a|^2, |b|^2) for two single-state CUDA tensors."""
    pa, ra, na, ca = _state_args(a)
    pb, rb, nb, cb = _state_args(b)
    if (ra, na, ca) != (1, nb, cb) or rb != 1:
        raise ValueError("fidelity takes two single states of equal size and dtype")
    fid, n1, n2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().hs_fidelity(pa, pb, na, ca, _stream(stream), ctypes.byref(fid), ctypes.byref(n1), ctypes.byref(n2)))
    return fid.value, n1.value, n2.value


def _check_out(out, n_doubles: int, like) -> None:
    """out must be a contiguous float64 CUDA tensor of at least n_doubles
    elements on the device of `like` (the library writes 8-byte values)."""
    import torch
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64:
        raise ValueError("out must be a CUDA float64 tensor")
    if out.device != like.device:
        raise ValueError("out must be on the device of the states")
    if not out.is_contiguous() or out.numel() < n_doubles:
        raise ValueError(f"out must be contiguous with at least {n_doubles} elements")


def hs_inner_device(a, b, out, stream=None) -> None:
    """out (CUDA float64 tensor of 4) <- (Re<a|b>, Im<a|b>, |a|^2, |b|^2), no synchronisation."""
    pa, ra, na, ca = _state_args(a)
    pb, rb, nb, cb = _state_args(b)
    if (ra, na, ca) != (1, nb, cb) or rb != 1:
        raise ValueError("inner product takes two single states of equal size and dtype")
    _check_out(out, 4, a)
    _check(lib().hs_inner_device(pa, pb, na, ca, out.data_ptr(), _stream(stream)))


def hs_plan_factors(x, z, n_qubits: int, diag_budget: int, dtype="c64"):
    """Structural dry run on the host (no GPU): list of (term_first, term_last, offsets)
    per factor and the device bytes the factor values will take."""
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    za = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    code = HS_C64 if dtype in ("c64", HS_C64) else HS_C128
    nf, no = ctypes.c_int(), ctypes.c_int()
    vb = ctypes.c_int64()
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check(lib().hs_plan_factors(xa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 za.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), xa.size, int(n_qubits),
                                 int(diag_budget), code, ctypes.byref(nf), ctypes.byref(no), None, None, None, None,
                                 ctypes.byref(vb), 0, 0))
    gf = np.zeros(nf.value, dtype=np.int32)
    gl = np.zeros(nf.value, dtype=np.int32)
    nd = np.zeros(nf.value, dtype=np.int32)
    offs = np.zeros(no.value, dtype=np.int64)
    _check(lib().hs_plan_factors(xa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 za.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), xa.size, int(n_qubits),
                                 int(diag_budget), code, ctypes.byref(nf), ctypes.byref(no), ip(gf), ip(gl), ip(nd),
                                 offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(vb), nf.value,
                                 no.value))
    out, k = [], 0
    for g in range(nf.value):
        out.append((int(gf[g]), int(gl[g]), [int(o) for o in offs[k:k + nd[g]]]))
        k += int(nd[g])
    return out, int(vb.value)


def hs_plan_schedule(x, z, n_qubits: int, diag_budget: int, n_steps: int, tile_bits: int, low_bits: int,
                     order: int = 1, dtype="c64", max_fuse: int = 0, commuting: bool = True):
    """Host-only launch schedule (no GPU): arrays (factor, step, sweep) per factor
    application, in the order the sweeps apply them."""
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    za = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    code = HS_C64 if dtype in ("c64", HS_C64) else HS_C128
    na, ns = ctypes.c_int(), ctypes.c_int()
    args = (xa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), za.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
            xa.size, int(n_qubits), int(diag_budget), int(order), code, int(n_steps), int(tile_bits), int(low_bits),
            int(max_fuse), int(bool(commuting)), ctypes.byref(na), ctypes.byref(ns))
    _check(lib().hs_plan_schedule(*args, None, None, None, 0))
    fac, st, sw = (np.zeros(na.value, dtype=np.int32) for _ in range(3))
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check(lib().hs_plan_schedule(*args, ip(fac), ip(st), ip(sw), na.value))
    return fac, st, sw


def hs_inner_batch_noalloc(a, b, out, stream=None) -> None:
    """out (CUDA float64 tensor (R, 4)) <- per state pair (Re<a_i|b_i>, Im<a_i|b_i>, |a_i|^2, |b_i|^2),
    computed without any device allocation (static scratch; see include/hs.h)."""
    pa, ra, na, ca = _state_args(a)
    pb, rb, nb, cb = _state_args(b)
    if (ra, na, ca) != (rb, nb, cb):
        raise ValueError("a and b differ in shape or dtype")
    _check_out(out, 4 * ra, a)
    _check(lib().hs_inner_batch_noalloc(pa, pb, na, ra, ca, out.data_ptr(), _stream(stream)))


class Batch:
    """Owner of an hs_batch handle; keeps its jobs' factor sets and states alive."""

    def __init__(self, handle: int, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep
        nl, ns = ctypes.c_int(), ctypes.c_int()
        nc, nu = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().hs_batch_info(self.handle, ctypes.byref(nl), ctypes.byref(nc), ctypes.byref(nu), ctypes.byref(ns)))
        self.n_levels, self.n_ctas, self.n_updates, self.n_separate = nl.value, nc.value, nu.value, ns.value

    def close(self, stream=None):
        """Free the batch; with a stream, in stream order without synchronising."""
        if self.handle and self.handle.value:
            if _lib is not None:
                if stream is None:
                    _lib.hs_batch_free(self.handle)
                else:
                    _lib.hs_batch_free_async(self.handle, _stream(stream))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hs_batch_create(jobs, tile_bits: int = 0, low_bits: int = 0, use_graph: bool = True, smem_kb: int = 0,
                    no_tables: bool = False, tiles_per_cta: int = 0, method: int = 0, reg_bits: int = 0) -> Batch:
    """jobs: sequence of (Factors, state tensor, n_steps)."""
    arr = (BatchJob * len(jobs))()
    keep = []
    for k, (f, psi, n_steps) in enumerate(jobs):
        ptr, n_rhs = _check_state(f, psi)
        arr[k] = BatchJob(f.handle.value, ptr, n_rhs, int(n_steps))
        keep.append((f, psi))
    o = BatchOpts(int(tile_bits), int(low_bits), int(bool(use_graph)), int(smem_kb), int(bool(no_tables)),
                  int(tiles_per_cta), int(method), int(reg_bits))
    out = ctypes.c_void_p()
    _check(lib().hs_batch_create(arr, len(jobs), ctypes.byref(o), ctypes.byref(out)))
    return Batch(out.value, keep)


def _batch_jobs(jobs):
    arr = (BatchJob * len(jobs))()
    keep = []
    for k, (f, psi, n_steps) in enumerate(jobs):
        ptr, n_rhs = _check_state(f, psi)
        arr[k] = BatchJob(f.handle.value, ptr, n_rhs, int(n_steps))
        keep.append((f, psi))
    return arr, keep


def hs_batch_autotune(jobs, use_graph: bool = False, stream=None) -> dict:
    """Time candidate batch options on scratch copies of the jobs' states; the
    fastest as keyword arguments for hs_batch_create."""
    arr, _ = _batch_jobs(jobs)
    o = BatchOpts()
    o.use_graph = int(bool(use_graph))
    _check(lib().hs_batch_autotune(arr, len(jobs), _stream(stream), ctypes.byref(o)))
    return dict(tile_bits=o.tile_bits, low_bits=o.low_bits, smem_kb=o.smem_kb, no_tables=bool(o.no_tables),
                tiles_per_cta=o.tiles_per_cta, method=o.method, reg_bits=o.reg_bits)


def hs_batch_launch(b: Batch, stream=None) -> None:
    _check(lib().hs_batch_launch(b.handle, _stream(stream)))


def hs_evolve_batch(jobs, stream=None) -> None:
    """jobs: sequence of (Factors, state tensor, n_steps); one call plans,
    launches and frees (in stream order) a batch of them."""
    n = len(jobs)
    fs = (ctypes.c_void_p * max(1, n))()
    ps = (ctypes.c_void_p * max(1, n))()
    nr = (ctypes.c_int * max(1, n))()
    ns = (ctypes.c_int * max(1, n))()
    for k, (f, psi, n_steps) in enumerate(jobs):
        ptr, n_rhs = _check_state(f, psi)
        fs[k], ps[k], nr[k], ns[k] = f.handle.value, ptr, n_rhs, int(n_steps)
    _check(lib().hs_evolve_batch(fs, ps, nr, ns, n, _stream(stream)))


# ---------------------------------------------------------------------------
# Single-factor Taylor mode (include/hs_dia.h): Alg. 2, Alg. 3, Eq. 5
# ---------------------------------------------------------------------------

class Dia:
    """Owner of an hs_dia handle: a device-resident matrix in the compact
    diagonal layout (freed on close or garbage collection)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        nq, nd, dt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nnz = ctypes.c_int64()
        _check(lib().hs_dia_info(self.handle, ctypes.byref(nq), ctypes.byref(nd), ctypes.byref(nnz),
                                 ctypes.byref(dt)))
        self.n_qubits, self.n_diags, self.nnz = nq.value, nd.value, nnz.value
        self.dtype = "c64" if dt.value == HS_C64 else "c128"

    @property
    def N(self) -> int:
        return 1 << self.n_qubits

    def offsets(self) -> np.ndarray:
        out = np.zeros(self.n_diags, dtype=np.int64)
        _check(lib().hs_dia_get(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None))
        return out

    def get(self):
        """(offsets, {offset: complex128 values}) copied to the host (Eq. 6 order)."""
        offs = self.offsets()
        total = int(sum(self.N - abs(int(d)) for d in offs))
        vals = np.zeros(2 * total, dtype=np.float64)
        _check(lib().hs_dia_get(self.handle, None, vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        c = vals.view(np.complex128)
        out, pos = {}, 0
        for d in offs:
            L = self.N - abs(int(d))
            out[int(d)] = c[pos:pos + L].copy()
            pos += L
        return offs, out

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().hs_dia_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _new_dia(fn, *args) -> Dia:
    out = ctypes.c_void_p()
    _check(fn(*args, ctypes.byref(out)))
    return Dia(out.value)


def hs_dia_from_terms(labels: Sequence[str], coeffs, stream=None) -> Dia:
    """H = sum_j c_j P_j in the compact layout (FP64, zero diagonals dropped)."""
    arr = (ctypes.c_char_p * len(labels))(*[l.encode() for l in labels])
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    return _new_dia(lib().hs_dia_from_terms, arr, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(labels),
                    _stream(stream))


def hs_dia_from_masks(x, z, coeffs, n_qubits: int, stream=None) -> Dia:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    return _new_dia(lib().hs_dia_from_masks, x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                    z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    len(c), int(n_qubits), _stream(stream))


def hs_dia_create(n_qubits: int, diags: dict, dtype="c128", stream=None) -> Dia:
    """A matrix from host diagonals {offset: complex values of length N - |offset|}."""
    offs = np.ascontiguousarray(np.asarray(list(diags.keys()), dtype=np.int64))
    vals = np.concatenate([np.asarray(diags[int(d)], dtype=np.complex128) for d in offs]) if len(offs) else \
        np.zeros(0, dtype=np.complex128)
    vals = np.ascontiguousarray(vals).view(np.float64)
    return _new_dia(lib().hs_dia_create, int(n_qubits), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    len(offs), vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _dtype_code(dtype),
                    _stream(stream))


def hs_spgemm(a: Dia, b: Dia, stream=None) -> Tuple[Dia, float]:
    """(A B, ||A B||_F)."""
    out, fro = ctypes.c_void_p(), ctypes.c_double()
    _check(lib().hs_spgemm(a.handle, b.handle, _stream(stream), ctypes.byref(out), ctypes.byref(fro)))
    return Dia(out.value), fro.value


def hs_spme(a: Dia, t: float, tol: float = 1e-6, max_iter: int = 100, stream=None) -> Tuple[Dia, int, bool]:
    """(exp(-i t A), Taylor terms used, converged)."""
    out, k, ok = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int()
    _check(lib().hs_spme(a.handle, float(t), float(tol), int(max_iter), _stream(stream), ctypes.byref(out),
                         ctypes.byref(k), ctypes.byref(ok)))
    return Dia(out.value), k.value, bool(ok.value)


def hs_estimate_timesteps(a: Dia, t: float, diag_budget: int, tol: float = 1e-6, max_iter: int = 100,
                          max_steps: int = 1 << 20, stream=None) -> int:
    r = ctypes.c_int()
    _check(lib().hs_estimate_timesteps(a.handle, float(t), int(diag_budget), float(tol), int(max_iter),
                                       int(max_steps), _stream(stream), ctypes.byref(r)))
    return r.value


def _dia_state(a: Dia, psi):
    ptr, n_rhs, n, dt = _state_args(psi)
    if n != a.n_qubits:
        raise ValueError("state size does not match the matrix")
    if dt != _dtype_code(a.dtype):
        raise ValueError("state dtype does not match the matrix")
    return ptr, n_rhs


def hs_spmv(a: Dia, x, y, stream=None) -> None:
    px, n_rhs = _dia_state(a, x)
    py, n_rhs_y = _dia_state(a, y)
    if n_rhs != n_rhs_y:
        raise ValueError("x and y hold different numbers of states")
    _check(lib().hs_spmv(a.handle, px, py, n_rhs, _stream(stream)))


def hs_dia_evolve(u: Dia, psi, n_steps: int, stream=None) -> None:
    p, n_rhs = _dia_state(u, psi)
    _check(lib().hs_dia_evolve(u.handle, p, n_rhs, int(n_steps), _stream(stream)))


def hs_dia_evolve_td(x, z, coeffs0, coeffs1, n_qubits: int, t: float, drive, psi, tol: float = 1e-6,
                     max_iter: int = 100, stream=None) -> None:
    """One single-factor Taylor step per drive sample under H0 + f H1, psi in place."""
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    za = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    a = np.ascontiguousarray(np.asarray(coeffs0, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(coeffs1, dtype=np.float64))
    if not (xa.size == za.size == a.size == b.size):
        raise ValueError("x, z, coeffs0 and coeffs1 differ in length")
    fv = np.ascontiguousarray(np.asarray(drive, dtype=np.float64).ravel())
    ptr, n_rhs, n, code = _state_args(psi)
    if n != int(n_qubits):
        raise ValueError("state size does not match n_qubits")
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().hs_dia_evolve_td(xa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                  za.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), a.ctypes.data_as(dp),
                                  b.ctypes.data_as(dp), xa.size, int(n_qubits), float(t), fv.ctypes.data_as(dp),
                                  fv.size, float(tol), int(max_iter), ptr, n_rhs, code, _stream(stream)))


def hs_dia_convert(a: Dia, dtype, stream=None) -> Dia:
    return _new_dia(lib().hs_dia_convert, a.handle, _dtype_code(dtype), _stream(stream))


def hs_expectation(a: Dia, psi, stream=None):
    """(<psi_r|A|psi_r> as complex128 array of n_rhs, <psi_r|psi_r> array), FP64."""
    p, n_rhs = _dia_state(a, psi)
    vals = np.zeros(2 * n_rhs, dtype=np.float64)
    norms = np.zeros(n_rhs, dtype=np.float64)
    _check(lib().hs_expectation(a.handle, p, n_rhs, _stream(stream), vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                norms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return vals.view(np.complex128), norms
