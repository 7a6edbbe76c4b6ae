"""Python binding of libkomega_gb300.so (ctypes; argument marshalling only).

Every step of the solve runs in the library's CUDA kernels.  PyTorch provides
device memory and the current CUDA stream.  The names mirror the C ABI in
include/komega_gb300.h.  There is no CPU fallback: if the library is missing
or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkomega_gb300.so")

KW_F64 = 0
KW_C32V_F64S = 1
KW_DF64 = 2
PRECISIONS = {"f64": KW_F64, "c32v_f64s": KW_C32V_F64S, "c32": KW_C32V_F64S, "df64": KW_DF64}

STATUS = {0: "KW_OK", 1: "KW_ERR_ARG", 2: "KW_ERR_CUDA", 3: "KW_ERR_OOM", 4: "KW_ERR_BREAKDOWN",
          5: "KW_ERR_NONFINITE", 6: "KW_ERR_CALLBACK", 7: "KW_ERR_TIMEOUT", 8: "KW_NOT_CONVERGED"}
KW_OK, KW_ERR_ARG, KW_ERR_CALLBACK, KW_NOT_CONVERGED = 0, 1, 6, 8
MAX_PROJ = 32


class kw_options(C.Structure):
    _fields_ = [("prec", C.c_int), ("tol", C.c_double), ("maxiter", C.c_int64), ("seed_switch", C.c_int),
                ("hist_stride", C.c_int64), ("hist_max", C.c_int64), ("use_graph", C.c_int),
                ("tune_cache", C.c_char_p)]

ABI_VERSION = 2   # KW_ABI_VERSION of the header these structures mirror


class kw_c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class kw_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("n_converged", C.c_int64), ("max_res", C.c_double),
                ("n_seed_switch", C.c_int64), ("updates", C.c_int64), ("seed", C.c_int64), ("status", C.c_int)]


class kw_csr_term(C.Structure):
    _fields_ = [("nnz", C.c_int64), ("rowptr_dev", C.c_void_p), ("col_dev", C.c_void_p), ("val_dev", C.c_void_p)]


class kw_instance(C.Structure):
    _fields_ = [("m", C.c_int64), ("nnz", C.c_int64), ("rowptr_dev", C.c_void_p), ("col_dev", C.c_void_p),
                ("val_dev", C.c_void_p), ("b_dev", C.c_void_p), ("nshift", C.c_int64), ("z_host", C.c_void_p),
                ("nleft", C.c_int64), ("left_dev", C.c_void_p), ("x_out_dev", C.c_void_p),
                ("proj_out_host", C.c_void_p), ("tol", C.c_double)]


class kw_rci_io(C.Structure):
    _fields_ = [("r", C.c_void_p), ("q", C.c_void_p), ("rt", C.c_void_p), ("qt", C.c_void_p), ("elem", C.c_int)]


class kw_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("timed_iters", C.c_int64), ("kernel_ms", C.c_double * 4),
                ("tune_runs", C.c_int64), ("tune_hits", C.c_int64)]


_lib = None


# kw_matvec_fn: (user, r_dev, q_dev, m, elem, cuda_stream) -> int
MATVEC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p)
KW_ELEM_C128, KW_ELEM_C64 = 0, 1
METHODS = {"cocg": 0, "cg": 1, "bicg": 2}


class _DeviceVector:
    """A borrowed device vector as (m, 2) real numbers, for torch.as_tensor."""

    def __init__(self, ptr: int, m: int, real_typestr: str):
        self.__cuda_array_interface__ = {"shape": (m, 2), "typestr": real_typestr, "data": (ptr, False),
                                         "strides": None, "version": 2}


def load_library(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2001_08707_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(path)
    lib.kw_abi_version.restype = C.c_int
    if lib.kw_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{path} has ABI version {lib.kw_abi_version()}, the binding expects {ABI_VERSION}: "
                           "rebuild it")
    P, I64, D = C.c_void_p, C.c_int64, C.c_double
    sig = {
        "kw_abi_version": (C.c_int, []),
        "kw_default_options": (None, [C.POINTER(kw_options)]),
        "kw_status_string": (C.c_char_p, [C.c_int]),
        "kw_create": (C.c_int, [C.POINTER(P), C.POINTER(kw_options), P]),
        "kw_destroy": (None, [P]),
        "kw_last_error": (C.c_int, [P, C.c_char_p, C.c_size_t]),
        "kw_set_csr": (C.c_int, [P, I64, I64, P, P, P]),
        "kw_solve": (C.c_int, [P, P, I64, P, I64, P, P, P, C.POINTER(kw_solve_info)]),
        "kw_solve_host": (C.c_int, [P, I64, I64, P, P, P, P, I64, P, I64, P, P, P, C.POINTER(kw_solve_info)]),
        "kw_get_shift_status": (C.c_int, [P, P, P]),
        "kw_get_residual_history": (C.c_int, [P, P, C.POINTER(I64)]),
        "kw_spmv_dot": (C.c_int, [P, kw_c128, P, P, C.POINTER(kw_c128)]),
        "kw_set_kernel_timing": (C.c_int, [P, I64]),
        "kw_get_stats": (C.c_int, [P, C.POINTER(kw_stats)]),
        "kw_set_spmv_config": (C.c_int, [P, C.c_int, C.c_int]),
        "kw_bilinear": (C.c_int, [P, I64, I64, C.POINTER(kw_csr_term), I64, P, P, P]),
        "kw_solve_batched": (C.c_int, [P, I64, C.POINTER(kw_instance), C.POINTER(kw_solve_info)]),
        "kw_spmv_dot_noalloc": (C.c_int, [I64, I64, P, P, P, kw_c128, P, P, C.POINTER(kw_c128), P]),
        "kw_get_spmv_config": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "kw_set_matvec": (C.c_int, [P, I64, MATVEC_FN, P]),
        "kw_set_spin_operator": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, P]),
        "kw_set_lattice3d": (C.c_int, [P, I64, I64, I64, P, D]),
        "kw_set_spin_table": (C.c_int, [P, C.c_int]),
        "kw_set_krylov_log": (C.c_int, [P, I64]),
        "kw_set_stream_overlap": (C.c_int, [P, C.c_int]),
        "kw_set_bulk_copy": (C.c_int, [P, C.c_int]),
        "kw_set_shift_storage": (C.c_int, [P, C.c_int]),
        "kw_set_seed_update": (C.c_int, [P, C.c_int]),
        "kw_set_update_tile": (C.c_int, [P, C.c_int]),
        "kw_shift_combine": (C.c_int, [P, I64, I64, P, C.c_int, I64, P, P]),
        "kw_get_update_tile": (C.c_int, [P, C.POINTER(C.c_int)]),
        "kw_bilinear_c64": (C.c_int, [P, I64, I64, C.POINTER(kw_csr_term), I64, P, P, P]),
        "kw_set_method": (C.c_int, [P, C.c_int, P]),
        "kw_resume": (C.c_int, [P, I64, P, C.POINTER(kw_solve_info)]),
        "kw_rci_init": (C.c_int, [P, I64, P, I64, P, I64, P, P, C.POINTER(kw_rci_io)]),
        "kw_rci_update": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(kw_rci_io)]),
        "kw_rci_get_residual": (C.c_int, [P, P]),
        "kw_rci_finalize": (C.c_int, [P, P, C.POINTER(kw_solve_info)]),
        "kw_set_matvec_adjoint": (C.c_int, [P, MATVEC_FN, P]),
        "kw_get_krylov_log": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(D), P, P]),
        "kw_recalc": (C.c_int, [P, I64, I64, D, P, P, I64, P, P, P, P, C.POINTER(kw_solve_info)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def spmv_dot_noalloc(rowptr, col, val, zs: complex, r, q, stream=None) -> complex:
    """kw_spmv_dot_noalloc: q = zs r - H r and t = r^T q in FP64 without any
    device allocation by the library (all arguments are contiguous tensors on
    the current CUDA device: int64 rowptr [m+1], int32 col and float64 val of
    equal length, complex128 r and q [m]).  Every type, device and length is
    checked here and a mismatch raises ValueError before the library is
    called; the row offsets and column indices themselves are the caller's
    promise (kw_set_csr's contract)."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    for name, v, dt in (("rowptr", rowptr, torch.int64), ("col", col, torch.int32), ("val", val, torch.float64)):
        if not isinstance(v, torch.Tensor) or v.device != dev or v.dtype != dt or not v.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt} tensor on {dev}")
    if rowptr.dim() != 1 or rowptr.numel() < 2:
        raise ValueError("rowptr must hold m + 1 >= 2 offsets")
    if col.numel() != val.numel():
        raise ValueError(f"col and val must have the same length, got {col.numel()} and {val.numel()}")
    m = rowptr.numel() - 1
    for name, v in (("r", r), ("q", q)):
        if not isinstance(v, torch.Tensor) or v.device != dev or v.dtype != torch.complex128:
            raise ValueError(f"{name} must be a complex128 tensor on {dev}")
        check_vector_bytes(name, v, m, 16)
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    t = kw_c128()
    st = lib.kw_spmv_dot_noalloc(m, col.numel(), C.c_void_p(rowptr.data_ptr()),
                                 C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()),
                                 kw_c128(zs.real, zs.imag), C.c_void_p(r.data_ptr()), C.c_void_p(q.data_ptr()),
                                 C.byref(t), C.c_void_p(s.cuda_stream))
    if st != KW_OK:
        raise KomegaError(st, "kw_spmv_dot_noalloc")
    return complex(t.re, t.im)


class KomegaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


@dataclass
class SolveResult:
    proj: np.ndarray          # [K, nleft+1] complex128; column 0 = b^T x_k
    x: object                 # torch tensor [K, m] (complex128 / complex64) in full mode, else None
    iters: int
    n_converged: int
    max_res: float
    n_seed_switch: int
    updates: int
    seed: int
    status: str


# Columns of a Krylov log row before P r_{n+1}: z_s, alpha_n, c_n, beta_n,
# ||r_{n+1}||^2, pi^j_{n+1}, pi^j_n (see kw_get_krylov_log).
LOG_FIXED = 7


@dataclass
class KrylovLog:
    """A solve's per-iteration record for recalculation at new shifts."""
    rows: np.ndarray          # [n_iter, LOG_FIXED + nproj] complex128
    w0: np.ndarray            # [nproj] complex128: P b
    thresh: float             # the solve's tol * ||b||
    n_run: int                # iterations of the solve (> n_iter when the log was cut short)

    @property
    def nproj(self) -> int:
        return self.rows.shape[1] - LOG_FIXED


@dataclass
class RecalcResult:
    proj: np.ndarray          # [K, nproj] complex128; column 0 = b^T x
    conv_iter: np.ndarray     # [K] rows replayed when the shift froze, -1 if never
    final_res: np.ndarray     # [K] last residual estimate
    iters: int                # rows replayed
    n_converged: int
    updates: int              # shift-rows replayed
    status: str


def check_solve_arrays(m, b, left, x_out, K, vec_dtype):
    """Sizes the C ABI cannot see (it takes bare pointers): b holds m values,
    left is [nleft][m] (or one row of m), and x_out, when given, is a
    contiguous [K][m] tensor of the form's complex type.  Raises ValueError."""
    if m is not None and b.numel() != m:
        raise ValueError(f"b has {b.numel()} entries, the operator has {m} rows")
    if left is not None and m is not None and (left.shape[-1] != m or left.dim() > 2):
        raise ValueError(f"left has shape {tuple(left.shape)}, expected [nleft, {m}]")
    if x_out is not None:
        if x_out.dtype != vec_dtype:
            raise ValueError(f"x_out has dtype {x_out.dtype}, the form writes {vec_dtype}")
        if not x_out.is_contiguous() or (m is not None and x_out.numel() != K * m):
            raise ValueError(f"x_out must be a contiguous [{K}, {m}] tensor, got {tuple(x_out.shape)}")


def check_vector_bytes(name, v, m, elem_bytes):
    """A device vector handed to the C ABI as a bare pointer: contiguous and
    exactly m elements of elem_bytes bytes.  Raises ValueError."""
    if m is not None and (not v.is_contiguous() or v.numel() * v.element_size() != m * elem_bytes):
        raise ValueError(f"{name} must be a contiguous vector of {m} elements of {elem_bytes} bytes, "
                         f"got {tuple(v.shape)} {v.dtype}")


def _z_array(z):
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    return z, z.ctypes.data_as(C.c_void_p)


class Solver:
    """A solver context (kw_ctx) on the current CUDA device and stream.

    use_graph: 1 (default) runs the iterations as a device-side loop in one CUDA
    graph; 0 has the host enqueue them in chunks; n >= 2 sets the iterations per
    trip of the device-side loop (kw_options.use_graph).  tune_cache: a file in
    which the product kernel's tuned layout is looked up and stored
    (kw_options.tune_cache).
    """

    def __init__(self, prec: str = "f64", tol: float = 1e-10, maxiter: int = 100000, seed_switch: bool = True,
                 hist_stride: int = 0, hist_max: int = 0, stream=None, method: str = "cocg",
                 use_graph: int = 1, tune_cache: str | None = None):
        import torch

        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("komega: no CUDA device (the solver has no CPU path)")
        lib = load_library()
        self._lib = lib
        self.prec = PRECISIONS[prec]
        opt = kw_options(self.prec, tol, maxiter, 1 if seed_switch else 0, hist_stride, hist_max, int(use_graph),
                         tune_cache.encode() if tune_cache else None)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        ctx = C.c_void_p()
        st = lib.kw_create(C.byref(ctx), C.byref(opt), C.c_void_p(s.cuda_stream))
        if st != KW_OK:
            raise KomegaError(st, "kw_create failed")
        self._ctx = ctx
        self._keep = []
        self.m = None
        if method != "cocg":
            self.set_method(method)
        self.vec_dtype = torch.complex64 if self.prec == KW_C32V_F64S else torch.complex128

    # ------------------------------------------------------------------ helpers
    def _err(self, st, what):
        buf = C.create_string_buffer(512)
        self._lib.kw_last_error(self._ctx, buf, 512)
        return KomegaError(st, f"{what}: {buf.value.decode()}")

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.kw_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype):
        t = self._torch
        if isinstance(a, t.Tensor):
            a = a.to(device="cuda", dtype=dtype)
        else:
            a = t.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")
        return a.contiguous()

    # ------------------------------------------------------------------ ABI calls
    def set_csr(self, rowptr, col, val):
        t = self._torch
        rp = self._dev(rowptr, t.int64)
        cl = self._dev(col, t.int32)
        vl = self._dev(val, t.float64)
        m = rp.numel() - 1
        nnz = cl.numel()
        st = self._lib.kw_set_csr(self._ctx, m, nnz, C.c_void_p(rp.data_ptr()), C.c_void_p(cl.data_ptr()),
                                  C.c_void_p(vl.data_ptr()))
        if st != KW_OK:
            raise self._err(st, "kw_set_csr")
        self._keep = [rp, cl, vl]     # borrowed by the context in FP64 mode
        self.m = m

    def solve(self, b, z, left=None, full: bool = False, x_out=None, check: bool = True) -> SolveResult:
        """kw_solve.  x_out (a CUDA tensor [K, m] of the form's complex type)
        receives x^(k) and implies full mode."""
        t = self._torch
        bd = self._dev(b, t.float64)
        zz, zp = _z_array(z)
        K = zz.size
        if left is not None:
            ld = self._dev(left, t.float64)
            nleft = ld.shape[0] if ld.dim() == 2 else 1
            lp = C.c_void_p(ld.data_ptr())
        else:
            ld, nleft, lp = None, 0, None
        if x_out is not None:
            if not x_out.is_cuda:
                raise ValueError("x_out must be a CUDA tensor")
            full = True
        check_solve_arrays(self.m, bd, ld, x_out, K, self.vec_dtype)
        x = None
        xp = None
        if full:
            x = x_out if x_out is not None else t.empty((K, bd.numel()), dtype=self.vec_dtype, device="cuda")
            xp = C.c_void_p(x.data_ptr())
        proj = np.zeros((K, nleft + 1), dtype=np.complex128)
        info = kw_solve_info()
        st = self._lib.kw_solve(self._ctx, C.c_void_p(bd.data_ptr()), K, zp, nleft, lp, xp,
                                proj.ctypes.data_as(C.c_void_p), C.byref(info))
        self._last_solve = (bd, zz, ld, x, proj.shape)   # kept alive for kw_resume
        if check and st not in (KW_OK, KW_NOT_CONVERGED):
            raise self._err(st, "kw_solve") from getattr(self, "_mv_error", None)
        return SolveResult(proj, x, info.iters, info.n_converged, info.max_res, info.n_seed_switch, info.updates,
                           info.seed, STATUS.get(st, str(st)))

    # ------------------------------------------------------------------ reverse communication
    def _rci_views(self, io):
        torch = self._torch
        ts = "<f8" if io.elem == KW_ELEM_C128 else "<f4"
        view = lambda ptr: None if not ptr else torch.view_as_complex(
            torch.as_tensor(_DeviceVector(ptr, self.m, ts), device="cuda"))
        return view(io.r), view(io.q), view(io.rt), view(io.qt)

    def rci_init(self, b, z, left=None, full: bool = False):
        """kw_rci_init: start a solve whose products the caller makes.  Returns
        (r, q, rt, qt) tensor views: write H r into q (and H^dagger rt into qt
        for BiCG), then call rci_update."""
        t = self._torch
        bd = self._dev(b, t.float64)
        zz, zp = _z_array(z)
        ld = None if left is None else self._dev(np.atleast_2d(left), t.float64)
        nleft = 0 if ld is None else ld.shape[0]
        self.m = bd.numel()
        x = t.empty((zz.size, self.m), dtype=self.vec_dtype, device="cuda") if full else None
        io = kw_rci_io()
        st = self._lib.kw_rci_init(self._ctx, self.m, C.c_void_p(bd.data_ptr()), zz.size, zp, nleft,
                                   None if ld is None else C.c_void_p(ld.data_ptr()),
                                   None if x is None else C.c_void_p(x.data_ptr()), C.byref(io))
        if st != KW_OK:
            raise self._err(st, "kw_rci_init")
        self._rci = (bd, zz, ld, x, (zz.size, nleft + 1))
        return self._rci_views(io)

    def rci_update(self):
        """kw_rci_update: finish the iteration; returns (done, (r, q, rt, qt))."""
        d = C.c_int()
        io = kw_rci_io()
        st = self._lib.kw_rci_update(self._ctx, C.byref(d), C.byref(io))
        if st != KW_OK:
            raise self._err(st, "kw_rci_update")
        return bool(d.value), self._rci_views(io)

    def rci_residual(self):
        K = self._rci[1].size
        res = np.zeros(K)
        st = self._lib.kw_rci_get_residual(self._ctx, res.ctypes.data_as(C.c_void_p))
        if st != KW_OK:
            raise self._err(st, "kw_rci_get_residual")
        return res

    def rci_finalize(self, check: bool = True) -> SolveResult:
        _, _, _, x, shape = self._rci
        proj = np.zeros(shape, dtype=np.complex128)
        info = kw_solve_info()
        st = self._lib.kw_rci_finalize(self._ctx, proj.ctypes.data_as(C.c_void_p), C.byref(info))
        if check and st not in (KW_OK, KW_NOT_CONVERGED):
            raise self._err(st, "kw_rci_finalize")
        return SolveResult(proj, x, info.iters, info.n_converged, info.max_res, info.n_seed_switch, info.updates,
                           info.seed, STATUS.get(st, str(st)))

    def resume(self, more_iters: int, check: bool = True) -> SolveResult:
        """kw_resume: continue the last solve (stopped at its iteration cap) for up
        to more_iters further iterations; x (full mode) is the same tensor."""
        last = getattr(self, "_last_solve", None)
        if last is None:
            raise KomegaError(KW_ERR_ARG, "resume: no solve to continue")
        _, _, _, x, shape = last
        proj = np.zeros(shape, dtype=np.complex128)
        info = kw_solve_info()
        st = self._lib.kw_resume(self._ctx, int(more_iters), proj.ctypes.data_as(C.c_void_p), C.byref(info))
        if check and st not in (KW_OK, KW_NOT_CONVERGED):
            raise self._err(st, "kw_resume")
        return SolveResult(proj, x, info.iters, info.n_converged, info.max_res, info.n_seed_switch, info.updates,
                           info.seed, STATUS.get(st, str(st)))

    def solve_host(self, rowptr, col, val, b, z, left=None, full: bool = False, check: bool = True):
        """kw_solve_host: all inputs and outputs in host (numpy) memory."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        vl = np.ascontiguousarray(val, dtype=np.float64)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        zz, zp = _z_array(z)
        K = zz.size
        m = rp.size - 1
        ll = None if left is None else np.ascontiguousarray(np.atleast_2d(left), dtype=np.float64)
        nleft = 0 if ll is None else ll.shape[0]
        x = None
        if full:
            x = np.zeros((K, m), dtype=np.complex64 if self.vec_dtype == self._torch.complex64 else np.complex128)
        proj = np.zeros((K, nleft + 1), dtype=np.complex128)
        info = kw_solve_info()
        vp = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        st = self._lib.kw_solve_host(self._ctx, m, cl.size, vp(rp), vp(cl), vp(vl), vp(bb), K, zp, nleft, vp(ll),
                                     vp(x), proj.ctypes.data_as(C.c_void_p), C.byref(info))
        if check and st not in (KW_OK, KW_NOT_CONVERGED):
            raise self._err(st, "kw_solve_host")
        self.m = m
        return SolveResult(proj, x, info.iters, info.n_converged, info.max_res, info.n_seed_switch, info.updates,
                           info.seed, STATUS.get(st, str(st)))

    def shift_status(self, K: int):
        ci = np.zeros(K, dtype=np.int64)
        fr = np.zeros(K, dtype=np.float64)
        st = self._lib.kw_get_shift_status(self._ctx, ci.ctypes.data_as(C.c_void_p), fr.ctypes.data_as(C.c_void_p))
        if st != KW_OK:
            raise self._err(st, "kw_get_shift_status")
        return ci, fr

    def residual_history(self, K: int):
        n = C.c_int64()
        st = self._lib.kw_get_residual_history(self._ctx, None, C.byref(n))
        if st != KW_OK:
            raise self._err(st, "kw_get_residual_history")
        h = np.zeros((max(n.value, 0), K), dtype=np.float64)
        if n.value > 0:
            st = self._lib.kw_get_residual_history(self._ctx, h.ctypes.data_as(C.c_void_p), C.byref(n))
            if st != KW_OK:
                raise self._err(st, "kw_get_residual_history")
        return h

    def set_matvec(self, fn, m: int, fn_adj=None):
        """kw_set_matvec: use ``fn(r, q)`` as the operator, where r and q are
        borrowed complex CUDA tensors of length m (complex64 in the FP32 form,
        complex128 otherwise) and fn must write H r into q with torch work on
        the current stream (the solver's).  fn_adj(r, q), if given, writes
        H^dagger r (kw_set_matvec_adjoint, for BiCG).  kw_set_csr ends it."""
        torch = self._torch
        self._mv_error = None

        def trampoline(user, r, q, mm, elem, stream):
            try:
                ts = "<f8" if elem == KW_ELEM_C128 else "<f4"
                rt = torch.view_as_complex(torch.as_tensor(_DeviceVector(r, mm, ts), device="cuda"))
                qt = torch.view_as_complex(torch.as_tensor(_DeviceVector(q, mm, ts), device="cuda"))
                # ctypes hands a NULL stream (the legacy default stream) over as None
                cs = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(cs):
                    fn(rt, qt)
                return 0
            except BaseException as exc:          # reported as KW_ERR_CALLBACK
                self._mv_error = exc
                return 1

        cb = MATVEC_FN(trampoline)
        st = self._lib.kw_set_matvec(self._ctx, int(m), cb, None)
        if st != KW_OK:
            raise self._err(st, "kw_set_matvec")
        self._mv_cb = cb                          # the library keeps the pointer
        if fn_adj is not None:
            def trampoline_adj(user, r, q, mm, elem, stream):
                try:
                    ts = "<f8" if elem == KW_ELEM_C128 else "<f4"
                    rt = torch.view_as_complex(torch.as_tensor(_DeviceVector(r, mm, ts), device="cuda"))
                    qt = torch.view_as_complex(torch.as_tensor(_DeviceVector(q, mm, ts), device="cuda"))
                    cs = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                    with torch.cuda.stream(cs):
                        fn_adj(rt, qt)
                    return 0
                except BaseException as exc:          # reported as KW_ERR_CALLBACK
                    self._mv_error = exc
                    return 1

            cba = MATVEC_FN(trampoline_adj)
            st = self._lib.kw_set_matvec_adjoint(self._ctx, cba, None)
            if st != KW_OK:
                raise self._err(st, "kw_set_matvec_adjoint")
            self._mv_cb_adj = cba
        self._keep = []
        self.m = int(m)

    def set_spin_operator(self, nsite: int, nup: int, bonds, J, h=None):
        """kw_set_spin_operator: H = sum_b J_b S_i.S_j + sum_i h_i S^z_i on the
        nsite-bit words with nup up spins, generated on the fly."""
        bd = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        Jv = np.ascontiguousarray(np.broadcast_to(np.asarray(J, dtype=np.float64), (bd.shape[0],)))
        hv = None if h is None else np.ascontiguousarray(np.asarray(h, dtype=np.float64))
        st = self._lib.kw_set_spin_operator(self._ctx, int(nsite), int(nup), bd.shape[0],
                                            bd.ctypes.data_as(C.c_void_p), Jv.ctypes.data_as(C.c_void_p),
                                            None if hv is None else hv.ctypes.data_as(C.c_void_p))
        if st != KW_OK:
            raise self._err(st, "kw_set_spin_operator")
        from math import comb

        self._keep = []
        self.m = comb(int(nsite), int(nup))

    def set_spin_table(self, on: bool):
        """kw_set_spin_table: keep an exchange table for the spin operator (True)
        or regenerate the exchanged rows in every product (False, default)."""
        st = self._lib.kw_set_spin_table(self._ctx, 1 if on else 0)
        if st != KW_OK:
            raise self._err(st, "kw_set_spin_table")

    def set_lattice3d(self, nx: int, ny: int, nz: int, eps, hopping: float = -1.0):
        """kw_set_lattice3d: periodic nearest-neighbour lattice, H_ii = eps_i,
        H_ij = hopping, generated on the fly (site i = x + nx (y + ny z))."""
        ed = self._dev(eps, self._torch.float64)
        st = self._lib.kw_set_lattice3d(self._ctx, int(nx), int(ny), int(nz), C.c_void_p(ed.data_ptr()),
                                        float(hopping))
        if st != KW_OK:
            raise self._err(st, "kw_set_lattice3d")
        self._keep = []
        self.m = int(nx) * int(ny) * int(nz)

    def set_method(self, method: str, btilde=None):
        """kw_set_method: 'cocg' (default), 'cg' (Hermitian A, real shifts) or
        'bicg' (shadow residual; btilde = its real start vector, default b)."""
        bt = None if btilde is None else self._dev(btilde, self._torch.float64)
        st = self._lib.kw_set_method(self._ctx, METHODS[method], None if bt is None else C.c_void_p(bt.data_ptr()))
        if st != KW_OK:
            raise self._err(st, "kw_set_method")
        self._btilde = bt                          # borrowed by the context

    def set_stream_overlap(self, on: bool):
        """kw_set_stream_overlap: run the shift scalars of iteration n beside the
        product of iteration n+1 and the x/p update of iteration n beside the next
        three-term update (True, the default: three streams), or all on one stream."""
        st = self._lib.kw_set_stream_overlap(self._ctx, 1 if on else 0)
        if st != KW_OK:
            raise self._err(st, "kw_set_stream_overlap")

    def set_shift_storage(self, fp32: bool):
        """kw_set_shift_storage: in full mode keep x^(k) and p^(k) as complex FP32
        (the seed recurrence keeps the form's precision); x tensors are then
        complex64 and the projections come from the projected recurrences."""
        st = self._lib.kw_set_shift_storage(self._ctx, int(bool(fp32)))
        if st != KW_OK:
            raise self._err(st, "kw_set_shift_storage")
        t = self._torch
        self.vec_dtype = t.complex64 if (fp32 or self.prec == KW_C32V_F64S) else t.complex128

    def set_update_tile(self, shifts: int):
        """kw_set_update_tile: shifts per tile of the x/p update (4, 8, 16), or 0
        to time the three at the next full-mode solve (the default)."""
        st = self._lib.kw_set_update_tile(self._ctx, int(shifts))
        if st != KW_OK:
            raise self._err(st, "kw_set_update_tile")

    def update_tile(self) -> int:
        """kw_get_update_tile: the x/p update tile of the last full-mode solve."""
        v = C.c_int()
        st = self._lib.kw_get_update_tile(self._ctx, C.byref(v))
        if st != KW_OK:
            raise self._err(st, "kw_get_update_tile")
        return v.value

    def set_seed_update(self, mode: int):
        """kw_set_seed_update: 1 = the row-group form of the three-term update
        (pair form; many projection rows), 0 = one element per thread, -1 (the
        default) = the row-group form above nine projection rows."""
        st = self._lib.kw_set_seed_update(self._ctx, int(mode))
        if st != KW_OK:
            raise self._err(st, "kw_set_seed_update")

    def set_bulk_copy(self, on):
        """kw_set_bulk_copy: stage the three-term update's tiles in shared memory
        with TMA bulk copies (True), read them with plain loads (False), or -1
        (the default) to stage only with more than 9 projection rows; 2 arms the
        stages for bytes that never arrive (a test of the bounded wait)."""
        st = self._lib.kw_set_bulk_copy(self._ctx, int(on))
        if st != KW_OK:
            raise self._err(st, "kw_set_bulk_copy")

    def set_krylov_log(self, max_iters: int):
        """Record the Krylov log (at most max_iters rows) in the next solves; 0 = off."""
        st = self._lib.kw_set_krylov_log(self._ctx, int(max_iters))
        if st != KW_OK:
            raise self._err(st, "kw_set_krylov_log")

    def krylov_log(self) -> KrylovLog:
        """The Krylov log of the last solve, copied to the host."""
        n, run, np_, thr = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
        st = self._lib.kw_get_krylov_log(self._ctx, C.byref(n), C.byref(run), C.byref(np_), C.byref(thr), None, None)
        if st != KW_OK:
            raise self._err(st, "kw_get_krylov_log")
        rows = np.zeros((n.value, LOG_FIXED + np_.value), dtype=np.complex128)
        w0 = np.zeros(np_.value, dtype=np.complex128)
        st = self._lib.kw_get_krylov_log(self._ctx, C.byref(n), C.byref(run), C.byref(np_), C.byref(thr),
                                         rows.ctypes.data_as(C.c_void_p), w0.ctypes.data_as(C.c_void_p))
        if st != KW_OK:
            raise self._err(st, "kw_get_krylov_log")
        return KrylovLog(rows, w0, thr.value, run.value)

    def recalc(self, z, log: KrylovLog | None = None, thresh: float | None = None, n_iter: int = -1,
               check: bool = True) -> RecalcResult:
        """kw_recalc: projections at shifts z from ``log`` (host) or, when log is
        None, from the device log of the last solve.  thresh defaults to the
        logged solve's tol*||b||."""
        zz, zp = _z_array(z)
        K = zz.size
        if log is not None:
            rows = np.ascontiguousarray(log.rows, dtype=np.complex128)
            w0 = np.ascontiguousarray(log.w0, dtype=np.complex128)
            n, npj = rows.shape[0] if n_iter < 0 else min(n_iter, rows.shape[0]), rows.shape[1] - LOG_FIXED
            thr = log.thresh if thresh is None else thresh
            lp, wp = rows.ctypes.data_as(C.c_void_p), w0.ctypes.data_as(C.c_void_p)
        else:
            nn, run, np_, t0 = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
            st = self._lib.kw_get_krylov_log(self._ctx, C.byref(nn), C.byref(run), C.byref(np_), C.byref(t0),
                                             None, None)
            if st != KW_OK:
                raise self._err(st, "kw_get_krylov_log")
            n, npj = n_iter, np_.value
            thr = t0.value if thresh is None else thresh
            lp, wp = None, None
        proj = np.zeros((K, max(npj, 1)), dtype=np.complex128)
        ci = np.zeros(K, dtype=np.int64)
        fr = np.zeros(K, dtype=np.float64)
        info = kw_solve_info()
        st = self._lib.kw_recalc(self._ctx, n, npj, thr, lp, wp, K, zp, proj.ctypes.data_as(C.c_void_p),
                                 ci.ctypes.data_as(C.c_void_p), fr.ctypes.data_as(C.c_void_p), C.byref(info))
        if check and st not in (KW_OK, KW_NOT_CONVERGED):
            raise self._err(st, "kw_recalc")
        return RecalcResult(proj[:, :npj], ci, fr, info.iters, info.n_converged, info.updates,
                            STATUS.get(st, str(st)))

    def set_kernel_timing(self, every: int):
        st = self._lib.kw_set_kernel_timing(self._ctx, every)
        if st != KW_OK:
            raise self._err(st, "kw_set_kernel_timing")

    def set_spmv_config(self, lanes: int = 0, val_f32: int = -1):
        st = self._lib.kw_set_spmv_config(self._ctx, lanes, val_f32)
        if st != KW_OK:
            raise self._err(st, "kw_set_spmv_config")

    def spmv_config(self):
        l, v = C.c_int(), C.c_int()
        st = self._lib.kw_get_spmv_config(self._ctx, C.byref(l), C.byref(v))
        if st != KW_OK:
            raise self._err(st, "kw_get_spmv_config")
        return l.value, v.value

    def stats(self) -> dict:
        s = kw_stats()
        st = self._lib.kw_get_stats(self._ctx, C.byref(s))
        if st != KW_OK:
            raise self._err(st, "kw_get_stats")
        return {"launches": s.launches, "timed_iters": s.timed_iters, "kernel_ms": list(s.kernel_ms),
                "tune_runs": s.tune_runs, "tune_hits": s.tune_hits}

    def prepare_batch(self, problems):
        """Device-resident inputs and outputs of a kw_solve_batched call, built once
        (problems as in solve_batched); run_batch(handle) then makes only the call."""
        t = self._torch
        n = len(problems)
        arr = (kw_instance * n)()
        keep, outs = [], []
        for i, pr in enumerate(problems):
            H = pr["H"]
            rp, cl, vl = self._dev(H.rowptr, t.int64), self._dev(H.col, t.int32), self._dev(H.val, t.float64)
            bd = self._dev(pr["b"], t.float64)
            zz, zp = _z_array(pr["z"])
            left = pr.get("left")
            ld = None if left is None else self._dev(np.atleast_2d(left), t.float64)
            nleft = 0 if ld is None else ld.shape[0]
            x = t.empty((zz.size, rp.numel() - 1), dtype=self.vec_dtype, device="cuda") if pr.get("full", True) \
                else None
            proj = np.zeros((zz.size, nleft + 1), dtype=np.complex128)
            keep += [rp, cl, vl, bd, zz, ld, x, proj]
            arr[i] = kw_instance(rp.numel() - 1, cl.numel(), rp.data_ptr(), cl.data_ptr(), vl.data_ptr(),
                                 bd.data_ptr(), zz.size, zp.value, nleft, None if ld is None else ld.data_ptr(),
                                 None if x is None else x.data_ptr(), proj.ctypes.data, float(pr.get("tol", 0.0)))
            outs.append((proj, x))
        return {"arr": arr, "keep": keep, "outs": outs, "n": n}

    def run_batch(self, handle, check: bool = True):
        """kw_solve_batched on a prepare_batch handle; one SolveResult per instance."""
        infos = (kw_solve_info * handle["n"])()
        st = self._lib.kw_solve_batched(self._ctx, handle["n"], handle["arr"], infos)
        if check and st not in (KW_OK, KW_NOT_CONVERGED):
            raise self._err(st, "kw_solve_batched")
        res = []
        for (proj, x), info in zip(handle["outs"], infos):
            res.append(SolveResult(proj.copy(), x, info.iters, info.n_converged, info.max_res, info.n_seed_switch,
                                   info.updates, info.seed, STATUS.get(info.status, str(info.status))))
        return res

    def solve_batched(self, problems, check: bool = True):
        """kw_solve_batched over a list of problems, each a dict with keys H (CSR with
        rowptr, col, val arrays), b, z and optionally left, full (default True) and
        tol.  Returns one SolveResult per problem."""
        return self.run_batch(self.prepare_batch(problems), check)

    def shift_combine(self, X, W):
        """kw_shift_combine: S = W X on the device for X a [K, m] complex128 or
        complex64 CUDA tensor and W a [nk, K] complex array (nk <= 16); returns the
        [nk, m] complex128 CUDA tensor S."""
        t = self._torch
        if X.dtype not in (t.complex128, t.complex64) or not X.is_cuda or not X.is_contiguous() or X.dim() != 2:
            raise ValueError("X must be a contiguous [K, m] complex128 or complex64 CUDA tensor")
        K, m = X.shape
        Wh = np.ascontiguousarray(np.asarray(W, dtype=np.complex128))
        if Wh.ndim != 2 or Wh.shape[1] != K:
            raise ValueError(f"W must be [nk, {K}]")
        S = t.empty((Wh.shape[0], m), dtype=t.complex128, device=X.device)
        elem = KW_ELEM_C64 if X.dtype == t.complex64 else KW_ELEM_C128
        st = self._lib.kw_shift_combine(self._ctx, m, K, C.c_void_p(X.data_ptr()), elem, Wh.shape[0],
                                        Wh.ctypes.data_as(C.c_void_p), C.c_void_p(S.data_ptr()))
        if st != KW_OK:
            raise self._err(st, "kw_shift_combine")
        return S

    def bilinear(self, terms, X, Y=None) -> np.ndarray:
        """kw_bilinear / kw_bilinear_c64: out[k][t] = y_k^T H_t x_k for device CSR terms
        (each a tuple of CUDA tensors (rowptr int64, col int32, val float64)) and X, Y
        [K, m] CUDA tensors, both complex128 or both complex64 (FP64 sums either way)."""
        t = self._torch
        K, m = X.shape
        if X.dtype not in (t.complex128, t.complex64) or not X.is_cuda or not X.is_contiguous():
            raise ValueError("X must be a contiguous complex128 or complex64 CUDA tensor [K, m]")
        if Y is not None and (Y.dtype != X.dtype or tuple(Y.shape) != tuple(X.shape) or not Y.is_cuda
                              or not Y.is_contiguous()):
            raise ValueError("Y must match X in dtype, shape and device and be contiguous")
        arr = (kw_csr_term * len(terms))()
        for i, (rp, cl, vl) in enumerate(terms):
            arr[i] = kw_csr_term(cl.numel(), rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
        out = np.zeros((K, len(terms)), dtype=np.complex128)
        fn, name = ((self._lib.kw_bilinear_c64, "kw_bilinear_c64") if X.dtype == t.complex64
                    else (self._lib.kw_bilinear, "kw_bilinear"))
        st = fn(self._ctx, m, len(terms), arr, K, C.c_void_p(X.data_ptr()),
                None if Y is None else C.c_void_p(Y.data_ptr()), out.ctypes.data_as(C.c_void_p))
        if st != KW_OK:
            raise self._err(st, name)
        return out

    def spmv_dot(self, zs: complex, r, q):
        """q = zs r - H r and t = r^T q on the device.  r, q: device tensors in the
        context's element layout (complex128 for f64, complex64 for c32, float32
        [m, 4] pairs (re.hi, re.lo, im.hi, im.lo) for df64)."""
        eb = 8 if self.prec == KW_C32V_F64S else 16
        for name, v in (("r", r), ("q", q)):
            if not v.is_cuda:
                raise ValueError(f"{name} must be a CUDA tensor")
            check_vector_bytes(name, v, self.m, eb)
        t = kw_c128()
        st = self._lib.kw_spmv_dot(self._ctx, kw_c128(zs.real, zs.imag), C.c_void_p(r.data_ptr()),
                                   C.c_void_p(q.data_ptr()), C.byref(t))
        if st != KW_OK:
            raise self._err(st, "kw_spmv_dot") from getattr(self, "_mv_error", None)
        return complex(t.re, t.im)
