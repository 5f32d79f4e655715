"""Python binding of the C ABI in include/dspg.h (argument marshalling only).

Every computation runs in the CUDA library ``libdspg.so``; this module only
turns numpy arrays (host memory) or torch tensors (device or host memory)
into pointers and sizes, and status codes into exceptions. There is no CPU
fallback: if the library cannot be loaded, ``load()`` raises.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

PLUS_TIMES_F64 = 0
MIN_PLUS_I32 = 1

SIZE_BOUND = 0
SIZE_EXACT = 1
SIZE_LEARNED = 2
EST_PARAMS = 4545

OP_INSERT = 0
OP_DELETE = 1
OP_SET = 2

_STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_STATE"}

_lock = threading.Lock()
_lib = None


class DspgError(RuntimeError):
    def __init__(self, status: int, msg: str, needed: int | None = None):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.needed = needed  # the result size a call reported with its error, where it reports one


class _Csr(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("on_device", C.c_int)]


class _Upd(C.Structure):
    _fields_ = [("n", C.c_int64), ("row", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("op", C.c_void_p), ("on_device", C.c_int)]


class _Opt(C.Structure):
    _fields_ = [("slack_min", C.c_int32), ("slack_div", C.c_int32), ("arena_headroom", C.c_double),
                ("keep_transpose", C.c_int32), ("exact_static", C.c_int32), ("bloom", C.c_int32)]


class _Form(C.Structure):
    _fields_ = [("trans_a", C.c_int32), ("trans_b", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double),
                ("alpha_i", C.c_int32), ("beta_i", C.c_int32), ("X", C.POINTER(_Csr))]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_updates", "n_unique", "n_insert", "n_update", "n_delete", "n_noop", "touched_rows", "affected_rows",
        "products", "nnz_written", "relocations", "compactions", "a_entries", "est_rows", "est_overflows",
        "algebraic", "table_slots", "masked_entries")]


class _Tuning(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("merge_k", "merge_ub", "lanes_min", "table_shift", "warp_max", "cta_max",
                                         "sort_max")]


def _debug() -> bool:
    return os.environ.get("DSPG_DEBUG", "") == "1"


def library_path() -> str:
    return _build.LIB_DEBUG if _debug() else _build.LIB


def load():
    """Load libdspg.so (compiling it first if it is missing or stale); with
    DSPG_DEBUG=1 in the environment, the debug build libdspg_debug.so, whose
    kernels check indices and room before their accesses."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build(debug=_debug())
        lib = C.CDLL(path)
        p, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        lib.dspg_build.restype = i32
        lib.dspg_build.argtypes = [C.POINTER(p), C.POINTER(_Csr), C.POINTER(_Csr), i32, C.POINTER(_Opt), p]
        lib.dspg_build_form.restype = i32
        lib.dspg_build_form.argtypes = [C.POINTER(p), C.POINTER(_Csr), C.POINTER(_Csr), i32, C.POINTER(_Form),
                                        C.POINTER(_Opt), p]
        lib.dspg_apply_batch.restype = i32
        lib.dspg_apply_batch.argtypes = [p, C.POINTER(_Upd), C.POINTER(_Upd), C.POINTER(_Stats), p]
        lib.dspg_apply_batch_algebraic.restype = i32
        lib.dspg_apply_batch_algebraic.argtypes = [p, C.POINTER(_Upd), C.POINTER(_Upd), C.POINTER(_Stats), p]
        for name in ("dspg_read_C", "dspg_read_A", "dspg_read_bloom"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [p, C.POINTER(i64), p, p, p, i32, p]
        lib.dspg_read_rows_C.restype = i32
        lib.dspg_read_rows_C.argtypes = [p, p, i64, C.POINTER(i64), p, p, p, i32, p]
        lib.dspg_debug_build.restype = i32
        lib.dspg_debug_build.argtypes = []
        lib.dspg_fault_inject.restype = i32
        lib.dspg_fault_inject.argtypes = [C.c_char_p]
        lib.dspg_read_affected_C.restype = i32
        lib.dspg_read_affected_C.argtypes = [p, i64, i64, C.POINTER(i64), C.POINTER(i64), p, p, p, p, i32, p]
        lib.dspg_apply_read_affected.restype = i32
        lib.dspg_apply_read_affected.argtypes = [p, C.POINTER(_Upd), C.POINTER(_Upd), i64, i64, C.POINTER(i64),
                                                 C.POINTER(i64), p, p, p, p, C.POINTER(_Stats), p]
        lib.dspg_last_affected.restype = i32
        lib.dspg_last_affected.argtypes = [p, C.POINTER(i64), p, i32, p]
        lib.dspg_recompute_all.restype = i32
        lib.dspg_recompute_all.argtypes = [p, p]
        lib.dspg_info.restype = i32
        lib.dspg_info.argtypes = [p] + [C.POINTER(i64)] * 5
        lib.dspg_set_profiling.restype = i32
        lib.dspg_set_profiling.argtypes = [p, i32]
        lib.dspg_stage_times.restype = i32
        lib.dspg_stage_times.argtypes = [p, C.POINTER(C.c_float), i32]
        lib.dspg_kernel_launches.restype = C.c_ulonglong
        lib.dspg_kernel_launches.argtypes = []
        lib.dspg_reserve.restype = i32
        lib.dspg_reserve.argtypes = [p, i64, i64, p]
        lib.dspg_run_counts.restype = i32
        lib.dspg_run_counts.argtypes = [p, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        lib.dspg_multiply_rows_noalloc.restype = i32
        lib.dspg_multiply_rows_noalloc.argtypes = [C.POINTER(_Csr), C.POINTER(_Csr), i32, p, i64, p, p, p, i64,
                                                   C.POINTER(i64), p]
        lib.dspg_set_tuning.restype = i32
        lib.dspg_set_tuning.argtypes = [p, C.POINTER(_Tuning)]
        lib.dspg_get_tuning.restype = i32
        lib.dspg_get_tuning.argtypes = [p, C.POINTER(_Tuning)]
        lib.dspg_tuning_candidate.restype = i32
        lib.dspg_tuning_candidate.argtypes = [i32, C.POINTER(_Tuning)]
        lib.dspg_autotune.restype = i32
        lib.dspg_autotune.argtypes = [p, C.POINTER(_Upd), C.POINTER(_Upd), i64, C.POINTER(_Tuning),
                                      C.POINTER(C.c_float), i32, C.POINTER(i32), p]
        lib.dspg_group_create.restype = i32
        lib.dspg_group_create.argtypes = [C.POINTER(p), C.POINTER(p), i64]
        lib.dspg_group_apply.restype = i32
        lib.dspg_group_apply.argtypes = [p, C.POINTER(_Upd), C.POINTER(_Upd), C.POINTER(_Stats), C.POINTER(i32), p]
        lib.dspg_group_destroy.restype = None
        lib.dspg_group_destroy.argtypes = [p]
        lib.dspg_group_last_error.restype = C.c_char_p
        lib.dspg_group_last_error.argtypes = [p]
        lib.dspg_estimator_create.restype = i32
        lib.dspg_estimator_create.argtypes = [C.POINTER(p), p]
        lib.dspg_estimator_params.restype = i32
        lib.dspg_estimator_params.argtypes = [p, p, p]
        lib.dspg_estimator_grad.restype = i32
        lib.dspg_estimator_grad.argtypes = [p, p, p, i64, p, C.POINTER(C.c_double), p]
        lib.dspg_estimator_train.restype = i32
        lib.dspg_estimator_train.argtypes = [p, p, p, i64, i64, i64, C.c_float, C.POINTER(C.c_double), p]
        lib.dspg_estimator_predict.restype = i32
        lib.dspg_estimator_predict.argtypes = [p, p, i64, p, p]
        lib.dspg_estimator_last_error.restype = C.c_char_p
        lib.dspg_estimator_last_error.argtypes = [p]
        lib.dspg_estimator_destroy.restype = None
        lib.dspg_estimator_destroy.argtypes = [p]
        lib.dspg_row_features.restype = i32
        lib.dspg_row_features.argtypes = [p, p, i64, p, p, p]
        lib.dspg_set_sizing.restype = i32
        lib.dspg_set_sizing.argtypes = [p, i32, p, i32, C.c_float]
        lib.dspg_footprint.restype = i32
        lib.dspg_footprint.argtypes = [p, C.POINTER(_Upd), p, p, i32, C.POINTER(i32), C.POINTER(i64), p]
        lib.dspg_footprint_batch.restype = i32
        lib.dspg_footprint_batch.argtypes = [p, C.POINTER(_Upd), i64, p, p, i32, C.POINTER(i32), C.POINTER(i64), p]
        lib.dspg_apply_batch_async.restype = i32
        lib.dspg_apply_batch_async.argtypes = [p, C.POINTER(_Upd), C.POINTER(_Upd), p]
        lib.dspg_apply_batch_wait.restype = i32
        lib.dspg_apply_batch_wait.argtypes = [p, C.POINTER(_Stats), p]
        lib.dspg_destroy.restype = None
        lib.dspg_destroy.argtypes = [p]
        lib.dspg_last_error.restype = C.c_char_p
        lib.dspg_last_error.argtypes = [p]
        _lib = lib
        return lib


EXPORTED = ["dspg_build", "dspg_build_form", "dspg_apply_batch", "dspg_apply_batch_algebraic", "dspg_read_C", "dspg_read_A",
            "dspg_read_bloom", "dspg_read_rows_C", "dspg_read_affected_C", "dspg_apply_read_affected",
            "dspg_fault_inject", "dspg_debug_build",
            "dspg_last_affected", "dspg_recompute_all", "dspg_info", "dspg_set_profiling", "dspg_stage_times",
            "dspg_kernel_launches", "dspg_run_counts", "dspg_reserve", "dspg_multiply_rows_noalloc", "dspg_set_tuning", "dspg_get_tuning",
            "dspg_tuning_candidate", "dspg_autotune", "dspg_group_create", "dspg_group_apply", "dspg_group_destroy",
            "dspg_group_last_error", "dspg_estimator_create", "dspg_estimator_params", "dspg_estimator_grad",
            "dspg_estimator_train", "dspg_estimator_predict", "dspg_estimator_last_error", "dspg_estimator_destroy",
            "dspg_row_features", "dspg_set_sizing", "dspg_footprint", "dspg_footprint_batch",
            "dspg_apply_batch_async", "dspg_apply_batch_wait", "dspg_destroy",
            "dspg_last_error"]

TUNING_FIELDS = [n for n, _ in _Tuning._fields_]


def _tuning_dict(t: _Tuning) -> dict:
    return {n: int(getattr(t, n)) for n in TUNING_FIELDS}


def tuning_candidates() -> list[dict]:
    """The autotuner's built-in candidate tunings, in its order."""
    lib, out, k = load(), [], 0
    while True:
        t = _Tuning()
        if lib.dspg_tuning_candidate(k, C.byref(t)) != 0:
            return out
        out.append(_tuning_dict(t))
        k += 1

STAGES = ["sort", "classify", "detect", "merge", "commit", "transpose", "size", "numeric"]


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().dspg_kernel_launches())


def _vdtype(sr: int):
    return np.float64 if sr == PLUS_TIMES_F64 else np.int32


_PINNED = {}


def _host_empty(n: int, dtype) -> np.ndarray:
    """An uninitialised host array for results copied from the device: page-
    locked memory from torch's caching host allocator when a GPU is there (the
    copy runs at full speed and touches no fresh pages; freed arrays give their
    blocks back for the next read), else plain numpy memory."""
    if _PINNED.get("ok") is None:
        try:
            import torch
            _PINNED["ok"] = bool(torch.cuda.is_available())
            _PINNED["torch"] = torch
        except ImportError:
            _PINNED["ok"] = False
    if not _PINNED["ok"]:
        return np.empty(n, dtype)
    torch = _PINNED["torch"]
    tdt = {np.dtype(np.int64): torch.int64, np.dtype(np.int32): torch.int32,
           np.dtype(np.float64): torch.float64}[np.dtype(dtype)]
    return torch.empty(n, dtype=tdt, pin_memory=True).numpy()


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, keep: list):
    """Pointer of a numpy array or torch tensor (contiguous); returns (ptr, on_device)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        x = x.contiguous()
        keep.append(x)
        return x.data_ptr(), int(x.is_cuda)
    a = np.ascontiguousarray(x)
    keep.append(a)
    return a.ctypes.data, 0


def _stream(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def fault_inject(spec: str | None) -> None:
    """Arm host-side fault injection (dspg_fault_inject): "alloc@N" fails the
    N-th device allocation, "validate@N" the N-th batch check; None or ""
    disarms."""
    lib = load()
    st = lib.dspg_fault_inject(spec.encode() if spec else None)
    if st != 0:
        raise DspgError(st, lib.dspg_last_error(None).decode())


class DynamicSpGEMM:
    """C = A B over a semiring, kept up to date under update batches.

    ``A`` (and ``B``) are objects with ``nrows, ncols, rowptr, col, val``
    (e.g. ``workloads.CSR``; arrays may be numpy or torch). ``B=None`` means
    C = A A with one batch updating both operands.

    The general form C = alpha op(A) op(B) (+) beta X (dspg_build_form):
    ``trans_a``/``trans_b`` multiply by the transposes, ``alpha``/``beta``
    scale (multiply in (+,.), add in (min,+)) and ``X`` is a fixed matrix of
    C's shape; batches stay in the caller's coordinates.

    ``bloom=True`` keeps C's Bloom filter F and applies every batch by the
    entry-level masked recompute of Algorithm 2 (``read_bloom`` reads F)."""

    def __init__(self, A, B=None, semiring: int | None = None, slack_min: int = 4, slack_div: int = 4,
                 arena_headroom: float = 1.5, keep_transpose: int = -1, exact_static: int = 0, stream=None,
                 trans_a: bool = False, trans_b: bool = False, alpha=None, beta=None, X=None, bloom: bool = False):
        self._lib = load()
        self._h = C.c_void_p()
        if semiring is None:
            semiring = PLUS_TIMES_F64 if np.dtype(_dtype_of(A.val)) == np.float64 else MIN_PLUS_I32
        self.sr = semiring
        keep: list = []
        ca = self._csr(A, keep)
        cb = self._csr(B, keep) if B is not None else None
        opt = _Opt(slack_min, slack_div, arena_headroom, keep_transpose, exact_static, int(bool(bloom)))
        if trans_a or trans_b or alpha is not None or beta is not None or X is not None:
            cx = self._csr(X, keep) if X is not None else None
            pt = semiring == PLUS_TIMES_F64
            form = _Form(int(trans_a), int(trans_b),
                         float(alpha if alpha is not None else 1.0) if pt else 0.0,
                         float(beta if beta is not None else 1.0) if pt else 0.0,
                         0 if pt else int(alpha if alpha is not None else 0),
                         0 if pt else int(beta if beta is not None else 0),
                         C.pointer(cx) if cx is not None else None)
            keep.append(cx)
            st = self._lib.dspg_build_form(C.byref(self._h), C.byref(ca), C.byref(cb) if cb is not None else None,
                                           semiring, C.byref(form), C.byref(opt), _stream(stream))
        else:
            st = self._lib.dspg_build(C.byref(self._h), C.byref(ca), C.byref(cb) if cb is not None else None,
                                      semiring, C.byref(opt), _stream(stream))
        if st != 0:
            raise DspgError(st, self._lib.dspg_last_error(None).decode())
        self.b_is_a = B is None
        self.a_shape = (int(A.nrows), int(A.ncols))  # the caller's A (read_A's shape)

    def _csr(self, M, keep) -> _Csr:
        rp, dev = _ptr(_as_int(M.rowptr, np.int64), keep)
        col, _ = _ptr(_as_int(M.col, np.int32), keep)
        val, _ = _ptr(_as_val(M.val, self.sr), keep)
        nnz = int(M.rowptr[-1])
        return _Csr(M.nrows, M.ncols, nnz, rp, col, val, dev)

    def _check(self, st):
        if st != 0:
            raise DspgError(st, self._lib.dspg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dspg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _upd(self, b, keep) -> _Upd:
        row, dev = _ptr(_as_int(b.row, np.int32), keep)
        col, _ = _ptr(_as_int(b.col, np.int32), keep)
        val, _ = _ptr(_as_val(b.val, self.sr), keep)
        op, _ = _ptr(_as_int(b.op, np.uint8), keep)
        return _Upd(len(b.row), row, col, val, op, dev)

    def apply_batch(self, dA=None, dB=None, stream=None, algebraic: bool = False) -> dict:
        """Apply a batch (dspg_apply_batch); with ``algebraic`` through
        dspg_apply_batch_algebraic (the delta path of Eq. 1 for batches that
        only insert, the row path otherwise)."""
        keep: list = []
        ua = self._upd(dA, keep) if dA is not None else None
        ub = self._upd(dB, keep) if dB is not None else None
        stats = _Stats()
        fn = self._lib.dspg_apply_batch_algebraic if algebraic else self._lib.dspg_apply_batch
        st = fn(self._h, C.byref(ua) if ua is not None else None, C.byref(ub) if ub is not None else None,
                C.byref(stats), _stream(stream))
        self._check(st)
        return {name: getattr(stats, name) for name, _ in _Stats._fields_}

    def _read(self, fn, ncols: int, stream=None, nrows: int | None = None) -> "CsrArrays":
        s = _stream(stream)
        nnz = C.c_int64()
        self._check(fn(self._h, C.byref(nnz), None, None, None, 0, s))
        n = self.info()["n"] if nrows is None else nrows
        rp = _host_empty(n + 1, np.int64)
        col = _host_empty(nnz.value, np.int32)
        val = _host_empty(nnz.value, _vdtype(self.sr))
        self._check(fn(self._h, C.byref(nnz), rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0, s))
        return CsrArrays(n, ncols, rp, col, val)

    def read_C(self, stream=None) -> "CsrArrays":
        """C' in canonical CSR (host numpy arrays)."""
        return self._read(self._lib.dspg_read_C, self.info()["m"], stream)

    def read_bloom(self, stream=None) -> "CsrArrays":
        """C's Bloom filter F (handles built with ``bloom=True``) in canonical
        CSR: the pattern of C with one uint64 word per entry as ``val``."""
        s = _stream(stream)
        nnz = C.c_int64()
        self._check(self._lib.dspg_read_bloom(self._h, C.byref(nnz), None, None, None, 0, s))
        n = self.info()["n"]
        rp = _host_empty(n + 1, np.int64)
        col = _host_empty(nnz.value, np.int32)
        words = _host_empty(nnz.value, np.int64).view(np.uint64)
        self._check(self._lib.dspg_read_bloom(self._h, C.byref(nnz), rp.ctypes.data, col.ctypes.data,
                                              words.ctypes.data, 0, s))
        return CsrArrays(n, self.info()["m"], rp, col, words)

    def read_A(self, stream=None) -> "CsrArrays":
        """A' in canonical CSR (host numpy arrays), in the caller's coordinates."""
        return self._read(self._lib.dspg_read_A, self.a_shape[1], stream, nrows=self.a_shape[0])

    def read_C_device(self, stream=None):
        """C as torch device tensors (rowptr, col, val)."""
        import torch
        nnz = C.c_int64()
        s = _stream(stream)
        self._check(self._lib.dspg_read_C(self._h, C.byref(nnz), None, None, None, 1, s))
        n = self.info()["n"]
        rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz.value, 1), dtype=torch.float64 if self.sr == PLUS_TIMES_F64 else torch.int32,
                          device="cuda")
        self._check(self._lib.dspg_read_C(self._h, C.byref(nnz), rp.data_ptr(), col.data_ptr(), val.data_ptr(), 1, s))
        return rp, col[: nnz.value], val[: nnz.value]

    def read_affected(self, stream=None, out=None):
        """(rows, rowptr, col, val) of the last batch's affected rows of C', in
        one call (dspg_read_affected_C): R ascending and its rows canonical,
        in page-locked host arrays sized with room for the next batches.
        out: caller-owned host arrays (rows int32, rowptr int64 with one more
        entry than rows, col int32, val of the semiring's type), reused when
        they hold the result (a loop that reads every batch keeps one set);
        the result is then views of them."""
        s = _stream(stream)
        n = C.c_int64()
        nnz = C.c_int64()
        cap = getattr(self, "_aff_cap", (0, 0))
        if out is not None:
            o_rows, o_rp, o_col, o_val = out
            if (o_rows.dtype != np.int32 or o_rp.dtype != np.int64 or o_col.dtype != np.int32
                    or o_val.dtype != _vdtype(self.sr) or o_rp.shape[0] < o_rows.shape[0] + 1
                    or o_val.shape[0] < o_col.shape[0]):
                raise ValueError("read_affected: out arrays of the wrong types or sizes")
            st = self._lib.dspg_read_affected_C(self._h, o_rows.shape[0], o_col.shape[0], C.byref(n), C.byref(nnz),
                                                o_rows.ctypes.data, o_rp.ctypes.data, o_col.ctypes.data,
                                                o_val.ctypes.data, 0, s)
            if st == 0:
                k, e = n.value, nnz.value
                return o_rows[:k], o_rp[:k + 1], o_col[:e], o_val[:e]
            if not (st == 1 and (n.value > o_rows.shape[0] or nnz.value > o_col.shape[0])):
                self._check(st)
            cap = (n.value + n.value // 4 + 1, nnz.value + nnz.value // 4 + 1)  # too small: arrays of our own
        for _ in range(2):
            if cap[0] == 0:  # sizes first
                self._check(self._lib.dspg_read_affected_C(self._h, 0, 0, C.byref(n), C.byref(nnz), None, None, None,
                                                           None, 0, s))
                cap = (n.value + n.value // 4 + 1, nnz.value + nnz.value // 4 + 1)  # room for the next batches
            rows = _host_empty(cap[0], np.int32)
            rp = _host_empty(cap[0] + 1, np.int64)
            col = _host_empty(cap[1], np.int32)
            val = _host_empty(cap[1], _vdtype(self.sr))
            st = self._lib.dspg_read_affected_C(self._h, cap[0], cap[1], C.byref(n), C.byref(nnz), rows.ctypes.data,
                                                rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0, s)
            if st == 1 and (n.value > cap[0] or nnz.value > cap[1]):
                cap = (max(n.value, cap[0]) + n.value // 4 + 1, max(nnz.value, cap[1]) + nnz.value // 4 + 1)
                continue
            self._check(st)
            self._aff_cap = (max(cap[0], n.value), max(cap[1], nnz.value))
            k, e = n.value, nnz.value
            return rows[:k], rp[:k + 1], col[:e], val[:e]
        raise DspgError(1, "read_affected: sizes kept changing")

    def apply_read_affected(self, dA=None, dB=None, stream=None, out=None):
        """apply_batch and then read_affected in one call
        (dspg_apply_read_affected): returns (stats, (rows, rowptr, col,
        val)).  With out (caller-owned page-locked arrays, as read_affected
        takes them) the read is enqueued behind the batch and the stream is
        synchronised once; without, the two calls run one after the other."""
        if out is None:
            stats = self.apply_batch(dA, dB, stream)
            return stats, self.read_affected(stream)
        o_rows, o_rp, o_col, o_val = out
        if (o_rows.dtype != np.int32 or o_rp.dtype != np.int64 or o_col.dtype != np.int32
                or o_val.dtype != _vdtype(self.sr) or o_rp.shape[0] < o_rows.shape[0] + 1
                or o_val.shape[0] < o_col.shape[0]):
            raise ValueError("apply_read_affected: out arrays of the wrong types or sizes")
        keep: list = []
        ua = self._upd(dA, keep) if dA is not None else None
        ub = self._upd(dB, keep) if dB is not None else None
        stats = _Stats()
        n = C.c_int64()
        nnz = C.c_int64()
        st = self._lib.dspg_apply_read_affected(self._h, C.byref(ua) if ua is not None else None,
                                                C.byref(ub) if ub is not None else None, o_rows.shape[0],
                                                o_col.shape[0], C.byref(n), C.byref(nnz), o_rows.ctypes.data,
                                                o_rp.ctypes.data, o_col.ctypes.data, o_val.ctypes.data,
                                                C.byref(stats), _stream(stream))
        sd = {name: getattr(stats, name) for name, _ in _Stats._fields_}
        if st == 0:
            k, e = n.value, nnz.value
            return sd, (o_rows[:k], o_rp[:k + 1], o_col[:e], o_val[:e])
        if st == 1 and (n.value > o_rows.shape[0] or nnz.value > o_col.shape[0]):
            return sd, self.read_affected(stream)  # applied; the arrays were too small for the read
        self._check(st)

    def read_rows_C(self, rows, stream=None):
        rows = np.ascontiguousarray(rows, np.int32)
        nnz = C.c_int64()
        s = _stream(stream)
        self._check(self._lib.dspg_read_rows_C(self._h, rows.ctypes.data, rows.shape[0], C.byref(nnz), None, None,
                                               None, 0, s))
        rp = _host_empty(rows.shape[0] + 1, np.int64)
        col = _host_empty(nnz.value, np.int32)
        val = _host_empty(nnz.value, _vdtype(self.sr))
        self._check(self._lib.dspg_read_rows_C(self._h, rows.ctypes.data, rows.shape[0], C.byref(nnz),
                                               rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0, s))
        return rp, col, val

    def last_affected(self, stream=None) -> np.ndarray:
        cnt = C.c_int64()
        s = _stream(stream)
        self._check(self._lib.dspg_last_affected(self._h, C.byref(cnt), None, 0, s))
        out = _host_empty(cnt.value, np.int32)
        self._check(self._lib.dspg_last_affected(self._h, C.byref(cnt), out.ctypes.data, 0, s))
        return out

    def set_profiling(self, on: bool = True) -> None:
        self._check(self._lib.dspg_set_profiling(self._h, int(on)))

    def stage_times(self) -> dict:
        ms = (C.c_float * len(STAGES))()
        self._check(self._lib.dspg_stage_times(self._h, ms, len(STAGES)))
        return dict(zip(STAGES, [float(x) for x in ms]))

    def set_tuning(self, tuning: dict | None = None) -> None:
        """Row-bin thresholds of the recompute (None: the defaults)."""
        t = _Tuning(**tuning) if tuning is not None else None
        self._check(self._lib.dspg_set_tuning(self._h, C.byref(t) if t is not None else None))

    def get_tuning(self) -> dict:
        t = _Tuning()
        self._check(self._lib.dspg_get_tuning(self._h, C.byref(t)))
        return _tuning_dict(t)

    def autotune(self, batches, batches_b=None, stream=None) -> tuple[dict, list[float]]:
        """Apply `batches` (real updates) while timing every candidate tuning
        on each batch's affected rows; keeps and returns the fastest, with the
        per-candidate total milliseconds."""
        keep: list = []
        ua = (_Upd * len(batches))(*[self._upd(b, keep) for b in batches])
        ub = (_Upd * len(batches))(*[self._upd(b, keep) for b in batches_b]) if batches_b is not None else None
        best = _Tuning()
        ms = (C.c_float * 64)()
        nc = C.c_int()
        self._check(self._lib.dspg_autotune(self._h, ua, ub, len(batches), C.byref(best), ms, 64, C.byref(nc),
                                            _stream(stream)))
        return _tuning_dict(best), [float(ms[k]) for k in range(nc.value)]

    def set_sizing(self, mode: int, estimator: "Estimator | None" = None, est_min: int = 128,
                   margin: float = 0.25) -> None:
        """How the recompute sizes its hash tables: SIZE_BOUND, SIZE_EXACT or
        SIZE_LEARNED (with an Estimator, whose weights are copied)."""
        e = estimator._e if estimator is not None else None
        self._check(self._lib.dspg_set_sizing(self._h, mode, e, est_min, margin))

    def row_features(self, rows=None, stream=None):
        """(X, y) as torch tensors on the device: the estimator's features of
        rows of C (all rows when rows is None) and log2(1 + nnz(C_i))."""
        import torch
        keep: list = []
        if rows is None:
            n = self.info()["n"]
            rp = None
        else:
            rows = rows if _is_torch(rows) and rows.is_cuda else torch.as_tensor(np.asarray(rows, np.int32)).cuda()
            n = int(rows.shape[0])
            rp, _ = _ptr(rows, keep)
        X = torch.empty((max(n, 1), 4), dtype=torch.float32, device="cuda")
        y = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        self._check(self._lib.dspg_row_features(self._h, rp, n, X.data_ptr(), y.data_ptr(), _stream(stream)))
        return X[:n], y[:n]

    def footprint(self, batch, f, u=None, or_anyway: bool = False, stream=None):
        """Write the footprint of an A batch into the device bitmap f (torch
        int32, ceil(n/32) words).  Returns (rows in f, admitted): with a wave
        bitmap u, admitted tells whether f was disjoint from u (and u |= f
        then, or always with or_anyway); without u, admitted is None."""
        keep: list = []
        ub = self._upd(batch, keep)
        adm = C.c_int()
        rows = C.c_int64()
        self._check(self._lib.dspg_footprint(self._h, C.byref(ub), f.data_ptr(), u.data_ptr() if u is not None else None,
                                             int(or_anyway), C.byref(adm), C.byref(rows), _stream(stream)))
        return int(rows.value), (bool(adm.value) if u is not None else None)

    def footprint_batch(self, batches, f, u, or_anyway: bool = False, stream=None):
        """Footprints of k batches into the rows of f (torch int32, k x
        ceil(n/32)) and their admission against the wave bitmap u, in one
        call (dspg_footprint_batch).  Returns (admitted, rows) lists."""
        k = len(batches)
        if k == 0:
            return [], []
        keep: list = []
        arr = (_Upd * k)(*[self._upd(b, keep) for b in batches])
        adm = (C.c_int * k)()
        rows = (C.c_int64 * k)()
        self._check(self._lib.dspg_footprint_batch(self._h, arr, k, f.data_ptr(), u.data_ptr(), int(or_anyway), adm,
                                                   rows, _stream(stream)))
        return [bool(x) for x in adm], [int(x) for x in rows]

    def apply_batch_async(self, dA=None, dB=None, stream=None):
        """Enqueue a batch and return (dspg_apply_batch_async); the arrays must
        stay alive until apply_batch_wait."""
        self._async_keep: list = []
        ua = self._upd(dA, self._async_keep) if dA is not None else None
        ub = self._upd(dB, self._async_keep) if dB is not None else None
        self._async_keep.extend([ua, ub, dA, dB])
        self._check(self._lib.dspg_apply_batch_async(self._h, C.byref(ua) if ua is not None else None,
                                                     C.byref(ub) if ub is not None else None, _stream(stream)))

    def apply_batch_wait(self, stream=None) -> dict:
        stats = _Stats()
        try:
            self._check(self._lib.dspg_apply_batch_wait(self._h, C.byref(stats), _stream(stream)))
        finally:
            self._async_keep = []
        return {name: getattr(stats, name) for name, _ in _Stats._fields_}

    def reserve(self, nA: int, nB: int = 0, stream=None) -> None:
        """Launch sizes for batches up to nA (nB) entries inside a group
        (dspg_reserve)."""
        self._check(self._lib.dspg_reserve(self._h, int(nA), int(nB), _stream(stream)))

    def run_counts(self) -> dict:
        """How this handle's batches ran: graph replays, captures, eager runs."""
        v = [C.c_int64() for _ in range(3)]
        self._check(self._lib.dspg_run_counts(self._h, *[C.byref(x) for x in v]))
        return dict(zip(("replayed", "captured", "eager"), [x.value for x in v]))

    def recompute_all(self, stream=None) -> None:
        self._check(self._lib.dspg_recompute_all(self._h, _stream(stream)))

    def info(self) -> dict:
        v = [C.c_int64() for _ in range(5)]
        self._check(self._lib.dspg_info(self._h, *[C.byref(x) for x in v]))
        return dict(zip(("n", "k", "m", "nnz_a", "nnz_c"), [x.value for x in v]))


class Estimator:
    """The learned row-size estimator (include/dspg.h): a 4-64-64-1 network
    with bfloat16 weights, trained on the GPU by the library's kernels."""

    def __init__(self, params):
        self._lib = load()
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if p.shape != (EST_PARAMS,):
            raise ValueError(f"need {EST_PARAMS} parameters")
        self._e = C.c_void_p()
        st = self._lib.dspg_estimator_create(C.byref(self._e), p.ctypes.data)
        if st != 0:
            raise DspgError(st, self._lib.dspg_last_error(None).decode())

    def _check(self, st):
        if st != 0:
            raise DspgError(st, self._lib.dspg_estimator_last_error(self._e).decode())

    def params(self, stream=None) -> np.ndarray:
        out = np.empty(EST_PARAMS, dtype=np.float32)
        self._check(self._lib.dspg_estimator_params(self._e, out.ctypes.data, _stream(stream)))
        return out

    @staticmethod
    def _dev(x, dt):
        import torch
        t = x if _is_torch(x) else torch.as_tensor(np.asarray(x, dtype=dt))
        return t.to(device="cuda", dtype=torch.float32).contiguous()

    def grad(self, X, y, stream=None):
        """(loss, dL/dw) at the current weights; the weights do not change."""
        X, y = self._dev(X, np.float32), self._dev(y, np.float32)
        g = np.empty(EST_PARAMS, dtype=np.float32)
        loss = C.c_double()
        self._check(self._lib.dspg_estimator_grad(self._e, X.data_ptr(), y.data_ptr(), int(X.shape[0]), g.ctypes.data,
                                                  C.byref(loss), _stream(stream)))
        return loss.value, g

    def train(self, X, y, batch: int = 4096, steps: int = 1000, lr: float = 1e-3, stream=None) -> float:
        X, y = self._dev(X, np.float32), self._dev(y, np.float32)
        loss = C.c_double()
        self._check(self._lib.dspg_estimator_train(self._e, X.data_ptr(), y.data_ptr(), int(X.shape[0]), batch, steps,
                                                   lr, C.byref(loss), _stream(stream)))
        return loss.value

    def predict(self, X, stream=None):
        import torch
        X = self._dev(X, np.float32)
        out = torch.empty(max(int(X.shape[0]), 1), dtype=torch.float32, device="cuda")
        self._check(self._lib.dspg_estimator_predict(self._e, X.data_ptr(), int(X.shape[0]), out.data_ptr(),
                                                     _stream(stream)))
        return out[:X.shape[0]]

    def close(self):
        if getattr(self, "_e", None) is not None and self._e.value:
            self._lib.dspg_estimator_destroy(self._e)
            self._e = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Several independent DynamicSpGEMM instances whose batches are applied
    together, as branches of one CUDA graph (one graph launch per apply once
    the batch sizes repeat)."""

    def __init__(self, members):
        self._lib = load()
        self.members = list(members)
        hs = (C.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        self._g = C.c_void_p()
        st = self._lib.dspg_group_create(C.byref(self._g), hs, len(self.members))
        if st != 0:
            raise DspgError(st, self._lib.dspg_group_last_error(None).decode())

    def apply(self, batches, batches_b=None, stream=None, raise_on_error: bool = True):
        """batches[t] (or None) for member t; returns (stats list, status list)."""
        n = len(self.members)
        if len(batches) != n:
            raise ValueError("one batch (or None) per member")
        keep: list = []
        empty = _Upd(0, None, None, None, None, 0)
        ua = (_Upd * n)(*[m._upd(b, keep) if b is not None else empty for m, b in zip(self.members, batches)])
        ub = None
        if batches_b is not None:
            ub = (_Upd * n)(*[m._upd(b, keep) if b is not None else empty for m, b in zip(self.members, batches_b)])
        stats = (_Stats * n)()
        status = (C.c_int * n)()
        st = self._lib.dspg_group_apply(self._g, ua, ub, stats, status, _stream(stream))
        if st != 0 and raise_on_error:
            raise DspgError(st, self._lib.dspg_group_last_error(self._g).decode())
        return ([{name: getattr(x, name) for name, _ in _Stats._fields_} for x in stats], [int(x) for x in status])

    def close(self):
        if getattr(self, "_g", None) is not None and self._g.value:
            self._lib.dspg_group_destroy(self._g)
            self._g = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def multiply_rows_noalloc(A, B, rows, semiring: int | None = None, stream=None, capacity: int | None = None,
                          query_only: bool = False):
    """Rows `rows` of C = A B through dspg_multiply_rows_noalloc, for callers
    that cannot let the library allocate device memory (the call itself
    allocates nothing: its working memory is a fixed array in the library).

    A and B are objects with ``nrows, ncols, rowptr, col, val`` whose arrays
    are CUDA tensors; rows is a CUDA int32 tensor.  The output tensors are
    allocated here by torch, on the caller's side of the boundary.  Returns
    (rowptr, col, val) as CUDA tensors; with ``query_only`` the size query
    alone, as (rowptr, nnz).  ``capacity`` sizes the output buffers of the
    second call (default: the size the query returned)."""
    import torch
    lib = load()
    keep: list = []
    if semiring is None:
        semiring = PLUS_TIMES_F64 if A.val.dtype == torch.float64 else MIN_PLUS_I32

    def csr(M):
        rp = M.rowptr.to(torch.int64).contiguous()
        col = M.col.to(torch.int32).contiguous()
        val = M.val.contiguous()
        keep.extend([rp, col, val])
        return _Csr(M.nrows, M.ncols, int(rp[-1].item()), rp.data_ptr(), col.data_ptr(), val.data_ptr(), 1)

    ca, cb = csr(A), csr(B)
    rows = rows.to(torch.int32).contiguous()
    n = rows.numel()
    rp = torch.empty(n + 1, dtype=torch.int64, device=rows.device)
    nnz = C.c_int64()
    s = _stream(stream)
    st = lib.dspg_multiply_rows_noalloc(C.byref(ca), C.byref(cb), semiring, rows.data_ptr(), n, rp.data_ptr(), None,
                                        None, 0, C.byref(nnz), s)
    if st != 0:
        raise DspgError(st, lib.dspg_last_error(None).decode())
    if query_only:
        return rp, nnz.value
    cap = max(nnz.value, 1) if capacity is None else int(capacity)
    col = torch.empty(max(cap, 1), dtype=torch.int32, device=rows.device)
    val = torch.empty(max(cap, 1), dtype=torch.float64 if semiring == PLUS_TIMES_F64 else torch.int32, device=rows.device)
    st = lib.dspg_multiply_rows_noalloc(C.byref(ca), C.byref(cb), semiring, rows.data_ptr(), n, rp.data_ptr(),
                                        col.data_ptr(), val.data_ptr(), cap, C.byref(nnz), s)
    if st != 0:
        raise DspgError(st, lib.dspg_last_error(None).decode(), needed=nnz.value)
    return rp, col[: nnz.value], val[: nnz.value]


class CsrArrays:
    """A canonical CSR read back from the library (rowptr int64, col int32,
    val float64 or int32)."""

    def __init__(self, nrows, ncols, rowptr, col, val):
        self.nrows, self.ncols, self.rowptr, self.col, self.val = nrows, ncols, rowptr, col, val

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.nrows, dtype=np.int64), np.diff(self.rowptr))


def _dtype_of(v):
    if _is_torch(v):
        import torch
        return np.float64 if v.dtype == torch.float64 else np.int32
    return np.asarray(v).dtype


def _as_int(x, dt):
    if _is_torch(x):
        import torch
        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.uint8: torch.uint8}[dt]
        return x.to(tdt)
    return np.ascontiguousarray(x, dtype=dt)


def _as_val(x, sr):
    if _is_torch(x):
        import torch
        return x.to(torch.float64 if sr == PLUS_TIMES_F64 else torch.int32)
    return np.ascontiguousarray(x, dtype=_vdtype(sr))
