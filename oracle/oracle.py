"""ctypes wrapper of the C oracle (test infrastructure only; see package docstring)."""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dspg_oracle.c")
_LIB = os.path.join(_HERE, "libdspg_oracle.so")
_lock = threading.Lock()
_lib = None

PLUS_TIMES_F64 = 0
MIN_PLUS_I32 = 1


class OracleError(RuntimeError):
    pass


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable flags only; with
    OpenMP for the all-cores timing when the compiler has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:-1] + ["-fopenmp", "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Threads of the oracle's row loops (1: single-threaded, the default)."""
    oracle_lib().orc_set_threads(int(n))


def oracle_lib():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle())
            p, i64, i32, u8p = C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_uint8)
            lib.orc_new.restype = p
            lib.orc_new.argtypes = [i64, i64, i32]
            lib.orc_free.argtypes = [p]
            lib.orc_nnz.restype = i64
            lib.orc_nnz.argtypes = [p]
            lib.orc_from_csr.restype = i32
            lib.orc_from_csr.argtypes = [C.POINTER(C.c_void_p), i64, i64, i32, p, p, p]
            lib.orc_to_csr.argtypes = [p, p, p, p]
            lib.orc_copy.restype = p
            lib.orc_copy.argtypes = [p]
            lib.orc_apply.restype = i32
            lib.orc_apply.argtypes = [p, i64, p, p, p, p]
            lib.orc_presence.argtypes = [p, i64, p, p, p]
            lib.orc_multiply.restype = p
            lib.orc_multiply.argtypes = [p, p, i32]
            lib.orc_multiply_rows.restype = i32
            lib.orc_multiply_rows.argtypes = [p, p, p, i64, i32, p, p, p]
            lib.orc_affected_rows.restype = i64
            lib.orc_affected_rows.argtypes = [p, i64, p, p, p, i64, p, p, p, i64, i32, p]
            lib.orc_bloom.restype = i32
            lib.orc_bloom.argtypes = [p, p, p, p, p]
            lib.orc_replace_rows.restype = i32
            lib.orc_replace_rows.argtypes = [p, p, p, p, i64]
            lib.orc_row_len.restype = C.c_int32
            lib.orc_row_len.argtypes = [p, i64]
            lib.orc_get_row.argtypes = [p, i64, p, p]
            lib.orc_set_threads.argtypes = [i32]
            lib.orc_set_threads.restype = None
            lib.orc_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _vdtype(sr: int):
    return np.float64 if sr == PLUS_TIMES_F64 else np.int32


class OMat:
    """An oracle-side matrix (rows of sorted (col, value) arrays)."""

    def __init__(self, handle: int, sr: int):
        if not handle:
            raise OracleError("oracle allocation failed")
        self._h = C.c_void_p(handle)
        self.sr = sr
        self._lib = oracle_lib()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    @property
    def nrows(self) -> int:
        return self._shape[0]

    @classmethod
    def from_csr(cls, csr) -> "OMat":
        lib = oracle_lib()
        sr = PLUS_TIMES_F64 if csr.val.dtype == np.float64 else MIN_PLUS_I32
        rp = np.ascontiguousarray(csr.rowptr, dtype=np.int64)
        col = np.ascontiguousarray(csr.col, dtype=np.int32)
        val = np.ascontiguousarray(csr.val, dtype=_vdtype(sr))
        out = C.c_void_p()
        st = lib.orc_from_csr(C.byref(out), csr.nrows, csr.ncols, sr, _ptr(rp), _ptr(col), _ptr(val))
        if st != 0:
            raise OracleError(f"orc_from_csr status {st}")
        m = cls(out.value, sr)
        m._shape = (csr.nrows, csr.ncols)
        return m

    def _wrap(self, handle, shape) -> "OMat":
        m = OMat(handle, self.sr)
        m._shape = shape
        return m

    def copy(self) -> "OMat":
        return self._wrap(self._lib.orc_copy(self._h), self._shape)

    @property
    def nnz(self) -> int:
        return int(self._lib.orc_nnz(self._h))

    def to_csr(self):
        from workloads import CSR
        n = self._shape[0]
        nnz = self.nnz
        rp = np.empty(n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, _vdtype(self.sr))
        self._lib.orc_to_csr(self._h, _ptr(rp), _ptr(col), _ptr(val))
        return CSR(self._shape[0], self._shape[1], rp, col, val)

    def apply(self, batch) -> None:
        row = np.ascontiguousarray(batch.row, np.int32)
        col = np.ascontiguousarray(batch.col, np.int32)
        val = np.ascontiguousarray(batch.val, _vdtype(self.sr))
        op = np.ascontiguousarray(batch.op, np.uint8)
        st = self._lib.orc_apply(self._h, row.shape[0], _ptr(row), _ptr(col), _ptr(val), _ptr(op))
        if st != 0:
            raise OracleError(f"orc_apply status {st}")

    def presence(self, batch) -> np.ndarray:
        row = np.ascontiguousarray(batch.row, np.int32)
        col = np.ascontiguousarray(batch.col, np.int32)
        out = np.zeros(row.shape[0], np.uint8)
        self._lib.orc_presence(self._h, row.shape[0], _ptr(row), _ptr(col), _ptr(out))
        return out

    def multiply(self, B: "OMat", absval: bool = False) -> "OMat":
        h = self._lib.orc_multiply(self._h, B._h, int(absval))
        if not h:
            raise OracleError("orc_multiply failed")
        return self._wrap(h, (self._shape[0], B._shape[1]))

    def multiply_rows(self, B: "OMat", rows, absval: bool = False):
        rows = np.ascontiguousarray(rows, np.int32)
        rp = np.empty(rows.shape[0] + 1, np.int64)
        st = self._lib.orc_multiply_rows(self._h, B._h, _ptr(rows), rows.shape[0], int(absval), _ptr(rp), None, None)
        if st != 0:
            raise OracleError(f"orc_multiply_rows status {st}")
        col = np.empty(int(rp[-1]), np.int32)
        val = np.empty(int(rp[-1]), _vdtype(self.sr))
        st = self._lib.orc_multiply_rows(self._h, B._h, _ptr(rows), rows.shape[0], int(absval), _ptr(rp), _ptr(col), _ptr(val))
        if st != 0:
            raise OracleError(f"orc_multiply_rows status {st}")
        return rp, col, val

    def bloom(self, B: "OMat"):
        """The Bloom filter F of self * B (Section 5.2, l = 64), by its
        definition: (rowptr, col, words) with words uint64."""
        n = self._shape[0]
        rp = np.empty(n + 1, np.int64)
        st = self._lib.orc_bloom(self._h, B._h, _ptr(rp), None, None)
        if st != 0:
            raise OracleError(f"orc_bloom status {st}")
        col = np.empty(int(rp[-1]), np.int32)
        words = np.empty(int(rp[-1]), np.uint64)
        st = self._lib.orc_bloom(self._h, B._h, _ptr(rp), _ptr(col), _ptr(words))
        if st != 0:
            raise OracleError(f"orc_bloom status {st}")
        return rp, col, words

    def replace_rows(self, A: "OMat", B: "OMat", rows) -> None:
        rows = np.ascontiguousarray(rows, np.int32)
        st = self._lib.orc_replace_rows(self._h, A._h, B._h, _ptr(rows), rows.shape[0])
        if st != 0:
            raise OracleError(f"orc_replace_rows status {st}")

    def row(self, i: int):
        n = int(self._lib.orc_row_len(self._h, i))
        col = np.empty(n, np.int32)
        val = np.empty(n, _vdtype(self.sr))
        self._lib.orc_get_row(self._h, i, _ptr(col), _ptr(val))
        return col, val


def affected_rows(a_new: OMat, batch_a, pre_a, post_a, batch_b=None, pre_b=None, post_b=None,
                  b_nrows: int | None = None, b_is_a: bool = True) -> np.ndarray:
    """R = rows(A*) u {i : A'(i,k) != 0, k in rows(B*)} (see dspg_oracle.c)."""
    lib = oracle_lib()
    arow = np.ascontiguousarray(batch_a.row, np.int32)
    apre = np.ascontiguousarray(pre_a, np.uint8)
    apost = np.ascontiguousarray(post_a, np.uint8)
    if batch_b is None:
        brow = np.zeros(0, np.int32)
        bpre = bpost = np.zeros(0, np.uint8)
    else:
        brow = np.ascontiguousarray(batch_b.row, np.int32)
        bpre = np.ascontiguousarray(pre_b, np.uint8)
        bpost = np.ascontiguousarray(post_b, np.uint8)
    if b_nrows is None:
        b_nrows = a_new._shape[1]
    out = np.empty(max(a_new._shape[0], 1), np.int32)
    cnt = lib.orc_affected_rows(a_new._h, arow.shape[0], _ptr(arow), _ptr(apre), _ptr(apost),
                                brow.shape[0], _ptr(brow), _ptr(bpre), _ptr(bpost),
                                b_nrows, int(b_is_a), _ptr(out))
    if cnt < 0:
        raise OracleError("orc_affected_rows failed")
    return out[:cnt].copy()


def row_dynamic(A: OMat, C: OMat, batch_a, B: OMat | None = None, batch_b=None) -> np.ndarray:
    """The oracle's row-dynamic route for one batch: apply the batch(es) in
    array order (Section 4.1), find the affected rows R of C (Section 5,
    general updates) and recompute exactly those rows of C in place.
    ``B is None`` means B is A (C = A A, one batch for both). Returns R."""
    if B is None:
        pre = A.presence(batch_a)
        A.apply(batch_a)
        post = A.presence(batch_a)
        R = affected_rows(A, batch_a, pre, post, b_nrows=A._shape[0], b_is_a=True)
        C.replace_rows(A, A, R)
        return R
    if batch_b is None:
        from workloads import Batch
        z = np.zeros(0, np.int32)
        batch_b = Batch(z, z, np.zeros(0, np.float64 if B.sr == PLUS_TIMES_F64 else np.int32), np.zeros(0, np.uint8))
    pre_a, pre_b = A.presence(batch_a), B.presence(batch_b)
    # validate both before mutating either: apply to copies first
    A2, B2 = A.copy(), B.copy()
    A2.apply(batch_a)
    B2.apply(batch_b)
    A.apply(batch_a)
    B.apply(batch_b)
    post_a, post_b = A.presence(batch_a), B.presence(batch_b)
    R = affected_rows(A, batch_a, pre_a, post_a, batch_b, pre_b, post_b,
                      b_nrows=B._shape[0], b_is_a=False)
    C.replace_rows(A, B, R)
    return R
