"""CPU oracle for GF(2^e) matrix multiplication and triangular solving (test
infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C, OpenMP over rows): the field
product of Section 2 (carry-less multiply, then reduction modulo f) and its
inverse, the cubic matrix product of Algorithm 1, the triangular solve of
Algorithm 5 (Section 4.3), the reduced row echelon form of Algorithm 4
(Section 4.1) and the PLE decomposition of Section 4.2, the packed representation of Section 3.1 and the slicing /
clinging conversions of Section 3.2 and Figure 1.  This module only compiles that file with gcc and
marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_default = None


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp a C source file into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, src], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(SOURCE):
        compile_source(SOURCE, _LIB_PATH)
    return _LIB_PATH


def elem_dtype(e: int):
    """Element storage: uint8 for e <= 8, uint16 for e in {9, 10}."""
    return np.uint8 if e <= 8 else np.uint16


def _as_u16(x, e: int, name: str) -> np.ndarray:
    x = np.asarray(x)
    if x.size and int(x.max()) >= (1 << e):
        raise ValueError(f"{name} has entries >= 2^{e}; the oracle takes field elements only")
    return np.ascontiguousarray(x, dtype=np.uint16)


class OracleLib:
    """numpy front end of one compiled copy of oracle.c."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        u32, i32, i64, vp = ctypes.c_uint32, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.oracle_gf_mul.restype = u32
        L.oracle_gf_mul.argtypes = [i32, u32, u32, u32]
        L.oracle_gf_mul_table.restype = None
        L.oracle_gf_mul_table.argtypes = [i32, u32, vp]
        L.oracle_set_threads.restype = None
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_get_threads.restype = i32
        L.oracle_get_threads.argtypes = []
        L.oracle_matmul.restype = None
        L.oracle_matmul.argtypes = [i32, u32, i64, i64, i64, vp, vp, vp, i32]
        L.oracle_slice.restype = None
        L.oracle_slice.argtypes = [i32, i64, i64, vp, vp, i64]
        L.oracle_cling.restype = None
        L.oracle_cling.argtypes = [i32, i64, i64, vp, i64, vp]
        L.oracle_packed_width.restype = i32
        L.oracle_packed_width.argtypes = [i32]
        L.oracle_pack.restype = None
        L.oracle_pack.argtypes = [i32, i64, i64, vp, vp, i64]
        L.oracle_unpack.restype = None
        L.oracle_unpack.argtypes = [i32, i64, i64, vp, i64, vp]
        L.oracle_gf_inv.restype = u32
        L.oracle_gf_inv.argtypes = [i32, u32, u32]
        L.oracle_trsm_upper_left.restype = i32
        L.oracle_trsm_upper_left.argtypes = [i32, u32, i64, i64, vp, vp]
        L.oracle_trsm_lower_left.restype = i32
        L.oracle_trsm_lower_left.argtypes = [i32, u32, i64, i64, vp, vp]
        L.oracle_echelon.restype = i64
        L.oracle_echelon.argtypes = [i32, u32, i64, i64, vp, vp]
        L.oracle_ple.restype = i64
        L.oracle_ple.argtypes = [i32, u32, i64, i64, vp, vp, vp]
        self.L = L
        self.path = path

    def set_threads(self, n: int) -> None:
        self.L.oracle_set_threads(int(n))

    def get_threads(self) -> int:
        return int(self.L.oracle_get_threads())

    def gf_mul(self, e: int, f: int, a: int, b: int) -> int:
        """Section 2: a * b in F2[x]/<f>."""
        return int(self.L.oracle_gf_mul(e, f, a, b))

    def mul_table(self, e: int, f: int) -> np.ndarray:
        """2^e x 2^e table of oracle_gf_mul."""
        q = 1 << e
        out = np.empty((q, q), dtype=np.uint16)
        self.L.oracle_gf_mul_table(e, f, out.ctypes.data)
        return out

    def _matmul(self, e, f, A, B, C, accumulate):
        A16 = _as_u16(A, e, "A")
        B16 = _as_u16(B, e, "B")
        if A16.ndim != 2 or B16.ndim != 2 or A16.shape[1] != B16.shape[0]:
            raise ValueError(f"shape mismatch {A16.shape} x {B16.shape}")
        m, k = A16.shape
        n = B16.shape[1]
        if C is None:
            C16 = np.zeros((m, n), dtype=np.uint16)
        else:
            C16 = _as_u16(C, e, "C").copy()
            if C16.shape != (m, n):
                raise ValueError("C has the wrong shape")
        if m and n:
            self.L.oracle_matmul(e, f, m, n, k, A16.ctypes.data, B16.ctypes.data, C16.ctypes.data,
                                 1 if accumulate else 0)
        return C16.astype(elem_dtype(e))

    def matmul(self, e: int, f: int, A, B) -> np.ndarray:
        """Algorithm 1: C = A * B over GF(2^e)."""
        return self._matmul(e, f, A, B, None, False)

    def addmul(self, e: int, f: int, A, B, C) -> np.ndarray:
        """C + A * B over GF(2^e) (addition is XOR); returns a new array."""
        return self._matmul(e, f, A, B, C, True)

    def slice_(self, e: int, elems, ld_words: int | None = None) -> np.ndarray:
        """Section 3.2: slicing.  Returns uint64 planes of shape (e, rows, ld_words)."""
        X = _as_u16(elems, e, "elems")
        rows, cols = X.shape
        if ld_words is None:
            ld_words = (cols + 63) // 64
        out = np.empty((e, rows, ld_words), dtype=np.uint64)
        self.L.oracle_slice(e, rows, cols, X.ctypes.data, out.ctypes.data, ld_words)
        return out

    def cling(self, e: int, slices, cols: int) -> np.ndarray:
        """Section 3.2: clinging (inverse of slicing)."""
        S = np.ascontiguousarray(slices, dtype=np.uint64)
        _, rows, ld_words = S.shape
        out = np.empty((rows, cols), dtype=np.uint16)
        self.L.oracle_cling(e, rows, cols, S.ctypes.data, ld_words, out.ctypes.data)
        return out.astype(elem_dtype(e))

    def packed_width(self, e: int) -> int:
        """Section 3.1: bits per element in the packed representation."""
        return int(self.L.oracle_packed_width(e))

    def to_packed(self, e: int, elems, ld_words: int | None = None) -> np.ndarray:
        """Section 3.1: packed representation, uint64 array (rows, ld_words)."""
        X = _as_u16(elems, e, "elems")
        rows, cols = X.shape
        per = 64 // self.packed_width(e)
        if ld_words is None:
            ld_words = (cols + per - 1) // per
        out = np.empty((rows, ld_words), dtype=np.uint64)
        self.L.oracle_pack(e, rows, cols, X.ctypes.data, out.ctypes.data, ld_words)
        return out

    def from_packed(self, e: int, words, cols: int) -> np.ndarray:
        """Section 3.1: elements of a packed matrix (padding ignored)."""
        Wd = np.ascontiguousarray(words, dtype=np.uint64)
        rows, ld_words = Wd.shape
        out = np.empty((rows, cols), dtype=np.uint16)
        self.L.oracle_unpack(e, rows, cols, Wd.ctypes.data, ld_words, out.ctypes.data)
        return out.astype(elem_dtype(e))

    def gf_inv(self, e: int, f: int, a: int) -> int:
        """a^(2^e - 2), the inverse of a != 0 (0 for a = 0)."""
        return int(self.L.oracle_gf_inv(e, f, a))

    def trsm(self, e: int, f: int, T, B, upper: bool = True) -> np.ndarray:
        """Algorithm 5: T^{-1} * B for T square triangular (upper or lower);
        returns a new array.  Raises ZeroDivisionError on a zero diagonal."""
        T16 = _as_u16(T, e, "T")
        B16 = _as_u16(B, e, "B").copy()
        if T16.ndim != 2 or T16.shape[0] != T16.shape[1] or B16.ndim != 2 or B16.shape[0] != T16.shape[0]:
            raise ValueError(f"shape mismatch: T {T16.shape}, B {B16.shape}")
        m, n = B16.shape
        fn = self.L.oracle_trsm_upper_left if upper else self.L.oracle_trsm_lower_left
        if m and fn(e, f, m, n, T16.ctypes.data, B16.ctypes.data) != 0:
            raise ZeroDivisionError("zero on the diagonal")
        return B16.astype(elem_dtype(e))

    def echelon(self, e: int, f: int, A):
        """Algorithm 4: (reduced row echelon form of A as a new array, rank,
        pivot columns of the first rank rows)."""
        A16 = _as_u16(A, e, "A").copy()
        if A16.ndim != 2:
            raise ValueError("A must be 2-D")
        m, n = A16.shape
        piv = np.zeros(max(1, min(m, n)), dtype=np.int64)
        r = int(self.L.oracle_echelon(e, f, m, n, A16.ctypes.data, piv.ctypes.data)) if m and n else 0
        return A16.astype(elem_dtype(e)), r, piv[:r].copy()

    def ple(self, e: int, f: int, A):
        """Section 4.2: (A overwritten with its PLE decomposition, as a new
        array; rank r; P (m swap partners); Q (n entries, the pivot columns
        first)).  Layout of the result: see oracle_ple in oracle.c."""
        A16 = _as_u16(A, e, "A").copy()
        if A16.ndim != 2:
            raise ValueError("A must be 2-D")
        m, n = A16.shape
        P = np.arange(max(1, m), dtype=np.int64)
        Q = np.arange(max(1, n), dtype=np.int64)
        r = int(self.L.oracle_ple(e, f, m, n, A16.ctypes.data, P.ctypes.data, Q.ctypes.data)) if m and n else 0
        return A16.astype(elem_dtype(e)), r, P[:m].copy(), Q[:n].copy()

    def freivalds(self, e: int, f: int, A, B, C, trials: int = 64, seed: int = 0) -> bool:
        """Randomised check that C == A * B: with X an n x trials matrix of
        uniform field elements, compare A(BX) with CX.  A wrong C passes one
        column with probability at most 2^-e."""
        rng = np.random.default_rng(seed)
        n = np.asarray(B).shape[1]
        X = rng.integers(0, 1 << e, size=(n, trials), dtype=np.uint16)
        lhs = self.matmul(e, f, A, self.matmul(e, f, B, X))
        rhs = self.matmul(e, f, C, X)
        return bool(np.array_equal(lhs, rhs))


def default() -> OracleLib:
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
    return _default


def set_threads(n: int) -> None:
    default().set_threads(n)


def get_threads() -> int:
    return default().get_threads()


def gf_mul(e, f, a, b):
    return default().gf_mul(e, f, a, b)


def mul_table(e, f):
    return default().mul_table(e, f)


def matmul(e, f, A, B):
    return default().matmul(e, f, A, B)


def addmul(e, f, A, B, C):
    return default().addmul(e, f, A, B, C)


def slice_(e, elems, ld_words=None):
    return default().slice_(e, elems, ld_words)


def cling(e, slices, cols):
    return default().cling(e, slices, cols)


def freivalds(e, f, A, B, C, trials=64, seed=0):
    return default().freivalds(e, f, A, B, C, trials, seed)


def gf_inv(e, f, a):
    return default().gf_inv(e, f, a)


def trsm(e, f, T, B, upper=True):
    return default().trsm(e, f, T, B, upper)


def echelon(e, f, A):
    return default().echelon(e, f, A)


def ple(e, f, A):
    return default().ple(e, f, A)


def packed_width(e):
    return default().packed_width(e)


def to_packed(e, elems, ld_words=None):
    return default().to_packed(e, elems, ld_words)


def from_packed(e, words, cols):
    return default().from_packed(e, words, cols)
