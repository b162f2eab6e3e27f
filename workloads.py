"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds data only: field polynomials, workload shapes and seeded
random field elements.  It contains none of the method's arithmetic, so both
the CPU oracle and the CUDA path can take their inputs from it.

Input recipe (the paper measures on random dense matrices, Section 4.1 and
Table 3; no dataset is involved): numpy ``default_rng(seed)``, entries drawn
i.i.d. uniform in [0, 2^e); for workload i the seed is 1000 + i and the
matrices are drawn in the order A, B, C; for batched instance j the seed is
40000 + j and the draw order is e, (m, n, k), A, B.  Triangular systems
(Section 4.3): the triangle of T (upper or lower) uniform, its diagonal
uniform in [1, 2^e) so that T is invertible, the other triangle zero, then B.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Field polynomial f per degree e, as an integer bitmask including x^e.
#   x^2+x+1, x^3+x+1, x^4+x+1, x^5+x^2+1, x^6+x+1, x^7+x+1,
#   x^8+x^4+x^3+x^2+1, x^9+x^4+1, x^10+x^3+1
FIELD_POLY = {2: 0x7, 3: 0xB, 4: 0x13, 5: 0x25, 6: 0x43, 7: 0x83, 8: 0x11D, 9: 0x211, 10: 0x409}


def elem_dtype(e: int):
    """uint8 storage for e <= 8, little-endian uint16 for e in {9, 10}."""
    return np.uint8 if e <= 8 else np.uint16


def elements(rng: np.random.Generator, e: int, shape) -> np.ndarray:
    """I.i.d. uniform field elements of GF(2^e) in their integer encoding."""
    return rng.integers(0, 1 << e, size=shape, dtype=np.uint16).astype(elem_dtype(e))


@dataclass(frozen=True)
class Workload:
    name: str
    op: str          # "mul" (C = A B) or "addmul" (C += A B)
    e: int
    m: int
    k: int
    n: int
    seed: int

    @property
    def f(self) -> int:
        return FIELD_POLY[self.e]

    @property
    def field_ops(self) -> float:
        """Nominal GF(2^e) field operations 2 m n k."""
        return 2.0 * self.m * self.n * self.k

    def inputs(self, rows: slice | None = None):
        """(A, B, C) for this workload; C is None for "mul".  ``rows`` selects a
        row panel of A and C after drawing the full matrices (same values)."""
        rng = np.random.default_rng(self.seed)
        A = elements(rng, self.e, (self.m, self.k))
        B = elements(rng, self.e, (self.k, self.n))
        C = elements(rng, self.e, (self.m, self.n)) if self.op == "addmul" else None
        if rows is not None:
            A = A[rows]
            C = None if C is None else C[rows]
        return A, B, C


WORKLOADS = {
    1: Workload("gf4_512_mul", "mul", 2, 512, 512, 512, 1001),
    2: Workload("gf16_4096_mul", "mul", 4, 4096, 4096, 4096, 1002),
    3: Workload("gf256_8192_addmul", "addmul", 8, 8192, 8192, 8192, 1003),
    5: Workload("gf1024_16384x4096x16384_mul", "mul", 10, 16384, 4096, 16384, 1005),
    # the rank-64 update of a reduced echelon form's panel step (Section 6),
    # C += A B with A 8192 x 64 and B 64 x 8192 over GF(2^8)
    "rank64": Workload("gf256_8192x64x8192_addmul", "addmul", 8, 8192, 64, 8192, 1006),
}

BATCHED_COUNT = 4096
BATCHED_E = (2, 8)                 # e uniform in {2..8}
BATCHED_DIM_STEP, BATCHED_DIM_MAX = 32, 1024   # m, n, k uniform in {32, 64, ..., 1024}


def batched_instance(j: int, dims_only: bool = False):
    """Instance j of the batched workload: (e, f, m, n, k, A, B)."""
    rng = np.random.default_rng(40000 + j)
    e = int(rng.integers(BATCHED_E[0], BATCHED_E[1] + 1))
    m, n, k = (int(v) * BATCHED_DIM_STEP for v in rng.integers(1, BATCHED_DIM_MAX // BATCHED_DIM_STEP + 1, size=3))
    if dims_only:
        return e, FIELD_POLY[e], m, n, k, None, None
    A = elements(rng, e, (m, k))
    B = elements(rng, e, (k, n))
    return e, FIELD_POLY[e], m, n, k, A, B


def random_problem(e: int, m: int, n: int, k: int, seed: int, with_c: bool = False):
    """Seeded (A, B, C) of the given shape; C is None unless with_c."""
    rng = np.random.default_rng(seed)
    A = elements(rng, e, (m, k))
    B = elements(rng, e, (k, n))
    C = elements(rng, e, (m, n)) if with_c else None
    return A, B, C


# Triangular solves B <- T^{-1} B, T m x m upper triangular, B m x n: (e, m, n, seed).
TRSM_WORKLOADS = {
    "trsm_gf16_4096": (4, 4096, 4096, 1100),
    "trsm_gf256_8192": (8, 8192, 8192, 1101),
}


def triangular_system(e: int, m: int, n: int, seed: int, upper: bool = True):
    """Seeded (T, B): T m x m triangular with a non-zero diagonal, B m x n."""
    rng = np.random.default_rng(seed)
    T = elements(rng, e, (m, m))
    T = np.triu(T) if upper else np.tril(T)
    T[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m).astype(T.dtype)
    B = elements(rng, e, (m, n))
    return T, B


# Reduced row echelon forms of random dense matrices (Section 4.1; the
# introduction's 4000 x 4000 over GF(4) and Table 2's 1000 x 1000 sizes):
# (e, m, n, seed).
ECHELON_WORKLOADS = {
    "rref_gf4_4000": (2, 4000, 4000, 1200),
    "rref_gf256_1000": (8, 1000, 1000, 1201),
    "rref_gf16_8192": (4, 8192, 8192, 1202),
}


# PLE decompositions (Section 4.2) of random dense matrices: (e, m, n, seed)
PLE_WORKLOADS = {
    "ple_gf4_4000": (2, 4000, 4000, 1300),
    "ple_gf256_1000": (8, 1000, 1000, 1301),
    "ple_gf16_8192": (4, 8192, 8192, 1302),
}


def echelon_matrix(e: int, m: int, n: int, seed: int):
    """Seeded m x n matrix, entries uniform in [0, 2^e)."""
    return elements(np.random.default_rng(seed), e, (m, n))
