"""Independent constructions used to pin the oracle (and the CUDA path's host logic).

Nothing here is shared with ``oracle/`` or with the product: these are the
textbook constructions the oracle is checked against, written separately.

* ``xtime``: multiplication by x modulo f, i.e. shift left and subtract f when
  the degree reaches e (the step of Algorithm 2 that computes alpha^k * B).
* ``exp_log_tables``: powers of alpha = x built by repeated ``xtime`` and
  their inverse (discrete logarithms), the Zech-logarithm style representation
  the Appendix describes for Magma.
* ``poly_mod`` / ``is_irreducible``: long division over F2[x] and trial
  division by every polynomial of degree <= e/2.
"""
from __future__ import annotations

import numpy as np


def xtime(e: int, f: int, a: int) -> int:
    a <<= 1
    if a >> e & 1:
        a ^= f
    return a


def poly_deg(p: int) -> int:
    return p.bit_length() - 1


def poly_mod(a: int, b: int) -> int:
    """Remainder of a modulo b in F2[x] (integers as coefficient bitmasks)."""
    db = poly_deg(b)
    while a and poly_deg(a) >= db:
        a ^= b << (poly_deg(a) - db)
    return a


def is_irreducible(f: int) -> bool:
    e = poly_deg(f)
    if e < 1:
        return False
    for d in range(2, 1 << (e // 2 + 1)):
        if poly_deg(d) >= 1 and poly_deg(d) <= e // 2 and poly_mod(f, d) == 0:
            return False
    return True


def order_of_x(e: int, f: int) -> int:
    """Multiplicative order of x modulo f (f irreducible of degree e)."""
    a, n = xtime(e, f, 1), 1
    while a != 1:
        a = xtime(e, f, a)
        n += 1
        if n > (1 << e):
            raise ValueError("x is not invertible")
    return n


def exp_log_tables(e: int, f: int):
    """exp[i] = alpha^i for i < 2^e - 1, log[exp[i]] = i (f must be primitive)."""
    q = (1 << e) - 1
    exp = np.zeros(q, dtype=np.int64)
    log = np.full(q + 1, -1, dtype=np.int64)
    a = 1
    for i in range(q):
        exp[i] = a
        log[a] = i
        a = xtime(e, f, a)
    if a != 1 or (log[1:] < 0).any():
        raise ValueError("f is not primitive")
    return exp, log


def log_table_product(e: int, f: int) -> np.ndarray:
    """2^e x 2^e multiplication table from discrete logarithms."""
    exp, log = exp_log_tables(e, f)
    q = (1 << e) - 1
    a = np.arange(q + 1)
    la, lb = np.meshgrid(log[a], log[a], indexing="ij")
    t = exp[(la + lb) % q]
    t[0, :] = 0
    t[:, 0] = 0
    return t


def x_power_mod(e: int, f: int, d: int) -> int:
    """x^d mod f as a coefficient bitmask."""
    a = 1
    for _ in range(d):
        a = xtime(e, f, a)
    return a


def bits(M: np.ndarray, i: int) -> np.ndarray:
    """Coefficient i of every entry, as an int64 0/1 matrix."""
    return (M.astype(np.int64) >> i) & 1


def gf2_matmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """GF(2) product of 0/1 matrices via the integer matmul of numpy."""
    return (X.astype(np.int64) @ Y.astype(np.int64)) & 1


def slice_product(e: int, f: int, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A * B over GF(2^e) by the reduction to GF(2) products of Section 5:
    C~_d = sum_{i+j=d} A_i B_j (schoolbook polynomial product of the slice
    polynomials), then C = sum_d C~_d * (x^d mod f)."""
    m, n = A.shape[0], B.shape[1]
    C = np.zeros((m, n), dtype=np.int64)
    for i in range(e):
        Ai = bits(A, i)
        for j in range(e):
            P = gf2_matmul(Ai, bits(B, j))
            C ^= P * x_power_mod(e, f, i + j)
    return C
