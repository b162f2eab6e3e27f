"""Pins of the oracle's PLE decomposition (Section 4.2) against facts fixed
independently of it: a decomposition worked by hand, P L E = A through the
test-side slice product, the pivot columns and rank of the separately pinned
reduced echelon form, the first-row pivot rule checked by enumerating row
spaces over GF(4), and the layout of the in-place result."""
import os

import numpy as np
import pytest

import oracle
import workloads
from tests import fieldref as fr
from tests import pleref
from tests.test_oracle import _row_space, random_invertible, random_rref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ple_gf4_hand.txt")


def read_hand_example():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    e = int(rows[0][1])
    f = int(rows[1][1])
    a = rows.index(["A"])
    res = rows.index(["result"])
    rk = next(i for i, r in enumerate(rows) if r[0] == "rank")
    A = np.array([[int(v) for v in r] for r in rows[a + 1:res]])
    R = np.array([[int(v) for v in r] for r in rows[res + 1:rk]])
    r = int(rows[rk][1])
    P = [int(v) for v in rows[rk + 1][1:]]
    Q = [int(v) for v in rows[rk + 2][1:]]
    return e, f, A, R, r, P, Q


def test_hand_worked_example():
    e, f, A, R, r, P, Q = read_hand_example()
    out, rk, p, q = oracle.ple(e, f, A.astype(np.uint8))
    assert rk == r
    np.testing.assert_array_equal(out.astype(np.int64), R)
    assert list(p) == P and list(q) == Q
    # the example's own check, through the test-side product
    np.testing.assert_array_equal(pleref.rebuild(e, f, out, rk, p, q, fr.slice_product), A)


def structured_inputs(e, f, rng):
    """Random dense, rank-deficient S R, zero rows on top (swaps from far
    below), a zero matrix, and tall / wide shapes."""
    out = []
    for m, n in ((7, 9), (9, 7), (12, 12), (1, 5), (5, 1)):
        out.append(rng.integers(0, 1 << e, size=(m, n)))
    for m, n, rank in ((10, 14, 6), (14, 10, 4), (12, 12, 11)):
        R, _ = random_rref(e, m, n, rank, rng)
        out.append(fr.slice_product(e, f, random_invertible(e, f, m, rng), R))
    Z = rng.integers(0, 1 << e, size=(11, 8))
    Z[:6] = 0
    Z[6:, :2] = 0
    out.append(Z)
    out.append(np.zeros((4, 6), np.int64))
    return out


@pytest.mark.parametrize("e", [2, 3, 4, 7, 8, 10])
def test_ple_rebuilds_a_and_agrees_with_the_echelon_form(e):
    """P L E = A (test-side product), the layout, and the pivot columns and
    rank equal to those of the reduced echelon form (a unique object, pinned
    on its own)."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(100 + e)
    for A in structured_inputs(e, f, rng):
        A = A.astype(np.uint16)
        out, r, P, Q = oracle.ple(e, f, A)
        assert pleref.layout_ok(out, r, P, Q), A
        np.testing.assert_array_equal(pleref.rebuild(e, f, out, r, P, Q, fr.slice_product), A)
        _, rr, piv = oracle.echelon(e, f, A)
        assert r == rr and list(Q[:r]) == list(piv)


def first_row_rule_ok(e, table, A, r, P, Q):
    """At step t the pivot row is the first row, in the arrangement left by
    the earlier swaps, whose entries in columns 0..Q[t] are outside the span
    of the t pivot rows' entries there (equivalently: its entry in column
    Q[t] is non-zero once those rows are eliminated).  Row spaces are
    enumerated, so small inputs only."""
    cur = np.array(A, np.int64)
    m = cur.shape[0]
    for t in range(r):
        span = _row_space(e, table, cur[:t, :Q[t] + 1]) if t else {tuple([0] * (Q[t] + 1))}
        first = next((i for i in range(t, m) if tuple(int(v) for v in cur[i, :Q[t] + 1]) not in span), None)
        if first != P[t]:
            return False
        cur[[t, first]] = cur[[first, t]]
    # nothing left outside the span of the r pivot rows
    if r < m:
        span = _row_space(e, table, cur[:r]) if r else {tuple([0] * cur.shape[1])}
        if any(tuple(int(v) for v in cur[i]) not in span for i in range(r, m)):
            return False
    return True


def test_first_row_pivot_rule_brute_force_gf4():
    """Every 2 x 2 matrix over GF(4) and a seeded sample of 3 x 3, 3 x 2 and
    2 x 3 ones (with zeros planted so that swaps and empty columns occur)."""
    e, f = 2, 7
    table = fr.log_table_product(e, f)
    cases = [np.array(v).reshape(2, 2) for v in np.ndindex(4, 4, 4, 4)]
    rng = np.random.default_rng(7)
    for shape in ((3, 3), (3, 2), (2, 3)):
        for _ in range(300):
            M = rng.integers(0, 4, size=shape)
            M[rng.random(shape) < 0.4] = 0
            cases.append(M)
    for A in cases:
        out, r, P, Q = oracle.ple(e, f, A.astype(np.uint8))
        assert pleref.layout_ok(out, r, P, Q), A
        assert first_row_rule_ok(e, table, A, r, P, Q), A
        np.testing.assert_array_equal(pleref.rebuild(e, f, out, r, P, Q, fr.slice_product), A)


def test_ple_of_an_invertible_matrix_without_swaps_is_its_lu():
    """A = L0 U0 with L0 lower triangular (non-zero diagonal) and U0 unit
    upper triangular: no row is ever zero in its pivot column, so P is the
    identity, Q = 0..n-1 and the factors are L0 and U0 themselves (the LU
    factorisation with a unit upper factor is unique)."""
    e, f = 5, workloads.FIELD_POLY[5]
    rng = np.random.default_rng(3)
    n = 9
    L0 = np.tril(rng.integers(0, 32, size=(n, n)), -1)
    L0[np.arange(n), np.arange(n)] = rng.integers(1, 32, size=n)
    U0 = np.triu(rng.integers(0, 32, size=(n, n)), 1) + np.eye(n, dtype=np.int64)
    A = fr.slice_product(e, f, L0, U0)
    out, r, P, Q = oracle.ple(e, f, A.astype(np.uint8))
    assert r == n and list(P) == list(range(n)) and list(Q) == list(range(n))
    L, E = pleref.factors(out, r, Q)
    np.testing.assert_array_equal(L, L0)
    np.testing.assert_array_equal(E, U0)


def test_ple_empty_shapes():
    for m, n in ((0, 3), (3, 0), (0, 0)):
        out, r, P, Q = oracle.ple(4, 0x13, np.zeros((m, n), np.uint8))
        assert r == 0 and out.shape == (m, n) and list(P) == list(range(m)) and list(Q) == list(range(n))
