"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something computed independently of it:
Figure 1, the GF(4) example of Section 5, textbook field products, logarithm
tables built from powers of alpha, brute force and matrix identities.  The
mutation tests at the end plant plausible mistakes into a copy of the
oracle's C source and check that the pins catch each one.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import workloads
from tests import fieldref as fr
from tests import pleref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fig1_sections():
    with open(os.path.join(GOLDEN, "fig1_gf8.txt")) as fh:
        lines = [l.split("#")[0].strip() for l in fh]
    lines = [l for l in lines if l]
    e = int(lines[0].split()[1])
    sections = {}
    i = 1
    while i < len(lines):
        sections[lines[i]] = [lines[i + 1].split(), lines[i + 2].split()]
        i += 3
    return e, sections


def _read_fig1():
    e, sec = _fig1_sections()
    elems = np.array([[int(v) for v in row] for row in sec["elements"]])
    slices = [np.array([[int(v) for v in row] for row in sec[f"slice {i}"]]) for i in range(e)]
    return e, elems, slices


def _read_fig1_packed():
    """Figure 1's packed row as a list of rows of bit-strings (highest bit first)."""
    _, sec = _fig1_sections()
    return sec["packed"]


# ---------------------------------------------------------------- Figure 1


def test_fig1_slicing_matches_figure():
    e, elems, slices = _read_fig1()
    planes = oracle.slice_(e, elems)
    assert planes.shape == (3, 2, 1)
    for i in range(e):
        got = np.array([[(int(planes[i, r, 0]) >> c) & 1 for c in range(2)] for r in range(2)])
        np.testing.assert_array_equal(got, slices[i], err_msg=f"slice {i}")
        # only the two columns may be set: padding bits are zero
        assert all(int(planes[i, r, 0]) >> 2 == 0 for r in range(2))


def test_fig1_clinging_inverts_slicing():
    e, elems, _ = _read_fig1()
    np.testing.assert_array_equal(oracle.cling(e, oracle.slice_(e, elems), 2), elems)


# ------------------------------------------------ packed representation


def test_fig1_packed_matches_figure():
    """Figure 1, second row: F_8 entries in 4-bit fields, the top (padding)
    bit zero.  The figure does not fix the order of the fields inside a word;
    the lowest field first (the slices' column order) is the reading used."""
    e, elems, _ = _read_fig1()
    fields = _read_fig1_packed()
    assert oracle.packed_width(e) == len(fields[0][0]) == 4
    W = oracle.to_packed(e, elems)
    assert W.shape == (2, 1)
    for r in range(2):
        want = sum(int(fields[r][c], 2) << (4 * c) for c in range(2))
        assert int(W[r, 0]) == want
    np.testing.assert_array_equal(oracle.from_packed(e, W, 2), elems)


def test_packed_widths():
    """Section 3.1: the next length dividing 64; F_32 entries take 8 bits
    (three zero coefficients on top)."""
    assert oracle.packed_width(5) == 8
    for e in range(2, 11):
        w = oracle.packed_width(e)
        assert 64 % w == 0 and w >= e and (w == 2 or w // 2 < e)


@pytest.mark.parametrize("e", list(range(2, 11)))
def test_packed_bits_and_roundtrip(e):
    """Every field of a packed word, read back bit by bit, is the element;
    padding fields and bits are zero; unpacking ignores padding."""
    rng = np.random.default_rng(70 + e)
    cols = 37
    X = workloads.elements(rng, e, (5, cols))
    w = oracle.packed_width(e)
    per = 64 // w
    W = oracle.to_packed(e, X, ld_words=(cols + per - 1) // per + 1)
    for r in range(5):
        for c in range(W.shape[1] * per):
            field = (int(W[r, c // per]) >> (w * (c % per))) & ((1 << w) - 1)
            assert field == (int(X[r, c]) if c < cols else 0)
    dirty = W.copy()
    dirty[:, -1] = np.uint64(0xFFFFFFFFFFFFFFFF)  # padding word
    np.testing.assert_array_equal(oracle.from_packed(e, dirty, cols), X)


def test_slice_cling_roundtrip_random_and_padding():
    rng = np.random.default_rng(5)
    for e in (2, 5, 8, 10):
        X = workloads.elements(rng, e, (7, 131))
        S = oracle.slice_(e, X, ld_words=4)   # wider than the 3 words needed
        assert S.shape == (e, 7, 4)
        assert (S[:, :, 3] == 0).all()
        assert (S[:, :, 2] >> np.uint64(131 - 128) == 0).all()
        # bit (c mod 64) of word c // 64 is coefficient i of column c
        for (r, c) in [(0, 0), (3, 63), (6, 64), (2, 130)]:
            for i in range(e):
                assert (int(S[i, r, c // 64]) >> (c % 64)) & 1 == (int(X[r, c]) >> i) & 1
        np.testing.assert_array_equal(oracle.cling(e, S, 131), X)


# ---------------------------------------------------------------- the field


@pytest.mark.parametrize("e", sorted(workloads.FIELD_POLY))
def test_field_polynomials_irreducible_and_primitive(e):
    f = workloads.FIELD_POLY[e]
    assert fr.poly_deg(f) == e
    assert fr.is_irreducible(f)
    assert fr.order_of_x(e, f) == (1 << e) - 1


def test_irreducibility_check_rejects_reducible():
    # x^4 + 1 = (x + 1)^4, x^2 + 1 = (x + 1)^2, x^8+x^4+x^3+x^2 has the root 0,
    # x^4 + x^2 + 1 = (x^2 + x + 1)^2
    for f in (0x11, 0x5, 0x11C, 0x15):
        assert not fr.is_irreducible(f)
    assert fr.is_irreducible(0x1F)  # x^4+x^3+x^2+x+1: irreducible, x has order 5
    assert fr.order_of_x(4, 0x1F) == 5


def test_aes_worked_products():
    with open(os.path.join(GOLDEN, "aes_gf256.txt")) as fh:
        rows = [l.split("#")[0].split() for l in fh]
    rows = [r for r in rows if r]
    e = int(rows[0][1])
    f = int(rows[1][1], 16)
    assert fr.is_irreducible(f) and fr.order_of_x(e, f) == 51
    for a, b, c in rows[2:]:
        assert oracle.gf_mul(e, f, int(a, 16), int(b, 16)) == int(c, 16)


@pytest.mark.parametrize("e", sorted(workloads.FIELD_POLY))
def test_product_equals_log_table_exhaustive(e):
    """All 2^(2e) products equal alpha^(log a + log b)."""
    f = workloads.FIELD_POLY[e]
    np.testing.assert_array_equal(oracle.mul_table(e, f).astype(np.int64), fr.log_table_product(e, f))


@pytest.mark.parametrize("e", [2, 3, 4])
def test_field_axioms_brute_force(e):
    f = workloads.FIELD_POLY[e]
    T = oracle.mul_table(e, f).astype(np.int64)
    q = 1 << e
    a = np.arange(q)
    assert (T == T.T).all()                       # commutative
    assert (T[1] == a).all() and (T[:, 0] == 0).all()   # identity, zero
    # associative: (ab)c == a(bc) for all triples
    A3, B3, C3 = np.meshgrid(a, a, a, indexing="ij")
    assert (T[T[A3, B3], C3] == T[A3, T[B3, C3]]).all()
    # distributive: a(b + c) == ab + ac
    assert (T[A3, B3 ^ C3] == (T[A3, B3] ^ T[A3, C3])).all()
    # every nonzero element has exactly one inverse
    for x in range(1, q):
        assert (T[x] == 1).sum() == 1
    assert (T[0] == 1).sum() == 0


def test_product_with_merely_irreducible_polynomial():
    """0x11B is irreducible with x of order 51: the product still follows the
    field axioms (checked against the xtime construction of b * x^i)."""
    e, f = 8, 0x11B
    T = oracle.mul_table(e, f).astype(np.int64)
    # a * x^i via repeated xtime, for all a and i < 8, and linearity in b
    for a in range(256):
        xi = a
        for i in range(8):
            assert T[a, 1 << i] == xi
            xi = fr.xtime(e, f, xi)
    b = np.arange(256)
    for a in (0x57, 0x83, 0xFF):
        expect = np.zeros(256, dtype=np.int64)
        for i in range(8):
            expect ^= ((b >> i) & 1) * T[a, 1 << i]
        assert (T[a] == expect).all()


# ---------------------------------------------------------------- matrices


def test_section5_gf4_example():
    """Section 5: over GF(4) with f = x^2+x+1, C = (A1B1 + A1B0 + A0B1) x + A0B0 + A1B1,
    and the 3-product form ((A1+A0)(B1+B0) + A0B0) x + A0B0 + A1B1."""
    e, f = 2, 0x7
    A, B, _ = workloads.random_problem(e, 23, 19, 37, seed=11)
    C = oracle.matmul(e, f, A, B).astype(np.int64)
    A0, A1, B0, B1 = fr.bits(A, 0), fr.bits(A, 1), fr.bits(B, 0), fr.bits(B, 1)
    P = fr.gf2_matmul
    C1 = P(A1, B1) ^ P(A1, B0) ^ P(A0, B1)
    C0 = P(A0, B0) ^ P(A1, B1)
    np.testing.assert_array_equal(C, C1 * 2 + C0)
    K1 = P(A1 ^ A0, B1 ^ B0) ^ P(A0, B0)
    np.testing.assert_array_equal(C, K1 * 2 + C0)


@pytest.mark.parametrize("e", sorted(workloads.FIELD_POLY))
def test_slice_decomposition_equals_oracle(e):
    """Special case reducing to a library routine: the GF(2) slice products via
    numpy integer matmul, recombined as a polynomial product and reduced mod f."""
    f = workloads.FIELD_POLY[e]
    A, B, _ = workloads.random_problem(e, 37, 41, 53, seed=100 + e)
    np.testing.assert_array_equal(oracle.matmul(e, f, A, B).astype(np.int64), fr.slice_product(e, f, A, B))


def test_brute_force_all_2x2x2_over_gf4():
    """Every pair of 2x2 matrices over GF(4), against the logarithm table."""
    e, f = 2, 0x7
    T = fr.log_table_product(e, f)
    mats = np.array(list(itertools.product(range(4), repeat=4)), dtype=np.int64).reshape(-1, 2, 2)
    # stack all A as rows of one tall matrix and all B side by side, one oracle call
    bigA = mats.reshape(-1, 2)                    # (256*2) x 2
    bigB = mats.transpose(1, 0, 2).reshape(2, -1)  # 2 x (256*2)
    got = oracle.matmul(e, f, bigA, bigB).astype(np.int64).reshape(256, 2, 256, 2).transpose(0, 2, 1, 3)
    expect = np.zeros((256, 256, 2, 2), dtype=np.int64)
    for t in range(2):
        expect ^= T[mats[:, None, :, t, None], mats[None, :, None, t, :]]
    np.testing.assert_array_equal(got, expect)


def test_one_by_one_products_are_the_table():
    for e in (3, 9):
        f = workloads.FIELD_POLY[e]
        T = fr.log_table_product(e, f)
        rng = np.random.default_rng(e)
        for a, b in rng.integers(0, 1 << e, size=(50, 2)):
            assert int(oracle.matmul(e, f, [[a]], [[b]])[0, 0]) == T[a, b]


@pytest.mark.parametrize("e", [2, 3, 8, 10])
def test_matrix_invariants(e):
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(7 * e)
    A = workloads.elements(rng, e, (9, 12))
    B = workloads.elements(rng, e, (12, 10))
    B2 = workloads.elements(rng, e, (12, 10))
    D = workloads.elements(rng, e, (10, 8))
    C0 = workloads.elements(rng, e, (9, 10))
    mm = lambda X, Y: oracle.matmul(e, f, X, Y).astype(np.int64)
    np.testing.assert_array_equal(mm(A, np.eye(12, dtype=np.int64)), A)
    np.testing.assert_array_equal(mm(np.eye(9, dtype=np.int64), A), A)
    assert (mm(A, np.zeros((12, 5), dtype=np.int64)) == 0).all()
    np.testing.assert_array_equal(mm(A, B ^ B2), mm(A, B) ^ mm(A, B2))
    np.testing.assert_array_equal(mm(mm(A, B), D), mm(A, mm(B, D)))
    np.testing.assert_array_equal(mm(A, B).T, mm(B.T, A.T))
    T = fr.log_table_product(e, f)
    for j in (1, e - 1, e + 3):
        aj = fr.x_power_mod(e, f, j)
        np.testing.assert_array_equal(mm(aj * np.eye(12, dtype=np.int64), B), T[aj, B.astype(np.int64)])
    C1 = oracle.addmul(e, f, A, B, C0).astype(np.int64)
    np.testing.assert_array_equal(C1, mm(A, B) ^ C0)
    np.testing.assert_array_equal(oracle.addmul(e, f, A, B, C1), C0)
    # k = 0: mul gives zero, addmul leaves C
    assert (mm(A[:, :0], B[:0]) == 0).all()
    np.testing.assert_array_equal(oracle.addmul(e, f, A[:, :0], B[:0], C0), C0)


def test_oracle_rejects_out_of_range_entries():
    with pytest.raises(ValueError):
        oracle.matmul(2, 0x7, [[4]], [[1]])


def test_freivalds_accepts_correct_and_rejects_planted_error():
    e, f = 4, 0x13
    A, B, _ = workloads.random_problem(e, 40, 30, 50, seed=3)
    C = oracle.matmul(e, f, A, B)
    assert oracle.freivalds(e, f, A, B, C, trials=16)
    bad = C.copy()
    bad[17, 11] ^= 1
    assert not oracle.freivalds(e, f, A, B, bad, trials=16)


def test_threads_setting():
    n = oracle.get_threads()
    assert n >= 1
    oracle.set_threads(1)
    assert oracle.get_threads() == 1
    oracle.set_threads(0)
    assert oracle.get_threads() == n


# ---------------------------------------------------------------- TRSM (Section 4.3, Algorithm 5)


def _triangular(e, m, upper, rng, junk=False):
    """Random triangular matrix with non-zero diagonal; `junk` fills the other
    triangle with random entries (which a solver must not read)."""
    T = rng.integers(0, 1 << e, size=(m, m)).astype(np.uint16)
    keep = np.triu(np.ones((m, m), bool)) if upper else np.tril(np.ones((m, m), bool))
    if not junk:
        T[~keep] = 0
    T[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m)
    return T


@pytest.mark.parametrize("e", [2, 3, 4, 5, 8, 9, 10])
def test_field_inverse_against_log_tables(e):
    f = workloads.FIELD_POLY[e]
    table = fr.log_table_product(e, f)
    for a in range(1, 1 << e):
        assert table[a, oracle.gf_inv(e, f, a)] == 1
    assert oracle.gf_inv(e, f, 0) == 0


@pytest.mark.parametrize("e", [2, 3, 4, 7, 8, 10])
@pytest.mark.parametrize("upper", [True, False])
def test_trsm_solves_the_system(e, upper):
    """T * X == B, the product formed by the slice decomposition of Section 5
    (fieldref), not by the oracle; X is unique because T is invertible."""
    rng = np.random.default_rng(100 + e)
    f = workloads.FIELD_POLY[e]
    m, n = 29, 17
    T = _triangular(e, m, upper, rng)
    B = rng.integers(0, 1 << e, size=(m, n)).astype(np.uint16)
    X = oracle.trsm(e, f, T, B, upper)
    assert np.array_equal(fr.slice_product(e, f, T, X), B.astype(np.int64))


@pytest.mark.parametrize("upper", [True, False])
def test_trsm_ignores_the_other_triangle(upper):
    rng = np.random.default_rng(7)
    e, f = 4, workloads.FIELD_POLY[4]
    T = _triangular(e, 20, upper, rng)
    J = T.copy()
    keep = np.triu(np.ones(T.shape, bool)) if upper else np.tril(np.ones(T.shape, bool))
    J[~keep] = rng.integers(0, 1 << e, size=int((~keep).sum()))
    B = rng.integers(0, 1 << e, size=(20, 9)).astype(np.uint16)
    assert np.array_equal(oracle.trsm(e, f, T, B, upper), oracle.trsm(e, f, J, B, upper))


def test_trsm_identity_and_diagonal():
    rng = np.random.default_rng(8)
    e, f = 8, workloads.FIELD_POLY[8]
    table = fr.log_table_product(e, f)
    B = rng.integers(0, 256, size=(12, 7)).astype(np.uint16)
    assert np.array_equal(oracle.trsm(e, f, np.eye(12, dtype=np.uint16), B), B)
    d = rng.integers(1, 256, size=12)
    D = np.diag(d).astype(np.uint16)
    X = oracle.trsm(e, f, D, B, upper=False)
    # D X = B row by row: d_i * X[i][c] == B[i][c] in the log-table field
    for i in range(12):
        assert all(table[d[i], X[i, c]] == B[i, c] for c in range(7))


def test_trsm_brute_force_2x2_over_gf4():
    """Every invertible upper-triangular 2x2 system over GF(4) with every
    right-hand side: the oracle's X is the unique x with T x = b."""
    e, f = 2, workloads.FIELD_POLY[2]
    table = fr.log_table_product(e, f)
    for t00, t01, t11, b0, b1 in itertools.product(range(1, 4), range(4), range(1, 4), range(4), range(4)):
        sols = [(x0, x1) for x0 in range(4) for x1 in range(4)
                if table[t00, x0] ^ table[t01, x1] == b0 and table[t11, x1] == b1]
        assert len(sols) == 1
        T = np.array([[t00, t01], [0, t11]], dtype=np.uint16)
        X = oracle.trsm(e, f, T, np.array([[b0], [b1]], dtype=np.uint16))
        assert (int(X[0, 0]), int(X[1, 0])) == sols[0]


def test_trsm_zero_diagonal_raises():
    T = np.array([[1, 2], [0, 0]], dtype=np.uint16)
    with pytest.raises(ZeroDivisionError):
        oracle.trsm(2, 7, T, np.ones((2, 3), dtype=np.uint16))


# ---------------------------------------------------------------- echelon form (Section 4.1, Algorithm 4)


def random_rref(e, m, n, rank, rng):
    """A random matrix in reduced row echelon form with the given rank: pivot
    columns drawn at random, leading 1s, zeros in the other rows of pivot
    columns and left of each pivot, random entries elsewhere."""
    piv = np.sort(rng.choice(n, size=rank, replace=False))
    R = np.zeros((m, n), dtype=np.int64)
    for i, p in enumerate(piv):
        R[i, p + 1:] = rng.integers(0, 1 << e, size=n - p - 1)
        R[i, p] = 1
    for i, p in enumerate(piv):
        R[:rank, p] = 0
        R[i, p] = 1
    return R, piv


def random_invertible(e, f, m, rng):
    """S = L U with L unit lower and U upper triangular with non-zero diagonal."""
    L = np.tril(rng.integers(0, 1 << e, size=(m, m)), -1) + np.eye(m, dtype=np.int64)
    U = np.triu(rng.integers(0, 1 << e, size=(m, m)), 1)
    U[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m)
    return fr.slice_product(e, f, L, U)


def is_rref(R, rank):
    lead = -1
    for i in range(R.shape[0]):
        nz = np.nonzero(R[i])[0]
        if i >= rank:
            if nz.size:
                return False
            continue
        if not nz.size or nz[0] <= lead or R[i, nz[0]] != 1:
            return False
        lead = nz[0]
        col = R[:, lead].copy()
        col[i] = 0
        if col.any():
            return False
    return True


@pytest.mark.parametrize("e,m,n,rank", [(2, 12, 15, 12), (3, 20, 11, 7), (4, 16, 16, 16), (8, 30, 40, 22),
                                        (10, 9, 25, 5), (5, 14, 14, 0)])
def test_echelon_recovers_a_constructed_rref(e, m, n, rank):
    """A = S R with R in reduced row echelon form and S invertible has the
    row space of R, so its reduced echelon form is exactly R (uniqueness)."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(e * 100 + m + n + rank)
    R, piv = random_rref(e, m, n, rank, rng)
    A = fr.slice_product(e, f, random_invertible(e, f, m, rng), R)
    E, r, p = oracle.echelon(e, f, A)
    assert r == rank
    assert np.array_equal(E.astype(np.int64), R)
    assert np.array_equal(p, piv)


def _row_space(e, table, M):
    """All linear combinations of the rows of M over GF(2^e) (small M only)."""
    rows = [tuple(int(v) for v in r) for r in M]
    space = {tuple([0] * M.shape[1])}
    for r in rows:
        space = {tuple(a ^ int(table[c, b]) for a, b in zip(v, r)) for v in space for c in range(1 << e)}
    return space


def test_echelon_brute_force_small_gf4():
    """Every 2 x 2 and a sample of 3 x 3 matrices over GF(4): the output is in
    reduced row echelon form, has the input's row space (enumerated), and its
    rank is the number of non-zero rows."""
    e, f = 2, workloads.FIELD_POLY[2]
    table = fr.log_table_product(e, f)
    cases = [np.array(v, dtype=np.uint8).reshape(2, 2) for v in itertools.product(range(4), repeat=4)]
    rng = np.random.default_rng(3)
    cases += [rng.integers(0, 4, size=(3, 3)).astype(np.uint8) for _ in range(300)]
    cases += [rng.integers(0, 4, size=(2, 4)).astype(np.uint8) for _ in range(100)]
    for A in cases:
        E, r, _ = oracle.echelon(e, f, A)
        assert is_rref(E.astype(np.int64), r), A
        assert _row_space(e, table, A) == _row_space(e, table, E), A
        assert r == int((E != 0).any(axis=1).sum())


def test_echelon_is_idempotent_and_zero_matrix():
    e, f = 7, workloads.FIELD_POLY[7]
    rng = np.random.default_rng(4)
    A = rng.integers(0, 128, size=(25, 31)).astype(np.uint8)
    E, r, p = oracle.echelon(e, f, A)
    E2, r2, p2 = oracle.echelon(e, f, E)
    assert np.array_equal(E, E2) and r == r2 and np.array_equal(p, p2)
    Z, rz, pz = oracle.echelon(e, f, np.zeros((5, 6), np.uint8))
    assert rz == 0 and not Z.any() and pz.size == 0


# ---------------------------------------------------------------- planted mistakes

_MUTANTS = {
    # reduction subtracts f at the wrong degree
    "reduce_shift": ("p ^= f << (d - e);", "p ^= f << (d - e + 1);"),
    # reduction skips the highest product term
    "reduce_top": ("for (int d = 2 * e - 2; d >= e; d--)", "for (int d = 2 * e - 3; d >= e; d--)"),
    # carry-less multiply drops the top coefficient of b
    "clmul_term": ("for (int i = 0; i < e; i++)\n        if ((b >> i) & 1u)", "for (int i = 0; i < e - 1; i++)\n        if ((b >> i) & 1u)"),
    # matmul drops the last term of the inner sum
    "dropped_t": ("for (int64_t t = 0; t < k; t++) {", "for (int64_t t = 0; t + 1 < k; t++) {"),
    # matmul reads A transposed (only visible on non-symmetric inputs)
    "transposed_a": ("uint32_t a = A[r * k + t];", "uint32_t a = A[(t % m) * k + (r % k)];"),
    # slicing uses most-significant-bit-first columns
    "slice_msb": ("row[c / 64] |= (uint64_t)1 << (c % 64);", "row[c / 64] |= (uint64_t)1 << (63 - c % 64);"),
    # accumulation that overwrites C instead of adding to it
    "addmul_overwrites": ("        if (!accumulate)\n            for (int64_t c = 0; c < n; c++)\n                crow[c] = 0;",
                          "        if (1)\n            for (int64_t c = 0; c < n; c++)\n                crow[c] = 0;"),
    # addition as OR instead of XOR
    "add_or": ("crow[c] ^= (uint16_t)oracle_gf_mul(e, f, a, brow[c]);", "crow[c] |= (uint16_t)oracle_gf_mul(e, f, a, brow[c]);"),
    # packed fields placed highest first in the word
    "packed_msb": ("row[c / per] |= (uint64_t)elems[r * cols + c] << (w * (c % per));",
                   "row[c / per] |= (uint64_t)elems[r * cols + c] << (w * (per - 1 - c % per));"),
    # packing as many elements as fit instead of padding to a length dividing 64
    "packed_no_pad": ("    while (w < e)\n        w *= 2;\n    return w;", "    return e;"),
    # field inverse with the wrong exponent
    "inv_exponent": ("x = (1u << e) - 2;", "x = (1u << e) - 3;"),
    # upper solve reads the multiplier from the transposed position
    "trsm_transposed": ("uint32_t x = U[j * m + i];", "uint32_t x = U[i * m + j];"),
    # lower solve skips the row just below the pivot row
    "trsm_skip_row": ("for (int64_t j = i + 1; j < m; j++) {", "for (int64_t j = i + 2; j < m; j++) {"),
    # echelon form without scaling the pivot row to a leading 1
    "echelon_no_scale": ("ai[c] = (uint16_t)oracle_gf_mul(e, f, inv, ai[c]);", "ai[c] = ai[c];"),
    # echelon form that clears only the rows below the pivot (not reduced)
    "echelon_below_only": ("for (int64_t k = 0; k < m; k++) {\n            if (k == r)", "for (int64_t k = r + 1; k < m; k++) {\n            if (k == r)"),
    # echelon form that searches for a pivot from the top instead of at or below the rank
    "echelon_search_from_top": ("        int64_t i = r;\n        while (i < m && A[i * n + j] == 0)\n            i++;\n        if (i == m)\n            continue;\n        uint32_t inv",
                                "        int64_t i = 0;\n        while (i < m && A[i * n + j] == 0)\n            i++;\n        if (i == m)\n            continue;\n        uint32_t inv"),
    # echelon form that leaves the pivot row where it was found
    "echelon_no_swap": ("        if (i != r) {\n            uint16_t *ar = A + r * n;", "        if (0) {\n            uint16_t *ar = A + r * n;"),
    # echelon form that records the pivot's row instead of its column
    "echelon_pivot_row": ("            pivots[r] = j;", "            pivots[r] = i;"),
    # echelon form that clears the other rows only right of the pivot column
    "echelon_keeps_pivot_column": ("            for (int64_t c = j; c < n; c++)\n                ak[c] ^=",
                                   "            for (int64_t c = j + 1; c < n; c++)\n                ak[c] ^="),
    # lower solve reads the multiplier from the transposed position
    "trsm_lower_transposed": ("            uint32_t x = L[j * m + i];", "            uint32_t x = L[i * m + j];"),
    # slices in reverse order (slice 0 = the highest coefficient)
    "slice_reversed": ("                if ((elems[r * cols + c] >> i) & 1u)", "                if ((elems[r * cols + c] >> (e - 1 - i)) & 1u)"),
    # clinging puts slice i at the wrong bit
    "cling_reversed": ("                v |= (uint32_t)((row[c / 64] >> (c % 64)) & 1u) << i;",
                       "                v |= (uint32_t)((row[c / 64] >> (c % 64)) & 1u) << (e - 1 - i);"),
    # unpacking keeps the padding bits of a field
    "unpack_keeps_padding": ("(uint16_t)((word >> (w * (c % per))) & ((1u << e) - 1u));",
                             "(uint16_t)((word >> (w * (c % per))) & ((1u << w) - 1u));"),
    # upper solve does not scale by the inverse diagonal entry
    # PLE: the pivot row left where it was found
    "ple_no_swap": ("        if (i != r) {\n            uint16_t *ai = A + i * n, *ar = A + r * n;",
                    "        if (0) {\n            uint16_t *ai = A + i * n, *ar = A + r * n;"),
    # PLE: the swap not recorded in P
    "ple_p_not_recorded": ("        P[r] = i;", "        P[r] = r;"),
    # PLE: Q records the pivot's row
    "ple_q_records_row": ("        Q[r] = j;", "        Q[r] = i;"),
    # PLE: the pivot row not scaled to a leading 1
    "ple_no_scale": ("            pr[c] = (uint16_t)oracle_gf_mul(e, f, inv, pr[c]);\n#pragma omp parallel for schedule(static) num_threads(nt) if ((m - r) * (n - j) > 65536)",
                     "            pr[c] = pr[c];\n#pragma omp parallel for schedule(static) num_threads(nt) if ((m - r) * (n - j) > 65536)"),
    # PLE: the addition starts at the pivot column, so L is overwritten
    "ple_clears_l": ("            for (int64_t c = j + 1; c < n; c++)\n                ak[c] ^= (uint16_t)oracle_gf_mul(e, f, x, pr[c]);\n        }\n        r++;",
                     "            for (int64_t c = j; c < n; c++)\n                ak[c] ^= (uint16_t)oracle_gf_mul(e, f, x, pr[c]);\n        }\n        r++;"),
    # PLE: the rows above the pivot cleared as well (reduced form)
    "ple_clears_above": ("        for (int64_t k = r + 1; k < m; k++) {\n            uint32_t x = A[k * n + j];",
                         "        for (int64_t k = 0; k < m; k++) {\n            uint32_t x = k == r ? 0 : A[k * n + j];"),
    # PLE: L left in the pivot columns
    "ple_no_compress": ("    for (int64_t t = 0; t < r; t++) {\n        int64_t q = Q[t];", "    for (int64_t t = 0; t < 0; t++) {\n        int64_t q = Q[t];"),
    # PLE: the column swaps applied to every row, not only on and below the diagonal
    "ple_compress_all_rows": ("        for (int64_t k = t; k < m; k++) {\n            uint16_t v = A[k * n + t];",
                              "        for (int64_t k = 0; k < m; k++) {\n            uint16_t v = A[k * n + t];"),
    # PLE: the last row with a non-zero entry becomes the pivot (a valid PLE, but not Algorithm 4's)
    "ple_last_row": ("        int64_t i = r;\n        while (i < m && A[i * n + j] == 0)\n            i++;\n        if (i == m)\n            continue;\n        if (i != r) {",
                     "        int64_t i = m - 1;\n        while (i >= r && A[i * n + j] == 0)\n            i--;\n        if (i < r)\n            continue;\n        if (i != r) {"),
    "trsm_no_scale": ("for (int64_t i = m - 1; i >= 0; i--) {\n        uint32_t d = U[i * m + i];\n        if (d == 0)\n            return -1;\n        uint32_t dinv = oracle_gf_inv(e, f, d);",
                      "for (int64_t i = m - 1; i >= 0; i--) {\n        uint32_t d = U[i * m + i];\n        if (d == 0)\n            return -1;\n        uint32_t dinv = 1;"),
}


def _pins_pass(O: oracle.OracleLib) -> bool:
    """The cheap pins of this file, run against one compiled copy of the oracle."""
    try:
        e, elems, slices = _read_fig1()
        planes = O.slice_(e, elems)
        for i in range(e):
            got = np.array([[(int(planes[i, r, 0]) >> c) & 1 for c in range(2)] for r in range(2)])
            if not np.array_equal(got, slices[i]):
                return False
        # clinging of the printed slices (built from the figure, not by slice_)
        printed = np.zeros((e, 2, 1), np.uint64)
        for i in range(e):
            for r in range(2):
                printed[i, r, 0] = sum(int(slices[i][r][c]) << c for c in range(2))
        if not np.array_equal(O.cling(e, printed, 2).astype(np.int64), np.asarray(elems, np.int64)):
            return False
        fields = _read_fig1_packed()
        if O.packed_width(e) != 4 or O.packed_width(5) != 8:
            return False
        Wd = O.to_packed(e, elems)
        if any(int(Wd[r, 0]) != sum(int(fields[r][c], 2) << (4 * c) for c in range(2)) for r in range(2)):
            return False
        # unpacking of the printed packed rows with every padding bit set: bit 3 of
        # each 4-bit field (above e = 3) and the unused fields 2..15
        dirty = np.zeros((2, 1), np.uint64)
        for r in range(2):
            word = sum(int(fields[r][c], 2) << (4 * c) for c in range(2))
            dirty[r, 0] = word | 0x88 | (((1 << 64) - 1) ^ 0xFF)
        if not np.array_equal(O.from_packed(e, dirty, 2).astype(np.int64), np.asarray(elems, np.int64)):
            return False
        # a pivot below the current row: the permutation matrix reduces to the identity
        E, r, p = O.echelon(2, 7, np.array([[0, 1], [1, 0]], np.uint8))
        if r != 2 or not np.array_equal(E.astype(np.int64), np.eye(2, dtype=np.int64)) or list(p) != [0, 1]:
            return False
        for e in (2, 4, 8, 10):
            f = workloads.FIELD_POLY[e]
            if not np.array_equal(O.mul_table(e, f).astype(np.int64), fr.log_table_product(e, f)):
                return False
        for e in (2, 5):
            f = workloads.FIELD_POLY[e]
            A, B, C = workloads.random_problem(e, 13, 11, 17, seed=9, with_c=True)
            if not np.array_equal(O.matmul(e, f, A, B).astype(np.int64), fr.slice_product(e, f, A, B)):
                return False
            if not np.array_equal(O.addmul(e, f, A, B, C).astype(np.int64),
                                  fr.slice_product(e, f, A, B) ^ C.astype(np.int64)):
                return False
        for e in (3, 8):
            f = workloads.FIELD_POLY[e]
            table = fr.log_table_product(e, f)
            if any(table[a, O.gf_inv(e, f, a)] != 1 for a in range(1, 1 << e)):
                return False
            rng = np.random.default_rng(e)
            for upper in (True, False):
                T = _triangular(e, 9, upper, rng)
                B = rng.integers(0, 1 << e, size=(9, 5)).astype(np.uint16)
                if not np.array_equal(fr.slice_product(e, f, T, O.trsm(e, f, T, B, upper)), B.astype(np.int64)):
                    return False
            R, piv = random_rref(e, 10, 14, 6, rng)
            A = fr.slice_product(e, f, random_invertible(e, f, 10, rng), R)
            E, r, p = O.echelon(e, f, A)
            if r != 6 or not np.array_equal(E.astype(np.int64), R) or not np.array_equal(p, piv):
                return False
            # PLE of the same S R and of a matrix with zero rows on top
            Z = rng.integers(0, 1 << e, size=(9, 7))
            Z[:4] = 0
            for M in (A, Z):
                out, r, P, Q = O.ple(e, f, M.astype(np.uint16))
                _, rr, pv = O.echelon(e, f, M)
                if not pleref.layout_ok(out, r, P, Q) or r != rr or list(Q[:r]) != list(pv):
                    return False
                if not np.array_equal(pleref.rebuild(e, f, out, r, P, Q, fr.slice_product), M.astype(np.int64)):
                    return False
        # the hand-worked PLE example
        from tests.test_oracle_ple import read_hand_example
        e, f, A, R, r, P, Q = read_hand_example()
        out, rk, p, q = O.ple(e, f, A.astype(np.uint8))
        if rk != r or not np.array_equal(out.astype(np.int64), R) or list(p) != P or list(q) != Q:
            return False
        return True
    except Exception:
        return False


def test_pins_pass_on_the_oracle():
    assert _pins_pass(oracle.default())


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = _MUTANTS[name]
    with open(oracle.SOURCE) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = tmp_path / f"oracle_{name}.c"
    mut.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mut), str(tmp_path / f"lib_{name}.so"))
    assert not _pins_pass(oracle.OracleLib(lib)), f"pins did not detect mutant {name}"
