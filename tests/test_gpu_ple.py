"""PLE decomposition (Section 4.2) on the GPU against the oracle.  With
Algorithm 4's first-row pivoting the decomposition is unique, so the
overwritten matrix, the rank, P and Q are compared bit for bit."""
import numpy as np
import pytest

import oracle
import workloads
from tests import pleref
from tests.test_oracle import random_rref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1111_6900_gb300 as m4  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check(ctx, e, A, lda_pad=0):
    f = workloads.FIELD_POLY[e]
    m, n = A.shape
    if lda_pad:
        big = np.zeros((m, n + lda_pad), dtype=A.dtype)
        big[:, :n] = A
        big[:, n:] = 1  # must stay untouched
        d = dev(big)
        rank, P, Q = ctx.ple(e, f, d[:, :n])
        got = d.cpu().numpy()
        assert (got[:, n:] == 1).all()
        got = got[:, :n]
    else:
        d = dev(A)
        rank, P, Q = ctx.ple(e, f, d)
        got = d.cpu().numpy()
    out, r, Po, Qo = oracle.ple(e, f, A)
    assert rank == r
    np.testing.assert_array_equal(P, Po)
    np.testing.assert_array_equal(Q, Qo)
    np.testing.assert_array_equal(got, out)
    assert ctx.device_status() == m4.OK


SHAPES = [(1, 1), (1, 7), (7, 1), (5, 9), (130, 70), (70, 130), (128, 128), (257, 300), (300, 257), (600, 129),
          (64, 1000), (1000, 64)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("e", [2, 4, 8])
def test_ple_random_matches_oracle(e, m, n):
    rng = np.random.default_rng(e * 7919 + m * 31 + n + 5)
    A = rng.integers(0, 1 << e, size=(m, n)).astype(workloads.elem_dtype(e))
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


@pytest.mark.parametrize("e", [3, 5, 6, 7, 9, 10])
def test_ple_every_field(e):
    rng = np.random.default_rng(e + 50)
    A = rng.integers(0, 1 << e, size=(150, 200)).astype(workloads.elem_dtype(e))
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


@pytest.mark.parametrize("e,m,n,rank", [(2, 300, 400, 170), (4, 260, 260, 259), (8, 500, 140, 60),
                                        (10, 200, 333, 100), (4, 90, 80, 0), (5, 180, 500, 150)])
def test_ple_rank_deficient(e, m, n, rank):
    """A = S R with R a random reduced echelon matrix of the given rank: most
    columns have no pivot, so rounds stop early and search the other rows."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(rank + m + 1)
    R, piv = random_rref(e, m, n, rank, rng)
    L = np.tril(rng.integers(0, 1 << e, size=(m, m)), -1) + np.eye(m, dtype=np.int64)
    U = np.triu(rng.integers(0, 1 << e, size=(m, m)), 1)
    U[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m)
    dt = workloads.elem_dtype(e)
    S = oracle.matmul(e, f, L.astype(dt), U.astype(dt))
    A = oracle.matmul(e, f, S, R.astype(dt))
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


def test_ple_pivots_far_below_the_candidates():
    """Column 0 is non-zero only in the last row and column 1 only in the one
    before: the first rounds find no pivot among the candidate rows and the
    rows found below are swapped up (Algorithm 4's swap)."""
    e = 4
    rng = np.random.default_rng(19)
    m, n = 1500, 300
    A = rng.integers(0, 16, size=(m, n)).astype(np.uint8)
    A[:, 0] = 0
    A[m - 1, 0] = 5
    A[:, 1] = 0
    A[m - 2, 1] = 3
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


@pytest.mark.parametrize("e", [2, 8])
def test_ple_sparse_and_zero_blocks(e):
    """Zero rows on top, zero columns, and 85% zero entries: swaps from far
    below, empty columns inside panels and short rounds."""
    rng = np.random.default_rng(e + 3)
    dt = workloads.elem_dtype(e)
    A = rng.integers(0, 1 << e, size=(700, 450)).astype(dt)
    A[:250] = 0
    A[:, 60:75] = 0
    A[:, 200] = 0
    ctx = m4.Context()
    check(ctx, e, A)
    B = rng.integers(0, 1 << e, size=(400, 380)).astype(dt)
    B[rng.random(B.shape) < 0.85] = 0
    check(ctx, e, B)
    ctx.close()


def test_ple_window_and_zero_matrix():
    ctx = m4.Context()
    rng = np.random.default_rng(11)
    check(ctx, 8, rng.integers(0, 256, size=(200, 150)).astype(np.uint8), lda_pad=37)
    check(ctx, 8, np.zeros((64, 80), np.uint8))
    ctx.close()


def test_ple_invalid_arguments_and_optional_outputs():
    ctx = m4.Context()
    A = torch.ones((8, 8), dtype=torch.uint8, device="cuda")
    L, h = m4.lib, ctx.handle
    assert L.m4rie_ple(h, 4, 0x13, 8, 8, A.data_ptr(), 7, None, None, None) == m4.ERR_ARG   # lda < n
    assert L.m4rie_ple(h, 4, 0x15, 8, 8, A.data_ptr(), 8, None, None, None) == m4.ERR_POLY
    assert L.m4rie_ple(h, 11, 0x13, 8, 8, A.data_ptr(), 8, None, None, None) == m4.ERR_ARG
    assert L.m4rie_ple(h, 4, 0x13, 0, 8, None, 8, None, None, None) == m4.OK
    # rank, P and Q may be NULL: the matrix is still decomposed
    rng = np.random.default_rng(2)
    X = rng.integers(0, 16, size=(40, 50)).astype(np.uint8)
    d = dev(X)
    assert L.m4rie_ple(h, 4, 0x13, 40, 50, d.data_ptr(), 50, None, None, None) == m4.OK
    out, _, _, _ = oracle.ple(4, 0x13, X)
    np.testing.assert_array_equal(d.cpu().numpy(), out)
    ctx.close()


def _prefix_check(e, f, A, got, rank, P, Q, c):
    """Against the oracle's PLE of the first c columns: the steps whose pivot
    columns lie there depend on those columns only, so P, Q, L's columns and
    E's entries left of column c of those steps must agree exactly.  The
    later steps touch L's first columns only through their row swaps, which
    are replayed on the oracle's result."""
    out, rc, Pc, Qc = oracle.ple(e, f, A[:, :c])
    assert rc <= rank
    np.testing.assert_array_equal(P[:rc], Pc[:rc])
    np.testing.assert_array_equal(Q[:rc], Qc[:rc])
    cur = np.array(out[:, :rc], copy=True)
    for t in range(rc, rank):
        cur[[t, P[t]]] = cur[[P[t], t]]
    np.testing.assert_array_equal(got[:, :rc], cur)
    for k in range(rc):
        np.testing.assert_array_equal(got[k, Q[k] + 1:c], out[k, Q[k] + 1:c])


def _freivalds(e, f, A, got, rank, P, Q, trials=4, seed=0):
    """P L E = A on random vectors: L (E X) with rows swapped as P says
    against A X (oracle products)."""
    rng = np.random.default_rng(seed)
    m, n = A.shape
    dt = workloads.elem_dtype(e)
    X = rng.integers(0, 1 << e, size=(n, trials)).astype(dt)
    Lf, Ef = pleref.factors(got, rank, Q)
    EX = oracle.matmul(e, f, Ef.astype(dt), X)
    LEX = oracle.matmul(e, f, Lf.astype(dt), EX)
    np.testing.assert_array_equal(pleref.apply_p(LEX, rank, P), oracle.matmul(e, f, A, X).astype(np.int64))


def test_ple_full_size_random_gf4_4000():
    """The 4000 x 4000 GF(4) workload of the benchmark: layout, P L E = A by
    Freivalds, and the first 192 columns' steps exactly."""
    e, f = 2, workloads.FIELD_POLY[2]
    A = workloads.echelon_matrix(e, 4000, 4000, 1300)
    ctx = m4.Context()
    d = dev(A)
    rank, P, Q = ctx.ple(e, f, d)
    got = d.cpu().numpy()
    assert ctx.device_status() == m4.OK
    assert pleref.layout_ok(got, rank, P, Q)
    assert rank >= 3990
    _freivalds(e, f, A, got, rank, P, Q)
    _prefix_check(e, f, A, got, rank, P, Q, 192)
    ctx.close()


@pytest.mark.parametrize("e,size", [(2, 4096), (8, 2048)])
def test_ple_full_size_by_construction(e, size):
    """A = S R built on the GPU (S = L U invertible, R a random reduced
    echelon matrix of rank size - 37): rank and pivot columns are R's, and
    the checks of the random case hold."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(size + e + 1)
    m = n = size
    rank = size - 37
    R, piv = random_rref(e, m, n, rank, rng)
    dt = workloads.elem_dtype(e)
    Lw = np.tril(rng.integers(0, 1 << e, size=(m, m)), -1).astype(dt)
    Lw[np.arange(m), np.arange(m)] = 1
    U = np.triu(rng.integers(0, 1 << e, size=(m, m)), 1).astype(dt)
    U[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m)
    ctx = m4.Context()
    dS = ctx.mul(e, f, dev(Lw), dev(U))
    dA = ctx.mul(e, f, dS, dev(R.astype(dt)))
    A = dA.cpu().numpy()
    r, P, Q = ctx.ple(e, f, dA)
    got = dA.cpu().numpy()
    assert ctx.device_status() == m4.OK
    assert r == rank
    assert list(Q[:r]) == [int(v) for v in piv]
    assert pleref.layout_ok(got, r, P, Q)
    _freivalds(e, f, A, got, r, P, Q)
    _prefix_check(e, f, A, got, r, P, Q, 160)
    ctx.close()
