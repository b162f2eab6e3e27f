"""Reduced row echelon form (Section 4.1, Algorithm 4) on the GPU against the
oracle.  The reduced echelon form is unique, so results are compared bit for
bit whatever rows the GPU picks as pivots."""
import numpy as np
import pytest

import oracle
import workloads
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
        rank, piv = ctx.echelonize(e, f, d[:, :n])
        got = d.cpu().numpy()
        assert (got[:, n:] == 1).all()
        got = got[:, :n]
    else:
        d = dev(A)
        rank, piv = ctx.echelonize(e, f, d)
        got = d.cpu().numpy()
    E, r, p = oracle.echelon(e, f, A)
    assert rank == r
    assert piv == list(p)
    np.testing.assert_array_equal(got, E)
    assert ctx.device_status() == m4.OK


SHAPES = [(1, 1), (1, 7), (7, 1), (5, 9), (130, 70), (70, 130), (128, 128), (257, 300), (300, 257), (600, 129),
          (64, 1000), (1000, 64)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("e", [2, 4, 8])
def test_echelon_random_matches_oracle(e, m, n):
    rng = np.random.default_rng(e * 7919 + m * 31 + n)
    A = rng.integers(0, 1 << e, size=(m, n)).astype(workloads.elem_dtype(e))
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


@pytest.mark.parametrize("e", [3, 5, 6, 7, 9, 10])
def test_echelon_every_field(e):
    rng = np.random.default_rng(e)
    A = rng.integers(0, 1 << e, size=(150, 200)).astype(workloads.elem_dtype(e))
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


@pytest.mark.parametrize("e,m,n,rank", [(2, 300, 400, 170), (4, 260, 260, 259), (8, 500, 140, 60),
                                        (10, 200, 333, 100), (4, 90, 80, 0)])
def test_echelon_rank_deficient(e, m, n, rank):
    """A = S R with R a random reduced echelon matrix of the given rank."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(rank + m)
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


def test_echelon_pivot_outside_the_first_candidates():
    """Column 0 is non-zero only in the last row and every row has non-zero
    entries further right, so the first candidate rows miss column 0: a
    second round finds it and the panel's rows are put back in order."""
    e = 4
    rng = np.random.default_rng(9)
    m, n = 1500, 300
    A = rng.integers(0, 16, size=(m, n)).astype(np.uint8)
    A[:, 0] = 0
    A[m - 1, 0] = 5
    A[:, 1] = 0
    A[m - 2, 1] = 3
    ctx = m4.Context()
    check(ctx, e, A)
    ctx.close()


def test_echelon_window_and_zero_matrix():
    ctx = m4.Context()
    rng = np.random.default_rng(10)
    check(ctx, 8, rng.integers(0, 256, size=(200, 150)).astype(np.uint8), lda_pad=37)
    check(ctx, 8, np.zeros((64, 80), np.uint8))
    ctx.close()


def test_echelon_invalid_arguments():
    ctx = m4.Context()
    A = torch.ones((8, 8), dtype=torch.uint8, device="cuda")
    L, h = m4.lib, ctx.handle
    assert L.m4rie_echelonize(h, 4, 0x13, 8, 8, A.data_ptr(), 7, None, None) == m4.ERR_ARG   # lda < n
    assert L.m4rie_echelonize(h, 4, 0x15, 8, 8, A.data_ptr(), 8, None, None) == m4.ERR_POLY
    assert L.m4rie_echelonize(h, 11, 0x13, 8, 8, A.data_ptr(), 8, None, None) == m4.ERR_ARG
    assert L.m4rie_echelonize(h, 4, 0x13, 0, 8, None, 8, None, None) == m4.OK
    ctx.close()


@pytest.mark.parametrize("e,size", [(2, 4096), (8, 2048)])
def test_echelon_full_size_by_construction(e, size):
    """A = S R built on the GPU (S = L U invertible, R a random reduced echelon
    matrix of rank size - 37): the echelon form must be exactly R."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(size + e)
    m = n = size
    rank = size - 37
    R, piv = random_rref(e, m, n, rank, rng)
    dt = workloads.elem_dtype(e)
    L = np.tril(rng.integers(0, 1 << e, size=(m, m)), -1).astype(dt)
    L[np.arange(m), np.arange(m)] = 1
    U = np.triu(rng.integers(0, 1 << e, size=(m, m)), 1).astype(dt)
    U[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m)
    ctx = m4.Context()
    dS = ctx.mul(e, f, dev(L), dev(U))
    dA = ctx.mul(e, f, dS, dev(R.astype(dt)))
    r, p = ctx.echelonize(e, f, dA)
    assert r == rank
    assert p == [int(v) for v in piv]
    assert torch.equal(dA, dev(R.astype(dt)))
    assert ctx.device_status() == m4.OK
    ctx.close()
