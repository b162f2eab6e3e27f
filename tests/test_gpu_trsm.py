"""Triangular solves (Section 4.3, Algorithm 5) and products on strided windows,
on the GPU, against the oracle."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1111_6900_gb300 as m4  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def triangular(e, m, upper, rng, junk=True):
    """Random triangular matrix with a non-zero diagonal; with `junk` the other
    triangle holds random entries, which the solver must not read."""
    T = rng.integers(0, 1 << e, size=(m, m)).astype(workloads.elem_dtype(e))
    if not junk:
        T = np.triu(T) if upper else np.tril(T)
    T[np.arange(m), np.arange(m)] = rng.integers(1, 1 << e, size=m)
    return T


def clean(T, upper):
    return np.triu(T) if upper else np.tril(T)


CASES = [(2, 1, 1), (3, 5, 7), (4, 127, 33), (4, 128, 64), (4, 129, 65), (5, 200, 100), (8, 300, 257),
         (9, 260, 40), (10, 385, 129), (6, 64, 1000), (7, 513, 31), (2, 640, 200)]


@pytest.mark.parametrize("e,m,n", CASES)
@pytest.mark.parametrize("upper", [True, False])
def test_trsm_matches_oracle(e, m, n, upper):
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(e * 1000 + m + n + upper)
    T = triangular(e, m, upper, rng)
    B = rng.integers(0, 1 << e, size=(m, n)).astype(workloads.elem_dtype(e))
    ctx = m4.Context()
    dB = dev(B)
    ctx.trsm(e, f, dev(T), dB, upper)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.trsm(e, f, clean(T, upper), B, upper))
    ctx.close()


@pytest.mark.parametrize("form,sched", [("popc", "alpha_b"), ("popc", "karatsuba"), ("tc_f8", "alpha_b"),
                                        ("tc_f8", "karatsuba"), ("tc_f4", "alpha_b"), ("tc_f4", "karatsuba"),
                                        ("mma_s8", "alpha_b"), ("mma_b1", "alpha_b")])
def test_trsm_every_form(form, sched):
    e, f = 4, workloads.FIELD_POLY[4]
    rng = np.random.default_rng(31)
    ctx = m4.Context()
    ctx.set_form(form)
    ctx.set_schedule(sched)
    for upper in (True, False):
        T = triangular(e, 333, upper, rng)
        B = rng.integers(0, 16, size=(333, 90)).astype(np.uint8)
        dB = dev(B)
        ctx.trsm(e, f, dev(T), dB, upper)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dB.cpu().numpy(), oracle.trsm(e, f, clean(T, upper), B, upper))
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_trsm_on_windows_leaves_the_rest_alone():
    e, f = 8, workloads.FIELD_POLY[8]
    rng = np.random.default_rng(5)
    m, n = 300, 70
    bigT = rng.integers(0, 256, size=(m + 9, m + 40)).astype(np.uint8)
    bigB = rng.integers(0, 256, size=(m + 5, n + 33)).astype(np.uint8)
    T = bigT[4:4 + m, 16:16 + m].copy()
    T[np.arange(m), np.arange(m)] = rng.integers(1, 256, size=m)
    bigT[4:4 + m, 16:16 + m] = T
    dT, dBig = dev(bigT), dev(bigB)
    ctx = m4.Context()
    ctx.trsm(e, f, dT[4:4 + m, 16:16 + m], dBig[3:3 + m, 16:16 + n], upper=True)
    torch.cuda.synchronize()
    got = dBig.cpu().numpy()
    want = bigB.copy()
    want[3:3 + m, 16:16 + n] = oracle.trsm(e, f, np.triu(T), bigB[3:3 + m, 16:16 + n], True)
    np.testing.assert_array_equal(got, want)
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_trsm_zero_diagonal_sets_singular():
    e, f = 4, workloads.FIELD_POLY[4]
    rng = np.random.default_rng(6)
    T = triangular(e, 200, True, rng)
    T[150, 150] = 0
    ctx = m4.Context()
    dB = dev(rng.integers(0, 16, size=(200, 8)).astype(np.uint8))
    ctx.trsm(e, f, dev(T), dB, True)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.ERR_SINGULAR
    assert ctx.device_status() == m4.OK   # the status word is cleared by reading it
    ctx.close()


def test_trsm_out_of_range_entry_sets_range():
    e, f = 3, workloads.FIELD_POLY[3]
    rng = np.random.default_rng(7)
    T = triangular(e, 40, False, rng)
    T[10, 3] = 9   # >= 2^3, inside the lower triangle
    ctx = m4.Context()
    dB = dev(rng.integers(0, 8, size=(40, 8)).astype(np.uint8))
    ctx.trsm(e, f, dev(T), dB, False)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.ERR_RANGE
    ctx.close()


def test_trsm_invalid_arguments():
    ctx = m4.Context()
    T = torch.ones((8, 8), dtype=torch.uint8, device="cuda")
    B = torch.ones((8, 4), dtype=torch.uint8, device="cuda")
    L = m4.lib
    h = ctx.handle
    assert L.m4rie_trsm_upper_left(h, 4, 0x13, 8, 4, T.data_ptr(), 7, B.data_ptr(), 4) == m4.ERR_ARG  # ldt < m
    assert L.m4rie_trsm_upper_left(h, 4, 0x13, 8, 4, T.data_ptr(), 8, B.data_ptr(), 3) == m4.ERR_ARG  # ldb < n
    assert L.m4rie_trsm_upper_left(h, 4, 0x15, 8, 4, T.data_ptr(), 8, B.data_ptr(), 4) == m4.ERR_POLY
    assert L.m4rie_trsm_lower_left(h, 4, 0x13, 8, 4, T.data_ptr(), 8, T.data_ptr(), 4) == m4.ERR_ALIAS
    assert L.m4rie_trsm_lower_left(h, 4, 0x13, 0, 4, None, 0, None, 4) == m4.OK  # empty system
    assert L.m4rie_trsm_lower_left(h, 4, 0x13, 8, 0, T.data_ptr(), 8, None, 0) == m4.OK
    ctx.close()


def test_trsm_replay_sees_new_contents():
    """Repeated solves on the same buffers replay the recorded graph; it must
    read the buffers' current contents, and a settings change re-records."""
    e, f = 4, workloads.FIELD_POLY[4]
    rng = np.random.default_rng(21)
    m, n = 700, 300
    T = triangular(e, m, True, rng)
    dT = dev(T)
    dB = torch.empty((m, n), dtype=torch.uint8, device="cuda")
    ctx = m4.Context()
    for trial in range(4):
        if trial == 2:                      # new matrix in the same buffer
            T = triangular(e, m, True, rng)
            dT.copy_(dev(T))
        if trial == 3:                      # other settings: a new recording
            ctx.set_form("popc")
        B = rng.integers(0, 16, size=(m, n)).astype(np.uint8)
        dB.copy_(dev(B))
        launches = ctx.kernel_launches()
        ctx.trsm(e, f, dT, dB, True)
        torch.cuda.synchronize()
        assert ctx.kernel_launches() > launches
        np.testing.assert_array_equal(dB.cpu().numpy(), oracle.trsm(e, f, np.triu(T), B, True), err_msg=f"trial {trial}")
    assert ctx.device_status() == m4.OK
    ctx.close()


def _solve_and_check_by_columns(e, m, n, upper, seed, sample=12):
    """Full-size solve: T X == B through the (separately parity-tested) GPU
    product, and sampled columns of X against the oracle (columns of a
    triangular solve are independent)."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(seed)
    T = triangular(e, m, upper, rng, junk=False)
    B = rng.integers(0, 1 << e, size=(m, n)).astype(workloads.elem_dtype(e))
    ctx = m4.Context()
    dT, dB = dev(T), dev(B)
    dX = dB.clone()
    ctx.trsm(e, f, dT, dX, upper)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    assert torch.equal(ctx.mul(e, f, dT, dX), dB)
    cols = np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=sample, replace=False)]))
    X = dX.cpu().numpy()
    np.testing.assert_array_equal(X[:, cols], oracle.trsm(e, f, T, B[:, cols], upper))
    ctx.close()


@pytest.mark.parametrize("upper", [True, False])
def test_trsm_2048_by_1000_gf256(upper):
    _solve_and_check_by_columns(8, 2048, 1000, upper, seed=11)


def test_trsm_full_size_gf16_4096():
    """The size the benchmark times: 4096 x 4096 over GF(2^4)."""
    _solve_and_check_by_columns(4, 4096, 4096, True, seed=12)


def test_trsm_gf1024_1100():
    _solve_and_check_by_columns(10, 1100, 300, False, seed=13)


# ---------------------------------------------------------------- strided products (m4rie_gemm)


@pytest.mark.parametrize("form,sched", [("popc", "alpha_b"), ("popc", "karatsuba"), ("tc_f8", "karatsuba"),
                                        ("tc_f4", "alpha_b"), ("tc_f4", "karatsuba"), ("mma_s8", "alpha_b"),
                                        ("mma_b1", "alpha_b")])
@pytest.mark.parametrize("e", [3, 8, 10])
def test_gemm_on_windows(form, sched, e):
    f = workloads.FIELD_POLY[e]
    dt = workloads.elem_dtype(e)
    rng = np.random.default_rng(e + 17)
    m, n, k = 150, 131, 77
    bigA = rng.integers(0, 1 << e, size=(m + 6, k + 40)).astype(dt)
    bigB = rng.integers(0, 1 << e, size=(k + 3, n + 21)).astype(dt)
    bigC = rng.integers(0, 1 << e, size=(m + 2, n + 50)).astype(dt)
    A, B = bigA[5:5 + m, 8:8 + k], bigB[2:2 + k, 16:16 + n]
    ctx = m4.Context()
    ctx.set_form(form)
    ctx.set_schedule(sched)
    for acc in (False, True):
        dA, dB, dC = dev(bigA), dev(bigB), dev(bigC)
        ctx.gemm(e, f, dA[5:5 + m, 8:8 + k], dB[2:2 + k, 16:16 + n], dC[1:1 + m, 32:32 + n], accumulate=acc)
        torch.cuda.synchronize()
        want = bigC.copy()
        want[1:1 + m, 32:32 + n] = (oracle.addmul(e, f, A, B, bigC[1:1 + m, 32:32 + n]) if acc
                                    else oracle.matmul(e, f, A, B))
        np.testing.assert_array_equal(dC.cpu().numpy(), want, err_msg=f"accumulate={acc}")
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_gemm_window_arguments():
    ctx = m4.Context()
    C = torch.zeros((10, 40), dtype=torch.uint8, device="cuda")
    A = torch.ones((10, 8), dtype=torch.uint8, device="cuda")
    B = torch.ones((8, 16), dtype=torch.uint8, device="cuda")
    L, h = m4.lib, ctx.handle
    # lda < k, ldb < n, ldc < n
    assert L.m4rie_gemm(h, 4, 0x13, 10, 16, 8, A.data_ptr(), 7, B.data_ptr(), 16, C.data_ptr(), 40, 0) == m4.ERR_ARG
    assert L.m4rie_gemm(h, 4, 0x13, 10, 16, 8, A.data_ptr(), 8, B.data_ptr(), 15, C.data_ptr(), 40, 0) == m4.ERR_ARG
    assert L.m4rie_gemm(h, 4, 0x13, 10, 16, 8, A.data_ptr(), 8, B.data_ptr(), 16, C.data_ptr(), 15, 0) == m4.ERR_ARG
    # C's window interleaves with an input's rows: spans overlap
    assert L.m4rie_gemm(h, 4, 0x13, 4, 16, 8, C.data_ptr(), 40, B.data_ptr(), 16, C.data_ptr() + 20, 40, 0) == m4.ERR_ALIAS
    # k = 0 on a window: only the window is zeroed
    C.fill_(7)
    assert L.m4rie_gemm(h, 4, 0x13, 3, 5, 0, None, 0, None, 5, C.data_ptr() + 41, 40, 0) == m4.OK
    torch.cuda.synchronize()
    want = torch.full((10, 40), 7, dtype=torch.uint8)
    want[1:4, 1:6] = 0
    assert torch.equal(C.cpu(), want)
    ctx.close()
