"""The packed representation (Section 3.1) and Newton-John multiplication
(Section 4, Algorithms 2 and 3) on the GPU against the oracle, through the C
ABI.  Every comparison is bit for bit: field arithmetic has one result."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1111_6900_gb300 as m4  # noqa: E402

ALL_E = list(range(2, 11))


@pytest.fixture(scope="module")
def ctx():
    c = m4.Context()
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def words_dev(W):
    return dev(np.ascontiguousarray(W).view(np.int64))


def words_host(t):
    return t.cpu().numpy().view(np.uint64)


def per_word(e):
    return 64 // oracle.packed_width(e)


# ---------------------------------------------------------------- conversions


@pytest.mark.parametrize("e", ALL_E)
def test_packed_width_matches_oracle(e):
    assert m4.packed_width(e) == oracle.packed_width(e)


@pytest.mark.parametrize("e", ALL_E)
@pytest.mark.parametrize("rows,cols", [(1, 1), (3, 17), (70, 129), (257, 1000)])
def test_to_packed_matches_oracle(ctx, e, rows, cols):
    rng = np.random.default_rng(e * 1000 + rows + cols)
    X = workloads.elements(rng, e, (rows, cols))
    ld = (cols + per_word(e) - 1) // per_word(e) + 2  # two padding words per row
    W = ctx.to_packed(e, dev(X), ld_words=ld)
    np.testing.assert_array_equal(words_host(W), oracle.to_packed(e, X, ld_words=ld))
    assert ctx.device_status() == m4.OK


@pytest.mark.parametrize("e", ALL_E)
def test_from_packed_ignores_padding(ctx, e):
    rng = np.random.default_rng(40 + e)
    rows, cols = 33, 77
    X = workloads.elements(rng, e, (rows, cols))
    W = oracle.to_packed(e, X, ld_words=(cols + per_word(e) - 1) // per_word(e) + 1)
    w = oracle.packed_width(e)
    per = per_word(e)
    dirty = W.copy()
    # set every bit that is not an element bit: field bits above e, padding fields, padding words
    junk = np.uint64(sum(((1 << w) - 1 - ((1 << e) - 1)) << (w * j) for j in range(per)))
    dirty |= junk
    dirty[:, cols // per + 1:] = np.uint64(0xFFFFFFFFFFFFFFFF)
    if cols % per:
        dirty[:, cols // per] |= np.uint64(((1 << 64) - 1) ^ ((1 << (w * (cols % per))) - 1))
    got = ctx.from_packed(e, words_dev(dirty), cols)
    np.testing.assert_array_equal(got.cpu().numpy(), X)


def test_to_packed_window_and_range_flag(ctx):
    e = 3
    rng = np.random.default_rng(3)
    big = workloads.elements(rng, e, (20, 50))
    win = dev(big)[2:15, 5:40]
    W = ctx.to_packed(e, win)
    np.testing.assert_array_equal(words_host(W), oracle.to_packed(e, big[2:15, 5:40]))
    assert ctx.device_status() == m4.OK
    bad = big.copy()
    bad[4, 7] = 13  # >= 2^3: flagged, low 3 bits used
    W = ctx.to_packed(e, dev(bad))
    assert ctx.device_status() == m4.ERR_RANGE
    fixed = bad.copy()
    fixed[4, 7] = 13 & 7
    np.testing.assert_array_equal(words_host(W), oracle.to_packed(e, fixed))


def test_packed_invalid_arguments(ctx):
    L, h = m4.lib, ctx.handle
    X = torch.zeros((4, 40), dtype=torch.uint8, device="cuda")
    W = torch.zeros((4, 10), dtype=torch.int64, device="cuda")
    assert L.m4rie_to_packed(h, 4, 4, 40, X.data_ptr(), 40, W.data_ptr(), 2) == m4.ERR_ARG   # 3 words needed
    assert L.m4rie_to_packed(h, 11, 4, 40, X.data_ptr(), 40, W.data_ptr(), 10) == m4.ERR_ARG
    assert L.m4rie_to_packed(h, 4, 4, 40, X.data_ptr(), 39, W.data_ptr(), 10) == m4.ERR_ARG  # lde < cols
    assert L.m4rie_to_packed(h, 4, 4, 40, W.data_ptr(), 40, W.data_ptr(), 10) == m4.ERR_ALIAS
    assert L.m4rie_from_packed(h, 4, 4, 40, W.data_ptr(), 2, X.data_ptr(), 40) == m4.ERR_ARG
    # e = 4: 16 fields per 64-bit word, so 40 columns take 3 words
    A = torch.zeros((40, 3), dtype=torch.int64, device="cuda")
    C = torch.zeros((40, 3), dtype=torch.int64, device="cuda")
    a, c = A.data_ptr(), C.data_ptr()
    assert L.m4rie_mul_packed(h, 4, 0x13, 40, 40, 40, a, 3, a, 3, c, 2, 0) == m4.ERR_ARG    # ldc < 3
    assert L.m4rie_mul_packed(h, 4, 0x13, 40, 40, 40, a, 2, a, 3, c, 3, 0) == m4.ERR_ARG    # lda < 3
    assert L.m4rie_mul_packed(h, 4, 0x15, 40, 40, 40, a, 3, a, 3, c, 3, 0) == m4.ERR_POLY
    assert L.m4rie_mul_packed(h, 4, 0x13, 40, 40, 40, a, 3, a, 3, a, 3, 0) == m4.ERR_ALIAS
    assert L.m4rie_mul_packed(h, 4, 0x13, 0, 40, 40, None, 3, a, 3, None, 3, 0) == m4.OK


# ---------------------------------------------------------------- Newton-John on element arrays

SHAPES = [(1, 1, 1), (5, 9, 7), (130, 70, 33), (257, 300, 129), (1000, 17, 64), (64, 1000, 3), (33, 20, 5000)]


def nj_mul(ctx, e, A, B, C0=None):
    ctx.set_form("newton_john")
    try:
        f = workloads.FIELD_POLY[e]
        if C0 is None:
            C = ctx.mul(e, f, dev(A), dev(B))
        else:
            C = dev(C0)
            ctx.addmul(e, f, dev(A), dev(B), C)
        torch.cuda.synchronize()
        assert ctx.device_status() == m4.OK
        return C.cpu().numpy()
    finally:
        ctx.set_form("auto")


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("e", ALL_E)
def test_newton_john_mul_matches_oracle(ctx, e, m, n, k):
    A, B, _ = workloads.random_problem(e, m, n, k, seed=e * 7 + m + n + k)
    np.testing.assert_array_equal(nj_mul(ctx, e, A, B), oracle.matmul(e, workloads.FIELD_POLY[e], A, B))


@pytest.mark.parametrize("e", [2, 5, 8, 10])
def test_newton_john_addmul_matches_oracle(ctx, e):
    A, B, C = workloads.random_problem(e, 200, 150, 77, seed=e, with_c=True)
    np.testing.assert_array_equal(nj_mul(ctx, e, A, B, C), oracle.addmul(e, workloads.FIELD_POLY[e], A, B, C))


@pytest.mark.parametrize("e", [3, 9])
def test_newton_john_windows(ctx, e):
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(e + 100)
    bigA = workloads.elements(rng, e, (90, 120))
    bigB = workloads.elements(rng, e, (130, 80))
    bigC = workloads.elements(rng, e, (70, 90))
    dA, dB, dC = dev(bigA), dev(bigB), dev(bigC)
    ctx.set_form("newton_john")
    try:
        ctx.gemm(e, f, dA[3:63, 10:110], dB[5:105, 7:57], dC[4:64, 20:70], accumulate=True)
    finally:
        ctx.set_form("auto")
    want = bigC.copy()
    want[4:64, 20:70] = oracle.addmul(e, f, bigA[3:63, 10:110], bigB[5:105, 7:57], bigC[4:64, 20:70])
    np.testing.assert_array_equal(dC.cpu().numpy(), want)


@pytest.mark.parametrize("e", ALL_E)
@pytest.mark.parametrize("accumulate", [False, True])
def test_newton_john_16_byte_rows(ctx, e, accumulate):
    """Rows of B and C on 16-byte boundaries (n = 208 elements): a lane's whole
    words move as 16-byte vectors; for e <= 4 the last words of a row are a
    partial group of four and go one by one."""
    f = workloads.FIELD_POLY[e]
    A, B, C = workloads.random_problem(e, 150, 208, 70, seed=e + 40, with_c=True)
    if accumulate:
        np.testing.assert_array_equal(nj_mul(ctx, e, A, B, C), oracle.addmul(e, f, A, B, C))
    else:
        np.testing.assert_array_equal(nj_mul(ctx, e, A, B), oracle.matmul(e, f, A, B))


@pytest.mark.parametrize("e", [2, 4, 8, 10])
def test_newton_john_16_byte_windows(ctx, e):
    """Windows whose rows start on 16-byte boundaries (16-byte path) inside
    larger matrices: nothing outside the window of C changes."""
    f = workloads.FIELD_POLY[e]
    rng = np.random.default_rng(e + 200)
    bigA = workloads.elements(rng, e, (90, 120))
    bigB = workloads.elements(rng, e, (130, 240))
    bigC = workloads.elements(rng, e, (70, 256))
    dA, dB, dC = dev(bigA), dev(bigB), dev(bigC)
    ctx.set_form("newton_john")
    try:
        ctx.gemm(e, f, dA[3:63, 10:110], dB[5:105, 16:224], dC[4:64, 32:240], accumulate=True)
        torch.cuda.synchronize()
        assert ctx.device_status() == m4.OK
    finally:
        ctx.set_form("auto")
    want = bigC.copy()
    want[4:64, 32:240] = oracle.addmul(e, f, bigA[3:63, 10:110], bigB[5:105, 16:224], bigC[4:64, 32:240])
    np.testing.assert_array_equal(dC.cpu().numpy(), want)


def test_newton_john_16_byte_range_flag(ctx):
    """Entries >= 2^e in B and in the old C, inside words that take the 16-byte
    path: the status says so and the product uses their low e bits."""
    e = 4
    f = workloads.FIELD_POLY[e]
    A, B, C = workloads.random_problem(e, 64, 256, 40, seed=77, with_c=True)
    B2, C2 = B.copy(), C.copy()
    B2[11, 5] = 0xF3
    C2[9, 130] = 0x5A
    ctx.set_form("newton_john")
    try:
        dC = dev(C2)
        ctx.addmul(e, f, dev(A), dev(B2), dC)
        torch.cuda.synchronize()
        assert ctx.device_status() == m4.ERR_RANGE
    finally:
        ctx.set_form("auto")
    B2[11, 5] &= 15
    C2[9, 130] &= 15
    np.testing.assert_array_equal(dC.cpu().numpy(), oracle.addmul(e, f, A, B2, C2))


def test_newton_john_range_flag(ctx):
    e = 5
    A, B, _ = workloads.random_problem(e, 40, 30, 50, seed=5)
    A2 = A.copy()
    A2[3, 4] = 200
    B2 = B.copy()
    B2[7, 9] = 77
    ctx.set_form("newton_john")
    try:
        C = ctx.mul(e, workloads.FIELD_POLY[e], dev(A2), dev(B2))
        assert ctx.device_status() == m4.ERR_RANGE
    finally:
        ctx.set_form("auto")
    A2[3, 4] &= 31
    B2[7, 9] &= 31
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.matmul(e, workloads.FIELD_POLY[e], A2, B2))


def test_newton_john_k_zero(ctx):
    ctx.set_form("newton_john")
    try:
        C = dev(np.full((5, 6), 3, np.uint8))
        ctx.mul(4, 0x13, dev(np.zeros((5, 0), np.uint8)), dev(np.zeros((0, 6), np.uint8)), C)
        assert int(C.to(torch.int32).sum()) == 0
    finally:
        ctx.set_form("auto")


# ---------------------------------------------------------------- Newton-John on packed matrices


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 33, 65), (129, 257, 100), (40, 16, 3000), (300, 1000, 64)])
@pytest.mark.parametrize("e", ALL_E)
@pytest.mark.parametrize("accumulate", [False, True])
def test_mul_packed_matches_oracle(ctx, e, m, n, k, accumulate):
    f = workloads.FIELD_POLY[e]
    A, B, C0 = workloads.random_problem(e, m, n, k, seed=e + m + n + k + accumulate, with_c=True)
    per = per_word(e)
    nw, kw = (n + per - 1) // per, (k + per - 1) // per
    PA = oracle.to_packed(e, A, ld_words=kw + 1)
    PB = oracle.to_packed(e, B, ld_words=nw + 2)
    PC = oracle.to_packed(e, C0, ld_words=nw + 1)
    # junk in C's padding: ignored as input, written as zero
    w = oracle.packed_width(e)
    if n % per:
        PC[:, nw - 1] |= np.uint64(((1 << 64) - 1) ^ ((1 << (w * (n % per))) - 1))
    PC[:, nw] = np.uint64(0xFFFFFFFFFFFFFFFF)
    dC = words_dev(PC)
    ctx.mul_packed(e, f, words_dev(PA), words_dev(PB), dC, n=n, k=k, accumulate=accumulate)
    got = words_host(dC)
    want = oracle.addmul(e, f, A, B, C0) if accumulate else oracle.matmul(e, f, A, B)
    np.testing.assert_array_equal(got[:, :nw], oracle.to_packed(e, want))
    np.testing.assert_array_equal(got[:, nw], PC[:, nw])  # beyond the row's words: untouched
    assert ctx.device_status() == m4.OK


def test_mul_packed_field_bits_above_e_are_flagged(ctx):
    e, f = 3, workloads.FIELD_POLY[3]
    A, B, _ = workloads.random_problem(e, 20, 30, 40, seed=1)
    PA = oracle.to_packed(e, A)
    PB = oracle.to_packed(e, B)
    PB[2, 0] |= np.uint64(8 << 4)  # bit 3 of the field of column 1: above e
    dC = words_dev(np.zeros((20, PB.shape[1]), np.uint64))
    ctx.mul_packed(e, f, words_dev(PA), words_dev(PB), dC, n=30, k=40)
    assert ctx.device_status() == m4.ERR_RANGE
    np.testing.assert_array_equal(words_host(dC), oracle.to_packed(e, oracle.matmul(e, f, A, B)))


# ---------------------------------------------------------------- larger products


@pytest.mark.parametrize("e,m,n,k", [(4, 4096, 4096, 4096), (2, 512, 512, 512), (8, 1024, 1024, 1024)])
def test_newton_john_full_size_against_tensor_form(ctx, e, m, n, k):
    """The Newton-John product equals the tcgen05 product bit for bit, sampled
    rows equal the oracle, and the whole product passes Freivalds' test against
    the oracle with 8 random columns (a wrong product passes with probability
    at most 2^-(8e))."""
    f = workloads.FIELD_POLY[e]
    A, B, _ = workloads.random_problem(e, m, n, k, seed=e + m)
    dA, dB = dev(A), dev(B)
    ctx.set_form("newton_john")
    C1 = ctx.mul(e, f, dA, dB)
    ctx.set_form("tc_f4")
    C2 = ctx.mul(e, f, dA, dB)
    ctx.set_form("auto")
    assert torch.equal(C1, C2)
    rows = np.random.default_rng(1).choice(m, size=8, replace=False)
    got = C1.cpu().numpy()
    np.testing.assert_array_equal(got[rows], oracle.matmul(e, f, A[rows], B))
    assert oracle.freivalds(e, f, A, B, got, trials=8, seed=m + k), "Freivalds' test failed"
    assert ctx.device_status() == m4.OK


def test_newton_john_batched_one_by_one(ctx):
    probs, want, keep = [], [], []
    rng = np.random.default_rng(77)
    for j in range(12):
        e = int(rng.integers(2, 11))
        f = workloads.FIELD_POLY[e]
        m, n, k = (int(x) for x in rng.integers(1, 300, size=3))
        A, B, C = workloads.random_problem(e, m, n, k, seed=j, with_c=True)
        acc = bool(j % 2)
        dA, dB, dC = dev(A), dev(B), dev(C)
        keep += [dA, dB, dC]
        probs.append((e, f, dA, dB, dC, acc))
        want.append(oracle.addmul(e, f, A, B, C) if acc else oracle.matmul(e, f, A, B))
    ctx.set_form("newton_john")
    try:
        ctx.mul_batched(probs)
        torch.cuda.synchronize()
    finally:
        ctx.set_form("auto")
    for p, w in zip(probs, want):
        np.testing.assert_array_equal(p[4].cpu().numpy(), w)
    assert ctx.device_status() == m4.OK
