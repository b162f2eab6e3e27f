"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Every comparison is bit-exact (field arithmetic has one correct result).
Small and ragged shapes are compared in full; the full-size workloads are
compared on sampled row panels that the oracle computes directly plus a
Freivalds check of the whole product.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1111_6900_gb300 as m4  # noqa: E402

FORMS = ["popc", "tc_f8", "tc_f4", "mma_s8", "mma_b1"]
# (form, schedule) pairs the library implements; the INT8 mma.sync form runs
# the alpha^j-B schedule only
FORM_SCHEDS = [(f, s) for f in FORMS for s in ("alpha_b", "karatsuba") if not (f.startswith("mma_") and s == "karatsuba")]


@pytest.fixture(scope="module")
def ctx():
    c = m4.Context()
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def run(ctx, form, sched, e, A, B, C0=None):
    ctx.set_form(form)
    ctx.set_schedule(sched)
    f = workloads.FIELD_POLY[e]
    dA, dB = dev(A), dev(B)
    if C0 is None:
        C = ctx.mul(e, f, dA, dB)
    else:
        C = dev(C0)
        ctx.addmul(e, f, dA, dB, C)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    return host(C)


# ---------------------------------------------------------------- slicing


def test_pack_figure1(ctx):
    e = 3
    X = np.array([[5, 2], [3, 1]], dtype=np.uint8)
    S = host(ctx.pack(e, dev(X))).view(np.uint64)
    expect = oracle.slice_(e, X)
    np.testing.assert_array_equal(S, expect)
    assert [int(S[i, r, 0]) for i in range(3) for r in range(2)] == [0b01, 0b11, 0b10, 0b01, 0b01, 0b00]
    np.testing.assert_array_equal(host(ctx.unpack(e, ctx.pack(e, dev(X)), 2)), X)


@pytest.mark.parametrize("e", [2, 4, 8, 9, 10])
@pytest.mark.parametrize("shape", [(1, 1), (7, 131), (64, 64), (33, 200)])
def test_pack_unpack_random(ctx, e, shape):
    rng = np.random.default_rng(e * 100 + shape[1])
    X = workloads.elements(rng, e, shape)
    ldw = (shape[1] + 63) // 64 + 1
    S = ctx.pack(e, dev(X), ld_words=ldw)
    np.testing.assert_array_equal(host(S).view(np.uint64), oracle.slice_(e, X, ld_words=ldw))
    np.testing.assert_array_equal(host(ctx.unpack(e, S, shape[1])), X)


# ---------------------------------------------------------------- products


@pytest.mark.parametrize("e", sorted(workloads.FIELD_POLY))
@pytest.mark.parametrize("form,sched", FORM_SCHEDS)
def test_mul_ragged_every_field(ctx, e, form, sched):
    """Several tiles in every direction plus a ragged tail."""
    f = workloads.FIELD_POLY[e]
    for (m, n, k) in [(33, 65, 129), (130, 300, 257)]:
        A, B, _ = workloads.random_problem(e, m, n, k, seed=e * 1000 + m)
        np.testing.assert_array_equal(run(ctx, form, sched, e, A, B), oracle.matmul(e, f, A, B),
                                      err_msg=f"{form} {sched} e={e} {m}x{k}x{n}")


@pytest.mark.parametrize("e", [2, 5, 8, 10])
@pytest.mark.parametrize("form,sched", FORM_SCHEDS)
def test_addmul(ctx, e, form, sched):
    f = workloads.FIELD_POLY[e]
    A, B, C0 = workloads.random_problem(e, 150, 97, 333, seed=77 + e, with_c=True)
    np.testing.assert_array_equal(run(ctx, form, sched, e, A, B, C0), oracle.addmul(e, f, A, B, C0))


@pytest.mark.parametrize("form,sched", FORM_SCHEDS)
def test_degenerate_shapes(ctx, form, sched):
    e, f = 4, workloads.FIELD_POLY[4]
    for (m, n, k) in [(1, 1, 1), (1, 300, 1), (300, 1, 1), (1, 1, 5000), (2, 3, 4096)]:
        A, B, _ = workloads.random_problem(e, m, n, k, seed=m + n + k)
        np.testing.assert_array_equal(run(ctx, form, sched, e, A, B), oracle.matmul(e, f, A, B))
    # k = 0: mul writes zeros, addmul leaves C unchanged; m = 0 / n = 0 are no-ops
    ctx.set_form(form)
    ctx.set_schedule(sched)
    A = torch.empty((5, 0), dtype=torch.uint8, device="cuda")
    B = torch.empty((0, 7), dtype=torch.uint8, device="cuda")
    C = torch.full((5, 7), 9, dtype=torch.uint8, device="cuda")
    ctx.mul(e, f, A, B, C)
    assert int(C.max()) == 0
    C.fill_(9)
    ctx.addmul(e, f, A, B, C)
    assert int(C.min()) == 9
    ctx.mul(e, f, torch.empty((0, 3), dtype=torch.uint8, device="cuda"), torch.ones((3, 4), dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK


@pytest.mark.parametrize("form", FORMS)
def test_out_of_range_entries_flagged_and_masked(ctx, form):
    e, f = 3, workloads.FIELD_POLY[3]
    A, B, _ = workloads.random_problem(e, 40, 30, 50, seed=5)
    A2 = A.copy()
    A2[3, 7] |= 0x80           # entry >= 2^e
    ctx.set_form(form)
    ctx.set_schedule("alpha_b")
    C = ctx.mul(e, f, dev(A2), dev(B))
    assert ctx.device_status() == m4.ERR_RANGE
    assert ctx.device_status() == m4.OK   # status is cleared once read
    np.testing.assert_array_equal(host(C), oracle.matmul(e, f, A, B))


@pytest.mark.parametrize("form", ["mma_s8", "mma_b1"])
def test_legacy_mma_forms_have_no_karatsuba_schedule(ctx, form):
    e, f = 4, workloads.FIELD_POLY[4]
    ctx.set_form(form)
    ctx.set_schedule("karatsuba")
    A = dev(np.ones((8, 8), np.uint8))
    with pytest.raises(m4.M4rieError) as ei:
        ctx.mul(e, f, A, A)
    assert ei.value.status == m4.ERR_UNSUPPORTED


def test_invalid_arguments_launch_nothing(ctx):
    e, f = 4, workloads.FIELD_POLY[4]
    A = dev(np.zeros((8, 8), np.uint8))
    before = ctx.kernel_launches()
    with pytest.raises(m4.M4rieError) as ei:
        ctx.mul(e, 0x11, A, A)        # reducible f
    assert ei.value.status == m4.ERR_POLY
    with pytest.raises(m4.M4rieError) as ei:
        ctx.mul(e, f, A, A, A)        # C aliases A
    assert ei.value.status == m4.ERR_ALIAS
    assert ctx.kernel_launches() == before


def test_host_buffer_entry_point(ctx):
    e, f = 5, workloads.FIELD_POLY[5]
    A, B, C0 = workloads.random_problem(e, 70, 90, 110, seed=3, with_c=True)
    for form in FORMS:
        ctx.set_form(form)
        ctx.set_schedule("alpha_b")
        C = np.zeros((70, 90), np.uint8)
        ctx.mul_host(e, f, A, B, C)
        np.testing.assert_array_equal(C, oracle.matmul(e, f, A, B))
        C = C0.copy()
        ctx.mul_host(e, f, A, B, C, accumulate=True)
        np.testing.assert_array_equal(C, oracle.addmul(e, f, A, B, C0))


def test_batched_matches_individual(ctx):
    ctx.set_form("auto")
    ctx.set_schedule("auto")
    probs, expect = [], []
    for j in range(12):
        e, f, m, n, k, A, B = workloads.batched_instance(j)
        m, n, k = max(1, m // 8), max(1, n // 8), max(1, k // 8)
        A, B = A[:m, :k].copy(), B[:k, :n].copy()
        C = torch.zeros((m, n), dtype=m4.elem_dtype_torch(e), device="cuda")
        probs.append((e, f, dev(A), dev(B), C, False))
        expect.append(oracle.matmul(e, f, A, B))
    ctx.mul_batched(probs)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    for (e, f, A, B, C, _), ex in zip(probs, expect):
        np.testing.assert_array_equal(host(C), ex)


# ---------------------------------------------------------------- full-size workloads

_panel_cache = {}


def _workload_panel(idx, rows):
    """Inputs of a workload and the oracle's product on a row panel."""
    key = (idx, rows.start, rows.stop)
    if key not in _panel_cache:
        w = workloads.WORKLOADS[idx]
        A, B, C0 = w.inputs()
        Ap = A[rows]
        ref = oracle.addmul(w.e, w.f, Ap, B, C0[rows]) if C0 is not None else oracle.matmul(w.e, w.f, Ap, B)
        _panel_cache[key] = (w, A, B, C0, ref)
    return _panel_cache[key]


def test_workload1_full(ctx):
    w = workloads.WORKLOADS[1]
    A, B, _ = w.inputs()
    ref = oracle.matmul(w.e, w.f, A, B)
    for form, sched in FORM_SCHEDS:
        np.testing.assert_array_equal(run(ctx, form, sched, w.e, A, B), ref, err_msg=f"{form} {sched}")


@pytest.mark.parametrize("idx", [2, 3, 5])
@pytest.mark.parametrize("form,sched", FORM_SCHEDS)
def test_full_size_workloads(ctx, idx, form, sched):
    w = workloads.WORKLOADS[idx]
    rows = slice(w.m // 2 - 8, w.m // 2 + 8)
    w, A, B, C0, ref = _workload_panel(idx, rows)
    C = run(ctx, form, sched, w.e, A, B, C0)
    np.testing.assert_array_equal(C[rows], ref)                 # sampled rows, exact
    np.testing.assert_array_equal(C[:4], (oracle.addmul(w.e, w.f, A[:4], B, C0[:4]) if C0 is not None
                                          else oracle.matmul(w.e, w.f, A[:4], B)))   # first rows (first tile)
    lhs = C if C0 is None else (C ^ C0)
    assert oracle.freivalds(w.e, w.f, A, B, lhs, trials=4, seed=idx)   # whole product, error <= 2^(-4e)


# ---------------------------------------------------------------- recombination in the epilogue


@pytest.mark.parametrize("form", ["tc_f8", "tc_f4"])
@pytest.mark.parametrize("e,m,n,k,add", [(2, 512, 700, 300, False), (4, 1024, 513, 257, True),
                                         (8, 768, 1100, 96, True), (5, 2048, 448, 640, False),
                                         (3, 2100, 333, 129, True)])
def test_karatsuba_recombined_in_the_epilogue(form, e, m, n, k, add, monkeypatch):
    """M4RIE_FUSE_RECOMBINE=1: the 2-SM tcgen05 GEMM runs every product of an
    output tile back to back and recombines them in its epilogue (no parity
    planes; m is a multiple of 256 or at least 2048, so the products run on
    2-SM pairs); the result must be the oracle's, ragged edges and
    accumulation included."""
    monkeypatch.setenv("M4RIE_FUSE_RECOMBINE", "1")
    c = m4.Context()
    try:
        c.set_form(form)
        c.set_schedule("karatsuba")
        f = workloads.FIELD_POLY[e]
        A, B, C0 = workloads.random_problem(e, m, n, k, seed=e * 100 + m, with_c=True)
        if add:
            C = dev(C0)
            c.addmul(e, f, dev(A), dev(B), C)
            want = oracle.addmul(e, f, A, B, C0)
        else:
            C = c.mul(e, f, dev(A), dev(B))
            want = oracle.matmul(e, f, A, B)
        torch.cuda.synchronize()
        assert c.device_status() == m4.OK
        np.testing.assert_array_equal(host(C), want)
    finally:
        c.close()


@pytest.mark.parametrize("form,sched", [("popc", "alpha_b"), ("tc_f4", "karatsuba"), ("tc_f8", "alpha_b"),
                                        ("newton_john", "alpha_b"), ("mma_s8", "alpha_b")])
def test_host_buffers_in_place_when_pinned(form, sched, monkeypatch):
    """M4RIE_ZERO_COPY=1: with pinned (device-mapped) host buffers the kernels
    read A, B and write C in host memory directly; pageable buffers still go
    through staging copies.  Both must give the oracle's result."""
    monkeypatch.setenv("M4RIE_ZERO_COPY", "1")
    c = m4.Context()
    try:
        c.set_form(form)
        c.set_schedule(sched)
        for e, (m, n, k) in [(4, (600, 520, 300)), (9, (130, 70, 257))]:
            f = workloads.FIELD_POLY[e]
            A, B, C0 = workloads.random_problem(e, m, n, k, seed=e + m, with_c=True)
            hA = torch.from_numpy(A).pin_memory()
            hB = torch.from_numpy(B).pin_memory()
            hC = torch.zeros((m, n), dtype=hA.dtype).pin_memory()
            c.mul_host(e, f, hA, hB, hC)
            np.testing.assert_array_equal(hC.numpy(), oracle.matmul(e, f, A, B))
            hC.copy_(torch.from_numpy(C0))
            c.mul_host(e, f, hA, hB, hC, accumulate=True)
            np.testing.assert_array_equal(hC.numpy(), oracle.addmul(e, f, A, B, C0))
            Cp = C0.copy()  # pageable: the staging path
            c.mul_host(e, f, A, B, Cp, accumulate=True)
            np.testing.assert_array_equal(Cp, oracle.addmul(e, f, A, B, C0))
        assert c.device_status() == m4.OK
    finally:
        c.close()


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("accumulate", [False, True])
def test_host_buffers_pipelined_row_panels(pinned, accumulate):
    """A host-buffer product of more than 32 MiB runs in four row panels whose
    copies overlap the other panels' products (B sliced once, reused).  The
    result equals the device-buffer product and, on rows sampled from every
    panel (including the ragged last one), the oracle."""
    e, f = 4, workloads.FIELD_POLY[4]
    m, n, k = 2148, 4096, 4096
    A, B, C0 = workloads.random_problem(e, m, n, k, seed=77, with_c=True)
    c = m4.Context()
    try:
        dC = dev(C0)
        if accumulate:
            c.addmul(e, f, dev(A), dev(B), dC)
        else:
            c.mul(e, f, dev(A), dev(B), dC)
        if pinned:
            hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
            hC = torch.from_numpy(C0.copy()).pin_memory()
            c.mul_host(e, f, hA, hB, hC, accumulate=accumulate)
            got = hC.numpy()
        else:
            got = C0.copy()
            c.mul_host(e, f, A, B, got, accumulate=accumulate)
        np.testing.assert_array_equal(got, host(dC))
        rows = np.array([0, 1, 600, 639, 640, 641, 1279, 1280, 1919, 1920, 2100, 2147])
        want = oracle.addmul(e, f, A[rows], B, C0[rows]) if accumulate else oracle.matmul(e, f, A[rows], B)
        np.testing.assert_array_equal(got[rows], want)
        assert c.device_status() == m4.OK
    finally:
        c.close()


@pytest.mark.parametrize("form", ["tc_f4", "tc_f8"])
@pytest.mark.parametrize("sched", ["alpha_b", "karatsuba"])
def test_counts_at_the_chunk_limit(ctx, form, sched):
    """Every entry of A and B has all its slice bits set, so the GF(2) counts
    reach the largest value an accumulation chunk allows (the tensor forms
    accumulate integer counts in FP32 on top of 2^23 and keep bit 0; a count
    that lost a low bit would flip an output bit).  k spans several chunks."""
    for e in (2, 4, 8):
        f = workloads.FIELD_POLY[e]
        m, n, k = 130, 70, 20000
        A = np.full((m, k), (1 << e) - 1, dtype=np.uint8)
        B = np.full((k, n), (1 << e) - 1, dtype=np.uint8)
        B[::3] = 1
        ctx.set_form(form)
        ctx.set_schedule(sched)
        got = ctx.mul(e, f, dev(A), dev(B)).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.matmul(e, f, A, B), err_msg=f"e={e}")
    ctx.set_form("auto")
    ctx.set_schedule("auto")
    assert ctx.device_status() == m4.OK
