"""Batched products (one persistent launch replayed from a CUDA graph) against
the oracle, including the full 4096-instance workload on sampled rows."""
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


def _problems(specs, seed0):
    probs, ref = [], []
    for j, (e, m, n, k, acc) in enumerate(specs):
        f = workloads.FIELD_POLY[e]
        A, B, C0 = workloads.random_problem(e, m, n, k, seed=seed0 + j, with_c=True)
        C = dev(C0)
        probs.append((e, f, dev(A), dev(B), C, acc))
        ref.append(oracle.addmul(e, f, A, B, C0) if acc else oracle.matmul(e, f, A, B))
    return probs, ref


SPECS = [(2, 33, 65, 129, False), (3, 130, 70, 300, True), (4, 1, 1, 1, False), (5, 200, 257, 64, False),
         (6, 64, 64, 64, True), (7, 17, 300, 90, False), (8, 129, 31, 1000, False), (9, 40, 50, 60, False),
         (10, 70, 33, 130, True), (4, 0, 5, 5, False), (4, 5, 5, 0, False), (8, 6, 7, 0, True)]


@pytest.mark.parametrize("form", ["auto", "tc_f8", "popc"])
def test_batched_mixed_fields_and_shapes(form):
    ctx = m4.Context()
    ctx.set_form(form)
    probs, ref = _problems(SPECS, 5000)
    ctx.mul_batched(probs)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    for (e, f, A, B, C, acc), r, spec in zip(probs, ref, SPECS):
        np.testing.assert_array_equal(C.cpu().numpy(), r, err_msg=str(spec))
    ctx.close()


KARA_SPECS = SPECS + [(5, 300, 20, 520, True), (6, 129, 33, 256, False), (8, 257, 229, 384, True),
                      (7, 64, 448, 130, False), (10, 130, 224, 257, False), (3, 1, 600, 33, True)]


@pytest.mark.parametrize("sched", ["karatsuba", "auto"])
@pytest.mark.parametrize("form", ["tc_f4", "tc_f8"])
def test_batched_karatsuba(monkeypatch, sched, form):
    """Batched products on the Karatsuba-like schedule: r GF(2) products per
    product written as blocked parity planes by the persistent GEMM, then one
    batched recombination; narrow n takes narrower tiles.  Mixed fields,
    ragged and degenerate shapes, accumulation; against the oracle."""
    monkeypatch.setenv("M4RIE_BATCHED_SCHED", sched)
    monkeypatch.setenv("M4RIE_BATCHED_KARA_MIN_MNK", "0")
    ctx = m4.Context()
    ctx.set_form(form)
    probs, ref = _problems(KARA_SPECS, 5100)
    ctx.mul_batched(probs)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    for (e, f, A, B, C, acc), r, spec in zip(probs, ref, KARA_SPECS):
        np.testing.assert_array_equal(C.cpu().numpy(), r, err_msg=str(spec))
    # a replay of the recorded graph gives the same products (accumulating ones again)
    for (e, f, A, B, C, acc), (_, m, n, k, _) in zip(probs, KARA_SPECS):
        if acc:
            C.zero_()
    ctx.mul_batched(probs)
    torch.cuda.synchronize()
    for (e, f, A, B, C, acc), spec in zip(probs, KARA_SPECS):
        want = oracle.matmul(e, workloads.FIELD_POLY[e], A.cpu().numpy(), B.cpu().numpy()) if acc else None
        if acc:
            np.testing.assert_array_equal(C.cpu().numpy(), want, err_msg=str(spec))
    assert ctx.device_status() == m4.OK
    ctx.close()


def _shape_class(m, n, k):
    return min(63, int(np.floor(np.log2(max(1.0, float(m) * n * k)))))


def test_tune_batched_then_mul(tmp_path):
    """m4rie_tune_batched times every (e, shape class) of a batch under both
    schedules on scratch inputs (the batch's tensors stay untouched), keeps
    the faster, and later batches use the choices; the batch's products are
    still equal to the oracle's.  With phase timing on, the replayed graph
    reports its plane, GEMM and recombination phases."""
    ctx = m4.Context()
    specs = [s for s in KARA_SPECS if s[1] and s[2] and s[3]]
    probs, ref = _problems(specs, 5200)
    before = [p[4].clone() for p in probs]
    ctx.tune_batched(probs)
    torch.cuda.synchronize()
    for p, c0 in zip(probs, before):
        assert torch.equal(p[4], c0)
    path = str(tmp_path / "tune.txt")
    ctx.tune_save(path)
    with open(path) as fh:
        lines = [w for w in (l.split() for l in fh) if w and w[0] == "B"]
    tuned = {(int(w[1]), int(w[2])): int(w[4]) for w in lines}
    want = {(e, _shape_class(m, n, k)) for e, m, n, k, _ in specs}
    assert set(tuned) == want
    assert set(tuned.values()) <= {m4.SCHED_ALPHA_B, m4.SCHED_KARATSUBA}
    assert {int(w[5]) for w in lines} <= {1, 2}          # tile width: wide or narrow
    ctx2 = m4.Context()                     # the cache file carries the choices
    ctx2.tune_load(path)
    for c in (ctx, ctx2):
        for p in probs:
            p[4].zero_()
        c.enable_timing(True)
        c.phase_times(reset=True)
        c.mul_batched(probs)
        torch.cuda.synchronize()
        pack_ms, gemm_ms, rec_ms, nprod = c.phase_times(reset=True)
        c.enable_timing(False)
        assert pack_ms > 0 and gemm_ms > 0 and rec_ms >= 0 and nprod == len(specs)
        for (e, f, A, B, C, acc), r, spec in zip(probs, ref, specs):
            want_c = oracle.matmul(e, f, A.cpu().numpy(), B.cpu().numpy()) if acc else r
            np.testing.assert_array_equal(C.cpu().numpy(), want_c, err_msg=str(spec))
        assert c.device_status() == m4.OK
    ctx2.close()
    ctx.close()


@pytest.mark.parametrize("width", [1, 2])
@pytest.mark.parametrize("sched", [1, 2])
def test_batched_tile_widths_from_the_tune_cache(tmp_path, sched, width):
    """Every (schedule, tile width) the tuner can pick, imposed through a tune
    cache, gives the oracle's products (narrow tiles cover few columns)."""
    specs = [(e, m, n, k, acc) for e, m, n, k, acc in KARA_SPECS if m and n and k]
    path = tmp_path / "cache.txt"
    with open(path, "w") as fh:
        for e, m, n, k, _ in specs:
            fh.write(f"B {e} {_shape_class(m, n, k)} {m4.FORM_TC_F4} {sched} {width} 1.0\n")
    ctx = m4.Context()
    ctx.tune_load(str(path))
    probs, ref = _problems(specs, 5300)
    ctx.mul_batched(probs)
    torch.cuda.synchronize()
    for (e, f, A, B, C, acc), r, spec in zip(probs, ref, specs):
        np.testing.assert_array_equal(C.cpu().numpy(), r, err_msg=str(spec))
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_batched_graph_replay_sees_new_inputs():
    ctx = m4.Context()
    specs = [(4, 100, 90, 80, False), (8, 50, 60, 70, False)]
    probs, _ = _problems(specs, 6000)
    ctx.mul_batched(probs)           # records the graph
    launches = ctx.kernel_launches()
    # new input values in the same buffers: the replay must compute them
    refs = []
    for (e, f, A, B, C, acc), (_, m, n, k, _) in zip(probs, specs):
        A2, B2, _ = workloads.random_problem(e, m, n, k, seed=77 + e)
        A.copy_(dev(A2))
        B.copy_(dev(B2))
        refs.append(oracle.matmul(e, f, A2, B2))
    ctx.mul_batched(probs)           # replays
    torch.cuda.synchronize()
    assert ctx.kernel_launches() > launches
    for (e, f, A, B, C, acc), r in zip(probs, refs):
        np.testing.assert_array_equal(C.cpu().numpy(), r)
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_batched_rejects_overlapping_outputs():
    ctx = m4.Context()
    e, f = 4, workloads.FIELD_POLY[4]
    A = dev(np.ones((8, 8), np.uint8))
    C = torch.zeros((16, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(m4.M4rieError) as ei:
        ctx.mul_batched([(e, f, A, A, C[:8], False), (e, f, A, A, C[4:12], False)])
    assert ei.value.status == m4.ERR_ALIAS
    with pytest.raises(m4.M4rieError) as ei:   # an output over another product's input
        ctx.mul_batched([(e, f, A, A, C[:8], False), (e, f, C[:8], A, C[8:], False)])
    assert ei.value.status == m4.ERR_ALIAS
    ctx.close()


def test_batched_workload_4096_instances():
    """The batched workload: 4096 instances, e in 2..8, m, n, k in 32..1024.
    Every instance is checked on its first and last rows against the oracle
    and as a whole by Freivalds' test with 8 random columns (a wrong instance
    passes with probability at most 2^-(8e)); 64 instances are compared with
    the oracle's product element by element."""
    ctx = m4.Context()
    probs, host = [], []
    for j in range(workloads.BATCHED_COUNT):
        e, f, m, n, k, A, B = workloads.batched_instance(j)
        C = torch.empty((m, n), dtype=m4.elem_dtype_torch(e), device="cuda")
        probs.append((e, f, dev(A), dev(B), C, False))
        host.append((A, B))
    ctx.mul_batched(probs)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    rng = np.random.default_rng(4)
    full = set(rng.choice(len(probs), size=64, replace=False).tolist())
    for j, ((e, f, dA, dB, C, _), (A, B)) in enumerate(zip(probs, host)):
        got = C.cpu().numpy()
        rows = [0, A.shape[0] - 1]
        np.testing.assert_array_equal(got[rows], oracle.matmul(e, f, A[rows], B), err_msg=f"instance {j}")
        assert oracle.freivalds(e, f, A, B, got, trials=8, seed=j), f"instance {j}: Freivalds' test failed"
        if j in full:
            np.testing.assert_array_equal(got, oracle.matmul(e, f, A, B), err_msg=f"instance {j}")
    ctx.close()
