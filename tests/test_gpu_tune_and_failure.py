"""Autotuner and failure detection on the GPU.

The failure test makes the bounded waits of the persistent tcgen05 kernel
run out (a wait limit of zero) instead of faulting anything: the kernel must
report M4RIE_ERR_TIMEOUT through the device status word, stop, free its tensor
memory and return, and the context must then compute correct products again.
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_autotuner_picks_a_correct_candidate_and_auto_uses_it(tmp_path):
    e, f = 4, workloads.FIELD_POLY[4]
    m = n = k = 512
    ctx = m4.Context()
    form, sched, ms = ctx.tune(e, f, m, n, k)
    assert form in ("popc", "tc_f8", "tc_f4", "newton_john") and sched in ("alpha_b", "karatsuba") and ms > 0
    assert ctx.resolve_form(e, m, n, k) == m4.FORMS[form]
    A, B, _ = workloads.random_problem(e, m, n, k, seed=31)
    C = ctx.mul(e, f, dev(A), dev(B))          # AUTO
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.matmul(e, f, A, B))
    path = str(tmp_path / "tune.txt")
    ctx.tune_save(path)
    with open(path, "a") as fh:
        fh.write("garbage line\n4 3 99 1 0 1.0\n")   # ignored: not a valid entry
    other = m4.Context()
    assert other.tuned_choice(e, m, n, k)[0] is None
    other.tune_load(path)
    assert other.tuned_choice(e, m, n, k)[:2] == (form, sched)
    other.close()
    os.environ["M4RIE_TUNE_CACHE"] = path
    try:
        third = m4.Context()
        assert third.tuned_choice(e, m, n, k)[:2] == (form, sched)
        third.close()
    finally:
        del os.environ["M4RIE_TUNE_CACHE"]
    ctx.close()


@pytest.mark.parametrize("form", ["tc_f8", "tc_f4"])
def test_bounded_wait_timeout_is_reported_and_context_recovers(form):
    e, f = 8, workloads.FIELD_POLY[8]
    A, B, _ = workloads.random_problem(e, 1024, 1024, 4096, seed=8)
    dA, dB = dev(A), dev(B)
    ctx = m4.Context()
    ctx.set_form(form)
    ctx.set_schedule("alpha_b")
    ctx.set_test_hook(1)                       # the epilogue waits on a barrier nothing signals
    ctx.set_wait_limit_ns(200_000_000)         # 0.2 s
    ctx.mul(e, f, dA, dB)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.ERR_TIMEOUT
    ctx.set_test_hook(0)
    ctx.set_wait_limit_ns(4_000_000_000)
    C = ctx.mul(e, f, dA, dB)
    torch.cuda.synchronize()
    assert ctx.device_status() == m4.OK
    rows = slice(0, 8)
    np.testing.assert_array_equal(C.cpu().numpy()[rows], oracle.matmul(e, f, A[rows], B))
    with pytest.raises(m4.M4rieError):
        ctx.set_test_hook(2)
    ctx.close()
