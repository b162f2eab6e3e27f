"""m4rie_mul_noalloc: the entry point for callers that may not allocate device
memory (their own allocator owns the GPU's memory, their footprint must be
fixed at load time, or cudaMalloc's possible device synchronisation is not
acceptable on their path).  It keeps its operand planes in a static device
array instead of a context workspace.

Its results must equal those of the existing entry points (bit-exact, as all
products here), on two calls in a row, since the calls share that array and
the second call finds the first call's planes still in it.  This file is
collected last so that a run stopping at the first failure has run every
other test.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1111_6900_gb300 as m4  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_noalloc_equals_existing_entry_point_twice():
    ctx = m4.Context()
    ctx.set_form("popc")
    ctx.set_schedule("alpha_b")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # two consecutive calls with different fields and shapes (the second, smaller
    # one runs over the planes left behind by the first), then an accumulate call
    cases = [(4, 300, 257, 520, False), (9, 70, 45, 130, False), (8, 129, 200, 64, True)]
    for e, m, n, k, acc in cases:
        f = workloads.FIELD_POLY[e]
        A, B, C0 = workloads.random_problem(e, m, n, k, seed=900 + e, with_c=True)
        dA, dB = _dev(A), _dev(B)
        ref = _dev(C0)
        if acc:
            ctx.addmul(e, f, dA, dB, ref)
        else:
            ctx.mul(e, f, dA, dB, ref)
        got = _dev(C0)
        assert m4.mul_noalloc(e, f, dA, dB, got, accumulate=acc, device_status=status) == m4.OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy(), err_msg=f"e={e} {m}x{k}x{n}")
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    e, f = 10, workloads.FIELD_POLY[10]
    A = torch.zeros((4096, 4096), dtype=torch.uint16, device="cuda")
    B = torch.zeros((4096, 4096), dtype=torch.uint16, device="cuda")
    C = torch.zeros((4096, 4096), dtype=torch.uint16, device="cuda")
    assert m4.mul_noalloc(e, f, A, B, C) == m4.ERR_SCRATCH
    assert m4.mul_noalloc(e, 0x401, A[:8, :8], B[:8, :8], C[:8, :8]) == m4.ERR_POLY
