"""m4rie_mul_noalloc: the entry point for callers that may not allocate device
memory (their own allocator owns the GPU's memory, their footprint must be
fixed at load time, or cudaMalloc's possible device synchronisation is not
acceptable on their path).  It keeps its operand planes in a static device
array instead of a context workspace.

Its results must equal those of the existing entry points and of the CPU
oracle (bit-exact, as all products here), on two calls in a row, since the
calls share that array and the second call finds the first call's planes
still in it.  This file is
collected last so that a run stopping at the first failure has run every
other test.
"""
import numpy as np
import pytest

import oracle
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
        expect = oracle.addmul(e, f, A, B, C0) if acc else oracle.matmul(e, f, A, B)
        np.testing.assert_array_equal(got.cpu().numpy(), expect, err_msg=f"oracle, e={e} {m}x{k}x{n}")
    assert ctx.device_status() == m4.OK
    ctx.close()


def test_noalloc_without_a_status_tensor():
    """device_status=None: the status bits go to a word of the scratch array
    that nothing reads; the product itself is unchanged (twice in a row)."""
    for e, m, n, k in ((4, 200, 131, 300), (2, 64, 520, 129)):
        f = workloads.FIELD_POLY[e]
        A, B, _ = workloads.random_problem(e, m, n, k, seed=950 + e)
        dA, dB = _dev(A), _dev(B)
        got = torch.empty((m, n), dtype=dA.dtype, device="cuda")
        assert m4.mul_noalloc(e, f, dA, dB, got) == m4.OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.matmul(e, f, A, B), err_msg=f"e={e}")


def test_noalloc_rejects_problems_beyond_its_scratch():
    e, f = 10, workloads.FIELD_POLY[10]
    A = torch.zeros((4096, 4096), dtype=torch.uint16, device="cuda")
    B = torch.zeros((4096, 4096), dtype=torch.uint16, device="cuda")
    C = torch.zeros((4096, 4096), dtype=torch.uint16, device="cuda")
    assert m4.mul_noalloc(e, f, A, B, C) == m4.ERR_SCRATCH
    a8, b8, c8 = A[:8, :8].contiguous(), B[:8, :8].contiguous(), C[:8, :8].contiguous()
    assert m4.mul_noalloc(e, 0x401, a8, b8, c8) == m4.ERR_POLY
    with pytest.raises(ValueError):
        m4.mul_noalloc(e, f, a8, b8, c8, device_status=torch.zeros(0, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        m4.mul_noalloc(e, f, A[:8, :8], b8, c8)   # a strided view
