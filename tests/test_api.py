"""Host-side tests of the C ABI that need no GPU: the library loads and exports
every declared entry point, argument validation returns the documented
status codes, and the GF(2)-product schedules compute the field product
(checked independently of the library with numpy GF(2) products)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import workloads
from tests import fieldref as fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(m4rie_\w+)\s*\(", text, flags=re.M):
            names.add(mt.group(1))
    return names


def test_library_exports_every_declared_symbol():
    import paper_1111_6900_gb300 as m4
    declared = _declared_functions()
    assert len(declared) >= 19
    lib = ctypes.CDLL(m4.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    import paper_1111_6900_gb300 as m4
    for s in range(9):
        assert m4.status_string(s)
    assert m4.status_string(0) == "ok"


def test_validation_codes():
    import paper_1111_6900_gb300 as m4
    v = m4.validate
    A, B, C = 0x10000, 0x20000, 0x30000
    assert v(4, 0x13, 8, 8, 8, A, B, C) == m4.OK
    assert v(1, 0x3, 8, 8, 8, A, B, C) == m4.ERR_ARG         # e < 2
    assert v(11, 0x805, 8, 8, 8, A, B, C) == m4.ERR_ARG       # e > 10
    assert v(4, 0x11, 8, 8, 8, A, B, C) == m4.ERR_POLY        # x^4 + 1 reducible
    assert v(4, 0x15, 8, 8, 8, A, B, C) == m4.ERR_POLY        # (x^2+x+1)^2
    assert v(4, 0x25, 8, 8, 8, A, B, C) == m4.ERR_POLY        # degree 5
    assert v(8, 0x11B, 8, 8, 8, A, B, C) == m4.OK             # irreducible, not primitive
    assert v(4, 0x13, -1, 8, 8, A, B, C) == m4.ERR_ARG
    assert v(4, 0x13, 8, 8, 8, None, B, C) == m4.ERR_ARG
    assert v(4, 0x13, 0, 8, 0, None, None, None) == m4.OK     # nothing to point to
    assert v(4, 0x13, 8, 8, 0, None, None, C) == m4.OK        # k = 0: only C needed
    assert v(4, 0x13, 16, 16, 16, A, B, A + 100) == m4.ERR_ALIAS
    assert v(4, 0x13, 16, 16, 16, A, B, B - 10) == m4.ERR_ALIAS
    assert v(4, 0x13, 16, 16, 16, A, B, A + 256) == m4.OK     # adjacent, no overlap
    assert v(10, 0x409, 16, 16, 16, A, B, A + 256) == m4.ERR_ALIAS  # 2-byte elements overlap


def test_every_configured_polynomial_accepted():
    import paper_1111_6900_gb300 as m4
    for e, f in workloads.FIELD_POLY.items():
        assert m4.validate(e, f, 4, 4, 4, 0x1000, 0x2000, 0x3000) == m4.OK


@pytest.mark.parametrize("e", sorted(workloads.FIELD_POLY))
@pytest.mark.parametrize("sched", ["alpha_b", "karatsuba"])
def test_schedule_is_the_field_product(e, sched):
    """Symbolic check on basis pairs (x^i, x^j), independent of the library:
    the schedule's output must be x^(i+j) mod f."""
    import paper_1111_6900_gb300 as m4
    f = workloads.FIELD_POLY[e]
    am, bm, om = m4.schedule_masks(e, f, sched)
    r = len(am)
    for i in range(e):
        for j in range(e):
            out = 0
            for p in range(r):
                if am[p] >> i & 1 and bm[p] >> j & 1:
                    if sched == "alpha_b":      # product p = i*e + j feeds slice p // e
                        out ^= 1 << (p // e)
                        continue
                    for s in range(e):
                        if om[s] >> p & 1:
                            out ^= 1 << s
            assert out == fr.x_power_mod(e, f, i + j), (i, j)


@pytest.mark.parametrize("e", [2, 3, 5, 6, 7, 8, 9, 10])
def test_karatsuba_schedule_on_matrices(e):
    """Run the Karatsuba schedule with numpy GF(2) products and compare with
    the oracle: the same recombination the GPU epilogue performs."""
    import oracle
    import paper_1111_6900_gb300 as m4
    f = workloads.FIELD_POLY[e]
    am, bm, om = m4.schedule_masks(e, f, "karatsuba")
    A, B, _ = workloads.random_problem(e, 21, 17, 29, seed=40 + e)

    def lin(M, mask):
        out = np.zeros(M.shape, dtype=np.int64)
        for i in range(e):
            if mask >> i & 1:
                out ^= fr.bits(M, i)
        return out
    P = [fr.gf2_matmul(lin(A, am[p]), lin(B, bm[p])) for p in range(len(am))]
    C = np.zeros((21, 17), dtype=np.int64)
    for s in range(e):
        acc = np.zeros_like(C)
        for p in range(len(am)):
            if om[s] >> p & 1:
                acc ^= P[p]
        C |= acc << s
    np.testing.assert_array_equal(C, oracle.matmul(e, f, A, B).astype(np.int64))


def test_product_counts():
    """alpha_b uses the schoolbook count e^2 (Table 3 'naive'); the
    Karatsuba-like schedules use fewer: Table 3's best-known polynomial counts
    for every e <= 8, or below them (the field product modulo f needs only 15
    and 24 products for e = 6 and 8, through GF(4))."""
    import paper_1111_6900_gb300 as m4
    with open(os.path.join(ROOT, "tests", "golden", "table3_counts.txt")) as fh:
        rows = [l.split("#")[0].split() for l in fh]
    table = {int(r[0]): (int(r[1]), int(r[2])) for r in rows if r}
    got = {}
    for e, f in workloads.FIELD_POLY.items():
        assert m4.schedule_products(e, f, "alpha_b") == e * e
        got[e] = m4.schedule_products(e, f, "karatsuba")
        assert got[e] < e * e
    for e, (naive, best) in table.items():
        assert naive == e * e
        assert got[e] <= best, (e, got[e], best)
    assert got == {2: 3, 3: 6, 4: 9, 5: 13, 6: 15, 7: 22, 8: 24, 9: 30, 10: 33}


# irreducible polynomials other than the workloads' (some not primitive)
OTHER_POLY = {5: [0x2F, 0x3D], 6: [0x5B, 0x49], 7: [0x89, 0xF7], 8: [0x11B, 0x187], 9: [0x221, 0x203],
              10: [0x481, 0x46F]}


@pytest.mark.parametrize("e", sorted(OTHER_POLY))
def test_table_formulas_carried_to_other_polynomials(e):
    """The searched formulas are written for one polynomial per e; for any
    other irreducible f the library carries them over by a field isomorphism.
    Checked here on every basis pair, with x^(i+j) mod f computed by the test,
    and with the same number of products as for the workload polynomial."""
    import paper_1111_6900_gb300 as m4
    r0 = m4.schedule_products(e, workloads.FIELD_POLY[e], "karatsuba")
    for f in OTHER_POLY[e]:
        assert fr.is_irreducible(f) and fr.poly_deg(f) == e, hex(f)
        am, bm, om = m4.schedule_masks(e, f, "karatsuba")
        assert len(am) == r0
        for i in range(e):
            for j in range(e):
                out = 0
                for p in range(len(am)):
                    if am[p] >> i & 1 and bm[p] >> j & 1:
                        for s in range(e):
                            if om[s] >> p & 1:
                                out ^= 1 << s
                assert out == fr.x_power_mod(e, f, i + j), (hex(f), i, j)


def test_host_matrix_checks():
    """The host-buffer entry point's argument check (no GPU needed): row-major
    integer matrices of the field's element width, of the stated shape."""
    import numpy as np
    import torch
    import paper_1111_6900_gb300 as m4
    a8 = np.zeros((3, 5), np.uint8)
    a16 = np.zeros((3, 5), np.uint16)
    assert m4._host_matrix(a8, 4, "A", (3, 5)).value == a8.ctypes.data
    assert m4._host_matrix(a16, 10, "A", (3, 5)).value == a16.ctypes.data
    t = torch.zeros((3, 5), dtype=torch.uint8)
    assert m4._host_matrix(t, 8, "A", (3, 5)).value == t.data_ptr()
    assert m4._host_matrix(np.zeros((0, 5), np.uint8), 4, "A", (0, 5)) is None
    with pytest.raises(TypeError):
        m4._host_matrix(a8, 10, "A", (3, 5))            # e > 8 stores two bytes per element
    with pytest.raises(TypeError):
        m4._host_matrix(a16, 4, "A", (3, 5))
    with pytest.raises(TypeError):
        m4._host_matrix(np.zeros((3, 5), np.float32), 4, "A", (3, 5))
    with pytest.raises(TypeError):
        m4._host_matrix([[0] * 5] * 3, 4, "A", (3, 5))   # a list would be a temporary copy
    with pytest.raises(ValueError):
        m4._host_matrix(np.zeros((3, 10), np.uint8)[:, ::2], 4, "A", (3, 5))
    with pytest.raises(ValueError):
        m4._host_matrix(a8, 4, "A", (5, 3))
    ro = np.zeros((3, 5), np.uint8)
    ro.flags.writeable = False
    assert m4._host_matrix(ro, 4, "A", (3, 5)) is not None
    with pytest.raises(ValueError):
        m4._host_matrix(ro, 4, "C", (3, 5), writable=True)


def test_mul_host_marshalling_reaches_the_library():
    """mul_host's whole Python path on the CPU: the arguments reach the C entry
    point, which rejects a null context before any CUDA call; a bad host array
    is refused before the call."""
    import numpy as np
    import paper_1111_6900_gb300 as m4

    class NoContext:
        handle = None
        seen = []

        def _raise(self, status, where):
            self.seen.append((status, where))

    A, B, C = np.zeros((4, 3), np.uint8), np.zeros((3, 5), np.uint8), np.zeros((4, 5), np.uint8)
    nc = NoContext()
    assert m4.Context.mul_host(nc, 4, 0x13, A, B, C) is C
    assert nc.seen == [(m4.ERR_ARG, "m4rie_mul_host")]
    with pytest.raises(ValueError):
        m4.Context.mul_host(nc, 4, 0x13, A, B, np.zeros((5, 4), np.uint8))
    assert len(nc.seen) == 1


def test_binding_shape_checks(monkeypatch):
    """The binding refuses mismatched shapes before the library could write past
    a buffer; matching shapes reach the C entry points (which reject the null
    context used here before any CUDA call).  The device checks are stubbed so
    that CPU tensors can stand in."""
    import torch
    import paper_1111_6900_gb300 as m4

    for name in ("_check_dev", "_check_words", "_check_word_window"):
        monkeypatch.setattr(m4, name, lambda *a, **k: None)

    class NoContext:
        handle = None

        def __init__(self):
            self.seen = []

        def _raise(self, status, where):
            self.seen.append((status, where))

    u8 = lambda *shape: torch.zeros(shape, dtype=torch.uint8)     # noqa: E731
    w64 = lambda *shape: torch.zeros(shape, dtype=torch.int64)    # noqa: E731
    nc = NoContext()
    Ctx = m4.Context
    # mul / addmul
    Ctx.mul(nc, 4, 0x13, u8(4, 3), u8(3, 5), u8(4, 5))
    Ctx.addmul(nc, 4, 0x13, u8(4, 3), u8(3, 5), u8(4, 5))
    assert [w for _, w in nc.seen] == ["m4rie_mul", "m4rie_addmul"]
    assert all(st == m4.ERR_ARG for st, _ in nc.seen)
    for bad in (lambda: Ctx.mul(nc, 4, 0x13, u8(4, 3), u8(2, 5)),
                lambda: Ctx.mul(nc, 4, 0x13, u8(4, 3), u8(3, 5), u8(5, 4)),
                lambda: Ctx.addmul(nc, 4, 0x13, u8(4, 3), u8(2, 5), u8(4, 5)),
                lambda: Ctx.addmul(nc, 4, 0x13, u8(4, 3), u8(3, 5), u8(4, 6)),
                lambda: Ctx.mul_batched(nc, [(4, 0x13, u8(4, 3), u8(3, 5), u8(4, 4), False)]),
                lambda: Ctx.unpack(nc, 4, w64(3, 2, 1), 10),                       # 3 slices for e = 4
                lambda: Ctx.from_packed(nc, 4, w64(2, 1), 10, out=u8(2, 11)),
                lambda: Ctx.mul_packed(nc, 4, 0x13, w64(5, 2), w64(40, 3), w64(5, 3), n=40, k=40),  # A: 3 words
                lambda: Ctx.mul_packed(nc, 4, 0x13, w64(5, 3), w64(40, 2), w64(5, 3), n=40, k=40),  # B: 3 words
                lambda: Ctx.mul_packed(nc, 11, 0x13, w64(5, 3), w64(40, 3), w64(5, 3), n=40, k=40)):
        with pytest.raises(ValueError):
            bad()
    assert len(nc.seen) == 2
    # matching shapes reach the library
    Ctx.mul_batched(nc, [(4, 0x13, u8(4, 3), u8(3, 5), u8(4, 5), False)])
    Ctx.unpack(nc, 4, w64(4, 2, 1), 10)
    Ctx.from_packed(nc, 4, w64(2, 1), 10, out=u8(2, 10))
    Ctx.mul_packed(nc, 4, 0x13, w64(5, 3), w64(40, 3), w64(5, 3), n=40, k=40)
    assert [w for _, w in nc.seen[2:]] == ["m4rie_mul_batched", "m4rie_unpack", "m4rie_from_packed",
                                          "m4rie_mul_packed"]
    assert all(st == m4.ERR_ARG for st, _ in nc.seen)


def test_noalloc_binding_checks(monkeypatch):
    """mul_noalloc's argument checks, before the bare-pointer entry point is
    reached: CUDA tensors of the field's element type, matching shapes, and a
    CUDA int32 status tensor.  Matching arguments reach the C entry point,
    which rejects an invalid field before any CUDA call."""
    import torch
    import paper_1111_6900_gb300 as m4

    class Stream:
        cuda_stream = 0

    u8 = lambda *shape: torch.zeros(shape, dtype=torch.uint8)     # noqa: E731
    # the real device check refuses host tensors and a wrong element type
    with pytest.raises(TypeError):
        m4.mul_noalloc(4, 0x13, u8(4, 3), u8(3, 5), u8(4, 5), stream=Stream())
    monkeypatch.setattr(m4, "_check_dev", lambda *a, **k: None)
    for bad in (lambda: m4.mul_noalloc(4, 0x13, u8(4, 3), u8(2, 5), u8(4, 5), stream=Stream()),
                lambda: m4.mul_noalloc(4, 0x13, u8(4, 3), u8(3, 5), u8(5, 4), stream=Stream()),
                lambda: m4.mul_noalloc(4, 0x13, u8(4, 3), u8(3, 5), u8(4, 6), stream=Stream()),
                lambda: m4.mul_noalloc(4, 0x13, u8(4, 3, 1), u8(3, 5), u8(4, 5), stream=Stream())):
        with pytest.raises(ValueError):
            bad()
    for status in (torch.zeros(1, dtype=torch.int32),            # host memory
                   torch.zeros(1, dtype=torch.int64), [0]):
        with pytest.raises(TypeError):
            m4.mul_noalloc(4, 0x13, u8(4, 3), u8(3, 5), u8(4, 5), device_status=status, stream=Stream())
    assert m4.mul_noalloc(11, 0x13, u8(4, 3), u8(3, 5), u8(4, 5), stream=Stream()) == m4.ERR_ARG
