"""CPU tests of the schedule sources (Section 5's bilinear formulas): the
subfield construction of schedules/towers.py, the stored table of field
formulas, and the flip-graph search program.  Every formula is checked on all
basis pairs (x^i, x^j) against x^(i+j) mod f computed by tests/fieldref.py."""
import os
import subprocess
import sys

import pytest

import workloads
from tests import fieldref as fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCHED = os.path.join(ROOT, "paper_1111_6900_gb300", "schedules")
sys.path.insert(0, SCHED)
import search  # noqa: E402
import towers  # noqa: E402


def field_formula_ok(e, f, terms):
    for i in range(e):
        for j in range(e):
            acc = 0
            for L, R, W in terms:
                if L >> i & 1 and R >> j & 1:
                    acc ^= W
            if acc != fr.x_power_mod(e, f, i + j):
                return False
    return True


@pytest.mark.parametrize("e,d,count", [(4, 2, 9), (6, 2, 15), (6, 3, 18), (8, 2, 24), (8, 4, 27), (9, 3, 30),
                                       (10, 2, 33), (10, 5, 39)])
def test_subfield_formulas(e, d, count):
    """GF(2^e) through GF(2^d): r(d) products per linear modulus (points of
    GF(2^d) and infinity) and 3 r(d) per irreducible quadratic, carried to the
    polynomial basis of the workload's field."""
    fd = search.FIELD_POLY[d]
    small = [(a, b, search.reduce_poly(d, fd, w)) for a, b, w in search.recursive_formula(d)]
    if d == 5:
        small = search.read_table()[5]
    assert field_formula_ok(d, fd, small)
    terms, tower_mul = towers.subfield_formula(d, e // d, fd, small)
    f = workloads.FIELD_POLY[e]
    assert search.FIELD_POLY[e] == f
    pf = towers.to_polynomial_basis(e, f, terms, tower_mul)
    assert len(pf) == count
    assert field_formula_ok(e, f, pf)


def test_gf2_chinese_remainder_formula_for_e7():
    """e = 7 over GF(2): residues modulo x^2, x + 1, x^2 + x + 1, the two
    irreducible cubics and the top two coefficients (degrees 2 + 1 + 2 + 3 + 3
    + 2 = 13 = 2e - 1): 3 + 1 + 3 + 6 + 6 + 3 = 22 products, the count of
    Table 3's best-known formula for e = 7."""
    forms = search.gf2_crt_formulas(7, search.read_table())
    assert len(forms) == 1 and len(forms[0]) == 22
    assert field_formula_ok(7, workloads.FIELD_POLY[7], forms[0])
    # the moduli must be coprime and add up to 2e - 1: a repeated cubic fails
    bad = [("pt", 0, 2), ("pt", 1, 1), ("inf", 2), ("irr", [1, 1, 1]), ("irr", [1, 1, 0, 1]), ("irr", [1, 1, 0, 1])]
    with pytest.raises(AssertionError):
        towers.gf2_crt_formula(7, bad, lambda k, q: [])


def test_subfield_formula_catches_a_wrong_small_formula():
    """A planted mistake: one term of the GF(4) formula dropped."""
    fd = search.FIELD_POLY[2]
    small = [(a, b, search.reduce_poly(2, fd, w)) for a, b, w in search.recursive_formula(2)][1:]
    terms, tower_mul = towers.subfield_formula(2, 3, fd, small)
    assert not field_formula_ok(6, 0x43, towers.to_polynomial_basis(6, 0x43, terms, tower_mul))


def test_stored_table():
    """Every stored formula is a field formula for its polynomial, with the
    library's counts for e >= 5."""
    table = search.read_table()
    want = {5: 13, 6: 15, 7: 22, 8: 24, 9: 30, 10: 33}
    for e, terms in table.items():
        assert field_formula_ok(e, search.FIELD_POLY[e], terms), e
    for e, r in want.items():
        assert len(table[e]) == r, e


def test_flip_search_reduces_the_schoolbook_formula(tmp_path):
    """The search program, from the 16-term schoolbook formula of GF(2^4),
    reaches the 9 terms of the nested Karatsuba formula (seeded, bounded)."""
    exe = str(tmp_path / "flip_search")
    subprocess.run(["gcc", "-O2", "-o", exe, os.path.join(SCHED, "flip_search.c")], check=True)
    e, f = 4, 0x13
    T = search.field_target(e, f)
    start = [(1 << i, 1 << j, T[i][j]) for i in range(e) for j in range(e)]
    inp = (f"{e} {e} {e} 9 50000000 200000 1\n" + " ".join(str(x) for row in T for x in row) + f"\n{len(start)}\n"
           + "\n".join(f"{a} {b} {c}" for a, b, c in start) + "\n")
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    words = out.stdout.split()
    r = int(words[0])
    terms = [tuple(int(x) for x in words[1 + 3 * q:4 + 3 * q]) for q in range(r)]
    assert r <= 10 and field_formula_ok(e, f, terms)
