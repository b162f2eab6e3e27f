"""Search for short bilinear schedules of GF(2^e) multiplication (Section 5)
and write them into the library's schedule table.

Section 5 reduces a GF(2^e) matrix product to GF(2) matrix products through a
bilinear formula for the product of two field elements: each of its r terms is
one GF(2) product L_p(A) * R_p(B) of XOR sums of slices, and each output slice
is an XOR sum of those products.  Fewer terms mean fewer GF(2) products.  The
paper's Table 3 lists the best known term counts of polynomial products for
e <= 8 (3, 6, 9, 13, 17, 22, 27).  This script searches the flip graph
(flip_search.c) of formulas for the field product itself (the polynomial
product already reduced modulo f), which can be shorter than the polynomial
product.  Every search starts from the schoolbook formula (e^2 terms), from
the recursive Karatsuba-like formula the library builds, and, for composite e,
from the subfield formulas of towers.py (evaluation and interpolation over
GF(2^d), d | e), runs several seeds in parallel for a few rounds, and keeps
the shortest formula found.

The table (csrc/schedule_table.inc) stores one formula per e for the field
polynomial f_e listed below; the library carries it over to any other
irreducible f of degree e through a field isomorphism and checks the result
on every basis pair before use.  An entry is replaced only by a shorter one.

Usage: python paper_1111_6900_gb300/schedules/search.py [e ...] [--rounds R]
       [--seeds S] [--steps N] [--rounds 0: constructions only]
"""
from __future__ import annotations

import argparse
import os
import re
import subprocess
import sys
import tempfile

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import towers  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(os.path.dirname(HERE), "csrc", "schedule_table.inc")
# the field polynomials of the benchmark workloads (primitive, degree e)
FIELD_POLY = {2: 0x7, 3: 0xB, 4: 0x13, 5: 0x25, 6: 0x43, 7: 0x83, 8: 0x11D, 9: 0x211, 10: 0x409}


def x_pow_mod(e: int, f: int, d: int) -> int:
    a = 1
    for _ in range(d):
        a <<= 1
        if a >> e & 1:
            a ^= f
    return a


def reduce_poly(e: int, f: int, w: int) -> int:
    """Output mask over field coefficients of a mask over x^0 .. x^(2e-2)."""
    v = 0
    for d in range(2 * e - 1):
        if w >> d & 1:
            v ^= x_pow_mod(e, f, d)
    return v


# ---- the recursive Karatsuba-like polynomial formulas (split and nest), as
# csrc/schedule.cpp builds them: terms (L, R, W), W over x^0 .. x^(2n-2)
def _base(n):
    if n == 1:
        return [(1, 1, 1)]
    if n == 2:
        return [(1, 1, 0x3), (2, 2, 0x6), (3, 3, 0x2)]
    return [(1, 1, 0x07), (2, 2, 0x0E), (4, 4, 0x1C), (3, 3, 0x02), (5, 5, 0x04), (6, 6, 0x08)]


def _split(H, Lo, h, lo_n):
    lm = (1 << lo_n) - 1
    out = [(a, b, w ^ (w << h)) for a, b, w in H]
    out += [(a << h, b << h, (w << 2 * h) ^ (w << h)) for a, b, w in Lo]
    out += [(a | ((a & lm) << h), b | ((b & lm) << h), w << h) for a, b, w in H]
    return out


def _nest(inner, u, outer, v):
    out = []
    for ao, bo, wo in outer:
        for ai, bi, wi in inner:
            L = R = W = 0
            for s in range(v):
                if ao >> s & 1:
                    L |= ai << (u * s)
                if bo >> s & 1:
                    R |= bi << (u * s)
            for d in range(2 * v - 1):
                if wo >> d & 1:
                    W ^= wi << (u * d)
            out.append((L, R, W))
    return out


def recursive_formula(n: int, memo={}):
    if n in memo:
        return memo[n]
    if n <= 3:
        b = _base(n)
    else:
        b = None
        for h in range((n + 1) // 2, n):
            c = _split(recursive_formula(h), recursive_formula(n - h), h, n - h)
            if b is None or len(c) < len(b):
                b = c
        for u in range(2, n):
            if n % u == 0:
                c = _nest(recursive_formula(u), u, recursive_formula(n // u), n // u)
                if len(c) < len(b):
                    b = c
    memo[n] = b
    return b


def field_target(e: int, f: int):
    return [[x_pow_mod(e, f, i + j) for j in range(e)] for i in range(e)]


def is_field_formula(e: int, f: int, terms) -> bool:
    T = field_target(e, f)
    for i in range(e):
        for j in range(e):
            acc = 0
            for a, b, c in terms:
                if a >> i & 1 and b >> j & 1:
                    acc ^= c
            if acc != T[i][j]:
                return False
    return True


def read_table(path: str = TABLE):
    """{e: [(L, R, W), ...]} from the table file (W over the e output slices)."""
    out = {}
    if not os.path.exists(path):
        return out
    with open(path) as fh:
        text = fh.read()
    for m in re.finditer(r"\{\s*(\d+)\s*,\s*0x([0-9A-Fa-f]+)\s*,\s*(\d+)\s*,\s*\{([^}]*)\}\s*\}", text):
        e, r = int(m.group(1)), int(m.group(3))
        nums = [int(x, 0) for x in m.group(4).replace("\n", " ").split(",") if x.strip()]
        out[e] = [tuple(nums[3 * p:3 * p + 3]) for p in range(r)]
    return out


def write_table(table, path: str = TABLE):
    lines = [
        "// Field-product formulas found by paper_1111_6900_gb300/schedules/search.py",
        "// (flip-graph search; do not edit by hand).  Entry: e, the field polynomial",
        "// f_e the formula is written for, the number of terms r, then r triples",
        "// (L, R, W): slice masks of A and of B and the mask of output slices that the",
        "// GF(2) product L(A) * R(B) is added to (Section 5, with the reduction mod f_e",
        "// folded into W).",
    ]
    for e in sorted(table):
        terms = table[e]
        body = ",\n     ".join(", ".join(f"0x{v:X}" for v in t) for t in terms)
        lines.append(f"{{{e}, 0x{FIELD_POLY[e]:X}, {len(terms)}, {{{body}}}}},")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def build_search(tmp: str) -> str:
    exe = os.path.join(tmp, "flip_search")
    subprocess.run(["gcc", "-O2", "-o", exe, os.path.join(HERE, "flip_search.c")], check=True)
    return exe


def run_seeds(exe, e, f, starts, target, steps, plateau, seed0):
    T = field_target(e, f)
    procs = []
    for i, start in enumerate(starts):
        inp = (f"{e} {e} {e} {target} {steps} {plateau} {seed0 + i}\n" + " ".join(str(x) for row in T for x in row)
               + f"\n{len(start)}\n" + "\n".join(f"{a} {b} {c}" for a, b, c in start) + "\n")
        p = subprocess.Popen([exe], stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        p.stdin.write(inp)
        p.stdin.close()
        procs.append(p)
    found = []
    for p in procs:
        out = p.stdout.read().split()
        p.wait()
        if p.returncode != 0 or not out:
            continue
        r = int(out[0])
        terms = [tuple(int(x) for x in out[1 + 3 * q:4 + 3 * q]) for q in range(r)]
        if is_field_formula(e, f, terms):
            found.append(terms)
    return found


def subfield_formulas(e, table):
    """Formulas through GF(2^d) for every divisor 2 <= d < e, each with the
    shortest GF(2^d) formula known (table or recursive)."""
    out = []
    for d in range(2, e):
        if e % d:
            continue
        fd = FIELD_POLY[d]
        small = [(a, b, reduce_poly(d, fd, w)) for a, b, w in recursive_formula(d)]
        if table.get(d) and len(table[d]) < len(small):
            small = table[d]
        terms, tower_mul = towers.subfield_formula(d, e // d, fd, small)
        pf = towers.to_polynomial_basis(e, FIELD_POLY[e], terms, tower_mul)
        if is_field_formula(e, FIELD_POLY[e], pf):
            out.append(pf)
    return out


# Chinese remaindering over GF(2) itself, for e where no subfield helps: the
# moduli (degrees adding up to 2e - 1) and their residue products' lengths
GF2_CRT_MODULI = {
    7: [("pt", 0, 2), ("pt", 1, 1), ("inf", 2), ("irr", [1, 1, 1]), ("irr", [1, 1, 0, 1]), ("irr", [1, 0, 1, 1])],
}


def gf2_crt_formulas(e, table):
    if e not in GF2_CRT_MODULI:
        return []

    def ring(k, q):  # the shortest known formula for GF(2)[y]/(q), deg q = k
        fk = FIELD_POLY[k]
        base = [(a, b, reduce_poly(k, fk, w)) for a, b, w in recursive_formula(k)]
        if table.get(k) and len(table[k]) < len(base):
            base = table[k]
        K = towers.GF(k, fk)
        return towers.to_polynomial_basis(k, q, base, K.mul)

    terms, tower_mul = towers.gf2_crt_formula(e, GF2_CRT_MODULI[e], ring)
    pf = towers.to_polynomial_basis(e, FIELD_POLY[e], terms, tower_mul)
    return [pf] if is_field_formula(e, FIELD_POLY[e], pf) else []


def search(e, rounds, seeds, steps, plateau, known, table=None, verbose=True):
    f = FIELD_POLY[e]
    naive = [(1 << i, 1 << j, x_pow_mod(e, f, i + j)) for i in range(e) for j in range(e)]
    rec = [(a, b, reduce_poly(e, f, w)) for a, b, w in recursive_formula(e)]
    pool = [t for t in [known, rec] + subfield_formulas(e, table or {}) + gf2_crt_formulas(e, table or {}) if t]
    best = min(pool, key=len)
    if verbose:
        print(f"e={e}: start formulas {sorted(len(t) for t in pool)}", flush=True)
    if rounds <= 0:
        return best
    with tempfile.TemporaryDirectory() as tmp:
        exe = build_search(tmp)
        for rnd in range(rounds):
            starts = [naive if (i % 2 == 0 and rnd == 0) else pool[i % len(pool)] for i in range(seeds)]
            found = run_seeds(exe, e, f, starts, 1, steps, plateau, 1000 * (rnd + 1) + 7 * e)
            found.sort(key=len)
            pool = (found[:max(1, seeds // 2)] + [best])
            if found and len(found[0]) < len(best):
                best = found[0]
            if verbose:
                print(f"e={e} round {rnd}: best {len(best)} (this round: {sorted(len(t) for t in found)})", flush=True)
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("e", nargs="*", type=int, default=list(range(2, 11)))
    ap.add_argument("--rounds", type=int, default=4)
    ap.add_argument("--seeds", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--steps", type=int, default=300_000_000)
    ap.add_argument("--plateau", type=int, default=1_000_000)
    args = ap.parse_args()
    table = read_table()
    for e in args.e:
        old = table.get(e)
        best = search(e, args.rounds, args.seeds, args.steps, args.plateau, old, table)
        if old is None or len(best) < len(old):
            table[e] = best
            write_table(table)
            print(f"e={e}: table entry now {len(best)} terms", flush=True)
        else:
            print(f"e={e}: kept the table entry ({len(old)} terms)", flush=True)


if __name__ == "__main__":
    main()
