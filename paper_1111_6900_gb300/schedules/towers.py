"""Bilinear formulas for GF(2^e) multiplication built through a subfield.

For e = d * t, GF(2^e) is GF(2^d)[y] / (g) with g irreducible of degree t
over GF(2^d).  Two elements are polynomials of degree < t over GF(2^d); their
product (degree <= 2t - 2) is recovered from its residues modulo pairwise
coprime moduli whose degrees add up to 2t - 1 (Chinese remaindering, the
evaluation-interpolation of Toom and Cook): linear factors y - c for points c
of GF(2^d), the point at infinity (the product's top coefficient), and monic
irreducible quadratics over GF(2^d) when GF(2^d) has too few points.  Each
residue product is one multiplication in GF(2^d) (linear moduli) or in
GF(2^d)[y] / (q) ~ GF(2^2d) (quadratics, three GF(2^d) multiplications by
Karatsuba), and each of those is a short GF(2) formula for GF(2^d).  Every
map between them is GF(2)-linear, so the whole is a GF(2)-bilinear formula
with (#linear moduli) * r(d) + (#quadratics) * 3 r(d) terms.  It is written in
the tower basis and carried to the polynomial basis of GF(2)[x] / (f) through
the isomorphism x -> tau, tau a root of f in the tower.

Only GF(2)-linear algebra on bit masks is used; the result is checked against
the field product on every basis pair by the caller.
"""
from __future__ import annotations


# ---------------------------------------------------------------- GF(2) linear maps
# A linear map F_2^n -> F_2^m is the list of its n column masks.

def apply(cols, v: int) -> int:
    out = 0
    i = 0
    while v:
        if v & 1:
            out ^= cols[i]
        v >>= 1
        i += 1
    return out


def parity(x: int) -> int:
    return bin(x).count("1") & 1


def pull_back(mask: int, cols) -> int:
    """The linear form `mask` (on the target) composed with the map `cols`."""
    return sum(parity(mask & c) << j for j, c in enumerate(cols))


def invert(cols, n: int):
    """Columns of the inverse of an invertible n x n map; None if singular."""
    rows = []
    for i in range(n):
        r = 1 << (n + i)
        for j in range(n):
            if cols[j] >> i & 1:
                r |= 1 << j
        rows.append(r)
    for c in range(n):
        piv = next((i for i in range(c, n) if rows[i] >> c & 1), None)
        if piv is None:
            return None
        rows[c], rows[piv] = rows[piv], rows[c]
        for i in range(n):
            if i != c and rows[i] >> c & 1:
                rows[i] ^= rows[c]
    return [sum(((rows[i] >> (n + j)) & 1) << i for i in range(n)) for j in range(n)]


# ---------------------------------------------------------------- GF(2^d) and polynomials over it

class GF:
    def __init__(self, d: int, f: int):
        self.d, self.f, self.q = d, f, 1 << d

    def mul(self, a: int, b: int) -> int:
        r = 0
        for i in range(self.d - 1, -1, -1):
            r <<= 1
            if r >> self.d & 1:
                r ^= self.f
            if b >> i & 1:
                r ^= a
        return r

    def pow(self, a: int, k: int) -> int:
        r = 1
        for _ in range(k):
            r = self.mul(r, a)
        return r

    def inv(self, a: int) -> int:
        return next(x for x in range(1, self.q) if self.mul(a, x) == 1)


def pmul(K: GF, a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] ^= K.mul(x, y)
    return out


def pmod(K: GF, a, m):
    """a mod m, m monic."""
    a = list(a)
    dm = len(m) - 1
    for i in range(len(a) - 1, dm - 1, -1):
        c = a[i]
        if c:
            for j in range(dm + 1):
                a[i - dm + j] ^= K.mul(c, m[j])
    out = a[:dm] + [0] * max(0, dm - len(a))
    return out[:dm]


def irreducible(K: GF, m) -> bool:
    """Monic m of degree <= 5 over K: no factor of degree <= deg(m) / 2."""
    dm = len(m) - 1
    for k in range(1, dm // 2 + 1):
        for low in range(K.q ** k):
            cand = [(low // K.q ** i) % K.q for i in range(k)] + [1]
            if not any(pmod(K, m, cand)):
                return False
    return True


def monic_irreducibles(K: GF, t: int):
    for low in range(K.q ** t):
        m = [(low // K.q ** i) % K.q for i in range(t)] + [1]
        if irreducible(K, m):
            yield m


# ---------------------------------------------------------------- the tower construction

def _block_bits(coeffs, d):
    return sum(c << (d * i) for i, c in enumerate(coeffs))


def _split(v: int, d: int, n: int):
    return [(v >> (d * i)) & ((1 << d) - 1) for i in range(n)]


def subfield_formula(d: int, t: int, fd: int, small):
    """The tower formula for GF(2^(d t)) = GF(2^d)[y] / (g): (terms, tower
    multiplication), terms over the tower basis (bit d j + k = bit k of the
    coefficient of y^j).  small: a formula for GF(2)[x] / (fd), terms
    (L, R, W) over d bits.  None if GF(2^d) has too few moduli of degree <= 2."""
    K = GF(d, fd)
    e = d * t
    g = next(monic_irreducibles(K, t))
    need = 2 * t - 1
    # moduli: linear points first, then infinity, then quadratics
    mods = [("lin", c) for c in range(K.q)][:need]
    if len(mods) < need:
        mods.append(("inf", None))
    quads = []
    if sum(1 for _ in mods) < need:
        qs = monic_irreducibles(K, 2)
        while len(mods) + 2 * len(quads) < need:
            quads.append(next(qs))
        if len(mods) + 2 * len(quads) != need:  # an odd remainder: drop one linear point
            mods.pop(0 if mods[0][0] == "lin" else 1)
    mods += [("quad", q) for q in quads]
    assert sum(2 if k == "quad" else 1 for k, _ in mods) == need

    def residue(coeffs, mod):
        kind, v = mod
        if kind == "lin":
            acc = 0
            for j in range(len(coeffs) - 1, -1, -1):
                acc = K.mul(acc, v) ^ coeffs[j]
            return acc
        if kind == "inf":  # the coefficient of y^(2t-2) of a product, the top coefficient of a factor
            return coeffs[-1] if len(coeffs) == need else coeffs[t - 1]
        return _block_bits(pmod(K, coeffs, v), d)

    def res_bits(mod):
        return 2 * d if mod[0] == "quad" else d

    # residue maps of a factor (tower, e bits) and the forward map of a product ((2t-1) d bits)
    fwd = []
    for i in range(need * d):
        P = _split(1 << i, d, need)
        v, off = 0, 0
        for mod in mods:
            v |= residue(P, mod) << off
            off += res_bits(mod)
        fwd.append(v)
    crt = invert(fwd, need * d)
    assert crt is not None, "moduli are not coprime"
    red = [_block_bits(pmod(K, _split(1 << i, d, need), g), d) for i in range(need * d)]

    # multiplication formula of GF(2^d)[y] / (q) (2d bits) by Karatsuba over GF(2^d)
    def quad_formula(q):
        # output map (c0, c1, c2) in GF^3 (3d bits) -> GF[y]/q (2d bits)
        out_map = [_block_bits(pmod(K, _split(1 << i, d, 3), q), d) for i in range(3 * d)]
        lo = (1 << d) - 1
        terms = []
        for selu, selv, blocks in ((1, 1, (0, 1)), (2, 2, (1, 2)), (3, 3, (1,))):
            for (l, r, w) in small:
                L = (l if selu & 1 else 0) | ((l << d) if selu & 2 else 0)
                R = (r if selv & 1 else 0) | ((r << d) if selv & 2 else 0)
                W = 0
                for b in blocks:
                    W ^= apply(out_map, (w & lo) << (d * b))
                terms.append((L, R, W))
        return terms

    terms = []
    off = 0
    for mod in mods:
        nb = res_bits(mod)
        rmap = [residue(_split(1 << i, d, t), mod) for i in range(e)]
        formula = small if nb == d else quad_formula(mod[1])
        for (l, r, w) in formula:
            L = pull_back(l, rmap)
            R = pull_back(r, rmap)
            W = apply(red, apply(crt, w << off))
            terms.append((L, R, W))
        off += nb

    def tower_mul(a: int, b: int) -> int:
        return _block_bits(pmod(K, pmul(K, _split(a, d, t), _split(b, d, t)), g), d)

    return terms, tower_mul


def to_polynomial_basis(e: int, f: int, terms, tower_mul):
    """Carry a formula in the tower basis to the basis 1, x, .., x^(e-1) of
    GF(2)[x] / (f): x -> tau with f(tau) = 0 in the tower."""
    def f_at(tau):
        acc = 0
        for k in range(e, -1, -1):
            acc = tower_mul(acc, tau) ^ ((f >> k) & 1)
        return acc
    tau = next(c for c in range(2, 1 << e) if f_at(c) == 0)
    psi = [1]
    for _ in range(e - 1):
        psi.append(tower_mul(psi[-1], tau))
    inv = invert(psi, e)
    return [(pull_back(L, psi), pull_back(R, psi), apply(inv, W)) for L, R, W in terms]
