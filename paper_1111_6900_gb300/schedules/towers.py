"""Bilinear formulas for GF(2^e) multiplication by Chinese remaindering.

For e = d * t, GF(2^e) is GF(2^d)[y] / (g) with g irreducible of degree t
over GF(2^d) (d = 1: GF(2)[y] / (g) itself).  Two elements are polynomials of
degree < t over GF(2^d); their product (degree <= 2t - 2) is recovered from
its residues modulo pairwise coprime moduli whose degrees add up to 2t - 1
(the evaluation-interpolation of Toom and Cook): powers (y - c)^k of linear
factors at points c of GF(2^d), the point at infinity (the product's top k
coefficients), and monic irreducible polynomials over GF(2^d).  Each residue
product is one multiplication in GF(2^d) (degree-1 moduli), a truncated
product of two degree-1 polynomials (three GF(2^d) multiplications by
Karatsuba, squared linear factors and infinity), or a multiplication in
GF(2^d)[y] / (q) (a field of 2^(d deg q) elements).  Every map between them is
GF(2)-linear, so the whole is a GF(2)-bilinear formula whose length is the
sum of the residue products' lengths.  It is written in the tower basis and
carried to the polynomial basis of GF(2)[x] / (f) through the isomorphism
x -> tau, tau a root of f in the tower.

Examples: e = 6 through GF(4) with its 4 points and infinity, 5 x 3 = 15
products; e = 7 over GF(2) with x^2, x + 1, infinity^2, x^2 + x + 1 and the two
irreducible cubics, 3 + 1 + 3 + 3 + 6 + 6 = 22.

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


# ---------------------------------------------------------------- Chinese remaindering

def _block_bits(coeffs, d):
    return sum(c << (d * i) for i, c in enumerate(coeffs))


def _split(v: int, d: int, n: int):
    return [(v >> (d * i)) & ((1 << d) - 1) for i in range(n)]


def _deg2_formula(d, small, out_map):
    """Formula for the product of two degree-1 polynomials over GF(2^d)
    (2d bits each) by Karatsuba (three GF(2^d) products: u0 v0, u1 v1,
    (u0 + u1)(v0 + v1)), the product's three coefficients (3d bits) sent
    through the linear map out_map (columns: 3d masks)."""
    lo = (1 << d) - 1
    terms = []
    for selu, blocks in ((1, (0, 1)), (2, (1, 2)), (3, (1,))):
        for (l, r, w) in small:
            L = (l if selu & 1 else 0) | ((l << d) if selu & 2 else 0)
            R = (r if selu & 1 else 0) | ((r << d) if selu & 2 else 0)
            W = 0
            for b in blocks:
                W ^= apply(out_map, (w & lo) << (d * b))
            terms.append((L, R, W))
    return terms


def crt_formula(d: int, t: int, fd: int, small, g, moduli, ring_formula=None):
    """GF(2)-bilinear formula for the product in GF(2^d)[y] / (g) (tower basis)
    from residues modulo the given moduli, whose degrees add up to 2t - 1:
      ("pt", c, k)   (y - c)^k, k = 1 or 2, residues in the basis 1, z (z = y - c);
      ("inf", k)     the top k coefficients of the product (k = 1 or 2);
      ("irr", q)     a monic irreducible q over GF(2^d) of degree >= 2 (coefficient list).
    small: formula for GF(2^d) = GF(2)[x]/(fd).  ring_formula(q): formula for
    GF(2^d)[y]/(q) in its basis 1, y, .. (default: Karatsuba for degree 2)."""
    K = GF(d, fd)
    e = d * t
    need = 2 * t - 1

    def degree(mod):
        return mod[2] if mod[0] == "pt" else mod[1] if mod[0] == "inf" else len(mod[1]) - 1

    assert sum(degree(m) for m in moduli) == need, "moduli degrees must add up to 2t - 1"

    def shift_at(coeffs, c):
        """Coefficients of a(z + c)."""
        out = [0] * len(coeffs)
        for i in range(len(coeffs) - 1, -1, -1):   # Horner: out = out * (z + c) + a_i
            nxt = [0] * len(coeffs)
            for j, x in enumerate(out):
                if x:
                    if j + 1 < len(nxt):
                        nxt[j + 1] ^= x
                    nxt[j] ^= K.mul(x, c)
            nxt[0] ^= coeffs[i]
            out = nxt
        return out

    def residue(coeffs, mod, product):
        kind = mod[0]
        if kind == "pt":
            return _block_bits(shift_at(coeffs, mod[1])[:mod[2]], d)
        if kind == "inf":  # reversed top coefficients: u0 = top, u1 = next
            top = len(coeffs) - 1 if product else t - 1
            return _block_bits([coeffs[top - i] if top - i >= 0 else 0 for i in range(mod[1])], d)
        return _block_bits(pmod(K, coeffs, mod[1]), d)

    def nbits(mod):
        return degree(mod) * d

    fwd = []
    for i in range(need * d):
        P = _split(1 << i, d, need)
        v, off = 0, 0
        for mod in moduli:
            v |= residue(P, mod, True) << off
            off += nbits(mod)
        fwd.append(v)
    crt = invert(fwd, need * d)
    assert crt is not None, "moduli are not coprime"
    red = [_block_bits(pmod(K, _split(1 << i, d, need), g), d) for i in range(need * d)]

    def mod_formula(mod):
        if degree(mod) == 1:
            return small
        if mod[0] in ("pt", "inf"):  # product mod z^2: keep c0, c1
            trunc = [_block_bits(_split(1 << i, d, 3)[:2], d) for i in range(3 * d)]
            return _deg2_formula(d, small, trunc)
        if ring_formula is not None:
            return ring_formula(mod[1])
        assert len(mod[1]) == 3, "irreducible moduli of degree > 2 need ring_formula"
        return _deg2_formula(d, small, [_block_bits(pmod(K, _split(1 << i, d, 3), mod[1]), d) for i in range(3 * d)])

    terms = []
    off = 0
    for mod in moduli:
        rmap = [residue(_split(1 << i, d, t), mod, False) for i in range(e)]
        for (l, r, w) in mod_formula(mod):
            terms.append((pull_back(l, rmap), pull_back(r, rmap), apply(red, apply(crt, w << off))))
        off += nbits(mod)

    def tower_mul(a: int, b: int) -> int:
        return _block_bits(pmod(K, pmul(K, _split(a, d, t), _split(b, d, t)), g), d)

    return terms, tower_mul


def subfield_formula(d: int, t: int, fd: int, small):
    """The tower formula for GF(2^(d t)) = GF(2^d)[y] / (g): (terms, tower
    multiplication), terms over the tower basis (bit d j + k = bit k of the
    coefficient of y^j).  small: a formula for GF(2)[x] / (fd), terms
    (L, R, W) over d bits.  Moduli: the points of GF(2^d), then infinity,
    then monic irreducible quadratics."""
    K = GF(d, fd)
    g = next(monic_irreducibles(K, t))
    need = 2 * t - 1
    mods = [("pt", c, 1) for c in range(K.q)][:need]
    if len(mods) < need:
        mods.append(("inf", 1))
    quads = []
    if len(mods) < need:
        qs = monic_irreducibles(K, 2)
        while len(mods) + 2 * len(quads) < need:
            quads.append(next(qs))
        if len(mods) + 2 * len(quads) != need:  # an odd remainder: drop one linear point
            mods.pop(0)
    mods += [("irr", q) for q in quads]
    return crt_formula(d, t, fd, small, g, mods)


def gf2_crt_formula(e: int, moduli, field_formula):
    """A formula for GF(2)[x]/(g) (g the first irreducible of degree e) from
    residues over GF(2) itself; field_formula(k, q) gives a formula for
    GF(2)[y]/(q) (q irreducible of degree k, as an integer bit mask)."""
    K = GF(1, 0b10)
    g = next(monic_irreducibles(K, e))
    def ring(q):
        qm = sum(c << i for i, c in enumerate(q))
        return field_formula(len(q) - 1, qm)
    return crt_formula(1, e, 0b10, [(1, 1, 1)], g, moduli, ring)


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
