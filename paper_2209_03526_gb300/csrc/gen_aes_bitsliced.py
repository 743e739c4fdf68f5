#!/usr/bin/env python3
"""Derive the bitsliced AES-128 S-box circuit used by aes_bitsliced.cuh and write that header.

The S-box is S(a) = A * a^{-1} + 0x63 (FIPS-197 Sec. 5.1.1): the inverse in GF(2^8) with the
AES polynomial x^8 + x^4 + x^3 + x + 1, then an affine map over GF(2).  A bitsliced S-box needs
that inverse as a circuit of AND and XOR gates on the eight bit planes.  This script builds it
in a tower field (a standard way to invert in GF(2^8) with few gates):

    GF(4)   = GF(2)[w] / (w^2 + w + 1)
    GF(16)  = GF(4)[z] / (z^2 + z + w)
    GF(256) = GF(16)[y] / (y^2 + y + lam)          (lam chosen below, trace 1)

In GF(q^2) = GF(q)[u] / (u^2 + u + c) the inverse of a1 u + a0 is
(a1 u + (a0 + a1)) / (c a1^2 + a1 a0 + a0^2), so an inverse in GF(256) costs three
multiplications and one inverse in GF(16), and that inverse three multiplications and one
inverse (a squaring, which is linear) in GF(4).  The isomorphism between the AES field and
the tower is the linear map sending x^k to g^k for a root g of the AES polynomial in the
tower; the output map is the affine matrix times that map's inverse.

Everything is checked here, exhaustively, against an S-box computed from its definition
(inverse by search, then the affine map) before the header is written.  Run from this
directory: python gen_aes_bitsliced.py  (writes aes_bitsliced_sbox.cuh).
"""
from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))

# ----------------------------------------------------------------- the AES field, by definition


def aes_mul(a: int, b: int) -> int:
    p = 0
    for _ in range(8):
        if b & 1:
            p ^= a
        hi = a & 0x80
        a = (a << 1) & 0xFF
        if hi:
            a ^= 0x1B
        b >>= 1
    return p


def aes_inv(a: int) -> int:
    return 0 if a == 0 else next(x for x in range(1, 256) if aes_mul(a, x) == 1)


def affine(b: int) -> int:
    s = 0
    for i in range(8):
        bit = ((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^ (b >> ((i + 6) % 8))
               ^ (b >> ((i + 7) % 8)) ^ (0x63 >> i)) & 1
        s |= bit << i
    return s


SBOX = [affine(aes_inv(a)) for a in range(256)]

# ----------------------------------------------------------------- the tower field on integers
# GF(4) element c1 w + c0 as (c1 << 1) | c0; GF(16) element b1 z + b0 as (b1 << 2) | b0;
# GF(256) element a1 y + a0 as (a1 << 4) | a0.


def m4(a, b):
    a1, a0, b1, b0 = a >> 1, a & 1, b >> 1, b & 1
    p, q, r = a1 & b1, a0 & b0, (a1 ^ a0) & (b1 ^ b0)
    return ((r ^ q) << 1) | (p ^ q)


def m16(a, b, phi=2):
    a1, a0, b1, b0 = a >> 2, a & 3, b >> 2, b & 3
    p, q, r = m4(a1, b1), m4(a0, b0), m4(a1 ^ a0, b1 ^ b0)
    return ((r ^ q) << 2) | (m4(phi, p) ^ q)


def m256(a, b, lam):
    a1, a0, b1, b0 = a >> 4, a & 15, b >> 4, b & 15
    p, q, r = m16(a1, b1), m16(a0, b0), m16(a1 ^ a0, b1 ^ b0)
    return ((r ^ q) << 4) | (m16(lam, p) ^ q)


def trace16(a):
    t, x = 0, a
    for _ in range(4):
        t ^= x
        x = m16(x, x)
    return t


def pow256(g, k, lam):
    r = 1
    for _ in range(k):
        r = m256(r, g, lam)
    return r


def column_matrix(cols):
    """8x8 GF(2) matrix whose column k is the bit vector cols[k]: rows[i] = bit mask over inputs."""
    return [sum(((cols[k] >> i) & 1) << k for k in range(8)) for i in range(8)]


def apply(rows, v):
    return sum((bin(rows[i] & v).count("1") & 1) << i for i in range(8))


def invert_matrix(rows):
    n = 8
    aug = [(rows[i] | (1 << (n + i))) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if (aug[r] >> c) & 1)
        aug[c], aug[piv] = aug[piv], aug[c]
        for r in range(n):
            if r != c and (aug[r] >> c) & 1:
                aug[r] ^= aug[c]
    return [aug[i] >> n for i in range(n)]


def matmul(a, b):
    """(a b)[i] as row masks: row i of a times b."""
    out = []
    for i in range(8):
        m = 0
        for j in range(8):
            if (a[i] >> j) & 1:
                m ^= b[j]
        out.append(m)
    return out


# ----------------------------------------------------------------- a gate-level circuit builder

class Circuit:
    def __init__(self):
        self.lines = []
        self.n = 0
        self.ands = 0
        self.xors = 0

    def tmp(self, expr):
        name = f"t{self.n}"
        self.n += 1
        self.lines.append(f"    const uint32_t {name} = {expr};")
        return name

    def xor(self, a, b):
        if a == "0":
            return b
        if b == "0":
            return a
        self.xors += 1
        return self.tmp(f"{a} ^ {b}")

    def and_(self, a, b):
        self.ands += 1
        return self.tmp(f"{a} & {b}")

    def lin(self, rows, ins, const=0):
        """outputs out_i = XOR of ins[j] with rows[i] bit j (+ the constant bit i as a NOT)."""
        outs = []
        for i in range(len(rows)):
            acc = "0"
            for j in range(len(ins)):
                if (rows[i] >> j) & 1:
                    acc = self.xor(acc, ins[j])
            if (const >> i) & 1:
                acc = self.tmp(f"~{acc}") if acc != "0" else self.tmp("0xFFFFFFFFu")
            outs.append(acc)
        return outs


# bit-plane circuits on the tower representation (lists of bit names, index 0 = LSB)

def c_m4(C, a, b):
    a0, a1, b0, b1 = a[0], a[1], b[0], b[1]
    p = C.and_(a1, b1)
    q = C.and_(a0, b0)
    r = C.and_(C.xor(a1, a0), C.xor(b1, b0))
    return [C.xor(p, q), C.xor(r, q)]


def c_m4_sum(C, a, b, asum, bsum):
    """GF(4) product with the operands' (hi + lo) precomputed."""
    p = C.and_(a[1], b[1])
    q = C.and_(a[0], b[0])
    r = C.and_(asum, bsum)
    return [C.xor(p, q), C.xor(r, q)]


def c_phi4(C, a):                      # w * a  (phi = w)
    return [a[1], C.xor(a[1], a[0])]


def c_add(C, a, b):
    return [C.xor(x, y) for x, y in zip(a, b)]


def c_m16(C, a, b):
    a0, a1, b0, b1 = a[0:2], a[2:4], b[0:2], b[2:4]
    p = c_m4_sum(C, a1, b1, C.xor(a1[0], a1[1]), C.xor(b1[0], b1[1]))
    q = c_m4_sum(C, a0, b0, C.xor(a0[0], a0[1]), C.xor(b0[0], b0[1]))
    asum, bsum = c_add(C, a1, a0), c_add(C, b1, b0)
    r = c_m4(C, asum, bsum)
    return c_add(C, c_phi4(C, p), q) + c_add(C, r, q)


def c_inv16(C, a):
    a0, a1 = a[0:2], a[2:4]
    # Delta = w a1^2 + a1 a0 + a0^2 in GF(4); a^2 = (a1, a1 + a0) in bit form [lo, hi]
    sq1 = [C.xor(a1[1], a1[0]), a1[1]]
    sq0 = [C.xor(a0[1], a0[0]), a0[1]]
    d = c_add(C, c_add(C, c_phi4(C, sq1), c_m4(C, a1, a0)), sq0)
    dinv = [C.xor(d[1], d[0]), d[1]]                    # inverse in GF(4) = square
    hi = c_m4(C, a1, dinv)
    lo = c_m4(C, c_add(C, a0, a1), dinv)
    return lo + hi


def build_sbox(lam):
    """The circuit for S on bit planes x0..x7 (x0 = bit 0); returns (Circuit, output names)."""
    # isomorphism: a root g of the AES polynomial in the tower
    g = next(c for c in range(2, 256)
             if pow256(c, 8, lam) ^ pow256(c, 4, lam) ^ pow256(c, 3, lam) ^ c ^ 1 == 0)
    to_tower = column_matrix([pow256(g, k, lam) for k in range(8)])
    from_tower = invert_matrix(to_tower)
    aff = column_matrix([affine(1 << k) ^ 0x63 for k in range(8)])   # linear part of the affine map
    out_rows = matmul(aff, from_tower)
    # sanity: the map is a field isomorphism on every pair
    for a in range(0, 256, 7):
        for b in range(0, 256, 5):
            assert apply(to_tower, aes_mul(a, b)) == m256(apply(to_tower, a), apply(to_tower, b), lam)
    C = Circuit()
    x = [f"x{i}" for i in range(8)]
    t = C.lin(to_tower, x)
    a0, a1 = t[0:4], t[4:8]
    # Delta = lam a1^2 + a1 a0 + a0^2 in GF(16): the squares and the constant product are
    # linear, so lam a1^2 + a0^2 is one linear map of the eight bits
    sq_rows = []
    for i in range(4):
        m = 0
        for k in range(8):
            v = 1 << k
            hi, lo = v >> 4, v & 15
            val = m16(lam, m16(hi, hi)) ^ m16(lo, lo)
            m |= ((val >> i) & 1) << k
        sq_rows.append(m)
    lin_part = C.lin(sq_rows, t)
    delta = c_add(C, lin_part, c_m16(C, a1, a0))
    dinv = c_inv16(C, delta)
    hi = c_m16(C, a1, dinv)
    lo = c_m16(C, c_add(C, a0, a1), dinv)
    y = lo + hi
    out = C.lin(out_rows, y, const=0x63)
    return C, out, to_tower, out_rows


def eval_circuit(C, out, v):
    env = {f"x{i}": (v >> i) & 1 for i in range(8)}
    for line in C.lines:
        lhs, rhs = line.split("=", 1)
        name = lhs.split()[-1]
        expr = rhs.strip().rstrip(";").replace("0xFFFFFFFFu", "1")
        val = eval(expr, {}, env)
        env[name] = val & 1
    return sum((env[o] & 1) << i for i, o in enumerate(out))


def header_text() -> str:
    """The generated header, after checking the circuit on all 256 inputs."""
    best = None
    for lam in range(1, 16):
        if trace16(lam) != 1:
            continue
        C, out, _, _ = build_sbox(lam)
        if best is None or C.ands + C.xors < best[0].ands + best[0].xors:
            best = (C, out, lam)
    C, out, lam = best
    for v in range(256):
        assert eval_circuit(C, out, v) == SBOX[v], v
    body = "\n".join(C.lines)
    outs = "\n".join(f"    x{i} = {o};" for i, o in enumerate(out))
    hdr = f"""// aes_bitsliced_sbox.cuh -- GENERATED by gen_aes_bitsliced.py; do not edit.
//
// The AES-128 S-box (FIPS-197 Sec. 5.1.1) on eight bit planes: bit i of byte b of each of
// 32 blocks is bit b of word x_i.  Inverse in GF(2^8) through the tower field
// GF(((2^2)^2)^2) (GF(256) over GF(16) with lambda = {lam}), then the affine map; checked
// exhaustively against the S-box's definition by the generator.  {C.ands} AND and {C.xors} XOR gates.
#pragma once
#include <cstdint>

namespace ogm {{

__device__ __forceinline__ void bs_sbox(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint32_t& x4,
                                        uint32_t& x5, uint32_t& x6, uint32_t& x7) {{
{body}
{outs}
}}

}}  // namespace ogm
"""
    return hdr


def main():
    hdr = header_text()
    with open(os.path.join(HERE, "aes_bitsliced_sbox.cuh"), "w") as f:
        f.write(hdr)
    print("wrote aes_bitsliced_sbox.cuh; all 256 inputs equal the S-box")


if __name__ == "__main__":
    main()
