// host_crypto.cpp -- host side of the oblivgm library: AES-128 (32-bit column
// T-table form), DPF/DCF key generation and the secure query token of
// Sec. V-C, and the servers' parsing of the three tokens into device keys.
//
// DPF: the tree construction of Boyle, Gilboa and Ishai ("Function Secret
// Sharing: Improvements and Extensions", CCS'16), cited by the paper for
// equality predicates.  DCF: the construction of Boyle et al. ("Function
// Secret Sharing for Mixed-Mode and Fixed-Point Secure Computation",
// Eurocrypt'21), cited for range predicates.  PRG: H_K(s) = AES_K(s) xor s under
// fixed public keys; the control bit is bit 0 of byte 0 and Convert into
// Z_{2^32} reads bytes 4..7 of a seed (bytes 0..3 of a DCF value block).
#include "host_crypto.h"

#include <cstring>
#include <mutex>

namespace ogm {

namespace {

inline uint32_t rotl(uint32_t x, int k) { return k == 0 ? x : (x << k) | (x >> (32 - k)); }
inline uint32_t ld32(const uint8_t* p) { uint32_t v; std::memcpy(&v, p, 4); return v; }   // LE host
inline void st32(uint8_t* p, uint32_t v) { std::memcpy(p, &v, 4); }
inline uint16_t ld16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }

// GF(2^8) through exponent/logarithm tables of the generator 3.
struct Gf {
    uint8_t exp[512], log[256];
    Gf() {
        uint8_t x = 1;
        for (int i = 0; i < 255; i++) {
            exp[i] = x;
            log[x] = (uint8_t)i;
            uint8_t x2 = (uint8_t)((x << 1) ^ ((x & 0x80) ? 0x1b : 0));
            x = (uint8_t)(x2 ^ x);   // x * 3
        }
        for (int i = 255; i < 512; i++) exp[i] = exp[i - 255];
        log[0] = 0;
    }
    uint8_t mul(uint8_t a, uint8_t b) const { return (a && b) ? exp[log[a] + log[b]] : 0; }
    uint8_t inv(uint8_t a) const { return a ? exp[255 - log[a]] : 0; }
};

AesTables build_tables() {
    Gf gf;
    AesTables t{};
    for (int x = 0; x < 256; x++) {
        uint8_t b = gf.inv((uint8_t)x);
        // affine map written with byte rotations: s = b ^ rotl(b,1) ^ rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ 0x63
        uint32_t bb = b;
        uint32_t r = bb ^ ((bb << 1) | (bb >> 7)) ^ ((bb << 2) | (bb >> 6)) ^ ((bb << 3) | (bb >> 5)) ^
                     ((bb << 4) | (bb >> 4));
        uint8_t s = (uint8_t)((r ^ 0x63) & 0xFF);
        t.sbox[x] = s;
        uint8_t s2 = gf.mul(s, 2), s3 = gf.mul(s, 3);
        t.te0[x] = (uint32_t)s2 | ((uint32_t)s << 8) | ((uint32_t)s << 16) | ((uint32_t)s3 << 24);
    }
    return t;
}

}  // namespace

const AesTables& aes_tables() {
    static const AesTables t = build_tables();
    return t;
}

RoundKeys expand_key(const uint8_t key[16]) {
    const AesTables& T = aes_tables();
    RoundKeys rk{};
    for (int i = 0; i < 4; i++) rk.w[i] = ld32(key + 4 * i);
    uint8_t rcon = 1;
    for (int i = 4; i < 44; i++) {
        uint32_t t = rk.w[i - 1];
        if (i % 4 == 0) {
            t = (t >> 8) | (t << 24);   // RotWord on little-endian bytes
            t = (uint32_t)T.sbox[t & 0xFF] | ((uint32_t)T.sbox[(t >> 8) & 0xFF] << 8) |
                ((uint32_t)T.sbox[(t >> 16) & 0xFF] << 16) | ((uint32_t)T.sbox[t >> 24] << 24);
            t ^= rcon;
            rcon = (uint8_t)((rcon << 1) ^ ((rcon & 0x80) ? 0x1b : 0));
        }
        rk.w[i] = rk.w[i - 4] ^ t;
    }
    return rk;
}

void aes_encrypt(const RoundKeys& rk, const uint32_t in[4], uint32_t out[4]) {
    const AesTables& T = aes_tables();
    uint32_t c[4], n[4];
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk.w[j];
    for (int r = 1; r < 10; r++) {
        for (int j = 0; j < 4; j++) {
            n[j] = T.te0[c[j] & 0xFF] ^ rotl(T.te0[(c[(j + 1) & 3] >> 8) & 0xFF], 8) ^
                   rotl(T.te0[(c[(j + 2) & 3] >> 16) & 0xFF], 16) ^ rotl(T.te0[c[(j + 3) & 3] >> 24], 24) ^
                   rk.w[4 * r + j];
        }
        std::memcpy(c, n, sizeof c);
    }
    for (int j = 0; j < 4; j++) {
        n[j] = (uint32_t)T.sbox[c[j] & 0xFF] | ((uint32_t)T.sbox[(c[(j + 1) & 3] >> 8) & 0xFF] << 8) |
               ((uint32_t)T.sbox[(c[(j + 2) & 3] >> 16) & 0xFF] << 16) |
               ((uint32_t)T.sbox[c[(j + 3) & 3] >> 24] << 24);
        out[j] = n[j] ^ rk.w[40 + j];
    }
}

const RoundKeys& fixed_key(int j) {
    static RoundKeys keys[4];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int k = 0; k < 4; k++) {
            uint8_t key[16];
            for (int i = 0; i < 16; i++) key[i] = (uint8_t)(16 * k + i);
            keys[k] = expand_key(key);
        }
    });
    return keys[j];
}

namespace {

struct Seed { uint32_t w[4]; };

Seed load_seed(const uint8_t* b) { Seed s; for (int i = 0; i < 4; i++) s.w[i] = ld32(b + 4 * i); return s; }
void store_seed(uint8_t* b, const Seed& s) { for (int i = 0; i < 4; i++) st32(b + 4 * i, s.w[i]); }

// H_K(s) = AES_K(s) xor s
Seed prg(int which, const Seed& s) {
    Seed o;
    aes_encrypt(fixed_key(which), s.w, o.w);
    for (int i = 0; i < 4; i++) o.w[i] ^= s.w[i];
    return o;
}

// child (seed, control bit) in direction dir (0 = L, 1 = R)
void expand(int dir, const Seed& s, Seed* cs, uint32_t* ct) {
    *cs = prg(dir, s);
    *ct = cs->w[0] & 1u;
    cs->w[0] &= ~1u;
}

inline uint32_t input_bit(uint32_t x, int n, int i) { return (x >> (n - i)) & 1u; }   // i = 1..n, MSB first

void put_header(uint8_t* k, uint32_t kind, int n, int party, const uint8_t seed[16], int group) {
    std::memset(k, 0, 8);
    k[0] = (uint8_t)kind;
    k[1] = (uint8_t)n;
    k[2] = (uint8_t)party;
    k[3] = (uint8_t)group;
    std::memcpy(k + 8, seed, 16);
}

// Convert into the output group: Z_{2^32} reads bytes 4..7 of a seed (bytes 0..3 of a
// value block); Z_2 reads bit 1 of byte 0 of a seed (bit 0 of byte 0 of a value block).
// Z_2 arithmetic is the Z_{2^32} arithmetic reduced mod 2, so only stored words are masked.
inline uint32_t conv_seed(const Seed& s, int group) { return group ? (s.w[0] >> 1) & 1u : s.w[1]; }
inline uint32_t conv_value(uint32_t w0, int group) { return group ? (w0 & 1u) : w0; }
inline uint32_t gmask(int group) { return group ? 1u : 0xFFFFFFFFu; }

}  // namespace

void dpf_gen(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0,
             uint8_t* k1, int group) {
    Seed s[2] = {load_seed(s0), load_seed(s1)};
    uint32_t t[2] = {0, 1};
    put_header(k0, OBLIVGM_KEY_DPF, n, 0, s0, group);
    put_header(k1, OBLIVGM_KEY_DPF, n, 1, s1, group);
    for (int i = 1; i <= n; i++) {
        Seed c[2][2];
        uint32_t tc[2][2];
        for (int b = 0; b < 2; b++) {
            expand(0, s[b], &c[b][0], &tc[b][0]);
            expand(1, s[b], &c[b][1], &tc[b][1]);
        }
        const uint32_t a = input_bit(alpha, n, i);
        const int keep = (int)a, lose = 1 - (int)a;
        Seed scw;
        for (int w = 0; w < 4; w++) scw.w[w] = c[0][lose].w[w] ^ c[1][lose].w[w];
        const uint32_t tlcw = tc[0][0] ^ tc[1][0] ^ a ^ 1u;
        const uint32_t trcw = tc[0][1] ^ tc[1][1] ^ a;
        const size_t off = 24 + (size_t)(i - 1) * 20;
        for (uint8_t* k : {k0, k1}) {
            store_seed(k + off, scw);
            k[off + 16] = (uint8_t)tlcw;
            k[off + 17] = (uint8_t)trcw;
            k[off + 18] = k[off + 19] = 0;
        }
        const uint32_t tkeep = keep ? trcw : tlcw;
        for (int b = 0; b < 2; b++) {
            const uint32_t m = 0u - t[b];
            for (int w = 0; w < 4; w++) s[b].w[w] = c[b][keep].w[w] ^ (scw.w[w] & m);
            t[b] = tc[b][keep] ^ (t[b] & tkeep);
        }
    }
    uint32_t cw = beta - conv_seed(s[0], group) + conv_seed(s[1], group);
    if (t[1]) cw = 0u - cw;
    cw &= gmask(group);
    st32(k0 + 24 + (size_t)n * 20, cw);
    st32(k1 + 24 + (size_t)n * 20, cw);
}

void dcf_gen(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0,
             uint8_t* k1, int group) {
    Seed s[2] = {load_seed(s0), load_seed(s1)};
    uint32_t t[2] = {0, 1};
    uint32_t valpha = 0;
    put_header(k0, OBLIVGM_KEY_DCF, n, 0, s0, group);
    put_header(k1, OBLIVGM_KEY_DCF, n, 1, s1, group);
    for (int i = 1; i <= n; i++) {
        Seed c[2][2];
        uint32_t tc[2][2], v[2][2];
        for (int b = 0; b < 2; b++) {
            for (int d = 0; d < 2; d++) {
                expand(d, s[b], &c[b][d], &tc[b][d]);
                v[b][d] = conv_value(prg(2 + d, s[b]).w[0], group);
            }
        }
        const uint32_t a = input_bit(alpha, n, i);
        const int keep = (int)a, lose = 1 - (int)a;
        Seed scw;
        for (int w = 0; w < 4; w++) scw.w[w] = c[0][lose].w[w] ^ c[1][lose].w[w];
        const bool neg = t[1] != 0;
        uint32_t vcw = v[1][lose] - v[0][lose] - valpha;
        if (neg) vcw = 0u - vcw;
        if (lose == 0) vcw += neg ? 0u - beta : beta;
        valpha = valpha - v[1][keep] + v[0][keep] + (neg ? 0u - vcw : vcw);
        const uint32_t tlcw = tc[0][0] ^ tc[1][0] ^ a ^ 1u;
        const uint32_t trcw = tc[0][1] ^ tc[1][1] ^ a;
        const size_t off = 24 + (size_t)(i - 1) * 24;
        for (uint8_t* k : {k0, k1}) {
            store_seed(k + off, scw);
            k[off + 16] = (uint8_t)tlcw;
            k[off + 17] = (uint8_t)trcw;
            k[off + 18] = k[off + 19] = 0;
            st32(k + off + 20, vcw & gmask(group));
        }
        const uint32_t tkeep = keep ? trcw : tlcw;
        for (int b = 0; b < 2; b++) {
            const uint32_t m = 0u - t[b];
            for (int w = 0; w < 4; w++) s[b].w[w] = c[b][keep].w[w] ^ (scw.w[w] & m);
            t[b] = tc[b][keep] ^ (t[b] & tkeep);
        }
    }
    uint32_t cw = conv_seed(s[1], group) - conv_seed(s[0], group) - valpha;
    if (t[1]) cw = 0u - cw;
    cw &= gmask(group);
    st32(k0 + 24 + (size_t)n * 24, cw);
    st32(k1 + 24 + (size_t)n * 24, cw);
}

namespace {

// A 2^m-bit vector as four words (bit j in word j / 32); bits from 2^m up cleared.
struct Vec { uint32_t w[4]; };

Vec vec_keep_low(Vec v, int m) {
    const int bits = 1 << m;
    for (int w = 0; w < 4; w++) {
        const int lo = 32 * w;
        if (bits <= lo) v.w[w] = 0;
        else if (bits < lo + 32) v.w[w] &= (1u << (bits - lo)) - 1u;
    }
    return v;
}

// H_{K_vdir}(s) cut to 2^m bits: a DCF level's value vector of child dir, and (dir 0)
// Conv of a leaf seed, the value block a further level would have computed.
Vec value_vec(int dir, const Seed& s, int m) {
    const Seed o = prg(2 + dir, s);
    Vec v;
    for (int w = 0; w < 4; w++) v.w[w] = o.w[w];
    return vec_keep_low(v, m);
}

Vec vec_xor(const Vec& a, const Vec& b) {
    Vec r;
    for (int w = 0; w < 4; w++) r.w[w] = a.w[w] ^ b.w[w];
    return r;
}

void store_vec(uint8_t* p, const Vec& v) { for (int w = 0; w < 4; w++) st32(p + 4 * w, v.w[w]); }

}  // namespace

// BGI16's early termination over Z_2 (the DPF the paper cites, Sec. IV-B), and the same
// for the BCG+21 DCF over the vector group Z_2^(2^m): the nu = n - m levels walk the high
// bits of alpha; a DCF level's lost branch carries the all-ones vector when alpha's bit is
// 1 (inputs there are smaller than alpha), and the final word puts e_{alpha_lo} (DPF) or
// the bits below alpha_lo (DCF) on alpha_hi's leaf.  Over Z_2 every sign is +.
void gen_et(uint32_t kind, int n, uint32_t alpha, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0,
            uint8_t* k1) {
    const bool dcf = kind == OBLIVGM_KEY_DCF;
    const int m = et_low_bits(n), nu = n - m;
    const size_t lb = dcf ? 36 : 20;
    put_header(k0, kind, n, 0, s0, 1);
    put_header(k1, kind, n, 1, s1, 1);
    Seed s[2] = {load_seed(s0), load_seed(s1)};
    uint32_t t[2] = {0, 1};
    Vec valpha{};
    const Vec ones = vec_keep_low(Vec{{~0u, ~0u, ~0u, ~0u}}, m);
    const uint32_t hi = alpha >> m, lo = alpha & ((1u << m) - 1u);
    for (int i = 1; i <= nu; i++) {
        Seed c[2][2];
        uint32_t tc[2][2];
        Vec v[2][2];
        for (int b = 0; b < 2; b++)
            for (int dir = 0; dir < 2; dir++) {
                expand(dir, s[b], &c[b][dir], &tc[b][dir]);
                if (dcf) v[b][dir] = value_vec(dir, s[b], m);
            }
        const uint32_t a = input_bit(hi, nu, i);
        const int keep = (int)a, lose = 1 - (int)a;
        Seed scw;
        for (int w = 0; w < 4; w++) scw.w[w] = c[0][lose].w[w] ^ c[1][lose].w[w];
        const uint32_t tlcw = tc[0][0] ^ tc[1][0] ^ a ^ 1u;
        const uint32_t trcw = tc[0][1] ^ tc[1][1] ^ a;
        const size_t off = 24 + (size_t)(i - 1) * lb;
        Vec vcw{};
        if (dcf) {
            vcw = vec_xor(vec_xor(v[0][lose], v[1][lose]), valpha);
            if (a) vcw = vec_xor(vcw, ones);
            valpha = vec_xor(vec_xor(valpha, vcw), vec_xor(v[0][keep], v[1][keep]));
        }
        for (uint8_t* k : {k0, k1}) {
            store_seed(k + off, scw);
            k[off + 16] = (uint8_t)tlcw;
            k[off + 17] = (uint8_t)trcw;
            k[off + 18] = k[off + 19] = 0;
            if (dcf) store_vec(k + off + 20, vcw);
        }
        const uint32_t tkeep = keep ? trcw : tlcw;
        for (int b = 0; b < 2; b++) {
            const uint32_t msk = 0u - t[b];
            for (int w = 0; w < 4; w++) s[b].w[w] = c[b][keep].w[w] ^ (scw.w[w] & msk);
            t[b] = tc[b][keep] ^ (t[b] & tkeep);
        }
    }
    Vec point{};
    if (dcf) {
        for (uint32_t j = 0; j < lo; j++) point.w[j / 32] |= 1u << (j % 32);
        point = vec_xor(point, valpha);
    } else {
        point.w[lo / 32] = 1u << (lo % 32);
    }
    const Vec cw = vec_xor(point, vec_xor(value_vec(0, s[0], m), value_vec(0, s[1], m)));
    store_vec(k0 + 24 + (size_t)nu * lb, cw);
    store_vec(k1 + 24 + (size_t)nu * lb, cw);
}

bool repack_key_et(const uint8_t* wire, size_t avail, uint32_t want_kind, int want_n, EtKey* out, std::string* err) {
    if (avail < 40) { *err = "key truncated"; return false; }
    const uint32_t kind = wire[0];
    const int n = wire[1];
    const uint32_t party = wire[2];
    if ((kind != OBLIVGM_KEY_DPF && kind != OBLIVGM_KEY_DCF) || (want_kind && kind != want_kind)) {
        *err = "unexpected key kind";
        return false;
    }
    if (n < 1 || n > kMaxOnehotBits || (want_n && n != want_n)) { *err = "key bit length mismatch"; return false; }
    if (party > 1 || wire[3] != 1) { *err = "bad key header"; return false; }
    if (avail < et_key_bytes(kind, n)) { *err = "key truncated"; return false; }
    std::memset(out, 0, sizeof *out);
    const int m = et_low_bits(n), nu = n - m;
    const size_t lb = kind == OBLIVGM_KEY_DPF ? 20 : 36;
    for (int w = 0; w < 4; w++) out->seed[w] = ld32(wire + 8 + 4 * w);
    for (int i = 0; i < nu; i++) {
        const uint8_t* lv = wire + 24 + i * lb;
        for (int w = 0; w < 4; w++) out->scw[i][w] = ld32(lv + 4 * w);
        if (lv[16] > 1 || lv[17] > 1) { *err = "bad control-bit correction"; return false; }
        out->tl |= (uint32_t)lv[16] << i;
        out->tr |= (uint32_t)lv[17] << i;
        if (kind == OBLIVGM_KEY_DCF)
            for (int w = 0; w < 4; w++) out->vcw[i][w] = ld32(lv + 20 + 4 * w);
    }
    for (int w = 0; w < 4; w++) out->cw_final[w] = ld32(wire + 24 + nu * lb + 4 * w);
    out->party = party;
    out->n = (uint32_t)n;
    out->kind = kind;
    out->low_bits = (uint32_t)m;
    out->levels = (uint32_t)nu;
    return true;
}

bool repack_key(const uint8_t* wire, size_t avail, uint32_t want_kind, int want_n, DevKey* out, std::string* err) {
    if (avail < 28) { *err = "key truncated"; return false; }
    const uint32_t kind = wire[0];
    const int n = wire[1];
    const uint32_t party = wire[2];
    if ((kind != OBLIVGM_KEY_DPF && kind != OBLIVGM_KEY_DCF) || (want_kind && kind != want_kind)) {
        *err = "unexpected key kind";
        return false;
    }
    if (n < 1 || n > kMaxBits || (want_n && n != want_n)) { *err = "key bit length mismatch"; return false; }
    if (party > 1 || wire[3] > 1) { *err = "bad key header"; return false; }
    if (avail < key_bytes(kind, n)) { *err = "key truncated"; return false; }
    std::memset(out, 0, sizeof *out);
    for (int w = 0; w < 4; w++) out->seed[w] = ld32(wire + 8 + 4 * w);
    const size_t lb = kind == OBLIVGM_KEY_DPF ? 20 : 24;
    for (int i = 0; i < n; i++) {
        const uint8_t* lv = wire + 24 + i * lb;
        for (int w = 0; w < 4; w++) out->scw[i][w] = ld32(lv + 4 * w);
        if (lv[16] > 1 || lv[17] > 1) { *err = "bad control-bit correction"; return false; }
        out->tl |= (uint32_t)lv[16] << i;
        out->tr |= (uint32_t)lv[17] << i;
        if (kind == OBLIVGM_KEY_DCF) out->vcw[i] = ld32(lv + 20);
    }
    out->cw_final = ld32(wire + 24 + n * lb);
    out->party = party;
    out->n = (uint32_t)n;
    out->kind = kind;
    out->group = wire[3];
    return true;
}

oblivgm_status parse_tokens(const uint8_t* const tok[3], const size_t tok_len[3], ParsedQuery* q, std::string* err) {
    if (!tok || !tok_len) { *err = "NULL token array"; return OBLIVGM_EINVAL; }
    int n = -1, np = -1;
    for (int i = 0; i < 3; i++) {
        const uint8_t* t = tok[i];
        if (!t || tok_len[i] < 16) { *err = "token missing or truncated"; return OBLIVGM_EINVAL; }
        if (ld32(t) != kTokenMagic || t[4] != 1 || t[5] != i + 1) { *err = "bad token header"; return OBLIVGM_EINVAL; }
        if (ld32(t + 12) != tok_len[i]) { *err = "token length field mismatch"; return OBLIVGM_EINVAL; }
        const int tn = t[6], tnp = ld16(t + 8);
        if (t[7] > 1 || t[7] != tok[0][7]) { *err = "bad or mismatched output group"; return OBLIVGM_EINVAL; }
        if (i == 0) { n = tn; np = tnp; }
        else if (tn != n || tnp != np) { *err = "tokens disagree on n or predicate count"; return OBLIVGM_EINVAL; }
    }
    if (n < 1 || n > kMaxBits || np < 1 || np > kMaxPreds) { *err = "token n or predicate count out of range"; return OBLIVGM_EINVAL; }
    const bool onehot = tok[0][7] == 1;
    if (onehot && n > kMaxOnehotBits) { *err = "one-hot token n above 16"; return OBLIVGM_EINVAL; }
    auto kbytes = [onehot](uint32_t kind, int nb) { return onehot ? et_key_bytes(kind, nb) : key_bytes(kind, nb); };
    q->n_bits = (uint32_t)n;
    q->out_group = tok[0][7];
    q->preds.clear();
    size_t off = 16;
    for (int p = 0; p < np; p++) {
        if (off + 24 > tok_len[0]) { *err = "token truncated"; return OBLIVGM_EINVAL; }
        const uint8_t* r0 = tok[0] + off;
        ParsedPred pp;
        pp.kind = r0[0];
        pp.n = r0[1];
        pp.table = ld16(r0 + 2);
        pp.attr = ld16(r0 + 4);
        pp.group = ld16(r0 + 6);
        pp.step = (uint32_t)p;
        if ((pp.kind != OBLIVGM_PRED_EQ && pp.kind != OBLIVGM_PRED_RANGE) || (int)pp.n != n) {
            *err = "bad predicate record";
            return OBLIVGM_EINVAL;
        }
        const uint32_t kkind = pp.kind == OBLIVGM_PRED_EQ ? OBLIVGM_KEY_DPF : OBLIVGM_KEY_DCF;
        const int nsub = pp.kind == OBLIVGM_PRED_EQ ? 1 : 2;
        const size_t half = nsub * kbytes(kkind, n);
        const size_t rec_len = 24 + 2 * half;
        for (int i = 0; i < 3; i++) {
            if (off + rec_len > tok_len[i]) { *err = "token truncated"; return OBLIVGM_EINVAL; }
            const uint8_t* ri = tok[i] + off;
            if (std::memcmp(ri, r0, 8) != 0) { *err = "tokens disagree on a predicate record"; return OBLIVGM_EINVAL; }
            pp.r[i] = ld32(ri + 8);
            if (ld32(ri + 16) != ld32(r0 + 16)) { *err = "tokens disagree on c*beta"; return OBLIVGM_EINVAL; }
        }
        // each server's second mask share must equal the next server's first
        for (int i = 0; i < 3; i++)
            if (ld32(tok[i] + off + 12) != pp.r[(i + 1) % 3]) { *err = "mask shares are not replicated"; return OBLIVGM_EINVAL; }
        pp.cbeta = ld32(r0 + 16);
        for (int i = 1; i < 3; i++)
            if (ld32(tok[i] + off + 20) != ld32(r0 + 20)) { *err = "tokens disagree on the combine field"; return OBLIVGM_EINVAL; }
        pp.combine = r0[20];
        if (pp.combine > OBLIVGM_COMBINE_OR || r0[21] || r0[22] || r0[23]) { *err = "bad combine field"; return OBLIVGM_EINVAL; }
        bool first_of_group = true;
        for (const ParsedPred& e : q->preds) first_of_group = first_of_group && e.group != pp.group;
        if (first_of_group && pp.combine != OBLIVGM_COMBINE_AND) {
            *err = "a group's first predicate must combine with AND";
            return OBLIVGM_EINVAL;
        }
        if (onehot) pp.et_keys.resize(6 * nsub);
        else pp.keys.resize(6 * nsub);
        for (int i = 0; i < 3; i++)
            for (int h = 0; h < 2; h++)
                for (int s = 0; s < nsub; s++) {
                    const uint8_t* kw = tok[i] + off + 24 + h * half + s * kbytes(kkind, n);
                    const size_t avail = tok_len[i] - (size_t)(kw - tok[i]);
                    if (onehot) {
                        if (!repack_key_et(kw, avail, kkind, n, &pp.et_keys[(i * 2 + h) * nsub + s], err))
                            return OBLIVGM_EINVAL;
                        continue;
                    }
                    DevKey& dk = pp.keys[(i * 2 + h) * nsub + s];
                    if (!repack_key(kw, avail, kkind, n, &dk, err))
                        return OBLIVGM_EINVAL;
                    if (dk.group != q->out_group) { *err = "key output group differs from the token's"; return OBLIVGM_EINVAL; }
                }
        q->preds.push_back(std::move(pp));
        off += rec_len;
    }
    for (int i = 0; i < 3; i++)
        if (off != tok_len[i]) { *err = "trailing bytes in token"; return OBLIVGM_EINVAL; }
    return OBLIVGM_OK;
}

bool check_combine(const oblivgm_pred* preds, uint32_t n_preds, std::string* err) {
    for (uint32_t p = 0; p < n_preds; p++) {
        if (preds[p].combine > OBLIVGM_COMBINE_OR) { *err = "combine must be AND, XOR or OR"; return false; }
        bool first_of_group = true;
        for (uint32_t e = 0; e < p; e++) first_of_group = first_of_group && preds[e].group != preds[p].group;
        if (first_of_group && preds[p].combine != OBLIVGM_COMBINE_AND) {
            *err = "a group's first predicate must combine with AND";
            return false;
        }
    }
    return true;
}

oblivgm_status keygen(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits, const uint8_t seed[16],
                      uint8_t* const tok[3], size_t cap, size_t out_len[3], std::string* err, bool onehot) {
    if (!preds || !seed || !out_len) { *err = "NULL argument"; return OBLIVGM_EINVAL; }
    if (n_preds == 0 || n_preds > (uint32_t)kMaxPreds) { *err = "predicate count must be 1..64"; return OBLIVGM_EINVAL; }
    if (n_bits < 1 || n_bits > (uint32_t)(onehot ? kMaxOnehotBits : kMaxBits)) {
        *err = onehot ? "one-hot n must be 1..16" : "n must be 1..32";
        return OBLIVGM_EINVAL;
    }
    const int group = onehot ? 1 : 0;
    const int n = (int)n_bits;
    const uint32_t m = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const size_t dpf = onehot ? et_key_bytes(OBLIVGM_KEY_DPF, n) : key_bytes(OBLIVGM_KEY_DPF, n);
    const size_t dcf = onehot ? et_key_bytes(OBLIVGM_KEY_DCF, n) : key_bytes(OBLIVGM_KEY_DCF, n);
    size_t total = 16;
    for (uint32_t p = 0; p < n_preds; p++) {
        const oblivgm_pred& q = preds[p];
        if (q.kind == OBLIVGM_PRED_EQ) {
            if (q.lo > m) { *err = "equality value outside the domain"; return OBLIVGM_EINVAL; }
            total += 24 + 2 * dpf;
        } else if (q.kind == OBLIVGM_PRED_RANGE) {
            if (q.lo > q.hi || q.hi > m) { *err = "empty range or bound outside the domain"; return OBLIVGM_EINVAL; }
            total += 24 + 4 * dcf;
        } else {
            *err = "unknown predicate kind";
            return OBLIVGM_EINVAL;
        }
        if (q.table > 0xFFFF || q.attr > 0xFFFF || q.group > 0xFFFF) { *err = "id above 65535"; return OBLIVGM_EINVAL; }
    }
    if (!check_combine(preds, n_preds, err)) return OBLIVGM_EINVAL;
    for (int i = 0; i < 3; i++) out_len[i] = total;
    if (!tok || !tok[0] || !tok[1] || !tok[2]) return OBLIVGM_OK;   // size query
    if (cap < total) { *err = "token buffer too small"; return OBLIVGM_ERANGE; }

    const RoundKeys rng_key = expand_key(seed);
    uint64_t ctr = 0;
    auto next_block = [&](uint8_t out[16]) {
        const uint32_t in[4] = {(uint32_t)ctr, (uint32_t)(ctr >> 32), 0u, 0u};
        uint32_t o[4];
        aes_encrypt(rng_key, in, o);
        for (int w = 0; w < 4; w++) st32(out + 4 * w, o[w]);
        ctr++;
    };
    for (int i = 0; i < 3; i++) {
        uint8_t* h = tok[i];
        std::memset(h, 0, 16);
        st32(h, kTokenMagic);
        h[4] = 1;
        h[5] = (uint8_t)(i + 1);
        h[6] = (uint8_t)n;
        h[7] = (uint8_t)group;
        h[8] = (uint8_t)n_preds;
        h[9] = (uint8_t)(n_preds >> 8);
        st32(h + 12, (uint32_t)total);
    }
    // halves held by server i: (pair, party) -- CS1 (1,0),(2,0); CS2 (2,1),(3,0); CS3 (3,1),(1,1)
    static const int kPair[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    static const int kParty[3][2] = {{0, 0}, {1, 0}, {1, 1}};
    std::vector<uint8_t> keys;
    size_t off = 16;
    for (uint32_t p = 0; p < n_preds; p++) {
        const oblivgm_pred& q = preds[p];
        // masked mode: a fresh mask r, replicated-shared; one-hot mode: no mask
        uint32_t r = 0, rs[3] = {0, 0, 0};
        if (!onehot) {
            uint8_t blk[16];
            next_block(blk);
            r = ld32(blk) & m;
            rs[0] = ld32(blk + 4) & m;
            rs[1] = ld32(blk + 8) & m;
            rs[2] = (r - rs[0] - rs[1]) & m;
        }
        const uint32_t beta = onehot ? 1u : kBetaPrime;
        const bool eq = q.kind == OBLIVGM_PRED_EQ;
        const size_t half = eq ? dpf : 2 * dcf;
        keys.assign(3 * 2 * half, 0);   // [pair][party][half]
        uint32_t cbeta = 0;
        const uint32_t a_eq = (q.lo + r) & m;
        const uint32_t a0 = (q.lo + r) & m, a1 = (q.hi + 1u + r) & m;
        if (!eq) cbeta = a1 <= a0 ? beta : 0u;
        for (int j = 0; j < 3; j++) {
            uint8_t* kp0 = keys.data() + (j * 2 + 0) * half;
            uint8_t* kp1 = keys.data() + (j * 2 + 1) * half;
            uint8_t s0[16], s1[16];
            next_block(s0);
            next_block(s1);
            if (eq) {
                if (onehot) gen_et(OBLIVGM_KEY_DPF, n, a_eq, s0, s1, kp0, kp1);
                else dpf_gen(n, a_eq, beta, s0, s1, kp0, kp1, group);
            } else {
                if (onehot) gen_et(OBLIVGM_KEY_DCF, n, a1, s0, s1, kp0, kp1);
                else dcf_gen(n, a1, beta, s0, s1, kp0, kp1, group);
                next_block(s0);
                next_block(s1);
                // over Z_2, -beta = beta = 1
                if (onehot) gen_et(OBLIVGM_KEY_DCF, n, a0, s0, s1, kp0 + dcf, kp1 + dcf);
                else dcf_gen(n, a0, 0u - beta, s0, s1, kp0 + dcf, kp1 + dcf, group);
            }
        }
        for (int i = 0; i < 3; i++) {
            uint8_t* rec = tok[i] + off;
            std::memset(rec, 0, 24);
            rec[0] = (uint8_t)q.kind;
            rec[1] = (uint8_t)n;
            rec[2] = (uint8_t)q.table; rec[3] = (uint8_t)(q.table >> 8);
            rec[4] = (uint8_t)q.attr;  rec[5] = (uint8_t)(q.attr >> 8);
            rec[6] = (uint8_t)q.group; rec[7] = (uint8_t)(q.group >> 8);
            st32(rec + 8, rs[i]);
            st32(rec + 12, rs[(i + 1) % 3]);
            st32(rec + 16, cbeta);
            rec[20] = (uint8_t)q.combine;
            for (int h = 0; h < 2; h++)
                std::memcpy(rec + 24 + h * half, keys.data() + (kPair[i][h] * 2 + kParty[i][h]) * half, half);
        }
        off += 24 + 2 * half;
    }
    return OBLIVGM_OK;
}

}  // namespace ogm
