// device_fss.cuh -- sm_103a device code of the oblivgm library: AES-128 from
// bank-replicated shared-memory T-tables, the fixed-key PRG, and one tree
// walk of DPF Eval / DCF Eval per (key, input) for E inputs per thread.
//
// Shared-memory table layout (128 KiB, dynamic shared memory offset 0):
//   table k in {0,1,2,3} = rotl(Te0, 8k); entry idx of table k for lane L sits
//   at byte (k >> 1) * 65536 + idx * 256 + (k & 1) * 128 + L * 4, so every lane
//   reads its own bank and a warp-wide lookup is conflict-free for any indices.
//   One PRMT builds idx * 256 + L * 4 from a state byte and the lane offset.
#pragma once
#include <cstdint>

#include "host_crypto.h"

namespace ogm {

constexpr int kTableBytes = 131072;

__device__ __forceinline__ uint32_t lane_offset() { return (threadIdx.x & 31u) * 4u; }

// Fill the replicated tables from the compact Te0 (256 words in global memory).  Each of
// the 1,024 (table, entry) pairs is one word replicated for the 32 lanes (128 bytes): eight
// threads write a pair with one 16-byte store each, so a warp's store covers four whole
// 128-byte rows (four wavefronts, no bank conflict).
__device__ __forceinline__ void fill_tables(uint32_t* tab, const uint32_t* __restrict__ te0) {
#pragma unroll 4
    for (int i = threadIdx.x; i < 4 * 256 * 8; i += blockDim.x) {
        const int pair = i >> 3, chunk = i & 7;
        const int k = pair >> 8, idx = pair & 255;
        const uint32_t w = __ldg(te0 + idx);
        const uint32_t v = __funnelshift_l(w, w, 8 * k);
        reinterpret_cast<uint4*>(tab + (k >> 1) * 16384 + idx * 64 + (k & 1) * 32)[chunk] = make_uint4(v, v, v, v);
    }
}

// Table access policies.  SmemTab: the bank-replicated shared-memory tables above
// (lookup of table TABLE at byte BYTE of column col).  GlobalTab: the four 1 KiB
// tables read straight from global memory through L1 (the plain path's layout).
struct SmemTab {
    const char* T;
    uint32_t lane4;
    template <int BYTE, int TABLE>
    __device__ __forceinline__ uint32_t lu(uint32_t col) const {
        const uint32_t off = __byte_perm(col, lane4, 0x5504u | (BYTE << 4));   // lane4 | byte << 8
        return *reinterpret_cast<const uint32_t*>(T + off + ((TABLE >> 1) * 65536 + (TABLE & 1) * 128));
    }
};

struct GlobalTab {
    const uint32_t* __restrict__ te;   // te[k * 256 + x] = rotl(Te0[x], 8 k)
    template <int BYTE, int TABLE>
    __device__ __forceinline__ uint32_t lu(uint32_t col) const {
        return __ldg(te + TABLE * 256 + ((col >> (8 * BYTE)) & 0xFFu));
    }
};

// One full AES round on four columns (SubBytes, ShiftRows, MixColumns, AddRoundKey).
template <class Tab>
__device__ __forceinline__ void aes_round(const Tab& T, uint32_t c[4], uint32_t k0, uint32_t k1, uint32_t k2,
                                          uint32_t k3) {
    const uint32_t n0 = T.template lu<0, 0>(c[0]) ^ T.template lu<1, 1>(c[1]) ^ T.template lu<2, 2>(c[2]) ^ T.template lu<3, 3>(c[3]) ^ k0;
    const uint32_t n1 = T.template lu<0, 0>(c[1]) ^ T.template lu<1, 1>(c[2]) ^ T.template lu<2, 2>(c[3]) ^ T.template lu<3, 3>(c[0]) ^ k1;
    const uint32_t n2 = T.template lu<0, 0>(c[2]) ^ T.template lu<1, 1>(c[3]) ^ T.template lu<2, 2>(c[0]) ^ T.template lu<3, 3>(c[1]) ^ k2;
    const uint32_t n3 = T.template lu<0, 0>(c[3]) ^ T.template lu<1, 1>(c[0]) ^ T.template lu<2, 2>(c[1]) ^ T.template lu<3, 3>(c[2]) ^ k3;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

// S-box byte r of the final round comes from table (r + 3) % 4, whose byte r holds S[x].
template <class Tab>
__device__ __forceinline__ uint32_t last_col(const Tab& T, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    const uint32_t x0 = T.template lu<0, 3>(a), x1 = T.template lu<1, 0>(b), x2 = T.template lu<2, 1>(c),
                   x3 = T.template lu<3, 2>(d);
    return __byte_perm(__byte_perm(x0, x1, 0x3250u), __byte_perm(x2, x3, 0x7210u), 0x7610u);
}

template <class Tab>
__device__ __forceinline__ void aes_last(const Tab& T, uint32_t c[4], uint32_t k0, uint32_t k1, uint32_t k2,
                                         uint32_t k3) {
    const uint32_t n0 = last_col(T, c[0], c[1], c[2], c[3]) ^ k0;
    const uint32_t n1 = last_col(T, c[1], c[2], c[3], c[0]) ^ k1;
    const uint32_t n2 = last_col(T, c[2], c[3], c[0], c[1]) ^ k2;
    const uint32_t n3 = last_col(T, c[3], c[0], c[1], c[2]) ^ k3;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

// AES-128 under round keys rk ^ (m & d): m = 0 selects key A, m = ~0 key B.
template <class Tab>
__device__ __forceinline__ void aes_sel(const Tab& T, const uint32_t* rk, const uint32_t* d, uint32_t m,
                                        const uint32_t in[4], uint32_t out[4]) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk[j] ^ (m & d[j]);
#pragma unroll
    for (int r = 1; r < 10; r++)
        aes_round(T, c, rk[4 * r] ^ (m & d[4 * r]), rk[4 * r + 1] ^ (m & d[4 * r + 1]),
                  rk[4 * r + 2] ^ (m & d[4 * r + 2]), rk[4 * r + 3] ^ (m & d[4 * r + 3]));
    aes_last(T, c, rk[40] ^ (m & d[40]), rk[41] ^ (m & d[41]), rk[42] ^ (m & d[42]), rk[43] ^ (m & d[43]));
#pragma unroll
    for (int j = 0; j < 4; j++) out[j] = c[j];
}

// Word 0 (bytes 0..3) of AES-128 under rk ^ (m & d): the final round computes only the
// output column it needs (4 lookups instead of 16).
template <class Tab>
__device__ __forceinline__ uint32_t aes_sel_w0(const Tab& T, const uint32_t* rk, const uint32_t* d, uint32_t m,
                                               const uint32_t in[4]) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk[j] ^ (m & d[j]);
#pragma unroll
    for (int r = 1; r < 10; r++)
        aes_round(T, c, rk[4 * r] ^ (m & d[4 * r]), rk[4 * r + 1] ^ (m & d[4 * r + 1]),
                  rk[4 * r + 2] ^ (m & d[4 * r + 2]), rk[4 * r + 3] ^ (m & d[4 * r + 3]));
    return last_col(T, c[0], c[1], c[2], c[3]) ^ rk[40] ^ (m & d[40]);
}

// Word 0 of AES-128 under one key.
template <class Tab>
__device__ __forceinline__ uint32_t aes_one_w0(const Tab& T, const uint32_t* rk, const uint32_t in[4]) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk[j];
#pragma unroll
    for (int r = 1; r < 10; r++) aes_round(T, c, rk[4 * r], rk[4 * r + 1], rk[4 * r + 2], rk[4 * r + 3]);
    return last_col(T, c[0], c[1], c[2], c[3]) ^ rk[40];
}

// AES-128 under one key.
template <class Tab>
__device__ __forceinline__ void aes_one(const Tab& T, const uint32_t* rk, const uint32_t in[4], uint32_t out[4]) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk[j];
#pragma unroll
    for (int r = 1; r < 10; r++) aes_round(T, c, rk[4 * r], rk[4 * r + 1], rk[4 * r + 2], rk[4 * r + 3]);
    aes_last(T, c, rk[40], rk[41], rk[42], rk[43]);
#pragma unroll
    for (int j = 0; j < 4; j++) out[j] = c[j];
}

// DPF Eval (BGI16) of one key at E inputs: per level one PRG call for the child
// the input bit selects, the conditional correction, and at the end
// (-1)^b (Convert(s) + t * CW_{n+1}).
// Z2 = true: output group Z_2 (one-hot mode): Convert(seed) = bit 1 of byte 0, the result mod 2.
template <int E, class Tab, bool Z2 = false>
__device__ __forceinline__ void dpf_walk(const Tab& T, const AesParams& A, const DevKey& K, const uint32_t xh[E],
                                         uint32_t y[E]) {
    uint32_t s[E][4], t[E];
    const uint32_t party = K.party;
#pragma unroll
    for (int e = 0; e < E; e++) {
#pragma unroll
        for (int w = 0; w < 4; w++) s[e][w] = K.seed[w];
        t[e] = party;
    }
    const int n = (int)K.n;
    const uint32_t tl = K.tl, tr = K.tr;
    for (int i = 0; i < n; i++) {
        const uint4 cw = *reinterpret_cast<const uint4*>(K.scw[i]);
        const int sh = n - 1 - i;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint32_t dir = (xh[e] >> sh) & 1u;
            uint32_t o[4];
            aes_sel(T, A.rk_st, A.d_st, 0u - dir, s[e], o);
#pragma unroll
            for (int w = 0; w < 4; w++) o[w] ^= s[e][w];
            uint32_t tn = o[0] & 1u;
            o[0] &= ~1u;
            const uint32_t tm = 0u - t[e];
            s[e][0] = o[0] ^ (cw.x & tm);
            s[e][1] = o[1] ^ (cw.y & tm);
            s[e][2] = o[2] ^ (cw.z & tm);
            s[e][3] = o[3] ^ (cw.w & tm);
            tn ^= t[e] & (((dir ? tr : tl) >> i) & 1u);
            t[e] = tn;
        }
    }
    const uint32_t cwf = K.cw_final;
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t conv = Z2 ? ((s[e][0] >> 1) & 1u) : s[e][1];
        const uint32_t v = conv + (t[e] ? cwf : 0u);
        y[e] = (party ? 0u - v : v) & (Z2 ? 1u : 0xFFFFFFFFu);
    }
}

// DCF Eval (BCG+21) of one key at E inputs: per level the seed/control block and
// the value block of the selected child (two PRG calls on the same seed),
// V += (-1)^b (Convert(v) + t * V_CW), then the final term.
template <int E, class Tab, bool Z2 = false>
__device__ __forceinline__ void dcf_walk(const Tab& T, const AesParams& A, const DevKey& K, const uint32_t xh[E],
                                         uint32_t y[E]) {
    uint32_t s[E][4], t[E], V[E];
    const uint32_t party = K.party;
#pragma unroll
    for (int e = 0; e < E; e++) {
#pragma unroll
        for (int w = 0; w < 4; w++) s[e][w] = K.seed[w];
        t[e] = party;
        V[e] = 0;
    }
    const int n = (int)K.n;
    const uint32_t tl = K.tl, tr = K.tr;
    for (int i = 0; i < n; i++) {
        const uint4 cw = *reinterpret_cast<const uint4*>(K.scw[i]);
        const uint32_t vcw = K.vcw[i];
        const int sh = n - 1 - i;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint32_t dir = (xh[e] >> sh) & 1u;
            const uint32_t m = 0u - dir;
            uint32_t o[4];
            aes_sel(T, A.rk_st, A.d_st, m, s[e], o);
            const uint32_t v0 = aes_sel_w0(T, A.rk_v, A.d_v, m, s[e]);   // Convert(v) needs bytes 0..3 only
            const uint32_t vconv = Z2 ? ((v0 ^ s[e][0]) & 1u) : (v0 ^ s[e][0]);
            const uint32_t term = vconv + (t[e] ? vcw : 0u);
            V[e] += party ? 0u - term : term;
#pragma unroll
            for (int w = 0; w < 4; w++) o[w] ^= s[e][w];
            uint32_t tn = o[0] & 1u;
            o[0] &= ~1u;
            const uint32_t tm = 0u - t[e];
            s[e][0] = o[0] ^ (cw.x & tm);
            s[e][1] = o[1] ^ (cw.y & tm);
            s[e][2] = o[2] ^ (cw.z & tm);
            s[e][3] = o[3] ^ (cw.w & tm);
            tn ^= t[e] & (((dir ? tr : tl) >> i) & 1u);
            t[e] = tn;
        }
    }
    const uint32_t cwf = K.cw_final;
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t conv = Z2 ? ((s[e][0] >> 1) & 1u) : s[e][1];
        const uint32_t term = conv + (t[e] ? cwf : 0u);
        y[e] = (V[e] + (party ? 0u - term : term)) & (Z2 ? 1u : 0xFFFFFFFFu);
    }
}

}  // namespace ogm
