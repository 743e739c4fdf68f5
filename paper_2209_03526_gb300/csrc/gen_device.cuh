// gen_device.cuh -- DPF / DCF Gen of one key pair on the device, for the batched key
// generation kernels.  The construction is the host's (BGI16 tree DPF, Boyle et al. DCF;
// H_K(s) = AES_K(s) xor s under the fixed keys, control bit = bit 0 of byte 0 of a child
// seed, Convert = bytes 4..7 of a seed / bytes 0..3 of a value block, input bits MSB
// first).  The correction words go to a Sink, which decides the key layout:
//   sink.level(lv, scw[4], tl, tr, vcw)   level lv = 0..n-1 (vcw only for DCF)
//   sink.final(cw)                        CW_{n+1}
#pragma once

#include <cstdint>

#include "device_fss.cuh"

namespace ogm {

// The round keys of the right-child PRG keys (K_R for the seed / control-bit block, K_vR
// for the DCF value block); the left-child ones are AesParams::rk_st and rk_v.  Gen
// expands both children of every node, so each AES runs under a fixed key.
struct GenRightKeys {
    uint32_t st[44];
    uint32_t v[44];
};

// child of a seed under the round keys rk of its direction: seed with bit 0 of byte 0
// cleared, control bit apart
__device__ __forceinline__ void gen_expand(const SmemTab& T, const uint32_t* rk, const uint32_t s[4], uint32_t cs[4],
                                           uint32_t& ct) {
    uint32_t o[4];
    aes_one(T, rk, s, o);
#pragma unroll
    for (int w = 0; w < 4; w++) cs[w] = o[w] ^ s[w];
    ct = cs[0] & 1u;
    cs[0] &= ~1u;
}

// Gen of f^=_{alpha,beta} (DCF = false) or g^<_{alpha,beta} (DCF = true) over Z_{2^32}
// from the root seeds s0, s1 (overwritten).  No runtime-indexed arrays: the L/R and
// keep/lose choices are selects, so everything stays in registers.  One instance per
// kind keeps the DPF loop free of the DCF's value blocks.
template <bool DCF, class Sink>
__device__ __forceinline__ void gen_pair(const SmemTab& T, const AesParams& A, const GenRightKeys& R, int n,
                                         uint32_t alpha, uint32_t beta, uint32_t s0[4], uint32_t s1[4], Sink& sink) {
    constexpr bool dcf = DCF;
    uint32_t t0 = 0u, t1 = 1u, valpha = 0u;
    for (int lv = 1; lv <= n; lv++) {
        uint32_t c0l[4], c0r[4], c1l[4], c1r[4], t0l, t0r, t1l, t1r;
        gen_expand(T, A.rk_st, s0, c0l, t0l);
        gen_expand(T, R.st, s0, c0r, t0r);
        gen_expand(T, A.rk_st, s1, c1l, t1l);
        gen_expand(T, R.st, s1, c1r, t1r);
        const uint32_t a = (alpha >> (n - lv)) & 1u;
        const uint32_t tl = t0l ^ t1l ^ a ^ 1u, tr = t0r ^ t1r ^ a;
        uint32_t scw[4];
#pragma unroll
        for (int w = 0; w < 4; w++) scw[w] = a ? (c0l[w] ^ c1l[w]) : (c0r[w] ^ c1r[w]);   // CW on the lose side
        uint32_t vcw = 0u;
        if (dcf) {
            const uint32_t v0l = aes_one_w0(T, A.rk_v, s0) ^ s0[0];
            const uint32_t v0r = aes_one_w0(T, R.v, s0) ^ s0[0];
            const uint32_t v1l = aes_one_w0(T, A.rk_v, s1) ^ s1[0];
            const uint32_t v1r = aes_one_w0(T, R.v, s1) ^ s1[0];
            const uint32_t v0_lose = a ? v0l : v0r, v1_lose = a ? v1l : v1r;
            const uint32_t v0_keep = a ? v0r : v0l, v1_keep = a ? v1r : v1l;
            const bool neg = t1 != 0;
            vcw = v1_lose - v0_lose - valpha;
            if (neg) vcw = 0u - vcw;
            if (a) vcw += neg ? 0u - beta : beta;          // lose side is L: inputs below alpha
            valpha = valpha - v1_keep + v0_keep + (neg ? 0u - vcw : vcw);
        }
        sink.level(lv - 1, scw, tl, tr, vcw);
        const uint32_t tkeep = a ? tr : tl;
        const uint32_t m0 = 0u - t0, m1 = 0u - t1;
#pragma unroll
        for (int w = 0; w < 4; w++) {
            s0[w] = (a ? c0r[w] : c0l[w]) ^ (scw[w] & m0);
            s1[w] = (a ? c1r[w] : c1l[w]) ^ (scw[w] & m1);
        }
        t0 = (a ? t0r : t0l) ^ (t0 & tkeep);
        t1 = (a ? t1r : t1l) ^ (t1 & tkeep);
    }
    uint32_t cw = dcf ? s1[1] - s0[1] - valpha : beta - s0[1] + s1[1];
    if (t1) cw = 0u - cw;
    sink.final(cw);
}

}  // namespace ogm
