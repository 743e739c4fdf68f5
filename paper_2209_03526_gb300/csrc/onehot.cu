// onehot.cu -- the one-hot mode of the oblivgm library: secEval exactly as the
// paper writes it (Sec. V-B, V-C, Eq. predEval, Alg. 3).  Attribute values are
// stored as binary-RSS shares of one-hot vectors of length D = 2^n (n <= 16),
// packed 32 positions per word.  Each server evaluates its FSS key halves (Z_2
// outputs, beta = 1) at every public position l and computes
//     x = XOR_l Eval(k, l) AND <e_v>_j[l]
// for the share j its key pair is tied to; it XORs its two results, re-shares them
// in binary RSS and the query element's predicates are folded (AND, XOR or OR) in binary RSS.
//
// Three steps per query:
//  * EvalAll, every key half at every position: the keys stop their trees early (a
//    leaf seed expands into the outputs of 2^min(n,7) consecutive positions, BGI16's
//    early termination for small output groups), and k_onehot_evalall_et gives each
//    (key, leaf) a lane pair that walks the n - 7 levels (seed chain and DCF value
//    chain side by side) and writes the leaf's 128 bits;
//  * the dot pass, one streaming pass over an attribute column's three share rows for
//    up to 4 predicates on that column: k_onehot_dots_pipe (D >= 2^12, persistent,
//    rows staged by per-lane cp.async, warps splitting the rows, each lane holding its
//    slice of the half vectors in registers) or k_onehot_dots (smaller D); parities
//    are XOR-reduced over the warp and each server's bit written packed;
//  * k_onehot_fold: every group in one launch, each element's bits re-shared in
//    binary RSS and folded in token order on whole 32-element words (one PRF AES
//    block from the shared-memory T-tables serves 128 elements); results are packed
//    32 elements per word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "device_fss.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "ptx_async.cuh"
#include "runtime.h"

namespace ogm {

namespace {

constexpr uint32_t kNoKey = 0xFFFFFFFFu;

struct HalfDesc {
    uint32_t key0, key1;   // one DPF key, or two DCF keys (a1, a0); key1 = kNoKey for DPF
    uint32_t cbit;         // public constant XORed in by party 0 of a range half
    uint32_t kind;         // OBLIVGM_KEY_DPF / OBLIVGM_KEY_DCF
};

struct KeySlot {
    uint32_t key;       // index into the keys
    uint32_t half;      // the half vector it is XORed into
    uint32_t cmask;     // all ones where party 0 of a range half adds the public constant
    uint32_t dcf;
};

struct EvalEtParams {
    AesParams aes;
    const uint32_t* te0;
    const EtKey* keys;
    const KeySlot* slots;
    uint32_t* hv;          // [half][words], zeroed before the launch
    uint32_t words;        // max(1, 2^n / 32)
    uint32_t leaves;       // 2^nu leaf seeds per key
    uint32_t n_slots;
};

// AES-128 whose round keys depend on the lane: key A (rkA ^ (m & dA)) where r = 0, key B
// (rkB ^ (m & dB)) where r = ~0.  The four schedules are launch parameters (uniform
// operands); the per-lane choice costs three LOP3s per round-key word.
template <class Tab>
__device__ __forceinline__ void aes_two_keys(const Tab& T, const uint32_t* rkA, const uint32_t* dA,
                                             const uint32_t* rkB, const uint32_t* dB, uint32_t m, uint32_t r,
                                             const uint32_t in[4], uint32_t out[4]) {
    auto key = [&](int w) {
        const uint32_t a = rkA[w] ^ (m & dA[w]), b = rkB[w] ^ (m & dB[w]);
        return a ^ ((a ^ b) & r);
    };
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ key(j);
#pragma unroll
    for (int rd = 1; rd < 10; rd++) aes_round(T, c, key(4 * rd), key(4 * rd + 1), key(4 * rd + 2), key(4 * rd + 3));
    aes_last(T, c, key(40), key(41), key(42), key(43));
#pragma unroll
    for (int j = 0; j < 4; j++) out[j] = c[j];
}

// Every key at every position.  Work item = (key slot, leaf), taken by a pair of lanes:
// at each of the nu levels the even lane computes the chosen child's seed block and the
// odd lane, for a DCF, its value block H_{K_vdir}(s) on the same seed (for a DPF its
// block is not used); the new seed and control bit reach the odd lane by shuffles.  The
// odd lane then expands the leaf seed into the 2^m output bits of positions
// leaf * 2^m + j,
//   y = V ^ H_{K_vL}(s) ^ t CW,
// and XORs them into the slot's half vector (a range half's two DCF keys land in the same
// words).  At n = 16 a key has 512 leaves of 9 levels: 36 keys are 18,432 items.
constexpr int kEvalEtMaxThreads = 512;

__global__ void __launch_bounds__(kEvalEtMaxThreads, 1) k_onehot_evalall_et(const __grid_constant__ EvalEtParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t lane = threadIdx.x & 31, role = lane & 1u, rmask = 0u - role, even = lane & ~1u;
    const uint64_t items = (uint64_t)P.n_slots * P.leaves;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x / 2;
    // the warp's first pair: the loop bound is the same for every lane of the warp, so the
    // shuffles below always have all 32 lanes; a pair past the end repeats the last item
    // and writes nothing
    const uint64_t warp_first = ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) / 2;
    for (uint64_t wf = warp_first; wf < items; wf += stride) {
        const uint64_t idx = wf + lane / 2;
        const bool live = idx < items;
        const uint64_t it = live ? idx : items - 1;
        const uint32_t slot = (uint32_t)(it / P.leaves), leaf = (uint32_t)(it % P.leaves);
        const KeySlot S = P.slots[slot];
        const EtKey& K = P.keys[S.key];
        const int nu = (int)K.levels, m = (int)K.low_bits;
        const uint32_t vmask = S.dcf ? rmask : 0u;    // the value chain runs on the odd lane of a DCF pair
        uint32_t s[4] = {K.seed[0], K.seed[1], K.seed[2], K.seed[3]};
        uint32_t t = K.party, V[4] = {0u, 0u, 0u, 0u};
        for (int i = 0; i < nu; i++) {
            const uint32_t dir = (leaf >> (nu - 1 - i)) & 1u, dm = 0u - dir, tm = 0u - t;
            uint32_t o[4];
            aes_two_keys(T, P.aes.rk_st, P.aes.d_st, P.aes.rk_v, P.aes.d_v, dm, rmask, s, o);
#pragma unroll
            for (int w = 0; w < 4; w++) {
                o[w] ^= s[w];
                V[w] ^= (o[w] ^ (K.vcw[i][w] & tm)) & vmask;
            }
            uint32_t tn = (o[0] & 1u) ^ (t & (((dir ? K.tr : K.tl) >> i) & 1u));
            o[0] &= ~1u;
#pragma unroll
            for (int w = 0; w < 4; w++) s[w] = __shfl_sync(0xFFFFFFFFu, o[w] ^ (K.scw[i][w] & tm), even);
            t = __shfl_sync(0xFFFFFFFFu, tn, even);
        }
        uint32_t c[4];
        aes_sel(T, P.aes.rk_v, P.aes.d_v, 0u, s, c);
        const uint32_t tm = 0u - t;
        const uint32_t bits = 1u << m;
        const uint32_t nw = bits >= 32 ? bits / 32 : 1u;
        const uint32_t keep = bits >= 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
        uint32_t* dst = P.hv + (uint64_t)S.half * P.words + (uint64_t)leaf * nw;
        if (live && role) {
#pragma unroll
            for (uint32_t w = 0; w < 4; w++)
                if (w < nw) atomicXor(dst + w, (V[w] ^ c[w] ^ s[w] ^ (K.cw_final[w] & tm) ^ S.cmask) & keep);
        }
    }
}

constexpr int kDotPreds = 4;   // predicates one streaming pass over a column serves

// Pass over one attribute column for up to kDotPreds predicates on it: every element's
// three share rows are read once and ANDed with the six half vectors of each predicate.
// Output: per predicate and server, the bit z_i = x(first half) xor x(second half),
// packed 32 elements per word into zbits[pred][server][word].
struct DotParams {
    const uint32_t* share[3];     // share set j at the column's first element: [elem][words]
    const uint32_t* hv;           // [half][words]
    uint32_t half_base[kDotPreds];
    uint32_t* zbits[kDotPreds];   // [3][ceil(n_elems / 32)] each
    uint64_t n_elems;
    uint32_t words;
    uint32_t n_preds;
    uint32_t pow2[32];            // pow2[i] = 2^i (read at run time by the staged pass)
};

// The unstaged pass, launched for domains below 2^12 and general in W.  One CTA per 32
// elements (one packed output word).  The CTA's warps split each share row: with
// W >= 128 words warp q covers words [128 q, 128 q + 128) of every row in steps of
// W' = 128 * warps (one uint4 per lane when W' = W); with W < 128 one warp reads the row
// word by word.  A lane keeps its slice of the predicates' half vectors in registers for
// all 32 elements and streams 8 elements' rows at a time; its parity bits of the 32
// elements are XORed over the warp by shuffles and over the warps through shared memory.
constexpr int kDotBatch = 8;

__device__ __forceinline__ void slice4(const uint32_t* row, uint32_t W, bool vec, uint32_t w0, uint32_t lane,
                                       uint32_t out[4]) {
    if (vec) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + w0));
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else {
#pragma unroll
        for (int r = 0; r < 4; r++) out[r] = lane + 32u * r < W ? __ldg(row + lane + 32u * r) : 0u;
    }
}

__global__ void __launch_bounds__(512) k_onehot_dots(const __grid_constant__ DotParams P) {
    __shared__ uint32_t zs[16][kDotPreds][3][2];      // per warp: element masks per (pred, share, half)
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const uint32_t W = P.words, np = P.n_preds;
    const bool vec = W >= 128;
    const uint64_t nwords = (P.n_elems + 31) / 32;
    const uint64_t wd = blockIdx.x;
    const uint64_t base = wd * 32;
    // lane 0 of each warp owns the warp's slots: cleared here, XORed into below
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kDotPreds; k++)
#pragma unroll
            for (int j = 0; j < 3; j++) zs[warp][k][j][0] = zs[warp][k][j][1] = 0;
    }
    // a lane's words: w0 .. w0 + 3 (vector path) or lane + 32 r (scalar path); the vector
    // path loops over the row in steps of 128 * warps words
    for (uint32_t w0 = vec ? warp * 128 + lane * 4 : 0; w0 < (vec ? W : 1u); w0 += vec ? warps * 128 : 1u) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            uint32_t h[kDotPreds][2][4];
#pragma unroll
            for (int k = 0; k < kDotPreds; k++) {
                if ((uint32_t)k < np) {
                    slice4(P.hv + (uint64_t)(P.half_base[k] + j * 2) * W, W, vec, w0, lane, h[k][0]);
                    slice4(P.hv + (uint64_t)(P.half_base[k] + ((j + 2) % 3) * 2 + 1) * W, W, vec, w0, lane, h[k][1]);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; r++) h[k][0][r] = h[k][1][r] = 0;
                }
            }
            // Lane-local parity bits of the 32 elements, XOR-reduced over the warp below.
            // Element c = 4 q + f sits at bit 8 f + q: a batch's popcounts (at most 32 each)
            // are added into the bytes of two words by shift-adds, and their low bits are
            // moved into place with one mask and one shift per four elements.
            uint32_t pl[kDotPreds][2];
#pragma unroll
            for (int k = 0; k < kDotPreds; k++) pl[k][0] = pl[k][1] = 0;
            for (uint32_t c0 = 0; c0 < 32; c0 += kDotBatch) {
                uint32_t v[kDotBatch][4];
#pragma unroll
                for (int b = 0; b < kDotBatch; b++) {
                    const uint64_t e = base + c0 + b;
                    if (e < P.n_elems) slice4(P.share[j] + e * W, W, vec, w0, lane, v[b]);
                    else v[b][0] = v[b][1] = v[b][2] = v[b][3] = 0;
                }
#pragma unroll
                for (int k = 0; k < kDotPreds; k++) {
                    if ((uint32_t)k >= np) break;
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                        uint32_t cnt[kDotBatch / 4] = {};
#pragma unroll
                        for (int b = 0; b < kDotBatch; b++) {
                            const uint32_t a = (v[b][0] & h[k][hh][0]) ^ (v[b][1] & h[k][hh][1]) ^
                                               (v[b][2] & h[k][hh][2]) ^ (v[b][3] & h[k][hh][3]);
                            cnt[b / 4] += (uint32_t)__popc(a) << (8 * (b % 4));
                        }
#pragma unroll
                        for (int q = 0; q < kDotBatch / 4; q++)
                            pl[k][hh] ^= (cnt[q] & 0x01010101u) << (c0 / 4 + q);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kDotPreds; k++) {
                if ((uint32_t)k >= np) break;
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    uint32_t m = pl[k][hh];
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) m ^= __shfl_xor_sync(0xFFFFFFFFu, m, off);
                    if (lane == 0) zs[warp][k][j][hh] ^= m;
                }
            }
        }
    }
    __syncthreads();
    // server i: first half with share i, second half with share i + 1; element c leaves
    // bit 8 (c % 4) + c / 4 for bit c of the packed output word
    if (threadIdx.x < np * 3) {
        const uint32_t k = threadIdx.x / 3, i = threadIdx.x % 3;
        uint32_t zp = 0;
        for (uint32_t q = 0; q < warps; q++) zp ^= zs[q][k][i][0] ^ zs[q][k][(i + 1) % 3][1];
        uint32_t z = 0;
#pragma unroll
        for (uint32_t c = 0; c < 32; c++) z |= ((zp >> (8 * (c % 4) + c / 4)) & 1u) << c;
        P.zbits[k][(uint64_t)i * nwords + wd] = z;
    }
}

// The same pass for rows of W = 128 * warps words (2^12 <= D <= 2^16), persistent (one
// CTA per SM walks the 32-element words wd = blockIdx.x, + gridDim.x, ...) with the element
// rows staged through shared memory so that two batches are always in flight while a
// third is combined, across word boundaries too.  Lane l of warp q owns words
// [128 q + 4 l, 128 q + 4 l + 4) of every row: it copies them with its own 16-byte
// cp.async into its own slots and reads back only those, so the pipeline needs no
// barrier.  A step is one share set and 8 elements; a word's 32 elements and 3 share sets
// take 12 steps.  The next share set's half-vector slices are loaded into registers
// during the last step of the current one.
constexpr int kPipeStages = 3;
constexpr int kPipeSteps = 3 * (32 / kDotBatch);
constexpr uint32_t kPipeSmemPerWarp = kPipeStages * kDotBatch * 32 * 16;

__device__ __forceinline__ void load_halves(const DotParams& P, uint32_t W, uint32_t w0, uint32_t np, int j,
                                            uint32_t h[kDotPreds][2][4]) {
#pragma unroll
    for (int k = 0; k < kDotPreds; k++) {
        if ((uint32_t)k < np) {
            const uint4 a = __ldg(reinterpret_cast<const uint4*>(P.hv + (uint64_t)(P.half_base[k] + j * 2) * W + w0));
            const uint4 b = __ldg(reinterpret_cast<const uint4*>(
                P.hv + (uint64_t)(P.half_base[k] + ((j + 2) % 3) * 2 + 1) * W + w0));
            h[k][0][0] = a.x; h[k][0][1] = a.y; h[k][0][2] = a.z; h[k][0][3] = a.w;
            h[k][1][0] = b.x; h[k][1][1] = b.y; h[k][1][2] = b.z; h[k][1][3] = b.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; r++) h[k][0][r] = h[k][1][r] = 0;
        }
    }
}

// acc ^ (a & b) in one instruction
__device__ __forceinline__ uint32_t xor_and(uint32_t acc, uint32_t a, uint32_t b) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x78;" : "=r"(d) : "r"(acc), "r"(a), "r"(b));
    return d;
}

__global__ void __launch_bounds__(512) k_onehot_dots_pipe(const __grid_constant__ DotParams P) {
    extern __shared__ __align__(16) unsigned char dsmem[];
    // 2^i for i < 32 from the launch parameters: a runtime factor, so that shifts into place
    // are multiply-adds on the FMA pipe and leave the ALU pipe to the AND / XOR work
    const uint32_t* pw = P.pow2;
    __shared__ uint32_t zs[2][16][kDotPreds][3][2];    // by word parity: per warp, masks per (pred, share, half)
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const uint32_t W = P.words, np = P.n_preds;
    const uint64_t nwords = (P.n_elems + 31) / 32;
    if (blockIdx.x >= nwords) return;
    const uint64_t my_words = (nwords - 1 - blockIdx.x) / gridDim.x + 1;
    const uint64_t total = my_words * kPipeSteps;
    const uint32_t w0 = warp * 128 + lane * 4;
    // slot (stage s, element b) of this lane: mine[(s * kDotBatch + b) * 32]
    uint4* mine = reinterpret_cast<uint4*>(dsmem + (size_t)warp * kPipeSmemPerWarp) + lane;
    // step T: word blockIdx.x + (T / 12) gridDim.x, share set (T % 12) / 4, elements 8 (T % 4) ..
    auto issue = [&](uint64_t T) {
        const int t = (int)(T % kPipeSteps), st = (int)(T % kPipeStages);
        const int j = t / (32 / kDotBatch), c0 = (t % (32 / kDotBatch)) * kDotBatch;
        const uint64_t e0 = (blockIdx.x + (T / kPipeSteps) * gridDim.x) * 32 + c0;
        uint4* dst = mine + st * kDotBatch * 32;
        const uint32_t* src = P.share[j] + e0 * W + w0;
        if (e0 + kDotBatch <= P.n_elems) {
#pragma unroll
            for (int b = 0; b < kDotBatch; b++) cp_async16(dst + b * 32, src + (size_t)b * W, 16u);
        } else {
            // the table's last word: rows past its end are zero-filled, nothing read
            const uint32_t* row0 = P.share[j] + (e0 - c0) * W + w0;
#pragma unroll
            for (int b = 0; b < kDotBatch; b++) {
                const bool ok = e0 + b < P.n_elems;
                cp_async16(dst + b * 32, ok ? src + (size_t)b * W : row0, ok ? 16u : 0u);
            }
        }
        cp_async_commit();
    };
    for (int d = 0; d < kPipeStages - 1; d++) {
        if ((uint64_t)d < total) issue(d);
        else cp_async_commit();                       // an empty group keeps the count uniform
    }
    uint32_t h[kDotPreds][2][4], hn[kDotPreds][2][4];
    load_halves(P, W, w0, np, 0, h);
    constexpr int kBatches = 32 / kDotBatch;          // steps per (word, share set)
#pragma unroll 1
    for (uint64_t T4 = 0; T4 < total; T4 += kBatches) {
        const int j = (int)((T4 / kBatches) % 3);
        const uint32_t par = (uint32_t)(T4 / kPipeSteps) & 1u;
        uint32_t pl[kDotPreds][2];
#pragma unroll
        for (int k = 0; k < kDotPreds; k++) pl[k][0] = pl[k][1] = 0;
#pragma unroll
        for (int cb = 0; cb < kBatches; cb++) {
            const uint64_t T = T4 + cb;
            if (T + kPipeStages - 1 < total) issue(T + kPipeStages - 1);
            else cp_async_commit();
            cp_async_wait<kPipeStages - 1>();         // this lane's copies of step T have landed
            if (cb == kBatches - 1) load_halves(P, W, w0, np, j < 2 ? j + 1 : 0, hn);
            const uint4* slot = mine + (int)(T % kPipeStages) * kDotBatch * 32;
            uint32_t v[kDotBatch][4];
#pragma unroll
            for (int b = 0; b < kDotBatch; b++) {
                const uint4 x = slot[b * 32];
                v[b][0] = x.x; v[b][1] = x.y; v[b][2] = x.z; v[b][3] = x.w;
            }
#pragma unroll
            for (int k = 0; k < kDotPreds; k++) {
                if ((uint32_t)k >= np) break;
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    uint32_t cnt[kDotBatch / 4] = {};
#pragma unroll
                    for (int b = 0; b < kDotBatch; b++) {
                        uint32_t a = v[b][0] & h[k][hh][0];
                        a = xor_and(a, v[b][1], h[k][hh][1]);
                        a = xor_and(a, v[b][2], h[k][hh][2]);
                        a = xor_and(a, v[b][3], h[k][hh][3]);
                        // popcount into byte b % 4 by a multiply-add (the FMA pipe, not the ALU)
                        cnt[b / 4] = (uint32_t)__popc(a) * pw[8 * (b % 4)] + cnt[b / 4];
                    }
                    // bit 8 f + q, q = cb * (kDotBatch / 4) + (b / 4): shifted by a multiply
#pragma unroll
                    for (int q = 0; q < kDotBatch / 4; q++) {
                        constexpr uint32_t M = 0x01010101u;
                        const int sh = cb * (kDotBatch / 4) + q;
                        pl[k][hh] = xor_and(pl[k][hh], cnt[q] * pw[sh], M << sh);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kDotPreds; k++) {
            if ((uint32_t)k >= np) break;
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                uint32_t m = pl[k][hh];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) m ^= __shfl_xor_sync(0xFFFFFFFFu, m, off);
                if (lane == 0) zs[par][warp][k][j][hh] = m;
            }
        }
#pragma unroll
        for (int k = 0; k < kDotPreds; k++)
#pragma unroll
            for (int hh = 0; hh < 2; hh++)
#pragma unroll
                for (int r = 0; r < 4; r++) h[k][hh][r] = hn[k][hh][r];
        if (j == 2) {
            // the word's masks are complete: combine the warps' and write the packed bits.
            // zs is double-buffered by word parity, so one barrier per word suffices.
            __syncthreads();
            if (threadIdx.x < np * 3) {
                const uint64_t wd = blockIdx.x + (T4 / kPipeSteps) * gridDim.x;
                const uint32_t k = threadIdx.x / 3, i = threadIdx.x % 3;
                uint32_t zp = 0;
                for (uint32_t q = 0; q < warps; q++) zp ^= zs[par][q][k][i][0] ^ zs[par][q][k][(i + 1) % 3][1];
                // element c sits at bit 8 (c % 4) + c / 4
                uint32_t z = 0;
#pragma unroll
                for (uint32_t c = 0; c < 32; c++) z |= ((zp >> (8 * (c % 4) + c / 4)) & 1u) << c;
                P.zbits[k][(uint64_t)i * nwords + wd] = z;
            }
        }
    }
    cp_async_wait<0>();
}

void launch_dots(const DotParams& D, uint64_t nwords, int sm_count, cudaStream_t s) {
    if (D.words >= 128 && D.words <= 128 * 16) {
        // persistent: as many CTAs as fit on the SMs (one of 16 warps per SM at D = 2^16)
        const uint32_t warps = D.words / 128;
        const uint32_t per_sm = std::max<uint32_t>(1, std::min<uint32_t>(227u * 1024 / (warps * kPipeSmemPerWarp + 4096), 32 / warps));
        const uint64_t grid = std::min<uint64_t>(nwords, (uint64_t)sm_count * per_sm);
        k_onehot_dots_pipe<<<(unsigned)grid, warps * 32, warps * kPipeSmemPerWarp, s>>>(D);
        return;
    }
    const uint32_t warps = D.words >= 128 ? std::min<uint32_t>(16, D.words / 128) : 1u;
    k_onehot_dots<<<(unsigned)nwords, warps * 32, 0, s>>>(D);
}

// All groups of a query in one launch: each element's predicate bits are re-shared in
// binary RSS and folded in token order.  The re-share PRF gives the bits of 128
// consecutive elements from one AES block (bit e mod 128 of AES_k(c), c = u64 (e div 128)
// | 2^63 || u16 step || u16 table || u32 query), and word q of that block holds the bits
// of the block's output word q, so a warp takes one (group, 128 elements) item and
// works on whole 32-element words: lane 4 b + q (b < 6) computes PRF block b (the three
// servers' keys at the predicate's step, then at its fold step) and keeps word q; shuffles
// bring each word's six PRF words to lane q, which re-shares, folds and stores word q.
// The AES reads the bank-replicated shared-memory T-tables (one persistent CTA per SM).
struct FoldGroup {
    uint32_t* out[3];
    uint64_t n_elems;
    uint64_t item_begin;     // first item (128-element block) of the group in the launch
    uint32_t first;          // index of the group's first predicate in zoff / steps
    uint32_t n_preds;
    uint32_t table_id;
    uint32_t pad;
};

struct FoldParams {
    uint32_t rk_prf[3][44];
    const uint32_t* te0;
    const uint32_t* zbase;             // the query's packed predicate bits
    const uint64_t* zoff;              // per predicate (group order): word offset of its [3][nwords] block
    const uint32_t* steps;             // per predicate: its index in the token | combine << 16
    const FoldGroup* groups;
    uint64_t total_items;
    uint32_t n_groups;
    uint32_t query_id;
};

constexpr int kFoldThreads = 768;
constexpr uint32_t kFoldBlockElems = 128;

__global__ void __launch_bounds__(kFoldThreads, 1) k_onehot_fold(const __grid_constant__ FoldParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    // this lane's PRF block: b = 0..2 server b's key at the step, 3..5 at the fold step
    // (lanes 24..31 repeat lanes 16..23; they keep a word nobody reads)
    const uint32_t b = lane < 24 ? lane >> 2 : (lane >> 2) - 2, q = lane & 3;
    const uint32_t* rk = P.rk_prf[b % 3];
    for (uint64_t item = (uint64_t)blockIdx.x * warps + (threadIdx.x >> 5); item < P.total_items;
         item += (uint64_t)gridDim.x * warps) {
        uint32_t g = 0;
        while (g + 1 < P.n_groups && P.groups[g + 1].item_begin <= item) g++;
        const FoldGroup& G = P.groups[g];
        const uint64_t nwords = (G.n_elems + 31) / 32;
        const uint64_t blk = item - G.item_begin;
        const uint64_t wd = blk * 4 + q;                  // this lane's output word
        const bool have = wd < nwords;
        const uint64_t rem = have ? G.n_elems - wd * 32 : 0;
        const uint32_t valid = rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
        const uint32_t c0 = (uint32_t)blk, c1 = (uint32_t)(blk >> 32) | 0x80000000u;
        uint32_t acc[3] = {0, 0, 0};
        for (uint32_t k = 0; k < G.n_preds; k++) {
            const uint64_t zo = P.zoff[G.first + k];
            const uint32_t sc = P.steps[G.first + k];
            const uint32_t step = sc & 0xFFFFu, combine = sc >> 16;
            // the predicate's bits of this word, loaded before the PRF's AES so the loads overlap it
            uint32_t z[3], r[3];
#pragma unroll
            for (int i = 0; i < 3; i++) z[i] = have ? P.zbase[zo + (uint64_t)i * nwords + wd] : 0u;
            uint32_t f = 0;
            if (b < 3 || k > 0) {
                const uint32_t ctr[4] = {c0, c1, (b < 3 ? step : 64u + step) | (G.table_id << 16), P.query_id};
                uint32_t o[4];
                aes_one(T, rk, ctr, o);
                f = q == 0 ? o[0] : q == 1 ? o[1] : q == 2 ? o[2] : o[3];
            }
            uint32_t F[6];
#pragma unroll
            for (int s = 0; s < 6; s++) F[s] = __shfl_sync(0xFFFFFFFFu, f, 4 * s + (int)q);
            // binary re-share: r_i = z_i xor F(k_i) xor F(k_{i-1})
#pragma unroll
            for (int i = 0; i < 3; i++) r[i] = z[i] ^ F[i] ^ F[(i + 2) % 3];
            if (k == 0) {
                acc[0] = r[0]; acc[1] = r[1]; acc[2] = r[2];
            } else {
                // fold over Z_2 (Sec. V-D): AND = a b, XOR = a ^ b, OR = a ^ b ^ a b
                const uint32_t lin = combine == OBLIVGM_COMBINE_AND ? 0u : 0xFFFFFFFFu;
                const uint32_t prod = combine == OBLIVGM_COMBINE_XOR ? 0u : 0xFFFFFFFFu;
                uint32_t w[3];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const int i1 = (i + 1) % 3;
                    const uint32_t pr = (acc[i] & r[i]) ^ (acc[i] & r[i1]) ^ (acc[i1] & r[i]);
                    w[i] = ((acc[i] ^ r[i]) & lin) ^ (pr & prod);
                }
#pragma unroll
                for (int i = 0; i < 3; i++) acc[i] = w[i] ^ F[3 + i] ^ F[3 + (i + 2) % 3];
            }
        }
        if (lane < 4 && have) {
#pragma unroll
            for (int i = 0; i < 3; i++) G.out[i][wd] = acc[i] & valid;
        }
    }
}

}  // namespace

}  // namespace ogm

// ====================================================================== host side

using namespace ogm;

extern "C" oblivgm_status oblivgm_keygen_onehot(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits,
                                                const uint8_t seed[16], uint8_t* const tok[3], size_t cap,
                                                size_t out_len[3]) {
    const NvtxRange nvtx_range("oblivgm_keygen_onehot");
    std::string err;
    oblivgm_status st = keygen(preds, n_preds, n_bits, seed, tok, cap, out_len, &err, /*onehot=*/true);
    if (st != OBLIVGM_OK) return fail(st, err);
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_load_onehot(oblivgm_ctx* ctx, uint32_t table_id, uint64_t n_elems,
                                              uint32_t n_attrs, uint32_t n_bits,
                                              const uint32_t* const share_sets[3], int32_t mem_kind, void* stream) {
    const NvtxRange nvtx_range("oblivgm_load_onehot");
    if (!ctx) return fail(OBLIVGM_EINVAL, "NULL context");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (table_id > 0xFFFF || n_attrs == 0 || n_attrs > 65536 || n_bits < 1 || n_bits > (uint32_t)kMaxOnehotBits ||
        !share_sets)
        return fail(OBLIVGM_EINVAL, "bad one-hot table arguments");
    if (mem_kind != OBLIVGM_MEM_HOST && mem_kind != OBLIVGM_MEM_DEVICE) return fail(OBLIVGM_EINVAL, "bad mem_kind");
    for (int j = 0; j < 3; j++)
        if (!share_sets[j] && n_elems) return fail(OBLIVGM_EINVAL, "NULL share set");
    const uint32_t words = n_bits >= 5 ? (1u << n_bits) / 32 : 1u;
    const size_t set_words = (size_t)n_attrs * n_elems * words;
    const size_t bytes = 3 * set_words * sizeof(uint32_t);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto it = ctx->onehot_tables.find(table_id);
    if (it != ctx->onehot_tables.end()) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
        cudaFree(it->second.dev);
        ctx->onehot_tables.erase(it);
    }
    OnehotTable tb{};
    tb.n_elems = n_elems; tb.n_attrs = n_attrs; tb.n_bits = n_bits; tb.words = words; tb.bytes = bytes;
    e = cudaMalloc(&tb.dev, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_fail(e, "one-hot table allocation");
    ctx->onehot_tables[table_id] = tb;
    const cudaMemcpyKind kind = mem_kind == OBLIVGM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int j = 0; j < 3 && set_words; j++) {
        e = cudaMemcpyAsync(tb.dev + j * set_words, share_sets[j], set_words * sizeof(uint32_t), kind, s);
        if (e != cudaSuccess) return cuda_fail(e, "one-hot share upload");
    }
    if (mem_kind == OBLIVGM_MEM_HOST) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    }
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_filter_onehot(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                                const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out,
                                                void* stream) {
    const NvtxRange nvtx_range("oblivgm_filter_onehot");
    if (!ctx || !tok || !tok_len || !out) return fail(OBLIVGM_EINVAL, "NULL argument");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    ParsedQuery q;
    std::string err;
    oblivgm_status st = parse_tokens(tok, tok_len, &q, &err);
    if (st != OBLIVGM_OK) return fail(st, err);
    if (q.out_group != 1) return fail(OBLIVGM_EINVAL, "a masked-mode token was given to the one-hot evaluation");
    if (n_groups == 0 || n_groups > OBLIVGM_MAX_GROUPS) return fail(OBLIVGM_EINVAL, "n_groups must be 1..64");
    std::vector<std::vector<uint32_t>> members(n_groups);   // predicate indices per group
    for (uint32_t p = 0; p < q.preds.size(); p++) {
        if (q.preds[p].group >= n_groups) return fail(OBLIVGM_EINVAL, "predicate group outside 0..n_groups-1");
        members[q.preds[p].group].push_back(p);
    }
    for (uint32_t g = 0; g < n_groups; g++) {
        if (members[g].empty()) return fail(OBLIVGM_EINVAL, "an AND-group has no predicate");
        const ParsedPred& p0 = q.preds[members[g][0]];
        auto it = ctx->onehot_tables.find(p0.table);
        if (it == ctx->onehot_tables.end()) return fail(OBLIVGM_ENOENT, "predicate on a one-hot table that is not loaded");
        for (uint32_t p : members[g]) {
            const ParsedPred& pp = q.preds[p];
            if (pp.table != p0.table) return fail(OBLIVGM_EINVAL, "an AND-group spans two tables");
            if (pp.attr >= it->second.n_attrs) return fail(OBLIVGM_EINVAL, "predicate attribute outside its table");
            if (pp.n != it->second.n_bits) return fail(OBLIVGM_EINVAL, "predicate domain differs from its table's");
        }
    }
    const uint32_t n = q.n_bits, domain = 1u << n, words = n >= 5 ? domain / 32 : 1u;
    // device keys and half descriptors: six halves per predicate, [server][half]
    std::vector<EtKey> keys;
    std::vector<HalfDesc> halves;
    for (const ParsedPred& pp : q.preds) {
        const bool eq = pp.kind == OBLIVGM_PRED_EQ;
        const uint32_t nsub = eq ? 1 : 2, k0 = (uint32_t)keys.size();
        keys.insert(keys.end(), pp.et_keys.begin(), pp.et_keys.end());
        for (uint32_t hh = 0; hh < 6; hh++) {
            HalfDesc h{};
            h.key0 = k0 + hh * nsub;
            h.key1 = eq ? kNoKey : k0 + hh * nsub + 1;
            h.kind = eq ? OBLIVGM_KEY_DPF : OBLIVGM_KEY_DCF;
            h.cbit = (!eq && pp.et_keys[hh * nsub].party == 0) ? (pp.cbeta & 1u) : 0u;
            halves.push_back(h);
        }
    }
    // packed predicate bits: per predicate [3][ceil(n_elems / 32)] words of its table
    std::vector<uint64_t> zoff(q.preds.size());
    uint64_t zwords = 0;
    for (uint32_t p = 0; p < q.preds.size(); p++) {
        const OnehotTable& tb = ctx->onehot_tables.at(q.preds[p].table);
        zoff[p] = zwords;
        zwords += 3 * ((tb.n_elems + 31) / 32);
    }
    // per group, the word offsets and token steps of its predicates (token order)
    std::vector<uint64_t> gzoff;
    std::vector<uint32_t> gstep;
    std::vector<size_t> gbegin;
    for (uint32_t g = 0; g < n_groups; g++) {
        gbegin.push_back(gzoff.size());
        for (uint32_t p : members[g]) {
            gzoff.push_back(zoff[p]);
            gstep.push_back(q.preds[p].step | q.preds[p].combine << 16);
        }
    }
    const size_t np = gzoff.size();
    // fold descriptors: the groups with elements, each with its first item
    std::vector<FoldGroup> fg;
    uint64_t fold_items = 0;
    for (uint32_t g = 0; g < n_groups; g++) {
        const OnehotTable& tb = ctx->onehot_tables.at(q.preds[members[g][0]].table);
        if (tb.n_elems == 0) continue;
        FoldGroup G{};
        for (int j = 0; j < 3; j++) {
            G.out[j] = out[3 * g + j];
            if (!G.out[j]) return fail(OBLIVGM_EINVAL, "NULL output pointer");
        }
        G.n_elems = tb.n_elems;
        G.item_begin = fold_items;
        G.first = (uint32_t)gbegin[g];
        G.n_preds = (uint32_t)members[g].size();
        G.table_id = q.preds[members[g][0]].table;
        fg.push_back(G);
        fold_items += (tb.n_elems + kFoldBlockElems - 1) / kFoldBlockElems;
    }
    // scratch: keys | halves | group offsets | group steps | key slots | fold groups | half vectors |
    // predicate bits
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t off_h = up(keys.size() * sizeof(EtKey));
    const size_t off_o = off_h + up(halves.size() * sizeof(HalfDesc));
    const size_t off_s = off_o + up(np * sizeof(uint64_t));
    std::vector<KeySlot> slots;             // DPF keys first, then DCF keys
    for (uint32_t kind = 0; kind < 2; kind++)
        for (uint32_t h = 0; h < halves.size(); h++) {
            const HalfDesc& H = halves[h];
            const uint32_t dcf = H.kind == OBLIVGM_KEY_DCF ? 1u : 0u;
            if (dcf != kind) continue;
            slots.push_back(KeySlot{H.key0, h, H.cbit ? 0xFFFFFFFFu : 0u, dcf});
            if (H.key1 != kNoKey) slots.push_back(KeySlot{H.key1, h, 0u, dcf});
        }
    const size_t off_k = off_s + up(np * sizeof(uint32_t));
    const size_t off_g = off_k + up(slots.size() * sizeof(KeySlot));
    const size_t off_v = off_g + up(fg.size() * sizeof(FoldGroup));
    const size_t off_z = off_v + up(halves.size() * words * sizeof(uint32_t));
    const size_t total = off_z + zwords * sizeof(uint32_t);
    std::vector<unsigned char> img(off_v, 0);
    std::memcpy(img.data(), keys.data(), keys.size() * sizeof(EtKey));
    std::memcpy(img.data() + off_h, halves.data(), halves.size() * sizeof(HalfDesc));
    std::memcpy(img.data() + off_o, gzoff.data(), np * sizeof(uint64_t));
    std::memcpy(img.data() + off_s, gstep.data(), np * sizeof(uint32_t));
    std::memcpy(img.data() + off_k, slots.data(), slots.size() * sizeof(KeySlot));
    if (!fg.empty()) std::memcpy(img.data() + off_g, fg.data(), fg.size() * sizeof(FoldGroup));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = nullptr;
    {
        const oblivgm_status as = ws_alloc(ctx, reinterpret_cast<void**>(&ws), total, s, "one-hot scratch");
        if (as != OBLIVGM_OK) return as;
    }
    ScratchGuard guard(ws, s);
    ce = cudaMemcpyAsync(ws, img.data(), off_v, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot descriptor upload");
    uint32_t* zbase = reinterpret_cast<uint32_t*>(ws + off_z);
    uint32_t* hv = reinterpret_cast<uint32_t*>(ws + off_v);
    ce = cudaMemsetAsync(hv, 0, halves.size() * words * sizeof(uint32_t), s);
    if (ce != cudaSuccess) return cuda_fail(ce, "half-vector clear");
    {
        EvalEtParams E{};
        E.aes = ctx->aes;
        E.te0 = ctx->d_te0;
        E.keys = reinterpret_cast<const EtKey*>(ws);
        E.slots = reinterpret_cast<const KeySlot*>(ws + off_k);
        E.hv = hv;
        E.words = words;
        E.leaves = 1u << (n - (uint32_t)et_low_bits((int)n));
        E.n_slots = (uint32_t)slots.size();
        const uint64_t items = (uint64_t)E.n_slots * E.leaves;
        // one CTA per SM (the tables take 128 KiB), as many threads as give every item a lane pair
        const uint64_t per_sm = (2 * items + ctx->sm_count - 1) / ctx->sm_count;
        const unsigned threads = (unsigned)std::min<uint64_t>(kEvalEtMaxThreads, std::max<uint64_t>(64, (per_sm + 31) / 32 * 32));
        const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((2 * items + threads - 1) / threads,
                                                                                 (uint64_t)ctx->sm_count));
        k_onehot_evalall_et<<<grid, threads, kTableBytes, s>>>(E);
    }
    ctx->launches++;
    // one streaming pass per (table, attribute) for up to kDotPreds predicates on it
    std::map<std::pair<uint32_t, uint32_t>, std::vector<uint32_t>> by_column;
    for (uint32_t p = 0; p < q.preds.size(); p++) by_column[{q.preds[p].table, q.preds[p].attr}].push_back(p);
    for (auto& col : by_column) {
        const OnehotTable& tb = ctx->onehot_tables.at(col.first.first);
        if (tb.n_elems == 0) continue;
        const size_t set_words = (size_t)tb.n_attrs * tb.n_elems * tb.words;
        const uint64_t nwords = (tb.n_elems + 31) / 32;
        const std::vector<uint32_t>& ps = col.second;
        for (size_t c0 = 0; c0 < ps.size(); c0 += kDotPreds) {
            DotParams D{};
            for (int j = 0; j < 3; j++) D.share[j] = tb.dev + j * set_words + (size_t)col.first.second * tb.n_elems * tb.words;
            D.hv = hv;
            D.n_preds = (uint32_t)std::min<size_t>(kDotPreds, ps.size() - c0);
            for (uint32_t k = 0; k < D.n_preds; k++) {
                D.half_base[k] = 6 * ps[c0 + k];
                D.zbits[k] = zbase + zoff[ps[c0 + k]];
            }
            D.n_elems = tb.n_elems;
            D.words = words;
            for (int i = 0; i < 32; i++) D.pow2[i] = 1u << i;
            launch_dots(D, nwords, ctx->sm_count, s);
            ctx->launches++;
        }
    }
    // every AND-group in one launch: binary re-share and fold, packed outputs
    if (!fg.empty()) {
        FoldParams F{};
        std::memcpy(F.rk_prf, ctx->rk_prf, sizeof F.rk_prf);
        F.te0 = ctx->d_te0;
        F.zbase = zbase;
        F.zoff = reinterpret_cast<const uint64_t*>(ws + off_o);
        F.steps = reinterpret_cast<const uint32_t*>(ws + off_s);
        F.groups = reinterpret_cast<const FoldGroup*>(ws + off_g);
        F.total_items = fold_items;
        F.n_groups = (uint32_t)fg.size();
        F.query_id = query_id;
        // a warp per item: as many warps per CTA as spread the items over every SM (at least 4)
        const uint64_t warps = std::min<uint64_t>(kFoldThreads / 32, std::max<uint64_t>(
                                                      4, (fold_items + ctx->sm_count - 1) / ctx->sm_count));
        const unsigned grid = (unsigned)std::min<uint64_t>((fold_items + warps - 1) / warps, (uint64_t)ctx->sm_count);
        k_onehot_fold<<<grid, (unsigned)(warps * 32), kTableBytes, s>>>(F);
        ctx->launches++;
    }
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot launch");
    guard.done();
    ce = cudaFreeAsync(ws, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot scratch release");
    return OBLIVGM_OK;
}

namespace ogm {

oblivgm_status set_onehot_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_onehot_evalall_et, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_onehot_dots_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 * kPipeSmemPerWarp);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_onehot_fold, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, "one-hot kernel attributes");
}

}  // namespace ogm
