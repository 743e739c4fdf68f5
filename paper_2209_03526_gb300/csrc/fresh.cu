// fresh.cu -- the masked-input approach with a fresh mask and fresh keys for every
// attribute value (Sec. V-C, the basic approach): predicate p meets element c with its
// own mask r_{c,p} and its own three key pairs, so no two opened values x^ share a mask.
//
//   k_keygen_fresh  the client's Gen, one thread per (element, predicate, pair, key):
//                   mask block and root seeds from AES under the client seed, then the
//                   DPF / DCF Gen of gen_device.cuh, written level-major so that the
//                   servers' reads are coalesced.
//   k_filter_fresh  the servers: open x^_c, walk element c's own six (EQ) or twelve
//                   (RANGE) key halves, sum per server (Eq. predEval, masked form),
//                   re-share to RSS and AND the group's predicates (Sec. III-B, V-D).
//
// Token layout (per server, device memory, little-endian, arrays 16-byte aligned,
// N4 = N rounded up to 4): a 64-byte header, 32 bytes per predicate, then per predicate
// rA[N4], rB[N4], (RANGE) cb[N4], and the key blocks (A,0), (A,1), (B,0), (B,1), each
// seed[N] (16 B), scw[n][N] (16 B), tl[N4], tr[N4], (DCF) vcw[n][N4], cw[N4].
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "device_fss.cuh"
#include "gen_device.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

constexpr uint32_t kFreshMagic = 0x464D474Fu;
constexpr int kFreshMaxPreds = 64;
constexpr int kFreshMaxJobs = kFreshMaxPreds * 6;
// client Gen: one CTA per SM (the tables take 128 KiB); both instances need more than the
// 80 registers a 768-thread CTA leaves
#ifndef OGM_FRESH_GEN_THREADS
#define OGM_FRESH_GEN_THREADS 512
#endif
template <bool DCF> constexpr int fresh_gen_threads() { return OGM_FRESH_GEN_THREADS; }
#ifndef OGM_FRESH_EVAL_THREADS
#define OGM_FRESH_EVAL_THREADS 768
#endif
constexpr int kFreshEvalThreads = OGM_FRESH_EVAL_THREADS;

// halves held by server i (0-based): (pair, party) -- CS1 (1,0),(2,0); CS2 (2,1),(3,0); CS3 (3,1),(1,1)
__constant__ uint8_t c_hold_party[3][2] = {{0, 0}, {1, 0}, {1, 1}};

struct FreshLayout {
    uint64_t N, N4;
    uint64_t key_block;    // bytes of one key block
    uint64_t keys_at;      // offset of the first key block in the data block
    uint64_t data_len;
};

__host__ __device__ inline FreshLayout fresh_layout(bool eq, uint32_t n, uint64_t N) {
    FreshLayout L;
    L.N = N;
    L.N4 = (N + 3) & ~uint64_t(3);
    L.key_block = 16 * N + 16 * (uint64_t)n * N + 12 * L.N4 + (eq ? 0 : 4 * (uint64_t)n * L.N4);
    L.keys_at = (eq ? 8 : 12) * L.N4;
    L.data_len = L.keys_at + (eq ? 2 : 4) * L.key_block;
    return L;
}

struct FreshPred {
    uint32_t kind, attr, lo, hi;
    uint32_t step;         // the predicate's index p in the query
    uint32_t combine;      // OBLIVGM_COMBINE_*: how the result joins the group's
    FreshLayout lay;
    uint8_t* data[3];      // the predicate's data block in each server token
};

// ------------------------------------------------------------------ client side

struct GenJob {
    uint16_t pred;
    uint8_t pair, sub;
};

struct FreshGenParams {
    AesParams aes;
    GenRightKeys right;
    uint32_t rk_client[44];
    const uint32_t* te0;
    uint32_t n, n_jobs;
    FreshPred preds[kFreshMaxPreds];
    GenJob jobs[kFreshMaxJobs];
    uint64_t job_start[kFreshMaxJobs + 1];   // prefix sums of the jobs' element counts
};

__device__ __forceinline__ void st_u32(uint8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }
__device__ __forceinline__ void st_u128(uint8_t* p, const uint32_t w[4]) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// level-major key blocks: element c's words of both keys of the pair
struct SoaSink {
    uint8_t* b[2];         // key block of party 0 and party 1
    uint64_t N, N4, c;
    uint32_t n, tlw, trw;
    bool dcf;
    __device__ __forceinline__ void level(int lv, const uint32_t scw[4], uint32_t tl, uint32_t tr, uint32_t vcw) {
        const uint64_t o = 16 * N + 16 * ((uint64_t)lv * N + c);
        st_u128(b[0] + o, scw);
        st_u128(b[1] + o, scw);
        tlw |= tl << lv;
        trw |= tr << lv;
        if (dcf) {
            const uint64_t ov = 16 * N + 16 * (uint64_t)n * N + 8 * N4 + 4 * ((uint64_t)lv * N4 + c);
            st_u32(b[0] + ov, vcw);
            st_u32(b[1] + ov, vcw);
        }
    }
    __device__ __forceinline__ void final(uint32_t cw) {
        const uint64_t ot = 16 * N + 16 * (uint64_t)n * N;
        const uint64_t oc = ot + 8 * N4 + (dcf ? 4 * (uint64_t)n * N4 : 0);
        for (int k = 0; k < 2; k++) {
            st_u32(b[k] + ot + 4 * c, tlw);
            st_u32(b[k] + ot + 4 * N4 + 4 * c, trw);
            st_u32(b[k] + oc + 4 * c, cw);
        }
    }
};

// AES under the client seed of B(c, p, tag, j) = u64 c || u16 p || u16 tag || u32 j
__device__ __forceinline__ void client_block(const SmemTab& T, const uint32_t* rk, uint64_t c, uint32_t p,
                                             uint32_t tag, uint32_t j, uint32_t out[4]) {
    const uint32_t in[4] = {(uint32_t)c, (uint32_t)(c >> 32), p | (tag << 16), j};
    aes_one(T, rk, in, out);
}

// one instance per predicate kind (EQ: DPF keys, RANGE: DCF keys), launched on its own jobs
template <bool DCF>
__global__ void __launch_bounds__(fresh_gen_threads<DCF>()) k_keygen_fresh(const __grid_constant__ FreshGenParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    constexpr bool eq = !DCF;
    const uint32_t n = P.n;
    const uint32_t m = n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    constexpr int nsub = eq ? 1 : 2;
    // one persistent grid over all (job, element) items of the launch, so no CTA waits on
    // a short last wave
    const uint64_t total = P.job_start[P.n_jobs];
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = P.n_jobs - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (P.job_start[mid] <= idx) lo = mid; else hi = mid - 1;
        }
        const GenJob J = P.jobs[lo];
        const FreshPred& Q = P.preds[J.pred];
        const FreshLayout& L = Q.lay;
        const uint64_t c = idx - P.job_start[lo];
        // owners (server, half) of the pair's two keys, from the assignment
        // CS1 (1,0),(2,0); CS2 (2,1),(3,0); CS3 (3,1),(1,1): party 0 of pairs 1, 2, 3 sits with
        // CS1 A, CS1 B, CS2 B; party 1 with CS3 B, CS2 A, CS3 A
        const uint32_t srv0 = J.pair == 2 ? 1u : 0u, half0 = J.pair == 0 ? 0u : 1u;
        const uint32_t srv1 = J.pair == 1 ? 1u : 2u, half1 = J.pair == 0 ? 1u : 0u;
        uint32_t w[4];
        client_block(T, P.rk_client, c, Q.step, 1u, 0u, w);
        const uint32_t r = w[0] & m;
        const uint32_t rs[3] = {w[1] & m, w[2] & m, (r - (w[1] & m) - (w[2] & m)) & m};
        const uint32_t a0 = (Q.lo + r) & m, a1 = (Q.hi + 1u + r) & m;
        if (J.pair == 0 && J.sub == 0) {
#pragma unroll
            for (int i = 0; i < 3; i++) {
                st_u32(Q.data[i] + 4 * c, rs[i]);
                st_u32(Q.data[i] + 4 * L.N4 + 4 * c, rs[(i + 1) % 3]);
                if (!eq) st_u32(Q.data[i] + 8 * L.N4 + 4 * c, a1 <= a0 ? kBetaPrime : 0u);
            }
        }
        const uint32_t alpha = eq ? a0 : (J.sub == 0 ? a1 : a0);
        const uint32_t beta = (eq || J.sub == 0) ? kBetaPrime : 0u - kBetaPrime;
        uint32_t s0[4], s1[4];
        client_block(T, P.rk_client, c, Q.step, 2u, 4u * J.pair + 2u * J.sub + 0u, s0);
        client_block(T, P.rk_client, c, Q.step, 2u, 4u * J.pair + 2u * J.sub + 1u, s1);
        SoaSink sink;
        sink.b[0] = Q.data[srv0] + L.keys_at + (uint64_t)(half0 * nsub + J.sub) * L.key_block;
        sink.b[1] = Q.data[srv1] + L.keys_at + (uint64_t)(half1 * nsub + J.sub) * L.key_block;
        st_u128(sink.b[0] + 16 * c, s0);
        st_u128(sink.b[1] + 16 * c, s1);
        sink.N = L.N;
        sink.N4 = L.N4;
        sink.c = c;
        sink.n = n;
        sink.tlw = sink.trw = 0;
        sink.dcf = !eq;
        gen_pair<DCF>(T, P.aes, P.right, (int)n, alpha, beta, s0, s1, sink);
    }
}

// ------------------------------------------------------------------ server side

struct FreshGroup {
    const uint32_t* share[3];   // share set j at attribute 0 of the group's table
    uint32_t* out[3];
    uint64_t stride;
    uint32_t pred_begin, n_preds, table, pad;
};

struct FreshEvalParams {
    AesParams aes;
    uint32_t rk_prf[3][44];
    const uint32_t* te0;
    uint32_t n, n_groups, query, pad;
    uint64_t item_start[OBLIVGM_MAX_GROUPS + 1];   // prefix sums of the groups' element counts
    FreshGroup groups[OBLIVGM_MAX_GROUPS];
    FreshPred preds[kFreshMaxPreds];
};

__device__ __forceinline__ uint32_t ldg1(const uint8_t* p) { return __ldg(reinterpret_cast<const uint32_t*>(p)); }

// DPF (DCF = false) or DCF Eval of element c's key in key block blk at input x.  The
// level-major arrays are walked with pointer increments, and the next level's
// correction word is loaded one level ahead of its use.
template <bool DCF>
__device__ __forceinline__ uint32_t walk_soa(const SmemTab& T, const AesParams& A, const uint8_t* blk, uint64_t N,
                                             uint64_t N4, uint64_t c, uint32_t n, uint32_t party, uint32_t x) {
    const uint4* scwp = reinterpret_cast<const uint4*>(blk + 16 * N) + c;
    const uint32_t* tp = reinterpret_cast<const uint32_t*>(blk + 16 * N + 16 * (uint64_t)n * N) + c;
    const uint32_t* vp = tp + 2 * N4;
    const uint32_t* cwp = vp + (DCF ? (uint64_t)n * N4 : 0);
    const uint4 s4 = __ldg(reinterpret_cast<const uint4*>(blk) + c);
    uint32_t s[4] = {s4.x, s4.y, s4.z, s4.w};
    const uint32_t tl = __ldg(tp), tr = __ldg(tp + N4), cwf = __ldg(cwp);
    uint32_t t = party, V = 0;
    uint4 cw_next = __ldg(scwp);
    uint32_t vcw_next = DCF ? __ldg(vp) : 0u;
    for (uint32_t i = 0; i < n; i++) {
        const uint4 cw = cw_next;
        const uint32_t vcw = vcw_next;
        if (i + 1 < n) {
            scwp += N;
            cw_next = __ldg(scwp);
            if (DCF) {
                vp += N4;
                vcw_next = __ldg(vp);
            }
        }
        const uint32_t dir = (x >> (n - 1 - i)) & 1u;
        const uint32_t msk = 0u - dir;
        uint32_t o[4];
        aes_sel(T, A.rk_st, A.d_st, msk, s, o);
        if (DCF) {
            const uint32_t v0 = aes_sel_w0(T, A.rk_v, A.d_v, msk, s) ^ s[0];
            const uint32_t term = v0 + (t ? vcw : 0u);
            V += party ? 0u - term : term;
        }
#pragma unroll
        for (int w = 0; w < 4; w++) o[w] ^= s[w];
        uint32_t tn = o[0] & 1u;
        o[0] &= ~1u;
        const uint32_t tm = 0u - t;
        s[0] = o[0] ^ (cw.x & tm);
        s[1] = o[1] ^ (cw.y & tm);
        s[2] = o[2] ^ (cw.z & tm);
        s[3] = o[3] ^ (cw.w & tm);
        tn ^= t & (((dir ? tr : tl) >> i) & 1u);
        t = tn;
    }
    const uint32_t term = s[1] + (t ? cwf : 0u);
    return V + (party ? 0u - term : term);
}

// r_i = z_i + F(k_i, ctr) - F(k_{i-1}, ctr), F = bytes 0..3 of AES_{k_i}(elem || step || table || query)
__device__ __forceinline__ void reshare1(const SmemTab& T, const uint32_t (&rk_prf)[3][44], const uint32_t z[3],
                                         uint32_t out[3], uint64_t el, uint32_t step, uint32_t table,
                                         uint32_t query) {
    out[0] = z[0];
    out[1] = z[1];
    out[2] = z[2];
    const uint32_t ctr[4] = {(uint32_t)el, (uint32_t)(el >> 32), step | (table << 16), query};
#pragma unroll 1
    for (int i = 0; i < 3; i++) {
        const uint32_t f = aes_one_w0(T, rk_prf[i], ctr);
        out[0] += i == 0 ? f : (i == 2 ? 0u - f : 0u);
        out[1] += i == 1 ? f : (i == 0 ? 0u - f : 0u);
        out[2] += i == 2 ? f : (i == 1 ? 0u - f : 0u);
    }
}

__global__ void __launch_bounds__(kFreshEvalThreads, 1) k_filter_fresh(const __grid_constant__ FreshEvalParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t n = P.n;
    const uint32_t mask = n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const uint64_t total = P.item_start[P.n_groups];
    for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t g = 0;
        while (g + 1 < P.n_groups && P.item_start[g + 1] <= f) g++;
        const FreshGroup& G = P.groups[g];
        const uint64_t c = f - P.item_start[g];
        uint32_t acc[3] = {0, 0, 0};
        for (uint32_t k = 0; k < G.n_preds; k++) {
            const FreshPred& Q = P.preds[G.pred_begin + k];
            const FreshLayout& L = Q.lay;
            const bool eq = Q.kind == OBLIVGM_PRED_EQ;
            // open x^ = <x>_1 + <x>_2 + <x>_3 + <r>_1 + <r>_2 + <r>_3 mod 2^n
            uint32_t xh = 0;
#pragma unroll
            for (int j = 0; j < 3; j++)
                xh += __ldg(G.share[j] + (uint64_t)Q.attr * G.stride + c) + ldg1(Q.data[j] + 4 * c);
            xh &= mask;
            uint32_t z[3] = {0, 0, 0};
            const int nsub = eq ? 1 : 2;
#pragma unroll 1
            for (int kk = 0; kk < 6 * nsub; kk++) {
                const int i = kk / (2 * nsub), h = (kk / nsub) & 1, sub = kk % nsub;
                const uint32_t party = c_hold_party[i][h];
                const uint8_t* blk = Q.data[i] + L.keys_at + (uint64_t)(h * nsub + sub) * L.key_block;
                uint32_t v = eq ? walk_soa<false>(T, P.aes, blk, L.N, L.N4, c, n, party, xh)
                                : walk_soa<true>(T, P.aes, blk, L.N, L.N4, c, n, party, xh);
                // RANGE: c * beta' joins party 0's half once
                if (!eq && sub == 0 && party == 0) v += ldg1(Q.data[i] + 8 * L.N4 + 4 * c);
                z[0] += i == 0 ? v : 0u;
                z[1] += i == 1 ? v : 0u;
                z[2] += i == 2 ? v : 0u;
            }
            uint32_t step = Q.step;
            const int passes = k == 0 ? 1 : 2;
#pragma unroll 1
            for (int pass = 0; pass < passes; pass++) {
                uint32_t r[3];
                reshare1(T, P.rk_prf, z, r, c, step, G.table, P.query);
                if (pass + 1 < passes) {
                    // fold (Sec. V-D): w = lin (a + b) + prod a b over 0/1 values
                    const uint32_t lin = Q.combine == OBLIVGM_COMBINE_AND ? 0u : 1u;
                    const uint32_t prod = Q.combine == OBLIVGM_COMBINE_AND   ? 1u
                                          : Q.combine == OBLIVGM_COMBINE_XOR ? 0xFFFFFFFEu
                                                                             : 0xFFFFFFFFu;
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        const int i1 = (i + 1) % 3;
                        z[i] = lin * (acc[i] + r[i]) + prod * (acc[i] * r[i] + acc[i] * r[i1] + acc[i1] * r[i]);
                    }
                    step = 64u + Q.step;
                } else {
                    acc[0] = r[0];
                    acc[1] = r[1];
                    acc[2] = r[2];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 3; i++) G.out[i][c] = acc[i];
    }
}

// ------------------------------------------------------------------ host helpers

void put_u64(uint8_t* p, uint64_t v) { std::memcpy(p, &v, 8); }
uint64_t get_u64(const uint8_t* p) {
    uint64_t v;
    std::memcpy(&v, p, 8);
    return v;
}

oblivgm_status check_fresh_preds(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits,
                                 const uint64_t* table_elems, uint32_t n_tables) {
    if (!preds || !table_elems) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (n_preds == 0 || n_preds > (uint32_t)kFreshMaxPreds) return fail(OBLIVGM_EINVAL, "predicate count must be 1..64");
    if (n_bits < 1 || n_bits > 32) return fail(OBLIVGM_EINVAL, "n must be 1..32");
    const uint32_t m = n_bits == 32 ? 0xFFFFFFFFu : ((1u << n_bits) - 1u);
    for (uint32_t p = 0; p < n_preds; p++) {
        const oblivgm_pred& q = preds[p];
        if (q.kind == OBLIVGM_PRED_EQ) {
            if (q.lo > m) return fail(OBLIVGM_EINVAL, "equality value outside the domain");
        } else if (q.kind == OBLIVGM_PRED_RANGE) {
            if (q.lo > q.hi || q.hi > m) return fail(OBLIVGM_EINVAL, "empty range or bound outside the domain");
        } else {
            return fail(OBLIVGM_EINVAL, "unknown predicate kind");
        }
        if (q.table >= n_tables) return fail(OBLIVGM_EINVAL, "predicate on a table outside table_elems");
        if (q.attr > 0xFFFF || q.group > 0xFFFF) return fail(OBLIVGM_EINVAL, "id above 65535");
        if (table_elems[q.table] >= (1ull << 40)) return fail(OBLIVGM_EINVAL, "table too large");
    }
    std::string err;
    if (!check_combine(preds, n_preds, &err)) return fail(OBLIVGM_EINVAL, err);
    return OBLIVGM_OK;
}

uint64_t fresh_total(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits, const uint64_t* table_elems) {
    uint64_t total = 64 + 32 * (uint64_t)n_preds;
    for (uint32_t p = 0; p < n_preds; p++)
        total += fresh_layout(preds[p].kind == OBLIVGM_PRED_EQ, n_bits, table_elems[preds[p].table]).data_len;
    return total;
}

}  // namespace

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_fresh_token_size(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits,
                                                   const uint64_t* table_elems, uint32_t n_tables, uint64_t* bytes) {
    if (!bytes) return fail(OBLIVGM_EINVAL, "NULL argument");
    const oblivgm_status st = check_fresh_preds(preds, n_preds, n_bits, table_elems, n_tables);
    if (st) return st;
    *bytes = fresh_total(preds, n_preds, n_bits, table_elems);
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_keygen_fresh(oblivgm_ctx* ctx, const oblivgm_pred* preds, uint32_t n_preds,
                                               uint32_t n_bits, const uint64_t* table_elems, uint32_t n_tables,
                                               const uint8_t seed[16], uint8_t* const tok[3], uint64_t cap,
                                               void* stream) {
    const NvtxRange nvtx_range("oblivgm_keygen_fresh");
    if (!ctx || !seed || !tok || !tok[0] || !tok[1] || !tok[2]) return fail(OBLIVGM_EINVAL, "NULL argument");
    oblivgm_status st = check_fresh_preds(preds, n_preds, n_bits, table_elems, n_tables);
    if (st) return st;
    const uint64_t total = fresh_total(preds, n_preds, n_bits, table_elems);
    if (cap < total) return fail(OBLIVGM_ERANGE, "fresh token buffer too small");
    for (int i = 0; i < 3; i++)
        if (reinterpret_cast<uintptr_t>(tok[i]) % 16) return fail(OBLIVGM_EINVAL, "token buffers must be 16-byte aligned");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    FreshGenParams P;
    std::memset(&P, 0, sizeof P);
    P.aes = ctx->aes;
    for (int w = 0; w < 44; w++) {
        P.right.st[w] = ctx->aes.rk_st[w] ^ ctx->aes.d_st[w];
        P.right.v[w] = ctx->aes.rk_v[w] ^ ctx->aes.d_v[w];
    }
    const RoundKeys rk = expand_key(seed);
    std::memcpy(P.rk_client, rk.w, sizeof P.rk_client);
    P.te0 = ctx->d_te0;
    P.n = n_bits;
    // headers and descriptors, written on the host and copied in front of each token
    const size_t head = 64 + 32 * (size_t)n_preds;
    std::vector<GenJob> eq_jobs, range_jobs;
    std::vector<uint8_t> hdr(3 * head, 0);
    uint64_t off = head, n_max = 0;
    for (uint32_t p = 0; p < n_preds; p++) {
        const oblivgm_pred& q = preds[p];
        const bool eq = q.kind == OBLIVGM_PRED_EQ;
        FreshPred& F = P.preds[p];
        F.kind = q.kind;
        F.attr = q.attr;
        F.lo = q.lo;
        F.hi = q.hi;
        F.step = p;
        F.combine = q.combine;
        F.lay = fresh_layout(eq, n_bits, table_elems[q.table]);
        for (int i = 0; i < 3; i++) {
            F.data[i] = tok[i] + off;
            uint8_t* d = hdr.data() + i * head + 64 + 32 * p;
            d[24] = (uint8_t)q.combine;
            d[0] = (uint8_t)q.kind;
            d[1] = (uint8_t)n_bits;
            d[2] = (uint8_t)q.table; d[3] = (uint8_t)(q.table >> 8);
            d[4] = (uint8_t)q.attr;  d[5] = (uint8_t)(q.attr >> 8);
            d[6] = (uint8_t)q.group; d[7] = (uint8_t)(q.group >> 8);
            put_u64(d + 8, F.lay.N);
            put_u64(d + 16, off);
        }
        for (uint8_t pair = 0; pair < 3; pair++)
            for (uint8_t sub = 0; sub < (eq ? 1 : 2); sub++) {
                std::vector<GenJob>& jl = eq ? eq_jobs : range_jobs;
                jl.push_back(GenJob{(uint16_t)p, pair, sub});
            }
        n_max = std::max(n_max, F.lay.N);
        off += F.lay.data_len;
    }
    for (int i = 0; i < 3; i++) {
        uint8_t* h = hdr.data() + i * head;
        const uint32_t magic = kFreshMagic;
        std::memcpy(h, &magic, 4);
        h[4] = 1;
        h[5] = (uint8_t)(i + 1);
        h[6] = (uint8_t)n_bits;
        h[8] = (uint8_t)n_preds;
        h[9] = (uint8_t)(n_preds >> 8);
        put_u64(h + 16, total);
        // pageable source: the copy is staged before cudaMemcpyAsync returns
        ce = cudaMemcpyAsync(tok[i], h, head, cudaMemcpyHostToDevice, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "fresh token header copy");
    }
    if (n_max == 0) return OBLIVGM_OK;
    // one launch per kind, a persistent grid over the launch's (job, element) items
    for (int kind = 0; kind < 2; kind++) {
        const std::vector<GenJob>& jl = kind ? range_jobs : eq_jobs;
        if (jl.empty()) continue;
        P.n_jobs = (uint32_t)jl.size();
        std::copy(jl.begin(), jl.end(), P.jobs);
        P.job_start[0] = 0;
        for (uint32_t j = 0; j < P.n_jobs; j++) P.job_start[j + 1] = P.job_start[j] + P.preds[jl[j].pred].lay.N;
        if (P.job_start[P.n_jobs] == 0) continue;
        const uint64_t threads = kind ? fresh_gen_threads<true>() : fresh_gen_threads<false>();
        const uint64_t grid = std::min<uint64_t>((P.job_start[P.n_jobs] + threads - 1) / threads, ctx->sm_count);
        if (kind) k_keygen_fresh<true><<<(unsigned)grid, (unsigned)threads, kTableBytes, s>>>(P);
        else k_keygen_fresh<false><<<(unsigned)grid, (unsigned)threads, kTableBytes, s>>>(P);
        ctx->launches++;
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "k_keygen_fresh launch");
    }
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_filter_fresh(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                               uint64_t tok_cap, uint32_t n_groups, uint32_t* const* out,
                                               void* stream) {
    const NvtxRange nvtx_range("oblivgm_filter_fresh");
    if (!ctx || !tok || !tok[0] || !tok[1] || !tok[2] || !out) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (n_groups == 0 || n_groups > OBLIVGM_MAX_GROUPS) return fail(OBLIVGM_EINVAL, "n_groups must be 1..64");
    for (int i = 0; i < 3; i++)
        if (reinterpret_cast<uintptr_t>(tok[i]) % 16) return fail(OBLIVGM_EINVAL, "token buffers must be 16-byte aligned");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tok_cap < 64) return fail(OBLIVGM_EINVAL, "fresh token buffer shorter than a header");
    // read the three headers and descriptor tables back (ordered after work already on the stream)
    uint8_t h[3][64];
    for (int i = 0; i < 3; i++) {
        ce = cudaMemcpyAsync(h[i], tok[i], 64, cudaMemcpyDeviceToHost, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "fresh token header read");
    }
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fresh token header read");
    uint32_t magic;
    std::memcpy(&magic, h[0], 4);
    const uint32_t n = h[0][6], np = h[0][8] | (h[0][9] << 8);
    for (int i = 0; i < 3; i++) {
        uint32_t mi;
        std::memcpy(&mi, h[i], 4);
        if (mi != kFreshMagic || h[i][4] != 1 || h[i][5] != i + 1) return fail(OBLIVGM_EINVAL, "not a fresh token");
        if (std::memcmp(h[i] + 6, h[0] + 6, 4) != 0 || get_u64(h[i] + 16) != get_u64(h[0] + 16))
            return fail(OBLIVGM_EINVAL, "the three fresh tokens disagree");
    }
    if (n < 1 || n > 32 || np < 1 || np > (uint32_t)kFreshMaxPreds) return fail(OBLIVGM_EINVAL, "bad fresh token header");
    if (get_u64(h[0] + 16) > tok_cap || 64 + 32 * (uint64_t)np > tok_cap)
        return fail(OBLIVGM_EINVAL, "fresh token longer than its buffer");
    std::vector<uint8_t> desc(3 * 32 * (size_t)np);
    for (int i = 0; i < 3; i++) {
        ce = cudaMemcpyAsync(desc.data() + i * 32 * np, tok[i] + 64, 32 * np, cudaMemcpyDeviceToHost, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "fresh token descriptor read");
    }
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fresh token descriptor read");
    for (int i = 1; i < 3; i++)
        if (std::memcmp(desc.data() + i * 32 * np, desc.data(), 32 * np) != 0)
            return fail(OBLIVGM_EINVAL, "the three fresh tokens disagree");

    FreshEvalParams* P = new FreshEvalParams;
    std::unique_ptr<FreshEvalParams> hold(P);
    std::memset(P, 0, sizeof *P);
    P->aes = ctx->aes;
    std::memcpy(P->rk_prf, ctx->rk_prf, sizeof P->rk_prf);
    P->te0 = ctx->d_te0;
    P->n = n;
    P->n_groups = n_groups;
    P->query = query_id;
    std::vector<std::vector<uint32_t>> members(n_groups);
    std::vector<int> gtable(n_groups, -1);
    uint64_t off = 64 + 32 * (uint64_t)np;
    for (uint32_t p = 0; p < np; p++) {
        const uint8_t* d = desc.data() + 32 * p;
        const uint32_t kind = d[0], table = d[2] | (d[3] << 8), attr = d[4] | (d[5] << 8), group = d[6] | (d[7] << 8);
        if (kind != OBLIVGM_PRED_EQ && kind != OBLIVGM_PRED_RANGE) return fail(OBLIVGM_EINVAL, "bad predicate kind");
        if (d[1] != n) return fail(OBLIVGM_EINVAL, "predicate n differs from the token's");
        if (group >= n_groups) return fail(OBLIVGM_EINVAL, "predicate group outside n_groups");
        auto it = ctx->tables.find(table);
        if (it == ctx->tables.end()) return fail(OBLIVGM_ENOENT, "predicate on a table that is not loaded");
        const Table& tb = it->second;
        const uint64_t N = get_u64(d + 8);
        if (N != tb.n_elems || attr >= tb.n_attrs || n != tb.n_bits)
            return fail(OBLIVGM_EINVAL, "predicate disagrees with the loaded table (elements, attribute or n)");
        if (get_u64(d + 16) != off) return fail(OBLIVGM_EINVAL, "fresh token layout offsets do not match");
        const uint32_t combine = d[24];
        for (int b = 25; b < 32; b++)
            if (d[b]) return fail(OBLIVGM_EINVAL, "bad fresh predicate descriptor");
        if (combine > OBLIVGM_COMBINE_OR) return fail(OBLIVGM_EINVAL, "bad combine field");
        if (members[group].empty() && combine != OBLIVGM_COMBINE_AND)
            return fail(OBLIVGM_EINVAL, "a group's first predicate must combine with AND");
        if (gtable[group] >= 0 && gtable[group] != (int)table)
            return fail(OBLIVGM_EINVAL, "an AND-group spans two tables");
        gtable[group] = (int)table;
        members[group].push_back(p);
        FreshPred& F = P->preds[p];
        F.kind = kind;
        F.attr = attr;
        F.step = p;
        F.combine = combine;
        F.lay = fresh_layout(kind == OBLIVGM_PRED_EQ, n, N);
        for (int i = 0; i < 3; i++) F.data[i] = const_cast<uint8_t*>(tok[i]) + off;
        off += F.lay.data_len;
    }
    if (off != get_u64(h[0] + 16)) return fail(OBLIVGM_EINVAL, "fresh token length does not match its predicates");
    // groups reference the predicates through index ranges: reorder into group order
    FreshPred ordered[kFreshMaxPreds];
    uint32_t at = 0;
    P->item_start[0] = 0;
    for (uint32_t g = 0; g < n_groups; g++) {
        if (members[g].empty()) return fail(OBLIVGM_EINVAL, "a group has no predicate");
        const Table& tb = ctx->tables[(uint32_t)gtable[g]];
        FreshGroup& G = P->groups[g];
        for (int j = 0; j < 3; j++) {
            G.share[j] = tb.dev + (uint64_t)j * tb.n_attrs * tb.stride;
            G.out[j] = out[3 * g + j];
            if (!G.out[j] && tb.n_elems) return fail(OBLIVGM_EINVAL, "NULL output");
        }
        G.stride = tb.stride;
        G.table = (uint32_t)gtable[g];
        G.pred_begin = at;
        G.n_preds = (uint32_t)members[g].size();
        for (uint32_t p : members[g]) ordered[at++] = P->preds[p];
        P->item_start[g + 1] = P->item_start[g] + tb.n_elems;
    }
    std::memcpy(P->preds, ordered, sizeof ordered);
    const uint64_t total = P->item_start[n_groups];
    if (total == 0) return OBLIVGM_OK;
    const uint64_t blocks = std::min<uint64_t>((total + kFreshEvalThreads - 1) / kFreshEvalThreads, ctx->sm_count);
    k_filter_fresh<<<(unsigned)blocks, kFreshEvalThreads, kTableBytes, s>>>(*P);
    ctx->launches++;
    ce = cudaGetLastError();
    return ce == cudaSuccess ? OBLIVGM_OK : cuda_fail(ce, "k_filter_fresh launch");
}

namespace ogm {
oblivgm_status set_fresh_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_keygen_fresh<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_keygen_fresh<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_filter_fresh, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, "fresh-key kernel attributes");
}
}  // namespace ogm
