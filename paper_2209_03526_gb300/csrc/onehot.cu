// onehot.cu -- the one-hot mode of the oblivgm library: secEval exactly as the
// paper writes it (Sec. V-B, V-C, Eq. predEval, Alg. 3).  Attribute values are
// stored as binary-RSS shares of one-hot vectors of length D = 2^n (n <= 16),
// packed 32 positions per word.  Each server evaluates its FSS key halves (Z_2
// outputs, beta = 1) at every public position l and computes
//     x = XOR_l Eval(k, l) AND <e_v>_j[l]
// for the share j its key pair is tied to; it XORs its two results, re-shares them
// in binary RSS and the query element's predicates are ANDed in binary RSS.
//
// Two kernels per query:
//  * k_onehot_evalall: every key half at every position, one tree walk per
//    position (the walk code of the masked mode with Z_2 outputs), 32 positions
//    packed into one word by a warp ballot;
//  * k_onehot_group: per AND-group, a warp per 32 elements streams each element's
//    three share rows from HBM, ANDs them with the six half vectors staged in
//    shared memory, reduces parities by ballots, then each lane re-shares and
//    folds its own element and the warp writes packed result words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_fss.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

constexpr uint32_t kNoKey = 0xFFFFFFFFu;

struct HalfDesc {
    uint32_t key0, key1;   // one DPF key, or two DCF keys (a1, a0); key1 = kNoKey for DPF
    uint32_t cbit;         // public constant XORed in by party 0 of a range half
    uint32_t kind;         // OBLIVGM_KEY_DPF / OBLIVGM_KEY_DCF
};

struct EvalAllParams {
    AesParams aes;
    const uint32_t* te0;
    const DevKey* keys;
    const HalfDesc* halves;
    uint32_t* hv;          // [half][words], zeroed before the launch
    uint32_t domain;       // D = 2^n
    uint32_t words;        // max(1, D / 32)
    uint32_t n_halves;
    int log_block;         // m = min(3, n): positions per work item = 2^m
};

// One tree level of DPF / DCF Eval (Z_2 outputs) in direction dir, as in the walks of the
// masked mode: the selected child's seed and control bit (and, for the DCF, the value
// term V += Convert(v) + t * V_CW, taken mod 2).
__device__ __forceinline__ void level_step(const SmemTab& T, const AesParams& A, const DevKey& K, int i, uint32_t dir,
                                           bool dcf, uint32_t s[4], uint32_t& t, uint32_t& V) {
    const uint32_t m = 0u - dir;
    uint32_t o[4];
    aes_sel(T, A.rk_st, A.d_st, m, s, o);
    if (dcf) {
        const uint32_t v0 = aes_sel_w0(T, A.rk_v, A.d_v, m, s);
        V ^= ((v0 ^ s[0]) & 1u) ^ (t & K.vcw[i] & 1u);
    }
#pragma unroll
    for (int w = 0; w < 4; w++) o[w] ^= s[w];
    uint32_t tn = o[0] & 1u;
    o[0] &= ~1u;
    const uint32_t tm = 0u - t;
#pragma unroll
    for (int w = 0; w < 4; w++) s[w] = o[w] ^ (K.scw[i][w] & tm);
    tn ^= t & (((dir ? K.tr : K.tl) >> i) & 1u);
    t = tn;
}

// Eval of one key at the 2^m consecutive positions prefix * 2^m + j, j < 2^m (m <= 3):
// walk the n - m shared levels once, then expand the last m levels depth first
// (2^(m+1) - 2 more levels instead of m per position).  Bit j of the result is
// position prefix * 2^m + j.
__device__ __forceinline__ uint32_t eval_block(const SmemTab& T, const AesParams& A, const DevKey& K, uint32_t prefix,
                                               int m) {
    const int n = (int)K.n;
    const bool dcf = K.kind == OBLIVGM_KEY_DCF;
    uint32_t s[4] = {K.seed[0], K.seed[1], K.seed[2], K.seed[3]};
    uint32_t t = K.party, V = 0;
    for (int i = 0; i < n - m; i++) level_step(T, A, K, i, (prefix >> (n - m - 1 - i)) & 1u, dcf, s, t, V);
    uint32_t bits = 0;
    const uint32_t cwf = K.cw_final & 1u;
    if (m == 0) {
        return V ^ ((s[0] >> 1) & 1u) ^ (t & cwf);
    }
    // depth-first over the last m levels (m = 1, 2 or 3), keeping one node per level
    uint32_t s1[4], t1, V1, s2[4], t2, V2;
    const int L1 = n - m;            // level index of the first expanded level
    for (uint32_t b1 = 0; b1 < 2; b1++) {
#pragma unroll
        for (int w = 0; w < 4; w++) s1[w] = s[w];
        t1 = t; V1 = V;
        level_step(T, A, K, L1, b1, dcf, s1, t1, V1);
        if (m == 1) { bits |= (V1 ^ ((s1[0] >> 1) & 1u) ^ (t1 & cwf)) << b1; continue; }
        for (uint32_t b2 = 0; b2 < 2; b2++) {
#pragma unroll
            for (int w = 0; w < 4; w++) s2[w] = s1[w];
            t2 = t1; V2 = V1;
            level_step(T, A, K, L1 + 1, b2, dcf, s2, t2, V2);
            if (m == 2) { bits |= (V2 ^ ((s2[0] >> 1) & 1u) ^ (t2 & cwf)) << (b1 * 2 + b2); continue; }
            for (uint32_t b3 = 0; b3 < 2; b3++) {
                uint32_t s3[4] = {s2[0], s2[1], s2[2], s2[3]}, t3 = t2, V3 = V2;
                level_step(T, A, K, L1 + 2, b3, dcf, s3, t3, V3);
                bits |= (V3 ^ ((s3[0] >> 1) & 1u) ^ (t3 & cwf)) << (b1 * 4 + b2 * 2 + b3);
            }
        }
    }
    return bits;
}

// Every key half at every position.  Work item = (half, block of 2^m positions); the
// items are spread over one persistent CTA per SM.  hv must be zeroed: each item ORs
// its 2^m bits into place.
__global__ void __launch_bounds__(1024, 1) k_onehot_evalall(const __grid_constant__ EvalAllParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const int m = P.log_block;
    const uint32_t per_half = P.domain >> m;
    const uint64_t items = (uint64_t)P.n_halves * per_half;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < items;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t half = (uint32_t)(idx / per_half), prefix = (uint32_t)(idx % per_half);
        const HalfDesc H = P.halves[half];
        uint32_t bits = eval_block(T, P.aes, P.keys[H.key0], prefix, m);
        if (H.key1 != kNoKey) bits ^= eval_block(T, P.aes, P.keys[H.key1], prefix, m);
        if (H.cbit) bits ^= (m == 5 ? 0xFFFFFFFFu : ((1u << (1u << m)) - 1u));
        const uint32_t pos = prefix << m;
        atomicOr(P.hv + (uint64_t)half * P.words + pos / 32, bits << (pos % 32));
    }
}

struct GroupParams {
    uint32_t rk_prf[3][44];
    const uint32_t* te4;          // global-memory T-tables for the re-share PRF
    const uint32_t* share[3];     // share set j of the table: [attr][elem][words]
    uint32_t* out[3];             // packed result share sets, ceil(n_elems / 32) words
    const uint32_t* hv;           // [half][words]
    const uint32_t* pred_attr;    // per predicate of the group
    const uint32_t* pred_step;
    const uint32_t* pred_half;    // index of the predicate's first half (6 in order [server][half])
    uint64_t n_elems;
    uint32_t words;
    uint32_t n_preds;
    uint32_t table_id, query_id;
};

__device__ __forceinline__ uint32_t prf_bit(const GlobalTab& T, const uint32_t* rk, uint64_t el, uint32_t step,
                                            uint32_t table, uint32_t query) {
    const uint32_t ctr[4] = {(uint32_t)el, (uint32_t)(el >> 32), step | (table << 16), query};
    return aes_one_w0(T, rk, ctr) & 1u;
}

// binary re-share: r_i = z_i xor F(k_i) xor F(k_{i-1})
__device__ __forceinline__ void reshare_bits(const GlobalTab& T, const GroupParams& P, const uint32_t z[3],
                                             uint32_t out[3], uint64_t el, uint32_t step) {
    uint32_t f[3];
#pragma unroll 1
    for (int i = 0; i < 3; i++) f[i] = prf_bit(T, P.rk_prf[i], el, step, P.table_id, P.query_id);
    out[0] = z[0] ^ f[0] ^ f[2];
    out[1] = z[1] ^ f[1] ^ f[0];
    out[2] = z[2] ^ f[2] ^ f[1];
}

__device__ __forceinline__ uint32_t warp_parity(uint32_t acc) {
    return __popc(__ballot_sync(0xFFFFFFFFu, __popc(acc) & 1u)) & 1u;
}

__global__ void __launch_bounds__(256) k_onehot_group(const __grid_constant__ GroupParams P) {
    extern __shared__ __align__(16) uint32_t hvs[];   // the current predicate's six half vectors
    const GlobalTab T{P.te4};
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t W = P.words;
    const uint64_t tile_elems = (uint64_t)blockDim.x;   // 32 elements per warp
    for (uint64_t tile = blockIdx.x; tile * tile_elems < P.n_elems; tile += gridDim.x) {
        const uint64_t base = tile * tile_elems + (uint64_t)warp * 32;
        const uint64_t my_e = base + lane;               // the element this lane folds
        uint32_t acc[3] = {0, 0, 0};
        for (uint32_t k = 0; k < P.n_preds; k++) {
            __syncthreads();
            const uint32_t* src = P.hv + (uint64_t)P.pred_half[k] * W;
            for (uint32_t i = threadIdx.x; i < 6 * W; i += blockDim.x) hvs[i] = src[i];
            __syncthreads();
            const uint64_t row = (uint64_t)P.pred_attr[k] * P.n_elems;
            uint32_t z[3] = {0, 0, 0};
            for (uint32_t c = 0; c < 32; c++) {
                const uint64_t e = base + c;
                if (e >= P.n_elems) break;                 // uniform across the warp
                // share j meets server j's first half and server j-1's second half
                uint32_t x[3][2];
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const uint32_t* d = P.share[j] + (row + e) * W;
                    const uint32_t* h0 = hvs + (j * 2 + 0) * W;
                    const uint32_t* h1 = hvs + (((j + 2) % 3) * 2 + 1) * W;
                    uint32_t a0 = 0, a1 = 0;
                    if ((W & 127u) == 0) {
                        for (uint32_t w = lane * 4; w < W; w += 128) {
                            const uint4 v = __ldg(reinterpret_cast<const uint4*>(d + w));
                            const uint4 p = *reinterpret_cast<const uint4*>(h0 + w);
                            const uint4 q = *reinterpret_cast<const uint4*>(h1 + w);
                            a0 ^= (v.x & p.x) ^ (v.y & p.y) ^ (v.z & p.z) ^ (v.w & p.w);
                            a1 ^= (v.x & q.x) ^ (v.y & q.y) ^ (v.z & q.z) ^ (v.w & q.w);
                        }
                    } else {
                        for (uint32_t w = lane; w < W; w += 32) {
                            const uint32_t v = __ldg(d + w);
                            a0 ^= v & h0[w];
                            a1 ^= v & h1[w];
                        }
                    }
                    x[j][0] = warp_parity(a0);
                    x[j][1] = warp_parity(a1);
                }
                // CS_i: its first half met share i, its second share i+1
                if (lane == c) {
                    z[0] = x[0][0] ^ x[1][1];
                    z[1] = x[1][0] ^ x[2][1];
                    z[2] = x[2][0] ^ x[0][1];
                }
            }
            uint32_t b[3];
            reshare_bits(T, P, z, b, my_e, P.pred_step[k]);
            if (k == 0) {
                acc[0] = b[0]; acc[1] = b[1]; acc[2] = b[2];
            } else {
                uint32_t w[3];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const int i1 = (i + 1) % 3;
                    w[i] = (acc[i] & b[i]) ^ (acc[i] & b[i1]) ^ (acc[i1] & b[i]);
                }
                reshare_bits(T, P, w, acc, my_e, 64u + P.pred_step[k]);
            }
        }
        const bool valid = my_e < P.n_elems;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, valid && (acc[i] & 1u));
            if (lane == 0 && base < P.n_elems) P.out[i][base / 32] = word;
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
    std::string err;
    oblivgm_status st = keygen(preds, n_preds, n_bits, seed, tok, cap, out_len, &err, /*onehot=*/true);
    if (st != OBLIVGM_OK) return fail(st, err);
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_load_onehot(oblivgm_ctx* ctx, uint32_t table_id, uint64_t n_elems,
                                              uint32_t n_attrs, uint32_t n_bits,
                                              const uint32_t* const share_sets[3], int32_t mem_kind, void* stream) {
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
    std::vector<DevKey> keys;
    std::vector<HalfDesc> halves;
    for (const ParsedPred& pp : q.preds) {
        const bool eq = pp.kind == OBLIVGM_PRED_EQ;
        const uint32_t nsub = eq ? 1 : 2, k0 = (uint32_t)keys.size();
        keys.insert(keys.end(), pp.keys.begin(), pp.keys.end());
        for (uint32_t hh = 0; hh < 6; hh++) {
            HalfDesc h{};
            h.key0 = k0 + hh * nsub;
            h.key1 = eq ? kNoKey : k0 + hh * nsub + 1;
            h.kind = eq ? OBLIVGM_KEY_DPF : OBLIVGM_KEY_DCF;
            h.cbit = (!eq && pp.keys[hh * nsub].party == 0) ? (pp.cbeta & 1u) : 0u;
            halves.push_back(h);
        }
    }
    std::vector<uint32_t> pattr, pstep, phalf;
    std::vector<size_t> gbegin;
    for (uint32_t g = 0; g < n_groups; g++) {
        gbegin.push_back(pattr.size());
        for (uint32_t p : members[g]) {
            pattr.push_back(q.preds[p].attr);
            pstep.push_back(q.preds[p].step);
            phalf.push_back(6 * p);
        }
    }
    const size_t np = pattr.size();
    // scratch: keys | halves | pred arrays (3 x np) | half vectors
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t off_h = up(keys.size() * sizeof(DevKey));
    const size_t off_p = off_h + up(halves.size() * sizeof(HalfDesc));
    const size_t off_v = off_p + up(3 * np * sizeof(uint32_t));
    const size_t total = off_v + halves.size() * words * sizeof(uint32_t);
    std::vector<unsigned char> img(off_v, 0);
    std::memcpy(img.data(), keys.data(), keys.size() * sizeof(DevKey));
    std::memcpy(img.data() + off_h, halves.data(), halves.size() * sizeof(HalfDesc));
    std::memcpy(img.data() + off_p, pattr.data(), np * 4);
    std::memcpy(img.data() + off_p + np * 4, pstep.data(), np * 4);
    std::memcpy(img.data() + off_p + 2 * np * 4, phalf.data(), np * 4);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = nullptr;
    ce = cudaMallocAsync(reinterpret_cast<void**>(&ws), total, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot scratch");
    ce = cudaMemcpyAsync(ws, img.data(), off_v, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot descriptor upload");
    EvalAllParams E{};
    E.aes = ctx->aes;
    E.te0 = ctx->d_te0;
    E.keys = reinterpret_cast<const DevKey*>(ws);
    E.halves = reinterpret_cast<const HalfDesc*>(ws + off_h);
    E.hv = reinterpret_cast<uint32_t*>(ws + off_v);
    E.domain = domain;
    E.words = words;
    E.n_halves = (uint32_t)halves.size();
    E.log_block = (int)std::min<uint32_t>(3, n);
    ce = cudaMemsetAsync(E.hv, 0, halves.size() * words * sizeof(uint32_t), s);
    if (ce != cudaSuccess) return cuda_fail(ce, "half-vector clear");
    {
        const uint64_t items = (uint64_t)halves.size() * (domain >> E.log_block);
        const unsigned grid = (unsigned)std::min<uint64_t>((items + 1023) / 1024, (uint64_t)ctx->sm_count);
        k_onehot_evalall<<<grid, 1024, kTableBytes, s>>>(E);
    }
    ctx->launches++;
    const size_t smem = 6 * (size_t)words * sizeof(uint32_t);
    for (uint32_t g = 0; g < n_groups; g++) {
        const OnehotTable& tb = ctx->onehot_tables.at(q.preds[members[g][0]].table);
        if (tb.n_elems == 0) continue;
        GroupParams G{};
        std::memcpy(G.rk_prf, ctx->rk_prf, sizeof G.rk_prf);
        G.te4 = ctx->d_te4;
        const size_t set_words = (size_t)tb.n_attrs * tb.n_elems * tb.words;
        for (int j = 0; j < 3; j++) {
            G.share[j] = tb.dev + j * set_words;
            G.out[j] = out[3 * g + j];
            if (!G.out[j]) return fail(OBLIVGM_EINVAL, "NULL output pointer");
        }
        G.hv = E.hv;
        const uint32_t* pa = reinterpret_cast<const uint32_t*>(ws + off_p);
        G.pred_attr = pa + gbegin[g];
        G.pred_step = pa + np + gbegin[g];
        G.pred_half = pa + 2 * np + gbegin[g];
        G.n_elems = tb.n_elems;
        G.words = words;
        G.n_preds = (uint32_t)members[g].size();
        G.table_id = q.preds[members[g][0]].table;
        G.query_id = query_id;
        const uint64_t tiles = (tb.n_elems + 255) / 256;
        const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)ctx->sm_count * 4);
        k_onehot_group<<<grid, 256, smem, s>>>(G);
        ctx->launches++;
    }
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot launch");
    ce = cudaFreeAsync(ws, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "one-hot scratch release");
    return OBLIVGM_OK;
}

namespace ogm {

oblivgm_status set_onehot_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_onehot_evalall, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_onehot_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 6 * (1 << kMaxOnehotBits) / 32 * (int)sizeof(uint32_t));
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, "one-hot kernel attributes");
}

}  // namespace ogm
