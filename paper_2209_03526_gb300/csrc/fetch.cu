// fetch.cu -- secFetch, case I (Alg. 4, Sec. V-D): fetch the one matching element of a
// filter obliviously.  With [[x_c]] the RSS result of an AND-group over a table's C
// elements (exactly one x_c = 1), the servers compute, over Z_{2^32},
//   index:   sum_c c * [[x_c]]            (public weights: linear, stays RSS)
//   attr a:  sum_c [[v_c]] (x) [[x_c]]     (RSS product per element, summed, one re-share)
// The re-share counter is (element = a, step = 256 + group, table, query).  Two kernels:
// k_fetch_clear zeroes the outputs and lets k_fetch, launched as its programmatic
// dependent, start at once: k_fetch streams the candidates while the clear runs and waits
// for it (griddepcontrol.wait) only before adding its sums into the outputs atomically.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>

#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

constexpr int kFetchMaxAttrs = 64;
constexpr uint32_t kFetchStep = 256;
constexpr int kFetchThreads = 256;
constexpr int kFetchCtasPerSm = 5;          // 48 registers: 1,280 threads per SM

struct FetchParams {
    const uint32_t* x[3];          // filter result share sets, n_elems each
    const uint32_t* v[3];          // table share set j at attribute 0: [attr][stride]
    uint64_t stride;
    uint64_t n_elems;
    uint32_t attrs[kFetchMaxAttrs];
    uint32_t n_attrs;
    uint32_t vec4;                 // the three result share sets are 16-byte aligned
    uint32_t mask[3][kFetchMaxAttrs];   // F(k_i, ctr) - F(k_{i-1}, ctr) per share set and attribute
    uint32_t* out;                 // [3][1 + n_attrs], zeroed by k_fetch_clear
};

// zero the outputs; the dependent k_fetch may launch right away
__global__ void k_fetch_clear(uint32_t* out, uint32_t n) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) out[t] = 0u;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

// one candidate's contribution to column k: the index row adds c * <x_c>_i, an attribute
// row the RSS product share w_i = v_i x_i + v_i x_{i+1} + v_{i+1} x_i
__device__ __forceinline__ void fetch_add(uint32_t acc[3], bool index_col, uint32_t c, const uint32_t x[3],
                                          const uint32_t v[3]) {
    if (index_col) {
        acc[0] += c * x[0]; acc[1] += c * x[1]; acc[2] += c * x[2];
    } else {
        acc[0] += v[0] * x[0] + v[0] * x[1] + v[1] * x[0];
        acc[1] += v[1] * x[1] + v[1] * x[2] + v[2] * x[1];
        acc[2] += v[2] * x[2] + v[2] * x[0] + v[0] * x[2];
    }
}

// Every output word is a sum mod 2^32, so each CTA adds its part straight into the
// zeroed outputs and the order of the additions does not matter:
//   index (column 0), share set i:    sum_c c * <x_c>_i
//   attribute a (column 1 + k), set i: sum_c w_i(c) + F(k_i, ctr) - F(k_{i-1}, ctr),
//   ctr = (a, 256 + group, table, query).
// CTA 0 adds the re-share masks (PRF blocks the host computes: they depend only on the
// attribute, the step, the table and the query); the index has public weights and needs none.
// Work split: the launch has a multiple of `cols` warps, and warp w always serves column
// w % cols, for blocks of 32 x 4 candidates w / cols, w / cols + W / cols, ... (W warps):
// each lane issues six 16-byte loads (its four candidates' result shares and the column's
// attribute shares) per step, every SM streams many such steps, and a warp keeps three
// accumulators.  The result shares are read once per column; the other columns' reads of
// the same block come from warps of the same CTA, mostly out of L1 / L2.
__global__ void __launch_bounds__(kFetchThreads, kFetchCtasPerSm) k_fetch(const __grid_constant__ FetchParams P) {
    __shared__ uint32_t part[1 + kFetchMaxAttrs][3];
    const uint32_t cols = 1 + P.n_attrs;
    for (uint32_t t = threadIdx.x; t < 3 * cols; t += blockDim.x) part[t / 3][t % 3] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t k = (uint32_t)(warp % cols);
    const uint64_t b0 = warp / cols, bstep = n_warps / cols;
    const bool index_col = k == 0;
    const uint64_t arow = index_col ? 0 : (uint64_t)P.attrs[k - 1] * P.stride;
    uint32_t acc[3] = {0, 0, 0};
    // 16-byte loads of four candidates while the result shares are 16-byte aligned (the
    // table rows always are), then one candidate at a time for the rest
    const uint64_t nq = P.vec4 ? P.n_elems / 4 : 0;
    for (uint64_t b = b0; b * 32 < nq; b += bstep) {
        const uint64_t q = b * 32 + lane;
        if (q < nq) {
            uint4 X[3], A[3];
#pragma unroll
            for (int j = 0; j < 3; j++) X[j] = __ldg(reinterpret_cast<const uint4*>(P.x[j]) + q);
            if (!index_col) {
#pragma unroll
                for (int j = 0; j < 3; j++) A[j] = __ldg(reinterpret_cast<const uint4*>(P.v[j] + arow) + q);
            } else {
#pragma unroll
                for (int j = 0; j < 3; j++) A[j] = make_uint4(0, 0, 0, 0);
            }
            const uint32_t c = (uint32_t)(4 * q);
            { const uint32_t x[3] = {X[0].x, X[1].x, X[2].x}, v[3] = {A[0].x, A[1].x, A[2].x}; fetch_add(acc, index_col, c, x, v); }
            { const uint32_t x[3] = {X[0].y, X[1].y, X[2].y}, v[3] = {A[0].y, A[1].y, A[2].y}; fetch_add(acc, index_col, c + 1, x, v); }
            { const uint32_t x[3] = {X[0].z, X[1].z, X[2].z}, v[3] = {A[0].z, A[1].z, A[2].z}; fetch_add(acc, index_col, c + 2, x, v); }
            { const uint32_t x[3] = {X[0].w, X[1].w, X[2].w}, v[3] = {A[0].w, A[1].w, A[2].w}; fetch_add(acc, index_col, c + 3, x, v); }
        }
    }
    for (uint64_t b = b0; 4 * nq + b * 32 < P.n_elems; b += bstep) {
        const uint64_t c = 4 * nq + b * 32 + lane;
        if (c < P.n_elems) {
            uint32_t x[3], v[3] = {0, 0, 0};
#pragma unroll
            for (int j = 0; j < 3; j++) x[j] = __ldg(P.x[j] + c);
            if (!index_col)
#pragma unroll
                for (int j = 0; j < 3; j++) v[j] = __ldg(P.v[j] + arow + c);
            fetch_add(acc, index_col, (uint32_t)c, x, v);   // weights mod 2^32
        }
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const uint32_t t = warp_sum(acc[i]);
        if (lane == 0) atomicAdd(&part[k][i], t);
    }
    __syncthreads();
    // the outputs are written only after k_fetch_clear has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (blockIdx.x == 0)
        for (uint32_t t = threadIdx.x; t < 3 * P.n_attrs; t += blockDim.x)
            atomicAdd(P.out + (t / P.n_attrs) * cols + 1 + t % P.n_attrs, P.mask[t / P.n_attrs][t % P.n_attrs]);
    for (uint32_t t = threadIdx.x; t < 3 * cols; t += blockDim.x) {
        const uint32_t col = t / 3, i = t % 3;
        atomicAdd(P.out + i * cols + col, part[col][i]);
    }
}

}  // namespace

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_fetch_unique(oblivgm_ctx* ctx, uint32_t query_id, uint32_t group,
                                               uint32_t table_id, const uint32_t* const x[3], uint32_t n_attrs,
                                               const uint32_t* attrs, uint32_t* out, void* stream) {
    const NvtxRange nvtx_range("oblivgm_fetch_unique");
    if (!ctx || !x || !out || (n_attrs && !attrs)) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (n_attrs > (uint32_t)kFetchMaxAttrs) return fail(OBLIVGM_EINVAL, "at most 64 attributes per fetch");
    if (group > 0xFFFF - kFetchStep) return fail(OBLIVGM_EINVAL, "group index too large");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    auto it = ctx->tables.find(table_id);
    if (it == ctx->tables.end()) return fail(OBLIVGM_ENOENT, "no such table");
    const Table& tb = it->second;
    for (int j = 0; j < 3; j++)
        if (!x[j] && tb.n_elems) return fail(OBLIVGM_EINVAL, "NULL filter share set");
    for (uint32_t a = 0; a < n_attrs; a++)
        if (attrs[a] >= tb.n_attrs) return fail(OBLIVGM_EINVAL, "attribute outside the table");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t cols = 1 + n_attrs;
    // warps: a multiple of cols (each warp serves one column), enough for one block of
    // 32 x 4 candidates per warp and column, at most kFetchCtasPerSm CTAs per SM
    const uint64_t warps_per_cta = kFetchThreads / 32;
    const uint64_t unit = cols / std::gcd<uint64_t>(cols, warps_per_cta);   // CTAs per whole round of columns
    const uint64_t blocks32 = std::max<uint64_t>(1, (tb.n_elems + 127) / 128);
    const uint64_t want = (blocks32 * cols + warps_per_cta - 1) / warps_per_cta;
    const uint64_t cap = std::max<uint64_t>(unit, (uint64_t)kFetchCtasPerSm * ctx->sm_count / unit * unit);
    const uint64_t blocks = std::min<uint64_t>((want + unit - 1) / unit * unit, cap);
    FetchParams F{};
    for (int j = 0; j < 3; j++) {
        F.x[j] = x[j];
        F.v[j] = tb.dev + (uint64_t)j * tb.n_attrs * tb.stride;
    }
    F.stride = tb.stride;
    F.n_elems = tb.n_elems;
    if (n_attrs) std::memcpy(F.attrs, attrs, n_attrs * sizeof(uint32_t));
    F.n_attrs = n_attrs;
    // re-share masks: F(k, ctr) = word 0 of AES_k(attr || step || table || query)
    for (uint32_t a = 0; a < n_attrs; a++) {
        const uint32_t ctr[4] = {attrs[a], 0u, (kFetchStep + group) | (table_id << 16), query_id};
        uint32_t f[3];
        for (int i = 0; i < 3; i++) {
            RoundKeys rk;
            std::memcpy(rk.w, ctx->rk_prf[i], sizeof rk.w);
            uint32_t o[4];
            aes_encrypt(rk, ctr, o);
            f[i] = o[0];
        }
        for (int i = 0; i < 3; i++) F.mask[i][a] = f[i] - f[(i + 2) % 3];
    }
    F.out = out;
    F.vec4 = 1;
    for (int j = 0; j < 3; j++)
        if (reinterpret_cast<uintptr_t>(x[j]) % 16) F.vec4 = 0;
    k_fetch_clear<<<1, 256, 0, s>>>(out, 3 * cols);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch clear launch");
    ctx->launches++;
    // the streaming kernel as a programmatic dependent of the clear: it starts at once and
    // waits (griddepcontrol.wait) for the clear only before it adds into the outputs
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)blocks);
    lc.blockDim = dim3(kFetchThreads);
    lc.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = la;
    lc.numAttrs = 1;
    ce = cudaLaunchKernelEx(&lc, k_fetch, F);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch launch");
    ctx->launches++;
    return OBLIVGM_OK;
}
