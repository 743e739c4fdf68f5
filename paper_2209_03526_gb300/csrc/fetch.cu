// fetch.cu -- secFetch, case I (Alg. 4, Sec. V-D): fetch the one matching element of a
// filter obliviously.  With [[x_c]] the RSS result of an AND-group over a table's C
// elements (exactly one x_c = 1), the servers compute, over Z_{2^32},
//   index:   sum_c c * [[x_c]]            (public weights: linear, stays RSS)
//   attr a:  sum_c [[v_c]] (x) [[x_c]]     (RSS product per element, summed, one re-share)
// The re-share counter is (element = a, step = 256 + group, table, query).  One kernel
// after a clear of the outputs: every CTA adds its sums into them atomically.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

constexpr int kFetchMaxAttrs = 64;
constexpr uint32_t kFetchStep = 256;

#ifndef OGM_FETCH_COLS
#define OGM_FETCH_COLS 6
#endif
#ifndef OGM_FETCH_CTAS_PER_SM
#define OGM_FETCH_CTAS_PER_SM 2
#endif
constexpr int kFetchThreads = 512;
constexpr uint32_t kFetchCols = OGM_FETCH_COLS;
constexpr int kFetchCtasPerSm = OGM_FETCH_CTAS_PER_SM;

struct FetchParams {
    const uint32_t* x[3];          // filter result share sets, n_elems each
    const uint32_t* v[3];          // table share set j at attribute 0: [attr][stride]
    uint64_t stride;
    uint64_t n_elems;
    uint32_t attrs[kFetchMaxAttrs];
    uint32_t n_attrs;
    uint32_t vec4;                 // the three result share sets are 16-byte aligned
    uint32_t mask[3][kFetchMaxAttrs];   // F(k_i, ctr) - F(k_{i-1}, ctr) per share set and attribute
    uint32_t* out;                 // [3][1 + n_attrs], zero before the launch
};

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

// sum of a value over the CTA (every thread gets it); red holds one word per warp
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* red) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; w++) t += red[w];
    return t;
}

// Every output word is a sum mod 2^32, so each CTA adds its part straight into the
// zeroed outputs and the order of the additions does not matter:
//   index (column 0), share set i:    sum_c c * <x_c>_i
//   attribute a (column 1 + k), set i: sum_c w_i(c) + F(k_i, ctr) - F(k_{i-1}, ctr),
//   w_i = v_i x_i + v_i x_{i+1} + v_{i+1} x_i (the RSS product), ctr = (a, 256 + group, table, query).
// CTA 0 adds the re-share masks (PRF blocks the host computes: they depend only on the
// attribute, the step, the table and the query); the index has public weights and needs none.  One pass over the candidates per group of up to 8 columns:
// each thread loads an element's result shares and every attribute share first, then sums.
__global__ void __launch_bounds__(kFetchThreads, kFetchCtasPerSm) k_fetch(const __grid_constant__ FetchParams P) {
    __shared__ uint32_t red[kFetchThreads / 32];
    const uint32_t cols = 1 + P.n_attrs;
    if (blockIdx.x == 0)
        for (uint32_t t = threadIdx.x; t < 3 * P.n_attrs; t += blockDim.x)
            atomicAdd(P.out + (t / P.n_attrs) * cols + 1 + t % P.n_attrs, P.mask[t / P.n_attrs][t % P.n_attrs]);
    for (uint32_t c0 = 0; c0 < cols; c0 += kFetchCols) {
        uint32_t acc[kFetchCols][3];
#pragma unroll
        for (uint32_t k = 0; k < kFetchCols; k++) acc[k][0] = acc[k][1] = acc[k][2] = 0;
        // 16-byte loads of four candidates while the result shares are 16-byte aligned (the
        // table rows always are), then one candidate at a time for the rest
        uint64_t c_begin = P.n_elems;
        if (P.vec4) {
            const uint64_t n4 = P.n_elems / 4;
            for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
                 q += (uint64_t)gridDim.x * blockDim.x) {
                const uint4 X0 = __ldg(reinterpret_cast<const uint4*>(P.x[0]) + q);
                const uint4 X1 = __ldg(reinterpret_cast<const uint4*>(P.x[1]) + q);
                const uint4 X2 = __ldg(reinterpret_cast<const uint4*>(P.x[2]) + q);
                const uint32_t xs[3][4] = {{X0.x, X0.y, X0.z, X0.w}, {X1.x, X1.y, X1.z, X1.w},
                                           {X2.x, X2.y, X2.z, X2.w}};
#pragma unroll
                for (uint32_t k = 0; k < kFetchCols; k++) {
                    const uint32_t col = c0 + k;
                    if (col == 0) {
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const uint32_t cw = (uint32_t)(4 * q + e);
                            acc[k][0] += cw * xs[0][e]; acc[k][1] += cw * xs[1][e]; acc[k][2] += cw * xs[2][e];
                        }
                    } else if (col < cols) {
                        const uint64_t off = ((uint64_t)P.attrs[col - 1] * P.stride) / 4 + q;
                        const uint4 A0 = __ldg(reinterpret_cast<const uint4*>(P.v[0]) + off);
                        const uint4 A1 = __ldg(reinterpret_cast<const uint4*>(P.v[1]) + off);
                        const uint4 A2 = __ldg(reinterpret_cast<const uint4*>(P.v[2]) + off);
                        const uint32_t as[3][4] = {{A0.x, A0.y, A0.z, A0.w}, {A1.x, A1.y, A1.z, A1.w},
                                                   {A2.x, A2.y, A2.z, A2.w}};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            acc[k][0] += as[0][e] * xs[0][e] + as[0][e] * xs[1][e] + as[1][e] * xs[0][e];
                            acc[k][1] += as[1][e] * xs[1][e] + as[1][e] * xs[2][e] + as[2][e] * xs[1][e];
                            acc[k][2] += as[2][e] * xs[2][e] + as[2][e] * xs[0][e] + as[0][e] * xs[2][e];
                        }
                    }
                }
            }
            c_begin = 4 * n4;
        } else {
            c_begin = 0;
        }
        for (uint64_t c = c_begin + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P.n_elems;
             c += (uint64_t)gridDim.x * blockDim.x) {
            const uint32_t x0 = __ldg(P.x[0] + c), x1 = __ldg(P.x[1] + c), x2 = __ldg(P.x[2] + c);
            uint32_t a[kFetchCols][3];
#pragma unroll
            for (uint32_t k = 0; k < kFetchCols; k++) {
                const uint32_t col = c0 + k;
                a[k][0] = a[k][1] = a[k][2] = 0;
                if (col >= 1 && col < cols) {
                    const uint64_t off = (uint64_t)P.attrs[col - 1] * P.stride + c;
                    a[k][0] = __ldg(P.v[0] + off);
                    a[k][1] = __ldg(P.v[1] + off);
                    a[k][2] = __ldg(P.v[2] + off);
                }
            }
#pragma unroll
            for (uint32_t k = 0; k < kFetchCols; k++) {
                if (c0 + k == 0) {
                    const uint32_t cw = (uint32_t)c;   // weights mod 2^32
                    acc[k][0] += cw * x0; acc[k][1] += cw * x1; acc[k][2] += cw * x2;
                } else {                               // zero for columns past the last
                    acc[k][0] += a[k][0] * x0 + a[k][0] * x1 + a[k][1] * x0;
                    acc[k][1] += a[k][1] * x1 + a[k][1] * x2 + a[k][2] * x1;
                    acc[k][2] += a[k][2] * x2 + a[k][2] * x0 + a[k][0] * x2;
                }
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < kFetchCols; k++) {
            if (c0 + k >= cols) break;
            for (int i = 0; i < 3; i++) {
                const uint32_t t = block_sum(acc[k][i], red);
                if (threadIdx.x == 0) atomicAdd(P.out + i * cols + c0 + k, t);
            }
        }
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
    ce = cudaMemsetAsync(out, 0, 3 * cols * sizeof(uint32_t), s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch output clear");
    // two 512-thread CTAs per SM (64 registers)
    const uint64_t blocks = std::max<uint64_t>(
        1, std::min<uint64_t>((tb.n_elems + kFetchThreads - 1) / kFetchThreads,
                              (uint64_t)kFetchCtasPerSm * ctx->sm_count));
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
    k_fetch<<<(unsigned)blocks, kFetchThreads, 0, s>>>(F);
    ctx->launches++;
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch launch");
    return OBLIVGM_OK;
}
