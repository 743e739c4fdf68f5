// fetch.cu -- secFetch, case I (Alg. 4, Sec. V-D): fetch the one matching element of a
// filter obliviously.  With [[x_c]] the RSS result of an AND-group over a table's C
// elements (exactly one x_c = 1), the servers compute, over Z_{2^32},
//   index:   sum_c c * [[x_c]]            (public weights: linear, stays RSS)
//   attr a:  sum_c [[v_c]] (x) [[x_c]]     (RSS product per element, summed, one re-share)
// The re-share counter is (element = a, step = 256 + group, table, query).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "device_fss.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

constexpr int kFetchMaxAttrs = 64;
constexpr uint32_t kFetchStep = 256;

struct FetchParams {
    const uint32_t* x[3];          // filter result share sets, n_elems each
    const uint32_t* v[3];          // table share set j at attribute 0: [attr][stride]
    uint64_t stride;
    uint64_t n_elems;
    uint32_t attrs[kFetchMaxAttrs];
    uint32_t* acc;                 // [1 + n_attrs][3], zeroed
};

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

// blockIdx.y = 0: index sums; y = 1 + a: the RSS products with attribute attrs[a]
__global__ void __launch_bounds__(256) k_fetch_sum(const __grid_constant__ FetchParams P) {
    const uint32_t y = blockIdx.y;
    uint32_t s[3] = {0, 0, 0};
    const uint32_t* v[3] = {nullptr, nullptr, nullptr};
    if (y > 0)
        for (int j = 0; j < 3; j++) v[j] = P.v[j] + (uint64_t)P.attrs[y - 1] * P.stride;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P.n_elems;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x0 = __ldg(P.x[0] + c), x1 = __ldg(P.x[1] + c), x2 = __ldg(P.x[2] + c);
        if (y == 0) {
            const uint32_t cw = (uint32_t)c;   // weights mod 2^32
            s[0] += cw * x0; s[1] += cw * x1; s[2] += cw * x2;
        } else {
            const uint32_t a0 = __ldg(v[0] + c), a1 = __ldg(v[1] + c), a2 = __ldg(v[2] + c);
            // w_i = v_i x_i + v_i x_{i+1} + v_{i+1} x_i
            s[0] += a0 * x0 + a0 * x1 + a1 * x0;
            s[1] += a1 * x1 + a1 * x2 + a2 * x1;
            s[2] += a2 * x2 + a2 * x0 + a0 * x2;
        }
    }
    __shared__ uint32_t part[8][3];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < 3; i++) {
        const uint32_t w = warp_sum(s[i]);
        if (lane == 0) part[warp][i] = w;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < blockDim.x / 32; w++) t += part[w][threadIdx.x];
        atomicAdd(P.acc + y * 3 + threadIdx.x, t);   // addition mod 2^32: order-independent
    }
}

struct FinishParams {
    uint32_t rk_prf[3][44];
    const uint32_t* te4;
    const uint32_t* acc;
    uint32_t* out;                 // [3][1 + n_attrs]
    uint32_t attrs[kFetchMaxAttrs];
    uint32_t n_attrs, step, table, query;
};

__global__ void k_fetch_finish(const __grid_constant__ FinishParams P) {
    const uint32_t t = threadIdx.x;
    const uint32_t cols = 1 + P.n_attrs;
    if (t >= cols) return;
    const uint32_t* a = P.acc + t * 3;
    if (t == 0) {                  // the index needs no re-share
        for (int i = 0; i < 3; i++) P.out[i * cols] = a[i];
        return;
    }
    const GlobalTab T{P.te4};
    const uint32_t ctr[4] = {P.attrs[t - 1], 0u, P.step | (P.table << 16), P.query};
    uint32_t f[3];
    for (int i = 0; i < 3; i++) f[i] = aes_one_w0(T, P.rk_prf[i], ctr);
    for (int i = 0; i < 3; i++) P.out[i * cols + t] = a[i] + f[i] - f[(i + 2) % 3];
}

}  // namespace

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_fetch_unique(oblivgm_ctx* ctx, uint32_t query_id, uint32_t group,
                                               uint32_t table_id, const uint32_t* const x[3], uint32_t n_attrs,
                                               const uint32_t* attrs, uint32_t* out, void* stream) {
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
    uint32_t* acc = nullptr;
    const size_t acc_bytes = (size_t)(1 + n_attrs) * 3 * sizeof(uint32_t);
    ce = cudaMallocAsync(reinterpret_cast<void**>(&acc), acc_bytes, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch scratch");
    ce = cudaMemsetAsync(acc, 0, acc_bytes, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch scratch clear");
    if (tb.n_elems) {
        FetchParams F{};
        for (int j = 0; j < 3; j++) {
            F.x[j] = x[j];
            F.v[j] = tb.dev + (uint64_t)j * tb.n_attrs * tb.stride;
        }
        F.stride = tb.stride;
        F.n_elems = tb.n_elems;
        std::memcpy(F.attrs, attrs, n_attrs * sizeof(uint32_t));
        F.acc = acc;
        const uint64_t blocks = std::min<uint64_t>((tb.n_elems + 255) / 256, (uint64_t)ctx->sm_count * 8);
        k_fetch_sum<<<dim3((unsigned)blocks, 1 + n_attrs), 256, 0, s>>>(F);
        ctx->launches++;
    }
    FinishParams Fn{};
    std::memcpy(Fn.rk_prf, ctx->rk_prf, sizeof Fn.rk_prf);
    Fn.te4 = ctx->d_te4;
    Fn.acc = acc;
    Fn.out = out;
    std::memcpy(Fn.attrs, attrs, n_attrs * sizeof(uint32_t));
    Fn.n_attrs = n_attrs;
    Fn.step = kFetchStep + group;
    Fn.table = table_id;
    Fn.query = query_id;
    k_fetch_finish<<<1, 96, 0, s>>>(Fn);
    ctx->launches++;
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch launch");
    ce = cudaFreeAsync(acc, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch scratch release");
    return OBLIVGM_OK;
}
