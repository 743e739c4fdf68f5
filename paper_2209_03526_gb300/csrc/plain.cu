// plain.cu -- the plain per-query GPU path, kept as the comparison point for the
// fused kernel: one launch per (predicate, key half) with the AES T-tables read
// from global memory, then separate launches for the mask-open, the per-server
// sums with the re-share, and each AND.  It computes exactly what
// oblivgm_filter_and_combine computes (same readings, same PRF counters).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "device_fss.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

struct PrfKeys { uint32_t rk[3][44]; };

__global__ void k_plain_open(const uint32_t* __restrict__ s0, const uint32_t* __restrict__ s1,
                             const uint32_t* __restrict__ s2, uint32_t rsum, uint32_t mask, uint64_t n,
                             uint32_t* __restrict__ xhat) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xhat[i] = (s0[i] + s1[i] + s2[i] + rsum) & mask;
}

template <uint32_t KIND>
__global__ void k_plain_walk(const __grid_constant__ AesParams A, const uint32_t* __restrict__ te,
                             const DevKey* __restrict__ key, const uint32_t* __restrict__ xhat, uint64_t n,
                             uint32_t add, uint32_t* __restrict__ y) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GlobalTab T{te};
    uint32_t x[1] = {xhat[i]}, v[1];
    if (KIND == OBLIVGM_KEY_DPF) dpf_walk<1>(T, A, *key, x, v);
    else dcf_walk<1>(T, A, *key, x, v);
    y[i] = v[0] + add;
}

__device__ __forceinline__ uint32_t prf(const GlobalTab& T, const uint32_t* rk, uint64_t el, uint32_t step,
                                        uint32_t table, uint32_t query) {
    const uint32_t ctr[4] = {(uint32_t)el, (uint32_t)(el >> 32), step | (table << 16), query};
    return aes_one_w0(T, rk, ctr);
}

// z_i = sum of server i's key-half outputs, then r_i = z_i + F(k_i) - F(k_{i-1})
__global__ void k_plain_sum_reshare(const __grid_constant__ PrfKeys K, const uint32_t* __restrict__ te,
                                    const uint32_t* __restrict__ y, int nsub, uint64_t n, uint32_t step,
                                    uint32_t table, uint32_t query, uint32_t* __restrict__ b) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GlobalTab T{te};
    uint32_t z[3];
    for (int s = 0; s < 3; s++) {
        z[s] = 0;
        for (int k = 0; k < 2 * nsub; k++) z[s] += y[(uint64_t)(s * 2 * nsub + k) * n + i];
    }
    uint32_t f[3];
    for (int s = 0; s < 3; s++) f[s] = prf(T, K.rk[s], i, step, table, query);
    for (int s = 0; s < 3; s++) b[(uint64_t)s * n + i] = z[s] + f[s] - f[(s + 2) % 3];
}

// acc <- reshare(acc OP b): w_i = lin (a_i + b_i) + prod (a_i b_i + a_i b_{i+1} + a_{i+1} b_i)
__global__ void k_plain_and(const __grid_constant__ PrfKeys K, const uint32_t* __restrict__ te,
                            const uint32_t* __restrict__ b, uint64_t n, uint32_t step, uint32_t table,
                            uint32_t query, uint32_t lin, uint32_t prod, uint32_t* __restrict__ acc) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GlobalTab T{te};
    uint32_t a[3], bb[3], w[3], f[3];
    for (int s = 0; s < 3; s++) { a[s] = acc[(uint64_t)s * n + i]; bb[s] = b[(uint64_t)s * n + i]; }
    for (int s = 0; s < 3; s++) {
        const int s1 = (s + 1) % 3;
        w[s] = lin * (a[s] + bb[s]) + prod * (a[s] * bb[s] + a[s] * bb[s1] + a[s1] * bb[s]);
    }
    for (int s = 0; s < 3; s++) f[s] = prf(T, K.rk[s], i, step, table, query);
    for (int s = 0; s < 3; s++) acc[(uint64_t)s * n + i] = w[s] + f[s] - f[(s + 2) % 3];
}

}  // namespace

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_filter_plain(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                               const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out,
                                               void* stream) {
    const NvtxRange nvtx_range("oblivgm_filter_plain");
    if (!ctx || !tok || !tok_len || !out) return fail(OBLIVGM_EINVAL, "NULL argument");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    ParsedQuery q;
    std::string err;
    oblivgm_status st = parse_tokens(tok, tok_len, &q, &err);
    if (st != OBLIVGM_OK) return fail(st, err);
    if (q.out_group != 0) return fail(OBLIVGM_EINVAL, "a one-hot token was given to the masked-mode evaluation");
    if (n_groups == 0 || n_groups > OBLIVGM_MAX_GROUPS) return fail(OBLIVGM_EINVAL, "n_groups must be 1..64");
    std::vector<std::vector<const ParsedPred*>> members(n_groups);
    for (const ParsedPred& p : q.preds) {
        if (p.group >= n_groups) return fail(OBLIVGM_EINVAL, "predicate group outside 0..n_groups-1");
        members[p.group].push_back(&p);
    }
    for (uint32_t g = 0; g < n_groups; g++) {
        if (members[g].empty()) return fail(OBLIVGM_EINVAL, "an AND-group has no predicate");
        auto it = ctx->tables.find(members[g][0]->table);
        if (it == ctx->tables.end()) return fail(OBLIVGM_ENOENT, "predicate on a table that is not loaded");
        for (const ParsedPred* p : members[g]) {
            if (p->table != members[g][0]->table) return fail(OBLIVGM_EINVAL, "an AND-group spans two tables");
            if (p->attr >= it->second.n_attrs) return fail(OBLIVGM_EINVAL, "predicate attribute outside its table");
            if (p->n != it->second.n_bits) return fail(OBLIVGM_EINVAL, "predicate bit length differs from its table's");
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PrfKeys K;
    std::memcpy(K.rk, ctx->rk_prf, sizeof K.rk);
    for (uint32_t g = 0; g < n_groups; g++) {
        const Table& tb = ctx->tables.at(members[g][0]->table);
        const uint64_t n = tb.n_elems;
        if (n == 0) continue;
        const uint32_t tid = members[g][0]->table;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        // scratch: xhat | y (12 n) | b (3 n) | 12 device keys
        const size_t words = n + 12 * n + 3 * n;
        unsigned char* ws = nullptr;
        {
            const oblivgm_status as =
                ws_alloc(ctx, reinterpret_cast<void**>(&ws), words * 4 + 12 * sizeof(DevKey) + 256, s, "plain-path scratch");
            if (as != OBLIVGM_OK) return as;
        }
        ScratchGuard guard(ws, s);
        uint32_t* xhat = reinterpret_cast<uint32_t*>(ws);
        uint32_t* y = xhat + n;
        uint32_t* b = y + 12 * n;
        DevKey* dkeys = reinterpret_cast<DevKey*>(ws + (words * 4 + 255) / 256 * 256);
        uint32_t* acc[3] = {out[3 * g], out[3 * g + 1], out[3 * g + 2]};
        bool first = true;
        for (const ParsedPred* p : members[g]) {
            const uint32_t mask = p->n >= 32 ? 0xFFFFFFFFu : ((1u << p->n) - 1u);
            const uint32_t* row[3];
            for (int j = 0; j < 3; j++) row[j] = tb.dev + ((uint64_t)j * tb.n_attrs + p->attr) * tb.stride;
            k_plain_open<<<blocks, 256, 0, s>>>(row[0], row[1], row[2], p->r[0] + p->r[1] + p->r[2], mask, n, xhat);
            ctx->launches++;
            ce = cudaMemcpyAsync(dkeys, p->keys.data(), p->keys.size() * sizeof(DevKey), cudaMemcpyHostToDevice, s);
            if (ce != cudaSuccess) return cuda_fail(ce, "plain-path key upload");
            const int nsub = p->kind == OBLIVGM_PRED_EQ ? 1 : 2;
            for (int k = 0; k < 6 * nsub; k++) {
                const uint32_t add = (nsub == 2 && k % 2 == 0 && p->keys[k].party == 0) ? p->cbeta : 0u;
                if (nsub == 1)
                    k_plain_walk<OBLIVGM_KEY_DPF><<<blocks, 256, 0, s>>>(ctx->aes, ctx->d_te4, dkeys + k, xhat, n, add, y + (uint64_t)k * n);
                else
                    k_plain_walk<OBLIVGM_KEY_DCF><<<blocks, 256, 0, s>>>(ctx->aes, ctx->d_te4, dkeys + k, xhat, n, add, y + (uint64_t)k * n);
                ctx->launches++;
            }
            // the predicate's RSS bit into b; the group's first predicate becomes the accumulator,
            // later ones are folded into it (the accumulator is staged through y's space)
            k_plain_sum_reshare<<<blocks, 256, 0, s>>>(K, ctx->d_te4, y, nsub, n, p->step, tid, query_id, b);
            ctx->launches++;
            if (first) {
                for (int j = 0; j < 3; j++) {
                    ce = cudaMemcpyAsync(acc[j], b + (uint64_t)j * n, n * 4, cudaMemcpyDeviceToDevice, s);
                    if (ce != cudaSuccess) return cuda_fail(ce, "plain-path copy");
                }
            } else {
                for (int j = 0; j < 3; j++) {
                    ce = cudaMemcpyAsync(y + (uint64_t)j * n, acc[j], n * 4, cudaMemcpyDeviceToDevice, s);
                    if (ce != cudaSuccess) return cuda_fail(ce, "plain-path copy");
                }
                uint32_t lin, prod;
                combine_coeffs(p->combine, &lin, &prod);
                k_plain_and<<<blocks, 256, 0, s>>>(K, ctx->d_te4, b, n, 64u + p->step, tid, query_id, lin, prod, y);
                ctx->launches++;
                for (int j = 0; j < 3; j++) {
                    ce = cudaMemcpyAsync(acc[j], y + (uint64_t)j * n, n * 4, cudaMemcpyDeviceToDevice, s);
                    if (ce != cudaSuccess) return cuda_fail(ce, "plain-path copy");
                }
            }
            first = false;
        }
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "plain-path launch");
        guard.done();
        ce = cudaFreeAsync(ws, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "plain-path scratch release");
    }
    return OBLIVGM_OK;
}
