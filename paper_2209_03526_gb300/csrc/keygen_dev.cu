// keygen_dev.cu -- batched FSS key generation on the GPU (client side of Sec. V-C):
// many DPF or DCF key pairs at once, for per-element keys.  Pair i is generated from
// root seeds s0 = AES_seed(2i), s1 = AES_seed(2i + 1) (counter blocks: u64 index || 0),
// with the same Gen as the host (BGI16 DPF / Boyle et al. DCF, H_K(s) = AES_K(s) xor s
// under the fixed keys, control bit = bit 0 of byte 0, Convert = bytes 4..7), and written
// in the key wire format: key 0 of pair i at byte 2 i L, key 1 at (2 i + 1) L.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "device_fss.cuh"
#include "gen_device.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

#ifndef OGM_KEYGEN_THREADS
#define OGM_KEYGEN_THREADS 768
#endif
constexpr int kKeygenThreads = OGM_KEYGEN_THREADS;   // one CTA per SM (the tables take 128 KiB)
// tables, then a staging area of 32 records of 6 words per warp for the stores
constexpr int kKeygenSmem = kTableBytes + (kKeygenThreads / 32) * 32 * 6 * 4;

struct KeygenParams {
    AesParams aes;
    GenRightKeys right;
    uint32_t rk_seed[44];          // round keys of the client's seed (root-seed stream)
    const uint32_t* te0;
    const uint32_t* alpha;         // per pair (device)
    const uint32_t* beta;          // per pair (device)
    uint8_t* out;                  // 2 * n_pairs keys of key_len bytes
    uint64_t n_pairs;
    uint32_t n, kind, key_len;
};

__device__ __forceinline__ void st32(uint8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

// Level records of the wire format, written by the whole warp.  A warp's 32 consecutive
// pairs own 64 consecutive keys; each level's record (the same for both keys of a pair)
// goes through shared memory, and the warp then stores the 64 records with lanes on
// consecutive words of a record, so a store instruction covers a few whole records
// instead of 32 scattered words.
template <bool DCF>
struct WarpWireSink {
    static constexpr uint32_t kWords = DCF ? 6 : 5;        // words per level record
    uint8_t* base;         // first key of the warp's 64
    uint32_t* stage;       // kWords words per lane
    uint32_t L, lane, n, n_keys;   // key length, lane, levels, keys of the warp that exist
    __device__ __forceinline__ void level(int lv, const uint32_t scw[4], uint32_t tl, uint32_t tr, uint32_t vcw) {
        uint32_t* my = stage + lane * kWords;
        my[0] = scw[0]; my[1] = scw[1]; my[2] = scw[2]; my[3] = scw[3];
        my[4] = tl | (tr << 8);
        if (DCF) my[5] = vcw;
        __syncwarp();
        const uint32_t off = 24u + (uint32_t)lv * kWords * 4;
#pragma unroll
        for (uint32_t j = 0; j < 2 * kWords; j++) {         // 64 records x kWords words
            const uint32_t w = 32 * j + lane, r = w / kWords, word = w - r * kWords;
            if (r < n_keys) st32(base + (uint64_t)r * L + off + 4 * word, stage[(r >> 1) * kWords + word]);
        }
        __syncwarp();
    }
    __device__ __forceinline__ void final(uint32_t cw) {
        const uint32_t off = 24u + n * kWords * 4;
        if (2 * lane < n_keys) {
            st32(base + (uint64_t)(2 * lane) * L + off, cw);
            st32(base + (uint64_t)(2 * lane + 1) * L + off, cw);
        }
    }
};

// The loop runs over warp-sized chunks of pairs so that the whole warp stays together
// for the cooperative stores; lanes past the last pair repeat the last pair's work and
// store nothing.
template <int kThreads, bool DCF>
__global__ void __launch_bounds__(kThreads) k_keygen(const __grid_constant__ KeygenParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t L = P.key_len;
    const int n = (int)P.n;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + kTableBytes) + warp * 32 * WarpWireSink<DCF>::kWords;
    const uint64_t warps_total = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t chunk = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; chunk * 32 < P.n_pairs;
         chunk += warps_total) {
        const uint64_t first = chunk * 32;
        const uint64_t i = first + lane < P.n_pairs ? first + lane : P.n_pairs - 1;
        const bool real = first + lane < P.n_pairs;
        uint32_t s0[4], s1[4];
        {
            const uint32_t c0[4] = {(uint32_t)(2 * i), (uint32_t)((2 * i) >> 32), 0u, 0u};
            const uint32_t c1[4] = {(uint32_t)(2 * i + 1), (uint32_t)((2 * i + 1) >> 32), 0u, 0u};
            aes_one(T, P.rk_seed, c0, s0);
            aes_one(T, P.rk_seed, c1, s1);
        }
        if (real) {
            uint8_t* const k0 = P.out + (2 * i) * L;
            uint8_t* const k1 = k0 + L;
            st32(k0, (uint32_t)P.kind | ((uint32_t)n << 8));
            st32(k1, (uint32_t)P.kind | ((uint32_t)n << 8) | (1u << 16));
            st32(k0 + 4, 0u);
            st32(k1 + 4, 0u);
#pragma unroll
            for (int w = 0; w < 4; w++) {
                st32(k0 + 8 + 4 * w, s0[w]);
                st32(k1 + 8 + 4 * w, s1[w]);
            }
        }
        WarpWireSink<DCF> sink;
        sink.base = P.out + 2 * first * L;
        sink.stage = stage;
        sink.L = L;
        sink.lane = lane;
        sink.n = (uint32_t)n;
        sink.n_keys = (uint32_t)(P.n_pairs - first < 32 ? 2 * (P.n_pairs - first) : 64);
        gen_pair<DCF>(T, P.aes, P.right, n, P.alpha[i], P.beta[i], s0, s1, sink);
    }
}

}  // namespace

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_keygen_device(oblivgm_ctx* ctx, uint32_t kind, uint32_t n_bits, uint64_t n_pairs,
                                                const uint32_t* alpha, const uint32_t* beta, const uint8_t seed[16],
                                                uint8_t* keys_out, uint64_t out_bytes, void* stream) {
    const NvtxRange nvtx_range("oblivgm_keygen_device");
    if (!ctx || !seed || (n_pairs && (!alpha || !beta || !keys_out))) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (kind != OBLIVGM_KEY_DPF && kind != OBLIVGM_KEY_DCF) return fail(OBLIVGM_EINVAL, "unknown key kind");
    if (n_bits < 1 || n_bits > (uint32_t)kMaxBits) return fail(OBLIVGM_EINVAL, "n must be 1..32");
    const uint32_t L = (uint32_t)key_bytes(kind, (int)n_bits);
    if (out_bytes < 2ull * L * n_pairs) return fail(OBLIVGM_ERANGE, "key buffer too small");
    if (reinterpret_cast<uintptr_t>(keys_out) % 4) return fail(OBLIVGM_EINVAL, "key buffer must be 4-byte aligned");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    if (n_pairs == 0) return OBLIVGM_OK;
    KeygenParams P{};
    P.aes = ctx->aes;
    for (int w = 0; w < 44; w++) {
        P.right.st[w] = ctx->aes.rk_st[w] ^ ctx->aes.d_st[w];
        P.right.v[w] = ctx->aes.rk_v[w] ^ ctx->aes.d_v[w];
    }
    const RoundKeys rk = expand_key(seed);
    std::memcpy(P.rk_seed, rk.w, sizeof P.rk_seed);
    P.te0 = ctx->d_te0;
    P.alpha = alpha;
    P.beta = beta;
    P.out = keys_out;
    P.n_pairs = n_pairs;
    P.n = n_bits;
    P.kind = kind;
    P.key_len = L;
    const unsigned grid =
        (unsigned)std::min<uint64_t>((n_pairs + kKeygenThreads - 1) / kKeygenThreads, (uint64_t)ctx->sm_count);
    if (kind == OBLIVGM_KEY_DCF)
        k_keygen<kKeygenThreads, true><<<grid, kKeygenThreads, kKeygenSmem, static_cast<cudaStream_t>(stream)>>>(P);
    else
        k_keygen<kKeygenThreads, false><<<grid, kKeygenThreads, kKeygenSmem, static_cast<cudaStream_t>(stream)>>>(P);
    ctx->launches++;
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "k_keygen launch");
    return OBLIVGM_OK;
}

namespace ogm {
oblivgm_status set_keygen_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_keygen<kKeygenThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kKeygenSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_keygen<kKeygenThreads, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kKeygenSmem);
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, "keygen kernel attributes");
}
}  // namespace ogm

// Wire-format keys already on the device -> DevKey, one thread per key.  A key whose
// header disagrees with (kind, n) or is malformed becomes a zero key of the expected
// shape and raises the context's fault flag (bit 2): the walks never see an n above 32.
namespace ogm {
namespace {
__global__ void k_repack(const uint8_t* __restrict__ wire, uint32_t kind, uint32_t n, uint32_t n_keys,
                         DevKey* __restrict__ out, uint32_t* error) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_keys) return;
    const uint32_t L = 28u + n * (kind == OBLIVGM_KEY_DPF ? 20u : 24u), lb = kind == OBLIVGM_KEY_DPF ? 20u : 24u;
    const uint8_t* k = wire + (uint64_t)i * L;
    DevKey d;
    memset(&d, 0, sizeof d);
    const bool ok = k[0] == kind && k[1] == n && k[2] <= 1 && k[3] == 0;
    d.n = n;
    d.kind = kind;
    if (ok) {
        for (int w = 0; w < 4; w++) d.seed[w] = *reinterpret_cast<const uint32_t*>(k + 8 + 4 * w);
        for (uint32_t lv = 0; lv < n; lv++) {
            const uint8_t* p = k + 24 + lv * lb;
            for (int w = 0; w < 4; w++) d.scw[lv][w] = *reinterpret_cast<const uint32_t*>(p + 4 * w);
            d.tl |= (uint32_t)(p[16] & 1u) << lv;
            d.tr |= (uint32_t)(p[17] & 1u) << lv;
            if (kind == OBLIVGM_KEY_DCF) d.vcw[lv] = *reinterpret_cast<const uint32_t*>(p + 20);
        }
        d.cw_final = *reinterpret_cast<const uint32_t*>(k + 24 + n * lb);
        d.party = k[2];
    } else {
        atomicOr(error, 4u);
    }
    out[i] = d;
}
}  // namespace

oblivgm_status repack_keys_device(oblivgm_ctx* ctx, const uint8_t* wire, uint32_t kind, uint32_t n, uint32_t n_keys,
                                  DevKey* out, cudaStream_t s) {
    if (reinterpret_cast<uintptr_t>(wire) % 4) return fail(OBLIVGM_EINVAL, "device keys must be 4-byte aligned");
    k_repack<<<(n_keys + 127) / 128, 128, 0, s>>>(wire, kind, n, n_keys, out, ctx->d_error);
    ctx->launches++;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, "k_repack launch");
}
}  // namespace ogm
