// aes_layouts.cu -- the fixed-key PRG H_K(s) = AES-128_K(s) xor s (the PRG of the DPF / DCF
// constructions cited in Sec. V-C, lambda = 128 as Sec. VII-A fixes it) in the two AES
// layouts a GPU can use, as a measured primitive and as the autotuner's AES-layout choice:
//
//  * T-table: the layout the walks use.  Four 1 KiB tables, bank-replicated in shared memory,
//    one block per thread; a round is 16 lookups (LDS) plus the XORs and byte selects.
//  * bitsliced: 32 blocks per thread, bit i of byte b of block e in bit e of word 8 b + i
//    (128 words in registers).  SubBytes is a gate circuit on the eight bit planes of each
//    byte (tower-field inverse, generated and checked exhaustively by gen_aes_bitsliced.py),
//    ShiftRows a renaming, MixColumns and AddRoundKey XORs; no tables, no loads.
//
// Both compute H_K(B_c) for counter blocks B_c = u64 c || 8 zero bytes, so the two layouts
// can be checked against each other and against a CPU AES.  An output is either every
// block (4 words) or, for timing, one parity word per 32 blocks: bit e of word g is the XOR
// of the 128 bits of H_K(B_{32 g + e}).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "aes_bitsliced_sbox.cuh"
#include "device_fss.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

// round keys of the four fixed PRG keys as bit-plane masks: kRkMask[key][round][8 b + i] is
// all ones when bit i of byte b of the round key is set
__constant__ uint32_t kRkMask[4][11][128];

struct PrgParams {
    const uint32_t* te0;
    uint32_t rk[44];          // T-table layout: round-key words of the chosen key
    uint32_t key;             // 0..3 (K_L, K_R, K_vL, K_vR)
    uint64_t first;           // first counter (a multiple of 32)
    uint64_t n_groups;        // blocks / 32
    uint32_t* out;            // full: [blocks][4]; parity: [n_groups]
    uint32_t parity;          // 1: one parity word per 32 blocks
};

// ---------------------------------------------------------------- T-table layout

__global__ void __launch_bounds__(768, 1) k_prg_ttable(const __grid_constant__ PrgParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint64_t n_blocks = P.n_groups * 32;
    // each warp takes 32 consecutive blocks (one parity word), lane e block 32 g + e
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_blocks;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = P.first + i;
        const uint32_t in[4] = {(uint32_t)c, (uint32_t)(c >> 32), 0u, 0u};
        uint32_t o[4];
        aes_one(T, P.rk, in, o);
#pragma unroll
        for (int w = 0; w < 4; w++) o[w] ^= in[w];
        if (P.parity) {
            const uint32_t bit = __popc(o[0] ^ o[1] ^ o[2] ^ o[3]) & 1u;
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
            if ((threadIdx.x & 31u) == 0) P.out[i / 32] = word;
        } else {
            reinterpret_cast<uint4*>(P.out)[i] = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

// ---------------------------------------------------------------- bitsliced layout

__device__ __forceinline__ void bs_xtime(const uint32_t u[8], uint32_t v[8]) {
    // multiply by x modulo x^8 + x^4 + x^3 + x + 1 (0x1b): shift up, fold bit 7 into bits 0, 1, 3, 4
    v[0] = u[7];
    v[1] = u[0] ^ u[7];
    v[2] = u[1];
    v[3] = u[2] ^ u[7];
    v[4] = u[3] ^ u[7];
    v[5] = u[4];
    v[6] = u[5];
    v[7] = u[6];
}

// SubBytes then ShiftRows (state byte b = r + 4 c takes the byte at r + 4 ((c + r) % 4)),
// then MixColumns when MIX, into n; AddRoundKey is the caller's.
template <bool MIX>
__device__ __forceinline__ void bs_round_body(uint32_t s[128], uint32_t n[128]) {
#pragma unroll
    for (int b = 0; b < 16; b++)
        bs_sbox(s[8 * b + 0], s[8 * b + 1], s[8 * b + 2], s[8 * b + 3], s[8 * b + 4], s[8 * b + 5], s[8 * b + 6],
                s[8 * b + 7]);
    if constexpr (!MIX) {
#pragma unroll
        for (int b = 0; b < 16; b++) {
            const int r = b % 4, c = b / 4, src = r + 4 * ((c + r) % 4);
#pragma unroll
            for (int i = 0; i < 8; i++) n[8 * b + i] = s[8 * src + i];
        }
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            // the column after ShiftRows: a_r = byte r + 4 ((c + r) % 4)
            const uint32_t* a[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = s + 8 * (r + 4 * ((c + r) % 4));
            uint32_t t[8];
#pragma unroll
            for (int i = 0; i < 8; i++) t[i] = a[0][i] ^ a[1][i] ^ a[2][i] ^ a[3][i];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                // out_r = a_r + t + 2 (a_r + a_{r+1})
                uint32_t u[8], v[8];
#pragma unroll
                for (int i = 0; i < 8; i++) u[i] = a[r][i] ^ a[(r + 1) % 4][i];
                bs_xtime(u, v);
#pragma unroll
                for (int i = 0; i < 8; i++) n[8 * (r + 4 * c) + i] = a[r][i] ^ t[i] ^ v[i];
            }
        }
    }
}

// 32 x 32 bit transpose in place: bit e of word j <-> bit j of word e
__device__ __forceinline__ void transpose32(uint32_t m[32]) {
    uint32_t mask = 0x0000FFFFu;
#pragma unroll
    for (int j = 16; j != 0; j >>= 1, mask ^= mask << j) {
#pragma unroll
        for (int k = 0; k < 32; k = ((k | j) + 1) & ~j) {
            const uint32_t t = ((m[k] >> j) ^ m[k | j]) & mask;
            m[k] ^= t << j;
            m[k | j] ^= t;
        }
    }
}

__global__ void __launch_bounds__(256) k_prg_bitsliced(const __grid_constant__ PrgParams P) {
    const uint32_t(*rk)[128] = kRkMask[P.key];
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P.n_groups;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c0 = P.first + 32 * g;   // a multiple of 32: bits 0..4 of the counter are e
        // bit planes of the 32 counter blocks: plane k (k < 64) is bit k of c0 + e over e
        uint32_t in[128], s[128];
#pragma unroll
        for (int k = 0; k < 128; k++) {
            uint32_t v;
            if (k == 0) v = 0xAAAAAAAAu;
            else if (k == 1) v = 0xCCCCCCCCu;
            else if (k == 2) v = 0xF0F0F0F0u;
            else if (k == 3) v = 0xFF00FF00u;
            else if (k == 4) v = 0xFFFF0000u;
            else if (k < 64) v = 0u - (uint32_t)((c0 >> k) & 1u);
            else v = 0u;
            in[k] = v;
            s[k] = v ^ rk[0][k];
        }
#pragma unroll 1
        for (int r = 1; r < 10; r++) {
            uint32_t n[128];
            bs_round_body<true>(s, n);
#pragma unroll
            for (int k = 0; k < 128; k++) s[k] = n[k] ^ rk[r][k];
        }
        {
            uint32_t n[128];
            bs_round_body<false>(s, n);
#pragma unroll
            for (int k = 0; k < 128; k++) s[k] = n[k] ^ rk[10][k] ^ in[k];   // MMO: xor the input
        }
        if (P.parity) {
            uint32_t par = 0;
#pragma unroll
            for (int k = 0; k < 128; k++) par ^= s[k];
            P.out[g] = par;
        } else {
            // block word w holds bytes 4 w .. 4 w + 3: planes 32 w .. 32 w + 31
#pragma unroll
            for (int w = 0; w < 4; w++) {
                uint32_t m[32];
#pragma unroll
                for (int j = 0; j < 32; j++) m[j] = s[32 * w + j];
                transpose32(m);
#pragma unroll
                for (int e = 0; e < 32; e++) P.out[(32 * g + e) * 4 + w] = m[e];
            }
        }
    }
}

}  // namespace

oblivgm_status set_prg_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_prg_ttable, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
    if (e != cudaSuccess) return cuda_fail(e, "PRG kernel attributes");
    // the fixed keys' round keys as bit-plane masks (once per process and device)
    static uint32_t masks[4][11][128];
    for (int j = 0; j < 4; j++) {
        const RoundKeys& K = fixed_key(j);
        for (int r = 0; r < 11; r++)
            for (int b = 0; b < 16; b++)
                for (int i = 0; i < 8; i++)
                    masks[j][r][8 * b + i] = 0u - ((K.w[4 * r + b / 4] >> (8 * (b % 4) + i)) & 1u);
    }
    e = cudaMemcpyToSymbol(kRkMask, masks, sizeof masks);
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, "PRG round-key masks");
}

oblivgm_status prg_launch(oblivgm_ctx* ctx, uint32_t layout, uint32_t key, uint64_t first, uint64_t n_blocks,
                          uint32_t flags, uint32_t* out, cudaStream_t s) {
    PrgParams P{};
    P.te0 = ctx->d_te0;
    std::memcpy(P.rk, fixed_key((int)key).w, sizeof P.rk);
    P.key = key;
    P.first = first;
    P.n_groups = n_blocks / 32;
    P.out = out;
    P.parity = (flags & OBLIVGM_PRG_PARITY) ? 1u : 0u;
    if (P.n_groups == 0) return OBLIVGM_OK;
    if (layout == OBLIVGM_AES_TTABLE) {
        const uint64_t want = (n_blocks + 767) / 768;
        k_prg_ttable<<<(unsigned)std::min<uint64_t>(want, (uint64_t)ctx->sm_count), 768, kTableBytes, s>>>(P);
    } else {
        const uint64_t want = (P.n_groups + 255) / 256;
        // registers hold 256 threads of this kernel per SM: one wave of CTAs per SM
        k_prg_bitsliced<<<(unsigned)std::min<uint64_t>(want, (uint64_t)ctx->sm_count), 256, 0, s>>>(P);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "PRG launch");
    ctx->launches++;
    return OBLIVGM_OK;
}

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_prg_batch(oblivgm_ctx* ctx, uint32_t layout, uint32_t key, uint64_t first,
                                            uint64_t n_blocks, uint32_t flags, uint32_t* out, uint64_t n_out,
                                            void* stream) {
    const NvtxRange nvtx_range("oblivgm_prg_batch");
    if (!ctx || (!out && n_blocks)) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (layout != OBLIVGM_AES_TTABLE && layout != OBLIVGM_AES_BITSLICED) return fail(OBLIVGM_EINVAL, "unknown AES layout");
    if (key > 3) return fail(OBLIVGM_EINVAL, "key must be 0..3 (K_L, K_R, K_vL, K_vR)");
    if (flags & ~OBLIVGM_PRG_PARITY) return fail(OBLIVGM_EINVAL, "unknown flags");
    if (first % 32 || n_blocks % 32) return fail(OBLIVGM_EINVAL, "first and n_blocks must be multiples of 32");
    const uint64_t need = (flags & OBLIVGM_PRG_PARITY) ? n_blocks / 32 : 4 * n_blocks;
    if (n_out < need) return fail(OBLIVGM_ERANGE, "output buffer too small");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return prg_launch(ctx, layout, key, first, n_blocks, flags, out, static_cast<cudaStream_t>(stream));
}

extern "C" oblivgm_status oblivgm_autotune_aes_layout(oblivgm_ctx* ctx, uint32_t* layout, double* ttable_blocks_per_s,
                                                      double* bitsliced_blocks_per_s) {
    const NvtxRange nvtx_range("oblivgm_autotune_aes_layout");
    if (!ctx) return fail(OBLIVGM_EINVAL, "NULL context");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    // 2^26 blocks of K_L per timing, parity outputs (8 MB): the AES work dominates
    const uint64_t n = 1ull << 26;
    uint32_t* out = nullptr;
    e = cudaMalloc(&out, n / 32 * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "layout tuning buffer");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double rate[2] = {0, 0};
    oblivgm_status st = OBLIVGM_OK;
    for (uint32_t lay = 0; lay < 2 && st == OBLIVGM_OK; lay++) {
        float best = 1e30f;
        for (int rep = 0; rep < 4 && st == OBLIVGM_OK; rep++) {   // the first run is a warm-up
            cudaEventRecord(a, 0);
            st = prg_launch(ctx, lay, 0, 0, n, OBLIVGM_PRG_PARITY, out, 0);
            cudaEventRecord(b, 0);
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) best = std::min(best, ms);
        }
        rate[lay] = (double)n / (best / 1e3);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (st != OBLIVGM_OK) return st;
    ctx->aes_layout = rate[1] > rate[0] ? OBLIVGM_AES_BITSLICED : OBLIVGM_AES_TTABLE;
    ctx->aes_layout_rate[0] = rate[0];
    ctx->aes_layout_rate[1] = rate[1];
    if (layout) *layout = ctx->aes_layout;
    if (ttable_blocks_per_s) *ttable_blocks_per_s = rate[0];
    if (bitsliced_blocks_per_s) *bitsliced_blocks_per_s = rate[1];
    return OBLIVGM_OK;
}
