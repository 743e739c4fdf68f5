// shuffle.cu -- secShuffle (Alg. 5) with the three servers simulated on one GPU, and
// secFetch case II (Alg. 4) on top of it.
//
//   k_feistel_tab the round function of each pair's Feistel PRP at all 2^h half-words
//   k_perms       the permutations (pi12, pi31 forward; all three inverse, the network run
//                 backwards) as index arrays: 4 table lookups per pass, cycle walking
//   k_compose     pi31 o pi12 (CS1's map) and pi31^-1 o pi23^-1 (CS3's map)
//   k_shuf_cs1    CS1: X1 = pi31(pi12(D1 + D2 + T12) + T31)
//   k_shuf_cs2    CS2: Y1 = pi12(D3 - T12); C1 = pi23(X1 + T23) - R2; its output share R2
//   k_shuf_cs3    CS3: C2 = pi23(pi31(Y1 - T31) - T23) - R1; R3 = C1 + C2; output shares R1, R3
//
// Each server kernel reads only what that server holds or receives.  Rows are row-major
// (width words), so a row read or written out of order is one contiguous run.  The masks T and R are AES
// blocks of the pair's seed, four words per block, made where used.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "device_fss.cuh"
#include "host_crypto.h"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

namespace {

#ifndef OGM_SHUF_THREADS
#define OGM_SHUF_THREADS 768
#endif
constexpr int kShufThreads = OGM_SHUF_THREADS;
constexpr uint32_t kShufMaxWidth = 64;

struct ShufParams {
    uint32_t rk[3][44];         // round keys of s12, s23, s31
    const uint32_t* te0;
    const uint32_t* d[3];       // input shares (rows of width words)
    uint32_t* s[3];             // output shares R1, R2, R3
    uint32_t* inv[3];           // pi12^-1, pi23^-1, pi31^-1
    uint32_t* fwd[2];           // pi12, pi31
    uint32_t* ftab;             // [which][round][2^h] Feistel round values
    uint32_t* comp1;            // pi31(pi12(i)): CS1 knows both permutations
    uint32_t* comp3;            // pi31^-1(pi23^-1(l)): CS3 knows both permutations
    uint32_t* x1;
    uint32_t* y1;
    uint32_t* c1;
    uint64_t n;
    uint32_t width, group;      // group: OBLIVGM_SHUFFLE_ADD or _XOR
    uint32_t half_bits;         // h of the Feistel network
};

constexpr int S12 = 0, S23 = 1, S31 = 2;

__device__ __forceinline__ uint32_t op_add(uint32_t g, uint32_t a, uint32_t b) { return g ? a ^ b : a + b; }
__device__ __forceinline__ uint32_t op_sub(uint32_t g, uint32_t a, uint32_t b) { return g ? a ^ b : a - b; }

// words 4 q .. 4 q + 3 of row i of table `tag` (1 = T, 2 = R) of a seed
__device__ __forceinline__ void mask_block(const SmemTab& T, const uint32_t* rk, uint32_t tag, uint64_t i, uint32_t q,
                                           uint32_t out[4]) {
    const uint32_t in[4] = {(uint32_t)i, (uint32_t)(i >> 32), tag | (q << 16), 0u};
    aes_one(T, rk, in, out);
}

// F_r(R) of the three permutations for every round r and every half-word R: the round
// function sees only h bits, so 4 * 2^h AES calls per permutation cover all inputs
__global__ void __launch_bounds__(kShufThreads, 1) k_feistel_tab(const __grid_constant__ ShufParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t h = P.half_bits, side = 1u << h, mask = side - 1u;
    const uint64_t total = 12ull * side;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t which = (uint32_t)(t / (4ull * side)), rem = (uint32_t)(t % (4ull * side));
        const uint32_t r = rem / side, R = rem % side;
        const uint32_t in[4] = {R, 0u, 3u | (r << 16), (uint32_t)P.n};
        P.ftab[t] = aes_one_w0(T, P.rk[which], in) & mask;
    }
}

__device__ __forceinline__ uint64_t feistel(const uint32_t* __restrict__ ft, uint64_t x, uint32_t h) {
    const uint32_t side = 1u << h, mask = side - 1u;
    uint32_t L = (uint32_t)(x >> h) & mask, R = (uint32_t)x & mask;
#pragma unroll
    for (uint32_t r = 0; r < 4; r++) {
        const uint32_t t = L ^ __ldg(ft + r * side + R);
        L = R;
        R = t;
    }
    return ((uint64_t)L << h) | R;
}

// the inverse of the Feistel network: rounds 3..0, each (L', R') -> (R' xor F_r(L'), L')
__device__ __forceinline__ uint64_t feistel_inv(const uint32_t* __restrict__ ft, uint64_t y, uint32_t h) {
    const uint32_t side = 1u << h, mask = side - 1u;
    uint32_t L = (uint32_t)(y >> h) & mask, R = (uint32_t)y & mask;
#pragma unroll
    for (int r = 3; r >= 0; r--) {
        const uint32_t prevL = R ^ __ldg(ft + (uint32_t)r * side + L);
        R = L;
        L = prevL;
    }
    return ((uint64_t)L << h) | R;
}

// pi^-1 of the three permutations, and pi12, pi31 forward, as index arrays.  The inverse
// of a cycle-walking permutation walks the inverse network until it re-enters [0, n).
// Items: 5 n, array a = item / n: 0..2 inverse of (12, 23, 31), 3 forward 12, 4 forward 31.
__global__ void __launch_bounds__(256) k_perms(const __grid_constant__ ShufParams P) {
    const uint32_t h = P.half_bits;
    const uint64_t dom = 1ull << (2 * h);
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 5 * P.n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / P.n);
        const int which = a < 3 ? a : (a == 3 ? S12 : S31);
        const bool fwd = a >= 3;
        const uint64_t y = t - (uint64_t)a * P.n;
        const uint32_t* ft = P.ftab + (uint64_t)which * 4 * (1ull << h);
        uint64_t x = 0;
        if (P.n > 1) {
            x = fwd ? feistel(ft, y, h) : feistel_inv(ft, y, h);
            // the cycle through y re-enters [0, n) within dom steps
            for (uint64_t guard = 0; x >= P.n && guard < dom; guard++)
                x = fwd ? feistel(ft, x, h) : feistel_inv(ft, x, h);
            if (x >= P.n) x = y;   // unreachable; keeps every later index inside the table
        }
        (fwd ? P.fwd[a - 3] : P.inv[which])[y] = (uint32_t)x;
    }
}

// CS1's map pi31(pi12(i)) and CS3's inverse map pi31^-1(pi23^-1(l)), so their row loops
// read indices in order
__global__ void __launch_bounds__(256) k_compose(const __grid_constant__ ShufParams P) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * P.n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        if (t < P.n) P.comp1[t] = P.fwd[1][P.fwd[0][t]];
        else P.comp3[t - P.n] = P.inv[S31][P.inv[S23][t - P.n]];
    }
}

// CS1 runs over its input rows (two rows of D read in order, one row of X1 written at
// pi31(pi12(i))); CS2 and CS3 run over their output rows and gather the input row the
// permutations bring there, so their index reads and row writes are in order.

// CS1: X1[k] = (D1 + D2 + T12)[i] + T31[j], j = pi12(i), k = pi31(j)
__global__ void __launch_bounds__(kShufThreads, 1) k_shuf_cs1(const __grid_constant__ ShufParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t W = P.width, g = P.group;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = P.fwd[0][i], k = P.comp1[i];
        for (uint32_t q = 0; q * 4 < W; q++) {
            uint32_t t12[4], t31[4];
            mask_block(T, P.rk[S12], 1u, i, q, t12);
            mask_block(T, P.rk[S31], 1u, j, q, t31);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t w = 4 * q + e;
                if (w < W) {
                    const uint64_t src = i * W + w;
                    const uint32_t a = op_add(g, op_add(g, __ldg(P.d[0] + src), __ldg(P.d[1] + src)), t12[e]);
                    P.x1[k * W + w] = op_add(g, a, t31[e]);
                }
            }
        }
    }
}

// CS2: items 0..n-1: Y1[j] = D3[i] - T12[i], i = pi12^-1(j);
//      items n..2n-1 (l = item - n): C1[l] = X1[k] + T23[k] - R2[l], k = pi23^-1(l); output R2[l]
__global__ void __launch_bounds__(kShufThreads, 1) k_shuf_cs2(const __grid_constant__ ShufParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t W = P.width, g = P.group;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * P.n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        if (t < P.n) {
            const uint64_t j = t, i = P.inv[S12][j];
            for (uint32_t q = 0; q * 4 < W; q++) {
                uint32_t t12[4];
                mask_block(T, P.rk[S12], 1u, i, q, t12);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t w = 4 * q + e;
                    if (w < W) P.y1[j * W + w] = op_sub(g, __ldg(P.d[2] + i * W + w), t12[e]);
                }
            }
        } else {
            const uint64_t l = t - P.n, k = P.inv[S23][l];
            for (uint32_t q = 0; q * 4 < W; q++) {
                uint32_t t23[4], r2[4];
                mask_block(T, P.rk[S23], 1u, k, q, t23);
                mask_block(T, P.rk[S12], 2u, l, q, r2);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t w = 4 * q + e;
                    if (w < W) {
                        P.c1[l * W + w] = op_sub(g, op_add(g, P.x1[k * W + w], t23[e]), r2[e]);
                        P.s[1][l * W + w] = r2[e];
                    }
                }
            }
        }
    }
}

// CS3: C2[l] = Y1[j] - T31[j] - T23[k] - R1[l], R3[l] = C1[l] + C2[l], with k = pi23^-1(l),
// j = pi31^-1(k); outputs R1[l] and R3[l]
__global__ void __launch_bounds__(kShufThreads, 1) k_shuf_cs3(const __grid_constant__ ShufParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    const uint32_t W = P.width, g = P.group;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < P.n; l += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = P.inv[S23][l], j = P.comp3[l];
        for (uint32_t q = 0; q * 4 < W; q++) {
            uint32_t t31[4], t23[4], r1[4];
            mask_block(T, P.rk[S31], 1u, j, q, t31);
            mask_block(T, P.rk[S23], 1u, k, q, t23);
            mask_block(T, P.rk[S31], 2u, l, q, r1);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t w = 4 * q + e;
                if (w < W) {
                    const uint32_t c2 = op_sub(g, op_sub(g, op_sub(g, P.y1[j * W + w], t31[e]), t23[e]), r1[e]);
                    P.s[2][l * W + w] = op_add(g, P.c1[l * W + w], c2);
                    P.s[0][l * W + w] = r1[e];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ secFetch case II

struct PackParams {
    const uint32_t* x[3];
    const uint32_t* v[3];       // table share set j at attribute 0
    uint32_t* d[3];
    uint64_t n, stride;
    uint32_t n_attrs, width;
    uint32_t attrs[kShufMaxWidth];
};

__global__ void k_fetch_pack(const __grid_constant__ PackParams P) {
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P.n; c += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            uint32_t* row = P.d[j] + c * P.width;
            row[0] = P.x[j][c];
            row[1] = j == 0 ? (uint32_t)c : 0u;
            for (uint32_t a = 0; a < P.n_attrs; a++) row[2 + a] = P.v[j][(uint64_t)P.attrs[a] * P.stride + c];
        }
    }
}

constexpr int kCompactRows = 1024;   // rows per block of the open-and-compact pass

struct CompactParams {
    const uint32_t* s[3];
    uint32_t* out[3];
    uint32_t* block_count;      // per block: rows with x^ = 1
    uint64_t n, cap;
    uint32_t width, n_blocks;
};

__device__ __forceinline__ bool opened_one(const CompactParams& P, uint64_t l) {
    return l < P.n && P.s[0][l * P.width] + P.s[1][l * P.width] + P.s[2][l * P.width] == 1u;
}

// open x^ for a block of rows and count the ones
__global__ void __launch_bounds__(kCompactRows) k_open_count(const __grid_constant__ CompactParams P) {
    __shared__ uint32_t warp_n[kCompactRows / 32];
    const uint64_t l = (uint64_t)blockIdx.x * kCompactRows + threadIdx.x;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, opened_one(P, l));
    if ((threadIdx.x & 31) == 0) warp_n[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kCompactRows / 32; w++) s += warp_n[w];
        P.block_count[blockIdx.x] = s;
    }
}

// exclusive scan of the block counts in place (one CTA); the total goes to block_count[n_blocks]
__global__ void __launch_bounds__(1024) k_scan_counts(uint32_t* c, uint32_t n_blocks) {
    __shared__ uint32_t part[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n_blocks; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < n_blocks ? c[i] : 0u;
        part[threadIdx.x] = v;
        __syncthreads();
        for (uint32_t off = 1; off < 1024; off <<= 1) {   // Hillis-Steele inclusive scan
            const uint32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n_blocks) c[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) c[n_blocks] = carry;
}

// write the kept rows (id and attributes of every share set) at their scanned offsets
__global__ void __launch_bounds__(kCompactRows) k_compact(const __grid_constant__ CompactParams P) {
    __shared__ uint32_t warp_off[kCompactRows / 32];
    const uint64_t l = (uint64_t)blockIdx.x * kCompactRows + threadIdx.x;
    const bool keep = opened_one(P, l);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_off[warp] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kCompactRows / 32; w++) {
            const uint32_t t = warp_off[w];
            warp_off[w] = s;
            s += t;
        }
    }
    __syncthreads();
    if (!keep) return;
    const uint64_t m = (uint64_t)P.block_count[blockIdx.x] + warp_off[warp] + __popc(b & ((1u << lane) - 1u));
    if (m >= P.cap) return;
    const uint32_t W = P.width;
#pragma unroll
    for (int j = 0; j < 3; j++)
        for (uint32_t w = 1; w < W; w++) P.out[j][m * (W - 1) + (w - 1)] = P.s[j][l * W + w];
}

}  // namespace

// the shuffle on device buffers; scratch from the stream-ordered pool
oblivgm_status shuffle_device(oblivgm_ctx* ctx, uint32_t group, uint64_t n, uint32_t width, const uint32_t* const in[3],
                              const uint8_t seeds[48], uint32_t* const out[3], cudaStream_t s) {
    if (n == 0) return OBLIVGM_OK;
    ShufParams P;
    std::memset(&P, 0, sizeof P);
    for (int k = 0; k < 3; k++) {
        const RoundKeys rk = expand_key(seeds + 16 * k);
        std::memcpy(P.rk[k], rk.w, sizeof P.rk[k]);
        P.d[k] = in[k];
        P.s[k] = out[k];
    }
    P.te0 = ctx->d_te0;
    P.n = n;
    P.width = width;
    P.group = group;
    uint32_t bits = 0;
    for (uint64_t v = n - 1; v; v >>= 1) bits++;
    P.half_bits = std::max<uint32_t>(1, (bits + 1) / 2);
    const size_t perm_bytes = (size_t)n * 4, tab_bytes = (size_t)n * width * 4;
    const size_t ftab_bytes = 12ull * (1ull << P.half_bits) * 4;
    const size_t total = 7 * ((perm_bytes + 255) & ~size_t(255)) + 3 * ((tab_bytes + 255) & ~size_t(255)) +
                         ((ftab_bytes + 255) & ~size_t(255));
    uint8_t* scratch = nullptr;
    const oblivgm_status as = ws_alloc(ctx, reinterpret_cast<void**>(&scratch), total, s, "shuffle scratch");
    if (as != OBLIVGM_OK) return as;
    cudaError_t ce = cudaSuccess;
    size_t off = 0;
    for (int k = 0; k < 3; k++) {
        P.inv[k] = reinterpret_cast<uint32_t*>(scratch + off);
        off += (perm_bytes + 255) & ~size_t(255);
    }
    uint32_t** tabs[3] = {&P.x1, &P.y1, &P.c1};
    for (int k = 0; k < 3; k++) {
        *tabs[k] = reinterpret_cast<uint32_t*>(scratch + off);
        off += (tab_bytes + 255) & ~size_t(255);
    }
    P.ftab = reinterpret_cast<uint32_t*>(scratch + off);
    off += (ftab_bytes + 255) & ~size_t(255);
    P.comp1 = reinterpret_cast<uint32_t*>(scratch + off);
    off += (perm_bytes + 255) & ~size_t(255);
    P.comp3 = reinterpret_cast<uint32_t*>(scratch + off);
    for (int k = 0; k < 2; k++) {
        off += (perm_bytes + 255) & ~size_t(255);
        P.fwd[k] = reinterpret_cast<uint32_t*>(scratch + off);
    }
    auto grid = [&](uint64_t items) {
        return (unsigned)std::min<uint64_t>((items + kShufThreads - 1) / kShufThreads, (uint64_t)ctx->sm_count);
    };
    k_feistel_tab<<<grid(12ull << P.half_bits), kShufThreads, kTableBytes, s>>>(P);
    k_perms<<<(unsigned)std::min<uint64_t>((5 * n + 255) / 256, 16ull * ctx->sm_count), 256, 0, s>>>(P);
    k_compose<<<(unsigned)std::min<uint64_t>((2 * n + 255) / 256, 16ull * ctx->sm_count), 256, 0, s>>>(P);
    k_shuf_cs1<<<grid(n), kShufThreads, kTableBytes, s>>>(P);
    k_shuf_cs2<<<grid(2 * n), kShufThreads, kTableBytes, s>>>(P);
    k_shuf_cs3<<<grid(n), kShufThreads, kTableBytes, s>>>(P);
    ctx->launches += 6;
    ce = cudaGetLastError();
    const cudaError_t fe = cudaFreeAsync(scratch, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "shuffle launch");
    ce = fe;
    return ce == cudaSuccess ? OBLIVGM_OK : cuda_fail(ce, "shuffle scratch release");
}

oblivgm_status set_shuffle_attrs() {
    const void* fns[4] = {reinterpret_cast<const void*>(k_feistel_tab), reinterpret_cast<const void*>(k_shuf_cs1),
                          reinterpret_cast<const void*>(k_shuf_cs2), reinterpret_cast<const void*>(k_shuf_cs3)};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes);
        if (e != cudaSuccess) return cuda_fail(e, "shuffle kernel attributes");
    }
    return OBLIVGM_OK;
}

}  // namespace ogm

using namespace ogm;

extern "C" oblivgm_status oblivgm_shuffle(oblivgm_ctx* ctx, uint32_t group, uint64_t n_rows, uint32_t width,
                                          const uint32_t* const in[3], const uint8_t seeds[48],
                                          uint32_t* const out[3], void* stream) {
    const NvtxRange nvtx_range("oblivgm_shuffle");
    if (!ctx || !in || !out || !seeds) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (group != OBLIVGM_SHUFFLE_ADD && group != OBLIVGM_SHUFFLE_XOR) return fail(OBLIVGM_EINVAL, "unknown share group");
    if (width < 1 || width > kShufMaxWidth) return fail(OBLIVGM_EINVAL, "width must be 1..64");
    if (n_rows >= (1ull << 31)) return fail(OBLIVGM_EINVAL, "at most 2^31 - 1 rows");
    for (int j = 0; j < 3; j++) {
        if (n_rows && (!in[j] || !out[j])) return fail(OBLIVGM_EINVAL, "NULL share set");
        if (reinterpret_cast<uintptr_t>(in[j]) % 4 || reinterpret_cast<uintptr_t>(out[j]) % 4)
            return fail(OBLIVGM_EINVAL, "share sets must be 4-byte aligned");
    }
    const cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    return shuffle_device(ctx, group, n_rows, width, in, seeds, out, static_cast<cudaStream_t>(stream));
}

extern "C" oblivgm_status oblivgm_fetch_multi(oblivgm_ctx* ctx, uint32_t table_id, const uint32_t* const x[3],
                                              uint32_t n_attrs, const uint32_t* attrs, const uint8_t seeds[48],
                                              uint32_t* const out[3], uint64_t cap, uint64_t* count, void* stream) {
    const NvtxRange nvtx_range("oblivgm_fetch_multi");
    if (!ctx || !x || !out || !seeds || !count || (n_attrs && !attrs)) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (n_attrs + 2 > kShufMaxWidth) return fail(OBLIVGM_EINVAL, "at most 62 attributes");
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    auto it = ctx->tables.find(table_id);
    if (it == ctx->tables.end()) return fail(OBLIVGM_ENOENT, "no such table");
    const Table& tb = it->second;
    for (uint32_t a = 0; a < n_attrs; a++)
        if (attrs[a] >= tb.n_attrs) return fail(OBLIVGM_EINVAL, "attribute outside the table");
    const uint64_t n = tb.n_elems;
    if (n >= (1ull << 31)) return fail(OBLIVGM_EINVAL, "at most 2^31 - 1 elements");
    for (int j = 0; j < 3; j++)
        if (n && (!x[j] || (cap && !out[j]))) return fail(OBLIVGM_EINVAL, "NULL share set");
    *count = 0;
    if (n == 0) return OBLIVGM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t W = 2 + n_attrs;
    const uint32_t n_blocks = (uint32_t)((n + kCompactRows - 1) / kCompactRows);
    const size_t tab = ((size_t)n * W * 4 + 255) & ~size_t(255);
    const size_t total = 6 * tab + ((size_t)(n_blocks + 1) * 4 + 255);
    uint8_t* scratch = nullptr;
    {
        const oblivgm_status as = ws_alloc(ctx, reinterpret_cast<void**>(&scratch), total, s, "fetch scratch");
        if (as != OBLIVGM_OK) return as;
    }
    PackParams K;
    std::memset(&K, 0, sizeof K);
    uint32_t* d[3];
    uint32_t* sh[3];
    for (int j = 0; j < 3; j++) {
        d[j] = reinterpret_cast<uint32_t*>(scratch + j * tab);
        sh[j] = reinterpret_cast<uint32_t*>(scratch + (3 + j) * tab);
        K.x[j] = x[j];
        K.v[j] = tb.dev + (uint64_t)j * tb.n_attrs * tb.stride;
        K.d[j] = d[j];
    }
    uint32_t* counts = reinterpret_cast<uint32_t*>(scratch + 6 * tab);
    K.n = n;
    K.stride = tb.stride;
    K.n_attrs = n_attrs;
    K.width = W;
    if (n_attrs) std::memcpy(K.attrs, attrs, n_attrs * sizeof(uint32_t));
    k_fetch_pack<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 8ull * ctx->sm_count), 256, 0, s>>>(K);
    ctx->launches++;
    const uint32_t* din[3] = {d[0], d[1], d[2]};
    uint32_t* dout[3] = {sh[0], sh[1], sh[2]};
    oblivgm_status st = shuffle_device(ctx, OBLIVGM_SHUFFLE_ADD, n, W, din, seeds, dout, s);
    if (st) {
        cudaFreeAsync(scratch, s);
        return st;
    }
    CompactParams C;
    std::memset(&C, 0, sizeof C);
    for (int j = 0; j < 3; j++) {
        C.s[j] = sh[j];
        C.out[j] = out[j];
    }
    C.block_count = counts;
    C.n = n;
    C.cap = cap;
    C.width = W;
    C.n_blocks = n_blocks;
    k_open_count<<<n_blocks, kCompactRows, 0, s>>>(C);
    k_scan_counts<<<1, 1024, 0, s>>>(counts, n_blocks);
    k_compact<<<n_blocks, kCompactRows, 0, s>>>(C);
    ctx->launches += 3;
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        cudaFreeAsync(scratch, s);
        return cuda_fail(ce, "fetch launch");
    }
    uint32_t total_count = 0;
    ce = cudaMemcpyAsync(&total_count, counts + n_blocks, 4, cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) {
        cudaFreeAsync(scratch, s);
        return cuda_fail(ce, "fetch count read");
    }
    ce = cudaFreeAsync(scratch, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch scratch release");
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "fetch synchronize");
    *count = total_count;
    return OBLIVGM_OK;
}
