// oblivgm.cu -- context, resident share store, raw DPF/DCF batches and the
// fused secEval kernels (mask-open, six key-half walks per predicate, per-server
// sums, PRF re-share, RSS fold of a group's predicates, output write) of the
// oblivgm library: k_filter (one thread per element) and k_filter_wp (one thread
// per key walk, for small batches), the batch planner that picks between them,
// prepared plans and the no-allocation entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "device_fss.cuh"
#include "host_crypto.h"
#include "ptx_async.cuh"
#include "oblivgm.h"
#include "runtime.h"

namespace ogm {

thread_local std::string g_last_error;

oblivgm_status fail(oblivgm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

const std::string& last_error_text() { return g_last_error; }

oblivgm_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? OBLIVGM_ENOMEM : OBLIVGM_ECUDA;
}

oblivgm_status ws_alloc(oblivgm_ctx* ctx, void** p, size_t bytes, cudaStream_t s, const char* what) {
    *p = nullptr;
    if (ctx->test_fail_alloc.exchange(false)) return fail(OBLIVGM_ENOMEM, std::string(what) + ": refused (test hook)");
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(OBLIVGM_ENOMEM, std::string(what) + ": out of device memory");
    }
    return e == cudaSuccess ? OBLIVGM_OK : cuda_fail(e, what);
}

#define OGM_CUDA(call, what)                      \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// ------------------------------------------------------------------ PTX helpers
// (mbarriers, bulk copies and the bounded wait are in ptx_async.cuh)

// ------------------------------------------------------------------ fused secEval

struct GroupDesc {
    const uint32_t* share[3];   // share set j of the group's table: [attr][stride]
    uint32_t* out[3];           // RSS share sets of the result, n_elems each
    uint64_t stride;
    uint64_t n_elems;
    uint32_t query_id, table_id, pred_begin, n_preds;
    uint32_t vec_out;           // out pointers are 16-byte aligned
    uint32_t tile;              // elements per work item of this group (k_filter_wp; k_filter uses the launch's)
    uint32_t slots;             // k_filter_wp: walk threads per element, 6 (equality predicates only) or 12
    uint32_t pad;
};

struct PredDesc {
    uint32_t kind, n_bits, attr, step;
    uint32_t r[3];
    uint32_t cbeta;
    uint32_t key_begin, n_keys;
    // fold into the group's result: w_i = lin (a_i + b_i) + prod (a_i b_i + a_i b_{i+1} + a_{i+1} b_i)
    uint32_t lin, prod;
};

struct FilterParams {
    AesParams aes;
    uint32_t rk_prf[3][44];
    const uint32_t* te0;
    const GroupDesc* groups;
    const PredDesc* preds;
    const DevKey* keys;
    const uint64_t* item_start;   // n_groups + 1 prefix sums of element tiles
    unsigned long long* counter;  // work queue head
    uint32_t* done;               // CTAs of the walk-parallel kernel that have finished (it resets both)
    uint32_t* error;              // context fault flags
    uint32_t n_groups;
    uint32_t tile;                // elements per item (a multiple of 32 E, at most blockDim.x * E)
    uint64_t wait_limit_ns;       // bound of every key-staging wait
    uint32_t expect_extra;        // failure-path test only: bytes expected beyond the copy (0 normally)
    uint32_t resident_bytes;      // walk-parallel kernel: nonzero when the workspace from `groups` to the
                                  // end of `item_start` (this many bytes) fits its shared memory whole
};

constexpr int kMaxKeysPerPred = 12;
constexpr int kFilterSmem = kTableBytes + kMaxKeysPerPred * (int)sizeof(DevKey);

// re-share of a 3-out-of-3 sharing z into RSS: r_i = z_i + F(k_i, ctr) - F(k_{i-1}, ctr).
// F(k_i) enters r_i with + and r_{i+1} with -; the loop over the three PRF keys is
// kept rolled so the code holds one AES body per element.
template <int E, class Tab>
__device__ __forceinline__ void reshare(const Tab& T, const uint32_t (&rk_prf)[3][44], const uint32_t z[3][E],
                                        uint32_t out[3][E], uint64_t e0, uint32_t step, uint32_t table,
                                        uint32_t query) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int e = 0; e < E; e++) out[i][e] = z[i][e];
#pragma unroll 1
    for (int i = 0; i < 3; i++) {
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint64_t el = e0 + (uint64_t)e;
            const uint32_t ctr[4] = {(uint32_t)el, (uint32_t)(el >> 32), step | (table << 16), query};
            const uint32_t f = aes_one_w0(T, rk_prf[i], ctr);   // F keeps bytes 0..3
            out[0][e] += i == 0 ? f : (i == 2 ? 0u - f : 0u);
            out[1][e] += i == 1 ? f : (i == 0 ? 0u - f : 0u);
            out[2][e] += i == 2 ? f : (i == 1 ? 0u - f : 0u);
        }
    }
}

template <int E>
__device__ __forceinline__ void load_col(const uint32_t* __restrict__ col, uint64_t e0, uint64_t n_elems, uint32_t v[E]) {
    if constexpr (E == 4) {
        if (e0 < n_elems) {   // stride is a multiple of 4, so the vector stays inside the row
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(col + e0));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            return;
        }
    } else if constexpr (E == 2) {
        if (e0 < n_elems) {
            const uint2 q = __ldg(reinterpret_cast<const uint2*>(col + e0));
            v[0] = q.x; v[1] = q.y;
            return;
        }
    } else {
        if (e0 < n_elems) { v[0] = __ldg(col + e0); return; }
    }
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = 0;
}

template <int E>
__device__ __forceinline__ void store_col(uint32_t* col, uint64_t e0, uint64_t n_elems, bool vec, const uint32_t v[E]) {
    if constexpr (E == 4) {
        if (vec && e0 + 3 < n_elems) {
            *reinterpret_cast<uint4*>(col + e0) = make_uint4(v[0], v[1], v[2], v[3]);
            return;
        }
    } else if constexpr (E == 2) {
        if (vec && e0 + 1 < n_elems) {
            *reinterpret_cast<uint2*>(col + e0) = make_uint2(v[0], v[1]);
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < E; e++)
        if (e0 + e < n_elems) col[e0 + e] = v[e];
}

// largest CTA each variant may be launched with (sets the register budget)
template <int E> constexpr int max_threads() { return E == 1 ? 1024 : 512; }

template <int E>
__global__ void __launch_bounds__(max_threads<E>(), 1) k_filter(const __grid_constant__ FilterParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    DevKey* kbuf = reinterpret_cast<DevKey*>(smem + kTableBytes);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ unsigned long long item_sh;

    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    if (threadIdx.x == 0) mbar_init(&mbar);
    __syncthreads();

    uint32_t phase = 0;
    const uint64_t n_items = P.item_start[P.n_groups];
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(P.counter, 1ull);
        __syncthreads();
        const uint64_t item = item_sh;
        if (item >= n_items) break;
        int lo = 0, hi = (int)P.n_groups - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.item_start[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const GroupDesc& G = P.groups[lo];
        // threads past the tile width (a multiple of 32 E, so whole warps) stay idle
        const bool in_tile = threadIdx.x * E < P.tile;
        const uint64_t e0 = (item - P.item_start[lo]) * P.tile + (uint64_t)threadIdx.x * E;
        const uint64_t n_elems = G.n_elems;
        const bool warp_busy = __any_sync(0xFFFFFFFFu, in_tile && e0 < n_elems);
        const uint32_t table = G.table_id, query = G.query_id;
        uint32_t acc[3][E];
        for (uint32_t k = 0; k < G.n_preds; k++) {
            const PredDesc& D = P.preds[G.pred_begin + k];
            __syncthreads();   // everyone is done with the previous predicate's keys
            if (threadIdx.x == 0) {
                const uint32_t bytes = D.n_keys * (uint32_t)sizeof(DevKey);
                mbar_expect_tx(&mbar, bytes + P.expect_extra);
                bulk_g2s(kbuf, P.keys + D.key_begin, bytes, &mbar);
            }
            const bool ok = mbar_wait_bounded(&mbar, phase, P.wait_limit_ns);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(P.error, kErrKeyWait);
                mbar_wait_bounded(&mbar, phase ^ 1u, P.wait_limit_ns);   // let an in-flight copy land
                return;
            }
            if (!warp_busy) continue;
            // open x^ = <x>_1 + <x>_2 + <x>_3 + <r>_1 + <r>_2 + <r>_3 mod 2^n
            const uint32_t mask = D.n_bits >= 32 ? 0xFFFFFFFFu : ((1u << D.n_bits) - 1u);
            uint32_t xh[E], sh[E];
            const uint64_t row = (uint64_t)D.attr * G.stride;
#pragma unroll
            for (int e = 0; e < E; e++) xh[e] = D.r[0] + D.r[1] + D.r[2];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                load_col<E>(G.share[j] + row, e0, n_elems, sh);
#pragma unroll
                for (int e = 0; e < E; e++) xh[e] += sh[e];
            }
#pragma unroll
            for (int e = 0; e < E; e++) xh[e] &= mask;
            // Eq. (predEval), masked form: CS_i sums the outputs of its two key halves.
            // keys are ordered [server i][half h][sub s]; one walk instance of each kind
            // is kept in the code and driven by a runtime loop
            uint32_t z[3][E];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int e = 0; e < E; e++) z[i][e] = 0;
            const bool eq = D.kind == OBLIVGM_PRED_EQ;
            const int nsub = eq ? 1 : 2;
            const int n_keys = 6 * nsub;
            for (int kk = 0; kk < n_keys; kk++) {
                const DevKey& K = kbuf[kk];
                uint32_t y[E];
                if (eq) dpf_walk<E>(T, P.aes, K, xh, y);
                else dcf_walk<E>(T, P.aes, K, xh, y);
                // RANGE: the public constant c * beta' joins party 0's half once
                const uint32_t add = (!eq && (kk % nsub) == 0 && K.party == 0) ? D.cbeta : 0u;
                const int i = kk / (2 * nsub);
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const uint32_t v = y[e] + add;
                    z[0][e] += i == 0 ? v : 0u;
                    z[1][e] += i == 1 ? v : 0u;
                    z[2][e] += i == 2 ? v : 0u;
                }
            }
            // re-share the predicate's sum to RSS (step p); from the second predicate on,
            // fold it into the accumulator -- the RSS product (Sec. III-B: a_i b_i + a_i b_{i+1}
            // + a_{i+1} b_i) plus, for XOR / OR, the linear terms (Sec. V-D) -- and re-share
            // the result (step 64 + p).  One re-share call site, two passes.
            uint32_t step = D.step;
            const int passes = k == 0 ? 1 : 2;
#pragma unroll 1
            for (int pass = 0; pass < passes; pass++) {
                uint32_t r[3][E];
                reshare<E>(T, P.rk_prf, z, r, e0, step, table, query);
                if (pass + 1 < passes) {
#pragma unroll
                    for (int i = 0; i < 3; i++)
#pragma unroll
                        for (int e = 0; e < E; e++) {
                            const int i1 = (i + 1) % 3;
                            const uint32_t pr = acc[i][e] * r[i][e] + acc[i][e] * r[i1][e] + acc[i1][e] * r[i][e];
                            z[i][e] = D.lin * (acc[i][e] + r[i][e]) + D.prod * pr;
                        }
                    step = 64u + D.step;
                } else {
#pragma unroll
                    for (int i = 0; i < 3; i++)
#pragma unroll
                        for (int e = 0; e < E; e++) acc[i][e] = r[i][e];
                }
            }
        }
        if (in_tile) {
#pragma unroll
            for (int i = 0; i < 3; i++) store_col<E>(G.out[i], e0, n_elems, G.vec_out != 0, acc[i]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ raw batches

struct RawParams {
    AesParams aes;
    const uint32_t* te0;
    const DevKey* keys;
    const uint32_t* points;
    const uint32_t* key_of_point;
    uint32_t* out;
    uint64_t n_points;
    uint32_t n_keys;
    uint32_t all_pairs;
};

template <uint32_t KIND>
__global__ void __launch_bounds__(256) k_eval_raw(const __grid_constant__ RawParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n_points) return;
    const uint32_t key = P.all_pairs ? blockIdx.y : P.key_of_point[i];
    uint64_t o = i;
    if (P.all_pairs) o = (uint64_t)key * P.n_points + i;
    if (key >= P.n_keys) { P.out[o] = 0u; return; }
    const DevKey& K = P.keys[key];
    const uint32_t mask = K.n >= 32 ? 0xFFFFFFFFu : ((1u << K.n) - 1u);
    uint32_t x[1] = {P.points[i] & mask}, y[1];
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    if (KIND == OBLIVGM_KEY_DPF) dpf_walk<1>(T, P.aes, K, x, y);
    else dcf_walk<1>(T, P.aes, K, x, y);
    P.out[o] = y[0];
}

}  // namespace ogm

// ====================================================================== host side

using namespace ogm;

namespace ogm {

// ------------------------------------------------------------------ walk-parallel filter
//
// For queries too small to give every SM its own tiles: every key walk of an element gets
// its own thread (the six DPF or twelve DCF keys of a predicate), so an element's walks run
// side by side instead of one after another in one thread; a DCF walk is split once more
// over two threads.  Each DCF level takes two PRG calls on the same seed s_i: the seed /
// control-bit block of the chosen child and its value block.  The walk's seed thread
// computes the first and the next seed, the walk's value thread the second, both at once:
// the seed thread leaves (s_i, t_i) in shared memory for its partner, and one barrier of
// the two threads' warps per level (all walks of a CTA have the same n) orders the hand-over.  The keys are staged
// as in k_filter; the walks' outputs meet in shared memory, and the element's first slot
// thread sums them per server, re-shares and folds exactly as k_filter does.

constexpr int kWpSlots = 12;                          // key walks per element
constexpr int kWpElems = 40;                          // elements per CTA (tile)
constexpr int kWpWalks = kWpSlots * kWpElems;         // 480 seed threads, then 480 value threads
constexpr int kWpEqSlots = 6;                         // walk threads per element of a group of equality predicates
constexpr int kWpEqElems = kWpWalks / kWpEqSlots;     // such a group's tile: up to 80 elements
constexpr int kWpThreads = 2 * kWpWalks;              // 960
static_assert(kWpWalks % 32 == 0 && kWpWalks / 32 <= 15, "one named barrier (1..15) per walk pair of warps");
constexpr int kWpPrf = 6;                             // re-share PRF words per element: 2 passes x 3 keys
constexpr int kWpResidentOff = kFilterSmem + (kWpWalks + kWpEqElems * kWpPrf) * 4 +   // walk outputs, PRF words
                               2 * kWpWalks * 16 + 2 * kWpWalks * 4 + kWpWalks * 4; // seed / control-bit hand-over, V
constexpr int kWpResidentBytes = 48 * 1024;   // descriptors, keys and tile offsets of a small launch
constexpr int kWpSmem = kWpResidentOff + kWpResidentBytes;
static_assert(kWpResidentOff % 16 == 0, "bulk copies need 16-byte aligned destinations");
// default switch-over: batches of at most this many elements per SM in all
constexpr uint64_t kWpDefaultElemsPerSm = 128;
// launches of at most this many groups get a tile width per group (walk-parallel kernel)
constexpr size_t kWpTileGroups = 4;

// The seed warp w (< 15) and the value warp 15 + w of a walk pair meet at named barrier
// 1 + w (64 threads): the per-level hand-over needs only the two of them, so pairs do not
// wait for one another and drift apart, which keeps the lookup and logic pipes busy.
__device__ __forceinline__ void wp_pair_sync(uint32_t walk) {
    asm volatile("bar.sync %0, 64;" ::"r"(1u + walk / 32u) : "memory");
}

__global__ void __launch_bounds__(kWpThreads, 1) k_filter_wp(const __grid_constant__ FilterParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemTab T{reinterpret_cast<const char*>(smem), lane_offset()};
    DevKey* kbuf = reinterpret_cast<DevKey*>(smem + kTableBytes);
    uint32_t* part = reinterpret_cast<uint32_t*>(smem + kFilterSmem);   // [element][slot]
    uint32_t* fprf = part + kWpWalks;                                      // [element][pass * 3 + key]
    uint4* sbuf = reinterpret_cast<uint4*>(fprf + kWpEqElems * kWpPrf);    // [2][walk]: s_i
    uint32_t* tbuf = reinterpret_cast<uint32_t*>(sbuf + 2 * kWpWalks);     // [2][walk]: t_i
    uint32_t* vbuf = tbuf + 2 * kWpWalks;                                  // [walk]: the value sum V
    unsigned char* wsm = smem + kWpResidentOff;                            // resident copy of the workspace
    __shared__ __align__(8) uint64_t mbar;
    __shared__ unsigned long long item_sh;

    // A small launch's descriptors, keys and tile offsets come into shared memory with one
    // bulk copy that runs while the tables fill; the items then read no global descriptor
    // and stage no keys.  Otherwise they are read from global memory and each predicate's
    // keys are staged as k_filter does.
    const bool resident = P.resident_bytes != 0;
    if (threadIdx.x == 0) {
        mbar_init(&mbar);
        if (resident) {
            mbar_expect_tx(&mbar, P.resident_bytes + P.expect_extra);
            bulk_g2s(wsm, P.groups, P.resident_bytes, &mbar);
        }
    }
    fill_tables(reinterpret_cast<uint32_t*>(smem), P.te0);
    __syncthreads();
    uint32_t phase = 0;
    bool failed = false;
    if (resident) {
        const bool ok = mbar_wait_bounded(&mbar, phase, P.wait_limit_ns);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(P.error, kErrKeyWait);
            mbar_wait_bounded(&mbar, phase ^ 1u, P.wait_limit_ns);   // let an in-flight copy land
            failed = true;
        }
    }
    const auto rel = [&](const void* p) {
        return wsm + (reinterpret_cast<const unsigned char*>(p) - reinterpret_cast<const unsigned char*>(P.groups));
    };
    const GroupDesc* groups = resident ? reinterpret_cast<const GroupDesc*>(wsm) : P.groups;
    const PredDesc* preds = resident ? reinterpret_cast<const PredDesc*>(rel(P.preds)) : P.preds;
    const DevKey* rkeys = reinterpret_cast<const DevKey*>(rel(P.keys));
    const uint64_t* item_start = resident ? reinterpret_cast<const uint64_t*>(rel(P.item_start)) : P.item_start;

    const bool value_thread = threadIdx.x >= (unsigned)kWpWalks;
    const uint32_t walk = threadIdx.x % kWpWalks;
    const uint64_t n_items = failed ? 0 : item_start[P.n_groups];
    // the first item of CTA b is item b (the grid has at most n_items CTAs); later ones come
    // from the work counter, past the first gridDim.x
    for (uint32_t round = 0;; round++) {
        if (threadIdx.x == 0) item_sh = round == 0 ? blockIdx.x : gridDim.x + atomicAdd(P.counter, 1ull);
        __syncthreads();
        const uint64_t item = item_sh;
        if (item >= n_items) break;
        int lo = 0, hi = (int)P.n_groups - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_start[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const GroupDesc& G = groups[lo];
        const uint32_t tile = G.tile, sw = G.slots;   // elements per item, walk threads per element
        const uint32_t el = walk / sw, slot = walk % sw;
        const uint64_t e = (item - item_start[lo]) * tile + el;
        const uint64_t n_elems = G.n_elems;
        const bool valid = el < tile && e < n_elems;
        const uint32_t table = G.table_id, query = G.query_id;
        uint32_t acc[3][1] = {{0}, {0}, {0}};
        for (uint32_t k = 0; k < G.n_preds; k++) {
            const PredDesc& D = preds[G.pred_begin + k];
            __syncthreads();   // everyone is done with the previous predicate's keys and outputs
            if (!resident) {
                if (threadIdx.x == 0) {
                    const uint32_t bytes = D.n_keys * (uint32_t)sizeof(DevKey);
                    mbar_expect_tx(&mbar, bytes + P.expect_extra);
                    bulk_g2s(kbuf, P.keys + D.key_begin, bytes, &mbar);
                }
                const bool ok = mbar_wait_bounded(&mbar, phase, P.wait_limit_ns);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) atomicOr(P.error, kErrKeyWait);
                    mbar_wait_bounded(&mbar, phase ^ 1u, P.wait_limit_ns);   // let an in-flight copy land
                    failed = true;
                    break;
                }
            }
            const DevKey* pkeys = resident ? rkeys + D.key_begin : kbuf;
            const bool eq = D.kind == OBLIVGM_PRED_EQ;
            const uint32_t nsub = eq ? 1u : 2u;
            const bool active = valid && slot < 6 * nsub;
            uint32_t xh = 0;
            if (active) {
                const uint32_t mask = D.n_bits >= 32 ? 0xFFFFFFFFu : ((1u << D.n_bits) - 1u);
                const uint64_t row = (uint64_t)D.attr * G.stride;
                xh = D.r[0] + D.r[1] + D.r[2];
#pragma unroll
                for (int j = 0; j < 3; j++) xh += __ldg(G.share[j] + row + e);
                xh &= mask;
            }
            const DevKey& K = pkeys[slot];
            uint32_t y = 0;
            // one loop for both kinds: the seed thread walks the seed / control-bit chain (a
            // DPF walk whole); for a DCF the value thread takes each level's value block on
            // the seed s_i the seed thread hands over, one barrier of the walk pair per level
            // (n and the kind are the same for every walk of the CTA)
            const int n = (int)D.n_bits;
            const uint32_t party = K.party;
            uint32_t s[4] = {0, 0, 0, 0}, t = party, V = 0;
            if (active && !value_thread) {
#pragma unroll
                for (int w = 0; w < 4; w++) s[w] = K.seed[w];
                if (!eq) {
                    sbuf[walk] = make_uint4(s[0], s[1], s[2], s[3]);
                    tbuf[walk] = t;
                }
            }
            if (!eq) wp_pair_sync(walk);
            for (int i = 0; i < n; i++) {
                const uint32_t dir = (xh >> (n - 1 - i)) & 1u;
                const uint32_t m = 0u - dir;
                if (active && !value_thread) {
                    // seed / control-bit block of the chosen child and its correction
                    uint32_t o[4];
                    aes_sel(T, P.aes.rk_st, P.aes.d_st, m, s, o);
                    const uint4 cw = *reinterpret_cast<const uint4*>(K.scw[i]);
#pragma unroll
                    for (int w = 0; w < 4; w++) o[w] ^= s[w];
                    uint32_t tn = o[0] & 1u;
                    o[0] &= ~1u;
                    const uint32_t tm = 0u - t;
                    s[0] = o[0] ^ (cw.x & tm);
                    s[1] = o[1] ^ (cw.y & tm);
                    s[2] = o[2] ^ (cw.z & tm);
                    s[3] = o[3] ^ (cw.w & tm);
                    tn ^= t & (((dir ? K.tr : K.tl) >> i) & 1u);
                    t = tn;
                    if (!eq) {
                        sbuf[((i + 1) & 1) * kWpWalks + walk] = make_uint4(s[0], s[1], s[2], s[3]);
                        tbuf[((i + 1) & 1) * kWpWalks + walk] = t;
                    }
                } else if (active && !eq) {
                    // value block on the same seed s_i: V += (-1)^b (Convert(v) + t_i V_CW)
                    const uint4 si = sbuf[(i & 1) * kWpWalks + walk];
                    const uint32_t ti = tbuf[(i & 1) * kWpWalks + walk];
                    const uint32_t sv[4] = {si.x, si.y, si.z, si.w};
                    const uint32_t v0 = aes_sel_w0(T, P.aes.rk_v, P.aes.d_v, m, sv);
                    const uint32_t term = (v0 ^ si.x) + (ti ? K.vcw[i] : 0u);
                    V += party ? 0u - term : term;
                }
                if (!eq) wp_pair_sync(walk);   // s_{i+1} visible; the partner is done reading s_i
            }
            if (!eq) {
                if (active && value_thread) vbuf[walk] = V;
                wp_pair_sync(walk);
            }
            if (active && !value_thread) {
                const uint32_t term = s[1] + (t ? K.cw_final : 0u);   // Convert(s_n): bytes 4..7
                y = (eq ? 0u : vbuf[walk]) + (party ? 0u - term : term);
                // RANGE: the public constant c * beta' joins party 0's half once
                if (!eq && (slot % nsub) == 0 && party == 0) y += D.cbeta;
            }
            if (!value_thread) part[el * sw + slot] = y;
            // The re-share PRF words depend only on (element, step, table, query), so six
            // value threads compute the (pass, key) pairs side by side (for an equality
            // predicate while the seed threads walk): pass p re-shares with step
            // D.step + 64 p (the fold's re-share, for every predicate after the first).
            const int passes = k == 0 ? 1 : 2;
            if (value_thread && valid && slot < 3u * passes) {
                const uint32_t pass = slot / 3, i = slot % 3;
                const uint32_t ctr[4] = {(uint32_t)e, (uint32_t)(e >> 32), (D.step + 64u * pass) | (table << 16),
                                         query};
                fprf[el * kWpPrf + slot] = aes_one_w0(T, P.rk_prf[i], ctr);   // F keeps bytes 0..3
            }
            __syncthreads();
            if (!value_thread && slot == 0 && valid) {
                // keys are ordered [server i][half h][sub s]: server i owns slots [2 nsub i, 2 nsub (i + 1))
                uint32_t z[3][1] = {{0}, {0}, {0}};
                for (uint32_t kk = 0; kk < 6 * nsub; kk++) {
                    const uint32_t v = part[el * sw + kk], i = kk / (2 * nsub);
                    z[0][0] += i == 0 ? v : 0u;
                    z[1][0] += i == 1 ? v : 0u;
                    z[2][0] += i == 2 ? v : 0u;
                }
#pragma unroll 1
                for (int pass = 0; pass < passes; pass++) {
                    // r_i = z_i + F(k_i) - F(k_{i-1}), as reshare() computes it
                    const uint32_t* f = fprf + el * kWpPrf + 3 * pass;
                    uint32_t r[3][1];
#pragma unroll
                    for (int i = 0; i < 3; i++) r[i][0] = z[i][0] + f[i] - f[(i + 2) % 3];
                    if (pass + 1 < passes) {
#pragma unroll
                        for (int i = 0; i < 3; i++) {
                            const int i1 = (i + 1) % 3;
                            const uint32_t pr = acc[i][0] * r[i][0] + acc[i][0] * r[i1][0] + acc[i1][0] * r[i][0];
                            z[i][0] = D.lin * (acc[i][0] + r[i][0]) + D.prod * pr;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 3; i++) acc[i][0] = r[i][0];
                    }
                }
            }
        }
        if (failed) break;   // the CTA records the fault and leaves its outputs alone
        if (!value_thread && slot == 0 && valid) {
#pragma unroll
            for (int i = 0; i < 3; i++) G.out[i][e] = acc[i][0];
        }
        __syncthreads();
    }
    // the last CTA to finish resets the work counter and this count, so that the next launch
    // of a prepared plan finds them at zero without a separate clear
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(P.done, 1u) == gridDim.x - 1) {
            *P.counter = 0ull;
            *P.done = 0u;
        }
    }
}

void build_aes_params(AesParams* a) {
    const RoundKeys &L = fixed_key(0), &R = fixed_key(1), &VL = fixed_key(2), &VR = fixed_key(3);
    for (int i = 0; i < 44; i++) {
        a->rk_st[i] = L.w[i];
        a->d_st[i] = L.w[i] ^ R.w[i];
        a->rk_v[i] = VL.w[i];
        a->d_v[i] = VL.w[i] ^ VR.w[i];
    }
}

static oblivgm_status check_ctx(oblivgm_ctx* ctx) {
    if (!ctx) return fail(OBLIVGM_EINVAL, "NULL context");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return OBLIVGM_OK;
}

// Build device descriptors of the given queries' groups (groups sorted by per-tile
// cost, most expensive first) into one contiguous host image.
struct Plan {
    uint32_t tile = 0, elems_per_thread = 1, threads = 0;
    bool wp = false;   // walk-parallel kernel (k_filter_wp)
    std::vector<GroupDesc> groups;
    std::vector<PredDesc> preds;
    std::vector<DevKey> keys;
    std::vector<uint64_t> item_start;
};

// Element tile per work item.  The items (group, tile) are taken by one persistent CTA
// per SM in cost order; a tile width that leaves the last wave half empty wastes the
// idle SMs' time, and a query too small to give every SM a full-width tile leaves SMs
// idle altogether, so widths from max_tile down to `step` are tried by simulating that
// greedy schedule, with item_time(group, width) as an item's time, and the width with
// the shortest makespan wins (the widest on ties).  Large item counts skip the search:
// their tail is already a small fraction.
// Makespan of the greedy schedule: items (group, tile) in group order, each taken by the CTA
// that is free first (one persistent CTA per SM); tile_of(g) is group g's width.
template <typename NF, typename WF, typename TF>
double simulate_makespan(size_t n_groups, NF n_elems_of, WF tile_of, TF item_time, int sm_count,
                         std::vector<double>& finish) {
    finish.assign((size_t)sm_count, 0.0);
    std::make_heap(finish.begin(), finish.end(), std::greater<double>());
    for (size_t g = 0; g < n_groups; g++) {
        const uint64_t n = n_elems_of(g), t = tile_of(g);
        for (uint64_t e = 0; e < n; e += t) {
            std::pop_heap(finish.begin(), finish.end(), std::greater<double>());
            finish.back() += item_time(g, std::min<uint64_t>(t, n - e));
            std::push_heap(finish.begin(), finish.end(), std::greater<double>());
        }
    }
    return *std::max_element(finish.begin(), finish.end());
}

template <typename NF, typename TF>
uint32_t choose_tile(size_t n_groups, NF n_elems_of, TF item_time, uint32_t max_tile, uint32_t step, int sm_count) {
    uint64_t items_at_max = 0;
    for (size_t g = 0; g < n_groups; g++) items_at_max += (n_elems_of(g) + max_tile - 1) / max_tile;
    if (items_at_max == 0 || items_at_max > 64ull * (uint64_t)sm_count || step == 0) return max_tile;
    uint32_t best_tile = max_tile;
    double best = -1.0;
    std::vector<double> finish;
    for (uint32_t t = max_tile; t >= step; t -= step) {
        if (best >= 0) {
            // skip a width whose work, spread evenly over the SMs, already takes longer
            double total = 0;
            for (size_t g = 0; g < n_groups; g++) {
                const uint64_t n = n_elems_of(g);
                total += (double)(n / t) * item_time(g, t) + (n % t ? item_time(g, n % t) : 0.0);
            }
            if (total / sm_count > best) {
                if (t < 2 * step) break;
                continue;
            }
        }
        const double makespan =
            simulate_makespan(n_groups, n_elems_of, [&](size_t) { return (uint64_t)t; }, item_time, sm_count, finish);
        if (best < 0 || makespan < best * (1.0 - 1e-9)) { best = makespan; best_tile = t; }
        if (t < 2 * step) break;
    }
    return best_tile;
}

// Per-group widths for a small launch of a few groups (the walk-parallel kernel): starting
// from the common width, each group's width in turn is set to the one (its maximum down to 1)
// that shortens the simulated makespan most (the widest on a tie), the others held, in two
// rounds.  An equality group's items are cheaper than a range group's, so the two kinds
// balance best at different widths, and fitting all items into one wave avoids a CTA
// taking two.
template <typename NF, typename TF, typename MF>
void choose_group_tiles(size_t n_groups, NF n_elems_of, TF item_time, MF max_tile_of, int sm_count,
                        std::vector<uint32_t>& tiles) {
    std::vector<double> finish;
    auto makespan = [&]() {
        return simulate_makespan(n_groups, n_elems_of, [&](size_t g) { return (uint64_t)tiles[g]; }, item_time,
                                 sm_count, finish);
    };
    // no schedule beats the work spread evenly over the SMs, nor its longest item
    auto lower_bound = [&]() {
        double total = 0, longest = 0;
        for (size_t g = 0; g < n_groups; g++) {
            const uint64_t n = n_elems_of(g), t = tiles[g];
            if (n == 0) continue;
            const double full = item_time(g, std::min<uint64_t>(t, n));
            total += (double)(n / t) * item_time(g, t) + (n % t ? item_time(g, n % t) : 0.0);
            longest = std::max(longest, full);
        }
        return std::max(total / sm_count, longest);
    };
    double best = makespan();
    for (int round = 0; round < 2; round++)
        for (size_t g = 0; g < n_groups; g++) {
            const uint32_t keep = tiles[g];
            uint32_t pick = keep;
            for (uint32_t t = max_tile_of(g); t >= 1; t--) {
                tiles[g] = t;
                if (lower_bound() > best * (1.0 + 1e-9)) continue;
                const double m = makespan();
                // on a tie the wider tile: fewer items leave more of the wave to the other groups
                if (m < best * (1.0 - 1e-9) || (m <= best * (1.0 + 1e-9) && t > pick)) { best = std::min(best, m); pick = t; }
            }
            tiles[g] = pick;
        }
}

// Item-time models (arbitrary units; only their ratios matter).
//  k_filter: one thread per element, so the time follows the cost of the group's walks
//  times the width rounded up to whole warps, but never less than for 64 elements: below
//  about two warps per SM the walks' own latency, not the shared-memory pipe, sets it.
//  k_filter_wp: one thread per walk (two per DCF walk); per predicate of n bits a fixed
//  cost (the key staging, the walk chain of one PRG call per level, the combine: about
//  656 n ns for EQ, 719 n ns for RANGE on GB300) plus a per-element term (20 n / 54 n ns:
//  the shared-memory lookups of an EQ / RANGE element).  Fitted to sweeps of tiles of 1..40
//  elements, one and two items per SM, n = 16 and 32.
struct GroupCost {
    uint64_t walk_cost = 0;            // k_filter: sum over predicates of 6 n (EQ) / 24 n (RANGE)
    uint64_t wp_lat = 0, wp_slope = 0; // k_filter_wp: latency and per-element terms, ns
};

double filter_item_time(const GroupCost& c, uint64_t width) {
    const uint64_t busy = std::max<uint64_t>((width + 31) / 32 * 32, 64);
    return (double)c.walk_cost * (double)busy;
}

double wp_item_time(const GroupCost& c, uint64_t width) {
    return (double)c.wp_lat + (double)c.wp_slope * (double)width;
}

oblivgm_status plan_queries(const std::map<uint32_t, Table>& tables, uint32_t n_queries, const uint32_t* query_ids,
                            const ParsedQuery* parsed, const uint32_t* n_groups, uint32_t* const* const* outs,
                            uint32_t tile, uint32_t step, bool wp, int sm_count, Plan* plan) {
    struct G { GroupDesc d; std::vector<const ParsedPred*> preds; GroupCost cost; };
    std::vector<G> all;
    for (uint32_t q = 0; q < n_queries; q++) {
        const ParsedQuery& pq = parsed[q];
        const uint32_t ng = n_groups[q];
        if (pq.out_group != 0) return fail(OBLIVGM_EINVAL, "a one-hot token was given to the masked-mode evaluation");
        if (ng == 0 || ng > OBLIVGM_MAX_GROUPS) return fail(OBLIVGM_EINVAL, "n_groups must be 1..64");
        std::vector<std::vector<const ParsedPred*>> members(ng);
        for (const ParsedPred& p : pq.preds) {
            if (p.group >= ng) return fail(OBLIVGM_EINVAL, "predicate group outside 0..n_groups-1");
            members[p.group].push_back(&p);
        }
        for (uint32_t g = 0; g < ng; g++) {
            if (members[g].empty()) return fail(OBLIVGM_EINVAL, "an AND-group has no predicate");
            const uint32_t tid = members[g][0]->table;
            auto it = tables.find(tid);
            if (it == tables.end()) return fail(OBLIVGM_ENOENT, "predicate on a table that is not loaded");
            const Table& tb = it->second;
            GroupCost cost;
            for (const ParsedPred* p : members[g]) {
                if (p->table != tid) return fail(OBLIVGM_EINVAL, "an AND-group spans two tables");
                if (p->attr >= tb.n_attrs) return fail(OBLIVGM_EINVAL, "predicate attribute outside its table");
                if (p->n != tb.n_bits) return fail(OBLIVGM_EINVAL, "predicate bit length differs from its table's");
                const bool eq = p->kind == OBLIVGM_PRED_EQ;
                cost.walk_cost += (eq ? 6ull : 24ull) * p->n;
                cost.wp_lat += (eq ? 656ull : 719ull) * p->n;
                cost.wp_slope += (eq ? 20ull : 54ull) * p->n;
            }
            G gr{};
            for (int j = 0; j < 3; j++) {
                gr.d.share[j] = tb.dev + (uint64_t)j * tb.n_attrs * tb.stride;
                gr.d.out[j] = outs[q][3 * g + j];
                if (!gr.d.out[j] && tb.n_elems) return fail(OBLIVGM_EINVAL, "NULL output pointer");
            }
            gr.d.vec_out = 1;
            for (int j = 0; j < 3; j++)
                if (reinterpret_cast<uintptr_t>(gr.d.out[j]) % 16) gr.d.vec_out = 0;
            gr.d.stride = tb.stride;
            gr.d.n_elems = tb.n_elems;
            // a group of equality predicates only needs 6 walk threads per element (k_filter_wp)
            gr.d.slots = (uint32_t)kWpSlots;
            bool all_eq = true;
            for (const ParsedPred* p : members[g]) all_eq = all_eq && p->kind == OBLIVGM_PRED_EQ;
            if (all_eq) gr.d.slots = (uint32_t)kWpEqSlots;
            gr.d.query_id = query_ids[q];
            gr.d.table_id = tid;
            gr.preds = members[g];
            gr.cost = cost;
            all.push_back(std::move(gr));
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const G& a, const G& b) { return a.cost.walk_cost > b.cost.walk_cost; });
    const uint32_t max_tile = tile;
    const auto n_of = [&](size_t i) { return all[i].d.n_elems; };
    const auto time_of = [&](size_t i, uint64_t w) {
        return wp ? wp_item_time(all[i].cost, w) : filter_item_time(all[i].cost, w);
    };
    tile = choose_tile(all.size(), n_of, time_of, max_tile, step, sm_count);
    std::vector<uint32_t> tiles(all.size(), tile);
    if (wp && step != 0 && all.size() > 1 && all.size() <= kWpTileGroups) {
        uint64_t items_at_max = 0;
        for (const G& g : all) items_at_max += (g.d.n_elems + max_tile - 1) / max_tile;
        if (items_at_max <= 4ull * (uint64_t)sm_count)
            choose_group_tiles(all.size(), n_of, time_of,
                               [&](size_t i) { return all[i].d.slots == (uint32_t)kWpEqSlots ? (uint32_t)kWpEqElems : max_tile; },
                               sm_count, tiles);
    }
    plan->groups.clear(); plan->preds.clear(); plan->keys.clear(); plan->item_start.clear();
    plan->tile = *std::max_element(tiles.begin(), tiles.end());
    uint64_t items = 0;
    for (size_t gi = 0; gi < all.size(); gi++) {
        G& g = all[gi];
        g.d.tile = tiles[gi];
        g.d.pred_begin = (uint32_t)plan->preds.size();
        g.d.n_preds = (uint32_t)g.preds.size();
        for (const ParsedPred* p : g.preds) {
            PredDesc d{};
            d.kind = p->kind; d.n_bits = p->n; d.attr = p->attr; d.step = p->step;
            for (int i = 0; i < 3; i++) d.r[i] = p->r[i];
            d.cbeta = p->cbeta;
            combine_coeffs(p->combine, &d.lin, &d.prod);
            d.key_begin = (uint32_t)plan->keys.size();
            d.n_keys = (uint32_t)p->keys.size();
            plan->keys.insert(plan->keys.end(), p->keys.begin(), p->keys.end());
            plan->preds.push_back(d);
        }
        plan->groups.push_back(g.d);
        plan->item_start.push_back(items);
        items += (g.d.n_elems + g.d.tile - 1) / g.d.tile;
    }
    plan->item_start.push_back(items);
    return OBLIVGM_OK;
}

// Plan a batch for the fused kernel in the context's launch shape; a batch whose groups
// hold at most ctx->wp_max_elems elements in all goes to the walk-parallel kernel instead,
// in tiles of kWpElems elements.
oblivgm_status plan_filter(oblivgm_ctx* ctx, const std::map<uint32_t, Table>& tables, uint32_t n_queries,
                           const uint32_t* query_ids, const ParsedQuery* parsed, const uint32_t* n_groups,
                           uint32_t* const* const* outs, Plan* plan) {
    const uint32_t threads = ctx->threads, E = ctx->elems_per_thread;
    plan->elems_per_thread = E;
    plan->threads = threads;
    plan->wp = false;
    oblivgm_status s = plan_queries(tables, n_queries, query_ids, parsed, n_groups, outs, threads * E, 32 * E,
                                    false, ctx->sm_count, plan);
    if (s != OBLIVGM_OK) return s;
    uint64_t total = 0;
    for (const GroupDesc& g : plan->groups) total += g.n_elems;
    if (total == 0 || total > ctx->wp_max_elems) return OBLIVGM_OK;
    // a forced tile (oblivgm_set_walk_parallel_tile) skips the search: step 0
    s = plan_queries(tables, n_queries, query_ids, parsed, n_groups, outs, ctx->wp_tile ? ctx->wp_tile : kWpElems,
                     ctx->wp_tile ? 0 : 1, true, ctx->sm_count, plan);
    if (s != OBLIVGM_OK) return s;
    plan->wp = true;
    plan->threads = kWpThreads;
    plan->elems_per_thread = 1;
    return OBLIVGM_OK;
}

// One launch of the planned kernel: grid = min(work items, SMs), one persistent CTA per SM.
cudaError_t launch_filter_kernel(const FilterParams& P, uint64_t n_items, int sm_count, uint32_t threads, uint32_t E,
                                 bool wp, cudaStream_t st) {
    const unsigned grid = (unsigned)std::min<uint64_t>(n_items, (uint64_t)sm_count);
    if (wp) {
        k_filter_wp<<<grid, kWpThreads, kWpSmem, st>>>(P);
    } else {
        switch (E) {
            case 1: k_filter<1><<<grid, threads, kFilterSmem, st>>>(P); break;
            case 2: k_filter<2><<<grid, threads, kFilterSmem, st>>>(P); break;
            default: k_filter<4><<<grid, threads, kFilterSmem, st>>>(P); break;
        }
    }
    return cudaGetLastError();
}

// Device workspace of one fused launch: work counter (and the walk-parallel kernel's count
// of finished CTAs at byte 8) | groups | preds | keys | tile offsets, each part 256-byte
// aligned.  The image is built on the host; its first 256 bytes are zero.
struct WsImage {
    size_t off_groups = 0, off_preds = 0, off_keys = 0, off_items = 0, total = 0;
    std::vector<unsigned char> bytes;
};

WsImage build_ws_image(const Plan& plan) {
    WsImage im;
    im.off_groups = 256;
    im.off_preds = im.off_groups + (plan.groups.size() * sizeof(GroupDesc) + 255) / 256 * 256;
    im.off_keys = im.off_preds + (plan.preds.size() * sizeof(PredDesc) + 255) / 256 * 256;
    im.off_items = im.off_keys + (plan.keys.size() * sizeof(DevKey) + 255) / 256 * 256;
    im.total = (im.off_items + plan.item_start.size() * sizeof(uint64_t) + 255) / 256 * 256;
    im.bytes.assign(im.total, 0);
    std::memcpy(im.bytes.data() + im.off_groups, plan.groups.data(), plan.groups.size() * sizeof(GroupDesc));
    std::memcpy(im.bytes.data() + im.off_preds, plan.preds.data(), plan.preds.size() * sizeof(PredDesc));
    std::memcpy(im.bytes.data() + im.off_keys, plan.keys.data(), plan.keys.size() * sizeof(DevKey));
    std::memcpy(im.bytes.data() + im.off_items, plan.item_start.data(), plan.item_start.size() * sizeof(uint64_t));
    return im;
}

// Fused-kernel parameters of a plan whose workspace image lives at device address `ws`.
FilterParams filter_params(const oblivgm_ctx* ctx, const Plan& plan, const WsImage& im, unsigned char* ws,
                           uint32_t* error_flag) {
    FilterParams P{};
    P.aes = ctx->aes;
    std::memcpy(P.rk_prf, ctx->rk_prf, sizeof P.rk_prf);
    P.te0 = ctx->d_te0;
    P.groups = reinterpret_cast<const GroupDesc*>(ws + im.off_groups);
    P.preds = reinterpret_cast<const PredDesc*>(ws + im.off_preds);
    P.keys = reinterpret_cast<const DevKey*>(ws + im.off_keys);
    P.item_start = reinterpret_cast<const uint64_t*>(ws + im.off_items);
    P.counter = reinterpret_cast<unsigned long long*>(ws);
    P.done = reinterpret_cast<uint32_t*>(ws + 8);
    P.error = error_flag;
    P.n_groups = (uint32_t)plan.groups.size();
    P.tile = plan.tile;
    P.wait_limit_ns = kWaitLimitNs;
    // the walk-parallel kernel keeps a small launch's workspace (from the groups on) in its
    // shared memory; the image is padded to 256 bytes, so the copy stays inside it
    const size_t res = im.total - im.off_groups;
    P.resident_bytes = plan.wp && res <= (size_t)kWpResidentBytes ? (uint32_t)res : 0u;
    return P;
}

// one-shot failure-path test (oblivgm_test_expire_next_wait): the next launch's first key
// staging expects 16 bytes more than it gets, under a short wait bound
void apply_test_expiry(oblivgm_ctx* ctx, FilterParams* P) {
    if (!ctx->test_expire_next) return;
    P->expect_extra = 16;
    P->wait_limit_ns = ctx->test_wait_limit_ns;
    ctx->test_expire_next = false;
}

oblivgm_status launch_plan(oblivgm_ctx* ctx, const Plan& plan, cudaStream_t st, uint32_t* error_flag) {
    if (plan.item_start.back() == 0) return OBLIVGM_OK;   // nothing to evaluate
    const WsImage im = build_ws_image(plan);
    unsigned char* ws = nullptr;
    oblivgm_status as = ws_alloc(ctx, reinterpret_cast<void**>(&ws), im.total, st, "workspace allocation");
    if (as != OBLIVGM_OK) return as;
    ScratchGuard guard(ws, st);
    OGM_CUDA(cudaMemcpyAsync(ws, im.bytes.data(), im.total, cudaMemcpyHostToDevice, st), "descriptor upload");
    FilterParams P = filter_params(ctx, plan, im, ws, error_flag);
    apply_test_expiry(ctx, &P);
    const cudaError_t e = launch_filter_kernel(P, plan.item_start.back(), ctx->sm_count, plan.threads,
                                               plan.elems_per_thread, plan.wp, st);
    if (e != cudaSuccess) return cuda_fail(e, "k_filter launch");
    ctx->launches++;
    guard.done();
    OGM_CUDA(cudaFreeAsync(ws, st), "workspace release");
    return OBLIVGM_OK;
}

oblivgm_status launch_parsed(oblivgm_ctx* ctx, uint32_t n_queries, const uint32_t* query_ids,
                             const ParsedQuery* parsed, const uint32_t* n_groups, uint32_t* const* const* outs,
                             const std::map<uint32_t, Table>& tables, cudaStream_t st) {
    Plan plan;
    oblivgm_status s = plan_filter(ctx, tables, n_queries, query_ids, parsed, n_groups, outs, &plan);
    if (s != OBLIVGM_OK) return s;
    return launch_plan(ctx, plan, st, ctx->d_error);
}

oblivgm_status set_filter_attrs() {
    OGM_CUDA(cudaFuncSetAttribute(k_filter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFilterSmem), "smem attr");
    OGM_CUDA(cudaFuncSetAttribute(k_filter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFilterSmem), "smem attr");
    OGM_CUDA(cudaFuncSetAttribute(k_filter<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFilterSmem), "smem attr");
    OGM_CUDA(cudaFuncSetAttribute(k_filter_wp, cudaFuncAttributeMaxDynamicSharedMemorySize, kWpSmem), "smem attr");
    OGM_CUDA(cudaFuncSetAttribute(k_eval_raw<OBLIVGM_KEY_DPF>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes), "smem attr");
    OGM_CUDA(cudaFuncSetAttribute(k_eval_raw<OBLIVGM_KEY_DCF>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTableBytes), "smem attr");
    return OBLIVGM_OK;
}

}  // namespace ogm

// ====================================================================== C ABI

extern "C" {

uint32_t oblivgm_version(void) { return 0x000100u; }

oblivgm_status oblivgm_last_error(char* buf, size_t n) {
    if (!buf || n == 0) return OBLIVGM_EINVAL;
    std::snprintf(buf, n, "%s", g_last_error.c_str());
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_create(oblivgm_ctx** out, int32_t device, const oblivgm_config* cfg) {
    if (!out || !cfg) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (cfg->flags != 0) return fail(OBLIVGM_EINVAL, "config flags must be 0");
    *out = nullptr;
    int count = 0;
    OGM_CUDA(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(OBLIVGM_EINVAL, "no such CUDA device");
    cudaDeviceProp prop;
    OGM_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3) return fail(OBLIVGM_EARCH, "this library is built for sm_103 (GB300) only");
    OGM_CUDA(cudaSetDevice(device), "cudaSetDevice");
    auto* ctx = new (std::nothrow) oblivgm_ctx();
    if (!ctx) return fail(OBLIVGM_ENOMEM, "host allocation");
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    ctx->wp_max_elems = (uint64_t)ctx->sm_count * kWpDefaultElemsPerSm;
    build_aes_params(&ctx->aes);
    for (int i = 0; i < 3; i++) {
        const RoundKeys rk = expand_key(cfg->prf_keys[i]);
        std::memcpy(ctx->rk_prf[i], rk.w, sizeof rk.w);
    }
    ctx->cfg = *cfg;
    oblivgm_status st = set_filter_attrs();
    if (st == OBLIVGM_OK) st = set_onehot_attrs();
    if (st == OBLIVGM_OK) st = set_keygen_attrs();
    if (st == OBLIVGM_OK) st = set_fresh_attrs();
    if (st == OBLIVGM_OK) st = set_shuffle_attrs();
    if (st == OBLIVGM_OK) st = set_prg_attrs();
    if (st != OBLIVGM_OK) { delete ctx; return st; }
    cudaError_t e = cudaMalloc(&ctx->d_te0, 256 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_te0, aes_tables().te0, 256 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_te4, 4 * 256 * sizeof(uint32_t));
    if (e == cudaSuccess) {
        uint32_t te4[4 * 256];
        for (int k = 0; k < 4; k++)
            for (int x = 0; x < 256; x++) {
                const uint32_t v = aes_tables().te0[x];
                te4[k * 256 + x] = k ? (v << (8 * k)) | (v >> (32 - 8 * k)) : v;
            }
        e = cudaMemcpy(ctx->d_te4, te4, sizeof te4, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_error, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_error, 0, sizeof(uint32_t));
    if (e == cudaSuccess) {
        cudaMemPool_t pool;
        e = cudaDeviceGetDefaultMemPool(&pool, device);
        uint64_t keep = UINT64_MAX;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        st = cuda_fail(e, "context set-up");
        oblivgm_destroy(ctx);
        return st;
    }
    st = serve_init(ctx);
    if (st != OBLIVGM_OK) { oblivgm_destroy(ctx); return st; }
    *out = ctx;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_destroy(oblivgm_ctx* ctx) {
    if (!ctx) return OBLIVGM_OK;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->tables) cudaFree(kv.second.dev);
    for (auto& kv : ctx->onehot_tables) cudaFree(kv.second.dev);
    if (ctx->d_te0) cudaFree(ctx->d_te0);
    if (ctx->d_te4) cudaFree(ctx->d_te4);
    if (ctx->d_error) cudaFree(ctx->d_error);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    delete ctx;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_sync(oblivgm_ctx* ctx, void* stream) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    OGM_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream synchronize");
    uint32_t flag = 0;
    OGM_CUDA(cudaMemcpy(&flag, ctx->d_error, sizeof flag, cudaMemcpyDeviceToHost), "read fault flag");
    if (flag) {
        cudaMemset(ctx->d_error, 0, sizeof flag);
        return fail(OBLIVGM_EFAULT_DEVICE, (flag & 1u) ? "a bounded device wait expired (key staging)"
                                                       : "a device-resident key had a malformed header");
    }
    return OBLIVGM_OK;
}

uint64_t oblivgm_launch_count(oblivgm_ctx* ctx) { return ctx ? ctx->launches.load() : 0ull; }

oblivgm_status oblivgm_load_shares(oblivgm_ctx* ctx, uint32_t table_id, uint64_t n_elems, uint32_t n_attrs,
                                   uint32_t n_bits, const uint32_t* const share_sets[3], int32_t mem_kind,
                                   void* stream) {
    const NvtxRange nvtx_range("oblivgm_load_shares");
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (table_id > 0xFFFF || n_attrs == 0 || n_attrs > 65536 || n_bits < 1 || n_bits > 32 || !share_sets)
        return fail(OBLIVGM_EINVAL, "bad table arguments");
    if (mem_kind != OBLIVGM_MEM_HOST && mem_kind != OBLIVGM_MEM_DEVICE) return fail(OBLIVGM_EINVAL, "bad mem_kind");
    for (int j = 0; j < 3; j++)
        if (!share_sets[j] && n_elems) return fail(OBLIVGM_EINVAL, "NULL share set");
    if (table_in_use(ctx, table_id)) return fail(OBLIVGM_EBUSY, "table is used by in-flight queries");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t stride = (n_elems + 3) / 4 * 4;
    const size_t row_bytes = stride * sizeof(uint32_t);
    const size_t bytes = 3ull * n_attrs * row_bytes;
    Table tb{};
    tb.n_elems = n_elems; tb.stride = stride; tb.n_attrs = n_attrs; tb.n_bits = n_bits;
    auto it = ctx->tables.find(table_id);
    if (it != ctx->tables.end() && it->second.bytes == bytes) {
        tb.dev = it->second.dev;   // same shape: reuse the allocation
        tb.bytes = bytes;
    } else {
        if (it != ctx->tables.end()) {
            OGM_CUDA(cudaStreamSynchronize(s), "stream synchronize");
            cudaFree(it->second.dev);
            ctx->tables.erase(it);
        }
        OGM_CUDA(cudaMalloc(&tb.dev, std::max<size_t>(bytes, 16)), "table allocation");
        tb.bytes = bytes;
    }
    ctx->tables[table_id] = tb;
    if (n_elems == 0) return OBLIVGM_OK;
    const size_t src_row = n_elems * sizeof(uint32_t);
    const cudaMemcpyKind kind = mem_kind == OBLIVGM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int j = 0; j < 3; j++) {
        // one 2-D copy per share set: n_attrs rows of n_elems words into rows of `stride` words
        OGM_CUDA(cudaMemcpy2DAsync(tb.dev + (uint64_t)j * n_attrs * stride, row_bytes, share_sets[j], src_row, src_row,
                                   n_attrs, kind, s),
                 "share upload");
    }
    if (mem_kind == OBLIVGM_MEM_HOST) {
        // pageable host sources are staged by the driver before the call returns only for
        // small copies; synchronise so the caller may reuse its buffers at once
        OGM_CUDA(cudaStreamSynchronize(s), "stream synchronize");
    }
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_unload_shares(oblivgm_ctx* ctx, uint32_t table_id) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->tables.find(table_id);
    if (it == ctx->tables.end()) return fail(OBLIVGM_ENOENT, "no such table");
    if (table_in_use(ctx, table_id)) return fail(OBLIVGM_EBUSY, "table is used by in-flight queries");
    cudaDeviceSynchronize();
    cudaFree(it->second.dev);
    ctx->tables.erase(it);
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_keygen(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits, const uint8_t seed[16],
                              uint8_t* const tok[3], size_t cap, size_t out_len[3]) {
    std::string err;
    oblivgm_status st = keygen(preds, n_preds, n_bits, seed, tok, cap, out_len, &err);
    if (st != OBLIVGM_OK) return fail(st, err);
    return OBLIVGM_OK;
}

static oblivgm_status eval_batch(oblivgm_ctx* ctx, uint32_t kind, const uint8_t* keys, uint32_t n_keys,
                                 const uint32_t* points, const uint32_t* key_of_point, uint64_t n_points,
                                 uint32_t flags, uint32_t* out, uint64_t n_out, void* stream) {
    const NvtxRange nvtx_range(kind == OBLIVGM_KEY_DPF ? "oblivgm_eval_dpf_batch" : "oblivgm_eval_dcf_batch");
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (!keys || n_keys == 0 || (n_points && (!points || !out))) return fail(OBLIVGM_EINVAL, "NULL or empty argument");
    const bool all = (flags & OBLIVGM_ALL_PAIRS) != 0;
    const bool dev_keys = (flags & OBLIVGM_KEYS_DEVICE) != 0;
    if (flags & ~(OBLIVGM_ALL_PAIRS | OBLIVGM_KEYS_DEVICE | 0xFF00u)) return fail(OBLIVGM_EINVAL, "unknown flags");
    if (!dev_keys && (flags & 0xFF00u)) return fail(OBLIVGM_EINVAL, "key bit length in flags needs OBLIVGM_KEYS_DEVICE");
    if (!all && n_points && !key_of_point) return fail(OBLIVGM_EINVAL, "key_of_point is NULL");
    if (all && n_keys > 65535) return fail(OBLIVGM_EINVAL, "ALL_PAIRS takes at most 65535 keys");
    const uint64_t need = all ? (uint64_t)n_keys * n_points : n_points;
    if (n_out < need) return fail(OBLIVGM_ERANGE, "output buffer too small");
    const int n = dev_keys ? (int)((flags >> 8) & 0xFFu) : keys[1];
    if (n < 1 || n > kMaxBits) return fail(OBLIVGM_EINVAL, "bad key bit length");
    if (n_points == 0) return OBLIVGM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevKey* d_keys = nullptr;
    st = ws_alloc(ctx, reinterpret_cast<void**>(&d_keys), (size_t)n_keys * sizeof(DevKey), s, "key buffer");
    if (st != OBLIVGM_OK) return st;
    ScratchGuard guard(d_keys, s);
    if (dev_keys) {
        st = repack_keys_device(ctx, keys, kind, (uint32_t)n, n_keys, d_keys, s);
        if (st != OBLIVGM_OK) return st;
    } else {
        const size_t klen = key_bytes(kind, n);
        std::vector<DevKey> dk(n_keys);
        std::string err;
        for (uint32_t k = 0; k < n_keys; k++)
            if (!repack_key(keys + (size_t)k * klen, klen, kind, n, &dk[k], &err)) return fail(OBLIVGM_EINVAL, err);
        OGM_CUDA(cudaMemcpyAsync(d_keys, dk.data(), dk.size() * sizeof(DevKey), cudaMemcpyHostToDevice, s), "key upload");
    }
    RawParams P{};
    P.aes = ctx->aes;
    P.te0 = ctx->d_te0;
    P.keys = d_keys;
    P.points = points;
    P.key_of_point = key_of_point;
    P.out = out;
    P.n_points = n_points;
    P.n_keys = n_keys;
    P.all_pairs = all ? 1u : 0u;
    const uint64_t blocks = (n_points + 255) / 256;
    if (blocks > 0x7FFFFFFFull) return fail(OBLIVGM_EINVAL, "too many points");
    dim3 grid((unsigned)blocks, all ? n_keys : 1);
    if (kind == OBLIVGM_KEY_DPF) k_eval_raw<OBLIVGM_KEY_DPF><<<grid, 256, kTableBytes, s>>>(P);
    else k_eval_raw<OBLIVGM_KEY_DCF><<<grid, 256, kTableBytes, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_eval_raw launch");
    ctx->launches++;
    guard.done();
    OGM_CUDA(cudaFreeAsync(d_keys, s), "key buffer release");
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_eval_dpf_batch(oblivgm_ctx* ctx, const uint8_t* keys, uint32_t n_keys, const uint32_t* points,
                                      const uint32_t* key_of_point, uint64_t n_points, uint32_t flags, uint32_t* out,
                                      uint64_t n_out, void* stream) {
    return eval_batch(ctx, OBLIVGM_KEY_DPF, keys, n_keys, points, key_of_point, n_points, flags, out, n_out, stream);
}

oblivgm_status oblivgm_eval_dcf_batch(oblivgm_ctx* ctx, const uint8_t* keys, uint32_t n_keys, const uint32_t* points,
                                      const uint32_t* key_of_point, uint64_t n_points, uint32_t flags, uint32_t* out,
                                      uint64_t n_out, void* stream) {
    return eval_batch(ctx, OBLIVGM_KEY_DCF, keys, n_keys, points, key_of_point, n_points, flags, out, n_out, stream);
}

oblivgm_status oblivgm_filter_batch(oblivgm_ctx* ctx, uint32_t n_queries, const uint32_t* query_ids,
                                    const uint8_t* const* toks, const size_t* tok_lens, const uint32_t* n_groups,
                                    uint32_t* const* const* outs, void* stream) {
    const NvtxRange nvtx_range("oblivgm_filter_batch");
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (n_queries == 0) return OBLIVGM_OK;
    if (!query_ids || !toks || !tok_lens || !n_groups || !outs) return fail(OBLIVGM_EINVAL, "NULL argument");
    std::vector<ParsedQuery> parsed(n_queries);
    std::string err;
    for (uint32_t q = 0; q < n_queries; q++) {
        if (!outs[q]) return fail(OBLIVGM_EINVAL, "NULL output array");
        st = parse_tokens(toks + 3 * q, tok_lens + 3 * q, &parsed[q], &err);
        if (st != OBLIVGM_OK) return fail(st, err);
    }
    return launch_parsed(ctx, n_queries, query_ids, parsed.data(), n_groups, outs, ctx->tables,
                         static_cast<cudaStream_t>(stream));
}

oblivgm_status oblivgm_filter_and_combine(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                          const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out,
                                          void* stream) {
    const NvtxRange nvtx_range("oblivgm_filter_and_combine");
    if (!tok || !tok_len || !out) return fail(OBLIVGM_EINVAL, "NULL argument");
    const uint8_t* toks[3] = {tok[0], tok[1], tok[2]};
    uint32_t* const* outs[1] = {out};
    return oblivgm_filter_batch(ctx, 1, &query_id, toks, tok_len, &n_groups, outs, stream);
}

oblivgm_status oblivgm_autotune(oblivgm_ctx* ctx, uint32_t* threads, uint32_t* elems_per_thread) {
    const NvtxRange nvtx_range("oblivgm_autotune");
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    // synthetic private table: 2^20 elements (every candidate shape gets at least one tile
    // per SM), one 32-bit attribute, one equality and one range predicate ANDed, so both
    // walk kinds and the fold are in the timing
    const uint64_t n = 1ull << 20;
    std::vector<uint32_t> h(n);
    uint32_t x = 0x9E3779B9u;
    for (auto& v : h) { x ^= x << 13; x ^= x >> 17; x ^= x << 5; v = x; }
    std::map<uint32_t, Table> tabs;
    Table tb{};
    tb.n_elems = n; tb.stride = n; tb.n_attrs = 1; tb.n_bits = 32; tb.bytes = 3 * n * 4;
    OGM_CUDA(cudaMalloc(&tb.dev, tb.bytes + 3 * n * 4), "autotune buffers");
    for (int j = 0; j < 3; j++)
        cudaMemcpy(tb.dev + j * n, h.data(), n * 4, cudaMemcpyHostToDevice);
    tabs[0] = tb;
    uint32_t* outp = tb.dev + 3 * n;
    uint32_t* outs3[3] = {outp, outp, outp};   // timing only: the three sets may overlap
    oblivgm_pred preds[2] = {{OBLIVGM_PRED_EQ, 0, 0, 0, 12345u, 0, OBLIVGM_COMBINE_AND},
                             {OBLIVGM_PRED_RANGE, 0, 0, 0, 1000u, 0x7FFFFFFFu, OBLIVGM_COMBINE_AND}};
    uint8_t seed[16] = {0};
    size_t len[3];
    std::string err;
    keygen(preds, 2, 32, seed, nullptr, 0, len, &err);
    std::vector<uint8_t> t0(len[0]), t1(len[1]), t2(len[2]);
    uint8_t* tk[3] = {t0.data(), t1.data(), t2.data()};
    keygen(preds, 2, 32, seed, tk, len[0], len, &err);
    const uint8_t* ctk[3] = {tk[0], tk[1], tk[2]};
    ParsedQuery pq;
    parse_tokens(ctk, len, &pq, &err);
    const uint32_t qid = 1, ng = 1;
    uint32_t* const* outs[1] = {outs3};
    struct Cand { uint32_t t, e; };
    const Cand cands[] = {{1024, 1}, {768, 1}, {512, 1}, {512, 2}, {256, 2}, {512, 4}, {256, 4}, {128, 4}};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const uint32_t keep_t = ctx->threads, keep_e = ctx->elems_per_thread;
    float best = 1e30f;
    Cand win{keep_t, keep_e};
    for (const Cand& c : cands) {
        ctx->threads = c.t;
        ctx->elems_per_thread = c.e;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(a, 0);
            st = launch_parsed(ctx, 1, &qid, &pq, &ng, outs, tabs, 0);
            cudaEventRecord(b, 0);
            if (st != OBLIVGM_OK) break;
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) ms_best = std::min(ms_best, ms);
        }
        if (st != OBLIVGM_OK) break;
        if (ms_best < best) { best = ms_best; win = c; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaDeviceSynchronize();
    cudaFree(tb.dev);
    if (st != OBLIVGM_OK) {
        ctx->threads = keep_t;
        ctx->elems_per_thread = keep_e;
        return st;
    }
    ctx->threads = win.t;
    ctx->elems_per_thread = win.e;
    if (threads) *threads = win.t;
    if (elems_per_thread) *elems_per_thread = win.e;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_test_fail_next_alloc(oblivgm_ctx* ctx) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    ctx->test_fail_alloc = true;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_test_expire_next_wait(oblivgm_ctx* ctx, uint32_t limit_us) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (limit_us == 0 || limit_us > 2000000) return fail(OBLIVGM_EINVAL, "limit must be 1..2000000 us");
    ctx->test_wait_limit_ns = (uint64_t)limit_us * 1000ull;
    ctx->test_expire_next = true;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_set_schedule(oblivgm_ctx* ctx, uint32_t threads, uint32_t elems_per_thread) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    const uint32_t t = threads ? threads : ctx->threads;
    const uint32_t e = elems_per_thread ? elems_per_thread : ctx->elems_per_thread;
    if (e != 1 && e != 2 && e != 4) return fail(OBLIVGM_EINVAL, "elems_per_thread must be 1, 2 or 4");
    const uint32_t tmax = e == 1 ? max_threads<1>() : max_threads<4>();
    if (t % 32 || t < 32 || t > tmax) return fail(OBLIVGM_EINVAL, "threads must be a multiple of 32, at most 1024 (E = 1) or 512 (E = 2, 4)");
    ctx->threads = t;
    ctx->elems_per_thread = e;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_set_walk_parallel_tile(oblivgm_ctx* ctx, uint32_t tile, uint32_t* previous) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (tile > (uint32_t)kWpElems) return fail(OBLIVGM_EINVAL, "the walk-parallel tile is at most 40 elements");
    if (previous) *previous = ctx->wp_tile;
    ctx->wp_tile = tile;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_set_walk_parallel(oblivgm_ctx* ctx, uint64_t max_elems, uint64_t* previous) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (previous) *previous = ctx->wp_max_elems;
    ctx->wp_max_elems = max_elems;
    return OBLIVGM_OK;
}

}  // extern "C"

// ====================================================================== no-allocation variant
//
// oblivgm_filter_and_combine_noalloc runs the same fused kernel as
// oblivgm_filter_and_combine, but its per-call workspace (work-queue counter,
// group and predicate descriptors, device keys, tile offsets) lives in the
// fixed device array below instead of memory obtained with cudaMallocAsync.
// It is for callers that must not allocate device memory at call time.  The
// array is part of the loaded module: every GPU that loads this library holds
// OBLIVGM_NOALLOC_SCRATCH_BYTES of it until the process exits.

namespace ogm {

static __device__ __align__(256) unsigned char g_noalloc_scratch[OBLIVGM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the host-side name of a __device__
// array is only a stand-in, so ask the runtime for the array's device address.
oblivgm_status scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return fail(OBLIVGM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[device]);
    return OBLIVGM_OK;
}

}  // namespace
}  // namespace ogm

extern "C" oblivgm_status oblivgm_filter_and_combine_noalloc(oblivgm_ctx* ctx, uint32_t query_id,
                                                             const uint8_t* const tok[3], const size_t tok_len[3],
                                                             uint32_t n_groups, uint32_t* const* out, void* stream) {
    const NvtxRange nvtx_range("oblivgm_filter_and_combine_noalloc");
    oblivgm_status st = check_ctx(ctx);   // also makes the context's device current
    if (st) return st;
    if (!tok || !tok_len || !out) return fail(OBLIVGM_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The workspace upload reads a host buffer that lives only for this call, so a graph
    // replay of a captured call would copy freed memory: refuse a capturing stream.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce == cudaErrorStreamCaptureImplicit) {   // the legacy stream while another stream captures
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    } else if (ce != cudaSuccess) {
        return cuda_fail(ce, "cudaStreamIsCapturing");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return fail(OBLIVGM_EINVAL, "the no-alloc entry point must not be called on a stream under capture");
    ParsedQuery parsed;
    std::string err;
    st = parse_tokens(tok, tok_len, &parsed, &err);
    if (st != OBLIVGM_OK) return fail(st, err);
    uint32_t* const* outs[1] = {out};
    Plan plan;
    st = plan_filter(ctx, ctx->tables, 1, &query_id, &parsed, &n_groups, outs, &plan);
    if (st != OBLIVGM_OK) return st;
    if (plan.item_start.back() == 0) return OBLIVGM_OK;
    const WsImage im = build_ws_image(plan);
    if (im.total > OBLIVGM_NOALLOC_SCRATCH_BYTES)
        return fail(OBLIVGM_ERANGE, "query needs " + std::to_string(im.total) +
                                        " workspace bytes; the no-alloc entry point holds " +
                                        std::to_string(OBLIVGM_NOALLOC_SCRATCH_BYTES));
    unsigned char* ws = nullptr;
    st = scratch_address(ctx->device, &ws);
    if (st != OBLIVGM_OK) return st;
    OGM_CUDA(cudaMemcpyAsync(ws, im.bytes.data(), im.total, cudaMemcpyHostToDevice, s), "no-alloc workspace upload");
    FilterParams P = filter_params(ctx, plan, im, ws, ctx->d_error);
    apply_test_expiry(ctx, &P);
    const cudaError_t e = launch_filter_kernel(P, plan.item_start.back(), ctx->sm_count, plan.threads,
                                               plan.elems_per_thread, plan.wp, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_filter launch (no-alloc)");
    ctx->launches++;
    return OBLIVGM_OK;
}

// ====================================================================== prepared plans (CUDA-graph capture)
//
// A plan holds a batch's descriptors and device keys in its own device buffer, so
// launching it is only a counter reset and one kernel launch: no host work, no
// allocation and no pageable copies, which is what stream capture into a CUDA graph
// needs.  Replaying the plan recomputes the same shares into the same outputs.

struct oblivgm_plan {
    oblivgm_ctx* ctx = nullptr;
    unsigned char* ws = nullptr;
    FilterParams params{};
    uint32_t threads = 0, E = 1;
    bool wp = false;
    uint64_t n_items = 0;
};

extern "C" oblivgm_status oblivgm_plan_create(oblivgm_ctx* ctx, uint32_t n_queries, const uint32_t* query_ids,
                                              const uint8_t* const* toks, const size_t* tok_lens,
                                              const uint32_t* n_groups, uint32_t* const* const* outs,
                                              oblivgm_plan** out_plan) {
    oblivgm_status st = check_ctx(ctx);
    if (st) return st;
    if (!out_plan || !query_ids || !toks || !tok_lens || !n_groups || !outs || n_queries == 0)
        return fail(OBLIVGM_EINVAL, "NULL or empty argument");
    *out_plan = nullptr;
    std::vector<ParsedQuery> parsed(n_queries);
    std::string err;
    for (uint32_t q = 0; q < n_queries; q++) {
        if (!outs[q]) return fail(OBLIVGM_EINVAL, "NULL output array");
        st = parse_tokens(toks + 3 * q, tok_lens + 3 * q, &parsed[q], &err);
        if (st != OBLIVGM_OK) return fail(st, err);
    }
    Plan plan;
    st = plan_filter(ctx, ctx->tables, n_queries, query_ids, parsed.data(), n_groups, outs, &plan);
    if (st != OBLIVGM_OK) return st;
    const WsImage im = build_ws_image(plan);
    auto* p = new (std::nothrow) oblivgm_plan();
    if (!p) return fail(OBLIVGM_ENOMEM, "host allocation");
    cudaError_t e = cudaMalloc(&p->ws, im.total);
    if (e == cudaSuccess) e = cudaMemcpy(p->ws, im.bytes.data(), im.total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p->ws) cudaFree(p->ws);
        delete p;
        return cuda_fail(e, "plan buffer");
    }
    p->ctx = ctx;
    p->params = filter_params(ctx, plan, im, p->ws, ctx->d_error);
    p->n_items = plan.item_start.back();
    p->threads = plan.threads;
    p->E = plan.elems_per_thread;
    p->wp = plan.wp;
    *out_plan = p;
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_plan_launch(oblivgm_plan* p, void* stream) {
    const NvtxRange nvtx_range("oblivgm_plan_launch");
    if (!p) return fail(OBLIVGM_EINVAL, "NULL plan");
    if (p->n_items == 0) return OBLIVGM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the walk-parallel kernel leaves its counters at zero when it ends; the per-element
    // kernel's counter is cleared before each launch
    if (!p->wp) OGM_CUDA(cudaMemsetAsync(p->ws, 0, sizeof(unsigned long long), s), "plan counter reset");
    const cudaError_t e = launch_filter_kernel(p->params, p->n_items, p->ctx->sm_count, p->threads, p->E, p->wp, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_filter launch (plan)");
    p->ctx->launches++;
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_plan_describe(const oblivgm_plan* p, uint32_t* walk_parallel, uint32_t* threads,
                                                uint32_t* tile, uint64_t* n_items, uint32_t* grid) {
    if (!p) return fail(OBLIVGM_EINVAL, "NULL plan");
    if (walk_parallel) *walk_parallel = p->wp ? 1u : 0u;
    if (threads) *threads = p->threads;
    if (tile) *tile = p->params.tile;
    if (n_items) *n_items = p->n_items;
    if (grid) *grid = (uint32_t)std::min<uint64_t>(p->n_items, (uint64_t)p->ctx->sm_count);
    return OBLIVGM_OK;
}

extern "C" oblivgm_status oblivgm_plan_destroy(oblivgm_plan* p) {
    if (!p) return OBLIVGM_OK;
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(p->ws);
    delete p;
    return OBLIVGM_OK;
}
