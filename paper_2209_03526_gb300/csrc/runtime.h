// runtime.h -- host runtime state of an oblivgm context: resident tables,
// schedule, fault flag, and the serving loop (admission by memory, continuous
// batching of admitted queries into shared launches).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "host_crypto.h"
#include "oblivgm.h"

namespace ogm {

// NVTX range around an ABI call (header-only NVTX v3: a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Releases a stream-ordered workspace (from ws_alloc) when an entry point returns early
// on an error; the normal path releases it itself, checking the result, after done().
struct ScratchGuard {
    void* p;
    cudaStream_t s;
    ScratchGuard(void* p_, cudaStream_t s_) : p(p_), s(s_) {}
    ~ScratchGuard() {
        if (p) cudaFreeAsync(p, s);
    }
    void done() { p = nullptr; }
    ScratchGuard(const ScratchGuard&) = delete;
    ScratchGuard& operator=(const ScratchGuard&) = delete;
};

struct Table {
    uint32_t* dev = nullptr;   // [share set j][attr][stride] uint32
    uint64_t n_elems = 0;
    uint64_t stride = 0;       // n_elems rounded up to a multiple of 4
    uint32_t n_attrs = 0;
    uint32_t n_bits = 0;
    size_t bytes = 0;
};

// one-hot table: binary-RSS shares of one-hot vectors, [share set j][attr][elem][words]
struct OnehotTable {
    uint32_t* dev = nullptr;
    uint64_t n_elems = 0;
    uint32_t n_attrs = 0;
    uint32_t n_bits = 0;       // one-hot length 2^n_bits
    uint32_t words = 0;        // max(1, 2^n_bits / 32)
    size_t bytes = 0;
};

struct ServeQuery {
    uint64_t ticket = 0;
    ParsedQuery parsed;
    uint32_t n_groups = 0;
    std::map<uint32_t, Table> tables;   // snapshot of the tables it reads
    std::vector<uint32_t*> outs;        // 3 * n_groups device arrays
    std::vector<uint64_t> n_elems;      // per group
    std::vector<uint32_t> group_table;  // per group
    size_t bytes = 0;
    double est_aes = 0;                 // algorithmic AES blocks, for batch sizing
    double t_submit = 0, t_done = 0;
    int state = 0;                      // 0 queued, 1 on the device, 2 done, 3 failed
    int stream = 0;
    std::string error;
};

struct ServeBatch;

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queued;
    std::map<uint64_t, std::unique_ptr<ServeQuery>> queries;
    std::map<uint32_t, int> table_refs;
    uint64_t next_ticket = 1;
    uint64_t arena = 0, reserved = 0;
    uint32_t max_inflight = 64, inflight = 0;
    uint64_t admitted = 0, completed = 0, rejected = 0;
    int running_batches = 0;
    double batch_aes_target = 3e9;     // a batch closes once it holds this much work
    uint32_t poll_limit_ms = OBLIVGM_POLL_LIMIT_DEFAULT_MS;   // longest wait of any poll
    bool stop = false;
    static constexpr int kStreams = 2;
    cudaStream_t streams[kStreams] = {};
    std::thread worker;
};

}  // namespace ogm

struct oblivgm_ctx {
    int device = 0;
    int sm_count = 0;
    oblivgm_config cfg{};
    ogm::AesParams aes{};
    uint32_t rk_prf[3][44] = {};
    uint32_t* d_te0 = nullptr;
    uint32_t* d_te4 = nullptr;   // the four T-tables, 4 x 256 words, for the plain path
    uint32_t* d_error = nullptr;
    void* h_stage = nullptr;
    std::map<uint32_t, ogm::Table> tables;
    std::map<uint32_t, ogm::OnehotTable> onehot_tables;
    uint32_t threads = 768;          // the autotuner's pick on GB300 (256 x 4 spills)
    uint32_t elems_per_thread = 1;
    uint64_t wp_max_elems = 0;       // batches with at most this many elements in all run walk-parallel
    uint32_t wp_tile = 0;            // walk-parallel elements per tile; 0 = chosen per launch
    std::atomic<uint64_t> launches{0};
    bool test_expire_next = false;      // failure-path test hook, one-shot
    std::atomic<bool> test_fail_alloc{false};   // failure-path test hook: refuse the next workspace allocation
    uint64_t test_wait_limit_ns = 0;
    uint32_t aes_layout = 0;             // OBLIVGM_AES_TTABLE until oblivgm_autotune_aes_layout measures
    double aes_layout_rate[2] = {0, 0};  // measured PRG blocks/s: T-table, bitsliced
    ogm::ServeState serve;
};

namespace ogm {

oblivgm_status fail(oblivgm_status st, const std::string& msg);
const std::string& last_error_text();   // the calling thread's last failure text
oblivgm_status cuda_fail(cudaError_t e, const char* what);

struct Plan;
oblivgm_status serve_init(oblivgm_ctx* ctx);
void serve_shutdown(oblivgm_ctx* ctx);
bool table_in_use(oblivgm_ctx* ctx, uint32_t table_id);

// plan + launch of the fused kernel over already-parsed queries (used by the serving loop)
oblivgm_status launch_parsed(oblivgm_ctx* ctx, uint32_t n_queries, const uint32_t* query_ids,
                             const ParsedQuery* parsed, const uint32_t* n_groups, uint32_t* const* const* outs,
                             const std::map<uint32_t, Table>& tables, cudaStream_t st);

double now_ms();
oblivgm_status set_onehot_attrs();
oblivgm_status set_keygen_attrs();
// stream-ordered device workspace; ENOMEM when the allocator refuses (or the test hook says so)
oblivgm_status ws_alloc(oblivgm_ctx* ctx, void** p, size_t bytes, cudaStream_t s, const char* what);
oblivgm_status set_fresh_attrs();
oblivgm_status set_shuffle_attrs();
oblivgm_status set_prg_attrs();
oblivgm_status repack_keys_device(oblivgm_ctx* ctx, const uint8_t* wire, uint32_t kind, uint32_t n, uint32_t n_keys,
                                  DevKey* out, cudaStream_t s);

}  // namespace ogm
