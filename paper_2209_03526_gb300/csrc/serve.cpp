// serve.cpp -- the serving loop of an oblivgm context.
//
// Queries are admitted by memory (their output share sets must fit in the
// serve arena) and by slot count.  A worker thread takes admitted queries in
// arrival order into a batch until the batch holds enough work to fill the GPU
// (about 3e9 AES blocks) and launches it as one fused kernel on one of two
// streams; the next batch goes to the other stream at once and takes over the
// SMs the running one releases (continuous batching).  A host callback on the
// batch's stream marks its queries done.
// Each query's shares depend only on its tokens, ticket and tables (the PRF
// counters carry element, step, table and query id), never on the batch it ran
// in.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "runtime.h"

namespace ogm {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct ServeBatch {
    oblivgm_ctx* ctx;
    std::vector<uint64_t> tickets;
};

namespace {

void CUDART_CB on_batch_done(void* arg) {
    // host callback: no CUDA calls allowed here
    ServeBatch* b = static_cast<ServeBatch*>(arg);
    ServeState& S = b->ctx->serve;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        const double t = now_ms();
        for (uint64_t tk : b->tickets) {
            auto it = S.queries.find(tk);
            if (it != S.queries.end() && it->second->state == 1) {
                it->second->state = 2;
                it->second->t_done = t;
                S.completed++;
            }
        }
        S.running_batches--;
    }
    S.cv_done.notify_all();
    S.cv_work.notify_all();
    delete b;
}

void worker_main(oblivgm_ctx* ctx) {
    ServeState& S = ctx->serve;
    cudaSetDevice(ctx->device);
    int next_stream = 0;
    std::unique_lock<std::mutex> lk(S.mu);
    for (;;) {
        S.cv_work.wait(lk, [&] { return S.stop || (!S.queued.empty() && S.running_batches < ServeState::kStreams); });
        if (S.stop) break;
        // take queued queries in arrival order until the batch holds enough work to fill the
        // GPU: small queries share a launch, a large one runs on its own, and a query that
        // arrives meanwhile starts in the next batch on the other stream
        std::vector<ServeQuery*> batch;
        double work = 0;
        while (!S.queued.empty() && work < S.batch_aes_target) {
            auto it = S.queries.find(S.queued.front());
            S.queued.pop_front();
            if (it != S.queries.end() && it->second->state == 0) {
                batch.push_back(it->second.get());
                work += it->second->est_aes;
            }
        }
        if (batch.empty()) continue;
        const int si = next_stream;
        next_stream = (next_stream + 1) % ServeState::kStreams;
        cudaStream_t st = S.streams[si];
        for (ServeQuery* q : batch) { q->state = 1; q->stream = si; }
        S.running_batches++;
        lk.unlock();

        // allocate outputs in stream order, then one fused launch for the whole batch
        std::vector<uint32_t> qids, ngroups;
        std::vector<uint32_t* const*> outs;
        std::vector<ParsedQuery> parsed;
        std::map<uint32_t, Table> tables;
        oblivgm_status st_code = OBLIVGM_OK;
        std::string err;
        for (ServeQuery* q : batch) {
            for (size_t g = 0; g < q->n_groups && st_code == OBLIVGM_OK; g++)
                for (int j = 0; j < 3; j++) {
                    void* p = nullptr;
                    cudaError_t e = cudaMallocAsync(&p, std::max<uint64_t>(q->n_elems[g], 4) * sizeof(uint32_t), st);
                    if (e != cudaSuccess) { st_code = OBLIVGM_ENOMEM; err = cudaGetErrorString(e); break; }
                    q->outs[3 * g + j] = static_cast<uint32_t*>(p);
                }
            qids.push_back((uint32_t)q->ticket);
            ngroups.push_back(q->n_groups);
            outs.push_back(q->outs.data());
            parsed.push_back(q->parsed);
            for (auto& kv : q->tables) tables[kv.first] = kv.second;
        }
        if (st_code == OBLIVGM_OK) {
            const NvtxRange nvtx_range("oblivgm_serve_batch");
            st_code = launch_parsed(ctx, (uint32_t)batch.size(), qids.data(), parsed.data(), ngroups.data(),
                                    outs.data(), tables, st);
            if (st_code != OBLIVGM_OK) err = last_error_text();   // this thread's failure text
        }
        auto* cb = new ServeBatch{ctx, {}};
        for (ServeQuery* q : batch) cb->tickets.push_back(q->ticket);
        if (st_code != OBLIVGM_OK) {
            lk.lock();
            for (ServeQuery* q : batch) { q->state = 3; q->error = "launch failed: " + err; }
            S.running_batches--;
            S.cv_done.notify_all();
            delete cb;
            continue;
        }
        cudaLaunchHostFunc(st, on_batch_done, cb);
        lk.lock();
    }
}

}  // namespace

oblivgm_status serve_init(oblivgm_ctx* ctx) {
    ServeState& S = ctx->serve;
    S.max_inflight = ctx->cfg.serve_max_inflight ? ctx->cfg.serve_max_inflight : 64;
    if (ctx->cfg.serve_arena_bytes) {
        S.arena = ctx->cfg.serve_arena_bytes;
    } else {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(OBLIVGM_ECUDA, "cudaMemGetInfo");
        S.arena = free_b / 4;
    }
    for (int i = 0; i < ServeState::kStreams; i++)
        if (cudaStreamCreateWithFlags(&S.streams[i], cudaStreamNonBlocking) != cudaSuccess)
            return fail(OBLIVGM_ECUDA, "stream creation");
    S.worker = std::thread(worker_main, ctx);
    return OBLIVGM_OK;
}

void serve_shutdown(oblivgm_ctx* ctx) {
    ServeState& S = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
    }
    S.cv_work.notify_all();
    if (S.worker.joinable()) S.worker.join();
    for (int i = 0; i < ServeState::kStreams; i++)
        if (S.streams[i]) cudaStreamSynchronize(S.streams[i]);
    for (auto& kv : S.queries)
        for (uint32_t* p : kv.second->outs)
            if (p) cudaFree(p);
    S.queries.clear();
    for (int i = 0; i < ServeState::kStreams; i++)
        if (S.streams[i]) cudaStreamDestroy(S.streams[i]);
}

bool table_in_use(oblivgm_ctx* ctx, uint32_t table_id) {
    std::lock_guard<std::mutex> lk(ctx->serve.mu);
    auto it = ctx->serve.table_refs.find(table_id);
    return it != ctx->serve.table_refs.end() && it->second > 0;
}

}  // namespace ogm

using namespace ogm;

extern "C" {

oblivgm_status oblivgm_submit(oblivgm_ctx* ctx, const uint8_t* const tok[3], const size_t tok_len[3],
                              uint64_t* ticket) {
    if (!ctx || !ticket) return fail(OBLIVGM_EINVAL, "NULL argument");
    auto q = std::make_unique<ServeQuery>();
    std::string err;
    oblivgm_status st = parse_tokens(tok, tok_len, &q->parsed, &err);
    if (st != OBLIVGM_OK) return fail(st, err);
    if (q->parsed.out_group != 0) return fail(OBLIVGM_EINVAL, "the serving loop evaluates masked-mode tokens only");
    uint32_t ng = 0;
    for (const ParsedPred& p : q->parsed.preds) ng = std::max(ng, p.group + 1);
    if (ng > OBLIVGM_MAX_GROUPS) return fail(OBLIVGM_EINVAL, "more than 64 AND-groups");
    q->n_groups = ng;
    q->n_elems.assign(ng, 0);
    q->group_table.assign(ng, 0xFFFFFFFFu);
    for (const ParsedPred& p : q->parsed.preds) {
        auto it = ctx->tables.find(p.table);
        if (it == ctx->tables.end()) return fail(OBLIVGM_ENOENT, "predicate on a table that is not loaded");
        q->tables[p.table] = it->second;
        if (q->group_table[p.group] == 0xFFFFFFFFu) q->group_table[p.group] = p.table;
        else if (q->group_table[p.group] != p.table) return fail(OBLIVGM_EINVAL, "an AND-group spans two tables");
        q->n_elems[p.group] = it->second.n_elems;
    }
    for (uint32_t g = 0; g < ng; g++)
        if (q->group_table[g] == 0xFFFFFFFFu) return fail(OBLIVGM_EINVAL, "an AND-group has no predicate");
    q->outs.assign(3 * ng, nullptr);
    for (const ParsedPred& p : q->parsed.preds) {
        // FSS walks of the predicate plus its re-shares (and the AND's), per element
        const double walks = p.kind == OBLIVGM_PRED_EQ ? 6.0 * p.n : 24.0 * p.n;
        q->est_aes += (walks + 6.0) * (double)q->n_elems[p.group];
    }
    q->bytes = 0;
    for (uint32_t g = 0; g < ng; g++) q->bytes += 3 * std::max<uint64_t>(q->n_elems[g], 4) * sizeof(uint32_t);
    ServeState& S = ctx->serve;
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.inflight >= S.max_inflight || S.reserved + q->bytes > S.arena) {
        S.rejected++;
        return fail(OBLIVGM_EAGAIN, "no serving slot or arena memory free");
    }
    q->ticket = S.next_ticket++;
    q->t_submit = now_ms();
    S.inflight++;
    S.reserved += q->bytes;
    S.admitted++;
    for (auto& kv : q->tables) S.table_refs[kv.first]++;
    *ticket = q->ticket;
    S.queued.push_back(q->ticket);
    S.queries[q->ticket] = std::move(q);
    S.cv_work.notify_all();
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_poll(oblivgm_ctx* ctx, uint64_t ticket, int32_t timeout_ms, oblivgm_result* out) {
    if (!ctx || !out) return fail(OBLIVGM_EINVAL, "NULL argument");
    ServeState& S = ctx->serve;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.queries.find(ticket);
    if (it == S.queries.end()) return fail(OBLIVGM_ENOENT, "unknown ticket");
    ServeQuery* q = it->second.get();
    auto done = [&] { return q->state >= 2; };
    if (!done()) {
        if (timeout_ms == 0) return OBLIVGM_EAGAIN;
        // a negative timeout waits up to the context's poll limit; so does a longer one
        const uint32_t wait_ms = timeout_ms < 0 ? S.poll_limit_ms : std::min<uint32_t>((uint32_t)timeout_ms,
                                                                                        S.poll_limit_ms);
        if (!S.cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), done))
            return fail(OBLIVGM_ETIMEOUT, timeout_ms < 0 || (uint32_t)timeout_ms > S.poll_limit_ms
                                              ? "query not finished within the context's poll limit"
                                              : "query not finished within the timeout");
    }
    if (q->state == 3) return fail(OBLIVGM_ECUDA, q->error);
    std::memset(out, 0, sizeof *out);
    out->n_groups = q->n_groups;
    for (uint32_t g = 0; g < q->n_groups; g++) {
        out->table[g] = q->group_table[g];
        out->n_elems[g] = q->n_elems[g];
        for (int j = 0; j < 3; j++) out->shares[g][j] = q->outs[3 * g + j];
    }
    out->latency_ms = q->t_done - q->t_submit;
    out->ticket = ticket;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_release(oblivgm_ctx* ctx, uint64_t ticket) {
    if (!ctx) return fail(OBLIVGM_EINVAL, "NULL argument");
    ServeState& S = ctx->serve;
    std::unique_ptr<ServeQuery> q;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        auto it = S.queries.find(ticket);
        if (it == S.queries.end()) return fail(OBLIVGM_ENOENT, "unknown ticket");
        if (it->second->state < 2) return fail(OBLIVGM_EAGAIN, "query still running");
        q = std::move(it->second);
        S.queries.erase(it);
        S.inflight--;
        S.reserved -= q->bytes;
        for (auto& kv : q->tables) S.table_refs[kv.first]--;
    }
    cudaSetDevice(ctx->device);
    for (uint32_t* p : q->outs)
        if (p) cudaFreeAsync(p, S.streams[q->stream]);
    S.cv_work.notify_all();
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_set_poll_limit(oblivgm_ctx* ctx, uint32_t max_ms, uint32_t* previous) {
    if (!ctx) return fail(OBLIVGM_EINVAL, "NULL argument");
    if (max_ms == 0) return fail(OBLIVGM_EINVAL, "the poll limit must be at least 1 ms");
    std::lock_guard<std::mutex> lk(ctx->serve.mu);
    if (previous) *previous = ctx->serve.poll_limit_ms;
    ctx->serve.poll_limit_ms = max_ms;
    return OBLIVGM_OK;
}

oblivgm_status oblivgm_serve_stats(oblivgm_ctx* ctx, uint64_t* admitted, uint64_t* completed, uint64_t* rejected,
                                   uint64_t* reserved_bytes) {
    if (!ctx) return fail(OBLIVGM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->serve.mu);
    if (admitted) *admitted = ctx->serve.admitted;
    if (completed) *completed = ctx->serve.completed;
    if (rejected) *rejected = ctx->serve.rejected;
    if (reserved_bytes) *reserved_bytes = ctx->serve.reserved;
    return OBLIVGM_OK;
}

}  // extern "C"
