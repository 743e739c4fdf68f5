/*
 * oblivgm.h -- C ABI of the GB300 library for OblivGM's secure predicate
 * evaluation (OblivGM: Oblivious Attributed Subgraph Matching as a Cloud
 * Service, arXiv 2209.03526).
 *
 * The library evaluates, on one GPU, what the three cloud servers CS1..CS3
 * compute in secEval (Alg. 3): every predicate of a query on every element
 * (vertex or edge) of a resident, secret-shared table, by DPF Eval (equality)
 * or DCF Eval (range) over masked attribute values, followed by the re-share
 * of Sec. III-B and the aggregation of Sec. V-D.  The three servers are
 * simulated as three share sets in one address space; "sending" a share is a
 * read of another share set.
 *
 * Conventions
 *  - Every function returns an oblivgm_status (0 on success, a negative code
 *    otherwise) and never throws.  oblivgm_last_error() gives the text of the
 *    calling thread's last failure.
 *  - "device pointer" means memory of the context's GPU (cudaMalloc, or a
 *    torch tensor's data_ptr()); "host pointer" means ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that take a stream only enqueue work on it; inputs that
 *    are host buffers may be reused as soon as the call returns.
 *  - All integers are little-endian.  Arithmetic is in Z_{2^32} unless
 *    stated; attribute domains are Z_{2^n}, 1 <= n <= 32.
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef OBLIVGM_H
#define OBLIVGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t oblivgm_status;

#define OBLIVGM_OK             0
#define OBLIVGM_EINVAL        (-1)   /* bad argument, malformed token or key            */
#define OBLIVGM_ENOMEM        (-2)   /* a device or host allocation failed              */
#define OBLIVGM_ECUDA         (-3)   /* a CUDA call failed (text in last_error)         */
#define OBLIVGM_EARCH         (-4)   /* the device is not compute capability 10.3       */
#define OBLIVGM_ERANGE        (-5)   /* output buffer too small; needed size reported   */
#define OBLIVGM_EBUSY         (-6)   /* table re-load while in-flight queries use it    */
#define OBLIVGM_EAGAIN        (-7)   /* submit: no slot/memory now; poll: not finished  */
#define OBLIVGM_ETIMEOUT      (-8)   /* poll: timeout expired before completion         */
#define OBLIVGM_ENOENT        (-9)   /* unknown table id or ticket                      */
#define OBLIVGM_EFAULT_DEVICE (-10)  /* a bounded device-side wait expired              */

/* predicate kinds (Sec. V-C: equality -> DPF, range -> DCF) */
#define OBLIVGM_PRED_EQ    1u
#define OBLIVGM_PRED_RANGE 2u

/* How a predicate's result joins its group's result (Sec. V-D, aggregation of
 * several predicates of one target vertex): the group's predicates are folded
 * left to right in list order, acc <- acc OP x_p, each step an RSS product
 * (Sec. III-B) plus local linear terms, then a re-share.  Over 0/1 values:
 *   AND  acc * x                 (all predicates hold; the paper's product)
 *   XOR  acc + x - 2 acc x       (the paper's "one of", written with XOR)
 *   OR   acc + x - acc x         (at least one holds)
 * In the one-hot mode (shares over Z_2) the same three are a b, a ^ b and
 * a ^ b ^ a b.  A group's first predicate must carry AND (0). */
#define OBLIVGM_COMBINE_AND 0u
#define OBLIVGM_COMBINE_XOR 1u
#define OBLIVGM_COMBINE_OR  2u

/* key kinds in the key wire format */
#define OBLIVGM_KEY_DPF 1u
#define OBLIVGM_KEY_DCF 2u

/* memory kinds of caller buffers */
#define OBLIVGM_MEM_HOST   0
#define OBLIVGM_MEM_DEVICE 1

/* flags of oblivgm_eval_*_batch */
#define OBLIVGM_ALL_PAIRS 1u
#define OBLIVGM_KEYS_DEVICE 2u   /* keys are device memory; put the key bit length n in flags bits 8..15 */

typedef struct oblivgm_ctx oblivgm_ctx;

typedef struct {
    /* k_1, k_2, k_3: AES-128 keys of the zero-sharing PRF F (Sec. III-B);
     * server i holds k_i and k_{i-1}.  F(k, ctr) = bytes 0..3 of AES_k(ctr). */
    uint8_t  prf_keys[3][16];
    /* serving loop: device bytes it may reserve for in-flight queries' outputs
     * (0 = 25 % of free memory at create time) and in-flight query slots
     * (0 = 64). */
    uint64_t serve_arena_bytes;
    uint32_t serve_max_inflight;
    uint32_t flags;   /* reserved, must be 0 */
} oblivgm_config;

/* One predicate of a query, as the client (graph owner) knows it. */
typedef struct {
    uint32_t kind;    /* OBLIVGM_PRED_EQ or OBLIVGM_PRED_RANGE                      */
    uint32_t table;   /* id of the element table the predicate reads (< 65536)      */
    uint32_t attr;    /* attribute row within that table (< 65536)                  */
    uint32_t group;   /* group of the query: all predicates of a group are on the
                         same table and their results are folded into one 0/1
                         result per element (Sec. V-D)                              */
    uint32_t lo;      /* EQ: the value alpha; RANGE: inclusive lower bound          */
    uint32_t hi;      /* RANGE: inclusive upper bound (lo <= hi); ignored for EQ    */
    uint32_t combine; /* OBLIVGM_COMBINE_*: how this result joins the group's result
                         so far; AND (0) for a group's first predicate              */
} oblivgm_pred;

/* Result of a served query: per group g, three device arrays of n_elems[g]
 * uint32 each, the RSS share sets 1..3 of the group's 0/1 result.  The memory
 * belongs to the library until oblivgm_release(). */
#define OBLIVGM_MAX_GROUPS 64
typedef struct {
    uint32_t  n_groups;
    uint32_t  table[OBLIVGM_MAX_GROUPS];
    uint64_t  n_elems[OBLIVGM_MAX_GROUPS];
    uint32_t* shares[OBLIVGM_MAX_GROUPS][3];
    double    latency_ms;        /* submit -> completion seen by poll, host clock */
    uint64_t  ticket;
} oblivgm_result;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  Builds the AES tables on the
 * device and the PRF round keys from cfg->prf_keys.  Errors: EINVAL (cfg NULL
 * or flags != 0), EARCH (device is not sm_103), ECUDA, ENOMEM. */
oblivgm_status oblivgm_create(oblivgm_ctx** out, int32_t device, const oblivgm_config* cfg);

/* Synchronise and free everything the context owns (tables, workspaces,
 * served results not yet released).  NULL is accepted. */
oblivgm_status oblivgm_destroy(oblivgm_ctx* ctx);

/* Text of the calling thread's last error ("" if none); always NUL-terminated. */
oblivgm_status oblivgm_last_error(char* buf, size_t n);

/* Library version as 0xMMmmpp. */
uint32_t oblivgm_version(void);

/* ------------------------------------------------------------- share store */

/* Load one element table into resident device memory (encGraph output,
 * Alg. 1, held by the servers; only the columns a query needs are loaded,
 * Sec. VII-A).  share_sets[j] (j = 0, 1, 2) points to n_attrs * n_elems
 * uint32 in row-major [attr][elem] order: the additive share <x>_{j+1} of
 * every attribute value, x = <x>_1 + <x>_2 + <x>_3 mod 2^n_bits.  mem_kind
 * says whether the three pointers are host or device memory.  The caller
 * keeps ownership; with host memory the call returns after the copy is
 * enqueued from a pinned staging buffer and the caller may reuse its buffers
 * at once.  Re-loading an existing id replaces it (EBUSY while served queries
 * still use it).  Errors: EINVAL (n_bits outside 1..32, n_attrs 0 or
 * > 65536, table_id > 65535, NULL pointer), ENOMEM, ECUDA. */
oblivgm_status oblivgm_load_shares(oblivgm_ctx* ctx, uint32_t table_id, uint64_t n_elems, uint32_t n_attrs,
                                   uint32_t n_bits, const uint32_t* const share_sets[3], int32_t mem_kind,
                                   void* stream);

/* Drop a resident table.  Errors: ENOENT, EBUSY. */
oblivgm_status oblivgm_unload_shares(oblivgm_ctx* ctx, uint32_t table_id);

/* ------------------------------------------------------------- the PRG */

/* The fixed-key PRG of the DPF / DCF constructions cited in Sec. V-C
 * (lambda = 128, Sec. VII-A): H_K(s) = AES-128_K(s) xor s under one of the four
 * public keys K_j[i] = 16 j + i (key 0 K_L, 1 K_R, 2 K_vL, 3 K_vR), on the
 * counter blocks B_c = u64 c || 8 zero bytes, c = first .. first + n_blocks - 1,
 * computed in one of two AES layouts:
 *   OBLIVGM_AES_TTABLE    one block per thread, bank-replicated shared-memory
 *                         T-tables (the layout of every walk in this library);
 *   OBLIVGM_AES_BITSLICED 32 blocks per thread as 128 bit planes in registers,
 *                         SubBytes as a gate circuit (tower-field inverse).
 * out (device, n_out uint32): flags 0 -> out[4 c' + w] = word w of
 * H_K(B_{first + c'}), n_out >= 4 n_blocks; flags & OBLIVGM_PRG_PARITY -> one
 * word per 32 blocks, bit e of out[g] = XOR of the 128 bits of
 * H_K(B_{first + 32 g + e}), n_out >= n_blocks / 32 (for timing the layouts).
 * first and n_blocks must be multiples of 32.  Asynchronous on stream.
 * Errors: EINVAL, ERANGE (n_out too small), ECUDA. */
#define OBLIVGM_AES_TTABLE    0u
#define OBLIVGM_AES_BITSLICED 1u
#define OBLIVGM_PRG_PARITY    1u
oblivgm_status oblivgm_prg_batch(oblivgm_ctx* ctx, uint32_t layout, uint32_t key, uint64_t first,
                                 uint64_t n_blocks, uint32_t flags, uint32_t* out, uint64_t n_out, void* stream);

/* The AES-layout dimension of the autotuner: times oblivgm_prg_batch in both
 * layouts on 2^26 blocks (parity outputs, best of three after a warm-up,
 * synchronous; allocates an 8 MB buffer) and reports the faster layout and
 * both rates in blocks per second (any pointer may be NULL).  The walks of the
 * filter, keygen, fresh-key and one-hot kernels are built in the T-table
 * layout: this measurement is what decides that layout for them. */
oblivgm_status oblivgm_autotune_aes_layout(oblivgm_ctx* ctx, uint32_t* layout, double* ttable_blocks_per_s,
                                           double* bitsliced_blocks_per_s);

/* ------------------------------------------------------------------ tokens */

/* Client-side secure query token generation (genToken, Sec. V-C), for the
 * masked-input evaluation: per predicate a fresh mask r (RSS-shared among the
 * servers) and three independent FSS key pairs for the shifted function
 * (EQ: DPF at alpha + r; RANGE [lo, hi]: DCFs at lo + r and hi + 1 + r),
 * every pair with output beta' = 3^{-1} mod 2^32 so the three pairs add up to
 * the predicate bit.  Server i receives tok[i] holding its two key halves:
 * CS1 (k^1_1, k^2_1), CS2 (k^2_2, k^3_1), CS3 (k^3_2, k^1_2).
 * Host only and deterministic in `seed` (AES-128 counter mode, counter block
 * = u64 index || 8 zero bytes; per predicate one block for the mask, bytes
 * 0..3 r, 4..7 <r>_1, 8..11 <r>_2, each mod 2^n, <r>_3 = r - <r>_1 - <r>_2,
 * then two root-seed blocks per key, pairs 1..3 in order, RANGE keys a1 then
 * a0).
 * Token of server i, all fields little-endian:
 *   header 16 B: u32 magic 0x544D474F, u8 version 1, u8 i (1..3), u8 n,
 *     u8 0, u16 n_preds, u16 0, u32 total length;
 *   per predicate a 24 B record: u8 kind, u8 n, u16 table, u16 attr,
 *     u16 group, u32 <r>_i, u32 <r>_{i+1}, u32 c*beta' (RANGE, c = [a1 <= a0];
 *     0 for EQ), u8 combine, 3 zero bytes; then key half A and key half B,
 *     each one DPF key (EQ)
 *     or two DCF keys, a1 = hi + 1 + r first, then a0 = lo + r (RANGE).
 *   key: u8 kind (1 DPF, 2 DCF), u8 n, u8 party b, u8 0, u32 0, seed[16],
 *     per level i = 1..n: s_CW[16], u8 t^L_CW, u8 t^R_CW, u16 0 and for DCF
 *     u32 V_CW; then u32 CW_{n+1}.
 * tok[i] may be NULL to query the size: out_len[i] is always set.  Errors:
 * EINVAL (0 or more than 64 predicates, empty range, value outside 2^n,
 * n outside 1..32, ids >= 65536, combine above 2 or not AND on a group's
 * first predicate), ERANGE (cap < out_len[i]). */
oblivgm_status oblivgm_keygen(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits,
                              const uint8_t seed[16], uint8_t* const tok[3], size_t cap, size_t out_len[3]);

/* --------------------------------------------------------- raw FSS batches */

/* DPF Eval (point function, Boyle-Gilboa-Ishai tree construction cited in
 * Sec. V-C) of wire-format keys on device-resident points.
 * keys: host pointer to n_keys keys back to back, all of the same kind and
 *       n (length 28 + 20 n bytes for DPF, 28 + 24 n for DCF).
 * points: device pointer, n_points uint32 (bits above n are ignored).
 * flags & OBLIVGM_ALL_PAIRS: out[k * n_points + i] = Eval(key k, points[i]),
 *       needs n_out >= n_keys * n_points; key_of_point is ignored.
 * otherwise: out[i] = Eval(key key_of_point[i], points[i]) with key_of_point
 *       a device pointer of n_points uint32; an index >= n_keys gives 0.
 * out: device pointer of n_out uint32, caller-owned.  Asynchronous on stream.
 * Errors: EINVAL (malformed key, kinds or n mixed, NULL), ERANGE (n_out too
 * small), ENOMEM, ECUDA. */
oblivgm_status oblivgm_eval_dpf_batch(oblivgm_ctx* ctx, const uint8_t* keys, uint32_t n_keys,
                                      const uint32_t* points, const uint32_t* key_of_point, uint64_t n_points,
                                      uint32_t flags, uint32_t* out, uint64_t n_out, void* stream);

/* With flags & OBLIVGM_KEYS_DEVICE (and n in flags bits 8..15) `keys` is a
 * 4-byte-aligned device pointer, e.g. the output of oblivgm_keygen_device;
 * the keys are repacked on the device, and a key whose header does not match
 * (kind, n) evaluates as a zero key and raises EFAULT_DEVICE at the next
 * oblivgm_sync. */

/* DCF Eval (comparison function x < alpha, construction of Boyle et al.
 * cited in Sec. V-C); same arguments and errors as oblivgm_eval_dpf_batch. */
oblivgm_status oblivgm_eval_dcf_batch(oblivgm_ctx* ctx, const uint8_t* keys, uint32_t n_keys,
                                      const uint32_t* points, const uint32_t* key_of_point, uint64_t n_points,
                                      uint32_t flags, uint32_t* out, uint64_t n_out, void* stream);

/* ---------------------------------------------------- filter and combine */

/* secEval (Alg. 3) of one query, fused: for every AND-group of the token and
 * every element of the group's table, open x^ = x + r (the masked-input
 * approach of Sec. V-C), evaluate the six key halves of each predicate
 * (Eq. predEval, masked form: CS_i sums its two halves), re-share each
 * predicate's 3-out-of-3 sum to RSS with the PRF zero-sharing (Sec. III-B,
 * counter = element, step p, table, query_id), and fold the group's
 * predicates in token order (AND, XOR or OR per predicate, OBLIVGM_COMBINE_*)
 * with RSS multiplication plus re-share (step 64 + p) (Sec. V-D).
 * tok[i], tok_len[i]: host pointers to server i+1's token from
 *       oblivgm_keygen (all three must come from the same keygen call).
 * out: host array of 3 * n_groups device pointers; out[3 g + i] receives
 *       share set i+1 of group g, n_elems(table of g) uint32, caller-owned.
 * Groups are numbered 0..n_groups-1 and must all be present in the token.
 * Asynchronous on stream.  Errors: EINVAL (malformed tokens, n_groups
 * mismatch, predicate on a missing table/attribute or with another n than
 * its table), ENOMEM, ECUDA, EFAULT_DEVICE (a key-staging wait expired;
 * detected at the next call that synchronises). */
oblivgm_status oblivgm_filter_and_combine(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                          const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out,
                                          void* stream);

/* The same for n_queries queries in ONE persistent launch (work items of all
 * queries' groups and element tiles in a shared queue, ordered by cost).
 * query_ids[q]; toks[3 q + i], tok_lens[3 q + i]; n_groups[q];
 * outs[q] is the query's array of 3 * n_groups[q] device pointers.
 * Each query's output equals what oblivgm_filter_and_combine gives for it
 * alone.  Errors as oblivgm_filter_and_combine. */
oblivgm_status oblivgm_filter_batch(oblivgm_ctx* ctx, uint32_t n_queries, const uint32_t* query_ids,
                                    const uint8_t* const* toks, const size_t* tok_lens, const uint32_t* n_groups,
                                    uint32_t* const* const* outs, void* stream);

/* Prepared batches for CUDA-graph capture.  oblivgm_plan_create parses the
 * queries (arguments as oblivgm_filter_batch), fixes the launch shape and
 * uploads descriptors and device keys into a plan-owned device buffer
 * (synchronous; allocates).  oblivgm_plan_launch then only resets the plan's
 * work counter and launches the fused kernel on `stream`: no host-side work,
 * no allocation and no pageable copies, so it may be captured into a CUDA
 * graph and replayed; every launch recomputes the same shares into the
 * outputs given at creation (which must stay valid).  Launches of one plan
 * must not overlap on the GPU.  oblivgm_plan_destroy synchronises the device
 * and frees the plan.  Errors as oblivgm_filter_batch. */
typedef struct oblivgm_plan oblivgm_plan;
oblivgm_status oblivgm_plan_create(oblivgm_ctx* ctx, uint32_t n_queries, const uint32_t* query_ids,
                                   const uint8_t* const* toks, const size_t* tok_lens, const uint32_t* n_groups,
                                   uint32_t* const* const* outs, oblivgm_plan** plan);
oblivgm_status oblivgm_plan_launch(oblivgm_plan* plan, void* stream);
oblivgm_status oblivgm_plan_destroy(oblivgm_plan* plan);

/* The launch a plan fixed: walk_parallel = 1 for the walk-parallel kernel
 * (one thread per key walk), 0 for the per-element kernel; threads per CTA;
 * elements per work item (tile: for the walk-parallel kernel, which may give
 * each of a few groups its own width, the widest); work items; CTAs launched
 * (one per SM at most).  Any output pointer may be NULL.  Errors: EINVAL for a
 * NULL plan. */
oblivgm_status oblivgm_plan_describe(const oblivgm_plan* plan, uint32_t* walk_parallel, uint32_t* threads,
                                     uint32_t* tile, uint64_t* n_items, uint32_t* grid);

/* The plain per-query GPU path: the same computation and results as
 * oblivgm_filter_and_combine (Alg. 3 + Eq. predEval + re-share + AND), but
 * launched the straightforward way -- per predicate one mask-open launch, one
 * launch per key half (6 DPF or 12 DCF walks, AES T-tables read from global
 * memory, one element per thread), one sum-and-re-share launch and one AND
 * launch -- with its scratch from cudaMallocAsync.  It is the comparison point
 * of the fused kernel and is parity-tested like it.  Errors as
 * oblivgm_filter_and_combine. */
oblivgm_status oblivgm_filter_plain(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                    const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out, void* stream);

/* Same inputs, outputs and results as oblivgm_filter_and_combine, for
 * callers that cannot allocate device memory while they run: code inside a
 * region where every allocation was made up front (a fixed memory budget, a
 * latency-critical serving thread), or a caller that has no business
 * touching the allocator at all.  The ordinary entry point takes its
 * per-call workspace (work-queue counter, descriptors and device keys) from
 * cudaMallocAsync; this one takes it from one fixed device array of
 * OBLIVGM_NOALLOC_SCRATCH_BYTES (256 KiB) compiled into the library, which
 * every GPU that loads the library holds until the process exits.  The
 * paper has no counterpart: it is an engineering variant only.
 * Limits and rules:
 *  - a query needing more workspace than the array (about 31 range or 62
 *    equality predicates) is rejected with ERANGE before anything runs;
 *  - the call makes no cudaMalloc/cudaFree or other device allocation (host
 *    memory is still used to parse the tokens);
 *  - all calls share the one array: the call overwrites it (and zeroes the
 *    work counter) in stream order, so calls that can overlap on the GPU --
 *    on different streams, or from several threads or contexts on the same
 *    device -- race and give wrong results; issue them on one stream (calls
 *    back to back on one stream are safe);
 *  - the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress);
 *  - the call uploads its workspace from a host buffer that lives only for
 *    the call, so it must not be captured into a CUDA graph: on a stream under
 *    capture (or the legacy stream while another stream captures) it returns
 *    EINVAL before doing anything.  Use oblivgm_plan_* for graphs.
 * Errors as oblivgm_filter_and_combine, plus ERANGE. */
#define OBLIVGM_NOALLOC_SCRATCH_BYTES (256u * 1024u)
oblivgm_status oblivgm_filter_and_combine_noalloc(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                                  const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out,
                                                  void* stream);

/* -------------------------------------------------- keys generated on GPU */

/* Batched FSS key generation on the GPU, the client's genToken (Sec. V-C)
 * for many functions at once -- e.g. one key pair per element, which makes
 * the masked-input approach's per-value keys (Sec. V-C) practical and
 * removes the one-mask-per-column leak.  Pair i (0 <= i < n_pairs) is
 * Gen(alpha[i], beta[i]) of `kind` (DPF: beta * [x == alpha]; DCF:
 * beta * [x < alpha]) over Z_{2^32} with n_bits input bits, from the root
 * seeds AES_seed(2 i) and AES_seed(2 i + 1) (counter block: u64 index, 8 zero
 * bytes); same construction, PRG and wire format as oblivgm_keygen's keys.
 * alpha, beta: device pointers of n_pairs uint32.  keys_out: device pointer,
 * 4-byte aligned, at least 2 * n_pairs * L bytes (L = 28 + 20 n for DPF,
 * 28 + 24 n for DCF); key b of pair i at byte (2 i + b) L.  Asynchronous on
 * stream.  Errors: EINVAL, ERANGE (out_bytes too small), ECUDA. */
oblivgm_status oblivgm_keygen_device(oblivgm_ctx* ctx, uint32_t kind, uint32_t n_bits, uint64_t n_pairs,
                                     const uint32_t* alpha, const uint32_t* beta, const uint8_t seed[16],
                                     uint8_t* keys_out, uint64_t out_bytes, void* stream);

/* ------------------------------------------ fresh masks and keys per element */

/* The masked-input approach with a fresh mask and fresh keys for every
 * attribute value (the basic approach of Sec. V-C): for predicate p and
 * element c of its table the client draws its own mask r_{c,p} and generates
 * the predicate's three key pairs at the shifted point(s), so the servers open
 * x^_c = x_c + r_{c,p} and no two opened values share a mask.  The client's
 * key generation runs on the GPU (oblivgm_keygen_fresh) and writes each
 * server's token to device memory in the layout below; the servers' filter
 * (oblivgm_filter_fresh) evaluates element c's own keys, then combines,
 * re-shares and ANDs exactly as oblivgm_filter_and_combine does (same PRF
 * counters: element, step p, table, query_id; AND step 64 + p).
 *
 * Client randomness: AES-128 under the 16-byte client seed of the block
 * B(c, p, tag, j) = u64 c || u16 p || u16 tag || u32 j (little-endian):
 *   tag 1, j 0: mask block; r = bytes 0..3, <r>_1 = bytes 4..7,
 *               <r>_2 = bytes 8..11, each mod 2^n; <r>_3 = r - <r>_1 - <r>_2.
 *   tag 2, j = 4 * pair + 2 * sub + b: root seed of party b of key `sub` of
 *               pair `pair` (0..2).
 * Keys (beta' = 3^{-1} mod 2^32): EQ: one DPF per pair at alpha = lo + r;
 * RANGE: sub 0 = DCF at a1 = hi + 1 + r with +beta', sub 1 = DCF at
 * a0 = lo + r with -beta', and c * beta' with c = [a1 <= a0] (all mod 2^n).
 * Server i (1..3) holds half A = (pair i, party HA) and half B =
 * (pair i + 1, party HB): (HA, HB) = (0, 0), (1, 0), (1, 1) for servers 1, 2, 3
 * (pairs numbered 1..3 here, 0..2 in the block index).
 *
 * Fresh token of server i, device memory, little-endian, every array 16-byte
 * aligned (N = the table's elements, N4 = N rounded up to a multiple of 4):
 *   header 64 B: u32 magic 0x464D474F, u8 version 1, u8 i, u8 n, u8 0,
 *     u16 n_preds, u16 0, u32 0, u64 total length, zero to byte 64;
 *   per predicate a 32 B descriptor: u8 kind, u8 n, u16 table, u16 attr,
 *     u16 group, u64 N, u64 byte offset of its data block, u8 combine,
 *     7 zero bytes;
 *   data block: u32 rA[N4] = <r_c>_i, u32 rB[N4] = <r_c>_{i+1}, RANGE only
 *     u32 cb[N4] = c_c * beta'; then the key blocks (A, sub 0), (A, sub 1),
 *     (B, sub 0), (B, sub 1) (sub 1 for RANGE only), each:
 *     uint4 seed[N], uint4 scw[n][N] (level-major), u32 tl[N4], u32 tr[N4]
 *     (bit l - 1 = t^L_CW / t^R_CW of level l), DCF only u32 vcw[n][N4],
 *     u32 cw[N4] (CW_{n+1}).
 * Seeds and correction words are the 16 bytes of the wire format's fields
 * read as four little-endian u32 words. */

/* Size in bytes of each server's fresh token (the same for the three).
 * table_elems[t] = elements of table t (n_tables entries).  Errors: EINVAL
 * (as oblivgm_keygen, or a predicate on a table >= n_tables). */
oblivgm_status oblivgm_fresh_token_size(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits,
                                        const uint64_t* table_elems, uint32_t n_tables, uint64_t* bytes);

/* Client key generation on the GPU: writes the three servers' fresh tokens
 * into tok[0..2] (device pointers, 16-byte aligned, cap bytes each).
 * Asynchronous on stream.  Errors: EINVAL, ERANGE (cap too small), ECUDA. */
oblivgm_status oblivgm_keygen_fresh(oblivgm_ctx* ctx, const oblivgm_pred* preds, uint32_t n_preds,
                                    uint32_t n_bits, const uint64_t* table_elems, uint32_t n_tables,
                                    const uint8_t seed[16], uint8_t* const tok[3], uint64_t cap, void* stream);

/* The servers' secEval (Alg. 3, masked form of Eq. predEval, re-share, AND)
 * on fresh tokens.  tok[i]: device pointer to server i+1's token, tok_cap
 * bytes readable at each (a token whose stated length exceeds tok_cap is
 * rejected before any kernel reads it); the headers are read back to the
 * host to plan the launch.  out as in oblivgm_filter_and_combine.
 * Asynchronous on stream apart from that header read.  Errors: EINVAL
 * (malformed, mismatched or truncated tokens, a predicate whose N, attribute
 * or n disagrees with the loaded table), ENOENT, ECUDA. */
oblivgm_status oblivgm_filter_fresh(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                    uint64_t tok_cap, uint32_t n_groups, uint32_t* const* out, void* stream);

/* --------------------------------------------- secShuffle, secFetch case II */

/* secShuffle (Alg. 5, the RSS shuffle of Araki et al. that the paper cites),
 * the three servers simulated on this GPU.  A table D of n_rows rows of
 * `width` uint32 words is 3-out-of-3 shared, D = D1 op D2 op D3, with op XOR
 * (OBLIVGM_SHUFFLE_XOR, binary RSS as Alg. 5 is written) or addition mod 2^32
 * (OBLIVGM_SHUFFLE_ADD, the arithmetic shares the masked filter produces).
 * seeds = s12 || s23 || s31, the seed each pair of servers shares.  From its
 * seed a pair derives
 *   pi_ab: a pseudo-random permutation of [0, n_rows): a 4-round balanced
 *     Feistel network on 2h bits, h = max(1, ceil(bits(n_rows - 1) / 2)),
 *     with cycle walking; round r maps (L, R) to (R, L xor F_r(R)),
 *     F_r(R) = word 0 of AES_s(u64 R || u16 3 || u16 r || u32 n_rows) mod 2^h;
 *   T_ab (tag 1) and R_a (tag 2): word w of row i is word w mod 4 of
 *     AES_s(u64 i || u16 tag || u16 w / 4 || u32 0).
 * pi moves row i to row pi(i).  With "+"/"-" XOR in the binary case:
 *   CS1: X1 = pi31(pi12(D1 + D2 + T12) + T31)                   (sent to CS2)
 *   CS2: Y1 = pi12(D3 - T12); C1 = pi23(X1 + T23) - R2           (sent to CS3)
 *   CS3: C2 = pi23(pi31(Y1 - T31) - T23) - R1; R3 = C1 + C2      (sent to CS2)
 * out[0] = R1, out[1] = R2, out[2] = R3, and R1 + R2 + R3 = pi23(pi31(pi12(D))).
 * in[j], out[j]: device pointers, n_rows x width row-major, 4-byte aligned;
 * out must not overlap in.  1 <= width <= 64, n_rows < 2^31.  Asynchronous on
 * stream.  Errors: EINVAL, ENOMEM, ECUDA. */
#define OBLIVGM_SHUFFLE_ADD 0u
#define OBLIVGM_SHUFFLE_XOR 1u
oblivgm_status oblivgm_shuffle(oblivgm_ctx* ctx, uint32_t group, uint64_t n_rows, uint32_t width,
                               const uint32_t* const in[3], const uint8_t seeds[48], uint32_t* const out[3],
                               void* stream);

/* secFetch case II (Alg. 4): fetch every matched element of a filter result
 * obliviously.  The records D_c = x_c || id_c || d_c (x: the filter's RSS
 * result over Z_{2^32}, three device share sets of the table's n_elems
 * values; id_c = c shared as (c, 0, 0); d_c: the attributes `attrs` of table
 * table_id) are shuffled with oblivgm_shuffle (additive), the shuffled x are
 * opened, and the records whose x = 1 are kept in shuffled order, still
 * shared.  out[j]: device pointer, cap rows of 1 + n_attrs uint32 (id, then
 * the attributes; attribute shares stay additive mod 2^n).  *count: the
 * number of matches (host pointer; may exceed cap, then cap rows are
 * written).  Waits for the stream to read the count.  Errors: EINVAL,
 * ENOENT, ENOMEM, ECUDA. */
oblivgm_status oblivgm_fetch_multi(oblivgm_ctx* ctx, uint32_t table_id, const uint32_t* const x[3], uint32_t n_attrs,
                                   const uint32_t* attrs, const uint8_t seeds[48], uint32_t* const out[3],
                                   uint64_t cap, uint64_t* count, void* stream);

/* ---------------------------------------------------------- secFetch case I */

/* secFetch, case I (Alg. 4, Sec. V-D): obliviously fetch the one element of a
 * table that a group matched.  x[0..2] are device pointers to the
 * group's RSS result (the three share sets written by
 * oblivgm_filter_and_combine for that group, n_elems of table_id each); the
 * result assumes exactly one x_c = 1 (with none it is 0, with several the
 * sum).  out (device, 3 * (1 + n_attrs) uint32, [share set][column]) gets
 * the RSS shares of the matched element's index (sum_c c * [[x_c]], column
 * 0, no re-share needed) and of each listed attribute
 * (sum_c [[v_c]] (x) [[x_c]] with one re-share; counter element = attribute
 * index, step = 256 + group, table, query), the attribute values reducing
 * mod 2^n of the table.  out is cleared and then accumulated into (each
 * word is a sum mod 2^32), so it must not be read or written by other work
 * until the call's stream work completes.  n_attrs <= 64.  Asynchronous on
 * stream.  Errors: EINVAL, ENOENT (table), ECUDA. */
oblivgm_status oblivgm_fetch_unique(oblivgm_ctx* ctx, uint32_t query_id, uint32_t group, uint32_t table_id,
                                    const uint32_t* const x[3], uint32_t n_attrs, const uint32_t* attrs,
                                    uint32_t* out, void* stream);

/* ------------------------------------------------------------- one-hot mode */

/* The paper's secEval as written (Sec. V-B, V-C, Eq. predEval, Alg. 3), for
 * attribute domains of at most 2^16 values.  An n-bit attribute value v is
 * the one-hot vector e_v in {0,1}^(2^n), shared in binary RSS
 * (e_v = <e>_1 xor <e>_2 xor <e>_3).  The FSS keys are evaluated at every
 * public position of that vector, with no mask, so the masked mode's leak of
 * value differences does not arise; outputs are bits (Z_2) throughout.
 *
 * oblivgm_keygen_onehot: genToken of Sec. V-C -- three key pairs per
 * predicate for the predicate itself, output group Z_2, beta = 1 (EQ: DPF at
 * alpha; RANGE [lo, hi]: DCFs at hi + 1 and lo, plus the constant 1 for
 * party 0 when hi is the domain's last value).  Same token layout as
 * oblivgm_keygen with header byte 7 = 1 and all <r> fields 0; the random
 * stream has no mask block.  The keys stop their trees early (BGI16's early
 * termination for small output groups, the DPF cited in Sec. IV-B; the DCF
 * the same over the vector group Z_2^(2^m)): with m = min(n, 7) a leaf seed s
 * expands into the outputs of the 2^m positions sharing x >> m, as the 2^m
 * low bits of H_{K_vL}(s) (bit j in byte j / 8, bit j % 8), so a key has
 * n - m levels, walked with x >> m:
 *   key: u8 kind (1 DPF, 2 DCF), u8 n, u8 party b, u8 1, u32 0, seed[16],
 *     per level i = 1..n-m: s_CW[16], u8 t^L_CW, u8 t^R_CW, u16 0 and for DCF
 *     V_CW[16] (a 2^m-bit vector); then CW[16] (2^m bits).
 * Eval at x: walk the levels; y = V ^ H_{K_vL}(s) ^ t CW, with V the XOR of
 * H_{K_vdir}(s_parent) ^ t V_CW over the DCF's levels; the output is bit
 * x mod 2^m of y.  n_bits 1..16.  Errors as oblivgm_keygen. */
oblivgm_status oblivgm_keygen_onehot(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits,
                                     const uint8_t seed[16], uint8_t* const tok[3], size_t cap, size_t out_len[3]);

/* Load a one-hot table: share_sets[j] holds n_attrs * n_elems * W uint32
 * (W = max(1, 2^n_bits / 32)) in [attr][elem][word] order; bit l of an
 * element's vector is bit l % 32 of word l / 32 (bits past 2^n_bits zero).
 * Replaces an existing one-hot table with that id.  Errors as
 * oblivgm_load_shares (n_bits 1..16). */
oblivgm_status oblivgm_load_onehot(oblivgm_ctx* ctx, uint32_t table_id, uint64_t n_elems, uint32_t n_attrs,
                                   uint32_t n_bits, const uint32_t* const share_sets[3], int32_t mem_kind,
                                   void* stream);

/* One-hot secEval of one query: per predicate each server evaluates its two
 * key halves at all 2^n positions (EvalAll) and takes the parity of their AND
 * with the binary share its key pair is tied to (CS_i: shares i and i+1);
 * it XORs its two bits, re-shares in binary RSS (F into Z_2: the bit of
 * element e is bit e mod 128 of AES_k(c), c = u64 (e div 128) | 2^63 || u16
 * step || u16 table || u32 query, bit j of a block in byte j / 8 at bit
 * j % 8; steps as in the masked mode) and the group's predicates are folded
 * in binary RSS (AND, XOR or OR per predicate).  out[3 g + i] receives share set i+1 of group g packed 32
 * elements per word (element e in bit e % 32 of word e / 32; ceil(n_elems / 32)
 * words; bits past n_elems are 0).  Asynchronous on stream.  Errors as
 * oblivgm_filter_and_combine; EINVAL for a masked-mode token. */
oblivgm_status oblivgm_filter_onehot(oblivgm_ctx* ctx, uint32_t query_id, const uint8_t* const tok[3],
                                     const size_t tok_len[3], uint32_t n_groups, uint32_t* const* out,
                                     void* stream);

/* --------------------------------------------------------------- serving */

/* Non-blocking admission of one query into the serving loop (continuous
 * batching).  Copies the tokens.  The query id used for the PRF counters is
 * the returned ticket (low 32 bits).  The query is admitted only if a slot is
 * free and its output shares fit in the serve arena; otherwise EAGAIN and
 * nothing is kept.  Admitted queries start on the device as soon as the loop
 * can launch them, overlapping queries already running.
 * Errors: EAGAIN, EINVAL (as filter_and_combine), ENOENT (table not loaded). */
oblivgm_status oblivgm_submit(oblivgm_ctx* ctx, const uint8_t* const tok[3], const size_t tok_len[3],
                              uint64_t* ticket);

/* Wait for a ticket: timeout_ms = 0 only checks; a positive timeout waits at
 * most that long; a negative one waits at most the context's poll limit
 * (oblivgm_set_poll_limit, default OBLIVGM_POLL_LIMIT_DEFAULT_MS = 10 min),
 * which also caps positive timeouts.  No poll blocks longer than its timeout
 * or that limit.
 * OK: *out describes the result (library-owned until oblivgm_release).
 * EAGAIN (timeout_ms == 0 and not finished), ETIMEOUT (the wait ran out, the
 * query keeps running and may be polled again), ENOENT (unknown or already
 * released ticket), ECUDA (its batch failed to launch; the text says why). */
#define OBLIVGM_POLL_LIMIT_DEFAULT_MS 600000u
oblivgm_status oblivgm_poll(oblivgm_ctx* ctx, uint64_t ticket, int32_t timeout_ms, oblivgm_result* out);

/* Longest wait of any oblivgm_poll on this context, in milliseconds (>= 1).
 * `previous` (may be NULL) receives the limit it replaces.  Errors: EINVAL
 * (NULL context, max_ms 0). */
oblivgm_status oblivgm_set_poll_limit(oblivgm_ctx* ctx, uint32_t max_ms, uint32_t* previous);

/* Return a served result's memory to the arena (re-admits waiting work). */
oblivgm_status oblivgm_release(oblivgm_ctx* ctx, uint64_t ticket);

/* Serving statistics: queries admitted, completed, rejected (EAGAIN), and the
 * device bytes currently reserved. */
oblivgm_status oblivgm_serve_stats(oblivgm_ctx* ctx, uint64_t* admitted, uint64_t* completed, uint64_t* rejected,
                                   uint64_t* reserved_bytes);

/* ---------------------------------------------------------------- tuning */

/* Autotuned launch shape of the fused evaluation kernel: threads per CTA and
 * elements per thread ("paths per thread").  oblivgm_autotune times the
 * candidates on a synthetic table and keeps the fastest; the choice is
 * reported (and may be forced with oblivgm_set_schedule, 0 = keep). */
oblivgm_status oblivgm_autotune(oblivgm_ctx* ctx, uint32_t* threads, uint32_t* elems_per_thread);
oblivgm_status oblivgm_set_schedule(oblivgm_ctx* ctx, uint32_t threads, uint32_t elems_per_thread);

/* Small batches (Alg. 3 over few elements): a batch whose groups hold at
 * most `max_elems` elements in all is evaluated by the walk-parallel kernel,
 * one thread per key walk (six DPF or twelve DCF walks of an element side by
 * side), instead of one thread per element.  Both kernels give identical
 * output.  Default: 128 x the SM count; 0 turns the walk-parallel kernel off,
 * UINT64_MAX uses it for every batch.  `previous` (may be NULL) receives the
 * setting it replaces.  Applies to oblivgm_filter_and_combine,
 * oblivgm_filter_batch, the no-alloc entry point, plans created afterwards and
 * the serving loop.  Errors: EINVAL for a NULL context. */
oblivgm_status oblivgm_set_walk_parallel(oblivgm_ctx* ctx, uint64_t max_elems, uint64_t* previous);

/* Elements per work item of the walk-parallel kernel: 1..40 fixes it for every
 * group, 0 (the default) lets each launch choose it by simulating its schedule
 * over the SMs (one width for all groups, then, in a launch of at most 4
 * groups, a width per group).  For tuning and measurement.  `previous` (may be NULL) receives the setting it
 * replaces.  Errors: EINVAL (NULL context, tile above 40). */
oblivgm_status oblivgm_set_walk_parallel_tile(oblivgm_ctx* ctx, uint32_t tile, uint32_t* previous);

/* Synchronise `stream` and report device-side faults recorded since the last
 * check: EFAULT_DEVICE if a bounded device wait (key staging) expired in a
 * kernel of this context, ECUDA on a CUDA error; the flag is cleared. */
oblivgm_status oblivgm_sync(oblivgm_ctx* ctx, void* stream);

/* Failure-path test hook.  The next fused launch of this context (filter,
 * batch, served batch or no-alloc call) asks its first key-staging barrier for 16 bytes
 * more than the copy delivers, so every CTA's bounded wait runs out after
 * limit_us microseconds (1..2,000,000) instead of the normal 2 s.  Each CTA
 * then records the fault and returns without touching its outputs, and
 * oblivgm_sync reports EFAULT_DEVICE; the context stays usable.  Nothing
 * faults, traps or spins without a bound.  For tests only. */
oblivgm_status oblivgm_test_expire_next_wait(oblivgm_ctx* ctx, uint32_t limit_us);

/* Failure-path test hook: the context's next device workspace allocation is
 * refused as if the device were out of memory, so that call returns ENOMEM
 * (nothing is launched); later calls allocate normally.  The paper has no
 * counterpart. */
oblivgm_status oblivgm_test_fail_next_alloc(oblivgm_ctx* ctx);

/* Count of this library's kernel launches so far on the context (for the
 * bench's launch accounting). */
uint64_t oblivgm_launch_count(oblivgm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* OBLIVGM_H */
