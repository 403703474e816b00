/*
 * ssh.h -- C ABI of the GB300 (sm_103a) SSH library.
 *
 * SSH (Sketch, Shingle & Hash; Luo & Shrivastava, arXiv:1610.07328) indexes
 * time series for similarity search under dynamic time warping (DTW):
 *   Sec. 4.1  a random Gaussian filter r of length W slides over a series with
 *             step delta and each window gives one sign bit;
 *   Sec. 4.2  the bit string is cut into all overlapping n-bit shingles, which
 *             form a weighted set (shingle id -> count);
 *   Sec. 4.3  weighted minhashes of that set (consistent weighted sampling)
 *             give K*L hash values, K per table, L tables;
 *   Alg. 1    every stored series goes into the L tables;
 *   Alg. 2    a query probes its bucket in each table, the union of the buckets
 *             is its candidate set, and the candidates are ranked by DTW
 *             (Sec. 2.1) after LB_Keogh pruning (Sec. 3) to give the top k.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an ssh_status. SSH_OK is 0. No function aborts the
 *    process; ssh_last_error() gives a one-line reason for the last failure on
 *    the calling thread.
 *  - Pointers named d_* are device pointers on the index's device; all others
 *    are host pointers. `stream` is a cudaStream_t passed as void* (NULL is the
 *    legacy default stream). The caller owns every buffer passed in; the
 *    library never frees or keeps them unless a flag below says so.
 *  - Series are FP32, stored back to back: series i occupies lengths[i]
 *    consecutive floats right after series i-1. Values must be finite and
 *    smaller than 1e15 in magnitude.
 *  - Ids are assigned from 0 in insertion order across all lengths. Series of
 *    one length form one sub-index; a query is answered from the sub-index of
 *    its own length.
 *  - Calls on one index are not thread-safe; use one index per host thread or
 *    serialise the calls.
 */
#ifndef SSH_H
#define SSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssh_index ssh_index; /* opaque; created by ssh_create, owned by the library */

typedef enum ssh_status {
    SSH_OK = 0,
    SSH_EINVAL = 1,   /* a parameter is out of range or a pointer is NULL */
    SSH_ENOMEM = 2,   /* a device or host allocation failed */
    SSH_ECUDA = 3,    /* a CUDA call failed; ssh_last_error() has the CUDA message */
    SSH_ELENGTH = 4,  /* a series is too short, too long, or a query length has no sub-index */
    SSH_EBUSY = 5,    /* admission refused: not enough free device memory */
    SSH_ETIMEOUT = 6, /* a bounded device wait gave up */
    SSH_ENOTSUP = 7   /* a parameter combination the library does not implement */
} ssh_status;

/* Name of a status code ("SSH_OK", ...). Never NULL. */
const char* ssh_status_str(ssh_status s);

/* One-line description of the last failing call on this thread ("" if none). */
const char* ssh_last_error(void);

/*
 * Create an index (Alg. 1 input: W, delta, n and the number of tables; Sec. 5.1
 * uses 20 tables of one hash each, here there are L tables keyed by K hashes each).
 *   W      filter length, 1 <= W <= 8192 (Sec. 4.1)
 *   delta  filter step, >= 1 (Sec. 4.1)
 *   n      shingle length in bits, 1 <= n <= 32 (Sec. 4.2); anything else SSH_EINVAL.
 *          For n <= 16 the minhash draws of every (hash, shingle id) are tabulated
 *          on the device; for 17..32 they are computed in FP64 as each series is
 *          hashed (exact, slower; the one-permutation minhash option needs n <= 16)
 *   K, L   hashes per table and number of tables, K*L <= 4096
 *   band   Sakoe-Chiba band as a fraction of the series length: the DTW radius
 *          is floor(band * m) (clamped to m-1); band >= 0
 *   seed   seeds the filter r and every minhash draw (Philox4x32-10)
 * The filter is generated on the host; the Sec. 4.3 draw tables are built on the
 * current CUDA device (which becomes the index's device) by kernels, from draws
 * whose logarithm is a fixed sequence of FP64 operations (the same bits on any
 * machine). On success *out owns about 90 bytes of device memory per (hash,
 * shingle id) for n <= 16 (290 MB at K*L = 100, n = 15), and under 1 MB for n > 16.
 */
ssh_status ssh_create(int W, int delta, int n, int K, int L, float band, uint64_t seed, ssh_index** out);

/* The paper's SRP baseline (Sec. 5.2, Table 2) behind the same index, table and
 * query API: hash j of a series x of length m is the sign of r_j . x over the
 * whole series, r_j of i.i.d. normal entries (Philox4x32-10 keyed by seed with
 * counter (i / 2, j, "SRP1", m), Box-Muller, rounded once to FP32; generated per
 * length on first use); table l keys the K bits of hashes lK .. lK+K-1 with the
 * same fold as the SSH pairs (hash value (bit, 0)). Bits are exact: a product
 * within tau_m ||r_j|| ||x|| of zero (tau_m = max(1e-4, 2 m 2^-24 / (1 - m 2^-24)))
 * is recomputed in FP64. Any length >= 1 is accepted. Batch plans, the server,
 * ssh_hash_device and the window add's shared sketch are SSH-only (batch and
 * server creation and ssh_hash_device return SSH_ENOTSUP; windows are hashed as rows). */
ssh_status ssh_create_srp(int K, int L, float band, uint64_t seed, ssh_index** out);

/* Release the index and all its device memory. NULL is a no-op. */
void ssh_destroy(ssh_index* idx);

/* Copy of the FP32 filter r (W floats) into r_out (host). */
ssh_status ssh_get_filter(const ssh_index* idx, float* r_out);

/* Alg. 1 on host series: copies `count` series (back to back, lengths[i] each)
 * to the device, hashes them and rebuilds the tables of the affected
 * sub-indexes. Every length must be at least W + (n-1)*delta (one shingle) and
 * give at most 65535 shingles, else SSH_ELENGTH and nothing is added.
 * *first_id (may be NULL) receives the id of the first added series. Synchronous. */
ssh_status ssh_index_add(ssh_index* idx, const float* series, const int32_t* lengths, int64_t count,
                         int64_t* first_id);

#define SSH_ADD_BORROW 1u /* keep d_series instead of copying it (see ssh_index_add_device) */

/* Alg. 1 on device series (d_series on the index's device, lengths on the host).
 * Without SSH_ADD_BORROW the series are copied into index-owned device memory.
 * With SSH_ADD_BORROW the index keeps d_series itself: the caller must keep that
 * buffer allocated and unchanged until ssh_index_clear or ssh_destroy.
 * Work is ordered on `stream` and the call returns once it is enqueued: later work
 * on `stream`, and every query of this library on any stream, runs after the
 * tables are rebuilt (queries wait for the index's latest add). */
ssh_status ssh_index_add_device(ssh_index* idx, const float* d_series, const int32_t* lengths, int64_t count,
                                uint32_t flags, void* stream, int64_t* first_id);

/* Sec. 5.1's workload: every length-t window of one long series. Adds the
 * windows d_stream[p, p + t) for p = 0, step, 2 step, ... with p + t <= stream_len
 * ((stream_len - t) / step + 1 windows) as series of length t with consecutive
 * ids (the first in *first_id, may be NULL), into the sub-index of length t.
 * The windows are borrowed: the index keeps pointers into d_stream (device, the
 * index's device), which must stay allocated and unchanged until
 * ssh_index_clear or ssh_destroy. Each window is hashed exactly as the same
 * samples added as a series would be. Stream-ordered like ssh_index_add_device.
 * SSH_EINVAL for step < 1 or stream_len < t; SSH_ELENGTH for a t that
 * ssh_index_add would refuse. */
ssh_status ssh_index_add_windows_device(ssh_index* idx, const float* d_stream, int64_t stream_len, int32_t t,
                                        int64_t step, void* stream, int64_t* first_id);

/* Drop every stored series and table; parameters, filter and draw tables stay.
 * Ids restart at 0. */
ssh_status ssh_index_clear(ssh_index* idx);

/* Number of stored series. */
ssh_status ssh_index_size(const ssh_index* idx, int64_t* count);

/* Alg. 2 on host queries: for query i (lengths[i] floats) write its k nearest
 * stored series of the same length by banded DTW into ids[i*k .. i*k+k-1] and
 * dists[i*k ..] in ascending (distance, id) order. Distances are sums of squared
 * differences along the best warping path (the square root of Sec. 2.1 is not
 * taken; it does not change the order). A query with fewer than k candidates
 * fills the remaining slots with id -1 and distance +inf. 1 <= k <= 1024.
 * SSH_ELENGTH if a query length has no sub-index. Synchronous. */
ssh_status ssh_query(ssh_index* idx, const float* queries, const int32_t* lengths, int64_t nq, int k,
                     int64_t* ids, float* dists);

/* Alg. 2 on device queries; d_ids / d_dists are device arrays of nq*k entries.
 * Work is ordered on `stream`; the call returns when the results are written. */
ssh_status ssh_query_device(ssh_index* idx, const float* d_queries, const int32_t* lengths, int64_t nq, int k,
                            int64_t* d_ids, float* d_dists, void* stream);

/* Alg. 2 over several indexes at once, for collections whose filter length W
 * depends on the series length (one index per (length, W)): query i goes to the
 * first handle in handles[0..nh) that stores series of length lengths[i], and
 * d_which[i] (device int32, may be NULL) receives that handle's position; ids
 * are that handle's ids. Results as in ssh_query_device. SSH_ELENGTH if no
 * handle stores a query's length. All handles must live on the current device. */
ssh_status ssh_group_query_device(ssh_index* const* handles, int nh, const float* d_queries, const int32_t* lengths,
                                  int64_t nq, int k, int64_t* d_ids, float* d_dists, int32_t* d_which, void* stream);

/* ---- batched queries: one CUDA graph per plan ----
 *
 * A batch plan answers Algorithm 2 for many queries of mixed lengths over the
 * nh indexes `handles` at once (a query goes to the first handle that stores
 * series of its length, as in ssh_group_query_device). Every kernel of the
 * plan's pipeline runs on a fixed grid and reads the batch's sizes from device
 * memory, so the pipeline is captured once as a CUDA graph and replayed for
 * each batch; the first batch of a plan runs directly and the graph is
 * captured from it. After hashing and the candidate unions, the rerank of
 * every length class (LB_Keogh, the seed DTWs, the bound, the survivors' DTW
 * with early abandoning, the top-k) runs, for a batch of up to 512 queries,
 * as one persistent cooperative launch whose blocks claim work items of all
 * classes from device counters (DTW items at their class's autotuned tiling;
 * a grid-barrier wait that runs out, about 4 s, ends the batch with
 * SSH_ETIMEOUT), and for larger batches as per-class kernels, which fill the
 * GPU by themselves; a plan keeps a captured graph of each form.
 * ssh_batch_create allocates every device buffer: room for
 * max_queries queries (1 .. 65535), top-k with k <= 1024, and max_pairs
 * (query, candidate) pairs in total (0: max(2^20, 2048 max_queries)); a batch
 * with more candidates grows the pair buffers and reruns. The DTW tiling of
 * each (length, band radius) is chosen at creation by timing the candidate
 * tilings (cached for the process). After an add to or clear of any of the
 * indexes the next ssh_batch_query rebuilds the plan. The indexes must outlive
 * the plan; one plan serves one thread at a time.
 *
 * ssh_batch_query: queries back to back in device memory (d_queries, lengths
 * on the host); d_ids/d_dists [nq][k] and d_which [nq] (may be NULL) as in
 * ssh_group_query_device. It waits for `stream`'s earlier work, and returns
 * when the results are in place (work is ordered before later work on
 * `stream`). SSH_ELENGTH for a length no index stores, SSH_EINVAL for
 * nq > max_queries. ssh_batch_stats: pairs (candidates) and DTW pairs of the
 * last batch, the pair capacity, and the kernels in the captured graph. */
typedef struct ssh_batch ssh_batch;
ssh_status ssh_batch_create(ssh_index* const* handles, int nh, int64_t max_queries, int k, int64_t max_pairs,
                            ssh_batch** out);
ssh_status ssh_batch_query(ssh_batch* b, const float* d_queries, const int32_t* lengths, int64_t nq, int64_t* d_ids,
                           float* d_dists, int32_t* d_which, void* stream);
ssh_status ssh_batch_stats(const ssh_batch* b, int64_t* pairs, int64_t* dtw, int64_t* pair_capacity,
                           int32_t* graph_kernels);
/* The rerank's form: mode 1, the one persistent launch; 0, per-class kernels
 * (envelope and LB_Keogh per class, selections, filters, DTW per class and
 * pass, top-k); -1 (the default), persistent for batches of at most 512
 * queries (the serving loop's slots use per-class kernels: slots share the GPU). Both forms give the same results bit for bit. The first batch of a
 * form runs directly and captures its graph. SSH_EINVAL for another mode. */
ssh_status ssh_batch_set_persistent(ssh_batch* b, int32_t mode);
void ssh_batch_destroy(ssh_batch* b);

/* ---- serving loop with continuous batching ----
 *
 * A server answers queries submitted from any thread while inserts stream in.
 * One worker thread owns the indexes (callers must not use them while the
 * server runs) and keeps up to max_slots batch plans ("slots"; as many as fit
 * while reserve_bytes of device memory stay free, at least one). Whenever a
 * slot is free and queries wait, it takes up to max_batch of them, copies them
 * to the device and launches the slot's batch (a replay of its CUDA graph)
 * without waiting, so batches of several slots run on the GPU at once while
 * later arrivals queue. Inserts are applied between batches (admission of
 * queries pauses until the slots drain); the plans follow the grown tables.
 * A query of a given length gets the same rows whether it is served alone or
 * in a mix (batching changes neither its candidates nor its DTW).
 *
 * ssh_server_submit copies the queries (host, back to back) and returns one
 * ticket each; arrival_s (may be NULL: now) gives each query's arrival on the
 * server clock (ssh_server_now, seconds since creation) for latency. SSH_ELENGTH
 * for a length no index stores. ssh_server_insert copies host series; they are
 * appended to the index that serves their length (the first storing it, else
 * the first index) with ids from that index's sequence. ssh_server_wait blocks
 * until a ticket is done (SSH_ETIMEOUT after timeout_s) and gives its k ids,
 * distances, handle position and latency in ms; ssh_server_collect takes up to
 * max_n finished requests in completion order (waiting up to timeout_s for the
 * first), with ids [n][k], dists [n][k], latency_ms [n] and status [n] (any of
 * the output arrays may be NULL). ssh_server_flush waits until every submitted
 * query and insert is done. ssh_server_destroy finishes the queued work first. */
typedef struct ssh_server ssh_server;
typedef struct ssh_server_stats {
    int64_t slots;              /* batch plans admitted at creation */
    int64_t queries_submitted, queries_done, errors;
    int64_t batches, max_inflight;
    double mean_batch;          /* queries per batch */
    int64_t inserts_submitted, inserts_applied, insert_errors, insert_batches;
    double insert_latency_ms_sum; /* submit-to-applied time summed over insert calls */
    int64_t max_inflight_device;  /* most batches executing on the GPU at once (a launch counts the
                                     other slots whose batch had not finished on the device) */
    int64_t deferred;           /* queries put back in the queue because their batch's candidates
                                   would have grown the pair buffers past the free-memory reserve */
    int64_t refused;            /* queries answered SSH_EBUSY: alone in a batch, their candidates
                                   still needed more pair memory than the reserve admits */
} ssh_server_stats;
/* reserve_bytes: device memory kept free, both when slots are created and when a
 * slot's candidate (pair) buffers grow; a batch that would breach it is split
 * (its queries requeued, later batches admitted at half the size) and a single
 * query that still does not fit completes with SSH_EBUSY. */
ssh_status ssh_server_create(ssh_index* const* handles, int nh, int k, int max_batch, int max_slots,
                             int64_t reserve_bytes, ssh_server** out);
/* ssh_server_create with the first pair capacity of every slot (0: the batch plan default). */
ssh_status ssh_server_create_ex(ssh_index* const* handles, int nh, int k, int max_batch, int max_slots,
                                int64_t reserve_bytes, int64_t max_pairs, ssh_server** out);
double ssh_server_now(const ssh_server* s);
ssh_status ssh_server_submit(ssh_server* s, const float* queries, const int32_t* lengths, int64_t n,
                             const double* arrival_s, int64_t* tickets);
ssh_status ssh_server_insert(ssh_server* s, const float* series, const int32_t* lengths, int64_t count);
ssh_status ssh_server_wait(ssh_server* s, int64_t ticket, double timeout_s, int64_t* ids, float* dists,
                           int32_t* which, double* latency_ms);
ssh_status ssh_server_collect(ssh_server* s, int64_t max_n, double timeout_s, int64_t* tickets, int64_t* ids,
                              float* dists, double* latency_ms, int32_t* status, int64_t* n_out);
ssh_status ssh_server_flush(ssh_server* s, double timeout_s);
ssh_status ssh_server_get_stats(ssh_server* s, ssh_server_stats* out);
void ssh_server_destroy(ssh_server* s);

/* Options. SSH_OPT_LB_PRUNE (default 1): LB_Keogh pruning before DTW in the
 * rerank; 0 computes DTW for every candidate (same results, more work).
 * SSH_OPT_KERNEL_TIMING (default 0): record CUDA events around each kernel
 * group on the stream it runs on; read them with ssh_get_kernel_times.
 * SSH_OPT_HASH_KERNEL (default 0): 0 hashes with the kernel specialised for the
 * index's (W, delta) and series length when one is compiled in, 1 always with
 * the generic kernel (same results; a diagnostic and test knob).
 * SSH_OPT_EXACT_SCAN (default 0): 1 makes ssh_query / ssh_query_device rank every
 * stored series of the query's length instead of the hashed candidates: exact
 * banded-DTW top-k through the same reporting step (LB_Keogh filter and
 * early-abandoning DTW, as in the UCR suite the paper compares against); the
 * comparator without hashing. Batch plans and the server always hash.
 * SSH_OPT_CWS_FP64 (default 0): 1 decides every weighted minhash by the FP64
 * recomputation instead of the FP32 fast path (same results, much slower; a
 * test knob for the recomputation itself).
 * SSH_OPT_LB_CASCADE (default 1): with LB pruning on, the UCR-style cascade of
 * the plain query path (ssh_query, ssh_query_device, the group query and the
 * exact scan): 0 the query-envelope LB_Keogh alone; 1 with the LB_Kim endpoint
 * costs folded into it; 2 as 1, then the reversed LB_Keogh (the candidate's
 * envelope against the query) on the candidates that pass, before their DTW
 * (it prunes more but builds each candidate's envelope, which costs more than
 * the DTW it saves at the band radii measured, up to 102). Batch plans use 1.
 * Same results in every mode: all are lower bounds of the banded DTW.
 * SSH_OPT_MINHASH (default 0): the weighted minhash of Sec. 4.3's last step. 0 is
 * Ioffe's consistent weighted sampling (ICWS); 1 is densified one-permutation
 * hashing of the set's copies (k, c), c = 1 .. S_k, one of the faster variants
 * the paper cites: each copy goes to one of the K*L bins by one hash, a bin keeps
 * its smallest copy and empty bins borrow by optimal densification; its collision
 * probability per hash is the same weighted Jaccard, at O(copies + K L) work per
 * series instead of O(distinct shingles x K L). Hashes and keys differ from
 * ICWS's. Settable only while the index is empty (else SSH_EBUSY) and for
 * K*L <= 256 and n <= 16 (else SSH_ENOTSUP); needs a compiled sketch shape (adds
 * return SSH_ENOTSUP otherwise). */
typedef enum ssh_option {
    SSH_OPT_LB_PRUNE = 1,
    SSH_OPT_KERNEL_TIMING = 2,
    SSH_OPT_HASH_KERNEL = 3,
    SSH_OPT_CWS_FP64 = 4,
    SSH_OPT_EXACT_SCAN = 5,
    SSH_OPT_LB_CASCADE = 6,
    SSH_OPT_MINHASH = 7
} ssh_option;
ssh_status ssh_set_option(ssh_index* idx, ssh_option opt, int64_t value);

/* Counters since the last ssh_reset_stats (all cumulative). */
typedef struct ssh_stats {
    int64_t series_hashed;     /* series and queries hashed (Sec. 4.1-4.3) */
    int64_t sketch_fp64;       /* sketch windows near the sign boundary (|r.x| <= tau ||r|| ||x||), decided
                                  apart from the FP32 pass: by an error-bounded compensated FP32 dot product,
                                  else in FP64 */
    int64_t cws_fp64;          /* minhashes recomputed in FP64 (near ties / floor steps) */
    int64_t queries;           /* queries answered */
    int64_t candidates;        /* sum over queries of |R| (Alg. 2 union) */
    int64_t dtw_computed;      /* candidates whose DTW was computed */
    int64_t lb_pruned;         /* candidates pruned by LB_Keogh */
    int64_t kernel_launches;   /* kernels launched by calls on this index */
    int64_t lb2_pruned;        /* of lb_pruned: candidates that passed LB_Keogh and were pruned by the
                                  reversed LB_Keogh (SSH_OPT_LB_CASCADE) */
    int64_t lb2_skipped;       /* queries whose requested reversed LB_Keogh pass (SSH_OPT_LB_CASCADE 2)
                                  did not run because the candidate envelopes of one series length do not
                                  fit in shared memory; their survivors all went to DTW (same results) */
} ssh_stats;
ssh_status ssh_get_stats(const ssh_index* idx, ssh_stats* out);
ssh_status ssh_reset_stats(ssh_index* idx);

/* Device time per kernel group since the last ssh_reset_stats, measured with
 * CUDA events while SSH_OPT_KERNEL_TIMING is on. Groups (prefix "add." for
 * ssh_index_add*, "query." for ssh_query*): "sketch", "sketch_fixup", "shingle",
 * "cws", "hash_generic" (units: series), "table_sort" (table entries),
 * "probe_union" (queries x tables), "lb_keogh" (candidate samples read),
 * "dtw" (DTW cells), "topk" (candidates).
 * Writes up to `cap` records to out and their number to *count; synchronises
 * on the recorded events. */
typedef struct ssh_kernel_time {
    char name[24];
    int64_t launches;   /* kernel launches in the group */
    int64_t calls;      /* timed regions (one region may launch several kernels) */
    double total_ms;    /* summed event time of the regions */
    double units;       /* work units processed (see above) */
} ssh_kernel_time;
ssh_status ssh_get_kernel_times(ssh_index* idx, ssh_kernel_time* out, int cap, int* count);

/* ---------------------------------------------------------------------------
 * Stage entry points. They run one step of the path on device buffers so that
 * each step can be checked and timed on its own; the index calls the same
 * kernels internally.
 * ------------------------------------------------------------------------- */

/* Sec. 4.1-4.3 plus the bucket keys of Alg. 1 for `count` series of length m
 * stored row-major at d_series (row stride m floats). Outputs (each may be NULL):
 *   d_bits    [count][ceil(N_B/32)] uint32, window i of a series is bit
 *             (31 - i%32) of word i/32, 1 for r.x >= 0; N_B = floor((m-W)/delta)+1
 *   d_sh_ids, d_sh_counts  [count][S] uint32, the distinct shingle ids of a
 *             series in ascending order and their counts, S = N_B - n + 1 slots
 *             per series, the first d_nnz[i] used
 *   d_nnz     [count] int32
 *   d_kstar, d_tstar  [count][K*L] uint32, the minhash (k*, t*) of each hash
 *   d_keys    [L][count] uint64, the bucket key of each table
 * SSH_ELENGTH if m gives no shingle or more than 65535. */
ssh_status ssh_hash_device(const ssh_index* idx, const float* d_series, int32_t m, int64_t count, void* stream,
                           uint32_t* d_bits, uint32_t* d_sh_ids, uint32_t* d_sh_counts, int32_t* d_nnz,
                           uint32_t* d_kstar, uint32_t* d_tstar, uint64_t* d_keys);

/* Size of the fixed device scratch used by ssh_hash_device_noalloc (16 MiB).
 * Every GPU on which the library's device code is loaded holds it until the
 * process exits. */
#define SSH_NOALLOC_SCRATCH_BYTES (16u << 20)

/* ssh_hash_device without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as a
 * process whose device memory is all handed out by another framework's pool
 * (an extra cudaMalloc could fail or fragment that pool), or a latency-bound
 * loop that must not pay for, or fail on, a device allocation while it runs.
 *
 * Arguments, outputs and results are those of ssh_hash_device. The working
 * buffers of the sketch / fix-up / shingle / minhash kernels live in one static
 * device array of SSH_NOALLOC_SCRATCH_BYTES bytes instead of memory allocated
 * per call. That limits how many series one call may hash (about 27,000 series
 * of length 512 with W = 80, delta = 3, n = 15): a larger count returns
 * SSH_EINVAL with the limit in ssh_last_error(), and nothing runs. Shapes for
 * which no specialised kernels are compiled run the single-kernel path, which
 * needs no scratch at all. The call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *
 * The first call on a device looks up the array's device address (the CUDA
 * symbol lookup, with that device current); make that first call before any
 * stream capture. Every call on a device uses the same array, which keeps the
 * previous call's contents, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
ssh_status ssh_hash_device_noalloc(const ssh_index* idx, const float* d_series, int32_t m, int64_t count,
                                   void* stream, uint32_t* d_bits, uint32_t* d_sh_ids, uint32_t* d_sh_counts,
                                   int32_t* d_nnz, uint32_t* d_kstar, uint32_t* d_tstar, uint64_t* d_keys);

/* Sec. 2.1 banded DTW for `npairs` pairs: d_out[p] = DTW(d_a + a_idx[p]*m, d_b + b_idx[p]*m)
 * with radius rb (0 <= rb < m), sum of squared costs. d_a_idx / d_b_idx are
 * int64 device arrays of row indexes into the row-major [*, m] arrays d_a, d_b.
 * Rows that share an a-row are best given consecutively. */
ssh_status ssh_dtw_device(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                          int64_t npairs, int32_t m, int32_t rb, float* d_out, void* stream);

/* ssh_dtw_device with an explicit tiling instead of the one the library's autotuner
 * picks for (m, rb): S band slots per lane (8, 14 or 26) and the kernel variant
 * (0, the only one built). Every tiling computes each cell from the same three
 * values in the same order, so all give the same distances bit for bit.
 * SSH_ENOTSUP for a tiling that is not compiled or needs more than 32 lanes per
 * pair at this radius. */
ssh_status ssh_dtw_device_tiled(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                                int64_t npairs, int32_t m, int32_t rb, int32_t S, int32_t variant, float* d_out,
                                void* stream);

/* Sec. 3 LB_Keogh for `npairs` pairs: d_out[p] = LB_Keogh of row d_b_idx[p] of d_b
 * against the envelope (radius rb) of row d_a_idx[p] of d_a. */
ssh_status ssh_lb_keogh_device(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                               int64_t npairs, int32_t m, int32_t rb, float* d_out, void* stream);

/* Lower bounds of the banded DTW for `npairs` pairs (a = query rows, b =
 * candidate rows, as in ssh_dtw_device), chosen by `kind`:
 *   0: LB_Keogh (Sec. 3): the envelope (radius rb) of the a-row against the
 *      b-row's samples, sum of squared excursions (= ssh_lb_keogh_device);
 *   1: kind 0 with the terms of samples 0 and m-1 replaced by the exact costs
 *      of the first and last cells, (a_0 - b_0)^2 and (a_{m-1} - b_{m-1})^2
 *      (the LB_Kim endpoint bound of the UCR suite folded into LB_Keogh);
 *   2: reversed LB_Keogh: the envelope of the b-row against the a-row's samples.
 * d_out[p] receives the bound of pair p. SSH_EINVAL for another kind or bad
 * sizes. */
ssh_status ssh_lb_bound_device(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                               int64_t npairs, int32_t m, int32_t rb, int32_t kind, float* d_out, void* stream);

/* ---- measurement-only export ----
 *
 * Not part of the method and not used by any other entry point: it gives the
 * benchmark the L2 read bandwidth that bounds the minhash kernel's gathers.
 * Reads the `bytes` bytes at d_buf
 * (16-byte aligned, bytes a multiple of 16) `passes` times in one kernel launch
 * on `stream`, with loads that bypass L1, and returns once the launch is enqueued.
 * A buffer that fits in L2 gives the L2 read bandwidth when the caller times the
 * launch with events on that stream: bytes * passes / time. The buffer is only
 * read. SSH_EINVAL for a null or unaligned buffer, a size that is zero or not a
 * multiple of 16, or passes < 1; SSH_ECUDA if the launch fails. */
ssh_status ssh_read_device(const void* d_buf, uint64_t bytes, int32_t passes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SSH_H */
