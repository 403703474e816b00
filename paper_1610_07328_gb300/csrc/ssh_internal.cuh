// ssh_internal.cuh -- internal declarations of the GB300 SSH library.
// Everything here is private to the library; the public surface is include/ssh.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "ssh.h"

struct ssh_index;
struct ssh_batch;

namespace ssh {

// ------------------------------------------------------------------ errors

void set_error(const char* fmt, ...);
ssh_status cuda_status(cudaError_t e, const char* what);
// set_error(fmt, ...) and return s
ssh_status fail_status(ssh_status s, const char* fmt, ...);
// Make the index's device current.
ssh_status check_device(const ssh_index* idx);

#define SSH_TRY(expr)                       \
    do {                                    \
        ssh_status _s = (expr);             \
        if (_s != SSH_OK) return _s;        \
    } while (0)

#define SSH_CUDA(expr)                                              \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return ::ssh::cuda_status(_e, #expr); \
    } while (0)

// Kernel launches made by this library in the calling process (all threads),
// and by the calling thread alone (per-call counts take differences of the
// latter, so calls on other threads do not inflate them).
extern std::atomic<long long> g_launches;
extern thread_local long long t_launches;
inline void note_launch(int n = 1) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}

// ------------------------------------------------------------- constants

// Value given to series samples outside [0, m) in the DTW wavefront. Any cost
// involving it is >= 1e36, far above every real path cost, so cells outside
// the grid never win a min (inputs are bounded by 1e15).
constexpr float kPad = 1.0e18f;

constexpr int kMaxShingleBits = 16;     // n limit of the tabulated minhash draws
constexpr int kMaxCount = 65535;        // shingles per series (u16 counts)
// Row stride (in hashes) of the per-shingle ln a / t tables: K L rounded up to
// 4, so a lane's 4 consecutive hashes are one aligned 16-byte (or 4-byte) load.
inline int tab_stride_of(int KL) { return (KL + 3) & ~3; }
// Row stride (in hashes) of the u16 rank table: K L rounded up to 64, so every
// row starts on a 128-byte line and a row's read touches the fewest lines and
// sectors; a lane's 4 consecutive ranks are one aligned 8-byte load.
inline int rank_stride_of(int KL) { return (KL + 63) & ~63; }
constexpr int kMaxTopK = 1024;
// The rerank's seeds are the kSeedFactor k candidates of smallest LB_Keogh; the
// k-th smallest DTW among them bounds the k-th best distance (pruning and early
// abandoning against it never change the result; more seeds give a tighter bound).
constexpr int kSeedFactor = 16;
constexpr int kTabCounts = 8;           // counts whose ln a is tabulated exactly rounded
constexpr int kMaxW = 8192;
constexpr int kMaxKL = 4096;

// Device-side counters (one array of these per index).
enum StatSlot { kStatSketch64 = 0, kStatCws64 = 1, kNumStatSlots = 4 };

// ----------------------------------------------------- hash kernel params

struct HashArgs {
    const float* series;     // row-major series, row i at series + i * stride ...
    int64_t stride;          // floats between consecutive rows
    const float* const* rows;// ... unless rows != NULL: row i at rows[i]
    int64_t count;           // rows to hash
    int m, W, delta, n, nb, nwords, S, K, L, KL;
    const float* r;          // [W] filter (device)
    const float* r_host;     // [W] the same filter in host memory
    float tau_norm;          // threshold factor tau * ||r|| (rounded up)
    float gamma_ss;          // relative inflation of the FP32 sum of squares
    const uint16_t* rank;    // [2^n][rank_stride] rank of the count-1 value of (j, k) among all k
    int rank_stride;         // KL rounded up to a multiple of 64 (row padding holds 0xFFFF)
    int force_generic;       // 1: use the generic kernel even when a specialised one exists
    int force_fp64;          // 1: decide every minhash by the FP64 recomputation (a test knob)
    int minhash;             // 0: ICWS (Sec. 4.3); 1: densified one-permutation hashing of the copies
    const uint2* kla;        // [KL][2^n] per rank: (shingle id, ln a at count 1 rounded once to FP32, as bits)
    const float4* p32;       // [2^n][KL] (r, 1/r, beta, ln c) rounded to FP32
    const double* p64;       // [KL][2^n][3] (r, beta, ln c) in FP64
    const float* lav;        // [2^n][kTabCounts][tab_stride] ln a of counts 1..kTabCounts, rounded once to FP32
    const uint8_t* tsm;      // [2^n][kTabCounts-1][tab_stride] t of counts 2..kTabCounts (255: not tabulated)
    int tab_stride;          // KL rounded up to a multiple of 4
    const float* lns32;      // [kMaxCount+1] ln s rounded to FP32
    const double* lns64;     // [kMaxCount+1] ln s in FP64
    uint64_t seed;
    // optional device [2] (first, end): hash rows first .. end-1 of `rows`/`series`
    // (at most `count` of them; keys at column key_col0 + row). NULL: rows 0 .. count-1.
    const int64_t* dev_range;
    uint64_t* keys;          // [L][key_stride], row i of this launch at column key_col0 + i
    int64_t key_stride;
    int64_t key_col0;
    // optional per-stage outputs
    uint32_t* bits_out;
    uint32_t* sh_ids_out;
    uint32_t* sh_counts_out;
    int32_t* nnz_out;
    uint32_t* kstar_out;
    uint32_t* tstar_out;
    unsigned long long* stats;
};

bool hash_fast_supported(const HashArgs& a);
// Sec. 4.3 draw tables of an index (and its ln s tables), built on the GPU on
// `st` (draws.cu); for n > kMaxShingleBits only ln s (draws are computed on the fly).
ssh_status build_draw_tables(ssh_index* idx, cudaStream_t st);
cudaError_t launch_hash_fast(const HashArgs& a, cudaStream_t st);

// Windows of one stream (row k = samples [k step, k step + m)): the sketch bits
// and shingle ids of every stream position computed once, then the windows'
// sets and the minhash. Stages 0 sketch, 1 FP64 fix-up, 2 ids and sets, 3 CWS
// and keys, over one scratch block of hash_windows_scratch_bytes(a, step) bytes;
// a.count = windows, a.keys / key_stride / key_col0 as for rows.
// The SRP baseline's hash (srp.cu): stages 0 bits, 1 FP64 fix-up, 2 keys, over
// srp_scratch_bytes(a) bytes of scratch; R / rn from the index's SrpTab for a.m.
size_t srp_scratch_bytes(const HashArgs& a);
cudaError_t launch_srp_hash(const HashArgs& a, const float* R, const float* rn, void* scratch, int stage,
                            cudaStream_t st);

bool hash_windows_supported(const HashArgs& a);
size_t hash_windows_scratch_bytes(const HashArgs& a, int64_t step);
cudaError_t hash_windows_stage(const HashArgs& a, const float* stream, int64_t step, void* scratch, int stage,
                               cudaStream_t st);

// The specialised hash path in stages (sketch -> FP64 fix-up -> shingle -> CWS)
// over one scratch block of hash_fast_scratch_bytes(a) bytes.
struct FastHashBuffers {
    uint32_t* bits;
    unsigned long long* nfix;
    unsigned long long* fix;
    unsigned long long fix_cap;
    uint32_t* sets;
    int2* sizes;
};
size_t hash_fast_scratch_bytes(const HashArgs& a);
FastHashBuffers hash_fast_buffers(const HashArgs& a, void* scratch);
cudaError_t hash_fast_sketch(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st);
cudaError_t hash_fast_fixup(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st);
cudaError_t hash_fast_shingle(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st);
cudaError_t hash_fast_cws(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st);
cudaError_t launch_hash_generic(const HashArgs& a, cudaStream_t st);
int hash_smem_bytes_per_warp(int m, int nwords, int S, int KL);

// Hash arguments of an index for series of length m (filter, draw tables,
// geometry); SSH_ELENGTH if m gives no shingle or too many.
ssh_status prepare_hash_args(const ssh_index* idx, int m, HashArgs* a);
int hash_warps_per_cta(int m, int nwords, int S, int KL);
cudaError_t launch_hash(const HashArgs& a, cudaStream_t st);

// ------------------------------------------------------------ bucket tables

// Bucket tables: per table, the (key, row) pairs of rows row0 .. row0+n-1
// (keys[l][row], row stride cap) partitioned into 2^bin_bits bins by the top
// bin_bits key bits into skeys/srows[l][0 .. n) (table stride out_stride);
// bins[l][b] .. bins[l][b+1] is bin b.
int table_bin_bits(int64_t n);
cudaError_t build_tables(const uint64_t* keys, int64_t row0, int64_t n, int L, int64_t cap, int64_t out_stride,
                         int bin_bits, uint32_t* bins, uint32_t* cursor, uint64_t* skeys, uint32_t* srows,
                         cudaStream_t st);

// -------------------------------------------------------------- queries

struct ProbeArgs {
    const uint64_t* qkeys;     // [L][nq]
    int64_t nq, L;
    const uint64_t* skeys;     // [L][cap] keys of the sub-index grouped by bin
    const uint32_t* srows;     // [L][cap] rows in the same order
    const uint32_t* bins;      // [L][2^bin_bits + 1] bin starts
    int bin_bits;
    int64_t cap, nrows;
    uint32_t* bitmap;          // [nq][words] candidate bitmap
    int64_t words;
    // the delta tables of the rows added since the main tables were built
    const uint64_t* dkeys;     // [L][dcap]
    const uint32_t* drows;     // [L][dcap]
    const uint32_t* dbins;     // [L][2^dbin_bits + 1]
    int dbin_bits;
    int64_t dcap, dcount;      // dcount = 0: no delta
};
cudaError_t launch_probe_union(const ProbeArgs& a, cudaStream_t st);
cudaError_t launch_bitmap_count(const uint32_t* bitmap, int64_t nq, int64_t words, int64_t* counts,
                                cudaStream_t st);
cudaError_t launch_bitmap_compact(const uint32_t* bitmap, int64_t nq, int64_t words, const int64_t* offsets,
                                  uint32_t* cand_rows, int32_t* cand_query, cudaStream_t st);

// A set of (query, candidate) pairs grouped by query: segment s has query
// series seg_a[s] (m floats) and pairs [seg_begin[s], seg_begin[s+1]); pair p
// compares seg_a[s] with pair_b[p] and writes out[pair_slot ? pair_slot[p] : p].
struct PairSet {
    const int64_t* seg_begin;   // [nseg + 1] device
    int64_t nseg;
    const float* const* seg_a;  // [nseg] device
    const float* const* pair_b; // [npairs] device
    const int64_t* pair_slot;   // [npairs] device, or NULL
    int64_t max_seg_pairs;      // upper bound of any segment's size (grid sizing)
    // optional device [2] (first, end): process only segments first .. end-1
    // (the launch then strides over them with its fixed grid). NULL: all nseg.
    const int64_t* seg_range = nullptr;
    int64_t env_stride = 0;     // floats between segments' envelopes (0: m)
    int64_t grid_y = 0;         // blocks striding over the segments (0: one per segment)
    // optional [nseg] per-segment bound (float bits; all ones: none): DTW stops a
    // warp's pairs once all of them certainly exceed it (distance reported +inf)
    const uint32_t* abandon = nullptr;
    float abandon_shrink = 1.f; // relative FP32 rounding margin of a path cost (1 - 4 (m + 3) 2^-24)
    // optional device counter: every pair adds the blocks of wavefront steps it ran
    // (all of them when it finishes, fewer when it is abandoned); see dtw_plan_blocks
    unsigned long long* blocks_done = nullptr;
};

cudaError_t launch_envelope(const float* const* seg_a, int64_t nseg, int m, int rb, float* upper, float* lower,
                            cudaStream_t st, const int64_t* seg_range = nullptr, int64_t env_stride = 0);
// kim: the endpoint samples take the exact first / last cell costs (LB_Kim folded in)
cudaError_t launch_lb_keogh(const PairSet& ps, const float* upper, const float* lower, int m, float* out,
                            cudaStream_t st, bool kim = false);
// Reversed LB_Keogh (the candidate's envelope, the query's samples). With U (per
// segment bound bits): clears pair_mut[p] of pairs whose LB * shrink > U and
// counts them in *pruned; without: writes out[slot].
// Whether the reversed LB_Keogh pass fits in shared memory at this (m, r_b).
bool lb_rev_fits(int m, int rb);
cudaError_t launch_lb_rev(const PairSet& ps, int m, int rb, float* out, const uint32_t* U, float shrink,
                          const float** pair_mut, unsigned long long* pruned, cudaStream_t st);

// A DTW tiling: S band slots per lane, G lanes per pair, the slot forced to +inf,
// and the kernel variant (0, the wavefront with paired square-adds, is the one built).
struct DtwPlan {
    int S, G, pmask;
    int variant = 0;
};
DtwPlan dtw_plan(int m, int rb);
bool dtw_tiling_compiled(int S, int variant);
// The plan of slot count S and variant at radius rb (S == 0: not compiled or too wide).
DtwPlan dtw_plan_for(int rb, int S, int variant);
// The tiling used for (m, rb): timed once per process over the candidate slot
// counts (the first call for a (m, rb) runs the timing on `st` and waits for it).
DtwPlan dtw_tuned_plan(int m, int rb, cudaStream_t st);
cudaError_t launch_dtw(const PairSet& ps, int m, int rb, float* out, cudaStream_t st);
// Blocks of wavefront steps a complete DTW of one pair takes under a plan: the
// cells a pair computed are blocks_done / dtw_plan_blocks of its m(2r+1) - r(r+1).
int64_t dtw_plan_blocks(int m, int rb, const DtwPlan& pl);
cudaError_t launch_dtw_plan(const PairSet& ps, int m, int rb, const DtwPlan& pl, float* out, cudaStream_t st);

// Raise (never lower) a kernel's dynamic shared memory limit on the current
// device to `bytes`: a launch captured in a CUDA graph keeps its size, so the
// limit must not drop below it later.
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes);

// Candidate filter of the rerank (one segment per query): mode 0 keeps the
// pairs with lb <= T[s] (the seeds), mode 1 those with T[s] < lb and
// lb * shrink <= U[s] (the survivors). Writes the kept pairs' candidate
// pointers and original slots segment by segment, begin[0 .. nseg] the
// offsets and *total their number. Grid: max_seg bounds a segment's size.
struct FilterArgs {
    const int64_t* seg_begin;
    int64_t nseg, max_seg;
    const float* lb;
    const uint32_t *T, *U;
    float shrink;
    int mode;
    int64_t* count;                 // [nseg] scratch
    unsigned long long* cursor;     // [nseg] scratch
    int64_t* begin;                 // [nseg + 1] out
    unsigned long long* total;      // [1] out (may be NULL)
    const float* const* pair_b;
    const float** pair_b_out;
    int64_t* slot_out;
};
cudaError_t launch_filter(const FilterArgs& f, cudaStream_t st);
cudaError_t launch_fill_f32(float* p, int64_t n, const int64_t* n_dev, float v, cudaStream_t st);
// Exclusive prefix sums (one block); cap > 0: a total above cap zeroes every
// offset and sets *overflow.
cudaError_t launch_scan(const int64_t* counts, int64_t n, int64_t* out, int64_t cap, unsigned long long* total_out,
                        unsigned long long* overflow, cudaStream_t st);
cudaError_t launch_topk_keys(const float* dist, const uint32_t* rows, int64_t n, const int64_t* n_dev, uint64_t* keys,
                             cudaStream_t st);
// Where the top-k of segment s goes: ids/dists rows qpos[s] (k each), the id of
// row r is gid[r] (or seg_gid[s][r]); which[qpos[s]] = seg_which[s] when which
// is given; segments at or past *nseg_dev (when given) are skipped.
struct TopkOut {
    int64_t* ids;
    float* dists;
    const int64_t* qpos;
    const int64_t* gid;
    const int64_t* const* seg_gid;
    int32_t* which;
    const int32_t* seg_which;
    const int64_t* nseg_dev;
};
cudaError_t launch_topk_output(const TopkOut& o, const uint64_t* keys, const int64_t* seg_begin, const uint64_t* kth,
                               int64_t nseg, int k, cudaStream_t st);

// The whole rerank of a batch plan in one persistent cooperative launch
// (batch_rerank.cu): per length class its length, radius and DTW tiling.
struct RerankClass {
    int m, rb, S, G, pmask;
    int64_t dtw_chunk;  // pairs per DTW work item
};
struct RerankArgs {
    const int64_t* nq;                // [1] queries of the batch (sorted by class)
    const int32_t* q_cls;             // [Q] class of each sorted query
    const float* const* q_ptr;        // [Q] query samples
    const RerankClass* cls;           // [C]
    const int64_t* seg_begin;         // [Q + 1] each query's candidate pairs
    const float** pair_b;             // [P] candidate rows
    const uint32_t* cand_rows;        // [P] their rows in the class's sub-index
    float *upper, *lower;             // [Q][env_stride] envelopes
    int64_t env_stride;
    float* lb;                        // [P]
    float* dist;                      // [P], +inf on entry
    const float** fb;                 // [P] the pass's pairs
    int64_t* fslot;                   // [P] their slots
    int64_t* fcount;                  // [Q]
    unsigned long long* fcursor;      // [Q]
    int64_t* fbegin;                  // [Q + 1]
    const int64_t* cls_begin;         // [C + 1] first sorted query of each class
    int C;                            // classes
    int64_t* item_off;                // [2 (C + 1)] item layouts of the LB pass and of a DTW pass
    uint32_t *T, *U;                  // [Q]
    int k;
    float shrink;
    TopkOut out;
    unsigned long long* dtw_counts;   // [2] pairs of the seed and survivor passes (added)
    const unsigned long long* overflow;
    unsigned long long* work;         // [kRerankWork] item counters, zero on entry
    unsigned* bar;                    // [2] grid barrier (count zero on entry, generation)
    unsigned* err;                    // set when a barrier wait ran out (zero on entry)
};
constexpr int kRerankWork = 12;
// Batches of at most this many queries rerank in the persistent launch by default
// (measured on mixed lengths 128 .. 2048: 1.07x faster at 64 queries, 1.67x at 256,
// 1.12x slower at 1024 and 1.49x slower at 4096, where per-class kernels fill the
// GPU by themselves).
constexpr int64_t kPersistentMaxQueries = 512;
size_t rerank_smem_bytes(int max_m);
int rerank_dtw_chunk(const DtwPlan& pl);
cudaError_t launch_rerank(const RerankArgs& a, int max_m, cudaStream_t st, int* grid_out);

// Batch plans, asynchronously (the server's slots): prepare writes the query
// table (queries back to back at d_queries), launch starts the batch on the
// plan's stream, done polls it, finish waits (and reruns an overflowed batch),
// outputs are the plan's device result rows in caller order.
ssh_status batch_prepare(ssh_batch* b, const float* d_queries, const int32_t* lengths, int64_t nq);
ssh_status batch_launch(ssh_batch* b);
bool batch_done(ssh_batch* b);
// Wait for the launched batch; on pair-buffer overflow grow the buffers and run
// it again. reserve_bytes >= 0: grow only while that much device memory stays
// free after the growth, else return SSH_EBUSY (nothing ranked; the plan stays
// valid for smaller batches). reserve_bytes < 0: grow unconditionally.
ssh_status batch_finish(ssh_batch* b, int64_t reserve_bytes = -1);
// Device bytes of one candidate pair in a plan's pair buffers.
constexpr int64_t kBatchPairBytes = 44;
ssh_status batch_refresh(ssh_batch* b);
void batch_outputs(const ssh_batch* b, const int64_t** ids, const float** dists, const int32_t** which);
cudaStream_t batch_stream(const ssh_batch* b);
size_t batch_device_bytes(const ssh_batch* b);
ssh_status batch_query_into(ssh_batch* b, const float* d_queries, const int32_t* lengths, int64_t nq,
                            int64_t* d_ids, float* d_dists, int32_t* d_which, cudaStream_t us);
int64_t batch_capacity(const ssh_batch* b);
int batch_k(const ssh_batch* b);

// k-th smallest key of each segment (keys read through `keys`, segment s is
// [seg_begin[s], seg_begin[s+1])); kth_out[s] = that key, or all-ones if the
// segment has fewer than k items.
cudaError_t launch_select_kth_u32(const uint32_t* keys, const int64_t* seg_begin, int64_t nseg, int k,
                                  uint32_t* kth_out, cudaStream_t st);
cudaError_t launch_select_kth_u64(const uint64_t* keys, const int64_t* seg_begin, int64_t nseg, int k,
                                  uint64_t* kth_out, cudaStream_t st);

}  // namespace ssh

// --------------------------------------------------------------- the index

struct SubIndex {
    int m = 0, nb = 0, nwords = 0, S = 0, rb = 0;
    int64_t count = 0, cap = 0;
    const float** row_ptr = nullptr;  // [cap] device: series pointer of each row
    int64_t* gid = nullptr;           // [cap] device: id of each row
    uint64_t* keys = nullptr;         // [L][cap] device: bucket keys by row
    uint64_t* skeys = nullptr;        // [L][cap] device: keys grouped by bin
    uint32_t* srows = nullptr;        // [L][cap] device: rows in the same order
    uint32_t* bins = nullptr;         // [L][2^bin_bits + 1] device: bin starts
    int bin_bits = 0, bins_alloc_bits = 0;
    // Rows [0, main_count) are in the main tables above; rows added later are in
    // the delta tables below (binned the same way, rows absolute) until the
    // delta outgrows an eighth of the main part and everything is rebinned.
    int64_t main_count = 0, dcount = 0, dcap = 0;
    uint64_t* dkeys = nullptr;        // [L][dcap]
    uint32_t* drows = nullptr;        // [L][dcap]
    uint32_t* dbins = nullptr;        // [L][2^dbin_bits + 1]
    int dbin_bits = 0, dbins_alloc_bits = 0;
};

struct KernelTimer {
    std::string name;
    cudaEvent_t start, stop;
    int launches;
    double units;
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool arena = false;  // carved from the index's arena (not freed on its own)
};

struct KernelTotals {
    int64_t launches = 0, calls = 0;
    double ms = 0.0, units = 0.0;
};

// The SRP baseline's projections for one series length m (device): R [KL][m]
// and rn[j] = tau_m ||r_j||, rounded up.
struct SrpTab {
    float* R = nullptr;
    float* rn = nullptr;
};

struct ssh_index {
    int W = 0, delta = 0, n = 0, K = 0, L = 0, KL = 0;
    int family = 0;                   // 0: SSH; 1: the SRP baseline (ssh_create_srp)
    int minhash = 0;                  // SSH_OPT_MINHASH: 0 ICWS, 1 densified one-permutation hashing
    std::map<int, SrpTab> srp;        // family 1: projections per series length
    bool timing = false;
    std::vector<KernelTimer> pending;
    std::map<std::string, KernelTotals> totals;
    float band = 0.f;
    uint64_t seed = 0;
    int device = 0;
    bool lb_prune = true;
    bool exact_scan = false;          // queries rank every stored series (no hashing)
    int lb_cascade = 1;               // SSH_OPT_LB_CASCADE: 0 none, 1 LB_Kim endpoints, 2 + reversed LB_Keogh
    int hash_kernel = 0;              // 0: fastest available, 1: always the generic kernel
    int cws_fp64 = 0;                 // 1: every minhash through the FP64 recomputation
    float tau_norm = 0.f;
    std::vector<float> h_r;           // host copy of the filter
    float* d_r = nullptr;
    uint16_t* d_rank = nullptr;
    uint2* d_kla = nullptr;
    float4* d_p32 = nullptr;
    double* d_p64 = nullptr;
    float* d_lav = nullptr;
    uint8_t* d_tsm = nullptr;
    float* d_lns32 = nullptr;
    double* d_lns64 = nullptr;
    unsigned long long* d_stats = nullptr;
    std::map<int, SubIndex> subs;
    int64_t next_id = 0;
    ssh_stats host_stats{};
    // series copies made by the library (host adds, non-borrowed device adds):
    // `owned` are referenced by stored rows; ssh_index_clear moves them to
    // `spare`, from which later host adds take their staging buffer
    std::vector<DevBuf> owned, spare;
    // small series copies (streamed inserts) are carved from arena chunks of
    // kArenaChunk bytes in order; ssh_index_clear rewinds to the first chunk
    std::vector<void*> arena;
    size_t arena_cur = 0, arena_off = 0;
    // host-API calls run on these non-blocking streams: hstream hashes and
    // queries, cstream copies host series in chunks ahead of the hashing
    cudaStream_t hstream = nullptr, cstream = nullptr;
    cudaEvent_t cevent = nullptr;
    unsigned long long* h_pinned = nullptr;  // small pinned host buffer for per-call device counters
    // recorded after the work of the latest add: device adds return once their
    // work is enqueued, and every query waits for this event on its own stream
    cudaEvent_t ready = nullptr;

    uint64_t version = 0;                    // bumped by every add and clear (batch plans check it)
};
