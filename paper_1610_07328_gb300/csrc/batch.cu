// batch.cu -- Algorithm 2 for a batch of queries of mixed lengths over several
// indexes, captured once as a CUDA graph and replayed for every batch.
//
// A plan fixes the classes (one per series length stored by the indexes; a
// length stored by several indexes goes to the first of them) and the buffer
// capacities: queries, candidate pairs, table and envelope strides. Every
// kernel of the pipeline runs on a fixed grid and takes the batch's sizes
// from device memory -- the query table (sorted by class), the class ranges,
// and the candidate offsets the pipeline computes itself -- so one captured
// graph serves any batch of the plan. The host writes the query table into
// pinned memory; the graph copies it in, hashes each class's queries (Sec.
// 4.1-4.3, with the specialised kernels where the class's shape has them),
// probes and unions the buckets (Algorithm 2), bounds the candidates
// by LB_Keogh (Sec. 3) and reranks them by banded DTW (Sec. 2.1) with the
// tiling the autotuner chose for the class's (length, radius), and writes the
// top-k. A batch whose candidates exceed the pair capacity sets a flag; the
// host then grows the capacity, captures again and reruns that batch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "ssh_internal.cuh"

namespace ssh {
namespace {

// One class on the device: the bucket tables and rows of one sub-index.
struct ClassDev {
    const uint64_t* skeys;
    const uint32_t* srows;
    const uint32_t* bins;
    const float* const* row_ptr;
    int64_t cap, nrows, words;
    int bin_bits, L;
    // delta tables (rows added since the main tables were built)
    const uint64_t* dkeys;
    const uint32_t* drows;
    const uint32_t* dbins;
    int64_t dcap, dcount;
    int dbin_bits;
};

ClassDev class_dev(const SubIndex& s, int L) {
    ClassDev d;
    d.skeys = s.skeys;
    d.srows = s.srows;
    d.bins = s.bins;
    d.row_ptr = s.row_ptr;
    d.cap = s.cap;
    d.nrows = s.count;
    d.words = (s.count + 31) / 32;
    d.bin_bits = s.bin_bits;
    d.L = L;
    d.dkeys = s.dkeys;
    d.drows = s.drows;
    d.dbins = s.dbins;
    d.dcap = s.dcap;
    d.dcount = s.dcount;
    d.dbin_bits = s.dbin_bits;
    return d;
}

// Device counters the host reads after a batch.
struct BatchStatus {
    unsigned long long pairs;     // candidates of the batch (counted even when over capacity)
    unsigned long long overflow;  // 1: pairs > capacity, nothing was ranked
    unsigned long long dtw[2];    // DTW pairs of the seed and survivor passes
    // the persistent rerank's work counters and grid barrier (zero on entry), and
    // its error flag (a barrier wait ran out)
    unsigned long long rr_work[kRerankWork];
    unsigned rr_bar[2];
    unsigned rr_err;
    unsigned rr_pad;
};

// The query table, in the order of the sorted queries (class by class).
struct PlanView {
    int64_t* nq;              // [1]
    int64_t* cls_begin;       // [C + 1] first sorted query of each class
    const float** q_ptr;      // [qcap] query samples
    int32_t* q_cls;           // [qcap] class
    int64_t* q_pos;           // [qcap] position in the caller's batch
    const int64_t** q_gid;    // [qcap] ids of the class's rows
    int32_t* q_which;         // [qcap] index (among the handles) the query went to
    size_t bytes;
};

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

PlanView plan_view(unsigned char* base, int64_t qcap, int C) {
    PlanView v;
    size_t off = 0;
    v.nq = reinterpret_cast<int64_t*>(base + off); off += a256(8);
    v.cls_begin = reinterpret_cast<int64_t*>(base + off); off += a256(8 * (size_t)(C + 1));
    v.q_ptr = reinterpret_cast<const float**>(base + off); off += a256(8 * (size_t)qcap);
    v.q_cls = reinterpret_cast<int32_t*>(base + off); off += a256(4 * (size_t)qcap);
    v.q_pos = reinterpret_cast<int64_t*>(base + off); off += a256(8 * (size_t)qcap);
    v.q_gid = reinterpret_cast<const int64_t**>(base + off); off += a256(8 * (size_t)qcap);
    v.q_which = reinterpret_cast<int32_t*>(base + off); off += a256(4 * (size_t)qcap);
    v.bytes = off;
    return v;
}

// Algorithm 2, probing: the bucket of sorted query q in table l of its class.
__global__ void batch_probe_kernel(const int64_t* nq, const int32_t* q_cls, const ClassDev* cls,
                                   const uint64_t* qkeys, int64_t key_stride, uint32_t* bitmap, int64_t bm_stride) {
    const int64_t q = blockIdx.x;
    const int l = blockIdx.y;
    if (q >= *nq) return;
    const ClassDev c = cls[q_cls[q]];
    if (l >= c.L) return;
    const uint64_t key = qkeys[(int64_t)l * key_stride + q];
    const uint64_t* sk = c.skeys + (int64_t)l * c.cap;
    const uint32_t* sr = c.srows + (int64_t)l * c.cap;
    const uint32_t* bn = c.bins + (int64_t)l * ((int64_t(1) << c.bin_bits) + 1);
    const uint32_t bin = (uint32_t)(key >> (64 - c.bin_bits));
    const int64_t b0 = bn[bin], b1 = bn[bin + 1];
    uint32_t* bm = bitmap + q * bm_stride;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        if (sk[i] != key) continue;
        const uint32_t row = sr[i];
        atomicOr(&bm[row >> 5], 1u << (row & 31));
    }
    if (c.dcount > 0) {  // rows added since the main tables were built
        const uint64_t* dk = c.dkeys + (int64_t)l * c.dcap;
        const uint32_t* dr = c.drows + (int64_t)l * c.dcap;
        const uint32_t* db = c.dbins + (int64_t)l * ((int64_t(1) << c.dbin_bits) + 1);
        const uint32_t dbin = (uint32_t)(key >> (64 - c.dbin_bits));
        for (int64_t i = db[dbin] + threadIdx.x; i < db[dbin + 1]; i += blockDim.x) {
            if (dk[i] != key) continue;
            const uint32_t row = dr[i];
            atomicOr(&bm[row >> 5], 1u << (row & 31));
        }
    }
}

constexpr unsigned kFull = 0xFFFFFFFFu;

// Candidates per query (the union's size); 0 past the batch.
__global__ void batch_count_kernel(const int64_t* nq, const int32_t* q_cls, const ClassDev* cls,
                                   const uint32_t* bitmap, int64_t bm_stride, int64_t* counts) {
    const int64_t q = blockIdx.x;
    __shared__ int64_t part[32];
    int64_t s = 0;
    if (q < *nq) {
        const int64_t words = cls[q_cls[q]].words;
        const uint32_t* bm = bitmap + q * bm_stride;
        for (int64_t w = threadIdx.x; w < words; w += blockDim.x) s += __popc(bm[w]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
        counts[q] = t;
    }
}

// The rows of query q's union in ascending order at offsets[q] .., with their
// series pointers; the bitmap words are cleared as they are read, so the
// bitmap is all zero again for the next batch (also when the batch overflowed
// and nothing is written).
__global__ void __launch_bounds__(1024) batch_compact_kernel(const int64_t* nq, const int32_t* q_cls,
                                                             const ClassDev* cls, uint32_t* bitmap, int64_t bm_stride,
                                                             const int64_t* offsets,
                                                             const unsigned long long* overflow, uint32_t* cand_rows,
                                                             const float** pair_b) {
    __shared__ int part[32];
    __shared__ int64_t s_base;
    const int64_t q = blockIdx.x;
    if (q >= *nq) return;
    const ClassDev c = cls[q_cls[q]];
    const bool write = *overflow == 0ull;
    uint32_t* bm = bitmap + q * bm_stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = offsets[q];
    __syncthreads();
    for (int64_t w0 = 0; w0 < c.words; w0 += blockDim.x) {
        const int64_t w = w0 + threadIdx.x;
        uint32_t bits = 0u;
        if (w < c.words) {
            bits = bm[w];
            if (bits) bm[w] = 0u;
        }
        const int cnt = __popc(bits);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) part[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int v = (lane < (int)(blockDim.x >> 5)) ? part[lane] : 0;
            int inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += u;
            }
            part[lane] = inc - v;
        }
        __syncthreads();
        int64_t pos = s_base + part[warp] + (incl - cnt);
        if (write) {
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const uint32_t row = (uint32_t)(w * 32 + b);
                cand_rows[pos] = row;
                pair_b[pos] = c.row_ptr[row];
                ++pos;
            }
        } else {
            pos += cnt;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base = pos;
        __syncthreads();
    }
}

}  // namespace
}  // namespace ssh

using namespace ssh;

struct ssh_batch {
    struct HostClass {
        int h = 0, m = 0, rb = 0, L = 0;
        DtwPlan plan{0, 0, 0, 0};
        HashArgs a;
    };
    std::vector<ssh_index*> handles;
    std::vector<uint64_t> versions;
    int64_t qcap = 0, pcap = 0;
    int k = 0;
    int device = 0;
    std::vector<HostClass> cls;
    std::map<int, int> class_of_length;
    int Lmax = 1, max_m = 1;
    int64_t max_words = 1;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_done = nullptr;
    cudaGraphExec_t execs[2] = {nullptr, nullptr};  // captured pipelines: per-class rerank, persistent rerank
    cudaGraphExec_t exec = nullptr;                 // the one the current batch runs
    bool eager = false;           // the launched batch ran without the graph (capture after it)
    int64_t nq = 0;               // queries of the prepared batch
    std::vector<int> q_class;     // their classes, in caller order
    int graph_kernels = 0;
    int graph_kernels_m[2] = {0, 0};
    int mode_pref = -1;           // -1: by batch size; 0: per-class rerank kernels; 1: persistent rerank
    bool persistent = true;       // the current batch's rerank: one persistent launch (else per-class kernels)
    int rerank_grid = 0;          // blocks of the persistent rerank's last launch
    RerankClass* d_rcls = nullptr;  // [C] lengths, radii and DTW tilings of the classes
    int64_t* item_off = nullptr;  // [2 (C + 1)] item layouts of the persistent rerank
    // plan (pinned host copy + device copy)
    unsigned char* h_plan = nullptr;
    unsigned char* d_plan = nullptr;
    PlanView hv{}, dv{};
    ClassDev* d_cls = nullptr;
    ClassDev* h_cls = nullptr;    // pinned staging of the class descriptors
    void* hscratch = nullptr;     // scratch of the specialised hash kernels (largest class, qcap rows)
    BatchStatus* h_status = nullptr;
    BatchStatus* d_status = nullptr;
    // per-query buffers
    uint64_t* qkeys = nullptr;    // [Lmax][qcap]
    uint32_t* bitmap = nullptr;   // [qcap][max_words]
    int64_t* counts = nullptr;    // [qcap]
    int64_t* seg_begin = nullptr; // [qcap + 1]
    float *upper = nullptr, *lower = nullptr;  // [qcap][max_m]
    uint32_t *T = nullptr, *U = nullptr;       // [qcap]
    int64_t* fcount = nullptr;    // [qcap]
    unsigned long long* cursor = nullptr;      // [qcap]
    int64_t* fbegin = nullptr;    // [qcap + 1]
    uint64_t* kth = nullptr;      // [qcap]
    int64_t* out_ids = nullptr;   // [qcap][k]
    float* out_dists = nullptr;   // [qcap][k]
    int32_t* out_which = nullptr; // [qcap]
    // per-pair buffers (capacity pcap)
    uint32_t* cand_rows = nullptr;
    const float** pair_b = nullptr;
    float *lb = nullptr, *dist = nullptr;
    const float** fb = nullptr;
    int64_t* fslot = nullptr;
    uint64_t* tkeys = nullptr;
};

namespace ssh {
namespace {

void free_pairs(ssh_batch* b) {
    cudaFree(b->cand_rows);
    cudaFree(b->pair_b);
    cudaFree(b->lb);
    cudaFree(b->dist);
    cudaFree(b->fb);
    cudaFree(b->fslot);
    cudaFree(b->tkeys);
    b->cand_rows = nullptr;
    b->pair_b = nullptr;
    b->lb = b->dist = nullptr;
    b->fb = nullptr;
    b->fslot = nullptr;
    b->tkeys = nullptr;
}

ssh_status alloc_pairs(ssh_batch* b, int64_t pcap) {
    free_pairs(b);
    const size_t n = (size_t)std::max<int64_t>(pcap, 1);
    cudaError_t e = cudaMalloc(&b->cand_rows, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->pair_b), n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->lb, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->dist, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->fb), n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->fslot, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->tkeys, n * 8);
    if (e != cudaSuccess) {
        free_pairs(b);
        return cuda_status(e, "batch pair buffers");
    }
    b->pcap = pcap;
    return SSH_OK;
}

void drop_graphs(ssh_batch* b) {
    for (int i = 0; i < 2; ++i) {
        if (b->execs[i]) cudaGraphExecDestroy(b->execs[i]);
        b->execs[i] = nullptr;
    }
    b->exec = nullptr;
}

void free_plan(ssh_batch* b) {
    drop_graphs(b);
    cudaFreeHost(b->h_plan);
    cudaFree(b->d_plan);
    cudaFree(b->d_cls);
    cudaFreeHost(b->h_cls);
    b->h_cls = nullptr;
    cudaFree(b->hscratch);
    cudaFree(b->d_rcls);
    cudaFree(b->item_off);
    b->d_rcls = nullptr;
    b->item_off = nullptr;
    b->hscratch = nullptr;
    cudaFree(b->qkeys);
    cudaFree(b->bitmap);
    cudaFree(b->counts);
    cudaFree(b->seg_begin);
    cudaFree(b->upper);
    cudaFree(b->lower);
    cudaFree(b->T);
    cudaFree(b->U);
    cudaFree(b->fcount);
    cudaFree(b->cursor);
    cudaFree(b->fbegin);
    cudaFree(b->kth);
    cudaFree(b->out_ids);
    cudaFree(b->out_dists);
    cudaFree(b->out_which);
    b->h_plan = b->d_plan = nullptr;
    b->d_cls = nullptr;
    b->qkeys = nullptr;
    b->bitmap = nullptr;
    b->counts = b->seg_begin = b->fcount = b->fbegin = nullptr;
    b->upper = b->lower = nullptr;
    b->T = b->U = nullptr;
    b->cursor = nullptr;
    b->kth = nullptr;
    b->out_ids = nullptr;
    b->out_dists = nullptr;
    b->out_which = nullptr;
    b->cls.clear();
    b->class_of_length.clear();
}

// Classes, tuned DTW tilings and every buffer but the pair buffers, from the
// indexes as they are now.
ssh_status build_plan(ssh_batch* b) {
    free_plan(b);
    b->versions.clear();
    for (ssh_index* idx : b->handles) b->versions.push_back(idx->version);
    b->Lmax = 1;
    b->max_m = 1;
    b->max_words = 1;
    std::vector<ClassDev> dev;
    for (int h = 0; h < (int)b->handles.size(); ++h) {
        ssh_index* idx = b->handles[h];
        for (auto& kv : idx->subs) {
            const SubIndex& s = kv.second;
            if (s.count == 0 || b->class_of_length.count(kv.first)) continue;
            ssh_batch::HostClass hc;
            hc.h = h;
            hc.m = s.m;
            hc.rb = s.rb;
            hc.L = idx->L;
            SSH_TRY(prepare_hash_args(idx, s.m, &hc.a));
            hc.plan = dtw_tuned_plan(s.m, s.rb, b->st);
            if (hc.plan.S == 0) return fail_status(SSH_ENOTSUP, "DTW radius %d (length %d) is not covered", s.rb, s.m);
            const ClassDev d = class_dev(s, idx->L);
            b->class_of_length[kv.first] = (int)b->cls.size();
            b->cls.push_back(hc);
            dev.push_back(d);
            b->Lmax = std::max(b->Lmax, idx->L);
            b->max_m = std::max(b->max_m, s.m);
            b->max_words = std::max(b->max_words, d.words);
        }
    }
    if (b->cls.empty()) return fail_status(SSH_ELENGTH, "the indexes of the batch store no series");
    const int C = (int)b->cls.size();
    const int64_t Q = b->qcap;
    const size_t plan_bytes = plan_view(nullptr, Q, C).bytes;
    cudaError_t e = cudaMallocHost(&b->h_plan, plan_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_plan, plan_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cls, C * sizeof(ClassDev));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_cls, C * sizeof(ClassDev));
    size_t hbytes = 256;
    for (const ssh_batch::HostClass& hc : b->cls) {
        HashArgs a = hc.a;
        a.count = Q;
        if (a.minhash != 0 && (a.force_generic || !hash_fast_supported(a))) {
            e = cudaErrorNotSupported;  // the one-permutation minhash runs in the split pipeline only
            break;
        }
        if (!a.force_generic && hash_fast_supported(a)) hbytes = std::max(hbytes, hash_fast_scratch_bytes(a));
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->hscratch, hbytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->qkeys, (size_t)b->Lmax * Q * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->bitmap, (size_t)Q * b->max_words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->counts, (size_t)Q * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->seg_begin, (size_t)(Q + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->upper, (size_t)Q * b->max_m * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->lower, (size_t)Q * b->max_m * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->T, (size_t)Q * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->U, (size_t)Q * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->fcount, (size_t)Q * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->cursor, (size_t)Q * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->fbegin, (size_t)(Q + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->kth, (size_t)Q * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->out_ids, (size_t)Q * b->k * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->out_dists, (size_t)Q * b->k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->out_which, (size_t)Q * 4);
    std::vector<RerankClass> rc(C);
    for (int c = 0; c < C; ++c) {
        const ssh_batch::HostClass& hc = b->cls[c];
        rc[c] = RerankClass{hc.m, hc.rb, hc.plan.S, hc.plan.G, hc.plan.pmask, (int64_t)rerank_dtw_chunk(hc.plan)};
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rcls, C * sizeof(RerankClass));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_rcls, rc.data(), C * sizeof(RerankClass), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->item_off, (size_t)2 * (C + 1) * 8);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_cls, dev.data(), C * sizeof(ClassDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->bitmap, 0, (size_t)Q * b->max_words * 4);
    if (e != cudaSuccess) {
        free_plan(b);
        return cuda_status(e, "batch buffers");
    }
    memset(b->h_plan, 0, plan_bytes);
    b->hv = plan_view(b->h_plan, Q, C);
    b->dv = plan_view(b->d_plan, Q, C);
    return SSH_OK;
}

// Fixed grids: kGridSegs block rows stride over a class's queries; the pair
// hints give 8 LB blocks, 4 DTW blocks and 4 filter blocks per query row.
constexpr int64_t kGridSegs = 1024;
constexpr int64_t kLbGridPairs = 64;
constexpr int64_t kDtwGridPairs = 512;
constexpr int64_t kFilterGridPairs = 1024;

// Enqueue the whole pipeline on b->st (inside a stream capture).
ssh_status enqueue_pipeline(ssh_batch* b) {
    cudaStream_t st = b->st;
    const int C = (int)b->cls.size();
    const int64_t Q = b->qcap;
    const PlanView& d = b->dv;
    SSH_CUDA(cudaMemcpyAsync(b->d_plan, b->h_plan, b->hv.bytes, cudaMemcpyHostToDevice, st));
    SSH_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(BatchStatus), st));
    // Sec. 4.1-4.3 + keys, class by class (rows cls_begin[c] .. cls_begin[c+1] of the sorted table)
    for (int c = 0; c < C; ++c) {
        HashArgs a = b->cls[c].a;
        a.rows = d.q_ptr;
        a.count = Q;
        a.dev_range = d.cls_begin + c;
        a.keys = b->qkeys;
        a.key_stride = Q;
        a.key_col0 = 0;
        if (!a.force_generic && hash_fast_supported(a)) {
            // the specialised kernels, on the plan's scratch (rows are absolute in the sorted table)
            const FastHashBuffers hb = hash_fast_buffers(a, b->hscratch);
            SSH_CUDA(hash_fast_sketch(a, hb, st));
            SSH_CUDA(hash_fast_fixup(a, hb, st));
            SSH_CUDA(hash_fast_shingle(a, hb, st));
            SSH_CUDA(hash_fast_cws(a, hb, st));
        } else {
            SSH_CUDA(launch_hash_generic(a, st));
        }
    }
    // Algorithm 2: probe, union, candidates
    batch_probe_kernel<<<dim3((unsigned)Q, (unsigned)b->Lmax), 256, 0, st>>>(d.nq, d.q_cls, b->d_cls, b->qkeys, Q,
                                                                              b->bitmap, b->max_words);
    note_launch();
    batch_count_kernel<<<(unsigned)Q, 512, 0, st>>>(d.nq, d.q_cls, b->d_cls, b->bitmap, b->max_words, b->counts);
    note_launch();
    SSH_CUDA(cudaGetLastError());
    SSH_CUDA(launch_scan(b->counts, Q, b->seg_begin, b->pcap, &b->d_status->pairs, &b->d_status->overflow, st));
    batch_compact_kernel<<<(unsigned)Q, 1024, 0, st>>>(d.nq, d.q_cls, b->d_cls, b->bitmap, b->max_words, b->seg_begin,
                                                       &b->d_status->overflow, b->cand_rows, b->pair_b);
    note_launch();
    SSH_CUDA(cudaGetLastError());
    const int64_t* n_pairs = b->seg_begin + Q;
    SSH_CUDA(launch_fill_f32(b->dist, b->pcap, n_pairs, __builtin_huge_valf(), st));
    const float shrink = (float)(1.0 - 4.0 * (b->max_m + 3) * std::ldexp(1.0, -24));
    if (b->persistent) {
        // Sec. 3 + Sec. 2.1 + the top-k of every class in one persistent launch
        RerankArgs ra;
        ra.nq = d.nq;
        ra.q_cls = d.q_cls;
        ra.q_ptr = d.q_ptr;
        ra.cls = b->d_rcls;
        ra.seg_begin = b->seg_begin;
        ra.pair_b = b->pair_b;
        ra.cand_rows = b->cand_rows;
        ra.upper = b->upper;
        ra.lower = b->lower;
        ra.env_stride = b->max_m;
        ra.lb = b->lb;
        ra.dist = b->dist;
        ra.fb = b->fb;
        ra.fslot = b->fslot;
        ra.fcount = b->fcount;
        ra.fcursor = b->cursor;
        ra.fbegin = b->fbegin;
        ra.cls_begin = d.cls_begin;
        ra.C = C;
        ra.item_off = b->item_off;
        ra.T = b->T;
        ra.U = b->U;
        ra.k = b->k;
        ra.shrink = shrink;
        ra.out = TopkOut{b->out_ids, b->out_dists, d.q_pos, nullptr, d.q_gid, b->out_which, d.q_which, d.nq};
        ra.dtw_counts = b->d_status->dtw;
        ra.overflow = &b->d_status->overflow;
        ra.work = b->d_status->rr_work;
        ra.bar = b->d_status->rr_bar;
        ra.err = &b->d_status->rr_err;
        SSH_CUDA(launch_rerank(ra, b->max_m, st, &b->rerank_grid));
        SSH_CUDA(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(BatchStatus), cudaMemcpyDeviceToHost, st));
        return SSH_OK;
    }
    // Sec. 3: LB_Keogh of every candidate against its query's envelope
    for (int c = 0; c < C; ++c) {
        const ssh_batch::HostClass& hc = b->cls[c];
        SSH_CUDA(launch_envelope(d.q_ptr, Q, hc.m, hc.rb, b->upper, b->lower, st, d.cls_begin + c, b->max_m));
        // the pair counts are on the device: size the grid for kLbGridPairs pairs per
        // segment at one pair per warp (the launcher plans about 8 per warp)
        PairSet ps{b->seg_begin, Q, d.q_ptr, b->pair_b, nullptr, 8 * kLbGridPairs, d.cls_begin + c, b->max_m,
                   std::min<int64_t>(kGridSegs, Q)};
        SSH_CUDA(launch_lb_keogh(ps, b->upper, b->lower, hc.m, b->lb, st, true));  // with the LB_Kim endpoints
    }
    // Sec. 2.1 rerank: DTW of the k smallest-LB candidates bounds the k-th
    // distance; DTW of the others only where LB (1 - eta) stays below it
    SSH_CUDA(launch_select_kth_u32(reinterpret_cast<const uint32_t*>(b->lb), b->seg_begin, Q, kSeedFactor * b->k, b->T,
                                       st));
    for (int mode = 0; mode < 2; ++mode) {
        if (mode == 1)
            SSH_CUDA(launch_select_kth_u32(reinterpret_cast<const uint32_t*>(b->dist), b->seg_begin, Q, b->k, b->U, st));
        FilterArgs f{b->seg_begin, Q, kFilterGridPairs, b->lb, b->T, b->U, shrink, mode, b->fcount, b->cursor, b->fbegin,
                     &b->d_status->dtw[mode], b->pair_b, b->fb, b->fslot};
        SSH_CUDA(launch_filter(f, st));
        for (int c = 0; c < C; ++c) {
            const ssh_batch::HostClass& hc = b->cls[c];
            PairSet ps{b->fbegin, Q, d.q_ptr, b->fb, b->fslot, kDtwGridPairs, d.cls_begin + c, 0,
                       std::min<int64_t>(kGridSegs, Q)};
            if (mode == 1) {  // survivors: stop at the bound U of the seeds' k-th distance
                ps.abandon = b->U;
                ps.abandon_shrink = shrink;
            }
            SSH_CUDA(launch_dtw_plan(ps, hc.m, hc.rb, hc.plan, b->dist, st));
        }
    }
    // top-k by (distance, row) per query, written at the caller's positions
    SSH_CUDA(launch_topk_keys(b->dist, b->cand_rows, b->pcap, n_pairs, b->tkeys, st));
    SSH_CUDA(launch_select_kth_u64(b->tkeys, b->seg_begin, Q, b->k, b->kth, st));
    TopkOut o{b->out_ids, b->out_dists, d.q_pos, nullptr, d.q_gid, b->out_which, d.q_which, d.nq};
    SSH_CUDA(launch_topk_output(o, b->tkeys, b->seg_begin, b->kth, Q, b->k, st));
    SSH_CUDA(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(BatchStatus), cudaMemcpyDeviceToHost, st));
    return SSH_OK;
}

ssh_status capture(ssh_batch* b) {
    const int mode = b->persistent ? 1 : 0;
    if (b->execs[mode]) {
        cudaGraphExecDestroy(b->execs[mode]);
        b->execs[mode] = nullptr;
    }
    b->exec = nullptr;
    const long long l0 = t_launches;
    SSH_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    ssh_status s = enqueue_pipeline(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    const long long captured = t_launches - l0;  // counted per replay instead
    t_launches -= captured;
    g_launches.fetch_sub(captured);
    if (s != SSH_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_status(e, "batch graph capture");
    size_t n = 0;
    e = cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(g, nodes.data(), &n);
    int kernels = 0;
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->execs[mode], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "batch graph instantiate");
    b->exec = b->execs[mode];
    b->graph_kernels = b->graph_kernels_m[mode] = kernels;
    return SSH_OK;
}

}  // namespace
}  // namespace ssh

namespace ssh {

// The indexes changed since the plan was built: when the classes are the same
// and every class still fits the bitmap stride, only the class descriptors
// (table pointers and sizes) are rewritten and the captured graph stays valid;
// otherwise the plan is rebuilt (and captured again on its next batch).
ssh_status batch_refresh(ssh_batch* b) {
    bool same = true;
    std::vector<ClassDev> dev(b->cls.size());
    std::map<int, int> seen;
    int ncls = 0;
    for (int h = 0; h < (int)b->handles.size() && same; ++h) {
        for (auto& kv : b->handles[h]->subs) {
            const SubIndex& s = kv.second;
            if (s.count == 0 || seen.count(kv.first)) continue;
            seen[kv.first] = h;
            ++ncls;
            auto it = b->class_of_length.find(kv.first);
            if (it == b->class_of_length.end() || b->cls[it->second].h != h || (s.count + 31) / 32 > b->max_words ||
                b->handles[h]->L != b->cls[it->second].L) {
                same = false;
                break;
            }
            dev[it->second] = class_dev(s, b->handles[h]->L);
        }
    }
    if (!same || ncls != (int)b->cls.size()) return build_plan(b);
    // stream-ordered on the plan's stream: after the batches that read the old
    // descriptors, before the next one (the pinned copy is not rewritten before
    // that batch has finished: every batch is finished before the next prepare)
    memcpy(b->h_cls, dev.data(), dev.size() * sizeof(ClassDev));
    SSH_CUDA(cudaMemcpyAsync(b->d_cls, b->h_cls, dev.size() * sizeof(ClassDev), cudaMemcpyHostToDevice, b->st));
    for (size_t h = 0; h < b->handles.size(); ++h) b->versions[h] = b->handles[h]->version;
    return SSH_OK;
}

// Route the queries (back to back at d_queries) to their classes and write
// the query table into the plan's pinned copy; rebuild or refresh a stale plan.
ssh_status batch_prepare(ssh_batch* b, const float* d_queries, const int32_t* lengths, int64_t nq) {
    if (nq > b->qcap) return fail_status(SSH_EINVAL, "%lld queries > the plan's %lld", (long long)nq, (long long)b->qcap);
    SSH_TRY(check_device(b->handles[0]));
    bool stale = false;
    for (size_t h = 0; h < b->handles.size(); ++h) stale |= b->handles[h]->version != b->versions[h];
    if (stale) SSH_TRY(batch_refresh(b));
    const int C = (int)b->cls.size();
    std::vector<int>& qc = b->q_class;
    qc.resize(nq);
    std::vector<int64_t> qoff(nq), per(C + 1, 0);
    int64_t off = 0;
    for (int64_t i = 0; i < nq; ++i) {
        auto it = b->class_of_length.find(lengths[i]);
        if (lengths[i] <= 0 || it == b->class_of_length.end())
            return fail_status(SSH_ELENGTH, "query %lld has length %d, which no index of the batch stores",
                               (long long)i, lengths[i]);
        qc[i] = it->second;
        qoff[i] = off;
        off += lengths[i];
        per[it->second + 1] += 1;
    }
    for (int c = 0; c < C; ++c) per[c + 1] += per[c];
    const PlanView& hv = b->hv;
    *hv.nq = nq;
    for (int c = 0; c <= C; ++c) hv.cls_begin[c] = per[c];
    std::vector<int64_t> fill(per.begin(), per.end() - 1);
    for (int64_t i = 0; i < nq; ++i) {
        const int c = qc[i];
        const int64_t s = fill[c]++;
        const ssh_batch::HostClass& hc = b->cls[c];
        hv.q_ptr[s] = d_queries + qoff[i];
        hv.q_cls[s] = c;
        hv.q_pos[s] = i;
        hv.q_gid[s] = b->handles[hc.h]->subs[hc.m].gid;
        hv.q_which[s] = hc.h;
    }
    b->nq = nq;
    return SSH_OK;
}

// Start the prepared batch on the plan's stream (the captured graph, or the
// kernels themselves for a plan's first batch); returns without waiting.
ssh_status batch_launch(ssh_batch* b) {
    for (ssh_index* h : b->handles) SSH_CUDA(cudaStreamWaitEvent(b->st, h->ready, 0));  // latest adds' tables
    // the rerank's form: one persistent launch balances the work of few queries over every
    // SM; a large batch fills the GPU with per-class kernels, which measured faster there
    const int mode = b->mode_pref >= 0 ? b->mode_pref : (b->nq <= kPersistentMaxQueries ? 1 : 0);
    b->persistent = mode == 1;
    b->exec = b->execs[mode];
    b->graph_kernels = b->graph_kernels_m[mode];
    b->eager = b->exec == nullptr;
    if (b->eager) {
        SSH_TRY(enqueue_pipeline(b));
    } else {
        SSH_CUDA(cudaGraphLaunch(b->exec, b->st));
        note_launch(b->graph_kernels);
    }
    SSH_CUDA(cudaEventRecord(b->ev_done, b->st));
    return SSH_OK;
}

bool batch_done(ssh_batch* b) { return cudaEventQuery(b->ev_done) != cudaErrorNotReady; }

// Wait for the launched batch; a batch whose candidates overflowed the pair
// buffers is run again with grown buffers. Captures the graph after a
// plan's first (direct) batch. Results: batch_outputs, rows in caller order.
ssh_status batch_finish(ssh_batch* b, int64_t reserve_bytes) {
    SSH_CUDA(cudaEventSynchronize(b->ev_done));
    for (int attempt = 0; b->h_status->overflow; ++attempt) {
        if (attempt == 1) return fail_status(SSH_ENOMEM, "batch candidates exceed the pair buffers");
        const int64_t need = (int64_t)b->h_status->pairs;
        const int64_t cap = need + need / 4 + 1024;
        if (reserve_bytes >= 0) {
            // admission by free memory: the old buffers are freed before the new ones are made
            size_t free_b = 0, total_b = 0;
            SSH_CUDA(cudaMemGetInfo(&free_b, &total_b));
            const int64_t grow = (cap - b->pcap) * kBatchPairBytes;
            if ((int64_t)free_b - grow < reserve_bytes)
                return fail_status(SSH_EBUSY, "%lld candidate pairs need %lld more bytes of pair buffers; %lld free, "
                                   "%lld reserved", (long long)need, (long long)grow, (long long)free_b,
                                   (long long)reserve_bytes);
        }
        SSH_TRY(alloc_pairs(b, cap));
        drop_graphs(b);  // both captured the old pair buffers
        SSH_TRY(batch_launch(b));
        SSH_CUDA(cudaEventSynchronize(b->ev_done));
    }
    if (b->h_status->rr_err)
        return fail_status(SSH_ETIMEOUT, "the persistent rerank's grid barrier gave up (a block did not arrive)");
    if (b->eager) SSH_TRY(capture(b));
    b->eager = false;
    for (size_t h = 0; h < b->handles.size(); ++h) {
        int64_t q_h = 0;
        for (int64_t i = 0; i < b->nq; ++i) q_h += b->cls[b->q_class[i]].h == (int)h;
        b->handles[h]->host_stats.queries += q_h;
    }
    b->handles[0]->host_stats.candidates += (int64_t)b->h_status->pairs;
    b->handles[0]->host_stats.dtw_computed += (int64_t)(b->h_status->dtw[0] + b->h_status->dtw[1]);
    return SSH_OK;
}

// Queries through a plan into the caller's rows, ordered on stream `us`.
ssh_status batch_query_into(ssh_batch* b, const float* d_queries, const int32_t* lengths, int64_t nq,
                            int64_t* d_ids, float* d_dists, int32_t* d_which, cudaStream_t us) {
    SSH_TRY(batch_prepare(b, d_queries, lengths, nq));
    SSH_CUDA(cudaEventRecord(b->ev_in, us));
    SSH_CUDA(cudaStreamWaitEvent(b->st, b->ev_in, 0));
    SSH_TRY(batch_launch(b));
    SSH_TRY(batch_finish(b));
    SSH_CUDA(cudaMemcpyAsync(d_ids, b->out_ids, (size_t)nq * b->k * 8, cudaMemcpyDeviceToDevice, b->st));
    SSH_CUDA(cudaMemcpyAsync(d_dists, b->out_dists, (size_t)nq * b->k * 4, cudaMemcpyDeviceToDevice, b->st));
    if (d_which) SSH_CUDA(cudaMemcpyAsync(d_which, b->out_which, (size_t)nq * 4, cudaMemcpyDeviceToDevice, b->st));
    SSH_CUDA(cudaEventRecord(b->ev_out, b->st));
    SSH_CUDA(cudaStreamWaitEvent(us, b->ev_out, 0));
    return SSH_OK;
}

int64_t batch_capacity(const ssh_batch* b) { return b->qcap; }
int batch_k(const ssh_batch* b) { return b->k; }

void batch_outputs(const ssh_batch* b, const int64_t** ids, const float** dists, const int32_t** which) {
    *ids = b->out_ids;
    *dists = b->out_dists;
    *which = b->out_which;
}

cudaStream_t batch_stream(const ssh_batch* b) { return b->st; }

size_t batch_device_bytes(const ssh_batch* b) {
    const int C = (int)b->cls.size();
    const size_t Q = (size_t)b->qcap;
    return plan_view(nullptr, b->qcap, C).bytes + C * sizeof(ClassDev) + (size_t)b->Lmax * Q * 8 +
           Q * (size_t)b->max_words * 4 + Q * 8 * 6 + Q * (size_t)b->max_m * 8 + Q * 4 * 2 + Q * 8 +
           Q * (size_t)b->k * 12 + Q * 4 + (size_t)b->pcap * kBatchPairBytes;
}

}  // namespace ssh

extern "C" {

ssh_status ssh_batch_create(ssh_index* const* handles, int nh, int64_t max_queries, int k, int64_t max_pairs,
                            ssh_batch** out) {
    if (!out) return fail_status(SSH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!handles || nh < 1) return fail_status(SSH_EINVAL, "no indexes");
    for (int h = 0; h < nh; ++h) {
        if (!handles[h]) return fail_status(SSH_EINVAL, "handle %d is NULL", h);
        if (handles[h]->family != 0) return fail_status(SSH_ENOTSUP, "batch plans hash with SSH; index %d is SRP", h);
    }
    if (max_queries < 1 || max_queries > 65535)
        return fail_status(SSH_EINVAL, "max_queries = %lld outside [1, 65535]", (long long)max_queries);
    if (k < 1 || k > kMaxTopK) return fail_status(SSH_EINVAL, "k = %d outside [1, %d]", k, kMaxTopK);
    if (max_pairs < 0) return fail_status(SSH_EINVAL, "max_pairs < 0");
    for (int h = 1; h < nh; ++h)
        if (handles[h]->device != handles[0]->device)
            return fail_status(SSH_EINVAL, "the indexes of a batch must be on one device");
    SSH_TRY(check_device(handles[0]));
    ssh_batch* b = new ssh_batch();
    b->handles.assign(handles, handles + nh);
    b->qcap = max_queries;
    b->k = k;
    b->device = handles[0]->device;
    cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(BatchStatus));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(BatchStatus));
    if (e != cudaSuccess) {
        ssh_status s = cuda_status(e, "ssh_batch_create");
        ssh_batch_destroy(b);
        return s;
    }
    ssh_status s = build_plan(b);
    if (s == SSH_OK) {
        int64_t pc = max_pairs;
        if (pc == 0) pc = std::max<int64_t>(1 << 20, max_queries * 2048);
        s = alloc_pairs(b, pc);
    }
    if (s != SSH_OK) {
        ssh_batch_destroy(b);
        return s;
    }
    *out = b;
    return SSH_OK;
}

ssh_status ssh_batch_query(ssh_batch* b, const float* d_queries, const int32_t* lengths, int64_t nq, int64_t* d_ids,
                           float* d_dists, int32_t* d_which, void* stream) {
    if (!b || nq < 0 || (nq > 0 && (!d_queries || !lengths || !d_ids || !d_dists)))
        return fail_status(SSH_EINVAL, "bad arguments");
    if (nq == 0) return SSH_OK;
    return batch_query_into(b, d_queries, lengths, nq, d_ids, d_dists, d_which, (cudaStream_t)stream);
}

ssh_status ssh_batch_stats(const ssh_batch* b, int64_t* pairs, int64_t* dtw, int64_t* pair_capacity,
                           int32_t* graph_kernels) {
    if (!b) return fail_status(SSH_EINVAL, "NULL batch");
    if (pairs) *pairs = (int64_t)b->h_status->pairs;
    if (dtw) *dtw = (int64_t)(b->h_status->dtw[0] + b->h_status->dtw[1]);
    if (pair_capacity) *pair_capacity = b->pcap;
    if (graph_kernels) *graph_kernels = b->graph_kernels;
    return SSH_OK;
}

ssh_status ssh_batch_set_persistent(ssh_batch* b, int32_t mode) {
    if (!b) return fail_status(SSH_EINVAL, "NULL batch");
    if (mode < -1 || mode > 1) return fail_status(SSH_EINVAL, "mode %d is not -1, 0 or 1", (int)mode);
    b->mode_pref = mode;
    return SSH_OK;
}

void ssh_batch_destroy(ssh_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    free_plan(b);
    free_pairs(b);
    cudaFreeHost(b->h_status);
    cudaFree(b->d_status);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

}  // extern "C"
