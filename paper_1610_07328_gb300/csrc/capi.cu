// capi.cu -- the C ABI of include/ssh.h: index lifetime, the host-side draw
// tables, and the device orchestration of Algorithm 1 (add) and Algorithm 2
// (query). All per-series and per-candidate work runs in the kernels of
// hash_kernels.cu, sort_kernels.cu and query_kernels.cu.
//
// This translation unit is compiled with -ffp-contract=off for the host: the
// FP64 draw tables must be rounded operation by operation, exactly as the
// definitions are written (Sec. 4.1 filter, Sec. 4.3 draws).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "ssh_internal.cuh"

// =================================================================== errors

namespace ssh {

static thread_local char g_err[512] = "";
std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ssh_status cuda_status(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? SSH_ENOMEM : SSH_ECUDA;
}

static ssh_status fail(ssh_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

// ============================================================ random draws
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the seed, with
// the counter naming what is drawn. Uniforms take the top 23 bits plus one
// half: ((x >> 9) + 0.5) * 2^-23, an odd multiple of 2^-24 in (0, 1), exact in
// FP32 and FP64.

namespace {

constexpr uint32_t kTagFilter = 0x46494C54u;  // "FILT"

void philox10(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

inline double unit(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

// Sec. 4.1: r_j ~ N(0,1) by Box-Muller, cosine branch for even j, sine for odd j.
void make_filter(uint64_t seed, int W, std::vector<float>& r) {
    r.resize(W);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < W; ++j) {
        const uint32_t ctr[4] = {(uint32_t)(j / 2), 0u, kTagFilter, 0u};
        uint32_t b[4];
        philox10(ctr, k0, k1, b);
        const double u1 = unit(b[0]), u2 = unit(b[1]);
        const double radius = std::sqrt(-2.0 * std::log(u1));
        const double angle = two_pi * u2;
        const double z = (j % 2 == 0) ? radius * std::cos(angle) : radius * std::sin(angle);
        r[j] = (float)z;
    }
}

constexpr uint32_t kTagSrp = 0x53525031u;     // "SRP1"

// The SRP baseline's projection j for series of length m: N(0,1) entries by
// Box-Muller on the Philox block with counter (i / 2, j, SRP1, m).
void make_srp_projection(uint64_t seed, int m, int j, float* r) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < m; ++i) {
        const uint32_t ctr[4] = {(uint32_t)(i / 2), (uint32_t)j, kTagSrp, (uint32_t)m};
        uint32_t b[4];
        philox10(ctr, k0, k1, b);
        const double u1 = unit(b[0]), u2 = unit(b[1]);
        const double radius = std::sqrt(-2.0 * std::log(u1));
        const double angle = two_pi * u2;
        r[i] = (float)((i % 2 == 0) ? radius * std::cos(angle) : radius * std::sin(angle));
    }
}

template <typename F>
void parallel_for(int64_t n, F f) {
    int nt = (int)std::thread::hardware_concurrency();
    if (nt < 1) nt = 1;
    if (nt > 64) nt = 64;
    if (n < 4096) nt = 1;
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        const int64_t b = t * chunk, e = std::min<int64_t>(n, b + chunk);
        if (b >= e) break;
        th.emplace_back([=]() {
            for (int64_t i = b; i < e; ++i) f(i);
        });
    }
    for (auto& x : th) x.join();
}

// ----------------------------------------------------------- device memory

template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
    return cudaMallocAsync(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T), st);
}

struct ScratchList {
    std::vector<void*> ptrs;
    cudaStream_t st;
    explicit ScratchList(cudaStream_t s) : st(s) {}
    template <typename T>
    ssh_status get(T** p, size_t count) {
        cudaError_t e = dalloc(p, count, st);
        if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync (scratch)");
        ptrs.push_back(*p);
        return SSH_OK;
    }
    ~ScratchList() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

// Records CUDA events around a group of kernels when the index's timing
// option is on; the events are read (and the device time summed) later by
// ssh_get_kernel_times.
struct TimedRegion {
    ssh_index* idx;
    cudaStream_t st;
    const char* name;
    double units;
    long long launches0;
    cudaEvent_t start = nullptr;
    TimedRegion(ssh_index* i, cudaStream_t s, const char* n, double u)
        : idx(i), st(s), name(n), units(u), launches0(t_launches) {
        if (idx->timing && cudaEventCreate(&start) == cudaSuccess) cudaEventRecord(start, st);
    }
    ~TimedRegion() {
        if (!start) return;
        cudaEvent_t stop;
        if (cudaEventCreate(&stop) != cudaSuccess) {
            cudaEventDestroy(start);
            return;
        }
        cudaEventRecord(stop, st);
        idx->pending.push_back(KernelTimer{name, start, stop, (int)(t_launches - launches0), units});
    }
};

double dtw_cells(int m, int rb) { return (double)m * (2.0 * rb + 1.0) - (double)rb * (rb + 1.0); }

// Sec. 4.1-4.3 + keys for a.count series, each stage in its own timed region
// named "<prefix>.<stage>" (units: series).
// The SRP baseline's projections for length m, generated on the host on first use.
ssh_status srp_tab(ssh_index* idx, int m, SrpTab** out) {
    auto it = idx->srp.find(m);
    if (it == idx->srp.end()) {
        const int KL = idx->KL;
        std::vector<float> R((size_t)KL * m), rn(KL);
        const double u = std::ldexp(1.0, -24), gm = m * u / (1.0 - m * u);
        const double tau = std::max(1e-4, 2.0 * gm);
        parallel_for(KL, [&](int64_t j) {
            make_srp_projection(idx->seed, m, (int)j, R.data() + (size_t)j * m);
            double nr = 0.0;
            for (int i = 0; i < m; ++i) nr += (double)R[(size_t)j * m + i] * (double)R[(size_t)j * m + i];
            rn[j] = std::nextafter((float)(tau * std::sqrt(nr) * (1.0 + 1e-6)), INFINITY);
        });
        SrpTab t;
        cudaError_t e = cudaMalloc(&t.R, R.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&t.rn, rn.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(t.R, R.data(), R.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(t.rn, rn.data(), rn.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(t.R);
            cudaFree(t.rn);
            return cuda_status(e, "SRP projections");
        }
        it = idx->srp.emplace(m, t).first;
    }
    *out = &it->second;
    return SSH_OK;
}

ssh_status run_srp(ssh_index* idx, const HashArgs& a, cudaStream_t st, const char* prefix) {
    SrpTab* t = nullptr;
    SSH_TRY(srp_tab(idx, a.m, &t));
    const bool q = prefix[0] == 'q';
    static const char* names[2][3] = {{"add.srp", "add.srp_fixup", "add.srp_keys"},
                                      {"query.srp", "query.srp_fixup", "query.srp_keys"}};
    void* scratch = nullptr;
    SSH_CUDA(cudaMallocAsync(&scratch, srp_scratch_bytes(a), st));
    cudaError_t e = cudaSuccess;
    for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
        TimedRegion tr(idx, st, names[q][stage], (double)a.count);
        e = launch_srp_hash(a, t->R, t->rn, scratch, stage, st);
    }
    cudaError_t f = cudaFreeAsync(scratch, st);
    SSH_CUDA(e);
    SSH_CUDA(f);
    return SSH_OK;
}

ssh_status run_hash(ssh_index* idx, const HashArgs& a, cudaStream_t st, const char* prefix) {
    if (a.count <= 0) return SSH_OK;
    if (idx->family == 1) return run_srp(idx, a, st, prefix);
    static const char* names[2][5] = {{"add.sketch", "add.sketch_fixup", "add.shingle", "add.cws", "add.hash_generic"},
                                      {"query.sketch", "query.sketch_fixup", "query.shingle", "query.cws",
                                       "query.hash_generic"}};
    const int w = (prefix[0] == 'q') ? 1 : 0;
    const double units = (double)a.count;
    if (a.force_generic || !hash_fast_supported(a)) {
        if (a.minhash != 0)
            return fail(SSH_ENOTSUP, "the one-permutation minhash needs a compiled sketch shape (W %d, delta %d)",
                        a.W, a.delta);
        TimedRegion tr(idx, st, names[w][4], units);
        SSH_CUDA(launch_hash_generic(a, st));
        return SSH_OK;
    }
    void* scratch = nullptr;
    SSH_CUDA(cudaMallocAsync(&scratch, hash_fast_scratch_bytes(a), st));
    const FastHashBuffers b = hash_fast_buffers(a, scratch);
    cudaError_t e;
    {
        TimedRegion tr(idx, st, names[w][0], units);
        e = hash_fast_sketch(a, b, st);
    }
    if (e == cudaSuccess) {
        TimedRegion tr(idx, st, names[w][1], units);
        e = hash_fast_fixup(a, b, st);
    }
    if (e == cudaSuccess) {
        TimedRegion tr(idx, st, names[w][2], units);
        e = hash_fast_shingle(a, b, st);
    }
    if (e == cudaSuccess) {
        TimedRegion tr(idx, st, names[w][3], units);
        e = hash_fast_cws(a, b, st);
    }
    cudaFreeAsync(scratch, st);
    SSH_CUDA(e);
    return SSH_OK;
}

// ------------------------------------------------------------ small kernels

__global__ void fill_rows_kernel(const float** row_ptr, int64_t* gid, int64_t n, const float* base, int64_t stride,
                                 int64_t first_gid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        row_ptr[i] = base + i * stride;
        gid[i] = first_gid + i;
    }
}

// Every segment of n lists all rows: rows[p] = p mod n.
__global__ void iota_rows_kernel(uint32_t* rows, int64_t total, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x)
        rows[p] = (uint32_t)(p % n);
}

__global__ void gather_ptrs_kernel(const uint32_t* rows, int64_t n, const float* const* row_ptr, const float** out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = row_ptr[rows[i]];
}


unsigned grid_for(int64_t n, int threads, int64_t cap = 65535) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

int min_length(const ssh_index* idx) { return idx->W + (idx->n - 1) * idx->delta; }

struct Geometry {
    int nb, nwords, S;
};

ssh_status geometry(const ssh_index* idx, int m, Geometry* g) {
    if (m < min_length(idx))
        return fail(SSH_ELENGTH, "series length %d is shorter than W + (n-1)*delta = %d", m, min_length(idx));
    const int64_t nb = (int64_t)(m - idx->W) / idx->delta + 1;
    const int64_t S = nb - idx->n + 1;
    if (S > kMaxCount) return fail(SSH_ELENGTH, "series length %d gives %lld shingles (max %d)", m, (long long)S, kMaxCount);
    g->nb = (int)nb;
    g->nwords = (int)((nb + 31) / 32);
    g->S = (int)S;
    return SSH_OK;
}

int band_radius(float band, int m) {
    if (!(band > 0.0f)) return 0;
    double rb = std::floor((double)band * (double)m);
    if (rb > (double)(m - 1)) rb = (double)(m - 1);
    return (int)rb;
}

HashArgs base_hash_args(const ssh_index* idx, int m, const Geometry& g) {
    HashArgs a;
    memset(&a, 0, sizeof(a));
    a.m = m;
    a.W = idx->W;
    a.delta = idx->delta;
    a.n = idx->n;
    a.nb = g.nb;
    a.nwords = g.nwords;
    a.S = g.S;
    a.K = idx->K;
    a.L = idx->L;
    a.KL = idx->KL;
    a.r = idx->d_r;
    a.r_host = idx->h_r.data();
    a.tau_norm = idx->tau_norm;
    const double gw = idx->W * std::ldexp(1.0, -24) / (1.0 - idx->W * std::ldexp(1.0, -24));
    a.gamma_ss = (float)(2.0 * gw);
    a.rank = idx->d_rank;
    a.rank_stride = rank_stride_of(idx->KL);
    a.tab_stride = tab_stride_of(idx->KL);
    a.force_generic = idx->hash_kernel == 1;
    a.force_fp64 = idx->cws_fp64;
    a.minhash = idx->minhash;
    a.kla = idx->d_kla;
    a.p32 = idx->d_p32;
    a.p64 = idx->d_p64;
    a.lav = idx->d_lav;
    a.tsm = idx->d_tsm;
    a.lns32 = idx->d_lns32;
    a.lns64 = idx->d_lns64;
    a.seed = idx->seed;
    a.stats = idx->d_stats;
    return a;
}

void free_sub(SubIndex& s) {
    cudaFree(s.row_ptr);
    cudaFree(s.gid);
    cudaFree(s.keys);
    cudaFree(s.skeys);
    cudaFree(s.srows);
    cudaFree(s.bins);
    cudaFree(s.dkeys);
    cudaFree(s.drows);
    cudaFree(s.dbins);
    s = SubIndex();
}

// Grow a sub-index to hold `need` rows, keeping the first `count` rows.
ssh_status reserve(ssh_index* idx, SubIndex& s, int64_t need, cudaStream_t st) {
    if (need <= s.cap) return SSH_OK;
    int64_t cap = std::max<int64_t>(need, s.cap + s.cap / 2);
    cap = std::max<int64_t>(cap, 1024);
    const int L = idx->L;
    const float** rp = nullptr;
    int64_t* gid = nullptr;
    uint64_t *keys = nullptr, *skeys = nullptr;
    uint32_t* srows = nullptr;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&rp, cap * sizeof(*rp));
    if (e == cudaSuccess) e = cudaMalloc(&gid, cap * sizeof(*gid));
    if (e == cudaSuccess) e = cudaMalloc(&keys, (size_t)L * cap * sizeof(*keys));
    if (e == cudaSuccess) e = cudaMalloc(&skeys, (size_t)L * cap * sizeof(*skeys));
    if (e == cudaSuccess) e = cudaMalloc(&srows, (size_t)L * cap * sizeof(*srows));
    if (e != cudaSuccess) {
        cudaFree(rp);
        cudaFree(gid);
        cudaFree(keys);
        cudaFree(skeys);
        cudaFree(srows);
        return cuda_status(e, "cudaMalloc (sub-index)");
    }
    if (s.count > 0) {
        SSH_CUDA(cudaMemcpyAsync(rp, s.row_ptr, s.count * sizeof(*rp), cudaMemcpyDeviceToDevice, st));
        SSH_CUDA(cudaMemcpyAsync(gid, s.gid, s.count * sizeof(*gid), cudaMemcpyDeviceToDevice, st));
        for (int l = 0; l < L; ++l)
            SSH_CUDA(cudaMemcpyAsync(keys + (size_t)l * cap, s.keys + (size_t)l * s.cap, s.count * sizeof(*keys),
                                     cudaMemcpyDeviceToDevice, st));
        SSH_CUDA(cudaStreamSynchronize(st));
    }
    cudaFree(s.row_ptr);
    cudaFree(s.gid);
    cudaFree(s.keys);
    cudaFree(s.skeys);
    cudaFree(s.srows);
    s.row_ptr = rp;
    s.gid = gid;
    s.keys = keys;
    s.skeys = skeys;
    s.srows = srows;
    s.cap = cap;
    s.main_count = 0;  // the main tables were not carried over: rebin every row
    s.dcount = 0;
    return SSH_OK;
}

// Rebuild the bucket tables of a sub-index from its per-row keys: only the
// delta tables (rows main_count .. count-1) while they stay within an eighth
// of the main part, else every row into the main tables and no delta.
ssh_status rebuild_tables(ssh_index* idx, SubIndex& s, cudaStream_t st) {
    const int L = idx->L;
    const int64_t nd = s.count - s.main_count;
    ScratchList sc(st);
    if (s.main_count > 0 && nd >= 0 && nd <= s.main_count / 8) {
        const int bits = table_bin_bits(nd);
        if (nd > s.dcap) {
            const int64_t dcap = std::max<int64_t>(nd, std::max<int64_t>(2 * s.dcap, 4096));
            cudaFree(s.dkeys);
            cudaFree(s.drows);
            s.dkeys = nullptr;
            s.drows = nullptr;
            s.dcap = 0;
            SSH_CUDA(cudaMalloc(&s.dkeys, (size_t)L * dcap * sizeof(uint64_t)));
            SSH_CUDA(cudaMalloc(&s.drows, (size_t)L * dcap * sizeof(uint32_t)));
            s.dcap = dcap;
        }
        if (bits > s.dbins_alloc_bits) {
            cudaFree(s.dbins);
            s.dbins = nullptr;
            s.dbins_alloc_bits = 0;
            SSH_CUDA(cudaMalloc(&s.dbins, (size_t)L * (((size_t)1 << bits) + 1) * sizeof(uint32_t)));
            s.dbins_alloc_bits = bits;
        }
        s.dbin_bits = bits;
        uint32_t* cursor;
        SSH_TRY(sc.get(&cursor, (size_t)L * (((size_t)1 << bits) + 1)));
        SSH_CUDA(build_tables(s.keys, s.main_count, nd, L, s.cap, s.dcap, bits, s.dbins, cursor, s.dkeys, s.drows, st));
        s.dcount = nd;
        return SSH_OK;
    }
    const int64_t n = s.count;
    const int bits = table_bin_bits(n);
    if (bits > s.bins_alloc_bits) {
        cudaFree(s.bins);
        s.bins = nullptr;
        s.bins_alloc_bits = 0;
        SSH_CUDA(cudaMalloc(&s.bins, (size_t)L * (((size_t)1 << bits) + 1) * sizeof(uint32_t)));
        s.bins_alloc_bits = bits;
    }
    s.bin_bits = bits;
    uint32_t* cursor;
    SSH_TRY(sc.get(&cursor, (size_t)L * (((size_t)1 << bits) + 1)));
    SSH_CUDA(build_tables(s.keys, 0, n, L, s.cap, s.cap, bits, s.bins, cursor, s.skeys, s.srows, st));
    s.main_count = n;
    s.dcount = 0;
    return SSH_OK;
}


// End of the run of equal lengths that starts at i: the first j > i with
// lengths[j] != lengths[i], or count. Whole chunks are tested with an OR of
// XORs (a loop the compiler vectorises), so a call of one length costs a
// fraction of a scalar compare loop.
int64_t run_end(const int32_t* lengths, int64_t i, int64_t count) {
    const uint32_t v = (uint32_t)lengths[i];
    int64_t j = i + 1;
    constexpr int64_t kChunk = 256;
    while (j + kChunk <= count) {
        uint32_t diff = 0;
        for (int64_t q = 0; q < kChunk; ++q) diff |= (uint32_t)lengths[j + q] ^ v;
        if (diff) break;
        j += kChunk;
    }
    while (j < count && (uint32_t)lengths[j] == v) ++j;
    return j;
}

// A run of consecutive series of one length: series [i, j) of a call, length m.
struct LengthRun {
    int64_t i, j;
    int m;
};

// Every length of a call must be valid before anything is added (each run of
// equal lengths is checked once); `runs` (may be NULL) receives the runs, so the
// lengths are scanned once per call.
ssh_status validate_lengths(ssh_index* idx, const int32_t* lengths, int64_t count,
                            std::vector<LengthRun>* runs = nullptr) {
    for (int64_t i = 0, j; i < count; i = j) {
        j = run_end(lengths, i, count);
        Geometry g;
        if (lengths[i] <= 0) return fail(SSH_ELENGTH, "series %lld has length %d", (long long)i, lengths[i]);
        SSH_TRY(geometry(idx, lengths[i], &g));
        const int rb = band_radius(idx->band, lengths[i]);
        if (dtw_plan(lengths[i], rb).S == 0)
            return fail(SSH_ENOTSUP, "DTW radius %d (length %d) is wider than the compiled DTW tilings cover", rb, lengths[i]);
        if (runs) runs->push_back(LengthRun{i, j, lengths[i]});
    }
    return SSH_OK;
}

// The sub-index of length m (created empty on first use).
SubIndex& sub_for(ssh_index* idx, int m, const Geometry& g) {
    SubIndex& s = idx->subs[m];
    if (s.m == 0) {
        s.m = m;
        s.nb = g.nb;
        s.nwords = g.nwords;
        s.S = g.S;
        s.rb = band_radius(idx->band, m);
    }
    return s;
}

// Algorithm 1 (sketch, shingle, minhash and row keys) for a list of runs of
// equal-length series of a call whose first id is id0 (run r holds the call's
// series [r.i, r.j), all of length r.m). `dev` holds the runs' series back to
// back, contiguously from runs[0].i on (run k starts after the floats of runs
// 0..k-1), in device memory that stays valid while the index uses it. The
// sub-indexes touched are added to `touched`; their tables are rebuilt later.
ssh_status hash_runs(ssh_index* idx, const float* dev, const std::vector<LengthRun>& runs, int64_t id0,
                     cudaStream_t st, std::vector<int>& touched) {
    int64_t run_off = 0;
    for (const LengthRun& r : runs) {
        const int64_t i = r.i, j = r.j;
        const int m = r.m;
        const int64_t nrun = j - i;
        Geometry g;
        SSH_TRY(geometry(idx, m, &g));
        SubIndex& s = sub_for(idx, m, g);
        if (std::find(touched.begin(), touched.end(), m) == touched.end()) touched.push_back(m);
        SSH_TRY(reserve(idx, s, s.count + nrun, st));
        fill_rows_kernel<<<grid_for(nrun, 256, 8192), 256, 0, st>>>(s.row_ptr + s.count, s.gid + s.count, nrun,
                                                                    dev + run_off, m, id0 + i);
        note_launch();
        SSH_CUDA(cudaGetLastError());
        HashArgs a = base_hash_args(idx, m, g);
        a.rows = s.row_ptr + s.count;
        a.count = nrun;
        a.keys = s.keys;
        a.key_stride = s.cap;
        a.key_col0 = s.count;
        SSH_TRY(run_hash(idx, a, st, "add"));
        s.count += nrun;
        idx->host_stats.series_hashed += nrun;
        run_off += (int64_t)m * nrun;
    }
    return SSH_OK;
}

ssh_status hash_range(ssh_index* idx, const float* dev, const int32_t* lengths, int64_t i0, int64_t i1, int64_t id0,
                      cudaStream_t st, std::vector<int>& touched) {
    std::vector<LengthRun> runs;
    for (int64_t i = i0, j; i < i1; i = j) {
        j = run_end(lengths, i, i1);
        runs.push_back(LengthRun{i, j, lengths[i]});
    }
    return hash_runs(idx, dev, runs, id0, st, touched);
}

// Rebuild the tables of the touched sub-indexes and mark the index ready after
// them (the event queries wait for); `sync`: also wait for the call's work.
ssh_status finish_add(ssh_index* idx, const std::vector<int>& touched, int64_t count, cudaStream_t st,
                      int64_t* first_id, bool sync) {
    for (int m : touched) {
        TimedRegion tr(idx, st, "add.table_sort", (double)idx->subs[m].count * idx->L);
        SSH_TRY(rebuild_tables(idx, idx->subs[m], st));
    }
    SSH_CUDA(cudaEventRecord(idx->ready, st));
    if (sync) SSH_CUDA(cudaStreamSynchronize(st));
    if (first_id) *first_id = idx->next_id;
    idx->next_id += count;
    idx->version += 1;
    return SSH_OK;
}

// Algorithm 1 for the series of one call, already in device memory.
ssh_status add_series(ssh_index* idx, const float* dev, const int32_t* lengths, int64_t count, cudaStream_t st,
                      int64_t* first_id) {
    std::vector<LengthRun> runs;
    SSH_TRY(validate_lengths(idx, lengths, count, &runs));
    std::vector<int> touched;
    SSH_TRY(hash_runs(idx, dev, runs, idx->next_id, st, touched));
    return finish_add(idx, touched, count, st, first_id, false);
}

constexpr size_t kArenaChunk = (size_t)256 << 20;
constexpr size_t kArenaMax = (size_t)16 << 20;

// A device buffer of at least `bytes` for a copy of series: small copies are
// carved from the arena (no allocation per streamed insert), larger ones take
// a spare buffer left by ssh_index_clear (the smallest that fits) or a new one.
ssh_status take_buffer(ssh_index* idx, size_t bytes, DevBuf* out) {
    if (bytes <= kArenaMax) {
        const size_t need = (bytes + 255) & ~(size_t)255;
        if (idx->arena.empty() || idx->arena_off + need > kArenaChunk) {
            if (!idx->arena.empty()) {
                ++idx->arena_cur;
                idx->arena_off = 0;
            }
            if (idx->arena_cur >= idx->arena.size()) {
                void* p = nullptr;
                SSH_CUDA(cudaMalloc(&p, kArenaChunk));
                idx->arena.push_back(p);
                idx->arena_cur = idx->arena.size() - 1;
            }
        }
        out->p = static_cast<unsigned char*>(idx->arena[idx->arena_cur]) + idx->arena_off;
        out->bytes = bytes;
        out->arena = true;
        idx->arena_off += need;
        return SSH_OK;
    }
    int best = -1;
    for (int q = 0; q < (int)idx->spare.size(); ++q)
        if (idx->spare[q].bytes >= bytes && (best < 0 || idx->spare[q].bytes < idx->spare[best].bytes)) best = q;
    if (best >= 0) {
        *out = idx->spare[best];
        idx->spare.erase(idx->spare.begin() + best);
        return SSH_OK;
    }
    DevBuf b;
    b.bytes = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, b.bytes);
    if (e != cudaSuccess) {
        // spare buffers too small to use: give their memory back and try once more
        for (DevBuf& f : idx->spare) cudaFree(f.p);
        idx->spare.clear();
        e = cudaMalloc(&b.p, b.bytes);
        if (e != cudaSuccess) return cuda_status(e, "cudaMalloc (series copy)");
    }
    *out = b;
    return SSH_OK;
}

// Algorithm 2 for the `nq` queries of one length m (dev_q[i] = query series,
// qpos[i] = its position in the caller's output).
ssh_status query_group(ssh_index* idx, SubIndex& s, const std::vector<const float*>& qptr,
                       const std::vector<int64_t>& qpos, int k, int64_t* d_ids, float* d_dists, cudaStream_t st) {
    const int64_t nq = (int64_t)qptr.size();
    const int m = s.m, L = idx->L;
    Geometry g{s.nb, s.nwords, s.S};
    ScratchList sc(st);
    const float** d_qptr;
    int64_t* d_qpos;
    SSH_TRY(sc.get(&d_qptr, nq));
    SSH_TRY(sc.get(&d_qpos, nq));
    SSH_CUDA(cudaMemcpyAsync(d_qptr, qptr.data(), nq * sizeof(float*), cudaMemcpyHostToDevice, st));
    SSH_CUDA(cudaMemcpyAsync(d_qpos, qpos.data(), nq * sizeof(int64_t), cudaMemcpyHostToDevice, st));

    // exact scan (the comparator without hashing): every stored series of the
    // query's length is a candidate of the reporting step below
    const bool exact = idx->exact_scan;
    const int64_t words = (s.count + 31) / 32;
    uint32_t* bitmap = nullptr;
    std::vector<int64_t> h_counts(nq, s.count), h_begin(nq + 1);
    if (!exact) {
        // Algorithm 2: hash the queries as the stored series were hashed
        uint64_t* qkeys;
        SSH_TRY(sc.get(&qkeys, (size_t)L * nq));
        HashArgs a = base_hash_args(idx, m, g);
        a.rows = d_qptr;
        a.count = nq;
        a.keys = qkeys;
        a.key_stride = nq;
        a.key_col0 = 0;
        SSH_TRY(run_hash(idx, a, st, "query"));
        idx->host_stats.series_hashed += nq;

        // Algorithm 2: probe every table, union of the buckets
        int64_t* counts;
        SSH_TRY(sc.get(&bitmap, (size_t)nq * words));
        SSH_TRY(sc.get(&counts, nq));
        SSH_CUDA(cudaMemsetAsync(bitmap, 0, (size_t)nq * words * sizeof(uint32_t), st));
        ProbeArgs pa{qkeys, nq, L, s.skeys, s.srows, s.bins, s.bin_bits, s.cap, s.count, bitmap, words,
                     s.dkeys, s.drows, s.dbins, s.dbin_bits, s.dcap, s.dcount};
        {
            TimedRegion tr(idx, st, "query.probe_union", (double)nq * L);
            SSH_CUDA(launch_probe_union(pa, st));
            SSH_CUDA(launch_bitmap_count(bitmap, nq, words, counts, st));
        }
        SSH_CUDA(cudaMemcpyAsync(h_counts.data(), counts, nq * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        SSH_CUDA(cudaStreamSynchronize(st));
    }
    h_begin[0] = 0;
    int64_t max_c = 0;
    for (int64_t q = 0; q < nq; ++q) {
        h_begin[q + 1] = h_begin[q] + h_counts[q];
        max_c = std::max(max_c, h_counts[q]);
    }
    const int64_t C = h_begin[nq];
    idx->host_stats.queries += nq;
    idx->host_stats.candidates += C;

    int64_t* seg_begin;
    uint32_t* cand_rows;
    const float** pair_b;
    float *lb, *dist;
    SSH_TRY(sc.get(&seg_begin, nq + 1));
    SSH_TRY(sc.get(&cand_rows, C));
    SSH_TRY(sc.get(&pair_b, C));
    SSH_TRY(sc.get(&lb, C));
    SSH_TRY(sc.get(&dist, C));
    SSH_CUDA(cudaMemcpyAsync(seg_begin, h_begin.data(), (nq + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (exact) {
        if (C > 0) {
            iota_rows_kernel<<<grid_for(C, 256, 8192), 256, 0, st>>>(cand_rows, C, s.count);
            note_launch();
            SSH_CUDA(cudaGetLastError());
        }
    } else {
        SSH_CUDA(launch_bitmap_compact(bitmap, nq, words, seg_begin, cand_rows, nullptr, st));
    }
    if (C > 0) {
        gather_ptrs_kernel<<<grid_for(C, 256, 8192), 256, 0, st>>>(cand_rows, C, s.row_ptr, pair_b);
        note_launch();
        SSH_CUDA(cudaGetLastError());
        SSH_CUDA(launch_fill_f32(dist, C, nullptr, __builtin_huge_valf(), st));
    }

    PairSet all{seg_begin, nq, d_qptr, pair_b, nullptr, max_c};
    const int rb = s.rb;
    unsigned long long* pruned_counts = nullptr;  // pinned: DTW pairs of the seed and survivor passes
    size_t pruned_slots[2] = {SIZE_MAX, SIZE_MAX};
    const DtwPlan dplan = (C > 0) ? dtw_tuned_plan(m, rb, st) : DtwPlan{0, 0, 0, 0};
    if (C > 0 && !idx->lb_prune) {
        {
            TimedRegion tr(idx, st, "query.dtw", (double)C * dtw_cells(m, rb));
            SSH_CUDA(launch_dtw_plan(all, m, rb, dplan, dist, st));
        }
        idx->host_stats.dtw_computed += C;
    } else if (C > 0) {
        // Algorithm 2 reporting step with UCR-style pruning: LB_Keogh of every candidate; DTW of the k
        // smallest-LB candidates gives a bound U on the k-th best distance; DTW of
        // the rest only where LB * (1 - eta) <= U.
        float *upper, *lower;
        SSH_TRY(sc.get(&upper, (size_t)nq * m));
        SSH_TRY(sc.get(&lower, (size_t)nq * m));
        {
            TimedRegion tr(idx, st, "query.lb_keogh", (double)C * m);
            SSH_CUDA(launch_envelope(d_qptr, nq, m, rb, upper, lower, st));
            SSH_CUDA(launch_lb_keogh(all, upper, lower, m, lb, st, idx->lb_cascade >= 1));
        }
        uint32_t *T, *U;
        SSH_TRY(sc.get(&T, nq));
        SSH_TRY(sc.get(&U, nq));
        SSH_CUDA(launch_select_kth_u32(reinterpret_cast<const uint32_t*>(lb), seg_begin, nq, kSeedFactor * k, T, st));
        // eta bounds the FP32 rounding of LB (m + 3 terms) and of DTW (2m terms): 4 (m + 3) 2^-24
        const float shrink = (float)(1.0 - 4.0 * (m + 3) * std::ldexp(1.0, -24));
        int64_t *fcount, *fbegin;
        unsigned long long *cursor, *ftotal;
        const float** fb;
        int64_t* fslot;
        SSH_TRY(sc.get(&fcount, nq));
        SSH_TRY(sc.get(&fbegin, nq + 1));
        SSH_TRY(sc.get(&cursor, nq));
        SSH_TRY(sc.get(&ftotal, 5));  // pairs of the two passes, reversed-LB prunes, DTW blocks of the two passes
        SSH_TRY(sc.get(&fb, C));
        SSH_TRY(sc.get(&fslot, C));
        unsigned long long* h_tot = idx->h_pinned;
        h_tot[0] = h_tot[1] = h_tot[2] = h_tot[3] = h_tot[4] = 0;
        const bool rev = idx->lb_cascade == 2;
        SSH_CUDA(cudaMemsetAsync(ftotal + 2, 0, 3 * sizeof(unsigned long long), st));
        ssh_status fst = SSH_OK;
        size_t tslot[2] = {SIZE_MAX, SIZE_MAX};  // the two DTW timings: cells are known after the sync
        for (int mode = 0; mode < 2 && fst == SSH_OK; ++mode) {
            cudaError_t e = cudaSuccess;
            if (mode == 1)
                e = launch_select_kth_u32(reinterpret_cast<const uint32_t*>(dist), seg_begin, nq, k, U, st);
            FilterArgs f{seg_begin, nq, max_c, lb, T, U, shrink, mode, fcount, cursor, fbegin, ftotal + mode, pair_b, fb,
                         fslot};
            if (e == cudaSuccess) e = launch_filter(f, st);
            // every filtered segment is no longer than its candidate segment, and a seed segment holds
            // about kSeedFactor * k pairs: size the DTW grid by that (a block whose share is empty
            // exits at once; a longer segment gives each block a larger share, see dtw_wave_kernel)
            const int64_t seg_pairs = mode == 0 ? std::min<int64_t>(max_c, (int64_t)kSeedFactor * k) : max_c;
            PairSet sub{fbegin, nq, d_qptr, fb, fslot, seg_pairs};
            sub.blocks_done = ftotal + 3 + mode;  // the cells actually computed (abandoned pairs stop early)
            if (mode == 1) {  // survivors: stop at the bound U of the seeds' k-th distance
                sub.abandon = U;
                sub.abandon_shrink = shrink;
                // UCR cascade: the reversed LB_Keogh clears the survivors it proves too far
                if (e == cudaSuccess && rev && !lb_rev_fits(m, rb)) {
                    idx->host_stats.lb2_skipped += nq;  // requested, but the envelopes do not fit
                } else if (e == cudaSuccess && rev) {
                    TimedRegion tr(idx, st, "query.lb_rev", 0.0);
                    e = launch_lb_rev(sub, m, rb, nullptr, U, shrink, fb, ftotal + 2, st);
                }
            }
            if (e == cudaSuccess) {
                {
                    TimedRegion tr(idx, st, "query.dtw", 0.0);
                    e = launch_dtw_plan(sub, m, rb, dplan, dist, st);
                }
                if (idx->timing && !idx->pending.empty()) tslot[mode] = idx->pending.size() - 1;
            }
            if (e != cudaSuccess) fst = cuda_status(e, "rerank");
        }
        if (fst == SSH_OK) {
            // read at the end of the query with the results
            cudaError_t e = cudaMemcpyAsync(h_tot, ftotal, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) fst = cuda_status(e, "rerank counts");
        }
        if (fst != SSH_OK) {
            cudaStreamSynchronize(st);
            return fst;
        }
        pruned_counts = h_tot;
        pruned_slots[0] = tslot[0];
        pruned_slots[1] = tslot[1];
    }
    // top-k by (distance, id): ids grow with rows inside a sub-index, so the key
    // (distance bits, row) orders exactly like (distance, id)
    uint64_t *tkeys, *kth;
    SSH_TRY(sc.get(&tkeys, C));
    SSH_TRY(sc.get(&kth, nq));
    cudaError_t e = cudaSuccess;
    {
        TimedRegion tr(idx, st, "query.topk", (double)C);
        if (C > 0) e = launch_topk_keys(dist, cand_rows, C, nullptr, tkeys, st);
        if (e == cudaSuccess) e = launch_select_kth_u64(tkeys, seg_begin, nq, k, kth, st);
        TopkOut o{d_ids, d_dists, d_qpos, s.gid, nullptr, nullptr, nullptr, nullptr};
        if (e == cudaSuccess) e = launch_topk_output(o, tkeys, seg_begin, kth, nq, k, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && pruned_counts) {
        const unsigned long long rev = pruned_counts[2];
        idx->host_stats.dtw_computed += (int64_t)(pruned_counts[0] + pruned_counts[1] - rev);
        idx->host_stats.lb2_pruned += (int64_t)rev;
        // DTW units: the cells computed, a pair's blocks of wavefront steps times its cells per block
        const double cells_per_block = dtw_cells(m, rb) / (double)dtw_plan_blocks(m, rb, dplan);
        for (int mode = 0; mode < 2; ++mode)
            if (pruned_slots[mode] != SIZE_MAX)
                idx->pending[pruned_slots[mode]].units = (double)pruned_counts[3 + mode] * cells_per_block;
    }
    idx->host_stats.lb_pruned = idx->host_stats.candidates - idx->host_stats.dtw_computed;
    SSH_CUDA(e);
    return SSH_OK;
}

ssh_status run_query(ssh_index* idx, const float* d_queries, const int32_t* lengths, int64_t nq, int k,
                     int64_t* d_ids, float* d_dists, cudaStream_t st) {
    if (k < 1 || k > kMaxTopK) return fail(SSH_EINVAL, "k = %d outside [1, %d]", k, kMaxTopK);
    SSH_CUDA(cudaStreamWaitEvent(st, idx->ready, 0));  // the latest add's tables
    std::map<int, std::pair<std::vector<const float*>, std::vector<int64_t>>> groups;
    int64_t off = 0;
    for (int64_t i = 0; i < nq; ++i) {
        const int m = lengths[i];
        auto it = idx->subs.find(m);
        if (m <= 0 || it == idx->subs.end() || it->second.count == 0)
            return fail(SSH_ELENGTH, "query %lld has length %d, which has no stored series", (long long)i, m);
        groups[m].first.push_back(d_queries + off);
        groups[m].second.push_back(i);
        off += m;
    }
    for (auto& kv : groups)
        SSH_TRY(query_group(idx, idx->subs[kv.first], kv.second.first, kv.second.second, k, d_ids, d_dists, st));
    return SSH_OK;
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, const int64_t* pos, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[pos[i]] = v;
}

}  // namespace

cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> have;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = have[{dev, fn}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

ssh_status check_device(const ssh_index* idx) {
    int dev = -1;
    SSH_CUDA(cudaGetDevice(&dev));
    if (dev != idx->device) SSH_CUDA(cudaSetDevice(idx->device));
    return SSH_OK;
}

ssh_status fail_status(ssh_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_error("%s", buf);
    return s;
}

ssh_status prepare_hash_args(const ssh_index* idx, int m, HashArgs* a) {
    SSH_TRY(check_device(idx));
    Geometry g;
    SSH_TRY(geometry(idx, m, &g));
    *a = base_hash_args(idx, m, g);
    return SSH_OK;
}

}  // namespace ssh

using namespace ssh;

// ================================================================= C ABI

extern "C" {

const char* ssh_status_str(ssh_status s) {
    switch (s) {
        case SSH_OK: return "SSH_OK";
        case SSH_EINVAL: return "SSH_EINVAL";
        case SSH_ENOMEM: return "SSH_ENOMEM";
        case SSH_ECUDA: return "SSH_ECUDA";
        case SSH_ELENGTH: return "SSH_ELENGTH";
        case SSH_EBUSY: return "SSH_EBUSY";
        case SSH_ETIMEOUT: return "SSH_ETIMEOUT";
        case SSH_ENOTSUP: return "SSH_ENOTSUP";
    }
    return "SSH_UNKNOWN";
}

const char* ssh_last_error(void) { return g_err; }

ssh_status ssh_create(int W, int delta, int n, int K, int L, float band, uint64_t seed, ssh_index** out) {
    if (!out) return fail(SSH_EINVAL, "out is NULL");
    *out = nullptr;
    if (W < 1 || W > kMaxW) return fail(SSH_EINVAL, "W = %d outside [1, %d]", W, kMaxW);
    if (delta < 1) return fail(SSH_EINVAL, "delta = %d < 1", delta);
    if (n < 1 || n > 32) return fail(SSH_EINVAL, "n = %d outside [1, 32]", n);
    if (K < 1 || L < 1 || (int64_t)K * L > kMaxKL) return fail(SSH_EINVAL, "K*L = %lld outside [1, %d]", (long long)K * L, kMaxKL);
    if (!(band >= 0.0f) || std::isinf(band)) return fail(SSH_EINVAL, "band must be finite and >= 0");

    ssh_index* idx = new ssh_index();
    idx->W = W;
    idx->delta = delta;
    idx->n = n;
    idx->K = K;
    idx->L = L;
    idx->KL = K * L;
    idx->band = band;
    idx->seed = seed;
    cudaError_t e = cudaGetDevice(&idx->device);
    if (e != cudaSuccess) {
        delete idx;
        return cuda_status(e, "cudaGetDevice");
    }
    {
        // scratch comes from the device's default stream-ordered pool: keep freed
        // blocks in the pool across synchronisations instead of returning them
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, idx->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    e = cudaStreamCreateWithFlags(&idx->hstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&idx->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&idx->cevent, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&idx->h_pinned, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&idx->ready, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ssh_status st = cuda_status(e, "ssh_create streams");
        ssh_destroy(idx);
        return st;
    }

    // Sec. 4.1 filter and the sign-test threshold tau * ||r|| (tau = max(1e-4, 2 gamma_W))
    make_filter(seed, W, idx->h_r);
    double nr = 0.0;
    for (float v : idx->h_r) nr += (double)v * (double)v;
    const double gw = W * std::ldexp(1.0, -24) / (1.0 - W * std::ldexp(1.0, -24));
    const double tau = std::max(1e-4, 2.0 * gw);
    idx->tau_norm = std::nextafter((float)(tau * std::sqrt(nr) * (1.0 + 1e-6)), INFINITY);

    // Sec. 4.3 draw tables for every (hash j, shingle k), built on the GPU (draws.cu)
    {
        ssh_status ts = build_draw_tables(idx, idx->hstream);
        if (ts != SSH_OK) {
            ssh_destroy(idx);
            return ts;
        }
    }
    e = cudaMalloc(reinterpret_cast<void**>(&idx->d_r), W * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(idx->d_r, idx->h_r.data(), W * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&idx->d_stats, kNumStatSlots * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(idx->d_stats, 0, kNumStatSlots * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        ssh_status st = cuda_status(e, "ssh_create device tables");
        ssh_destroy(idx);
        return st;
    }
    *out = idx;
    return SSH_OK;
}

ssh_status ssh_create_srp(int K, int L, float band, uint64_t seed, ssh_index** out) {
    // the SSH parameters W = delta = n = 1 make every length >= 1 valid and the draw tables tiny
    SSH_TRY(ssh_create(1, 1, 1, K, L, band, seed, out));
    (*out)->family = 1;
    return SSH_OK;
}

void ssh_destroy(ssh_index* idx) {
    if (!idx) return;
    cudaSetDevice(idx->device);
    cudaDeviceSynchronize();
    for (auto& kv : idx->subs) free_sub(kv.second);
    for (auto& kv : idx->srp) {
        cudaFree(kv.second.R);
        cudaFree(kv.second.rn);
    }
    for (DevBuf& b : idx->owned) cudaFree(b.p);
    for (DevBuf& b : idx->spare) cudaFree(b.p);
    for (void* p : idx->arena) cudaFree(p);
    if (idx->cevent) cudaEventDestroy(idx->cevent);
    if (idx->h_pinned) cudaFreeHost(idx->h_pinned);
    if (idx->ready) cudaEventDestroy(idx->ready);
    if (idx->hstream) cudaStreamDestroy(idx->hstream);
    if (idx->cstream) cudaStreamDestroy(idx->cstream);
    for (auto& t : idx->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    cudaFree(idx->d_r);
    cudaFree(idx->d_rank);
    cudaFree(idx->d_kla);
    cudaFree(idx->d_p32);
    cudaFree(idx->d_p64);
    cudaFree(idx->d_lav);
    cudaFree(idx->d_tsm);
    cudaFree(idx->d_lns32);
    cudaFree(idx->d_lns64);
    cudaFree(idx->d_stats);
    delete idx;
}

ssh_status ssh_get_filter(const ssh_index* idx, float* r_out) {
    if (!idx || !r_out) return fail(SSH_EINVAL, "NULL argument");
    memcpy(r_out, idx->h_r.data(), idx->W * sizeof(float));
    return SSH_OK;
}

static ssh_status index_add_impl(ssh_index* idx, const float* series, const int32_t* lengths, int64_t count,
                                 int64_t* first_id) {
    if (!idx || (count > 0 && (!series || !lengths)) || count < 0) return fail(SSH_EINVAL, "bad arguments");
    SSH_TRY(check_device(idx));
    if (count == 0) {
        if (first_id) *first_id = idx->next_id;
        return SSH_OK;
    }
    SSH_TRY(validate_lengths(idx, lengths, count));
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) total += lengths[i];
    DevBuf buf;
    SSH_TRY(take_buffer(idx, (size_t)total * sizeof(float), &buf));
    float* dev = static_cast<float*>(buf.p);
    // copy in chunks of about kAddChunkBytes on cstream; hashing of a chunk on
    // hstream waits only for that chunk's copy, so copies and hashing overlap
    constexpr int64_t kAddChunkBytes = 128ll << 20;
    cudaStream_t st = idx->hstream, cs = idx->cstream;
    std::vector<int> touched;
    ssh_status status = SSH_OK;
    int64_t i = 0, off = 0;
    while (i < count && status == SSH_OK) {
        int64_t j = i, bytes = 0;
        while (j < count && (j == i || bytes + (int64_t)lengths[j] * 4 <= kAddChunkBytes)) bytes += (int64_t)lengths[j++] * 4;
        cudaError_t e = cudaMemcpyAsync(dev + off, series + off, bytes, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(idx->cevent, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, idx->cevent, 0);
        if (e != cudaSuccess) {
            status = cuda_status(e, "series copy");
            break;
        }
        status = hash_range(idx, dev + off, lengths, i, j, idx->next_id, st, touched);
        off += bytes / 4;
        i = j;
    }
    if (status == SSH_OK) status = finish_add(idx, touched, count, st, first_id, true);
    if (status != SSH_OK) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(st);
        if (!buf.arena) idx->spare.push_back(buf);
        return status;
    }
    if (!buf.arena) idx->owned.push_back(buf);  // referenced by the stored rows until ssh_index_clear
    return SSH_OK;
}

static ssh_status index_add_device_impl(ssh_index* idx, const float* d_series, const int32_t* lengths,
                                        int64_t count, uint32_t flags, void* stream, int64_t* first_id);
static ssh_status query_impl(ssh_index* idx, const float* queries, const int32_t* lengths, int64_t nq, int k,
                             int64_t* ids, float* dists);

// Adds the kernel launches made during one public call to the index's counter.
struct LaunchCount {
    ssh_stats* st;
    long long l0;
    explicit LaunchCount(const ssh_index* idx)
        : st(idx ? const_cast<ssh_stats*>(&idx->host_stats) : nullptr), l0(t_launches) {}
    ~LaunchCount() {
        if (st) __atomic_fetch_add(&st->kernel_launches, (int64_t)(t_launches - l0), __ATOMIC_RELAXED);
    }
};

ssh_status ssh_index_add(ssh_index* idx, const float* series, const int32_t* lengths, int64_t count,
                         int64_t* first_id) {
    LaunchCount lc(idx);
    return index_add_impl(idx, series, lengths, count, first_id);
}

ssh_status ssh_index_add_device(ssh_index* idx, const float* d_series, const int32_t* lengths, int64_t count,
                                uint32_t flags, void* stream, int64_t* first_id) {
    LaunchCount lc(idx);
    return index_add_device_impl(idx, d_series, lengths, count, flags, stream, first_id);
}

ssh_status ssh_index_add_windows_device(ssh_index* idx, const float* d_stream, int64_t stream_len, int32_t t,
                                        int64_t step, void* stream, int64_t* first_id) {
    LaunchCount lc(idx);
    if (!idx || !d_stream || step < 1 || t < 1 || stream_len < t)
        return fail(SSH_EINVAL, "windows: need a stream, step >= 1 and 1 <= t <= stream_len");
    SSH_TRY(check_device(idx));
    SSH_TRY(validate_lengths(idx, &t, 1));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t count = (stream_len - t) / step + 1;
    Geometry g;
    SSH_TRY(geometry(idx, t, &g));
    SubIndex& s = sub_for(idx, t, g);
    SSH_TRY(reserve(idx, s, s.count + count, st));
    // row p of the call is the window that starts at sample p * step
    fill_rows_kernel<<<grid_for(count, 256, 8192), 256, 0, st>>>(s.row_ptr + s.count, s.gid + s.count, count,
                                                                 d_stream, step, idx->next_id);
    note_launch();
    SSH_CUDA(cudaGetLastError());
    HashArgs a = base_hash_args(idx, t, g);
    a.rows = s.row_ptr + s.count;
    a.count = count;
    a.keys = s.keys;
    a.key_stride = s.cap;
    a.key_col0 = s.count;
    if (idx->family == 0 && !a.force_generic && step < g.nb && hash_windows_supported(a)) {
        // overlapping windows share their sketch positions: the stream's bits and
        // shingle ids are computed once (N_B / step times fewer dot products)
        static const char* names[4] = {"add.sketch", "add.sketch_fixup", "add.shingle", "add.cws"};
        void* scratch = nullptr;
        SSH_CUDA(cudaMallocAsync(&scratch, hash_windows_scratch_bytes(a, step), st));
        cudaError_t e = cudaSuccess;
        for (int stage = 0; stage < 4 && e == cudaSuccess; ++stage) {
            TimedRegion tr(idx, st, names[stage], (double)count);
            e = hash_windows_stage(a, d_stream, step, scratch, stage, st);
        }
        cudaError_t f = cudaFreeAsync(scratch, st);
        SSH_CUDA(e);
        SSH_CUDA(f);
    } else {
        SSH_TRY(run_hash(idx, a, st, "add"));
    }
    s.count += count;
    idx->host_stats.series_hashed += count;
    return finish_add(idx, std::vector<int>{t}, count, st, first_id, false);
}

ssh_status ssh_query(ssh_index* idx, const float* queries, const int32_t* lengths, int64_t nq, int k, int64_t* ids,
                     float* dists) {
    LaunchCount lc(idx);
    return query_impl(idx, queries, lengths, nq, k, ids, dists);
}

static ssh_status index_add_device_impl(ssh_index* idx, const float* d_series, const int32_t* lengths,
                                        int64_t count, uint32_t flags, void* stream, int64_t* first_id) {
    if (!idx || (count > 0 && (!d_series || !lengths)) || count < 0) return fail(SSH_EINVAL, "bad arguments");
    SSH_TRY(check_device(idx));
    cudaStream_t st = (cudaStream_t)stream;
    if (count == 0) {
        if (first_id) *first_id = idx->next_id;
        return SSH_OK;
    }
    const float* src = d_series;
    DevBuf own;
    if (!(flags & SSH_ADD_BORROW)) {
        SSH_TRY(validate_lengths(idx, lengths, count));
        int64_t total = 0;
        for (int64_t i = 0; i < count; ++i) total += lengths[i];
        SSH_TRY(take_buffer(idx, (size_t)total * sizeof(float), &own));
        cudaError_t e = cudaMemcpyAsync(own.p, d_series, total * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            if (!own.arena) idx->spare.push_back(own);
            return cuda_status(e, "cudaMemcpyAsync (series)");
        }
        src = static_cast<const float*>(own.p);
    }
    ssh_status s = add_series(idx, src, lengths, count, st, first_id);
    if (s != SSH_OK) {
        if (own.p && !own.arena) {
            cudaStreamSynchronize(st);
            idx->spare.push_back(own);
        }
        return s;
    }
    if (own.p && !own.arena) idx->owned.push_back(own);
    return SSH_OK;
}

ssh_status ssh_index_clear(ssh_index* idx) {
    if (!idx) return fail(SSH_EINVAL, "NULL index");
    SSH_TRY(check_device(idx));
    SSH_CUDA(cudaDeviceSynchronize());
    for (auto& kv : idx->subs) {  // keep the capacity for the next add
        kv.second.count = 0;
        kv.second.main_count = 0;
        kv.second.dcount = 0;
    }
    idx->version += 1;
    // the copies of the cleared series become staging buffers for later adds
    for (DevBuf& b : idx->owned) idx->spare.push_back(b);
    idx->owned.clear();
    idx->arena_cur = 0;
    idx->arena_off = 0;
    idx->next_id = 0;
    return SSH_OK;
}

ssh_status ssh_index_size(const ssh_index* idx, int64_t* count) {
    if (!idx || !count) return fail(SSH_EINVAL, "NULL argument");
    int64_t c = 0;
    for (auto& kv : idx->subs) c += kv.second.count;
    *count = c;
    return SSH_OK;
}

static ssh_status query_impl(ssh_index* idx, const float* queries, const int32_t* lengths, int64_t nq, int k,
                             int64_t* ids, float* dists) {
    if (!idx || nq < 0 || (nq > 0 && (!queries || !lengths || !ids || !dists))) return fail(SSH_EINVAL, "bad arguments");
    SSH_TRY(check_device(idx));
    if (nq == 0) return SSH_OK;
    int64_t total = 0;
    for (int64_t i = 0; i < nq; ++i) total += std::max(lengths[i], 0);
    cudaStream_t st = idx->hstream;
    float* dq = nullptr;
    int64_t* did = nullptr;
    float* dd = nullptr;
    cudaError_t e = cudaMallocAsync(&dq, std::max<int64_t>(total, 1) * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&did, nq * k * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dd, nq * k * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dq, queries, total * sizeof(float), cudaMemcpyHostToDevice, st);
    ssh_status s = (e == cudaSuccess) ? run_query(idx, dq, lengths, nq, k, did, dd, st)
                                      : cuda_status(e, "ssh_query staging");
    if (s == SSH_OK) {
        e = cudaMemcpyAsync(ids, did, nq * k * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dists, dd, nq * k * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "ssh_query results");
    }
    cudaFreeAsync(dq, st);
    cudaFreeAsync(did, st);
    cudaFreeAsync(dd, st);
    cudaStreamSynchronize(st);
    return s;
}

ssh_status ssh_query_device(ssh_index* idx, const float* d_queries, const int32_t* lengths, int64_t nq, int k,
                            int64_t* d_ids, float* d_dists, void* stream) {
    if (!idx || nq < 0 || (nq > 0 && (!d_queries || !lengths || !d_ids || !d_dists)))
        return fail(SSH_EINVAL, "bad arguments");
    SSH_TRY(check_device(idx));
    if (nq == 0) return SSH_OK;
    LaunchCount lc(idx);
    return run_query(idx, d_queries, lengths, nq, k, d_ids, d_dists, (cudaStream_t)stream);
}

ssh_status ssh_group_query_device(ssh_index* const* handles, int nh, const float* d_queries, const int32_t* lengths,
                                  int64_t nq, int k, int64_t* d_ids, float* d_dists, int32_t* d_which, void* stream) {
    if (!handles || nh < 1 || nq < 0 || (nq > 0 && (!d_queries || !lengths || !d_ids || !d_dists)))
        return fail(SSH_EINVAL, "bad arguments");
    for (int h = 0; h < nh; ++h)
        if (!handles[h]) return fail(SSH_EINVAL, "handle %d is NULL", h);
    if (k < 1 || k > kMaxTopK) return fail(SSH_EINVAL, "k = %d outside [1, %d]", k, kMaxTopK);
    if (nq == 0) return SSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // route every query to the first handle holding series of its length
    std::map<std::pair<int, int>, std::pair<std::vector<const float*>, std::vector<int64_t>>> groups;
    int64_t off = 0;
    for (int64_t i = 0; i < nq; ++i) {
        const int m = lengths[i];
        int owner = -1;
        for (int h = 0; h < nh && owner < 0; ++h) {
            auto it = handles[h]->subs.find(m);
            if (it != handles[h]->subs.end() && it->second.count > 0) owner = h;
        }
        if (m <= 0 || owner < 0)
            return fail(SSH_ELENGTH, "query %lld has length %d, which no handle stores", (long long)i, m);
        auto& g = groups[{owner, m}];
        g.first.push_back(d_queries + off);
        g.second.push_back(i);
        off += m;
    }
    for (auto& kv : groups) {
        ssh_index* idx = handles[kv.first.first];
        SSH_TRY(check_device(idx));
        SSH_CUDA(cudaStreamWaitEvent(st, idx->ready, 0));  // the latest add's tables
        LaunchCount lc(idx);
        SSH_TRY(query_group(idx, idx->subs[kv.first.second], kv.second.first, kv.second.second, k, d_ids, d_dists, st));
        if (d_which) {
            const std::vector<int64_t>& pos = kv.second.second;
            int64_t* d_pos = nullptr;
            SSH_CUDA(cudaMallocAsync(&d_pos, pos.size() * sizeof(int64_t), st));
            cudaError_t e = cudaMemcpyAsync(d_pos, pos.data(), pos.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) {
                fill_i32_kernel<<<grid_for((int64_t)pos.size(), 256, 1024), 256, 0, st>>>(d_which, (int64_t)pos.size(),
                                                                                       d_pos, kv.first.first);
                note_launch();
                e = cudaGetLastError();
            }
            cudaFreeAsync(d_pos, st);
            SSH_CUDA(e);
        }
    }
    SSH_CUDA(cudaStreamSynchronize(st));
    return SSH_OK;
}

ssh_status ssh_set_option(ssh_index* idx, ssh_option opt, int64_t value) {
    if (!idx) return fail(SSH_EINVAL, "NULL index");
    switch (opt) {
        case SSH_OPT_LB_PRUNE:
            idx->lb_prune = value != 0;
            return SSH_OK;
        case SSH_OPT_KERNEL_TIMING:
            idx->timing = value != 0;
            return SSH_OK;
        case SSH_OPT_CWS_FP64:
            idx->cws_fp64 = value != 0;
            return SSH_OK;
        case SSH_OPT_MINHASH: {
            if (value < 0 || value > 1) return fail(SSH_EINVAL, "SSH_OPT_MINHASH takes 0 or 1");
            if (value == 1 && idx->KL > 256)
                return fail(SSH_ENOTSUP, "the one-permutation minhash covers K*L <= 256 (this index: %d)", idx->KL);
            if (value == 1 && idx->n > kMaxShingleBits)
                return fail(SSH_ENOTSUP, "the one-permutation minhash covers n <= %d (this index: %d)",
                            kMaxShingleBits, idx->n);
            for (const auto& kv : idx->subs)
                if (kv.second.count > 0) return fail(SSH_EBUSY, "SSH_OPT_MINHASH changes only an empty index");
            idx->minhash = (int)value;
            return SSH_OK;
        }
        case SSH_OPT_LB_CASCADE:
            if (value < 0 || value > 2) return fail(SSH_EINVAL, "SSH_OPT_LB_CASCADE takes 0, 1 or 2");
            idx->lb_cascade = (int)value;
            return SSH_OK;
        case SSH_OPT_EXACT_SCAN:
            idx->exact_scan = value != 0;
            return SSH_OK;
        case SSH_OPT_HASH_KERNEL:
            if (value < 0 || value > 1) return fail(SSH_EINVAL, "SSH_OPT_HASH_KERNEL takes 0 or 1");
            idx->hash_kernel = (int)value;
            return SSH_OK;
    }
    return fail(SSH_EINVAL, "unknown option %d", (int)opt);
}

ssh_status ssh_get_stats(const ssh_index* idx, ssh_stats* out) {
    if (!idx || !out) return fail(SSH_EINVAL, "NULL argument");
    SSH_CUDA(cudaEventSynchronize(idx->ready));
    unsigned long long dev[kNumStatSlots] = {0};
    SSH_CUDA(cudaMemcpy(dev, idx->d_stats, sizeof(dev), cudaMemcpyDeviceToHost));
    *out = idx->host_stats;
    out->sketch_fp64 = (int64_t)dev[kStatSketch64];
    out->cws_fp64 = (int64_t)dev[kStatCws64];
    return SSH_OK;
}

ssh_status ssh_reset_stats(ssh_index* idx) {
    if (!idx) return fail(SSH_EINVAL, "NULL index");
    SSH_CUDA(cudaMemset(idx->d_stats, 0, kNumStatSlots * sizeof(unsigned long long)));
    idx->host_stats = ssh_stats{};
    for (auto& t : idx->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    idx->pending.clear();
    idx->totals.clear();
    return SSH_OK;
}

ssh_status ssh_get_kernel_times(ssh_index* idx, ssh_kernel_time* out, int cap, int* count) {
    if (!idx || !count || (cap > 0 && !out)) return fail(SSH_EINVAL, "NULL argument");
    for (auto& t : idx->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(t.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.start, t.stop);
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
        if (e != cudaSuccess) return cuda_status(e, "kernel timing events");
        KernelTotals& k = idx->totals[t.name];
        k.launches += t.launches;
        k.calls += 1;
        k.ms += ms;
        k.units += t.units;
    }
    idx->pending.clear();
    int n = 0;
    for (auto& kv : idx->totals) {
        if (n < cap) {
            ssh_kernel_time& o = out[n];
            memset(&o, 0, sizeof(o));
            snprintf(o.name, sizeof(o.name), "%s", kv.first.c_str());
            o.launches = kv.second.launches;
            o.calls = kv.second.calls;
            o.total_ms = kv.second.ms;
            o.units = kv.second.units;
        }
        ++n;
    }
    *count = n;
    return SSH_OK;
}

ssh_status ssh_hash_device(const ssh_index* idx, const float* d_series, int32_t m, int64_t count, void* stream,
                           uint32_t* d_bits, uint32_t* d_sh_ids, uint32_t* d_sh_counts, int32_t* d_nnz,
                           uint32_t* d_kstar, uint32_t* d_tstar, uint64_t* d_keys) {
    if (!idx || count < 0 || (count > 0 && !d_series)) return fail(SSH_EINVAL, "bad arguments");
    if ((d_sh_ids == nullptr) != (d_sh_counts == nullptr) || (d_kstar == nullptr) != (d_tstar == nullptr))
        return fail(SSH_EINVAL, "shingle ids/counts and kstar/tstar come in pairs");
    if (idx->family != 0) return fail(SSH_ENOTSUP, "ssh_hash_device computes SSH hashes; this index is SRP");
    SSH_TRY(check_device(idx));
    Geometry g;
    SSH_TRY(geometry(idx, m, &g));
    HashArgs a = base_hash_args(idx, m, g);
    a.series = d_series;
    a.stride = m;
    a.count = count;
    a.keys = d_keys;
    a.key_stride = count;
    a.key_col0 = 0;
    a.bits_out = d_bits;
    a.sh_ids_out = d_sh_ids;
    a.sh_counts_out = d_sh_counts;
    a.nnz_out = d_nnz;
    a.kstar_out = d_kstar;
    a.tstar_out = d_tstar;
    LaunchCount lc(idx);
    SSH_CUDA(launch_hash(a, (cudaStream_t)stream));
    return SSH_OK;
}

// lb: -1 DTW, 0 LB_Keogh, 1 LB_Keogh with the LB_Kim endpoints, 2 reversed LB_Keogh
static ssh_status pairwise(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                           int64_t npairs, int32_t m, int32_t rb, float* d_out, cudaStream_t st, int lb,
                           const DtwPlan* forced = nullptr) {
    if (npairs < 0 || m < 1 || rb < 0 || rb >= m || (npairs > 0 && (!d_a || !d_a_idx || !d_b || !d_b_idx || !d_out)))
        return fail(SSH_EINVAL, "bad arguments");
    if (npairs == 0) return SSH_OK;
    // group the pairs by a-row on the host: segments of equal a_idx
    std::vector<int64_t> ai(npairs), bi(npairs);
    SSH_CUDA(cudaMemcpyAsync(ai.data(), d_a_idx, npairs * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SSH_CUDA(cudaMemcpyAsync(bi.data(), d_b_idx, npairs * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SSH_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> order(npairs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return ai[x] < ai[y]; });
    std::vector<int64_t> begin;
    std::vector<const float*> sa, pb(npairs);
    std::vector<int64_t> slot(npairs);
    int64_t mx = 0;
    for (int64_t t = 0; t < npairs; ++t) {
        const int64_t p = order[t];
        if (t == 0 || ai[p] != ai[order[t - 1]]) {
            if (!begin.empty()) mx = std::max(mx, t - begin.back());
            begin.push_back(t);
            sa.push_back(d_a + ai[p] * m);
        }
        pb[t] = d_b + bi[p] * m;
        slot[t] = p;
    }
    mx = std::max(mx, npairs - begin.back());
    begin.push_back(npairs);
    const int64_t nseg = (int64_t)sa.size();
    ScratchList sc(st);
    int64_t *dbeg, *dslot;
    const float **dsa, **dpb;
    SSH_TRY(sc.get(&dbeg, nseg + 1));
    SSH_TRY(sc.get(&dslot, npairs));
    SSH_TRY(sc.get(&dsa, nseg));
    SSH_TRY(sc.get(&dpb, npairs));
    SSH_CUDA(cudaMemcpyAsync(dbeg, begin.data(), (nseg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SSH_CUDA(cudaMemcpyAsync(dslot, slot.data(), npairs * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SSH_CUDA(cudaMemcpyAsync(dsa, sa.data(), nseg * sizeof(float*), cudaMemcpyHostToDevice, st));
    SSH_CUDA(cudaMemcpyAsync(dpb, pb.data(), npairs * sizeof(float*), cudaMemcpyHostToDevice, st));
    PairSet ps{dbeg, nseg, dsa, dpb, dslot, mx};
    if (lb == 0 || lb == 1) {
        float *up, *lo;
        SSH_TRY(sc.get(&up, (size_t)nseg * m));
        SSH_TRY(sc.get(&lo, (size_t)nseg * m));
        SSH_CUDA(launch_envelope(dsa, nseg, m, rb, up, lo, st));
        SSH_CUDA(launch_lb_keogh(ps, up, lo, m, d_out, st, lb == 1));
    } else if (lb == 2) {
        SSH_CUDA(launch_lb_rev(ps, m, rb, d_out, nullptr, 1.f, nullptr, nullptr, st));
    } else {
        cudaError_t e = launch_dtw_plan(ps, m, rb, forced ? *forced : dtw_tuned_plan(m, rb, st), d_out, st);
        if (e == cudaErrorNotSupported) return fail(SSH_ENOTSUP, "DTW radius %d is wider than the compiled DTW tilings cover", rb);
        SSH_CUDA(e);
    }
    SSH_CUDA(cudaStreamSynchronize(st));
    return SSH_OK;
}

ssh_status ssh_dtw_device(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                          int64_t npairs, int32_t m, int32_t rb, float* d_out, void* stream) {
    return pairwise(d_a, d_a_idx, d_b, d_b_idx, npairs, m, rb, d_out, (cudaStream_t)stream, -1);
}

ssh_status ssh_dtw_device_tiled(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                                int64_t npairs, int32_t m, int32_t rb, int32_t S, int32_t variant, float* d_out,
                                void* stream) {
    if (rb < 0 || rb >= m) return fail(SSH_EINVAL, "bad arguments");
    const DtwPlan pl = dtw_plan_for(rb, S, variant);
    if (pl.S == 0)
        return fail(SSH_ENOTSUP, "no compiled DTW tiling with S = %d, variant %d at radius %d", (int)S, (int)variant,
                    (int)rb);
    return pairwise(d_a, d_a_idx, d_b, d_b_idx, npairs, m, rb, d_out, (cudaStream_t)stream, -1, &pl);
}

ssh_status ssh_lb_keogh_device(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                               int64_t npairs, int32_t m, int32_t rb, float* d_out, void* stream) {
    return pairwise(d_a, d_a_idx, d_b, d_b_idx, npairs, m, rb, d_out, (cudaStream_t)stream, 0);
}

ssh_status ssh_lb_bound_device(const float* d_a, const int64_t* d_a_idx, const float* d_b, const int64_t* d_b_idx,
                               int64_t npairs, int32_t m, int32_t rb, int32_t kind, float* d_out, void* stream) {
    if (kind < 0 || kind > 2) return fail(SSH_EINVAL, "LB kind %d is not 0, 1 or 2", (int)kind);
    return pairwise(d_a, d_a_idx, d_b, d_b_idx, npairs, m, rb, d_out, (cudaStream_t)stream, kind);
}

}  // extern "C"
