// batch_rerank.cu -- the reporting step of Algorithm 2 for a whole mixed-length
// batch as one persistent launch: LB_Keogh of every candidate (Sec. 3, with the
// LB_Kim endpoint costs), the seeds (the kSeedFactor k smallest bounds) and
// their banded DTW (Sec. 2.1), the bound U (the k-th smallest seed distance),
// the survivors' DTW with early abandoning, and the top-k, for the queries of
// every length class. The work of a phase is split into items that the blocks
// claim from a counter, the largest length class first and, within a class,
// chunk by chunk across its queries (chunk c of every query, then chunk c + 1:
// the candidates are in row order, so the blocks at work read nearby rows and
// share them in L2); the phases are separated
// by a grid barrier (the launch is cooperative, so every block is resident);
// DTW items run the tiling the library's autotuner chose for their class. The
// arithmetic is the one of the per-class kernels (the same LB loop, the same
// wavefront device function, the same selections), so results are identical.
//
// Phases (q: a sorted query of the batch; pairs [sb, se) its candidates):
//  0 envelopes of every query; block 0 also lays out the LB items of each class
//  1 LB_Keogh items: (q, 64 pairs)
//  2 per query: T = (kSeedFactor k)-th smallest LB; seed count (lb <= T)
//  3 block 0: offsets of the seed lists, and the DTW items of each class
//  4 per query: the seeds into fb / fslot at their offsets
//  5 seed DTW items: (q, a chunk sized to the class's lane groups)
//  6 per query: U = k-th smallest distance; survivor count (T < lb, lb (1 - eta) <= U)
//  7 block 0: offsets of the survivor lists, and their DTW items
//  8 per query: the survivors into fb / fslot
//  9 survivor DTW items, abandoning against U
// 10 per query: the top-k (distance, row) keys, ordered, written at the caller's position
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dtw_wave.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLbChunk = 64;                 // pairs per LB item (8 per warp)
constexpr int kLbLoads = 32;                 // candidate loads in flight per lane in the LB loop
constexpr int kDtwPairsPerGroup = 16;        // pairs per lane group in one DTW item
constexpr long long kBarrierSpins = 1ll << 26;  // about 4 s of 64 ns sleeps, then the launch gives up
constexpr unsigned kFullMask = 0xFFFFFFFFu;

// Grid barrier over co-resident blocks: arrive on st[0], the last block resets it
// and bumps the generation st[1]. A wait that runs out of spins sets *err and
// returns; every block checks *err after each barrier and leaves.
__device__ bool grid_barrier(unsigned* st, unsigned nblocks, unsigned* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = st + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(st, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(st, 0u);
            __threadfence();
            atomicAdd(st + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (++spins > kBarrierSpins || *(volatile unsigned*)err) {
                    atomicExch(err, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile unsigned*)err == 0u;
}

// Next item of a phase (one claim per block, broadcast through shared memory).
__device__ __forceinline__ long long claim(unsigned long long* ctr, long long* s_item) {
    __syncthreads();
    if (threadIdx.x == 0) *s_item = (long long)atomicAdd(ctr, 1ull);
    __syncthreads();
    return *s_item;
}

// The k-th smallest (1-based) of n keys key(i), i in [0, n), by 8-bit radix
// passes over the block (all ones when n < k). Called by the whole block.
template <typename T, typename F>
__device__ T block_select_kth(int64_t n, int k, F key, uint32_t* hist, T* s_prefix, uint32_t* s_rem) {
    constexpr int kBits = sizeof(T) * 8;
    if (n < k) return ~(T)0;
    if (threadIdx.x == 0) {
        *s_prefix = 0;
        *s_rem = (uint32_t)k;
    }
    T mask = 0;
    for (int shift = kBits - 8; shift >= 0; shift -= 8) {
        for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0u;
        __syncthreads();
        const T prefix = *s_prefix;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const T v = key(i);
            if ((v & mask) == prefix) atomicAdd(&hist[(uint32_t)(v >> shift) & 0xFFu], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t rem = *s_rem;
            int d = 0;
            for (; d < 256; ++d) {
                if (hist[d] >= rem) break;
                rem -= hist[d];
            }
            *s_rem = rem;
            *s_prefix = prefix | ((T)d << shift);
        }
        mask |= ((T)0xFF << shift);
        __syncthreads();
    }
    return *s_prefix;
}

// Exclusive prefix sums of v(i), i in [0, n), into out[0 .. n] by one block.
template <typename F>
__device__ void block_scan(int64_t n, F v, int64_t* out, int64_t* part) {
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += v(i);
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int64_t x = part[t];
            part[t] = run;
            run += x;
        }
        out[n] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        out[i] = run;
        run += v(i);
    }
    __syncthreads();
}

// Items a query's list of `cnt` entries makes, `per` entries each.
__device__ __forceinline__ int64_t items_of(int64_t cnt, int64_t per) { return (cnt + per - 1) / per; }

// Item layout of a phase (block 0): class j of the processing order is c = C-1-j
// (longest series first); its items are (chunk, query) with the query fastest,
// as many chunks as its longest list (shorter lists leave empty items).
// off[j] = first item of the j-th class processed, off[C] = all items.
template <typename F>
__device__ void layout_items(int C, const int64_t* cls_begin, F chunks, int64_t* off, int64_t* part) {
    if (threadIdx.x == 0) off[0] = 0;
    for (int j = 0; j < C; ++j) {
        const int c = C - 1 - j;
        const int64_t q0 = cls_begin[c], q1 = cls_begin[c + 1];
        int64_t mx = 0;
        for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) mx = max(mx, chunks(q, c));
        part[threadIdx.x] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 1; t < (int)blockDim.x; ++t) mx = max(mx, part[t]);
            mx = max(mx, part[0]);
            off[j + 1] = off[j] + mx * (q1 - q0);
        }
        __syncthreads();
    }
}

// Item u of a phase laid out by layout_items: its query and chunk (chunk = -1: none).
__device__ __forceinline__ void item_of(int64_t u, int C, const int64_t* cls_begin, const int64_t* off, int64_t* q,
                                        int64_t* chunk, int* cls) {
    int j = 0;
    while (j + 1 < C && off[j + 1] <= u) ++j;
    const int c = C - 1 - j;
    const int64_t q0 = cls_begin[c], nqc = cls_begin[c + 1] - q0;
    const int64_t local = u - off[j];
    *cls = c;
    *q = q0 + local % nqc;
    *chunk = local / nqc;
}

template <int S, int PM>
__device__ __noinline__ void dtw_item(const float* q_s, const float* qg, int m, int rb, int G,
                                      const float* const* pair_b, const int64_t* pair_slot, int64_t b1,
                                      unsigned long long* s_next, float bound, float shrink, float* out) {
    wave::dtw_wave_pairs<S, PM>(q_s, qg, m, rb, G, pair_b, pair_slot, b1, s_next, bound, shrink, out, nullptr);
}

// The class's compiled tiling (S, pmask) for the pairs [*s_next, b1).
__device__ void dtw_dispatch(const RerankClass& c, const float* q_s, const float* qg, const float* const* pair_b,
                             const int64_t* pair_slot, int64_t b1, unsigned long long* s_next, float bound,
                             float shrink, float* out) {
#define SSH_RR_CASE(SS, PP)                                                                                 \
    if (c.S == SS && c.pmask == PP) {                                                                       \
        dtw_item<SS, PP>(q_s, qg, c.m, c.rb, c.G, pair_b, pair_slot, b1, s_next, bound, shrink, out);     \
        return;                                                                                             \
    }
    SSH_RR_CASE(8, 0) SSH_RR_CASE(8, 2) SSH_RR_CASE(8, 4) SSH_RR_CASE(8, 6)
    SSH_RR_CASE(14, 0) SSH_RR_CASE(14, 2) SSH_RR_CASE(14, 4) SSH_RR_CASE(14, 6) SSH_RR_CASE(14, 8)
    SSH_RR_CASE(14, 10) SSH_RR_CASE(14, 12)
    SSH_RR_CASE(26, 0) SSH_RR_CASE(26, 2) SSH_RR_CASE(26, 4) SSH_RR_CASE(26, 6) SSH_RR_CASE(26, 8)
    SSH_RR_CASE(26, 10) SSH_RR_CASE(26, 12) SSH_RR_CASE(26, 14) SSH_RR_CASE(26, 16) SSH_RR_CASE(26, 18)
    SSH_RR_CASE(26, 20) SSH_RR_CASE(26, 22) SSH_RR_CASE(26, 24)
#undef SSH_RR_CASE
}

__global__ void __launch_bounds__(kThreads, 2) rerank_kernel(RerankArgs a) {
    extern __shared__ __align__(16) float rsm[];  // [max(2, kWarps) max_m]: an envelope, or a query per warp
    __shared__ uint32_t hist[256];
    __shared__ uint64_t s_prefix64;
    __shared__ uint32_t s_prefix32, s_rem;
    __shared__ long long s_item;
    __shared__ unsigned long long w_next[kWarps];  // next unclaimed pair of each warp's DTW item
    __shared__ int64_t part[kThreads];
    __shared__ uint64_t topbuf[kMaxTopK];
    __shared__ int s_cnt;
    // every argument in a register of its own (lambdas capture these by value)
    const int32_t* q_cls = a.q_cls;
    const float* const* q_ptr = a.q_ptr;
    const RerankClass* cls = a.cls;
    const int64_t* seg_begin = a.seg_begin;
    const float** pair_b = a.pair_b;
    const uint32_t* cand_rows = a.cand_rows;
    float* upper = a.upper;
    float* lower = a.lower;
    const int64_t env_stride = a.env_stride;
    float* lb = a.lb;
    float* dist = a.dist;
    const float** fb = a.fb;
    int64_t* fslot = a.fslot;
    int64_t* fcount = a.fcount;
    unsigned long long* fcursor = a.fcursor;
    int64_t* fbegin = a.fbegin;
    const int64_t* cls_begin = a.cls_begin;
    const int C = a.C;
    int64_t* lb_off = a.item_off;            // [C + 1] LB items
    int64_t* dtw_off = a.item_off + (C + 1);  // [C + 1] DTW items of the current pass
    uint32_t* Tq = a.T;
    uint32_t* Uq = a.U;
    const int k = a.k;
    const float shrink = a.shrink;
    unsigned long long* dtw_counts = a.dtw_counts;
    unsigned long long* work = a.work;
    unsigned* bar = a.bar;
    unsigned* err = a.err;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (*a.overflow) return;  // the candidates did not fit: nothing is ranked (uniform)
    const int64_t nq = *a.nq;
    const float INF = __int_as_float(0x7F800000);

    // ---- phase 0: envelopes; block 0 first lays out the LB items
    if (blockIdx.x == 0)
        layout_items(C, cls_begin, [=](int64_t q, int) { return items_of(seg_begin[q + 1] - seg_begin[q], kLbChunk); },
                     lb_off, part);
    for (long long it = claim(&work[0], &s_item); it < nq; it = claim(&work[0], &s_item)) {
        const int64_t q = nq - 1 - it;
        const RerankClass c = cls[q_cls[q]];
        const float* qg = q_ptr[q];
        for (int i = threadIdx.x; i < c.m; i += blockDim.x) {
            const int lo = max(0, i - c.rb), hi = min(c.m - 1, i + c.rb);
            float u = qg[lo], l = qg[lo];
            for (int t = lo + 1; t <= hi; ++t) {
                const float v = qg[t];
                u = fmaxf(u, v);
                l = fminf(l, v);
            }
            upper[q * env_stride + i] = u;
            lower[q * env_stride + i] = l;
        }
    }
    if (!grid_barrier(bar, nblocks, err)) return;

    // ---- phase 1: LB_Keogh with the LB_Kim endpoints, 64 pairs per item (8 per warp)
    {
        const int64_t nitems = lb_off[C];
        int64_t staged = -1;
        for (long long it = claim(&work[1], &s_item); it < nitems; it = claim(&work[1], &s_item)) {
            int64_t q, chunk;
            int ci;
            item_of(it, C, cls_begin, lb_off, &q, &chunk, &ci);
            const int64_t sb = seg_begin[q] + chunk * kLbChunk;
            const int64_t se = min(seg_begin[q + 1], sb + kLbChunk);
            if (sb >= se) continue;  // an empty item (uniform over the block)
            const int m = cls[ci].m;
            if (q != staged) {  // uniform over the block (the claim synchronised it)
                const float* qa = q_ptr[q];
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    const bool endpoint = (i == 0 || i == m - 1);
                    rsm[i] = endpoint ? qa[i] : upper[q * env_stride + i];
                    rsm[m + i] = endpoint ? qa[i] : lower[q * env_stride + i];
                }
                staged = q;
                __syncthreads();
            }
            // two pairs per warp at a time, kLbLoads / 2 loads of each in flight per lane (this
            // kernel runs 16 warps per SM); each lane adds its terms in sample order, as the
            // per-class kernel does, so the bounds are the same bits
            for (int64_t p0 = sb + warp; p0 < se; p0 += 2 * kWarps) {
                const int64_t p1 = p0 + kWarps;
                const bool two = p1 < se;  // uniform over the warp
                const float* ca = pair_b[p0];
                const float* cb = two ? pair_b[p1] : ca;
                float acc0 = 0.f, acc1 = 0.f;
                int i = lane;
                constexpr int kH = kLbLoads / 2;
                for (; i + 32 * (kH - 1) < m; i += 32 * kH) {
                    float va[kH], vb[kH];
#pragma unroll
                    for (int t = 0; t < kH; ++t) va[t] = __ldg(ca + i + 32 * t);
#pragma unroll
                    for (int t = 0; t < kH; ++t) vb[t] = __ldg(cb + i + 32 * t);
#pragma unroll
                    for (int t = 0; t < kH; ++t) {
                        const int j = i + 32 * t;
                        const float up = rsm[j], lo = rsm[m + j];
                        const float du = va[t] - up, dl = va[t] - lo;
                        const float d = du > 0.f ? du : (dl < 0.f ? dl : 0.f);
                        acc0 = fmaf(d, d, acc0);
                        const float eu = vb[t] - up, el = vb[t] - lo;
                        const float e = eu > 0.f ? eu : (el < 0.f ? el : 0.f);
                        acc1 = fmaf(e, e, acc1);
                    }
                }
                for (; i < m; i += 32) {
                    const float up = rsm[i], lo = rsm[m + i];
                    const float va = __ldg(ca + i), vb = __ldg(cb + i);
                    const float du = va - up, dl = va - lo;
                    const float d = du > 0.f ? du : (dl < 0.f ? dl : 0.f);
                    acc0 = fmaf(d, d, acc0);
                    const float eu = vb - up, el = vb - lo;
                    const float e = eu > 0.f ? eu : (el < 0.f ? el : 0.f);
                    acc1 = fmaf(e, e, acc1);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    acc0 += __shfl_xor_sync(kFullMask, acc0, o);
                    acc1 += __shfl_xor_sync(kFullMask, acc1, o);
                }
                if (lane == 0) {
                    lb[p0] = acc0;
                    if (two) lb[p1] = acc1;
                }
            }
        }
    }
    if (!grid_barrier(bar, nblocks, err)) return;

    for (int mode = 0; mode < 2; ++mode) {
        // ---- phase 2 / 6: the bound (T, then U) and the size of the pass's list
        for (long long it = claim(&work[2 + 4 * mode], &s_item); it < nq; it = claim(&work[2 + 4 * mode], &s_item)) {
            const int64_t q = nq - 1 - it;
            const int64_t sb = seg_begin[q], se = seg_begin[q + 1];
            if (mode == 0) {
                const uint32_t t = block_select_kth<uint32_t>(
                    se - sb, kSeedFactor * k, [=](int64_t i) { return __float_as_uint(lb[sb + i]); }, hist,
                    &s_prefix32, &s_rem);
                if (threadIdx.x == 0) Tq[q] = t;
            } else {
                const uint32_t u = block_select_kth<uint32_t>(
                    se - sb, k, [=](int64_t i) { return __float_as_uint(dist[sb + i]); }, hist, &s_prefix32, &s_rem);
                if (threadIdx.x == 0) Uq[q] = u;
            }
            __syncthreads();
            const uint32_t tb = Tq[q];
            const float t = (tb == 0xFFFFFFFFu) ? INF : __uint_as_float(tb);
            const float ub = mode ? __uint_as_float(Uq[q]) : 0.f;
            int64_t cnt = 0;
            for (int64_t p = sb + threadIdx.x; p < se; p += blockDim.x) {
                const float v = lb[p];
                cnt += mode == 0 ? (v <= t) : (v > t && v * shrink <= ub);
            }
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFullMask, cnt, o);
            if (lane == 0) part[warp] = cnt;
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t tot = 0;
                for (int w = 0; w < kWarps; ++w) tot += part[w];
                fcount[q] = tot;
                fcursor[q] = 0ull;
                if (tot) atomicAdd(&dtw_counts[mode], (unsigned long long)tot);
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, nblocks, err)) return;

        // ---- phase 3 / 7: offsets of the lists and the layout of their DTW items (block 0)
        if (blockIdx.x == 0) {
            block_scan(nq, [=](int64_t q) { return fcount[q]; }, fbegin, part);
            layout_items(C, cls_begin, [=](int64_t q, int c) { return items_of(fcount[q], cls[c].dtw_chunk); },
                         dtw_off, part);
        }
        if (!grid_barrier(bar, nblocks, err)) return;

        // ---- phase 4 / 8: the pass's pairs into fb / fslot
        for (long long it = claim(&work[3 + 4 * mode], &s_item); it < nq; it = claim(&work[3 + 4 * mode], &s_item)) {
            const int64_t q = nq - 1 - it;
            const int64_t sb = seg_begin[q], se = seg_begin[q + 1];
            const uint32_t tb = Tq[q];
            const float t = (tb == 0xFFFFFFFFu) ? INF : __uint_as_float(tb);
            const float ub = mode ? __uint_as_float(Uq[q]) : 0.f;
            const int64_t base = fbegin[q];
            for (int64_t p = sb + threadIdx.x; p < se; p += blockDim.x) {
                const float v = lb[p];
                const bool keep = mode == 0 ? (v <= t) : (v > t && v * shrink <= ub);
                if (keep) {
                    const int64_t at = base + (int64_t)atomicAdd(&fcursor[q], 1ull);
                    fb[at] = pair_b[p];
                    fslot[at] = p;
                }
            }
        }
        if (!grid_barrier(bar, nblocks, err)) return;

        // ---- phase 5 / 9: DTW items at the class's tiling, claimed by single warps (each with
        // its own copy of its query), so a warp whose pairs end early takes the next item
        // instead of waiting for the block
        {
            const int64_t nitems = dtw_off[C];
            float* wq = rsm + (size_t)warp * env_stride;
            int64_t staged = -1;
            while (true) {
                unsigned long long it = 0;
                if (lane == 0) it = atomicAdd(&work[4 + 4 * mode], 1ull);
                it = __shfl_sync(kFullMask, it, 0);
                if ((int64_t)it >= nitems) break;
                int64_t q, chunk;
                int ci;
                item_of((int64_t)it, C, cls_begin, dtw_off, &q, &chunk, &ci);
                const RerankClass c = cls[ci];
                const int64_t f0 = fbegin[q] + chunk * c.dtw_chunk;
                const int64_t f1 = min(fbegin[q + 1], f0 + c.dtw_chunk);
                if (f0 >= f1) continue;  // an empty item (uniform over the warp)
                const float* qg = q_ptr[q];
                if (q != staged) {
                    for (int i = lane; i < c.m; i += 32) wq[i] = qg[i];
                    staged = q;
                }
                if (lane == 0) w_next[warp] = (unsigned long long)f0;
                __syncwarp();
                float bound = INF;
                if (mode == 1 && Uq[q] != 0xFFFFFFFFu) bound = __uint_as_float(Uq[q]);
                dtw_dispatch(c, wq, qg, fb, fslot, f1, &w_next[warp], bound, shrink, dist);
                __syncwarp();
            }
        }
        if (!grid_barrier(bar, nblocks, err)) return;
    }

    // ---- phase 10: top-k by (distance, row), written at the caller's position
    const TopkOut& o = a.out;
    for (long long it = claim(&work[10], &s_item); it < nq; it = claim(&work[10], &s_item)) {
        const int64_t q = nq - 1 - it;
        const int64_t sb = seg_begin[q], se = seg_begin[q + 1];
        auto key = [=](int64_t i) {
            return ((uint64_t)__float_as_uint(dist[sb + i]) << 32) | (uint64_t)cand_rows[sb + i];
        };
        const uint64_t lim = block_select_kth<uint64_t>(se - sb, k, key, hist, &s_prefix64, &s_rem);
        if (threadIdx.x == 0) s_cnt = 0;
        for (int i = threadIdx.x; i < kMaxTopK; i += blockDim.x) topbuf[i] = ~0ull;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < se - sb; i += blockDim.x) {
            const uint64_t v = key(i);
            if (v <= lim) {
                const int at = atomicAdd(&s_cnt, 1);
                if (at < kMaxTopK) topbuf[at] = v;
            }
        }
        __syncthreads();
        int n2 = 1;
        while (n2 < k) n2 <<= 1;
        for (int kk = 2; kk <= n2; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const uint64_t x = topbuf[i], y = topbuf[l];
                        const bool up = (i & kk) == 0;
                        if ((x > y) == up) {
                            topbuf[i] = y;
                            topbuf[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        const int64_t* gid = o.seg_gid ? o.seg_gid[q] : o.gid;
        const int64_t out0 = o.qpos[q] * (int64_t)k;
        for (int t = threadIdx.x; t < k; t += blockDim.x) {
            const uint64_t v = topbuf[t];
            const uint32_t dbits = (uint32_t)(v >> 32);
            const bool real = (v != ~0ull) && dbits < 0x7F800000u;
            o.ids[out0 + t] = real ? gid[(uint32_t)v] : -1;
            o.dists[out0 + t] = real ? __uint_as_float(dbits) : INF;
        }
        if (o.which && threadIdx.x == 0) o.which[o.qpos[q]] = o.seg_which[q];
    }
}

}  // namespace

size_t rerank_smem_bytes(int max_m) { return (size_t)kWarps * (size_t)std::max(max_m, 1) * sizeof(float); }

int rerank_dtw_chunk(const DtwPlan& pl) {
    // kDtwPairsPerGroup pairs per lane group of a warp: a group that finishes early (its
    // pairs abandoned) takes the next pair of the item instead of waiting for the others
    return kDtwPairsPerGroup * (32 / std::max(pl.G, 1));
}

cudaError_t launch_rerank(const RerankArgs& a, int max_m, cudaStream_t st, int* grid_out) {
    const size_t smem = rerank_smem_bytes(max_m);
    cudaError_t e = ensure_dynamic_smem((const void*)rerank_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rerank_kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)(sms * per_sm);
    if (grid_out) *grid_out = (int)grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, rerank_kernel, a);
    note_launch();
    return e;
}

}  // namespace ssh
