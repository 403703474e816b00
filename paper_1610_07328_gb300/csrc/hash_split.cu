// hash_split.cu -- the hash path for the compiled-in shapes as two kernels and
// a fix-up (Sec. 4.1-4.3 and the keys of Algorithm 1):
//
//  sketch_kernel<W, DELTA, R>: one warp per series at a time (persistent, with
//    the next series staged into shared memory by cp.async while the current
//    one is processed). Lane l owns the R consecutive windows [lR, lR + R); the
//    filter r sits in registers and the loop over the lane's W + (R-1) DELTA
//    samples is unrolled, so each sample read from shared memory feeds up to R
//    FMAs. A window whose |r.x| is not above tau ||r|| ||x_series|| is checked
//    again against its own energy tau ||r|| ||x_window||; if it stays below, it
//    goes to a fix-up list with a provisional bit 0. Bits are packed 32 per
//    word (window i -> bit 31 - i%32 of word i/32) into global memory.
//  sketch_fixup_kernel: one thread per listed window recomputes the dot product
//    in FP64 in the definition's order and sets the bit when it is >= 0.
//  shingle_cws_kernel<E>: one warp per series: the S = N_B - n + 1 shingle ids
//    (first bit most significant) are sorted by a bitonic network over 32E
//    registers with warp shuffles and run-length encoded with a ballot scan;
//    each lane then owns 4 consecutive hash functions: one 64-bit load brings
//    the 4 exact count-1 ranks of a shingle and SIMD u16 mins keep the minima,
//    repeated shingles go through the certified FP32 interval track, and an
//    uncertain hash is recomputed in FP64 (hash_common.cuh). Its shared memory
//    is small, so many warps per SM hide the L2 latency of the rank lookups.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hash_common.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSketchWarps = 8;
constexpr int kCwsWarps = 8;

__host__ __device__ inline int a16(int b) { return (b + 15) & ~15; }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ const float* row_ptr(const HashArgs& a, int64_t row) {
    return a.rows ? a.rows[row] : a.series + row * a.stride;
}

// Start copying series `row` into dst (m floats); misaligned rows load synchronously.
__device__ __forceinline__ void fetch_row(const HashArgs& a, int64_t row, float* dst, int lane) {
    const float* src = row_ptr(a, row);
    const int m = a.m;
    if (((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (m & 3) == 0) {
        for (int c = lane; c < (m >> 2); c += 32) cp_async16(dst + 4 * c, src + 4 * c);
    } else {
        for (int i = lane; i < m; i += 32) dst[i] = __ldg(src + i);
    }
}

__host__ __device__ inline int sketch_xb(int m, int W, int DELTA, int R) {
    int xb = m;
    const int need = 32 * R * DELTA + W;  // samples read by the padded windows of the last lanes
    if (need > xb) xb = need;
    return (xb + 3) & ~3;
}

// The filter as a by-value kernel parameter: it sits in the constant bank and
// every FMA reads its tap from there, leaving the registers to the windows.
template <int W>
struct FilterParam {
    float v[W];
};

// Provisional bits go to `bits`; windows needing FP64 go to fix[0..cap) as
// (row << 16 | window), counted in *nfix. If the list is full the window is
// recomputed in place.
template <int W, int DELTA, int R>
__global__ void __launch_bounds__(kSketchWarps * 32, 3)
    sketch_kernel(HashArgs a, const FilterParam<W> rp, uint32_t* bits, unsigned long long* fix,
                  unsigned long long fix_cap, unsigned long long* nfix) {
    constexpr int STRIP = W + (R - 1) * DELTA;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = a.m, nb = a.nb, nwords = a.nwords;
    const int xb = sketch_xb(m, W, DELTA, R);
    float* r_s = reinterpret_cast<float*>(smem);
    unsigned char* wb = smem + a16(4 * W) + (size_t)warp * (2 * a16(4 * xb) + a16(32 * R));
    float* xbuf[2] = {reinterpret_cast<float*>(wb), reinterpret_cast<float*>(wb + a16(4 * xb))};
    unsigned char* bytes = wb + 2 * a16(4 * xb);
    for (int j = threadIdx.x; j < W; j += blockDim.x) r_s[j] = a.r[j];
    for (int i = m + lane; i < xb; i += 32) {  // samples past the end feed only windows past N_B
        xbuf[0][i] = 0.f;
        xbuf[1][i] = 0.f;
    }
    __syncthreads();

    const int64_t nwarps = (int64_t)gridDim.x * kSketchWarps;
    const int64_t first = (int64_t)blockIdx.x * kSketchWarps + warp;
    unsigned long long n_inplace = 0;
    if (first < a.count) fetch_row(a, first, xbuf[0], lane);
    cp_async_commit();
    int it = 0;
    for (int64_t row = first; row < a.count; row += nwarps, ++it) {
        const int cur = it & 1;
        if (row + nwarps < a.count) fetch_row(a, row + nwarps, xbuf[cur ^ 1], lane);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const float* x = xbuf[cur];
        // series energy: ||x_window||^2 <= sum over the series; the loose test uses it
        float e = 0.f;
        for (int i = lane; i < m; i += 32) e = fmaf(x[i], x[i], e);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(kFull, e, o);
        // e carries at most (m/32 + 5) roundings of relative 2^-24 each; inflate by 2m 2^-24
        const float e_up = __fmul_ru(e, 1.0f + (float)(2 * m + 64) * 5.9604645e-08f);
        const float thr_loose = __fmul_ru(a.tau_norm, __fsqrt_ru(__fmul_ru(e_up, 1.0f + a.gamma_ss)));

        float acc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = 0.f;
        const float* xs = x + lane * R * DELTA;
#pragma unroll
        for (int t = 0; t < STRIP; ++t) {
            const float xv = xs[t];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int j = t - k * DELTA;
                if (j >= 0 && j < W) acc[k] = fmaf(rp.v[j], xv, acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int i = lane * R + k;
            uint8_t bit = 0;
            if (i < nb) {
                if (fabsf(acc[k]) > thr_loose) {
                    bit = acc[k] >= 0.f;
                } else {
                    // the window's own energy (sequential FMAs: at most W roundings)
                    const float* xw = xs + k * DELTA;
                    float ss = 0.f;
#pragma unroll 1
                    for (int j = 0; j < W; ++j) ss = fmaf(xw[j], xw[j], ss);
                    const float thr = __fmul_ru(a.tau_norm, __fsqrt_ru(__fmul_ru(ss, 1.0f + a.gamma_ss)));
                    if (fabsf(acc[k]) > thr) {
                        bit = acc[k] >= 0.f;
                    } else {
                        const unsigned long long slot = atomicAdd(nfix, 1ull);
                        if (slot < fix_cap) {
                            fix[slot] = ((unsigned long long)row << 16) | (unsigned long long)i;
                        } else {
                            double d = 0.0;  // list full: the definition's FP64 order, in place
#pragma unroll 1
                            for (int j = 0; j < W; ++j) d = fma((double)r_s[j], (double)xw[j], d);
                            bit = d >= 0.0;
                            n_inplace += 1;
                        }
                    }
                }
            }
            bytes[lane * R + k] = bit;
        }
        __syncwarp();
        uint32_t* out = bits + row * nwords;
        for (int w = lane; w < nwords; w += 32) {
            uint32_t word = 0;
            const uint32_t* b4 = reinterpret_cast<const uint32_t*>(bytes) + w * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t v = (w * 32 + q * 4 < 32 * R) ? b4[q] : 0u;
                word |= (((v * 0x08040201u) >> 24) & 0xFu) << (28 - 4 * q);  // bytes 0..3 -> bits 3..0
            }
            out[w] = word;
        }
        __syncwarp();
    }
    if (n_inplace && a.stats) atomicAdd(&a.stats[kStatSketch64], n_inplace);
}

// One thread per listed window: FP64 in the definition's order (the FP32 x FP32
// products are exact in FP64, so an FMA equals the separate multiply and add).
__global__ void sketch_fixup_kernel(HashArgs a, uint32_t* bits, const unsigned long long* fix,
                                    const unsigned long long* nfix, unsigned long long cap) {
    const unsigned long long n = min(*nfix, cap);
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long v = fix[t];
        const int64_t row = (int64_t)(v >> 16);
        const int i = (int)(v & 0xFFFFu);
        const float* xw = row_ptr(a, row) + i * a.delta;
        double d = 0.0;
        for (int j = 0; j < a.W; ++j) d = fma((double)a.r[j], (double)xw[j], d);
        if (d >= 0.0) atomicOr(&bits[row * a.nwords + (i >> 5)], 1u << (31 - (i & 31)));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats && n) atomicAdd(&a.stats[kStatSketch64], n);
}

// Per-series weighted set as written by shingle_kernel: S slots of u32, the n1
// shingles seen once first (id), then the nm repeated ones (id | count << 16),
// each group in ascending id order; sizes[row] = (n1, nm).
__device__ __forceinline__ uint32_t set_id(uint32_t v) { return v & 0xFFFFu; }
__device__ __forceinline__ uint32_t set_count(uint32_t v) { return v >> 16; }

struct ShingleLayout {
    int bits, hpos, cid, total;
};

__host__ __device__ inline ShingleLayout shingle_layout(int nwords, int S) {
    ShingleLayout L;
    int off = 0;
    L.bits = off; off += a16(4 * (nwords + 2));
    L.hpos = off; off += a16(4 * (S + 1));
    L.cid = off; off += a16(4 * S);
    L.total = off;
    return L;
}

template <int E>
__global__ void __launch_bounds__(kCwsWarps * 32) shingle_kernel(HashArgs a, const uint32_t* gbits, uint32_t* sets,
                                                                  int2* sizes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwords = a.nwords, S = a.S, n = a.n;
    const ShingleLayout lay = shingle_layout(nwords, S);
    unsigned char* wb = smem + (size_t)warp * lay.total;
    uint32_t* bits = reinterpret_cast<uint32_t*>(wb + lay.bits);
    int* hpos = reinterpret_cast<int*>(wb + lay.hpos);
    uint32_t* cid = reinterpret_cast<uint32_t*>(wb + lay.cid);
    const int64_t nwarps = (int64_t)gridDim.x * kCwsWarps;
    for (int64_t row = (int64_t)blockIdx.x * kCwsWarps + warp; row < a.count; row += nwarps) {
        for (int w = lane; w < nwords + 2; w += 32) bits[w] = (w < nwords) ? __ldg(gbits + row * nwords + w) : 0u;
        __syncwarp();
        int nnz;
        {
            uint32_t v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane * E + e;
                uint32_t id = 0xFFFFFFFFu;
                if (i < S) {
                    const uint64_t bb = ((uint64_t)bits[i >> 5] << 32) | (uint64_t)bits[(i >> 5) + 1];
                    id = (uint32_t)((bb << (i & 31)) >> (64 - n));
                }
                v[e] = id;
            }
            // bitonic sort, ascending; element index i = lane*E + e (blocked layout)
#pragma unroll
            for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    if (j < E) {
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            const int p = e ^ j;
                            if (p > e) {
                                const bool up = (((lane * E + e) & k) == 0);
                                const uint32_t lo = min(v[e], v[p]), hi = max(v[e], v[p]);
                                v[e] = up ? lo : hi;
                                v[p] = up ? hi : lo;
                            }
                        }
                    } else {
                        const int lm = j / E;
                        const bool lower = (lane & lm) == 0;
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            const uint32_t o = __shfl_xor_sync(kFull, v[e], lm);
                            const bool up = (((lane * E + e) & k) == 0);
                            v[e] = (up == lower) ? min(v[e], o) : max(v[e], o);
                        }
                    }
                }
            }
            // run-length encoding: run heads and their positions by a warp scan
            const uint32_t prev = __shfl_up_sync(kFull, v[E - 1], 1);
            int nh = 0;
            bool head[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane * E + e;
                head[e] = (i < S) && (i == 0 || v[e] != ((e == 0) ? prev : v[e - 1]));
                nh += head[e];
            }
            int incl = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            int pos = incl - nh;
            nnz = __shfl_sync(kFull, incl, 31);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (head[e]) {
                    cid[pos] = v[e];
                    hpos[pos] = lane * E + e;
                    ++pos;
                }
        }
        __syncwarp();
        // counts, then the set in two ascending groups: seen once, seen more than once
        uint32_t* out = sets + row * S;
        int n1 = 0, nm = 0;
        for (int e0 = 0; e0 < nnz; e0 += 32) {
            const int e = e0 + lane;
            uint32_t c = 0, id = 0;
            if (e < nnz) {
                c = (uint32_t)(((e + 1 < nnz) ? hpos[e + 1] : S) - hpos[e]);
                id = cid[e];
                if (a.sh_ids_out) {
                    a.sh_ids_out[row * S + e] = id;
                    a.sh_counts_out[row * S + e] = c;
                }
            }
            const bool one = (e < nnz) && c == 1u, more = (e < nnz) && c > 1u;
            const unsigned b1 = __ballot_sync(kFull, one), bm = __ballot_sync(kFull, more);
            const unsigned lt = (1u << lane) - 1u;
            if (one) cid[n1 + __popc(b1 & lt)] = id;              // in place: n1 <= e0 + lane
            if (more) hpos[nm + __popc(bm & lt)] = (int)(id | (c << 16));
            n1 += __popc(b1);
            nm += __popc(bm);
            __syncwarp();
        }
        for (int e = lane; e < n1 + nm; e += 32) out[e] = (e < n1) ? cid[e] : (uint32_t)hpos[e - n1];
        if (lane == 0) {
            sizes[row] = make_int2(n1, nm);
            if (a.nnz_out) a.nnz_out[row] = nnz;
        }
        __syncwarp();
    }
}

// Shingles of one series by a warp-level counting sort, for 10 <= n <= 16:
// every shingle id sets its bit in a shared-memory occupancy bitmap of the 2^n
// ids (lane l owns the ids [l 2^n/32, (l+1) 2^n/32) and a summary word marking
// which of its bitmap words are non-zero); walking the lanes' ranges in order
// gives the distinct ids ascending, and an id whose bit was already set is a
// repeat that adds to its run count (found by binary search in the sorted ids).
// Only the touched words are cleared afterwards. Output layout as shingle_kernel.
constexpr int kMaxShingleIdsPerLane = 32;  // ceil(S / 32) for S <= 1024

struct BitmapLayout {
    int bm, sum, pid, cid, cnt, total;
};

__host__ __device__ inline BitmapLayout bitmap_layout(int n, int S) {
    BitmapLayout L;
    int off = 0;
    L.bm = off; off += a16(4 * (1 << (n - 5)));
    L.sum = off; off += a16(4 * (1 << (n - 10)));
    L.pid = off; off += a16(4 * S);
    L.cid = off; off += a16(4 * S);
    L.cnt = off; off += a16(4 * S);
    L.total = off;
    return L;
}

__global__ void __launch_bounds__(kCwsWarps * 32) shingle_bitmap_kernel(HashArgs a, const uint32_t* gbits,
                                                                         uint32_t* sets, int2* sizes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwords = a.nwords, S = a.S, n = a.n;
    const BitmapLayout lay = bitmap_layout(n, S);
    unsigned char* wb = smem + (size_t)warp * lay.total;
    uint32_t* bm = reinterpret_cast<uint32_t*>(wb + lay.bm);
    uint32_t* sum = reinterpret_cast<uint32_t*>(wb + lay.sum);
    uint32_t* pid = reinterpret_cast<uint32_t*>(wb + lay.pid);  // the id at each position
    uint32_t* cid = reinterpret_cast<uint32_t*>(wb + lay.cid);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(wb + lay.cnt);
    const int nbm = 1 << (n - 5);         // bitmap words
    const int wpl = nbm >> 5;             // bitmap words per lane (>= 1 for n >= 10)
    const int spl = (wpl + 31) >> 5;      // summary words per lane
    for (int w = lane; w < nbm; w += 32) bm[w] = 0u;
    for (int w = lane; w < 32 * spl; w += 32) sum[w] = 0u;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int rounds = (S + 31) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kCwsWarps;
    for (int64_t row = (int64_t)blockIdx.x * kCwsWarps + warp; row < a.count; row += nwarps) {
        const uint32_t* brow = gbits + row * nwords;
        uint32_t dup = 0;  // bit t set: position lane + 32 t repeats an earlier id
        for (int t = 0; t < rounds; ++t) {
            const int i = lane + 32 * t;
            if (i < S) {
                const int w0 = i >> 5;
                const uint32_t hi = __ldg(brow + w0);
                const uint32_t lo = (w0 + 1 < nwords) ? __ldg(brow + w0 + 1) : 0u;
                const uint64_t bb = ((uint64_t)hi << 32) | (uint64_t)lo;
                const uint32_t id = (uint32_t)((bb << (i & 31)) >> (64 - n));
                pid[i] = id;
                const uint32_t bit = 1u << (id & 31);
                const uint32_t old = atomicOr(&bm[id >> 5], bit);
                if (old & bit) dup |= 1u << t;
                else if (old == 0u) atomicOr(&sum[(id >> 5) >> 5], 1u << ((id >> 5) & 31));
            }
        }
        __syncwarp();
        // sorted distinct ids: count per lane range, warp scan, then emit
        int mine = 0;
        for (int q = 0; q < spl; ++q) {
            uint32_t sw = sum[lane * spl + q];
            while (sw) {
                const int b = __ffs(sw) - 1;
                sw &= sw - 1;
                mine += __popc(bm[(lane * spl + q) * 32 + b]);
            }
        }
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        int pos = incl - mine;
        const int nnz = __shfl_sync(kFull, incl, 31);
        for (int q = 0; q < spl; ++q) {
            const int sidx = lane * spl + q;
            uint32_t sw = sum[sidx];
            while (sw) {
                const int b = __ffs(sw) - 1;
                sw &= sw - 1;
                const int w = sidx * 32 + b;
                uint32_t word = bm[w];
                while (word) {
                    const int c = __ffs(word) - 1;
                    word &= word - 1;
                    cid[pos] = ((uint32_t)w << 5) | (uint32_t)c;
                    cnt[pos] = 1u;
                    ++pos;
                }
            }
        }
        __syncwarp();
        // repeats: add to the run of their id
        for (int t = 0; t < rounds; ++t) {
            if ((dup >> t) & 1u) {
                const uint32_t id = pid[lane + 32 * t];
                int lo = 0, hi = nnz - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cid[mid] < id) lo = mid + 1; else hi = mid;
                }
                atomicAdd(&cnt[lo], 1u);
            }
        }
        __syncwarp();
        // clear the touched words for the next series
        for (int i = lane; i < S; i += 32) bm[pid[i] >> 5] = 0u;
        for (int q = 0; q < spl; ++q) sum[lane * spl + q] = 0u;
        // the set in two ascending groups: seen once, then seen more than once (id | count << 16)
        uint32_t* out = sets + row * S;
        int n1 = 0, nm = 0;
        for (int e0 = 0; e0 < nnz; e0 += 32) {
            const int e = e0 + lane;
            uint32_t c = 0, id = 0;
            if (e < nnz) {
                c = cnt[e];
                id = cid[e];
                if (a.sh_ids_out) {
                    a.sh_ids_out[row * S + e] = id;
                    a.sh_counts_out[row * S + e] = c;
                }
            }
            const bool one = (e < nnz) && c == 1u, more = (e < nnz) && c > 1u;
            const unsigned b1 = __ballot_sync(kFull, one), bmm = __ballot_sync(kFull, more);
            __syncwarp();
            if (one) cid[n1 + __popc(b1 & lt)] = id;                    // in place: n1 <= e0 + lane
            if (more) cnt[nm + __popc(bmm & lt)] = id | (c << 16);      // in place: nm <= e0 + lane
            n1 += __popc(b1);
            nm += __popc(bmm);
            __syncwarp();
        }
        for (int e = lane; e < n1 + nm; e += 32) out[e] = (e < n1) ? cid[e] : cnt[e - n1];
        if (lane == 0) {
            sizes[row] = make_int2(n1, nm);
            if (a.nnz_out) a.nnz_out[row] = nnz;
        }
        __syncwarp();
    }
}

constexpr int kCwsDepth = 16;  // rank loads in flight per lane

struct CwsLayout {
    int set, kst, tst, total;
};

__host__ __device__ inline CwsLayout cws_layout(int S, int KL) {
    CwsLayout L;
    int off = 0;
    L.set = off; off += a16(4 * S);
    L.kst = off; off += a16(4 * KL);
    L.tst = off; off += a16(4 * KL);
    L.total = off;
    return L;
}

// FP64 recomputation of hash j over a set in the shingle_kernel layout.
__device__ inline void cws_fp64_set(const HashArgs& a, int j, const uint32_t* set, int n1, int nm, uint32_t* kout,
                                    uint32_t* tout) {
    const size_t nk = (size_t)1 << a.n;
    double best = __longlong_as_double(0x7FF0000000000000ll);
    uint32_t bk = 0xFFFFFFFFu, bt = 0;
#pragma unroll 1
    for (int e = 0; e < n1 + nm; ++e) {
        const uint32_t k = (e < n1) ? set[e] : set_id(set[e]);
        const uint32_t c = (e < n1) ? 1u : set_count(set[e]);
        const double* p = a.p64 + ((size_t)j * nk + k) * 3;
        const double r = p[0], beta = p[1], lnc = p[2];
        const double t = floor(__dadd_rn(__ddiv_rn(a.lns64[c], r), beta));
        const double la = __dsub_rn(lnc, __dmul_rn(r, __dadd_rn(__dsub_rn(t, beta), 1.0)));
        if (la < best || (la == best && k < bk)) {  // smallest ln a, ties to the smaller id
            best = la;
            bk = k;
            bt = (uint32_t)t;
        }
    }
    *kout = bk;
    *tout = bt;
}

__global__ void __launch_bounds__(kCwsWarps * 32, 4) cws_kernel(HashArgs a, const uint32_t* sets, const int2* sizes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = a.S, KL = a.KL;
    const CwsLayout lay = cws_layout(S, KL);
    unsigned char* wb = smem + (size_t)warp * lay.total;
    uint32_t* set = reinterpret_cast<uint32_t*>(wb + lay.set);
    uint32_t* kst = reinterpret_cast<uint32_t*>(wb + lay.kst);
    uint32_t* tst = reinterpret_cast<uint32_t*>(wb + lay.tst);
    const size_t nk = (size_t)1 << a.n;
    const int kstride = a.rank_stride;
    unsigned long long n64c = 0;
    const int64_t nwarps = (int64_t)gridDim.x * kCwsWarps;
    for (int64_t row = (int64_t)blockIdx.x * kCwsWarps + warp; row < a.count; row += nwarps) {
        const int2 sz = __ldg(sizes + row);
        const int n1 = sz.x, nm = sz.y;
        for (int e = lane; e < n1 + nm; e += 32) set[e] = __ldg(sets + row * S + e);
        __syncwarp();
        for (int jb = 0; jb < KL; jb += 128) {
            const int j0 = jb + 4 * lane;
            if (j0 < KL) {
                uint32_t m01 = 0xFFFFFFFFu, m23 = 0xFFFFFFFFu;
                const uint16_t* rk = a.rank + j0;
                int e = 0;
                for (; e + kCwsDepth <= n1; e += kCwsDepth) {
                    uint2 rv[kCwsDepth];
#pragma unroll
                    for (int u = 0; u < kCwsDepth; ++u)
                        rv[u] = __ldg(reinterpret_cast<const uint2*>(rk + set[e + u] * (uint32_t)kstride));
#pragma unroll
                    for (int u = 0; u < kCwsDepth; ++u) {
                        m01 = __vminu2(m01, rv[u].x);
                        m23 = __vminu2(m23, rv[u].y);
                    }
                }
#pragma unroll 1
                for (; e < n1; ++e) {
                    const uint2 r2 = __ldg(reinterpret_cast<const uint2*>(rk + set[e] * (uint32_t)kstride));
                    m01 = __vminu2(m01, r2.x);
                    m23 = __vminu2(m23, r2.y);
                }
                const uint32_t rmin[4] = {m01 & 0xFFFFu, m01 >> 16, m23 & 0xFFFFu, m23 >> 16};
                // exact group: the count-1 winner and every shingle seen 2..kTabCounts times
                ExactMin ex[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ex[q].init();
                    if (n1 > 0 && j0 + q < KL) {
                        const uint32_t kA = __ldg(a.kinv + (size_t)(j0 + q) * nk + rmin[q]);
                        ex[q].add(__ldg(a.lav + (size_t)kA * kTabCounts * kstride + j0 + q), kA, 0u);
                    }
                }
                int nlarge = 0;
#pragma unroll 1
                for (int t = 0; t < nm; ++t) {
                    const uint32_t v = set[n1 + t];
                    const uint32_t k = set_id(v), c = set_count(v);
                    if (c <= (uint32_t)kTabCounts) {
                        const float4 L = __ldg(reinterpret_cast<const float4*>(
                            a.lav + ((size_t)k * kTabCounts + (c - 1)) * kstride + j0));
                        const uchar4 T = __ldg(reinterpret_cast<const uchar4*>(
                            a.tsm + ((size_t)k * (kTabCounts - 1) + (c - 2)) * kstride + j0));
                        ex[0].add(L.x, k, T.x);
                        ex[1].add(L.y, k, T.y);
                        ex[2].add(L.z, k, T.z);
                        ex[3].add(L.w, k, T.w);
                    } else {
                        ++nlarge;
                    }
                }
                if (nlarge == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = j0 + q;
                        if (j < KL) {
                            uint32_t ks = ex[q].k, ts = ex[q].t;
                            if (ex[q].tie || ts == 255u || a.force_fp64) {
                                cws_fp64_set(a, j, set, n1, nm, &ks, &ts);
                                n64c += 1;
                            }
                            kst[j] = ks;
                            tst[j] = ts;
                        }
                    }
                } else {
                    // counts above the table: certified FP32 intervals
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = j0 + q;
                        if (j >= KL) continue;
                        CwsTrack tr;
                        tr.init();
#pragma unroll 1
                        for (int t = 0; t < nm; ++t) {
                            const uint32_t v = set[n1 + t];
                            const uint32_t k = set_id(v), c = set_count(v);
                            if (c > (uint32_t)kTabCounts)
                                tr.add(__ldg(a.p32 + (size_t)k * KL + j), __ldg(a.lns32 + c), k);
                        }
                        uint32_t ks, ts;
                        if (!exact_decide(ex[q], tr, &ks, &ts) || a.force_fp64) {
                            cws_fp64_set(a, j, set, n1, nm, &ks, &ts);
                            n64c += 1;
                        }
                        kst[j] = ks;
                        tst[j] = ts;
                    }
                }
            }
        }
        __syncwarp();
        if (a.kstar_out)
            for (int j = lane; j < KL; j += 32) {
                a.kstar_out[row * KL + j] = kst[j];
                a.tstar_out[row * KL + j] = tst[j];
            }
        if (a.keys)
            for (int l = lane; l < a.L; l += 32)
                a.keys[(int64_t)l * a.key_stride + a.key_col0 + row] = bucket_key(a.seed, l, a.K, kst, tst);
        __syncwarp();
    }
    if (n64c && a.stats) atomicAdd(&a.stats[kStatCws64], n64c);
}

int sms_of_device() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <int W, int DELTA, int R>
cudaError_t launch_sketch_t(const HashArgs& a, uint32_t* bits, unsigned long long* fix, unsigned long long cap,
                            unsigned long long* nfix, cudaStream_t st) {
    const int xb = sketch_xb(a.m, W, DELTA, R);
    const size_t smem = (size_t)a16(4 * W) + (size_t)kSketchWarps * (2 * a16(4 * xb) + a16(32 * R));
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(sketch_kernel<W, DELTA, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_kernel<W, DELTA, R>, kSketchWarps * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + kSketchWarps - 1) / kSketchWarps;
    if (grid > need) grid = need;
    FilterParam<W> rp;
    if (!a.r_host) return cudaErrorInvalidValue;
    for (int j = 0; j < W; ++j) rp.v[j] = a.r_host[j];
    sketch_kernel<W, DELTA, R><<<(unsigned)grid, kSketchWarps * 32, smem, st>>>(a, rp, bits, fix, cap, nfix);
    note_launch();
    return cudaGetLastError();
}

template <int E>
cudaError_t launch_shingle_t(const HashArgs& a, const uint32_t* bits, uint32_t* sets, int2* sizes, cudaStream_t st) {
    const ShingleLayout lay = shingle_layout(a.nwords, a.S);
    const size_t smem = (size_t)kCwsWarps * lay.total;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(shingle_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shingle_kernel<E>, kCwsWarps * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + kCwsWarps - 1) / kCwsWarps;
    if (grid > need) grid = need;
    shingle_kernel<E><<<(unsigned)grid, kCwsWarps * 32, smem, st>>>(a, bits, sets, sizes);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_shingle_bitmap(const HashArgs& a, const uint32_t* bits, uint32_t* sets, int2* sizes,
                                  cudaStream_t st) {
    const BitmapLayout lay = bitmap_layout(a.n, a.S);
    const size_t smem = (size_t)kCwsWarps * lay.total;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(shingle_bitmap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shingle_bitmap_kernel, kCwsWarps * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + kCwsWarps - 1) / kCwsWarps;
    if (grid > need) grid = need;
    shingle_bitmap_kernel<<<(unsigned)grid, kCwsWarps * 32, smem, st>>>(a, bits, sets, sizes);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_cws(const HashArgs& a, const uint32_t* sets, const int2* sizes, cudaStream_t st) {
    const CwsLayout lay = cws_layout(a.S, a.KL);
    const size_t smem = (size_t)kCwsWarps * lay.total;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(cws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cws_kernel, kCwsWarps * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + kCwsWarps - 1) / kCwsWarps;
    if (grid > need) grid = need;
    cws_kernel<<<(unsigned)grid, kCwsWarps * 32, smem, st>>>(a, sets, sizes);
    note_launch();
    return cudaGetLastError();
}

struct SketchShape {
    int W, delta, R;
};
const SketchShape kSketchShapes[] = {
    {80, 3, 5},  {32, 3, 2},  {120, 5, 6}, {16, 3, 2}, {32, 3, 3}, {64, 3, 5}, {128, 3, 10},
};

bool sketch_shape_ok(const SketchShape& s, const HashArgs& a) {
    return s.W == a.W && s.delta == a.delta && a.nb <= 32 * s.R && a.nb > 32 * (s.R - 1) && a.nb < 65536;
}

int cws_e(int S) {
    for (int E = 1; E <= 32; E <<= 1)
        if (S <= 32 * E) return E;
    return 0;
}

}  // namespace

bool hash_fast_supported(const HashArgs& a) {
    bool ok = false;
    for (const SketchShape& s : kSketchShapes) ok |= sketch_shape_ok(s, a);
    const int E = cws_e(a.S);
    return ok && E >= 1 && E <= 16 && a.n <= 16;
}

// Scratch of the split hash path: bits [count][nwords], the fix-up counter and
// list, the weighted sets [count][S] and their sizes [count].
struct FastScratch {
    size_t bits, nfix, fix, sets, sizes, total;
    unsigned long long fix_cap;
};

FastScratch fast_scratch(const HashArgs& a) {
    FastScratch f;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    f.fix_cap = (unsigned long long)a.count * 4ull + 65536ull;
    size_t off = 0;
    f.bits = off; off += up((size_t)a.count * a.nwords * sizeof(uint32_t));
    f.nfix = off; off += 256;
    f.fix = off; off += up((size_t)f.fix_cap * sizeof(unsigned long long));
    f.sets = off; off += up((size_t)a.count * a.S * sizeof(uint32_t));
    f.sizes = off; off += up((size_t)a.count * sizeof(int2));
    f.total = off;
    return f;
}

size_t hash_fast_scratch_bytes(const HashArgs& a) { return fast_scratch(a).total; }

FastHashBuffers hash_fast_buffers(const HashArgs& a, void* scratch) {
    const FastScratch f = fast_scratch(a);
    unsigned char* p = static_cast<unsigned char*>(scratch);
    FastHashBuffers b;
    b.bits = a.bits_out ? a.bits_out : reinterpret_cast<uint32_t*>(p + f.bits);
    b.nfix = reinterpret_cast<unsigned long long*>(p + f.nfix);
    b.fix = reinterpret_cast<unsigned long long*>(p + f.fix);
    b.fix_cap = f.fix_cap;
    b.sets = reinterpret_cast<uint32_t*>(p + f.sets);
    b.sizes = reinterpret_cast<int2*>(p + f.sizes);
    return b;
}

cudaError_t hash_fast_sketch(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.nfix, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    for (const SketchShape& s : kSketchShapes) {
        if (!sketch_shape_ok(s, a)) continue;
#define SSH_SKETCH_CASE(W_, D_, R_) \
    if (s.W == W_ && s.delta == D_ && s.R == R_) return launch_sketch_t<W_, D_, R_>(a, b.bits, b.fix, b.fix_cap, b.nfix, st);
        SSH_SKETCH_CASE(80, 3, 5)
        SSH_SKETCH_CASE(32, 3, 2)
        SSH_SKETCH_CASE(120, 5, 6)
        SSH_SKETCH_CASE(16, 3, 2)
        SSH_SKETCH_CASE(32, 3, 3)
        SSH_SKETCH_CASE(64, 3, 5)
        SSH_SKETCH_CASE(128, 3, 10)
#undef SSH_SKETCH_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t hash_fast_fixup(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st) {
    // the list length is only known on the device: size the grid for up to one
    // listed window per 8 series and let surplus blocks exit
    int64_t g = ((int64_t)(a.count / 8) + 255) / 256;
    if (g < 1) g = 1;
    if (g > 8192) g = 8192;
    sketch_fixup_kernel<<<(unsigned)g, 256, 0, st>>>(a, b.bits, b.fix, b.nfix, b.fix_cap);
    note_launch();
    return cudaGetLastError();
}

cudaError_t hash_fast_shingle(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st) {
    if (a.n >= 10 && a.S <= 32 * kMaxShingleIdsPerLane) return launch_shingle_bitmap(a, b.bits, b.sets, b.sizes, st);
    switch (cws_e(a.S)) {
        case 1: return launch_shingle_t<1>(a, b.bits, b.sets, b.sizes, st);
        case 2: return launch_shingle_t<2>(a, b.bits, b.sets, b.sizes, st);
        case 4: return launch_shingle_t<4>(a, b.bits, b.sets, b.sizes, st);
        case 8: return launch_shingle_t<8>(a, b.bits, b.sets, b.sizes, st);
        case 16: return launch_shingle_t<16>(a, b.bits, b.sets, b.sizes, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t hash_fast_cws(const HashArgs& a, const FastHashBuffers& b, cudaStream_t st) {
    return launch_cws(a, b.sets, b.sizes, st);
}

cudaError_t launch_hash_fast(const HashArgs& a, cudaStream_t st) {
    const size_t bytes = hash_fast_scratch_bytes(a);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, st);
    if (e != cudaSuccess) return e;
    const FastHashBuffers b = hash_fast_buffers(a, scratch);
    e = hash_fast_sketch(a, b, st);
    if (e == cudaSuccess) e = hash_fast_fixup(a, b, st);
    if (e == cudaSuccess) e = hash_fast_shingle(a, b, st);
    if (e == cudaSuccess) e = hash_fast_cws(a, b, st);
    cudaError_t f = cudaFreeAsync(scratch, st);
    return e != cudaSuccess ? e : f;
}

}  // namespace ssh
