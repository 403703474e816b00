// hash_split.cu -- the hash path for the compiled-in shapes as two kernels and
// a fix-up (Sec. 4.1-4.3 and the keys of Algorithm 1):
//
//  sketch_kernel<W, DELTA, R, SPW>: one warp per SPW series at a time
//    (persistent, with the next series staged into shared memory by cp.async
//    while the current one is processed). Lane l of a series' 32 / SPW lanes
//    owns the R consecutive windows [lR, lR + R); the
//    filter r sits in registers and the loop over the lane's W + (R-1) DELTA
//    samples is unrolled, so each sample read from shared memory feeds up to R
//    FMAs and the strip's energy. A window whose |r.x| is not above
//    tau ||r|| ||x_strip|| (>= tau ||r|| ||x_window||) goes to a fix-up list
//    with a provisional bit 0. Bits are packed 32 per
//    word (window i -> bit 31 - i%32 of word i/32) into global memory.
//  sketch_fixup_kernel: one thread per listed window recomputes the dot product
//    in FP64 in the definition's order and sets the bit when it is >= 0.
//  shingle_kernel: one warp per series: the S = N_B - n + 1 shingle ids (first
//    bit most significant) go into a per-warp open-addressing table in shared
//    memory that counts repeats; the owners of the distinct ids write the
//    weighted set, ids seen once first.
//  cws_kernel: one warp per series; each lane owns 4 consecutive hash
//    functions: one 64-bit load brings the 4 exact count-1 ranks of a shingle
//    and SIMD u16 mins keep the minima, repeated shingles go through the
//    tabulated exact values or the certified FP32 interval track, and an
//    uncertain hash is recomputed in FP64 (hash_common.cuh). Its shared memory
//    is small, so many warps per SM hide the L2 latency of the rank lookups.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "hash_common.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSketchWarps = 8;

__host__ __device__ inline int a16(int b) { return (b + 15) & ~15; }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Rows [r0, r1) a launch hashes: 0 .. count-1, or the device range of a batch
// plan (rows are then absolute in the plan's sorted query table and scratch).
__device__ __forceinline__ void row_range(const HashArgs& a, int64_t* r0, int64_t* r1) {
    if (a.dev_range) {
        *r0 = a.dev_range[0];
        *r1 = min(a.dev_range[1], *r0 + a.count);
    } else {
        *r0 = 0;
        *r1 = a.count;
    }
}

__device__ __forceinline__ const float* row_ptr(const HashArgs& a, int64_t row) {
    return a.rows ? a.rows[row] : a.series + row * a.stride;
}

// Start copying series `row` into dst (m floats); misaligned rows load synchronously.
// (copied by the lanes l, l + lanes, ... of the series' lanes)
__device__ __forceinline__ void fetch_row(const HashArgs& a, int64_t row, float* dst, int lane, int lanes) {
    const float* src = row_ptr(a, row);
    const int m = a.m;
    if (((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (m & 3) == 0) {
        for (int c = lane; c < (m >> 2); c += lanes) cp_async16(dst + 4 * c, src + 4 * c);
    } else {
        for (int i = lane; i < m; i += lanes) dst[i] = __ldg(src + i);
    }
}

__host__ __device__ inline int sketch_xb(int m, int W, int DELTA, int R, int LPS) {
    int xb = m;
    const int need = LPS * R * DELTA + W;  // samples read by the padded windows of the last lanes
    if (need > xb) xb = need;
    return (xb + 3) & ~3;
}

// The filter as a by-value kernel parameter: it sits in the constant bank and
// every FMA reads its tap from there, leaving the registers to the windows.
// v2[j] packs the taps that sample t meets in two neighbouring windows k, k+1
// of a lane (j = t - k DELTA): r[j] (0 past the filter) in the low half and
// r[j - DELTA] (0 before it) in the high half, for one paired FMA.
template <int W, int DELTA>
struct FilterParam {
    float v[W];
    unsigned long long v2[W + DELTA];
};

#ifndef SSH_SKETCH_PAIRED
#define SSH_SKETCH_PAIRED 1
#endif

// (d.lo, d.hi) = (a.lo * b.lo + c.lo, a.hi * b.hi + c.hi), each half rounded once as fmaf.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Provisional bits go to `bits`; windows needing FP64 go to fix[0..cap) as
// (row << 16 | window), counted in *nfix. If the list is full the window is
// recomputed in place.
// SPW series per warp (1 or 2): the LPS = 32 / SPW lanes of a series own
// R consecutive windows each; with two series per warp a lane's R windows share
// one strip of W + (R-1) DELTA samples, so R can be twice as large for the same
// number of windows and each sample read from shared memory feeds twice as many
// FMAs.
template <int W, int DELTA, int R, int SPW>
__global__ void __launch_bounds__(kSketchWarps * 32, 3)
    sketch_kernel(HashArgs a, const FilterParam<W, DELTA> rp, uint32_t* bits, unsigned long long* fix,
                  unsigned long long fix_cap, unsigned long long* nfix) {
    constexpr int STRIP = W + (R - 1) * DELTA;
    constexpr int LPS = 32 / SPW;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = lane / LPS, ll = lane - sl * LPS;  // series slot of the warp, lane within the series
    const int m = a.m, nb = a.nb, nwords = a.nwords;
    const int xb = sketch_xb(m, W, DELTA, R, LPS);
    float* r_s = reinterpret_cast<float*>(smem);
    const size_t per_slot = 2 * (size_t)a16(4 * xb) + a16(LPS * R);
    unsigned char* wb = smem + a16(4 * W) + (size_t)(warp * SPW + sl) * per_slot;
    float* xbuf[2] = {reinterpret_cast<float*>(wb), reinterpret_cast<float*>(wb + a16(4 * xb))};
    unsigned char* bytes = wb + 2 * a16(4 * xb);
    for (int j = threadIdx.x; j < W; j += blockDim.x) r_s[j] = a.r[j];
    for (int i = m + ll; i < xb; i += LPS) {  // samples past the end feed only windows past N_B
        xbuf[0][i] = 0.f;
        xbuf[1][i] = 0.f;
    }
    __syncthreads();

    // the warp takes SPW consecutive rows at a time: group g holds rows g SPW .. g SPW + SPW - 1
    int64_t r0, r1;
    row_range(a, &r0, &r1);
    const int64_t ngroups = (r1 - r0 + SPW - 1) / SPW;
    const int64_t gstride = (int64_t)gridDim.x * kSketchWarps;
    const int64_t first = (int64_t)blockIdx.x * kSketchWarps + warp;
    unsigned long long n_inplace = 0;
    if (first < ngroups && r0 + first * SPW + sl < r1) fetch_row(a, r0 + first * SPW + sl, xbuf[0], ll, LPS);
    cp_async_commit();
    int it = 0;
    for (int64_t g = first; g < ngroups; g += gstride, ++it) {
        const int cur = it & 1;
        const int64_t row = r0 + g * SPW + sl;
        const int64_t nrow = r0 + (g + gstride) * SPW + sl;
        if (g + gstride < ngroups && nrow < r1) fetch_row(a, nrow, xbuf[cur ^ 1], ll, LPS);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        if (row < r1) {
            const float* x = xbuf[cur];
            // the R dot products and the energy of the lane's strip of STRIP samples,
            // which holds every window of the lane: ||x_window||^2 <= strip energy
            float acc[R];
            float e = 0.f;
            const float* xs = x + ll * R * DELTA;
            // windows 2p and 2p + 1 in one paired FMA per sample: each half gets the
            // same FMAs in the same order as alone (the zero taps only add +-0 to a
            // sum, which changes no nonzero value and no sign test). Up to 10 windows
            // per lane: more leave too few registers for the pairs.
            if constexpr (SSH_SKETCH_PAIRED && R <= 10) {
            constexpr int NP = R / 2;
            unsigned long long acc2[NP > 0 ? NP : 1];
#pragma unroll
            for (int q = 0; q < NP; ++q) acc2[q] = 0ull;
            float acc_odd = 0.f;
#pragma unroll
            for (int t = 0; t < STRIP; ++t) {
                const float xv = xs[t];
                e = fmaf(xv, xv, e);
                unsigned long long xx;
                asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(xv));
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const int j = t - 2 * q * DELTA;
                    if (j >= 0 && j < W + DELTA) acc2[q] = ffma2(rp.v2[j], xx, acc2[q]);
                }
                if constexpr ((R & 1) != 0) {
                    const int j = t - (R - 1) * DELTA;
                    if (j >= 0 && j < W) acc_odd = fmaf(rp.v[j], xv, acc_odd);
                }
            }
#pragma unroll
            for (int q = 0; q < NP; ++q)
                asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * q]), "=f"(acc[2 * q + 1]) : "l"(acc2[q]));
            if constexpr ((R & 1) != 0) acc[R - 1] = acc_odd;
            } else {
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = 0.f;
#pragma unroll
            for (int t = 0; t < STRIP; ++t) {
                const float xv = xs[t];
                e = fmaf(xv, xv, e);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int j = t - k * DELTA;
                    if (j >= 0 && j < W) acc[k] = fmaf(rp.v[j], xv, acc[k]);
                }
            }
            }
            // e carries at most STRIP roundings of relative 2^-24 each: inflate it past them
            const float e_up = __fmul_ru(e, 1.0f + (float)(2 * STRIP + 64) * 5.9604645e-08f);
            const float thr = __fmul_ru(a.tau_norm, __fsqrt_ru(__fmul_ru(e_up, 1.0f + a.gamma_ss)));
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int i = ll * R + k;
                uint8_t bit = 0;
                if (i < nb) {
                    if (fabsf(acc[k]) > thr) {
                        bit = acc[k] >= 0.f;
                    } else {
                        const unsigned long long slot = atomicAdd(nfix, 1ull);
                        if (slot < fix_cap) {
                            fix[slot] = ((unsigned long long)row << 16) | (unsigned long long)i;
                        } else {
                            const float* xw = xs + k * DELTA;
                            double d = 0.0;  // list full: the definition's FP64 order, in place
#pragma unroll 1
                            for (int j = 0; j < W; ++j) d = fma((double)r_s[j], (double)xw[j], d);
                            bit = d >= 0.0;
                            n_inplace += 1;
                        }
                    }
                }
                bytes[ll * R + k] = bit;
            }
        }
        __syncwarp();
        if (row < r1) {
            uint32_t* out = bits + row * nwords;
            for (int w = ll; w < nwords; w += LPS) {
                uint32_t word = 0;
                const uint32_t* b4 = reinterpret_cast<const uint32_t*>(bytes) + w * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t v = (w * 32 + q * 4 < LPS * R) ? b4[q] : 0u;
                    word |= (((v * 0x08040201u) >> 24) & 0xFu) << (28 - 4 * q);  // bytes 0..3 -> bits 3..0
                }
                out[w] = word;
            }
        }
        __syncwarp();
    }
    if (n_inplace && a.stats) atomicAdd(&a.stats[kStatSketch64], n_inplace);
}

// Sign of the FP64 dot product r . x (W terms, FP32 inputs, summed in order as
// the definition does) from FP32 arithmetic where an error bound settles it:
// Ogita, Rump & Oishi's Dot2 ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26(6), 2005: TwoProduct by FMA, TwoSum, the errors summed apart)
// returns res with |res - r.x| <= u |r.x| + g^2 sum |r_i x_i| (u = 2^-24,
// g = W u / (1 - W u)), and the FP64 chain errs by at most
// g64 sum |r_i x_i| (g64 = W 2^-53 / (1 - W 2^-53)). When |res| exceeds both
// with a margin, r.x and its FP64 value are nonzero and have the sign of res.
// Returns 1 (bit 1), 0 (bit 0) or -1 (not settled: recompute in FP64). Terms
// whose error-free product could underflow (a nonzero factor below 2^-50) are
// left to FP64 too.
struct Dot2 {
    float p = 0.f, s = 0.f, sabs = 0.f;
    bool tiny = false;
    __device__ __forceinline__ void add(float rj, float xj) {
        const float ar = fabsf(rj), ax = fabsf(xj);
        tiny |= (ar != 0.f && ar < 8.8817842e-16f) || (ax != 0.f && ax < 8.8817842e-16f);  // 2^-50
        const float h = __fmul_rn(rj, xj);
        const float e = __fmaf_rn(rj, xj, -h);  // rj xj = h + e exactly
        const float q = __fadd_rn(p, h);        // TwoSum(p, h) = q + f exactly
        const float z = __fsub_rn(q, p);
        const float f = __fadd_rn(__fsub_rn(p, __fsub_rn(q, z)), __fsub_rn(h, z));
        p = q;
        s = __fadd_rn(s, __fadd_rn(f, e));
        sabs = __fmaf_ru(ar, ax, sabs);  // an upper bound of sum |r_j x_j|
    }
};

__device__ __forceinline__ int dot2_sign(const float* r, const float* x, int W) {
    Dot2 d;
    int j = 0;
    for (; j + 8 <= W; j += 8) {  // groups of 8: the loads are issued together
        float rv[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            rv[u] = __ldg(r + j + u);
            xv[u] = __ldg(x + j + u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) d.add(rv[u], xv[u]);
    }
    for (; j < W; ++j) d.add(__ldg(r + j), __ldg(x + j));
    const float p = d.p, s = d.s, sabs = d.sabs;
    const bool tiny = d.tiny;
    const float res = __fadd_rn(p, s);
    // 2 (g^2 + g64) <= 2.002 (W u)^2 + 2.221e-16 W for W <= 8192 (W u <= 5e-4); FP32 rounding of
    // the factor is covered by the slack in its constants
    const float wu = (float)W * 5.9604645e-08f;
    const float fac = 2.01f * wu * wu + 2.3e-16f * (float)W;
    const float bound = __fadd_ru(__fmul_ru(fac, sabs), __fmul_ru(fabsf(res), 2.384185791015625e-07f));
    if (tiny || !(fabsf(res) > bound)) return -1;
    return res > 0.f ? 1 : 0;
}

// One thread per listed window: the sign by dot2_sign, else FP64 in the
// definition's order (the FP32 x FP32 products are exact in FP64, so an FMA
// equals the separate multiply and add).
__global__ void sketch_fixup_kernel(HashArgs a, uint32_t* bits, const unsigned long long* fix,
                                    const unsigned long long* nfix, unsigned long long cap) {
    const unsigned long long n = min(*nfix, cap);
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long v = fix[t];
        const int64_t row = (int64_t)(v >> 16);
        const int i = (int)(v & 0xFFFFu);
        const float* xw = row_ptr(a, row) + i * a.delta;
        const int sg = dot2_sign(a.r, xw, a.W);
        if (sg >= 0) {
            if (sg) atomicOr(&bits[row * a.nwords + (i >> 5)], 1u << (31 - (i & 31)));
            continue;
        }
        double d = 0.0;
        int j = 0;
        // groups of 8: the loads are issued together, the FMAs stay in the definition's order
        for (; j + 8 <= a.W; j += 8) {
            float xv[8], rv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                xv[u] = __ldg(xw + j + u);
                rv[u] = __ldg(a.r + j + u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) d = fma((double)rv[u], (double)xv[u], d);
        }
        for (; j < a.W; ++j) d = fma((double)__ldg(a.r + j), (double)__ldg(xw + j), d);
        if (d >= 0.0) atomicOr(&bits[row * a.nwords + (i >> 5)], 1u << (31 - (i & 31)));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats && n) atomicAdd(&a.stats[kStatSketch64], n);
}

// Per-series weighted set as written by shingle_kernel: S slots of u32, the n1
// shingles seen once first (id), then the nm repeated ones (id | count << 16);
// sizes[row] = (n1, nm). Within a group the order is that of first occurrence:
// every consumer takes an argmin with an explicit tie rule, so the order of a
// set does not matter.
__device__ __forceinline__ uint32_t set_id(uint32_t v) { return v & 0xFFFFu; }
__device__ __forceinline__ uint32_t set_count(uint32_t v) { return v >> 16; }

// Shared memory of one shingle warp: an open-addressing table of 2^tbits slots
// (2^tbits >= 2S, so at most half full), the slot of each position (bit 31: the
// position inserted the id first), and, when the caller asked for the sorted
// set, the set itself for ranking.
struct ShingleLayout {
    int tbits, tab, pos, stage, cid, total;
};

__host__ __device__ inline ShingleLayout shingle_layout(int S, bool sorted_out) {
    ShingleLayout L;
    L.tbits = 6;
    while ((1 << L.tbits) < 2 * S) ++L.tbits;
    int off = 0;
    L.tab = off; off += a16(4 << L.tbits);
    L.pos = off; off += a16(4 * S);
    L.stage = off; off += a16(4 * S);  // the repeated shingles before they follow the count-1 ones
    L.cid = off; off += sorted_out ? a16(4 * S) : 0;
    L.total = off;
    return L;
}

// Shingles of one series (Sec. 4.2) by hashing instead of sorting: position
// i = lane + 32 t reads sketch bits i .. i+n-1 (first bit most significant),
// which lie in words t and t+1, so every lane of a round reads the same two
// words. Each id is inserted into the warp's table (slot word = count << 16 |
// id; 0 is empty since counts start at 1): the lane whose compare-and-swap
// fills an empty slot owns the id, a lane that meets its id adds 1 to the
// count, any other id in the slot moves it on to the next slot. The owners
// then write the set, count-1 ids first, and clear their slots.
// WIN: the rows are the windows of one stream (window k starts at sample
// k * step) and shingle i of window k is the id precomputed at stream position
// k * step + i * delta (stream_ids_kernel); otherwise ids come from the row's bits.
template <bool WIN>
__global__ void __launch_bounds__(256) shingle_kernel(HashArgs a, const uint32_t* gbits, uint32_t* sets,
                                                      int2* sizes, const uint16_t* sh, int64_t step) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int nwords = a.nwords, S = a.S, n = a.n;
    const bool sorted_out = a.sh_ids_out != nullptr;
    const ShingleLayout lay = shingle_layout(S, sorted_out);
    unsigned char* wb = smem + (size_t)warp * lay.total;
    uint32_t* tab = reinterpret_cast<uint32_t*>(wb + lay.tab);
    uint32_t* pos = reinterpret_cast<uint32_t*>(wb + lay.pos);
    uint32_t* stage = reinterpret_cast<uint32_t*>(wb + lay.stage);
    uint32_t* cid = reinterpret_cast<uint32_t*>(wb + lay.cid);
    const uint32_t tmask = (1u << lay.tbits) - 1u;
    const int tshift = 32 - lay.tbits;
    constexpr uint32_t kOwner = 0x80000000u;
    for (uint32_t w = lane; w <= tmask; w += 32) tab[w] = 0u;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int rounds = (S + 31) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    int64_t r0, r1;
    row_range(a, &r0, &r1);
    for (int64_t row = r0 + (int64_t)blockIdx.x * wpb + warp; row < r1; row += nwarps) {
        const uint32_t* brow = WIN ? nullptr : gbits + row * nwords;
        uint32_t hi = WIN ? 0u : __ldg(brow);
        for (int t = 0; t < rounds; ++t) {
            const uint32_t lo = (!WIN && t + 1 < nwords) ? __ldg(brow + t + 1) : 0u;
            const int i = lane + 32 * t;
            if (i < S) {
                uint32_t id;
                if constexpr (WIN) {
                    id = __ldg(sh + row * step + (int64_t)i * a.delta);
                } else {
                    const uint64_t bb = ((uint64_t)hi << 32) | (uint64_t)lo;
                    id = (uint32_t)((bb << lane) >> (64 - n));
                }
                uint32_t h = (id * 0x9E3779B1u) >> tshift;
                uint32_t own = 0u;
                // at most S distinct ids in 2S slots: an empty slot or the id itself
                // is met within tmask + 1 probes
                for (uint32_t probe = 0; probe <= tmask; ++probe) {
                    const uint32_t old = atomicCAS(&tab[h], 0u, id | 0x10000u);
                    if (old == 0u) {
                        own = kOwner;
                        break;
                    }
                    if ((old & 0xFFFFu) == id) {
                        atomicAdd(&tab[h], 0x10000u);
                        break;
                    }
                    h = (h + 1u) & tmask;
                }
                pos[i] = h | own;
            }
            hi = lo;
        }
        __syncwarp();
        // one pass over the positions: owners write count-1 ids at once and stage the
        // repeated ones (they follow the count-1 ids), and clear their slots
        uint32_t* out = sets + row * S;
        int o1 = 0, om = 0;
        for (int t = 0; t < rounds; ++t) {
            const int i = lane + 32 * t;
            bool one = false, more = false;
            uint32_t v = 0u;
            if (i < S) {
                const uint32_t p = pos[i];
                if (p & kOwner) {
                    v = tab[p & ~kOwner];
                    tab[p & ~kOwner] = 0u;
                    one = set_count(v) == 1u;
                    more = !one;
                }
            }
            const unsigned b1 = __ballot_sync(kFull, one), bm = __ballot_sync(kFull, more);
            if (one) {
                const int e = o1 + __popc(b1 & lt);
                out[e] = set_id(v);
                if (sorted_out) cid[e] = v;
            }
            if (more) stage[om + __popc(bm & lt)] = v;
            o1 += __popc(b1);
            om += __popc(bm);
        }
        __syncwarp();
        const int n1 = o1, nm = om;
        for (int e = lane; e < nm; e += 32) {
            out[n1 + e] = stage[e];
            if (sorted_out) cid[n1 + e] = stage[e];
        }
        __syncwarp();
        const int nnz = n1 + nm;
        if (sorted_out) {
            // the sorted (id, count) list: the rank of an id among the distinct ids
            for (int e = lane; e < nnz; e += 32) {
                const uint32_t v = cid[e], id = set_id(v);
                int rank = 0;
#pragma unroll 1
                for (int f = 0; f < nnz; ++f) rank += set_id(cid[f]) < id;
                a.sh_ids_out[row * S + rank] = id;
                a.sh_counts_out[row * S + rank] = set_count(v);
            }
        }
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

__global__ void __launch_bounds__(256, 4) cws_kernel(HashArgs a, const uint32_t* sets, const int2* sizes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int S = a.S, KL = a.KL;
    const CwsLayout lay = cws_layout(S, KL);
    unsigned char* wb = smem + (size_t)warp * lay.total;
    uint32_t* set = reinterpret_cast<uint32_t*>(wb + lay.set);
    uint32_t* kst = reinterpret_cast<uint32_t*>(wb + lay.kst);
    uint32_t* tst = reinterpret_cast<uint32_t*>(wb + lay.tst);
    const size_t nk = (size_t)1 << a.n;
    const int kstride = a.rank_stride, tstride = a.tab_stride;
    unsigned long long n64c = 0;
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    int64_t r0, r1;
    row_range(a, &r0, &r1);
    for (int64_t row = r0 + (int64_t)blockIdx.x * wpb + warp; row < r1; row += nwarps) {
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
                for (; e < n1; e += 4) {
                    uint2 rv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        rv[u] = __ldg(reinterpret_cast<const uint2*>(rk + set[min(e + u, n1 - 1)] * (uint32_t)kstride));
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        m01 = __vminu2(m01, rv[u].x);
                        m23 = __vminu2(m23, rv[u].y);
                    }
                }
                const uint32_t rmin[4] = {m01 & 0xFFFFu, m01 >> 16, m23 & 0xFFFFu, m23 >> 16};
                // exact group: the count-1 winner and every shingle seen 2..kTabCounts times
                ExactMin ex[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ex[q].init();
                    if (n1 > 0 && j0 + q < KL) {
                        const uint2 w = __ldg(a.kla + (size_t)(j0 + q) * nk + rmin[q]);
                        ex[q].add(__uint_as_float(w.y), w.x, 0u);
                    }
                }
                int nlarge = 0;
#pragma unroll 1
                for (int t = 0; t < nm; ++t) {
                    const uint32_t v = set[n1 + t];
                    const uint32_t k = set_id(v), c = set_count(v);
                    if (c <= (uint32_t)kTabCounts) {
                        const float4 L = __ldg(reinterpret_cast<const float4*>(
                            a.lav + ((size_t)k * kTabCounts + (c - 1)) * tstride + j0));
                        const uchar4 T = __ldg(reinterpret_cast<const uchar4*>(
                            a.tsm + ((size_t)k * (kTabCounts - 1) + (c - 2)) * tstride + j0));
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

// Densified one-permutation weighted minhash of the copies (k, c), c = 1 .. S_k:
// one warp per series, the nhash = K L bins in shared memory (64-bit atomicMin of
// value << 32 | k << 16 | c), then each empty bin takes the bin of the first
// non-empty one of its pseudo-random sequence (after 64 K L tries, the next
// non-empty bin). Integer-only, so the hashes equal the definition exactly.
constexpr uint64_t kDophBin = 0xD0F1B1A5C0FFEE01ull;
constexpr uint64_t kDophFill = 0xDE45E1F1A11B0B02ull;
constexpr int kDophPerLane = 8;  // bins per lane: K L <= 256

__device__ __forceinline__ uint32_t doph_scale(uint64_t v, int nh) {
    return (uint32_t)(((v >> 32) * (uint64_t)nh) >> 32);
}

__global__ void __launch_bounds__(256) doph_kernel(HashArgs a, const uint32_t* sets, const int2* sizes) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int KL = a.KL, S = a.S;
    const size_t per_warp = (size_t)KL * 16;
    unsigned long long* bins = reinterpret_cast<unsigned long long*>(dsm + (size_t)warp * per_warp);
    uint32_t* kst = reinterpret_cast<uint32_t*>(bins + KL);
    uint32_t* tst = kst + KL;
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    int64_t r0, r1;
    row_range(a, &r0, &r1);
    for (int64_t row = r0 + (int64_t)blockIdx.x * wpb + warp; row < r1; row += nwarps) {
        for (int j = lane; j < KL; j += 32) bins[j] = ~0ull;
        __syncwarp();
        const int2 sz = __ldg(sizes + row);
        const int n1 = sz.x, nnz = sz.x + sz.y;
        for (int e = lane; e < nnz; e += 32) {
            const uint32_t v = __ldg(sets + row * S + e);
            const uint32_t k = (e < n1) ? v : set_id(v), cnt = (e < n1) ? 1u : set_count(v);
            for (uint32_t c = 1; c <= cnt; ++c) {
                const uint64_t h = mix64(a.seed ^ kDophBin ^ (((uint64_t)k << 32) | c));
                const uint64_t key = ((uint64_t)(uint32_t)mix64(h) << 32) | ((uint64_t)k << 16) | c;
                atomicMin(&bins[doph_scale(h, KL)], (unsigned long long)key);
            }
        }
        __syncwarp();
        // each bin's owner publishes its copy (k, c) (k = all ones: empty) ...
        for (int i = lane; i < KL; i += 32) {
            const unsigned long long key = bins[i];
            kst[i] = (key == ~0ull) ? 0xFFFFFFFFu : (uint32_t)((key >> 16) & 0xFFFFu);
            tst[i] = (key == ~0ull) ? 0u : (uint32_t)(key & 0xFFFFu);
        }
        __syncwarp();
        // ... then empty bins borrow from the published non-empty ones (into registers, so
        // no borrowed value is visible to another bin's probes), and store after a sync
        uint32_t rk[kDophPerLane], rt[kDophPerLane];
#pragma unroll
        for (int q = 0; q < kDophPerLane; ++q) {
            const int i = lane + 32 * q;
            rk[q] = 0xFFFFFFFFu;
            rt[q] = 0u;
            if (i >= KL) continue;
            uint32_t k = kst[i], c = tst[i];
            if (k == 0xFFFFFFFFu && nnz > 0) {
                const uint32_t tries = 64u * (uint32_t)KL;
                for (uint32_t t = 0; t < tries && k == 0xFFFFFFFFu; ++t) {
                    const uint32_t j =
                        doph_scale(mix64(a.seed ^ kDophFill ^ (((uint64_t)(uint32_t)i << 32) | (uint64_t)t)), KL);
                    k = kst[j];
                    c = tst[j];
                }
                for (int d = 1; d < KL && k == 0xFFFFFFFFu; ++d) {
                    k = kst[(i + d) % KL];
                    c = tst[(i + d) % KL];
                }
            }
            rk[q] = k;
            rt[q] = c;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kDophPerLane; ++q) {
            const int i = lane + 32 * q;
            if (i < KL) {
                kst[i] = rk[q];
                tst[i] = rt[q];
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
}

int sms_of_device() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <int W, int DELTA, int R, int SPW>
cudaError_t launch_sketch_t(const HashArgs& a, uint32_t* bits, unsigned long long* fix, unsigned long long cap,
                            unsigned long long* nfix, cudaStream_t st) {
    const int xb = sketch_xb(a.m, W, DELTA, R, 32 / SPW);
    const size_t smem = (size_t)a16(4 * W) + (size_t)kSketchWarps * SPW * (2 * a16(4 * xb) + a16((32 / SPW) * R));
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = ensure_dynamic_smem((const void*)sketch_kernel<W, DELTA, R, SPW>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_kernel<W, DELTA, R, SPW>, kSketchWarps * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = ((a.count + SPW - 1) / SPW + kSketchWarps - 1) / kSketchWarps;
    if (grid > need) grid = need;
    FilterParam<W, DELTA> rp;
    if (!a.r_host) return cudaErrorInvalidValue;
    for (int j = 0; j < W; ++j) rp.v[j] = a.r_host[j];
    for (int j = 0; j < W + DELTA; ++j) {
        const float lo = j < W ? a.r_host[j] : 0.f, hi = j >= DELTA ? a.r_host[j - DELTA] : 0.f;
        uint32_t ul, uh;
        memcpy(&ul, &lo, 4);
        memcpy(&uh, &hi, 4);
        rp.v2[j] = ((unsigned long long)uh << 32) | ul;
    }
    sketch_kernel<W, DELTA, R, SPW><<<(unsigned)grid, kSketchWarps * 32, smem, st>>>(a, rp, bits, fix, cap, nfix);
    note_launch();
    return cudaGetLastError();
}

// Warps per block for a kernel whose warps each take `per_warp` bytes of shared
// memory (8, fewer when they do not fit; 0 when one warp does not fit).
int warps_for(size_t per_warp) {
    int w = 8;
    while (w > 0 && (size_t)w * per_warp > 227 * 1024) --w;
    return w;
}

template <bool WIN>
cudaError_t launch_shingle_t(const HashArgs& a, const uint32_t* bits, uint32_t* sets, int2* sizes, const uint16_t* sh,
                             int64_t step, cudaStream_t st) {
    const ShingleLayout lay = shingle_layout(a.S, a.sh_ids_out != nullptr);
    const int wpb = warps_for((size_t)lay.total);
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)wpb * lay.total;
    cudaError_t e = ensure_dynamic_smem((const void*)shingle_kernel<WIN>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shingle_kernel<WIN>, wpb * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + wpb - 1) / wpb;
    if (grid > need) grid = need;
    shingle_kernel<WIN><<<(unsigned)grid, wpb * 32, smem, st>>>(a, bits, sets, sizes, sh, step);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_shingle(const HashArgs& a, const uint32_t* bits, uint32_t* sets, int2* sizes, cudaStream_t st) {
    return launch_shingle_t<false>(a, bits, sets, sizes, nullptr, 0, st);
}

cudaError_t launch_doph(const HashArgs& a, const uint32_t* sets, const int2* sizes, cudaStream_t st) {
    if (a.KL > 32 * kDophPerLane) return cudaErrorInvalidValue;
    const int wpb = warps_for((size_t)a.KL * 16);
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)wpb * a.KL * 16;
    cudaError_t e = ensure_dynamic_smem((const void*)doph_kernel, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, doph_kernel, wpb * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + wpb - 1) / wpb;
    if (grid > need) grid = need;
    doph_kernel<<<(unsigned)std::max<int64_t>(grid, 1), wpb * 32, smem, st>>>(a, sets, sizes);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_cws(const HashArgs& a, const uint32_t* sets, const int2* sizes, cudaStream_t st) {
    if (a.minhash == 1) return launch_doph(a, sets, sizes, st);
    const CwsLayout lay = cws_layout(a.S, a.KL);
    const int wpb = warps_for((size_t)lay.total);
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)wpb * lay.total;
    cudaError_t e = ensure_dynamic_smem((const void*)cws_kernel, smem);
    if (e != cudaSuccess) return e;
    // the rank rows are re-read from L1: ask for no more shared memory than 4 blocks use
    const int pct = (int)std::min<size_t>(100, (4 * smem * 100 + 228 * 1024 - 1) / (228 * 1024));
    e = cudaFuncSetAttribute(cws_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cws_kernel, wpb * 32, smem);
    int64_t grid = (int64_t)sms_of_device() * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (a.count + wpb - 1) / wpb;
    if (grid > need) grid = need;
    cws_kernel<<<(unsigned)grid, wpb * 32, smem, st>>>(a, sets, sizes);
    note_launch();
    return cudaGetLastError();
}

// Compiled (W, DELTA, R, series per warp) shapes; a shape serves the N_B in
// (LPS (R-1), LPS R] with LPS = 32 / SPW. The first match wins, so the
// two-series shapes come first.
struct SketchShape {
    int W, delta, R, spw;
};
const SketchShape kSketchShapes[] = {
    {80, 3, 10, 2},  {64, 3, 10, 2}, {32, 3, 3, 2},  {32, 3, 5, 2}, {16, 3, 3, 2}, {120, 5, 12, 2},
    {128, 3, 19, 2}, {80, 3, 5, 1},  {32, 3, 2, 1},  {120, 5, 6, 1}, {16, 3, 2, 1}, {32, 3, 3, 1},
    {64, 3, 5, 1},   {128, 3, 10, 1}, {256, 3, 19, 1},
};

// ---------------------------------------------- windows of one stream (Sec. 5.1)
//
// Window k of a stream starts at sample k * step; its sketch bit i is the sign
// of r . s[k step + i delta, + W), which depends only on the stream position
// j = k step + i delta. So the bits of every position are computed once
// (stream_sketch_kernel, with the same FP64 fix-up rule as sketch_kernel), then
// the n-bit shingle id of every position (stream_ids_kernel: bits j, j + delta,
// ..., j + (n-1) delta, first bit most significant), and a window's shingles
// are the ids at positions k step + i delta, i < S (shingle_kernel<true>).

// Bits of positions [0, J): word j / 32, bit 31 - j % 32. A thread per position;
// a block stages its 256 positions' samples (256 + W - 1) and r in shared memory.
__global__ void __launch_bounds__(256) stream_sketch_kernel(HashArgs a, const float* s, int64_t J, uint32_t* bits,
                                                            unsigned long long* fix, unsigned long long cap,
                                                            unsigned long long* nfix) {
    extern __shared__ float ssm[];
    const int W = a.W;
    float* r_s = ssm;
    float* xs = ssm + ((W + 3) & ~3);
    for (int i = threadIdx.x; i < W; i += blockDim.x) r_s[i] = a.r[i];
    unsigned long long n_inplace = 0;
    const int64_t send = J + W - 1;  // samples the positions read
    for (int64_t j0 = (int64_t)blockIdx.x * 256; j0 < J; j0 += (int64_t)gridDim.x * 256) {
        __syncthreads();
        for (int i = threadIdx.x; i < 256 + W - 1; i += blockDim.x) xs[i] = (j0 + i < send) ? __ldg(s + j0 + i) : 0.f;
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        bool bit = false;
        if (j < J) {
            float acc = 0.f, e = 0.f;
            for (int t = 0; t < W; ++t) {
                const float xv = xs[threadIdx.x + t];
                acc = fmaf(r_s[t], xv, acc);
                e = fmaf(xv, xv, e);
            }
            // e carries at most W roundings of relative 2^-24 each: inflate it past them
            const float e_up = __fmul_ru(e, 1.0f + (float)(2 * W + 64) * 5.9604645e-08f);
            const float thr = __fmul_ru(a.tau_norm, __fsqrt_ru(__fmul_ru(e_up, 1.0f + a.gamma_ss)));
            if (fabsf(acc) > thr) {
                bit = acc >= 0.f;
            } else {
                const unsigned long long slot = atomicAdd(nfix, 1ull);
                if (slot < cap) {
                    fix[slot] = (unsigned long long)j;
                } else {
                    double d = 0.0;  // list full: the definition's FP64 order, in place
                    for (int t = 0; t < W; ++t) d = fma((double)r_s[t], (double)xs[threadIdx.x + t], d);
                    bit = d >= 0.0;
                    n_inplace += 1;
                }
            }
        }
        const unsigned bal = __ballot_sync(kFull, bit);
        const int64_t jw = j0 + (threadIdx.x & ~31);
        if ((threadIdx.x & 31) == 0 && jw < J) bits[jw >> 5] = __brev(bal);
    }
    if (n_inplace && a.stats) atomicAdd(&a.stats[kStatSketch64], n_inplace);
}

// One thread per listed position: FP64 in the definition's order, as sketch_fixup_kernel.
__global__ void stream_fixup_kernel(HashArgs a, const float* s, uint32_t* bits, const unsigned long long* fix,
                                    const unsigned long long* nfix, unsigned long long cap) {
    const unsigned long long n = min(*nfix, cap);
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const int64_t j = (int64_t)fix[t];
        const float* xw = s + j;
        const int sg = dot2_sign(a.r, xw, a.W);
        if (sg >= 0) {
            if (sg) atomicOr(&bits[j >> 5], 1u << (31 - (j & 31)));
            continue;
        }
        double d = 0.0;
        for (int q = 0; q < a.W; ++q) d = fma((double)__ldg(a.r + q), (double)__ldg(xw + q), d);
        if (d >= 0.0) atomicOr(&bits[j >> 5], 1u << (31 - (j & 31)));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats && n) atomicAdd(&a.stats[kStatSketch64], n);
}

// The n-bit shingle id of every position j in [0, Jsh): bits j + b delta, b < n, first bit most significant.
__global__ void stream_ids_kernel(const uint32_t* bits, int64_t Jsh, int n, int delta, uint16_t* sh) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Jsh; j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t id = 0;
        for (int b = 0; b < n; ++b) {
            const int64_t q = j + (int64_t)b * delta;
            id = (id << 1) | ((__ldg(bits + (q >> 5)) >> (31 - (q & 31))) & 1u);
        }
        sh[j] = (uint16_t)id;
    }
}

bool sketch_shape_ok(const SketchShape& s, const HashArgs& a) {
    const int lps = 32 / s.spw;
    return s.W == a.W && s.delta == a.delta && a.nb <= lps * s.R && a.nb > lps * (s.R - 1) && a.nb < 65536;
}

}  // namespace

bool hash_fast_supported(const HashArgs& a) {
    bool ok = false;
    for (const SketchShape& s : kSketchShapes) ok |= sketch_shape_ok(s, a);
    return ok && a.n <= 16 && a.S >= 1 && warps_for((size_t)shingle_layout(a.S, true).total) >= 1 &&
           warps_for((size_t)cws_layout(a.S, a.KL).total) >= 1;
}

bool hash_windows_supported(const HashArgs& a) {
    return a.n <= 16 && a.S >= 1 && warps_for((size_t)shingle_layout(a.S, a.sh_ids_out != nullptr).total) >= 1 &&
           warps_for((size_t)cws_layout(a.S, a.KL).total) >= 1;
}

// Scratch of the window path: position bits, the fix-up counter and list, the
// position ids, the windows' weighted sets [count][S] and sizes [count].
struct WinScratch {
    size_t bits, nfix, fix, sh, sets, sizes, total;
    int64_t J, Jsh;
    unsigned long long fix_cap;
};

WinScratch win_scratch(const HashArgs& a, int64_t step) {
    WinScratch f;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    f.J = (a.count - 1) * step + (int64_t)(a.nb - 1) * a.delta + 1;
    f.Jsh = (a.count - 1) * step + (int64_t)(a.S - 1) * a.delta + 1;
    f.fix_cap = (unsigned long long)f.J / 8ull + 65536ull;
    size_t off = 0;
    f.bits = off; off += up((size_t)((f.J + 31) / 32) * sizeof(uint32_t));
    f.nfix = off; off += 256;
    f.fix = off; off += up((size_t)f.fix_cap * sizeof(unsigned long long));
    f.sh = off; off += up((size_t)f.Jsh * sizeof(uint16_t));
    f.sets = off; off += up((size_t)a.count * a.S * sizeof(uint32_t));
    f.sizes = off; off += up((size_t)a.count * sizeof(int2));
    f.total = off;
    return f;
}

size_t hash_windows_scratch_bytes(const HashArgs& a, int64_t step) { return win_scratch(a, step).total; }

cudaError_t hash_windows_stage(const HashArgs& a, const float* s, int64_t step, void* scratch, int stage,
                               cudaStream_t st) {
    const WinScratch f = win_scratch(a, step);
    unsigned char* p = static_cast<unsigned char*>(scratch);
    uint32_t* bits = reinterpret_cast<uint32_t*>(p + f.bits);
    unsigned long long* nfix = reinterpret_cast<unsigned long long*>(p + f.nfix);
    unsigned long long* fix = reinterpret_cast<unsigned long long*>(p + f.fix);
    uint16_t* sh = reinterpret_cast<uint16_t*>(p + f.sh);
    uint32_t* sets = reinterpret_cast<uint32_t*>(p + f.sets);
    int2* sizes = reinterpret_cast<int2*>(p + f.sizes);
    cudaError_t e = cudaSuccess;
    if (stage == 0) {  // sketch of every position
        e = cudaMemsetAsync(nfix, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        const size_t smem = (size_t)(((a.W + 3) & ~3) + 256 + a.W) * sizeof(float);
        e = ensure_dynamic_smem((const void*)stream_sketch_kernel, smem);
        if (e != cudaSuccess) return e;
        const int64_t g = std::min<int64_t>((f.J + 255) / 256, (int64_t)sms_of_device() * 8);
        stream_sketch_kernel<<<(unsigned)std::max<int64_t>(g, 1), 256, smem, st>>>(a, s, f.J, bits, fix, f.fix_cap,
                                                                                   nfix);
        note_launch();
        return cudaGetLastError();
    }
    if (stage == 1) {  // FP64 fix-up of the listed positions
        const int64_t g = std::max<int64_t>(1, std::min<int64_t>((f.J / 64 + 255) / 256, 8192));
        stream_fixup_kernel<<<(unsigned)g, 256, 0, st>>>(a, s, bits, fix, nfix, f.fix_cap);
        note_launch();
        return cudaGetLastError();
    }
    if (stage == 2) {  // position ids, then the windows' weighted sets
        const int64_t g = std::max<int64_t>(1, std::min<int64_t>((f.Jsh + 255) / 256, 8192));
        stream_ids_kernel<<<(unsigned)g, 256, 0, st>>>(bits, f.Jsh, a.n, a.delta, sh);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_shingle_t<true>(a, nullptr, sets, sizes, sh, step, st);
    }
    return launch_cws(a, sets, sizes, st);  // stage 3: weighted minhash and bucket keys
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
#define SSH_SKETCH_CASE(W_, D_, R_, P_)                                           \
    if (s.W == W_ && s.delta == D_ && s.R == R_ && s.spw == P_)                     \
        return launch_sketch_t<W_, D_, R_, P_>(a, b.bits, b.fix, b.fix_cap, b.nfix, st);
        SSH_SKETCH_CASE(80, 3, 10, 2)
        SSH_SKETCH_CASE(64, 3, 10, 2)
        SSH_SKETCH_CASE(32, 3, 3, 2)
        SSH_SKETCH_CASE(32, 3, 5, 2)
        SSH_SKETCH_CASE(16, 3, 3, 2)
        SSH_SKETCH_CASE(120, 5, 12, 2)
        SSH_SKETCH_CASE(128, 3, 19, 2)
        SSH_SKETCH_CASE(80, 3, 5, 1)
        SSH_SKETCH_CASE(32, 3, 2, 1)
        SSH_SKETCH_CASE(120, 5, 6, 1)
        SSH_SKETCH_CASE(16, 3, 2, 1)
        SSH_SKETCH_CASE(32, 3, 3, 1)
        SSH_SKETCH_CASE(64, 3, 5, 1)
        SSH_SKETCH_CASE(128, 3, 10, 1)
        SSH_SKETCH_CASE(256, 3, 19, 1)
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
    return launch_shingle(a, b.bits, b.sets, b.sizes, st);
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
