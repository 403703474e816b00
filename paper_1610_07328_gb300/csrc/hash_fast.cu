// hash_fast.cu -- the hash kernel specialised at compile time for a filter
// length W, step DELTA, windows per lane R and sort width 32*E (Sec. 4.1-4.3 and
// the keys of Algorithm 1). One warp hashes one series at a time, looping over
// series (persistent), with the next series copied into shared memory by
// cp.async while the current one is processed.
//
//  Sketch: lane l owns the R consecutive windows [l R, l R + R). The filter r
//  sits in registers and the loop over the lane's W + (R-1) DELTA samples is
//  unrolled, so every sample read from shared memory feeds up to R FMAs. The
//  window energies ||x_win||^2 come from a running sum of squares over the same
//  samples. Bits go to shared memory as bytes and are packed 32 per word.
//  Shingles: the S = N_B - n + 1 ids are sorted by a bitonic network over 32*E
//  registers (E per lane, blocked layout) with warp shuffles, then run-length
//  encoded with a ballot scan.
//  Weighted minhash: lane l owns the 4 hashes 4l .. 4l+3 (per 128 hashes): one
//  64-bit load brings the 4 count-1 ranks of a shingle, two SIMD u16 mins keep
//  the running minima; repeated shingles go through the certified FP32 track.
//  Exactness rules are those of hash_kernels.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hash_common.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kFastWarps = 8;

__host__ __device__ inline int a16(int b) { return (b + 15) & ~15; }

struct FastLayout {
    int xb;  // floats per x buffer
    int x0, x1, bytes, bits, hpos, cid, ccnt, kst, tst, total;
};

__host__ __device__ inline FastLayout fast_layout(int m, int W, int DELTA, int R, int nwords, int S, int KL) {
    FastLayout L;
    int xb = m;
    const int need = 32 * R * DELTA + W;  // samples read by the padded windows of the last lanes
    if (need > xb) xb = need;
    xb = (xb + 3) & ~3;
    L.xb = xb;
    int off = 0;
    L.x0 = off; off += a16(4 * xb);
    L.x1 = off; off += a16(4 * xb);
    L.bytes = off; off += a16(32 * R);
    L.bits = off; off += a16(4 * (nwords + 2));
    L.hpos = off; off += a16(4 * (S + 1));
    L.cid = off; off += a16(4 * S);
    L.ccnt = off; off += a16(4 * S);
    L.kst = off; off += a16(4 * KL);
    L.tst = off; off += a16(4 * KL);
    L.total = off;
    return L;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Start copying series `row` into dst (m floats); misaligned rows load synchronously.
__device__ __forceinline__ void fetch_row(const HashArgs& a, int64_t row, float* dst, int lane) {
    const float* src = a.rows ? a.rows[row] : a.series + row * a.stride;
    const int m = a.m;
    if (((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (m & 3) == 0) {
        for (int c = lane; c < (m >> 2); c += 32) cp_async16(dst + 4 * c, src + 4 * c);
    } else {
        for (int i = lane; i < m; i += 32) dst[i] = __ldg(src + i);
    }
}

template <int W, int DELTA, int R, int E>
__global__ void __launch_bounds__(kFastWarps * 32, 2) hash_fast_kernel(HashArgs a) {
    constexpr int STRIP = W + (R - 1) * DELTA;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int m = a.m, nb = a.nb, nwords = a.nwords, S = a.S, KL = a.KL, n = a.n;
    const FastLayout lay = fast_layout(m, W, DELTA, R, nwords, S, KL);

    float* r_s = reinterpret_cast<float*>(smem);
    double* r64 = reinterpret_cast<double*>(smem + a16(4 * W));
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        r_s[j] = a.r[j];
        r64[j] = (double)a.r[j];
    }
    unsigned char* wb = smem + a16(4 * W) + a16(8 * W) + (size_t)warp * lay.total;
    float* xbuf[2] = {reinterpret_cast<float*>(wb + lay.x0), reinterpret_cast<float*>(wb + lay.x1)};
    unsigned char* bytes = wb + lay.bytes;
    uint32_t* bits = reinterpret_cast<uint32_t*>(wb + lay.bits);
    int* hpos = reinterpret_cast<int*>(wb + lay.hpos);
    uint32_t* cid = reinterpret_cast<uint32_t*>(wb + lay.cid);
    uint32_t* ccnt = reinterpret_cast<uint32_t*>(wb + lay.ccnt);
    uint32_t* kst = reinterpret_cast<uint32_t*>(wb + lay.kst);
    uint32_t* tst = reinterpret_cast<uint32_t*>(wb + lay.tst);
    // samples past the series end are read only by windows past N_B: keep them finite (zero)
    for (int i = m + lane; i < lay.xb; i += 32) {
        xbuf[0][i] = 0.f;
        xbuf[1][i] = 0.f;
    }
    __syncthreads();

    const int64_t nwarps = (int64_t)gridDim.x * kFastWarps;
    const int64_t first = (int64_t)blockIdx.x * kFastWarps + warp;
    unsigned long long n64s = 0, n64c = 0;
    const size_t nk = (size_t)1 << n;
    const int kstride = a.rank_stride;

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

        // ---------------------------------------------------- Sec. 4.1 sketch
        {
            float rr[W];
#pragma unroll
            for (int j = 0; j < W; ++j) rr[j] = r_s[j];
            float acc[R];
            float ssq[R + 1];  // running sum of squares captured at window boundaries
            float run = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = 0.f;
            float s_lo[R], s_hi[R];
            const float* xs = x + lane * R * DELTA;
#pragma unroll
            for (int t = 0; t < STRIP; ++t) {
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (t == k * DELTA) s_lo[k] = run;
                const float xv = xs[t];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int j = t - k * DELTA;
                    if (j >= 0 && j < W) acc[k] = fmaf(rr[j], xv, acc[k]);
                }
                run = fmaf(xv, xv, run);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (t == k * DELTA + W - 1) s_hi[k] = run;
            }
            (void)ssq;
            // |sum-of-squares error| <= 2 STRIP u run(end): a margin that keeps the bound an upper bound
            const float margin = __fmul_ru(run, (float)(2.02 * STRIP) * 5.9604645e-08f);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int i = lane * R + k;
                uint8_t bit = 0;
                if (i < nb) {
                    const float ss = __fadd_ru(__fsub_ru(s_hi[k], s_lo[k]), margin);
                    const float thr = __fmul_ru(a.tau_norm, __fsqrt_ru(__fmul_ru(fmaxf(ss, 0.f), 1.0f + a.gamma_ss)));
                    if (fabsf(acc[k]) > thr) {
                        bit = acc[k] >= 0.f;
                    } else {
                        // FP64 in the definition's order (the FP32 x FP32 products are exact in FP64)
                        double d = 0.0;
                        const float* xw = xs + k * DELTA;
                        for (int j = 0; j < W; ++j) d = fma(r64[j], (double)xw[j], d);
                        bit = d >= 0.0;
                        n64s += 1;
                    }
                }
                bytes[lane * R + k] = bit;
            }
        }
        __syncwarp();
        for (int w = lane; w < nwords + 2; w += 32) {
            uint32_t word = 0;
            if (w < nwords) {
                const uint32_t* b4 = reinterpret_cast<const uint32_t*>(bytes) + w * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i0 = w * 32 + q * 4;
                    uint32_t v = (i0 < 32 * R) ? b4[q] : 0u;
                    const uint32_t nib = ((v * 0x08040201u) >> 24) & 0xFu;  // bytes 0..3 -> bits 3..0
                    word |= nib << (28 - 4 * q);
                }
            }
            bits[w] = word;
        }
        __syncwarp();
        if (a.bits_out)
            for (int w = lane; w < nwords; w += 32) a.bits_out[row * nwords + w] = bits[w];

        // ---------------------------------------------------- Sec. 4.2 shingles
        int nnz = 0;
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
            // bitonic sort, ascending, of 32*E keys; element index i = lane*E + e
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
            // run-length encoding: heads of runs, their positions by a warp scan
            uint32_t prev = __shfl_up_sync(kFull, v[E - 1], 1);
            int nh = 0;
            bool head[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane * E + e;
                const uint32_t pv = (e == 0) ? prev : v[e - 1];
                head[e] = (i < S) && (i == 0 || v[e] != pv);
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
        int n1 = 0;  // shingles seen once
        for (int e0 = 0; e0 < nnz; e0 += 32) {
            const int e = e0 + lane;
            uint32_t c = 0;
            if (e < nnz) {
                const int end = (e + 1 < nnz) ? hpos[e + 1] : S;
                c = (uint32_t)(end - hpos[e]);
                ccnt[e] = c;
            }
            n1 += __popc(__ballot_sync(kFull, c == 1u));
        }
        __syncwarp();
        if (a.nnz_out && lane == 0) a.nnz_out[row] = nnz;
        if (a.sh_ids_out)
            for (int e = lane; e < nnz; e += 32) {
                a.sh_ids_out[row * S + e] = cid[e];
                a.sh_counts_out[row * S + e] = ccnt[e];
            }

        // ---------------------------------------------------- Sec. 4.3 weighted minhash
        for (int jb = 0; jb < KL; jb += 128) {
            const int j0 = jb + 4 * lane;
            if (j0 < KL) {
                uint32_t m01 = 0xFFFFFFFFu, m23 = 0xFFFFFFFFu;
                CwsTrack tr[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) tr[q].init();
                const uint16_t* rk = a.rank + j0;
                int e = 0;
                for (; e + 4 <= nnz; e += 4) {
                    uint2 rv[4];
                    uint32_t kk[4], cc[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        kk[u] = cid[e + u];
                        cc[u] = ccnt[e + u];
                        rv[u] = (cc[u] == 1u) ? __ldg(reinterpret_cast<const uint2*>(rk + (size_t)kk[u] * kstride))
                                              : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        m01 = __vminu2(m01, rv[u].x);
                        m23 = __vminu2(m23, rv[u].y);
                        if (cc[u] != 1u) {
                            const float ls = __ldg(a.lns32 + cc[u]);
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (j0 + q < KL) tr[q].add(__ldg(a.p32 + (size_t)kk[u] * KL + j0 + q), ls, kk[u]);
                        }
                    }
                }
                for (; e < nnz; ++e) {
                    const uint32_t k = cid[e], c = ccnt[e];
                    if (c == 1u) {
                        const uint2 r2 = __ldg(reinterpret_cast<const uint2*>(rk + (size_t)k * kstride));
                        m01 = __vminu2(m01, r2.x);
                        m23 = __vminu2(m23, r2.y);
                    } else {
                        const float ls = __ldg(a.lns32 + c);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (j0 + q < KL) tr[q].add(__ldg(a.p32 + (size_t)k * KL + j0 + q), ls, k);
                    }
                }
                const uint32_t rmin[4] = {m01 & 0xFFFFu, m01 >> 16, m23 & 0xFFFFu, m23 >> 16};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = j0 + q;
                    if (j < KL) {
                        uint32_t kA = 0;
                        float4 pA = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (n1 > 0) {
                            kA = __ldg(a.kinv + (size_t)j * nk + rmin[q]);
                            pA = __ldg(a.p32 + (size_t)kA * KL + j);
                        }
                        uint32_t ks, ts;
                        if (!cws_decide(n1 > 0, kA, pA, tr[q], &ks, &ts)) {
                            cws_fp64(a, j, cid, ccnt, nnz, &ks, &ts);
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
    if (a.stats) {
        if (n64s) atomicAdd(&a.stats[kStatSketch64], n64s);
        if (n64c) atomicAdd(&a.stats[kStatCws64], n64c);
    }
}

template <int W, int DELTA, int R, int E>
cudaError_t launch_fast_t(const HashArgs& a, cudaStream_t st) {
    const FastLayout lay = fast_layout(a.m, W, DELTA, R, a.nwords, a.S, a.KL);
    const size_t smem = (size_t)a16(4 * W) + a16(8 * W) + (size_t)kFastWarps * lay.total;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(hash_fast_kernel<W, DELTA, R, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hash_fast_kernel<W, DELTA, R, E>, kFastWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = (a.count + kFastWarps - 1) / kFastWarps;
    if (grid > need) grid = need;
    hash_fast_kernel<W, DELTA, R, E><<<(unsigned)grid, kFastWarps * 32, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

// The shapes compiled ahead of time: (W, delta) of the benchmark workloads, R
// windows per lane covering N_B <= 32 R, and a sort of 32 E >= S keys.
struct FastShape {
    int W, delta, R, E;
};
static const FastShape kShapes[] = {
    {80, 3, 5, 8},    // m = 512, W = 80, delta = 3 (N_B 145, S 131 at n = 15)
    {32, 3, 2, 1},    // m = 128, W = 32, delta = 3 (N_B 33, S 26 at n = 8)
    {120, 5, 6, 8},   // m = 1024, W = 120, delta = 5 (N_B 181, S 167 at n = 15)
    {16, 3, 2, 1},    // m = 128, W = 16 (N_B 38, S 24)
    {32, 3, 3, 2},    // m = 256, W = 32 (N_B 75, S 61)
    {64, 3, 5, 8},    // m = 512, W = 64 (N_B 150, S 136)
    {128, 3, 10, 16}, // m = 1024, W = 128 (N_B 299, S 285)
};

bool hash_fast_supported(const HashArgs& a) {
    for (const FastShape& s : kShapes)
        if (s.W == a.W && s.delta == a.delta && a.nb <= 32 * s.R && a.nb > 32 * (s.R - 1) && a.S <= 32 * s.E &&
            a.S > 16 * s.E)
            return true;
    return false;
}

cudaError_t launch_hash_fast(const HashArgs& a, cudaStream_t st) {
    for (const FastShape& s : kShapes) {
        if (!(s.W == a.W && s.delta == a.delta && a.nb <= 32 * s.R && a.nb > 32 * (s.R - 1) && a.S <= 32 * s.E &&
              a.S > 16 * s.E))
            continue;
#define SSH_FAST_CASE(W_, D_, R_, E_) \
    if (s.W == W_ && s.delta == D_ && s.R == R_ && s.E == E_) return launch_fast_t<W_, D_, R_, E_>(a, st);
        SSH_FAST_CASE(80, 3, 5, 8)
        SSH_FAST_CASE(32, 3, 2, 1)
        SSH_FAST_CASE(120, 5, 6, 8)
        SSH_FAST_CASE(16, 3, 2, 1)
        SSH_FAST_CASE(32, 3, 3, 2)
        SSH_FAST_CASE(64, 3, 5, 8)
        SSH_FAST_CASE(128, 3, 10, 16)
#undef SSH_FAST_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace ssh
