// hash_kernels.cu -- Sec. 4.1 (sketch), Sec. 4.2 (shingles), Sec. 4.3 (weighted
// minhash by consistent weighted sampling) and the bucket keys of Algorithm 1,
// fused into one kernel: one warp hashes one series, and the series, its bits,
// its shingles and its hashes never leave shared memory.
//
// Exactness. Sign bits, shingles, (k*, t*) and keys must equal the FP64 CPU
// definition bit for bit, while the arithmetic here is FP32:
//  - a sketch bit is taken from the FP32 dot product only when |dot| exceeds
//    tau * ||r|| * ||x_window|| with tau = max(1e-4, 2 * gamma_W) (gamma_W is
//    the FP32 error bound of a W-term FMA chain); otherwise the window is
//    recomputed in FP64 in the definition's summation order;
//  - for shingles seen once, ln a_k = ln c_k - r_k (1 - beta_k) depends only on
//    (hash, shingle), so the draw tables hold its exact rank among all shingles
//    (computed from FP64 values at index creation) and the argmin over them is
//    an integer min;
//  - for repeated shingles and for the final comparison, ln a is evaluated in
//    FP32 together with a guaranteed error interval (relative width >= 1e-6,
//    directed rounding); if the winner's interval overlaps another candidate's,
//    or a floor() is within its error of an integer step, the whole hash is
//    recomputed in FP64 exactly as the definition orders the operations;
//  - for n > kMaxShingleBits there are no tables: each hash is the FP64 argmin
//    with its draws computed here (Philox, ln_fixed), the definition itself.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hash_common.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr int kMaxWarpsPerCta = 8;
constexpr unsigned kFull = 0xFFFFFFFFu;

__host__ __device__ inline int align16(int bytes) { return (bytes + 15) & ~15; }

__host__ __device__ inline int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct WarpSmem {
    int x, bits, sbuf, hpos, cid, ccnt, kst, tst, total;
};

__host__ __device__ inline WarpSmem warp_layout(int m, int nwords, int S, int KL) {
    WarpSmem L;
    int off = 0;
    L.x = off;    off += align16(4 * m);
    L.bits = off; off += align16(4 * (nwords + 2));
    L.sbuf = off; off += align16(4 * next_pow2(S));
    L.hpos = off; off += align16(4 * (S + 1));
    L.cid = off;  off += align16(4 * S);
    L.ccnt = off; off += align16(4 * S);
    L.kst = off;  off += align16(4 * KL);
    L.tst = off;  off += align16(4 * KL);
    L.total = off;
    return L;
}

__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) hash_kernel(HashArgs a, int warps_per_cta) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = a.W, m = a.m, delta = a.delta, n = a.n, nb = a.nb, nwords = a.nwords, S = a.S, KL = a.KL;

    float* r_s = reinterpret_cast<float*>(smem);
    for (int j = threadIdx.x; j < W; j += blockDim.x) r_s[j] = a.r[j];
    const WarpSmem lay = warp_layout(m, nwords, S, KL);
    unsigned char* wbase = smem + align16(4 * W) + (size_t)warp * lay.total;
    float* x_s = reinterpret_cast<float*>(wbase + lay.x);
    uint32_t* bits_s = reinterpret_cast<uint32_t*>(wbase + lay.bits);
    uint32_t* sbuf = reinterpret_cast<uint32_t*>(wbase + lay.sbuf);
    int* hpos = reinterpret_cast<int*>(wbase + lay.hpos);
    uint32_t* cid = reinterpret_cast<uint32_t*>(wbase + lay.cid);
    uint32_t* ccnt = reinterpret_cast<uint32_t*>(wbase + lay.ccnt);
    uint32_t* kst = reinterpret_cast<uint32_t*>(wbase + lay.kst);
    uint32_t* tst = reinterpret_cast<uint32_t*>(wbase + lay.tst);
    __syncthreads();

    int64_t row = (int64_t)blockIdx.x * warps_per_cta + warp;
    if (a.dev_range) {
        const int64_t r0 = a.dev_range[0], r1 = min(a.dev_range[1], r0 + a.count);
        row += r0;
        if (row >= r1) return;
    } else if (row >= a.count) {
        return;
    }
    const float* xg = a.rows ? a.rows[row] : a.series + row * a.stride;

    // ---- load the series (float4 when aligned)
    if (((reinterpret_cast<uintptr_t>(xg) & 15) == 0) && (m & 3) == 0) {
        const float4* x4 = reinterpret_cast<const float4*>(xg);
        float4* xs4 = reinterpret_cast<float4*>(x_s);
        for (int i = lane; i < (m >> 2); i += 32) xs4[i] = __ldg(x4 + i);
    } else {
        for (int i = lane; i < m; i += 32) x_s[i] = __ldg(xg + i);
    }
    __syncwarp();

    // ---- Sec. 4.1: sketch bits, one window per lane, packed by ballot
    unsigned long long n64 = 0;
    for (int w = 0; w < nwords; ++w) {
        const int i = w * 32 + lane;
        bool bit = false;
        if (i < nb) {
            const float* xw = x_s + i * delta;
            float acc = 0.f, ss = 0.f;
            for (int j = 0; j < W; ++j) {
                float xv = xw[j];
                acc = fmaf(r_s[j], xv, acc);
                ss = fmaf(xv, xv, ss);
            }
            float thr = __fmul_ru(a.tau_norm, __fsqrt_ru(__fmul_ru(ss, 1.0f + a.gamma_ss)));
            if (fabsf(acc) > thr) {
                bit = acc >= 0.f;
            } else {
                double d = 0.0;
                for (int j = 0; j < W; ++j) d = __dadd_rn(d, __dmul_rn((double)r_s[j], (double)xw[j]));
                bit = d >= 0.0;
                n64 += 1;
            }
        }
        unsigned bal = __ballot_sync(kFull, bit);
        if (lane == 0) bits_s[w] = __brev(bal);
    }
    if (lane == 0) {
        bits_s[nwords] = 0u;
        bits_s[nwords + 1] = 0u;
    }
    if (n64 && a.stats) atomicAdd(&a.stats[kStatSketch64], n64);
    __syncwarp();
    if (a.bits_out)
        for (int w = lane; w < nwords; w += 32) a.bits_out[row * nwords + w] = bits_s[w];

    // ---- Sec. 4.2: shingle ids (first bit most significant), warp bitonic sort, run-length encode
    const int S2 = next_pow2(S);
    for (int i = lane; i < S2; i += 32) {
        uint32_t id = 0xFFFFFFFFu;
        if (i < S) {
            uint64_t v = ((uint64_t)bits_s[i >> 5] << 32) | (uint64_t)bits_s[(i >> 5) + 1];
            id = (uint32_t)((v << (i & 31)) >> (64 - n));
        }
        sbuf[i] = id;
    }
    __syncwarp();
    for (int k = 2; k <= S2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < (S2 >> 1); t += 32) {
                int i = 2 * jj * (t / jj) + (t % jj);
                int l = i + jj;
                uint32_t u = sbuf[i], v = sbuf[l];
                bool up = (i & k) == 0;
                if ((u > v) == up) {
                    sbuf[i] = v;
                    sbuf[l] = u;
                }
            }
            __syncwarp();
        }
    }
    int nnz = 0;
    for (int base = 0; base < S; base += 32) {
        int i = base + lane;
        bool head = (i < S) && (i == 0 || sbuf[i] != sbuf[i - 1]);
        unsigned bal = __ballot_sync(kFull, head);
        if (head) {
            int pos = nnz + __popc(bal & ((1u << lane) - 1u));
            cid[pos] = sbuf[i];
            hpos[pos] = i;
        }
        nnz += __popc(bal);
    }
    __syncwarp();
    for (int e = lane; e < nnz; e += 32) {
        int end = (e + 1 < nnz) ? hpos[e + 1] : S;
        ccnt[e] = (uint32_t)(end - hpos[e]);
    }
    __syncwarp();
    if (a.nnz_out && lane == 0) a.nnz_out[row] = nnz;
    if (a.sh_ids_out)
        for (int e = lane; e < nnz; e += 32) {
            a.sh_ids_out[row * S + e] = cid[e];
            a.sh_counts_out[row * S + e] = ccnt[e];
        }

    // ---- Sec. 4.3: weighted minhash (Improved Consistent Sampling) per hash j
    unsigned long long c64 = 0;
    const size_t nk = (size_t)1 << n;
    for (int j0 = 0; j0 < KL; j0 += 32) {
        const int j = j0 + lane;
        if (j < KL && n > kMaxShingleBits) {
            // no draw tables for shingles this long: every draw in FP64 here, exactly as defined
            uint32_t ks, ts;
            cws_fp64_otf(a, j, cid, ccnt, nnz, &ks, &ts);
            kst[j] = ks;
            tst[j] = ts;
        } else if (j < KL) {
            uint32_t rmin = 0xFFFFFFFFu;
            bool hasA = false;
            CwsTrack tr;
            tr.init();
            for (int e = 0; e < nnz; ++e) {
                const uint32_t k = cid[e];
                const uint32_t s = ccnt[e];
                if (s == 1) {
                    rmin = min(rmin, (uint32_t)__ldg(a.rank + (size_t)k * a.rank_stride + j));
                    hasA = true;
                } else {
                    tr.add(__ldg(a.p32 + (size_t)k * KL + j), __ldg(a.lns32 + s), k);
                }
            }
            uint32_t kA = 0, ks, ts;
            float4 pA = make_float4(0.f, 0.f, 0.f, 0.f);
            if (hasA) {
                kA = __ldg(a.kla + (size_t)j * nk + rmin).x;
                pA = __ldg(a.p32 + (size_t)kA * KL + j);
            }
            if (!cws_decide(hasA, kA, pA, tr, &ks, &ts) || a.force_fp64) {
                cws_fp64(a, j, cid, ccnt, nnz, &ks, &ts);
                c64 += 1;
            }
            kst[j] = ks;
            tst[j] = ts;
        }
    }
    if (c64 && a.stats) atomicAdd(&a.stats[kStatCws64], c64);
    __syncwarp();
    if (a.kstar_out)
        for (int j = lane; j < KL; j += 32) {
            a.kstar_out[row * KL + j] = kst[j];
            a.tstar_out[row * KL + j] = tst[j];
        }

    // ---- Algorithm 1: one bucket key per table from its K hashes
    if (a.keys)
        for (int l = lane; l < a.L; l += 32)
            a.keys[(int64_t)l * a.key_stride + a.key_col0 + row] = bucket_key(a.seed, l, a.K, kst, tst);
}

}  // namespace

int hash_smem_bytes_per_warp(int m, int nwords, int S, int KL) { return warp_layout(m, nwords, S, KL).total; }

int hash_warps_per_cta(int m, int nwords, int S, int KL) {
    const int per = hash_smem_bytes_per_warp(m, nwords, S, KL);
    int w = kMaxWarpsPerCta;
    while (w > 1 && w * per > 160 * 1024) w >>= 1;
    return w;
}

cudaError_t launch_hash_generic(const HashArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    const int wpc = hash_warps_per_cta(a.m, a.nwords, a.S, a.KL);
    const size_t smem = (size_t)align16(4 * a.W) + (size_t)wpc * hash_smem_bytes_per_warp(a.m, a.nwords, a.S, a.KL);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = ensure_dynamic_smem((const void*)hash_kernel, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.count + wpc - 1) / wpc;
    hash_kernel<<<(unsigned)grid, wpc * 32, smem, st>>>(a, wpc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_hash(const HashArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (!a.force_generic && hash_fast_supported(a)) return launch_hash_fast(a, st);
    return launch_hash_generic(a, st);
}

}  // namespace ssh
