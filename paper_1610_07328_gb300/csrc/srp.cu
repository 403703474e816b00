// srp.cu -- the paper's SRP baseline (Sec. 5.2, Table 2): each hash is the sign
// of a random projection of the whole series, K of them per table, folded into
// the bucket key like the (k*, t*) pairs of the weighted minhash (hash value
// (bit, 0)). Three kernels:
//
//  srp_bits_kernel: a tiled FP32 product of 64 series x 128 projections per
//    block pass (series and projection tiles of 32 samples in shared memory,
//    8 x 4 accumulators per thread, each summing in sample order). A bit whose
//    |r_j . x| is not above tau_m ||r_j|| ||x|| is listed for the FP64 fix-up;
//    the FP32 sum of m products errs by at most gamma_m ||r_j|| ||x|| and
//    tau_m = max(1e-4, 2 gamma_m).
//  srp_fixup_kernel: one thread per listed bit, the dot product in FP64 in the
//    definition's order.
//  srp_keys_kernel: one warp per series, the L bucket keys from its K L bits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hash_common.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSrpSeries = 64;  // series per block tile
constexpr int kSrpHashes = 128; // projections per block pass
constexpr int kSrpChunk = 32;   // samples per staged chunk

__device__ __forceinline__ const float* srp_row(const HashArgs& a, int64_t row) {
    return a.rows ? a.rows[row] : a.series + row * a.stride;
}

__global__ void __launch_bounds__(256) srp_bits_kernel(HashArgs a, const float* R, const float* rn, uint8_t* bits,
                                                       unsigned long long* fix, unsigned long long cap,
                                                       unsigned long long* nfix) {
    __shared__ float xs[kSrpSeries][kSrpChunk + 1];
    __shared__ float rs[kSrpHashes][kSrpChunk + 1];
    __shared__ float es[kSrpSeries];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;  // wy: series group, lane: projection column
    const int m = a.m, KL = a.KL;
    for (int64_t s0 = (int64_t)blockIdx.x * kSrpSeries; s0 < a.count; s0 += (int64_t)gridDim.x * kSrpSeries) {
        for (int h0 = 0; h0 < KL; h0 += kSrpHashes) {
            float acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
            if (h0 == 0 && threadIdx.x < kSrpSeries) es[threadIdx.x] = 0.f;
            for (int k0 = 0; k0 < m; k0 += kSrpChunk) {
                __syncthreads();  // the previous chunk (and es initialisation) are done
                const int kk = k0 + lane;
#pragma unroll
                for (int i = 0; i < 8; ++i) {  // warp wy stages series rows wy*8 .. wy*8+7
                    const int r = wy * 8 + i;
                    const int64_t row = s0 + r;
                    const float x = (row < a.count && kk < m) ? __ldg(srp_row(a, row) + kk) : 0.f;
                    xs[r][lane] = x;
                    if (h0 == 0) {
                        float e = x * x;
                        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(kFull, e, o);
                        if (lane == 0) es[r] += e;
                    }
                }
#pragma unroll 4
                for (int i = 0; i < 16; ++i) {  // warp wy stages projections wy*16 .. wy*16+15
                    const int h = wy * 16 + i;
                    rs[h][lane] = (h0 + h < KL && kk < m) ? __ldg(R + (size_t)(h0 + h) * m + kk) : 0.f;
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < kSrpChunk; ++k) {
                    float xv[8], rv[4];
#pragma unroll
                    for (int i = 0; i < 8; ++i) xv[i] = xs[wy * 8 + i][k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) rv[q] = rs[lane + 32 * q][k];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(xv[i], rv[q], acc[i][q]);
                }
            }
            __syncthreads();  // es is complete
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t row = s0 + wy * 8 + i;
                if (row >= a.count) continue;
                // es carries at most m + 32 roundings of relative 2^-24: inflate it past them
                const float e_up = __fmul_ru(es[wy * 8 + i], 1.0f + (float)(2 * m + 64) * 5.9604645e-08f);
                const float xn = __fsqrt_ru(e_up);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = h0 + lane + 32 * q;
                    if (j >= KL) continue;
                    const float v = acc[i][q];
                    uint8_t bit = 0;
                    if (fabsf(v) > __fmul_ru(__ldg(rn + j), xn)) {
                        bit = v >= 0.f;
                    } else {
                        const unsigned long long slot = atomicAdd(nfix, 1ull);
                        if (slot < cap) {
                            fix[slot] = ((unsigned long long)row << 16) | (unsigned long long)j;
                        } else {  // list full: the definition's FP64 order, here
                            const float* x = srp_row(a, row);
                            double d = 0.0;
                            for (int t = 0; t < m; ++t) d = fma((double)__ldg(R + (size_t)j * m + t), (double)__ldg(x + t), d);
                            bit = d >= 0.0;
                        }
                    }
                    bits[row * KL + j] = bit;
                }
            }
        }
    }
}

__global__ void srp_fixup_kernel(HashArgs a, const float* R, uint8_t* bits, const unsigned long long* fix,
                                 const unsigned long long* nfix, unsigned long long cap) {
    const unsigned long long n = min(*nfix, cap);
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long v = fix[t];
        const int64_t row = (int64_t)(v >> 16);
        const int j = (int)(v & 0xFFFFu);
        const float* x = srp_row(a, row);
        const float* r = R + (size_t)j * a.m;
        double d = 0.0;  // the FP32 x FP32 products are exact in FP64: fma = multiply, then add
        for (int i = 0; i < a.m; ++i) d = fma((double)__ldg(r + i), (double)__ldg(x + i), d);
        bits[row * a.KL + j] = d >= 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats && n) atomicAdd(&a.stats[kStatSketch64], n);
}

__global__ void __launch_bounds__(256) srp_keys_kernel(HashArgs a, const uint8_t* bits) {
    extern __shared__ uint32_t ksm[];  // per warp: K L bits as u32, then K L zeros
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int KL = a.KL;
    uint32_t* kst = ksm + (size_t)warp * 2 * KL;
    uint32_t* tst = kst + KL;
    for (int j = lane; j < KL; j += 32) tst[j] = 0u;
    for (int64_t row = (int64_t)blockIdx.x * wpb + warp; row < a.count; row += (int64_t)gridDim.x * wpb) {
        __syncwarp();
        for (int j = lane; j < KL; j += 32) kst[j] = bits[row * KL + j];
        __syncwarp();
        for (int l = lane; l < a.L; l += 32)
            a.keys[(int64_t)l * a.key_stride + a.key_col0 + row] = bucket_key(a.seed, l, a.K, kst, tst);
    }
}

}  // namespace

size_t srp_scratch_bytes(const HashArgs& a) {
    const size_t bits = ((size_t)a.count * a.KL + 255) & ~(size_t)255;
    const size_t cap = (size_t)a.count * 2 + 65536;
    return bits + 256 + cap * sizeof(unsigned long long);
}

cudaError_t launch_srp_hash(const HashArgs& a, const float* R, const float* rn, void* scratch, int stage,
                            cudaStream_t st) {
    unsigned char* p = static_cast<unsigned char*>(scratch);
    const size_t bits_b = ((size_t)a.count * a.KL + 255) & ~(size_t)255;
    uint8_t* bits = p;
    unsigned long long* nfix = reinterpret_cast<unsigned long long*>(p + bits_b);
    unsigned long long* fix = nfix + 32;
    const unsigned long long cap = (unsigned long long)a.count * 2ull + 65536ull;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (stage == 0) {
        cudaError_t e = cudaMemsetAsync(nfix, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        const int64_t tiles = (a.count + kSrpSeries - 1) / kSrpSeries;
        const int64_t g = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * 8));
        srp_bits_kernel<<<(unsigned)g, 256, 0, st>>>(a, R, rn, bits, fix, cap, nfix);
        note_launch();
        return cudaGetLastError();
    }
    if (stage == 1) {
        const int64_t g = std::max<int64_t>(1, std::min<int64_t>((a.count / 4 + 255) / 256, 4096));
        srp_fixup_kernel<<<(unsigned)g, 256, 0, st>>>(a, R, bits, fix, nfix, cap);
        note_launch();
        return cudaGetLastError();
    }
    const size_t smem = (size_t)8 * 2 * a.KL * sizeof(uint32_t);
    cudaError_t e = ensure_dynamic_smem((const void*)srp_keys_kernel, smem);
    if (e != cudaSuccess) return e;
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>((a.count + 7) / 8, (int64_t)sms * 16));
    srp_keys_kernel<<<(unsigned)g, 256, smem, st>>>(a, bits);
    note_launch();
    return cudaGetLastError();
}

}  // namespace ssh
