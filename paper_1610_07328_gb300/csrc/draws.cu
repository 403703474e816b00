// draws.cu -- the Sec. 4.3 draw tables of an index, built on the GPU at
// ssh_create from the same definition the minhash kernels use (Philox draws,
// Ioffe's ICWS, ln by ln_fixed, every FP64 operation rounded to nearest):
//
//   p64   [KL][2^n][3]      (r, beta, ln c)
//   p32   [2^n][KL]         (r, 1/r, beta, ln c) rounded to FP32
//   lav   [2^n][8][KLp]     ln a of counts 1..8 rounded once to FP32
//   tsm   [2^n][7][KLp]     t of counts 2..8 (255: not tabulated)
//   rank  [2^n][KLr]        rank of the count-1 ln a of (j, k) among all k (ties: smaller k first)
//   kla   [KL][2^n]         per rank: (k, bits of its FP32 count-1 ln a)
//   lns64, lns32 [0..kMaxCount]  ln s (s = 0: -inf, never read)
//
// The ranks come from a bitonic sort of (order-preserving 64-bit key of the FP64
// value, k) per hash, a chunk of hashes at a time: passes with a stride of 1024
// or more go through global memory, the rest of each stage through a 2048-entry
// tile in shared memory. Keys are distinct (k breaks ties), so the unstable
// network gives the same order as a stable sort by (value, k).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hash_common.cuh"
#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr int kTile = 2048;  // entries per shared-memory tile of the sort (1024 threads)

struct DrawTables {
    int n, KL, KLr, KLp;
    int64_t nk;
    uint64_t seed;
    double* p64;
    float4* p32;
    float* lav;
    uint8_t* tsm;
};

__global__ void lns_kernel(double* lns64, float* lns32, int nmax) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= nmax; s += gridDim.x * blockDim.x) {
        const double v = (s == 0) ? __longlong_as_double(0xFFF0000000000000ll) : ln_fixed((double)s);
        lns64[s] = v;
        lns32[s] = __double2float_rn(v);
    }
}

// FP64 -> u64 with the same order (-0 counted as +0): the sort key of a count-1 ln a.
__device__ __forceinline__ uint64_t order_key(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(__dadd_rn(v, 0.0));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// One thread per (k, j) with j fastest, for hashes [j0, j0 + nj): every table
// entry of (j, k), and the sort key of its count-1 value in row j - j0.
__global__ void draws_kernel(DrawTables t, const double* lns64, int j0, int nj, uint64_t* keys, uint32_t* ids) {
    const int64_t total = t.nk * nj;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int jj = (int)(i % nj);
        const int64_t k = i / nj;
        const int j = j0 + jj;
        double r, beta, lnc;
        cws_draw_dev(t.seed, (uint32_t)j, (uint32_t)k, &r, &beta, &lnc);
        double* q = t.p64 + ((size_t)j * t.nk + k) * 3;
        q[0] = r;
        q[1] = beta;
        q[2] = lnc;
        t.p32[(size_t)k * t.KL + j] = make_float4(__double2float_rn(r), __double2float_rn(__ddiv_rn(1.0, r)),
                                                  __double2float_rn(beta), __double2float_rn(lnc));
        double la1 = 0.0;
        for (int c = 1; c <= kTabCounts; ++c) {
            const double lns = lns64[c];
            const double tt = floor(__dadd_rn(__ddiv_rn(lns, r), beta));
            const double la = __dsub_rn(lnc, __dmul_rn(r, __dadd_rn(__dsub_rn(tt, beta), 1.0)));
            if (c == 1) la1 = la;
            t.lav[((size_t)k * kTabCounts + (c - 1)) * t.KLp + j] = __double2float_rn(la);
            if (c >= 2)
                t.tsm[((size_t)k * (kTabCounts - 1) + (c - 2)) * t.KLp + j] =
                    (tt >= 0.0 && tt < 255.0) ? (uint8_t)tt : (uint8_t)255;
        }
        keys[(size_t)jj * t.nk + k] = order_key(la1);
        ids[(size_t)jj * t.nk + k] = (uint32_t)k;
    }
}

__device__ __forceinline__ bool key_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// One compare-exchange step of the bitonic network (stage size `stage`, stride
// `stride`) on every row: thread t handles the pair (i, i + stride).
__global__ void bitonic_global_kernel(uint64_t* keys, uint32_t* ids, int64_t nk, int rows, int64_t stage,
                                      int64_t stride) {
    const int64_t half = nk >> 1;
    const int64_t total = half * rows;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / half, u = t - row * half;
        const int64_t i = 2 * stride * (u / stride) + (u % stride);
        const int64_t l = i + stride;
        uint64_t* kr = keys + row * nk;
        uint32_t* ir = ids + row * nk;
        const bool up = (i & stage) == 0;
        const uint64_t ka = kr[i], kb = kr[l];
        const uint32_t ia = ir[i], ib = ir[l];
        if (key_less(kb, ib, ka, ia) == up) {
            kr[i] = kb;
            kr[l] = ka;
            ir[i] = ib;
            ir[l] = ia;
        }
    }
}

// The strides stride0, stride0/2, .., 1 of stage `stage` on tiles of kTile entries
// (stride0 < kTile), or, with stage == 0, every stage 2 .. kTile whole (the tile's
// first sort). One block of kTile/2 threads per tile.
__global__ void __launch_bounds__(kTile / 2) bitonic_tile_kernel(uint64_t* keys, uint32_t* ids, int64_t nk,
                                                                 int64_t stage, int stride0) {
    __shared__ uint64_t sk[kTile];
    __shared__ uint32_t si[kTile];
    const int64_t tiles_per_row = nk / kTile;
    const int64_t row = blockIdx.x / tiles_per_row;
    const int64_t base = row * nk + (blockIdx.x - row * tiles_per_row) * kTile;
    const int64_t gbase = (blockIdx.x - row * tiles_per_row) * kTile;  // index within the row
    for (int x = threadIdx.x; x < kTile; x += blockDim.x) {
        sk[x] = keys[base + x];
        si[x] = ids[base + x];
    }
    __syncthreads();
    const int u = threadIdx.x;
    auto step = [&](int64_t stg, int stride) {
        const int i = 2 * stride * (u / stride) + (u % stride);
        const int l = i + stride;
        const bool up = ((gbase + i) & stg) == 0;
        const uint64_t ka = sk[i], kb = sk[l];
        const uint32_t ia = si[i], ib = si[l];
        if (key_less(kb, ib, ka, ia) == up) {
            sk[i] = kb;
            sk[l] = ka;
            si[i] = ib;
            si[l] = ia;
        }
        __syncthreads();
    };
    if (stage == 0) {
        for (int stg = 2; stg <= kTile; stg <<= 1)
            for (int stride = stg >> 1; stride > 0; stride >>= 1) step(stg, stride);
    } else {
        for (int stride = stride0; stride > 0; stride >>= 1) step(stage, stride);
    }
    for (int x = threadIdx.x; x < kTile; x += blockDim.x) {
        keys[base + x] = sk[x];
        ids[base + x] = si[x];
    }
}

// Sorted rows -> rank[k][j] and kla[j][rank] (k, FP32 count-1 ln a bits).
__global__ void rank_kernel(DrawTables t, int j0, int nj, const uint32_t* ids, uint16_t* rank, uint2* kla) {
    const int64_t total = t.nk * nj;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int jj = (int)(i / t.nk);
        const int64_t pos = i - (int64_t)jj * t.nk;
        const int j = j0 + jj;
        const uint32_t k = ids[i];
        rank[(size_t)k * t.KLr + j] = (uint16_t)pos;
        kla[(size_t)j * t.nk + pos] = make_uint2(k, __float_as_uint(t.lav[(size_t)k * kTabCounts * t.KLp + j]));
    }
}

unsigned grid_of(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 64));
}

}  // namespace

ssh_status build_draw_tables(ssh_index* idx, cudaStream_t st) {
    const int n = idx->n, KL = idx->KL;
    // ln s for every count (also used by the tables-free minhash of n > kMaxShingleBits)
    SSH_CUDA(cudaMalloc(&idx->d_lns64, (kMaxCount + 1) * sizeof(double)));
    SSH_CUDA(cudaMalloc(&idx->d_lns32, (kMaxCount + 1) * sizeof(float)));
    lns_kernel<<<grid_of(kMaxCount + 1, 256), 256, 0, st>>>(idx->d_lns64, idx->d_lns32, kMaxCount);
    note_launch();
    SSH_CUDA(cudaGetLastError());
    if (n > kMaxShingleBits) return SSH_OK;  // draws computed on the fly by the minhash kernel

    DrawTables t;
    t.n = n;
    t.KL = KL;
    t.KLr = rank_stride_of(KL);
    t.KLp = tab_stride_of(KL);
    t.nk = (int64_t)1 << n;
    t.seed = idx->seed;
    SSH_CUDA(cudaMalloc(&idx->d_p64, (size_t)KL * t.nk * 3 * sizeof(double)));
    SSH_CUDA(cudaMalloc(&idx->d_p32, (size_t)t.nk * KL * sizeof(float4)));
    SSH_CUDA(cudaMalloc(&idx->d_lav, (size_t)t.nk * kTabCounts * t.KLp * sizeof(float)));
    SSH_CUDA(cudaMalloc(&idx->d_tsm, (size_t)t.nk * (kTabCounts - 1) * t.KLp));
    SSH_CUDA(cudaMalloc(&idx->d_rank, (size_t)t.nk * t.KLr * sizeof(uint16_t)));
    SSH_CUDA(cudaMalloc(&idx->d_kla, (size_t)KL * t.nk * sizeof(uint2)));
    SSH_CUDA(cudaMemsetAsync(idx->d_lav, 0, (size_t)t.nk * kTabCounts * t.KLp * sizeof(float), st));
    SSH_CUDA(cudaMemsetAsync(idx->d_tsm, 0xFF, (size_t)t.nk * (kTabCounts - 1) * t.KLp, st));
    SSH_CUDA(cudaMemsetAsync(idx->d_rank, 0xFF, (size_t)t.nk * t.KLr * sizeof(uint16_t), st));
    t.p64 = idx->d_p64;
    t.p32 = idx->d_p32;
    t.lav = idx->d_lav;
    t.tsm = idx->d_tsm;

    // sort scratch for a chunk of hashes: at most ~512 MB of (key, id) rows
    const int64_t row_bytes = t.nk * (int64_t)(sizeof(uint64_t) + sizeof(uint32_t));
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(KL, (512ll << 20) / row_bytes));
    uint64_t* keys = nullptr;
    uint32_t* ids = nullptr;
    SSH_CUDA(cudaMallocAsync(&keys, (size_t)chunk * t.nk * sizeof(uint64_t), st));
    cudaError_t e = cudaMallocAsync(&ids, (size_t)chunk * t.nk * sizeof(uint32_t), st);
    for (int j0 = 0; j0 < KL && e == cudaSuccess; j0 += chunk) {
        const int nj = std::min(chunk, KL - j0);
        draws_kernel<<<grid_of(t.nk * nj, 256), 256, 0, st>>>(t, idx->d_lns64, j0, nj, keys, ids);
        note_launch();
        e = cudaGetLastError();
        if (t.nk < kTile) {
            // rows shorter than a tile: the whole network in global memory
            for (int64_t stage = 2; stage <= t.nk && e == cudaSuccess; stage <<= 1)
                for (int64_t stride = stage >> 1; stride > 0 && e == cudaSuccess; stride >>= 1) {
                    bitonic_global_kernel<<<grid_of((t.nk >> 1) * nj, 256), 256, 0, st>>>(keys, ids, t.nk, nj,
                                                                                          stage, stride);
                    note_launch();
                    e = cudaGetLastError();
                }
        } else {
            const unsigned tiles = (unsigned)(t.nk / kTile * nj);
            bitonic_tile_kernel<<<tiles, kTile / 2, 0, st>>>(keys, ids, t.nk, 0, 0);
            note_launch();
            e = cudaGetLastError();
            for (int64_t stage = 2 * kTile; stage <= t.nk && e == cudaSuccess; stage <<= 1) {
                int64_t stride = stage >> 1;
                for (; stride >= kTile && e == cudaSuccess; stride >>= 1) {
                    bitonic_global_kernel<<<grid_of((t.nk >> 1) * nj, 256), 256, 0, st>>>(keys, ids, t.nk, nj,
                                                                                          stage, stride);
                    note_launch();
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) {
                    bitonic_tile_kernel<<<tiles, kTile / 2, 0, st>>>(keys, ids, t.nk, stage, (int)stride);
                    note_launch();
                    e = cudaGetLastError();
                }
            }
        }
        if (e == cudaSuccess) {
            rank_kernel<<<grid_of(t.nk * nj, 256), 256, 0, st>>>(t, j0, nj, ids, idx->d_rank, idx->d_kla);
            note_launch();
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(keys, st);
    if (ids) cudaFreeAsync(ids, st);
    SSH_CUDA(e);
    SSH_CUDA(cudaStreamSynchronize(st));
    return SSH_OK;
}

}  // namespace ssh
