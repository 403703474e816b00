// sort_kernels.cu -- the device-resident bucket tables of Algorithm 1 and the
// selections of Algorithm 2.
//
// Tables: one most-significant-digit radix pass per table. The top B bits of
// each 64-bit bucket key pick one of 2^B bins (B chosen so a bin holds about
// 16 rows); a histogram, an exclusive scan and a scatter place every (key, row)
// in its bin. Equal keys always share a bin, so a probe scans the query key's
// bin and compares full keys; the order inside a bin is not used.
// Selections: per-segment radix select of the k-th smallest key.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr int kRadix = 256;

// ------------------------------------------------------------ radix select

template <typename T>
__global__ void __launch_bounds__(512) select_kth_kernel(const T* keys, const int64_t* seg_begin, int k, T* kth_out) {
    constexpr int kBits = sizeof(T) * 8;
    __shared__ uint32_t h[kRadix];
    __shared__ T s_prefix;
    __shared__ uint32_t s_remaining;
    const int seg = blockIdx.x;
    const int64_t b = seg_begin[seg], e = seg_begin[seg + 1];
    if (e - b < k) {
        if (threadIdx.x == 0) kth_out[seg] = ~(T)0;
        return;
    }
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_remaining = (uint32_t)k;
    }
    T mask = 0;
    for (int shift = kBits - 8; shift >= 0; shift -= 8) {
        for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
        __syncthreads();
        const T prefix = s_prefix;
        for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            const T v = keys[i];
            if ((v & mask) == prefix) atomicAdd(&h[(uint32_t)(v >> shift) & 0xFFu], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t rem = s_remaining;
            int d = 0;
            for (; d < kRadix; ++d) {
                if (h[d] >= rem) break;
                rem -= h[d];
            }
            s_remaining = rem;
            s_prefix = prefix | ((T)d << shift);
        }
        mask |= ((T)0xFF << shift);
        __syncthreads();
    }
    if (threadIdx.x == 0) kth_out[seg] = s_prefix;
}

// ---------------------------------------------------- table partition

__global__ void bin_hist_kernel(const uint64_t* keys, int64_t row0, int64_t n, int64_t cap, int shift, int nbins,
                                uint32_t* counts) {
    const int l = blockIdx.y;
    const uint64_t* k = keys + (int64_t)l * cap + row0;
    uint32_t* c = counts + (int64_t)l * (nbins + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[(uint32_t)(k[i] >> shift)], 1u);
}

// Exclusive scan of one table's bin counts in place (nbins + 1 entries: the
// last becomes n), and a copy into the scatter cursors.
__global__ void __launch_bounds__(1024) bin_scan_kernel(uint32_t* counts, uint32_t* cursor, int nbins) {
    __shared__ uint32_t part[1024];
    const int l = blockIdx.x;
    uint32_t* c = counts + (int64_t)l * (nbins + 1);
    uint32_t* cur = cursor + (int64_t)l * (nbins + 1);
    const int total = nbins + 1;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(total, b + per);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += c[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = b; i < e; ++i) {
        const uint32_t v = c[i];
        c[i] = run;
        cur[i] = run;
        run += v;
    }
}

__global__ void bin_scatter_kernel(const uint64_t* keys, int64_t row0, int64_t n, int64_t cap, int64_t out_stride,
                                   int shift, int nbins, uint32_t* cursor, uint64_t* skeys, uint32_t* srows) {
    const int l = blockIdx.y;
    const uint64_t* k = keys + (int64_t)l * cap + row0;
    uint32_t* cur = cursor + (int64_t)l * (nbins + 1);
    uint64_t* sk = skeys + (int64_t)l * out_stride;
    uint32_t* sr = srows + (int64_t)l * out_stride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = k[i];
        const uint32_t pos = atomicAdd(&cur[(uint32_t)(key >> shift)], 1u);
        sk[pos] = key;
        sr[pos] = (uint32_t)(row0 + i);
    }
}

}  // namespace

int table_bin_bits(int64_t n) {
    int b = 1;
    while (b < 30 && ((int64_t)1 << (b + 4)) < n) ++b;  // about 16 rows per bin
    if (b < 8) b = 8;
    if (b > 24) b = 24;
    return b;
}

cudaError_t build_tables(const uint64_t* keys, int64_t row0, int64_t n, int L, int64_t cap, int64_t out_stride,
                         int bin_bits, uint32_t* bins, uint32_t* cursor, uint64_t* skeys, uint32_t* srows,
                         cudaStream_t st) {
    const int nbins = 1 << bin_bits;
    const int shift = 64 - bin_bits;
    cudaError_t e = cudaMemsetAsync(bins, 0, (size_t)L * (nbins + 1) * sizeof(uint32_t), st);
    if (e != cudaSuccess || n <= 0) return e;
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    dim3 grid((unsigned)g, (unsigned)L);
    bin_hist_kernel<<<grid, 256, 0, st>>>(keys, row0, n, cap, shift, nbins, bins);
    note_launch();
    bin_scan_kernel<<<(unsigned)L, 1024, 0, st>>>(bins, cursor, nbins);
    note_launch();
    bin_scatter_kernel<<<grid, 256, 0, st>>>(keys, row0, n, cap, out_stride, shift, nbins, cursor, skeys, srows);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_select_kth_u32(const uint32_t* keys, const int64_t* seg_begin, int64_t nseg, int k,
                                  uint32_t* kth_out, cudaStream_t st) {
    if (nseg <= 0) return cudaSuccess;
    select_kth_kernel<uint32_t><<<(unsigned)nseg, 512, 0, st>>>(keys, seg_begin, k, kth_out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_select_kth_u64(const uint64_t* keys, const int64_t* seg_begin, int64_t nseg, int k,
                                  uint64_t* kth_out, cudaStream_t st) {
    if (nseg <= 0) return cudaSuccess;
    select_kth_kernel<unsigned long long><<<(unsigned)nseg, 512, 0, st>>>(
        reinterpret_cast<const unsigned long long*>(keys), seg_begin, k,
        reinterpret_cast<unsigned long long*>(kth_out));
    note_launch();
    return cudaGetLastError();
}

}  // namespace ssh
