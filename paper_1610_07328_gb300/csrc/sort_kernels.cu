// sort_kernels.cu -- device-resident bucket tables of Algorithm 1 are built by a
// stable LSD radix sort of (64-bit key, 32-bit row) pairs, one segment per
// table; the top-k of Algorithm 2 uses a per-segment radix select.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ssh_internal.cuh"

namespace ssh {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                       // items per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 items per CTA
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadix = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t* keys, int64_t n, int64_t seg_stride,
                                                                  int shift, int ntiles, uint32_t* counts) {
    __shared__ uint32_t h[kRadix];
    const int seg = blockIdx.y, tile = blockIdx.x;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const uint64_t* k = keys + (int64_t)seg * seg_stride;
    const int64_t base = (int64_t)tile * kSortTile;
    for (int t = threadIdx.x; t < kSortTile; t += blockDim.x) {
        const int64_t i = base + t;
        if (i < n) atomicAdd(&h[(uint32_t)(k[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    uint32_t* c = counts + (int64_t)seg * kRadix * ntiles;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) c[(int64_t)d * ntiles + tile] = h[d];
}

// Exclusive scan of one segment's digit-major counts (kRadix * ntiles values).
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* counts, int ntiles) {
    __shared__ uint32_t part[1024];
    const int seg = blockIdx.x;
    uint32_t* c = counts + (int64_t)seg * kRadix * ntiles;
    const int64_t total = (int64_t)kRadix * ntiles;
    const int64_t per = (total + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(total, b + per);
    uint32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += c[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int64_t i = b; i < e; ++i) {
        uint32_t v = c[i];
        c[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint64_t* keys_in, const uint32_t* vals_in,
                                                                     uint64_t* keys_out, uint32_t* vals_out, int64_t n,
                                                                     int64_t seg_stride, int shift, int ntiles,
                                                                     const uint32_t* offsets) {
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    const int seg = blockIdx.y, tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < kRadix; d += 32) wcnt[warp][d] = 0;
    __syncwarp();
    const uint64_t* ki = keys_in + (int64_t)seg * seg_stride;
    const uint32_t* vi = vals_in + (int64_t)seg * seg_stride;
    const int64_t wbase = (int64_t)tile * kSortTile + (int64_t)warp * (32 * kSortItems);
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t loc[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const bool ok = i < n;
        key[r] = ok ? ki[i] : 0ull;
        val[r] = ok ? vi[i] : 0u;
        const uint32_t d = ok ? ((uint32_t)(key[r] >> shift) & 0xFFu) : 0x100u;
        const unsigned peers = __match_any_sync(kFull, d);
        const uint32_t before = (d < 0x100u) ? wcnt[warp][d] : 0u;
        loc[r] = before + __popc(peers & lt);
        __syncwarp();
        if (d < 0x100u && (peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // prefix over warps per digit (warp order = item order within the tile)
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t v = wcnt[w][d];
            wcnt[w][d] = run;
            run += v;
        }
    }
    __syncthreads();
    const uint32_t* off = offsets + (int64_t)seg * kRadix * ntiles;
    uint64_t* ko = keys_out + (int64_t)seg * seg_stride;
    uint32_t* vo = vals_out + (int64_t)seg * seg_stride;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)(key[r] >> shift) & 0xFFu;
            const int64_t dst = (int64_t)off[(int64_t)d * ntiles + tile] + wcnt[warp][d] + loc[r];
            ko[dst] = key[r];
            vo[dst] = val[r];
        }
    }
}

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

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n, int nseg) {
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    return (size_t)nseg * kRadix * (size_t)(ntiles > 0 ? ntiles : 1) * sizeof(uint32_t);
}

cudaError_t radix_sort_pairs_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                                 int nseg, int64_t seg_stride, void* scratch, size_t scratch_bytes, cudaStream_t st,
                                 int first_bit) {
    if (n <= 1 || nseg <= 0) return cudaSuccess;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    if (scratch_bytes < radix_sort_scratch_bytes(n, nseg) || ntiles > (1 << 24)) return cudaErrorInvalidValue;
    uint32_t* counts = static_cast<uint32_t*>(scratch);
    uint64_t* kin = keys;
    uint32_t* vin = vals;
    uint64_t* kout = keys_alt;
    uint32_t* vout = vals_alt;
    dim3 grid((unsigned)ntiles, (unsigned)nseg);
    if (first_bit < 0 || first_bit > 56 || (first_bit % 16) != 0) return cudaErrorInvalidValue;
    for (int shift = first_bit; shift < 64; shift += 8) {
        radix_hist_kernel<<<grid, kSortThreads, 0, st>>>(kin, n, seg_stride, shift, (int)ntiles, counts);
        note_launch();
        radix_scan_kernel<<<nseg, 1024, 0, st>>>(counts, (int)ntiles);
        note_launch();
        radix_scatter_kernel<<<grid, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, seg_stride, shift, (int)ntiles,
                                                            counts);
        note_launch();
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    return cudaGetLastError();  // an even number of passes: the sorted data is back in (keys, vals)
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
