// sort_kernels.cu -- the device-resident bucket tables of Algorithm 1 and the
// selections of Algorithm 2.
//
// Tables: one most-significant-digit radix pass per table. The top B bits of
// each 64-bit bucket key pick one of 2^B bins (B chosen so a bin holds about
// 16 rows); a histogram, an exclusive scan and a scatter place every (key, row)
// in its bin (large tables take two passes, below). Equal keys always share a
// bin, so a probe scans the query key's bin and compares full keys; the order
// inside a bin is not used.
// Selections: per-segment radix select of the k-th smallest key.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

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

// ----------------------------------------- two-pass partition of large tables
//
// Bins of about 16 rows number 2^B (B up to 24): one scatter into all of them
// writes every entry to a random place. Large tables are partitioned in two
// passes instead: pass 1 scatters by the top b1 = min(12, B - 7) key bits
// through per-block shared-memory histograms over chunks of 4,096 rows, so each
// block writes contiguous runs per bucket; pass 2 takes one bucket (1-2K
// entries at the usual sizes) per block and places its entries into the
// bucket's 2^(B-b1) bins in shared memory before writing them out.

constexpr int kPartThreads = 512;
constexpr int kPartItems = 8;                             // rows per thread of pass 1
constexpr int kPartChunk = kPartThreads * kPartItems;     // rows per block of pass 1

// Exclusive prefix sums of a[0 .. count) in shared memory (all threads of the block).
__device__ void block_exclusive_scan(uint32_t* a, int count, uint32_t* part) {
    const int per = (count + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(count, b + per);
    uint32_t sum = 0;
    for (int i = b; i < e; ++i) sum += a[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = b; i < e; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPartThreads) part_hist_kernel(const uint64_t* keys, int64_t row0, int64_t n,
                                                                 int64_t cap, int b1, int nblk, uint32_t* counts) {
    extern __shared__ uint32_t h[];
    const int l = blockIdx.y, blk = blockIdx.x, nb = 1 << b1;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const uint64_t* k = keys + (int64_t)l * cap + row0;
    const int64_t lo = (int64_t)blk * kPartChunk, hi = min(n, lo + kPartChunk);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[(uint32_t)(k[i] >> (64 - b1))], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += blockDim.x) counts[((int64_t)l * nb + d) * nblk + blk] = h[d];
}

// Offsets of pass 1, in two steps. part_scan_blocks_kernel: one warp per
// (table, bucket) turns the bucket's per-block counts into exclusive offsets
// within the bucket and writes the bucket's total into bstart[l][d].
// part_scan_buckets_kernel: one block per table turns the totals into the
// buckets' starts (bstart[l][nb] = n). The scatter adds the two.
__global__ void part_scan_blocks_kernel(uint32_t* counts, int nb, int nblk, int L, uint32_t* bstart) {
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)L * nb) return;  // whole warps only (blockDim is a multiple of 32)
    const int l = (int)(wid / nb), d = (int)(wid - (int64_t)l * nb);
    uint32_t* c = counts + ((int64_t)l * nb + d) * nblk;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nblk; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t v = (b < nblk) ? c[b] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += u;
        }
        if (b < nblk) c[b] = carry + incl - v;
        carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) bstart[(int64_t)l * (nb + 1) + d] = carry;
}

__global__ void __launch_bounds__(1024) part_scan_buckets_kernel(int nb, uint32_t* bstart) {
    __shared__ uint32_t part[1024];
    uint32_t* bs = bstart + (int64_t)blockIdx.x * (nb + 1);
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(nb, b + per);
    uint32_t sum = 0;
    for (int i = b; i < e; ++i) sum += bs[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = b; i < e; ++i) {
        const uint32_t v = bs[i];
        bs[i] = run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) bs[nb] = part[blockDim.x - 1];
}

// Pass 1 scatter: the block's chunk is first ordered by bucket in shared
// memory, then each bucket's run is written out with consecutive threads on
// consecutive addresses.
__global__ void __launch_bounds__(kPartThreads) part_scatter_kernel(const uint64_t* keys, int64_t row0, int64_t n,
                                                                    int64_t cap, int b1, int nblk,
                                                                    const uint32_t* offs, const uint32_t* bstart,
                                                                    uint64_t* tk, uint32_t* tr) {
    extern __shared__ __align__(16) unsigned char psm[];
    const int l = blockIdx.y, blk = blockIdx.x, nb = 1 << b1;
    uint64_t* skey = reinterpret_cast<uint64_t*>(psm);                          // [kPartChunk]
    uint32_t* srow = reinterpret_cast<uint32_t*>(skey + kPartChunk);            // [kPartChunk]
    uint32_t* lstart = srow + kPartChunk;                                       // [nb] local run starts
    uint32_t* gbase = lstart + nb;                                              // [nb] global run starts
    uint32_t* part = gbase + nb;                                                // [kPartThreads]
    for (int d = threadIdx.x; d < nb; d += blockDim.x) {
        lstart[d] = 0u;
        gbase[d] = bstart[(int64_t)l * (nb + 1) + d] + offs[((int64_t)l * nb + d) * nblk + blk];
    }
    __syncthreads();
    const uint64_t* k = keys + (int64_t)l * cap + row0;
    const int64_t lo = (int64_t)blk * kPartChunk;
    const int cnt = (int)min((int64_t)kPartChunk, n - lo);
    uint64_t key[kPartItems];
    uint32_t rnk[kPartItems];
#pragma unroll
    for (int t = 0; t < kPartItems; ++t) {
        const int i = t * kPartThreads + threadIdx.x;
        if (i < cnt) {
            key[t] = k[lo + i];
            rnk[t] = atomicAdd(&lstart[(uint32_t)(key[t] >> (64 - b1))], 1u);
        }
    }
    __syncthreads();
    block_exclusive_scan(lstart, nb, part);
#pragma unroll
    for (int t = 0; t < kPartItems; ++t) {
        const int i = t * kPartThreads + threadIdx.x;
        if (i < cnt) {
            const uint32_t at = lstart[(uint32_t)(key[t] >> (64 - b1))] + rnk[t];
            skey[at] = key[t];
            srow[at] = (uint32_t)(row0 + lo + i);
        }
    }
    __syncthreads();
    uint64_t* tkl = tk + (int64_t)l * n;
    uint32_t* trl = tr + (int64_t)l * n;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const uint64_t kj = skey[j];
        const uint32_t d = (uint32_t)(kj >> (64 - b1));
        const uint32_t pos = gbase[d] + ((uint32_t)j - lstart[d]);
        tkl[pos] = kj;
        trl[pos] = srow[j];
    }
}

// Pass 2: bucket d of table l into its 2^b2 bins (bins[l][(d << b2) + e] = bin
// start; the bucket's block also writes bins[l][2^B] = n when it is the last).
// A bucket of at most kRegionTile entries (all of them at the usual sizes) is
// read once into registers, counted, placed in shared memory at its bin's
// position and written out with consecutive threads on consecutive addresses.
// A larger bucket is taken a tile at a time: one pass counts, a second places
// each entry straight into the output through the shared bin cursors.
constexpr int kRegionThreads = 256;
constexpr int kRegionItems = 12;
constexpr int kRegionTile = kRegionThreads * kRegionItems;

size_t region_smem(int b2) {
    return (size_t)kRegionTile * 12 + ((size_t)(1 << b2) + kRegionThreads) * sizeof(uint32_t);
}

__global__ void __launch_bounds__(kRegionThreads) part_region_kernel(const uint64_t* tk, const uint32_t* tr, int64_t n,
                                                                     const uint32_t* bstart, int b1, int b2,
                                                                     int64_t out_stride, uint32_t* bins,
                                                                     uint64_t* skeys, uint32_t* srows) {
    extern __shared__ __align__(16) unsigned char rsm[];
    const int d = blockIdx.x, l = blockIdx.y, nb = 1 << b1, n2 = 1 << b2;
    uint64_t* pkey = reinterpret_cast<uint64_t*>(rsm);                                   // [kRegionTile]
    uint32_t* prow = reinterpret_cast<uint32_t*>(pkey + kRegionTile);                    // [kRegionTile]
    uint32_t* h = prow + kRegionTile;                                                    // [2^b2]
    uint32_t* part = h + n2;                                                             // [blockDim.x]
    const uint32_t* bs = bstart + (int64_t)l * (nb + 1);
    const int64_t s0 = bs[d], s1 = bs[d + 1];
    const uint64_t* tkl = tk + (int64_t)l * n;
    const uint32_t* trl = tr + (int64_t)l * n;
    const int shift = 64 - b1 - b2;
    const uint32_t mask = (uint32_t)n2 - 1u;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    uint32_t* bl = bins + (int64_t)l * (((int64_t)nb << b2) + 1);
    uint64_t* sk = skeys + (int64_t)l * out_stride;
    uint32_t* sr = srows + (int64_t)l * out_stride;
    uint64_t key[kRegionItems];
    uint32_t row[kRegionItems];
    if (s1 - s0 <= kRegionTile) {
        const int cnt = (int)(s1 - s0);
        uint32_t rnk[kRegionItems];
#pragma unroll
        for (int u = 0; u < kRegionItems; ++u) {
            const int i = u * kRegionThreads + threadIdx.x;
            if (i < cnt) {
                key[u] = tkl[s0 + i];
                row[u] = trl[s0 + i];
            }
        }
#pragma unroll
        for (int u = 0; u < kRegionItems; ++u)
            if (u * kRegionThreads + (int)threadIdx.x < cnt) rnk[u] = atomicAdd(&h[(uint32_t)(key[u] >> shift) & mask], 1u);
        __syncthreads();
        block_exclusive_scan(h, n2, part);
        for (int i = threadIdx.x; i < n2; i += blockDim.x) bl[((int64_t)d << b2) + i] = (uint32_t)s0 + h[i];
        if (d == nb - 1 && threadIdx.x == 0) bl[(int64_t)nb << b2] = (uint32_t)s1;
#pragma unroll
        for (int u = 0; u < kRegionItems; ++u) {
            if (u * kRegionThreads + (int)threadIdx.x < cnt) {
                const uint32_t at = h[(uint32_t)(key[u] >> shift) & mask] + rnk[u];  // < cnt
                pkey[at] = key[u];
                prow[at] = row[u];
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            sk[s0 + j] = pkey[j];
            sr[s0 + j] = prow[j];
        }
        return;
    }
    // counts (the first tile stays in registers for the placement)
    for (int64_t t0 = s0; t0 < s1; t0 += kRegionTile) {
#pragma unroll
        for (int u = 0; u < kRegionItems; ++u) {
            const int64_t i = t0 + u * kRegionThreads + threadIdx.x;
            uint64_t kk = 0;
            if (i < s1) kk = tkl[i];
            if (t0 == s0) key[u] = kk;
            if (i < s1) atomicAdd(&h[(uint32_t)(kk >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    block_exclusive_scan(h, n2, part);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        bl[((int64_t)d << b2) + i] = (uint32_t)s0 + h[i];
        h[i] += (uint32_t)s0;  // now the placement cursors
    }
    if (d == nb - 1 && threadIdx.x == 0) bl[(int64_t)nb << b2] = (uint32_t)s1;
    __syncthreads();
    for (int64_t t0 = s0; t0 < s1; t0 += kRegionTile) {
#pragma unroll
        for (int u = 0; u < kRegionItems; ++u) {
            const int64_t i = t0 + u * kRegionThreads + threadIdx.x;
            if (i < s1) {
                if (t0 != s0) key[u] = tkl[i];
                row[u] = trl[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kRegionItems; ++u) {
            const int64_t i = t0 + u * kRegionThreads + threadIdx.x;
            if (i < s1) {
                const uint32_t pos = atomicAdd(&h[(uint32_t)(key[u] >> shift) & mask], 1u);
                sk[pos] = key[u];
                sr[pos] = row[u];
            }
        }
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
    if (bin_bits >= 12 && n >= 65536) {
        // two passes: buckets of the top b1 bits, then the bins inside each bucket
        // bins of ~16 rows, 2^7 of them per bucket: buckets of ~2K entries (b1 at most 12)
        const int b1 = std::min(12, bin_bits - 7), b2 = bin_bits - b1, nb = 1 << b1;
        const int nblk = (int)((n + kPartChunk - 1) / kPartChunk);
        uint32_t *counts = nullptr, *bstart = nullptr, *tr = nullptr;
        uint64_t* tk = nullptr;
        cudaError_t e = cudaMallocAsync(&counts, (size_t)L * nb * nblk * sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaMallocAsync(&bstart, (size_t)L * (nb + 1) * sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaMallocAsync(&tk, (size_t)L * n * sizeof(uint64_t), st);
        if (e == cudaSuccess) e = cudaMallocAsync(&tr, (size_t)L * n * sizeof(uint32_t), st);
        if (e == cudaSuccess) {
            const dim3 g1((unsigned)nblk, (unsigned)L);
            part_hist_kernel<<<g1, kPartThreads, nb * sizeof(uint32_t), st>>>(keys, row0, n, cap, b1, nblk, counts);
            const int64_t warps = (int64_t)L * nb;
            part_scan_blocks_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(counts, nb, nblk, L, bstart);
            part_scan_buckets_kernel<<<(unsigned)L, 1024, 0, st>>>(nb, bstart);
            const size_t smem1 = (size_t)kPartChunk * 12 + ((size_t)2 * nb + kPartThreads) * sizeof(uint32_t);
            e = ensure_dynamic_smem((const void*)part_scatter_kernel, smem1);
            if (e == cudaSuccess)
                part_scatter_kernel<<<g1, kPartThreads, smem1, st>>>(keys, row0, n, cap, b1, nblk, counts, bstart,
                                                                    tk, tr);
            const size_t smem2 = region_smem(b2);
            if (e == cudaSuccess) e = ensure_dynamic_smem((const void*)part_region_kernel, smem2);
            if (e == cudaSuccess)
                part_region_kernel<<<dim3((unsigned)nb, (unsigned)L), kRegionThreads, smem2, st>>>(
                    tk, tr, n, bstart, b1, b2, out_stride, bins, skeys, srows);
            note_launch(5);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        cudaFreeAsync(counts, st);
        cudaFreeAsync(bstart, st);
        cudaFreeAsync(tk, st);
        cudaFreeAsync(tr, st);
        (void)cursor;
        return e;
    }
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
