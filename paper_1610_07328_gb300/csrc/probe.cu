// A plain read of a device buffer through L2 (loads that skip L1), used to put a
// measured L2 read bandwidth beside the minhash kernel's gather rate. Not part of
// the method: it computes nothing the search uses.
#include <cstdint>

#include "ssh_internal.cuh"

using namespace ssh;

namespace {

__device__ unsigned long long g_read_sink;

// Every pass reads all n16 16-byte words once: thread t of block b reads words
// (b' * blockDim + t) + j * stride, with b' = (b + 37 * pass) mod grid, so each
// pass hands every block other addresses. Four loads are in flight per thread.
__global__ void __launch_bounds__(512) read_l2_kernel(const uint4* __restrict__ p, size_t n16, int passes) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < passes; ++r) {
        const size_t blk = ((size_t)blockIdx.x + (size_t)r * 37) % gridDim.x;
        size_t i = blk * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride);
            const uint4 c = __ldcg(p + i + 2 * stride), d = __ldcg(p + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9e3779b9u) atomicAdd(&g_read_sink, 1ull);  // keeps the loads; almost never taken
}

}  // namespace

extern "C" ssh_status ssh_read_device(const void* d_buf, uint64_t bytes, int32_t passes, void* stream) {
    if (!d_buf || bytes == 0 || bytes % 16 != 0 || (reinterpret_cast<uintptr_t>(d_buf) & 15) != 0 || passes < 1)
        return fail_status(SSH_EINVAL, "ssh_read_device: needs a 16-byte aligned buffer, bytes > 0 and a "
                                       "multiple of 16, passes >= 1");
    int dev = 0, sms = 0, per_sm = 0;
    SSH_CUDA(cudaGetDevice(&dev));
    SSH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SSH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, read_l2_kernel, 512, 0));
    read_l2_kernel<<<sms * (per_sm > 0 ? per_sm : 1), 512, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4*>(d_buf), bytes / 16, passes);
    SSH_CUDA(cudaGetLastError());
    return SSH_OK;
}
