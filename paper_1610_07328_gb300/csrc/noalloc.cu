// noalloc.cu -- ssh_hash_device_noalloc: the hashing entry point (sketch,
// FP64 fix-up, shingle and weighted-minhash kernels) with its scratch memory
// in a fixed device array of this library instead of a device allocation, for
// callers that cannot call cudaMalloc (see include/ssh.h).
//
// The array below is a file-scope __device__ variable: in host code its name
// is only a host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress once per device (the first call on a device, with that
// device current) and that address is what the kernels receive.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>

#include "ssh_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)SSH_NOALLOC_SCRATCH_BYTES;

// Scratch shared by every ssh_hash_device_noalloc call on a device. It keeps
// the last call's contents; the one value that must start at zero (the FP64
// fix-up counter) is cleared by each call on its stream.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
std::map<int, void*> g_scratch_addr;  // device ordinal -> device address of g_noalloc_scratch

// Device address of the scratch array on the current device (looked up once per device).
ssh_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ssh::cuda_status(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    auto it = g_scratch_addr.find(dev);
    if (it != g_scratch_addr.end()) {
        *out = it->second;
        return SSH_OK;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return ssh::cuda_status(e, "cudaGetSymbolAddress (no-alloc scratch)");
    g_scratch_addr[dev] = p;
    *out = p;
    return SSH_OK;
}

}  // namespace

extern "C" ssh_status ssh_hash_device_noalloc(const ssh_index* idx, const float* d_series, int32_t m, int64_t count,
                                              void* stream, uint32_t* d_bits, uint32_t* d_sh_ids,
                                              uint32_t* d_sh_counts, int32_t* d_nnz, uint32_t* d_kstar,
                                              uint32_t* d_tstar, uint64_t* d_keys) {
    using namespace ssh;
    if (!idx || count < 0 || (count > 0 && !d_series)) {
        set_error("bad arguments");
        return SSH_EINVAL;
    }
    if (idx->family != 0) {
        set_error("ssh_hash_device_noalloc computes SSH hashes; this index is SRP");
        return SSH_ENOTSUP;
    }
    if ((d_sh_ids == nullptr) != (d_sh_counts == nullptr) || (d_kstar == nullptr) != (d_tstar == nullptr)) {
        set_error("shingle ids/counts and kstar/tstar come in pairs");
        return SSH_EINVAL;
    }
    HashArgs a;
    SSH_TRY(prepare_hash_args(idx, m, &a));
    a.series = d_series;
    a.stride = m;
    a.count = count;
    a.keys = d_keys;
    a.key_stride = count;
    a.key_col0 = 0;
    a.bits_out = d_bits;
    a.sh_ids_out = d_sh_ids;
    a.sh_counts_out = d_sh_counts;
    a.nnz_out = d_nnz;
    a.kstar_out = d_kstar;
    a.tstar_out = d_tstar;
    if (count == 0) return SSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const long long l0 = t_launches;  // this thread's launches: calls on other threads do not count here
    ssh_status status = SSH_OK;
    if ((a.force_generic || !hash_fast_supported(a)) && a.minhash != 0) {
        set_error("the one-permutation minhash needs a compiled sketch shape");
        return SSH_ENOTSUP;
    }
    if (a.force_generic || !hash_fast_supported(a)) {
        // shapes without a specialised pipeline: the single-kernel path needs no scratch
        cudaError_t e = launch_hash_generic(a, st);
        if (e != cudaSuccess) status = cuda_status(e, "generic hash kernel");
    } else {
        const size_t need = hash_fast_scratch_bytes(a);
        if (need > kNoAllocScratchBytes) {
            // the largest count that fits: the scratch size never decreases as the count grows
            // (each sub-buffer grows with it, rounded up to 256 bytes), so bisect on it
            long long lo = 0, hi = (long long)count;  // fits(lo) holds, fits(hi) does not
            while (hi - lo > 1) {
                const long long mid = lo + (hi - lo) / 2;
                HashArgs t = a;
                t.count = mid;
                if (hash_fast_scratch_bytes(t) <= kNoAllocScratchBytes) lo = mid;
                else hi = mid;
            }
            const long long fit = lo;
            set_error("ssh_hash_device_noalloc: %lld series of length %d need %zu bytes of scratch; the fixed "
                      "scratch holds %zu bytes (at most %lld series of this length per call)",
                      (long long)count, m, need, kNoAllocScratchBytes, fit);
            return SSH_EINVAL;
        }
        void* scratch = nullptr;
        SSH_TRY(scratch_address(&scratch));
        const FastHashBuffers b = hash_fast_buffers(a, scratch);
        cudaError_t e = hash_fast_sketch(a, b, st);
        if (e == cudaSuccess) e = hash_fast_fixup(a, b, st);
        if (e == cudaSuccess) e = hash_fast_shingle(a, b, st);
        if (e == cudaSuccess) e = hash_fast_cws(a, b, st);
        if (e != cudaSuccess) status = cuda_status(e, "no-alloc hash pipeline");
    }
    // the index is shared by concurrent callers: add this call's launches atomically
    __atomic_fetch_add(&const_cast<ssh_index*>(idx)->host_stats.kernel_launches, (int64_t)(t_launches - l0),
                       __ATOMIC_RELAXED);
    return status;
}
