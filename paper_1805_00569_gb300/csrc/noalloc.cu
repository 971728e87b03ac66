// noalloc.cu -- krr_gather_noalloc: the row-grouping step of krr_partition
// (rows grouped by partition, ascending row order inside a partition) for
// callers that must not allocate device memory.
//
// Who needs it: code whose device memory is wholly owned by another
// allocator (a framework's caching allocator that has reserved the GPU, where
// a raw cudaMalloc fails or fragments the pool), and latency-bound request
// loops that forbid allocation on the request path because cudaMalloc and
// cudaFree may synchronise the device and take unbounded time.  Such callers
// already own the input and output buffers and pass them in; the only memory
// the grouping needs beyond them -- one count per (1024-row block, partition)
// -- lives in a fixed file-scope device array instead of being allocated.
//
// The array is part of the library image: every GPU that loads libkrr keeps
// KRR_GATHER_SCRATCH_ENTRIES * 8 bytes (4 MiB) for it until the process
// exits.  All calls share it and it keeps the last call's contents; the
// kernels overwrite every entry they read, so nothing needs clearing, but two
// calls that overlap on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include <mutex>

#include "common.cuh"
#include "internal.h"

#define KRR_GATHER_SCRATCH_ENTRIES (1 << 19)
#define KRR_GATHER_BLOCK 1024
#define KRR_MAX_DEVICES 64

namespace krr {
// the stable-gather kernels of partition.cu, reused unchanged
__global__ void gather_count_kernel(const int32_t *__restrict__ a, int64_t n, int32_t p,
                                    long long *__restrict__ bcount);
__global__ void gather_scan_kernel(long long *__restrict__ bcount, int64_t nblk, int32_t p,
                                   int64_t *__restrict__ offsets);
__global__ void gather_scatter_kernel(const int32_t *__restrict__ a, int64_t n, int32_t p,
                                      const long long *__restrict__ bstart, int64_t *__restrict__ perm);
}  // namespace krr

// Scratch for the per-block partition counts.  In host code this name is a
// host-side stand-in, not a device address: only the address obtained with
// cudaGetSymbolAddress below may be handed to a kernel.
static __device__ __align__(256) long long g_gather_scratch[KRR_GATHER_SCRATCH_ENTRIES];

static std::mutex g_scratch_mu;
static long long *g_scratch_addr[KRR_MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does the lookup).
static cudaError_t scratch_on_current_device(long long **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= KRR_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gather_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<long long *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

extern "C" krr_status krr_gather_noalloc(void *cuda_stream, const int32_t *assign, int64_t n, int32_t p,
                                         int64_t *perm, int64_t *offsets) {
    if (n < 0 || p <= 0 || !offsets || (n > 0 && (!assign || !perm))) return KRR_ERR_ARG;
    const int64_t nblk = (n + KRR_GATHER_BLOCK - 1) / KRR_GATHER_BLOCK;
    // capacity: one count per (block, partition); the count kernel keeps one
    // int per partition in shared memory (48 KiB without opt-in)
    if (nblk * (int64_t)p > KRR_GATHER_SCRATCH_ENTRIES || (int64_t)p * 4 > 48 * 1024) return KRR_ERR_ARG;
    long long *scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return KRR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (nblk > 0) {
        KRR_LAUNCHED(), krr::gather_count_kernel<<<(unsigned)nblk, 256, p * sizeof(int), st>>>(assign, n, p,
                                                                                             scratch);
    }
    // the scan keeps one total per partition in shared memory (p <= 12288: 96 KiB)
    if (krr::allow_max_dyn_smem(krr::gather_scan_kernel) != cudaSuccess) return KRR_ERR_CUDA;
    KRR_LAUNCHED(), krr::gather_scan_kernel<<<1, 1024, (size_t)p * sizeof(long long), st>>>(scratch, nblk, p,
                                                                                            offsets);
    if (nblk > 0) {
        KRR_LAUNCHED(), krr::gather_scatter_kernel<<<(unsigned)nblk, 128, KRR_GATHER_BLOCK * sizeof(int32_t), st>>>(
            assign, n, p, scratch, perm);
    }
    return cudaGetLastError() == cudaSuccess ? KRR_OK : KRR_ERR_CUDA;
}
