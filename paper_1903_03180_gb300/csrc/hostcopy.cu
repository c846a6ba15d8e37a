// Bulk copies between page-locked host memory and device memory, done by a
// kernel that reads or writes the host side over the CPU-GPU link.
//
// On a Grace-attached GB300 the copy engines' host-to-device rate falls from
// about 210 GB/s to 25-60 GB/s for seconds at a time once copies have run for
// a while, and device-to-host copies follow at times.  Loads and stores issued
// by SMs over the same link hold 209-211 GB/s (up) and 192 GB/s (down) the
// whole time, and a few dozen SMs already reach those rates.  So every bulk
// frame copy of the host-memory paths goes through k_link_copy; the rest of
// the GPU stays free for the carving kernels and the scan.  A host pointer
// that the device cannot address (pageable memory without a mapping) falls
// back to cudaMemcpyAsync.
#include <cuda_runtime.h>

#include <cstdint>

#include "scpl.h"
#include "scpl_internal.cuh"

namespace scpl {

namespace {

// 16 CTAs of 1024 threads.  Such a copy holds the link's rate both ways
// (4 loads of 16 bytes in flight per thread, about 1 MB in all) while it
// shares only 16 SMs with the kernels it overlaps.  Measured on the streamed
// 1080p clips (page-locked in and out, one GB300), the steady time per clip
// was 19.5 ms against 18.9 ms with no copies at all; copies spread over more
// SMs disturbed the carving more (48 x 512: 27.3 ms, 152 x 128: 30.3 ms,
// 24 x 512: 21.0 ms), and fewer SMs could not keep up (6 x 1024: 26.3 ms).
constexpr int LINK_CTAS = 16;
constexpr int LINK_THREADS = 1024;

// dst[0, n) = src[0, n).  When both pointers share their offset within 16
// bytes, the bytes up to the first 16-byte boundary go singly, the body as
// 16-byte streaming loads and stores, and the tail singly; otherwise every
// byte goes singly.  Every index stays below n.
__global__ void __launch_bounds__(LINK_THREADS)
k_link_copy(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, size_t n) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    const uintptr_t ms = reinterpret_cast<uintptr_t>(src) & 15u;
    const uintptr_t md = reinterpret_cast<uintptr_t>(dst) & 15u;
    if (ms != md) {
        for (size_t i = tid; i < n; i += nth) dst[i] = src[i];
        return;
    }
    size_t head = (16u - md) & 15u;
    if (head > n) head = n;
    if (tid < head) dst[tid] = src[tid];
    const size_t n16 = (n - head) / 16;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
#pragma unroll 4
    for (size_t i = tid; i < n16; i += nth) __stcs(d4 + i, __ldcs(s4 + i));
    for (size_t i = head + n16 * 16 + tid; i < n; i += nth) dst[i] = src[i];
}

// The device-side address of p if it is page-locked (allocated or
// registered with CUDA) or device memory; NULL if the device cannot address it.
const void *device_view(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();   // an unknown pointer is not an error here
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        // the pointer may lie inside the allocation: keep its offset
        const char *base_h = static_cast<const char *>(a.hostPointer);
        const char *base_d = static_cast<const char *>(a.devicePointer);
        return base_h ? base_d + (static_cast<const char *>(p) - base_h) : a.devicePointer;
    }
    return nullptr;
}

}  // namespace

cudaError_t link_copy(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    const void *sv = device_view(src);
    void *dv = const_cast<void *>(device_view(dst));
    // unmapped memory, or offsets within 16 bytes that differ (the kernel
    // would copy byte by byte): the copy engine
    if (!sv || !dv || ((reinterpret_cast<uintptr_t>(sv) ^ reinterpret_cast<uintptr_t>(dv)) & 15u))
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    const size_t blocks_needed = (bytes + (size_t)LINK_THREADS * 16 - 1) / ((size_t)LINK_THREADS * 16);
    const int blocks = (int)(blocks_needed < (size_t)LINK_CTAS ? blocks_needed : LINK_CTAS);
    k_link_copy<<<blocks, LINK_THREADS, 0, s>>>(static_cast<const uint8_t *>(sv),
                                                 static_cast<uint8_t *>(dv), bytes);
    return cudaGetLastError();
}

}  // namespace scpl

extern "C" scpl_status scpl_copy(void *dst, const void *src, size_t bytes, void *stream) {
    if ((!dst || !src) && bytes) return SCPL_EINVAL;
    return scpl::link_copy(dst, src, bytes, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SCPL_OK
               : SCPL_ECUDA;
}
