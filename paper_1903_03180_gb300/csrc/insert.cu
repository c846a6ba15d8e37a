// Seam insertion: widening a clip by the seams that SCPL carving removes.
//
// k_insert_seams: grid (H, nb), IB threads.  For row i of buffer b the CTA
// marks the buffer's m inserted original columns (the seams carving removed
// from the buffer, in removal order) in a bitmap, takes the exclusive prefix
// of the words' bit counts, and then writes that row of every frame of the
// buffer: original pixel x goes to x + (inserted columns before x), and after
// an inserted column x comes the rounded mean of pixels x and x+1 (x itself
// at the last column).
#include <cuda_runtime.h>

#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int IB = 256;            // threads per CTA; one bitmap word each
constexpr int IMAXW = IB * 32;     // widest frame: 8192 columns

__global__ void __launch_bounds__(IB)
k_insert_seams(const uint8_t *__restrict__ frames, int H, int W, int target,
               const int16_t *__restrict__ seams, long seam_stride, int m,
               const int *__restrict__ starts, int b0, uint8_t *__restrict__ out) {
    __shared__ uint32_t bits[IB];
    __shared__ int before[IB];
    __shared__ int wsum[IB / 32];
    const int i = blockIdx.x, b = b0 + blockIdx.y, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nw = (W + 31) >> 5;
    bits[tid] = 0;
    __syncthreads();
    const int16_t *sb = seams + (long)b * seam_stride;
    for (int s = tid; s < m; s += IB) {
        const int c = sb[(long)s * H + i];
        if (c >= 0 && c < W) atomicOr(&bits[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
    // exclusive prefix of the words' bit counts
    const int n = tid < nw ? __popc(bits[tid]) : 0;
    int inc = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int off = 0;
    for (int x = 0; x < warp; ++x) off += wsum[x];
    before[tid] = off + inc - n;
    __syncthreads();

    const int t0 = starts[b], t1 = starts[b + 1];
    for (int t = t0; t < t1; ++t) {
        const uint8_t *src = frames + ((long)t * H + i) * W * 3;
        uint8_t *dst = out + ((long)t * H + i) * target * 3;
        for (int x = tid; x < W; x += IB) {
            const uint32_t w = bits[x >> 5];
            const int pos = x + before[x >> 5] + __popc(w & ((1u << (x & 31)) - 1u));
            const uint8_t r = src[3 * x], g = src[3 * x + 1], bl = src[3 * x + 2];
            if (pos < target) {
                dst[3 * pos] = r;
                dst[3 * pos + 1] = g;
                dst[3 * pos + 2] = bl;
            }
            if (((w >> (x & 31)) & 1u) && pos + 1 < target) {
                const int xn = min(x + 1, W - 1);
                dst[3 * pos + 3] = (uint8_t)((r + src[3 * xn] + 1) >> 1);
                dst[3 * pos + 4] = (uint8_t)((g + src[3 * xn + 1] + 1) >> 1);
                dst[3 * pos + 5] = (uint8_t)((bl + src[3 * xn + 2] + 1) >> 1);
            }
        }
    }
}

}  // namespace

cudaError_t launch_insert_seams(const uint8_t *frames, int H, int W, int target,
                                const int16_t *seams, long seam_stride, int m,
                                const int *starts, int nb, uint8_t *out, cudaStream_t s) {
    if (W > IMAXW) return cudaErrorInvalidValue;
    for (int b0 = 0; b0 < nb; b0 += 65535) {   // grid y is at most 65535
        const int n = nb - b0 < 65535 ? nb - b0 : 65535;
        k_insert_seams<<<dim3(H, n), IB, 0, s>>>(frames, H, W, target, seams, seam_stride, m,
                                                 starts, b0, out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace scpl
