// Quality measure of a retargeted video: the sharpness of blends of
// consecutive frames, a numeric stand-in for the paper's Fig. 9 (Sec. 4).
// On a nearly static clip, frames from which the same seams were removed
// blend into a sharp image; frames carved independently displace their
// content and blend into a blurred one.
//
// For every run of `window` frames t .. t+window-1 the blend is the sum of
// their integer BT.601 luma maps; num adds the L1 Sobel magnitude
// |Gx| + |Gy| (3x3, replicate border) of the blend, den the magnitudes of the
// run's frames.  Both are exact 64-bit sums.
#include <cuda_runtime.h>

#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int QB = 256;   // threads per block of k_blend_sobel

__global__ void k_luma_frames(const uint8_t *__restrict__ rgb, long n, uint8_t *__restrict__ Y) {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x) {
        const uint8_t *p = rgb + q * 3;
        Y[q] = (uint8_t)((77u * p[0] + 150u * p[1] + 29u * p[2] + 128u) >> 8);
    }
}

__device__ __forceinline__ int sobel_l1(const int (&v)[3][3]) {
    const int gx = (v[0][2] + 2 * v[1][2] + v[2][2]) - (v[0][0] + 2 * v[1][0] + v[2][0]);
    const int gy = (v[2][0] + 2 * v[2][1] + v[2][2]) - (v[0][0] + 2 * v[0][1] + v[0][2]);
    return abs(gx) + abs(gy);
}

// grid (ceil(W/QB), H, T - window + 1): one thread per pixel of one run
__global__ void __launch_bounds__(QB) k_blend_sobel(const uint8_t *__restrict__ Y, int H, int W,
                                                    int window,
                                                    unsigned long long *__restrict__ acc) {
    __shared__ unsigned long long s_num[QB / 32], s_den[QB / 32];
    const int j = blockIdx.x * QB + threadIdx.x, i = blockIdx.y, t = blockIdx.z;
    unsigned long long num = 0, den = 0;
    if (j < W) {
        const int rows[3] = {max(i - 1, 0), i, min(i + 1, H - 1)};
        const int cols[3] = {max(j - 1, 0), j, min(j + 1, W - 1)};
        int blend[3][3] = {};
        for (int w = 0; w < window; ++w) {
            const uint8_t *f = Y + (long)(t + w) * H * W;
            int v[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    v[a][c] = f[(long)rows[a] * W + cols[c]];
                    blend[a][c] += v[a][c];
                }
            den += (unsigned long long)sobel_l1(v);
        }
        num = (unsigned long long)sobel_l1(blend);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_num[warp] = num;
        s_den[warp] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int x = 0; x < QB / 32; ++x) {
            a += s_num[x];
            b += s_den[x];
        }
        atomicAdd(acc, a);
        atomicAdd(acc + 1, b);
    }
}

}  // namespace

cudaError_t launch_blend_sharpness(const uint8_t *frames, int T, int H, int W, int window,
                                   uint8_t *Y, unsigned long long *acc, cudaStream_t s) {
    const long n = (long)T * H * W;
    k_luma_frames<<<(unsigned)std::min<long>((n + 255) / 256, 152L * 16), 256, 0, s>>>(frames, n, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int runs = T - window + 1;
    for (int t0 = 0; t0 < runs; t0 += 65535) {   // grid z is at most 65535
        const int nr = std::min(runs - t0, 65535);
        k_blend_sobel<<<dim3((W + QB - 1) / QB, H, nr), QB, 0, s>>>(Y + (long)t0 * H * W, H, W,
                                                                    window, acc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace scpl
