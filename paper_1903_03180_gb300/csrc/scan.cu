// Energy of the frames (Sec. 3.3) and the dynamic spatiotemporal buffer scan
// (Sec. 3.2, Eq. 7-9).
//
// k_scan is one persistent cooperative launch over the whole clip.  Each CTA
// owns a fixed set of 8x64 pixel tiles.  For every frame t it
//   (1) computes luma, the Sobel gradient, the frame difference and the energy
//       e_t of its tiles (independent of any buffer decision) and writes Y_t,
//       D_t and e_t;
//   (2) waits until every CTA has published its partial sums for frame t-1,
//       reduces them and takes the buffer decision for t-1 (every CTA takes
//       the same decision from the same integers);
//   (3) folds e_{t-1} into its running sums S1, S2 as that decision says, and
//       publishes its partial A_t = sum floor(sqrt(65536 (n S2 - S1^2))) with
//       frame t added, plus the partial maximum of e_t.
// Step (1) of frame t overlaps the device-wide reduction of frame t-1.
//
// Several clips can share one launch: a table gives each clip its own range
// of CTAs, and the waits and reductions above then run among that range only.
#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int TR = 8, TC = 64, SCAN_THREADS = 256;
enum { DEC_JOIN = 0, DEC_FLUSH = 1, DEC_CLOSE = 2 };

__device__ __forceinline__ int luma_px(const uint8_t *p) {
    return (77 * (int)p[0] + 150 * (int)p[1] + 29 * (int)p[2] + 128) >> 8;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// floor(sqrt(x)) for x < 2^62: a single-precision estimate corrected exactly
// with integer arithmetic.
__device__ __forceinline__ unsigned long long isqrt_u64(unsigned long long x) {
    unsigned long long s = (unsigned long long)__fsqrt_rn(__ull2float_rn(x));
    while (s * s > x) --s;
    while ((s + 1) * (s + 1) <= x) ++s;
    return s;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sobel |Gx| + |Gy| at the centre of a 3x3 window w[r][c] (r, c in 0..2).
__device__ __forceinline__ int sobel3(int a00, int a01, int a02, int a10, int a12, int a20,
                                      int a21, int a22) {
    int gx = (a02 + 2 * a12 + a22) - (a00 + 2 * a10 + a20);
    int gy = (a20 + 2 * a21 + a22) - (a00 + 2 * a01 + a02);
    return abs(gx) + abs(gy);
}

// ---------------------------------------------------------------------------
// Energy of every frame (the scpl_energy entry point).
__global__ void k_energy_api(const uint8_t *__restrict__ rgb, int T, int H, int W, int wg, int wm,
                             int32_t *__restrict__ energy) {
    long hw = (long)H * W;
    long total = hw * T;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x) {
        int t = (int)(q / hw);
        long p = q - (long)t * hw;
        int i = (int)(p / W), j = (int)(p - (long)i * W);
        const uint8_t *f = rgb + (long)t * hw * 3;
        int y[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                y[a][b] = luma_px(f + ((long)clampi(i + a - 1, 0, H - 1) * W +
                                       clampi(j + b - 1, 0, W - 1)) * 3);
        int g = sobel3(y[0][0], y[0][1], y[0][2], y[1][0], y[1][2], y[2][0], y[2][1], y[2][2]);
        int d = 0;
        if (t > 0) d = abs(y[1][1] - luma_px(f - hw * 3 + p * 3));
        energy[q] = wg * g + wm * d;
    }
}

// ---------------------------------------------------------------------------
struct DecState {
    int n;          // frames in the open buffer
    long long M;    // Eq. 9 maxval of the open buffer
    int start;      // first frame of the open buffer
    int nb;         // buffers closed so far
};

// Buffer decision for frame t given the device-wide A_t and max e_t (all CTAs
// evaluate it identically).  Eq. 9: phi(n) = alpha*M*sqrt(n-1)/n, and
// ASDE > phi(n)  <=>  A > 256*alpha*M*sqrt(n-1)*H*W, products left to right.
__device__ int decide(DecState &s, long long A, long long emax, int t, const ScanArgs &a,
                      bool write) {
    int n1 = s.n + 1;
    long long M1 = a.maxval_mode == 1 ? a.maxval_theory : (emax > s.M ? emax : s.M);
    bool exceeds = false;
    if (n1 >= 2) {
        double thr = __dmul_rn(256.0, a.alpha);
        thr = __dmul_rn(thr, __ll2double_rn(M1));
        thr = __dmul_rn(thr, __dsqrt_rn(__int2double_rn(n1 - 1)));
        thr = __dmul_rn(thr, __int2double_rn(a.H));
        thr = __dmul_rn(thr, __int2double_rn(a.W));
        exceeds = __ll2double_rn(A) > thr;
    }
    if (exceeds) {
        if (write) a.starts[s.nb] = s.start;
        s.nb += 1;
        s.start = t;
        s.n = 1;
        s.M = a.maxval_mode == 1 ? a.maxval_theory : emax;
        return DEC_FLUSH;
    }
    s.n = n1;
    s.M = M1;
    if (s.n == a.t_max) {
        if (write) a.starts[s.nb] = s.start;
        s.nb += 1;
        s.start = t + 1;
        s.n = 0;
        s.M = 0;
        return DEC_CLOSE;
    }
    return DEC_JOIN;
}

// Warp 0 waits for every CTA's partials of frame t, reduces them and decides.
// Returns false (and sets the status word) if the wait ran out of time or
// another CTA gave up.
__device__ bool wait_and_decide(const ScanArgs &a, int t, int G, DecState &s, int *dec_out) {
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        int ok = 1;
        if (lane == 0) {
            unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_u32(&a.count[t]) < (unsigned)G) {
                if (*(volatile int *)a.err != DEV_OK) { ok = 0; break; }
                if (globaltimer_ns() - t0 > a.spin_limit_ns) {
                    atomicCAS(a.err, DEV_OK, DEV_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
            __threadfence();
            long long A = 0;
            int m = 0;
            for (int c = lane; c < G; c += 32) {
                A += __ldcg(&a.partA[(long)t * G + c]);
                m = max(m, __ldcg(&a.partM[(long)t * G + c]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                A += __shfl_xor_sync(0xffffffffu, A, o);
                m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            }
            if (lane == 0) *dec_out = decide(s, A, m, t, a, blockIdx.x == (unsigned)a.cta0);
        }
        if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One clip per launch (tab == NULL, every CTA works on a0) or one clip per
// range of CTAs (clip of CTA x = tab[block_clip[x]], CTAs [cta0, cta0 + G)).
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan(ScanArgs a0, const ScanArgs *__restrict__ tab, const int *__restrict__ block_clip) {
    __shared__ ScanArgs a;
    __shared__ uint8_t lum[TR + 2][TC + 2];
    __shared__ long long red_a[SCAN_THREADS / 32];
    __shared__ int red_m[SCAN_THREADS / 32];
    __shared__ DecState st;
    __shared__ int s_dec;

    const int tid = threadIdx.x;
    if (tid == 0) {
        if (tab) {
            a = tab[block_clip[blockIdx.x]];
        } else {
            a = a0;
            a.cta0 = 0;
            a.G = gridDim.x;
        }
    }
    __syncthreads();
    const int G = a.G;
    const int lb = blockIdx.x - a.cta0;   // CTA index within the clip's range
    const int tiles_x = (a.W + TC - 1) / TC;
    const int ntiles = ((a.H + TR - 1) / TR) * tiles_x;
    const long hw = (long)a.H * a.W;
    if (tid == 0) {
        st.n = 0; st.M = 0; st.start = 0; st.nb = 0;
        s_dec = DEC_JOIN;
    }
    __syncthreads();

    for (int t = 0; t < a.T; ++t) {
        // ---- (1) energy of frame t on this CTA's tiles ----------------------
        const uint8_t *f = a.rgb + (long)t * hw * 3;
        uint16_t *ecur = a.ering + (long)(t & 1) * hw;
        int emax = 0;
        for (int tile = lb; tile < ntiles; tile += G) {
            int r0 = (tile / tiles_x) * TR, c0 = (tile % tiles_x) * TC;
            for (int q = tid; q < (TR + 2) * (TC + 2); q += SCAN_THREADS) {
                int r = q / (TC + 2), c = q % (TC + 2);
                int gi = clampi(r0 + r - 1, 0, a.H - 1), gj = clampi(c0 + c - 1, 0, a.W - 1);
                lum[r][c] = (uint8_t)luma_px(f + ((long)gi * a.W + gj) * 3);
            }
            __syncthreads();
            for (int q = tid; q < TR * TC; q += SCAN_THREADS) {
                int r = q / TC, c = q % TC;
                int gi = r0 + r, gj = c0 + c;
                if (gi < a.H && gj < a.W) {
                    int g = sobel3(lum[r][c], lum[r][c + 1], lum[r][c + 2], lum[r + 1][c],
                                   lum[r + 1][c + 2], lum[r + 2][c], lum[r + 2][c + 1],
                                   lum[r + 2][c + 2]);
                    int y = lum[r + 1][c + 1];
                    long yo = (long)t * a.H * a.ypitch + (long)gi * a.ypitch + gj;
                    int d = 0;
                    if (t > 0) d = abs(y - (int)a.Y[yo - (long)a.H * a.ypitch]);
                    int e = a.wg * g + a.wm * d;
                    a.Y[yo] = (uint8_t)y;
                    a.D[yo] = (uint8_t)d;
                    ecur[(long)gi * a.W + gj] = (uint16_t)e;
                    emax = max(emax, e);
                }
            }
            __syncthreads();
        }

        // ---- (2) buffer decision for frame t-1 -------------------------------
        if (t > 0) {
            if (!wait_and_decide(a, t - 1, G, st, &s_dec)) return;
        }
        const int dec = s_dec;
        const int n1 = st.n + 1;

        // ---- (3) fold e_{t-1} into S1/S2, partial A_t ------------------------
        const uint16_t *eprev = a.ering + (long)((t + 1) & 1) * hw;
        unsigned long long acc = 0;
        for (int tile = lb; tile < ntiles; tile += G) {
            int r0 = (tile / tiles_x) * TR, c0 = (tile % tiles_x) * TC;
            for (int q = tid; q < TR * TC; q += SCAN_THREADS) {
                int gi = r0 + q / TC, gj = c0 + q % TC;
                if (gi < a.H && gj < a.W) {
                    long p = (long)gi * a.W + gj;
                    uint32_t s1 = 0, s2 = 0;   // the sums start at zero (no memset)
                    if (t > 0) {
                        s1 = a.S1[p];
                        s2 = a.S2[p];
                        uint32_t ep = eprev[p];
                        if (dec == DEC_JOIN) { s1 += ep; s2 += ep * ep; }
                        else if (dec == DEC_FLUSH) { s1 = ep; s2 = ep * ep; }
                        else { s1 = 0; s2 = 0; }
                    }
                    uint32_t ec = ecur[p];
                    unsigned long long a1 = s1 + ec;
                    unsigned long long a2 = (unsigned long long)s2 + ec * ec;
                    unsigned long long Q = (unsigned long long)n1 * a2 - a1 * a1;
                    acc += isqrt_u64(Q << 16);
                    a.S1[p] = s1;
                    a.S2[p] = s2;
                }
            }
        }
        // block reduction of (acc, emax)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        }
        if ((tid & 31) == 0) { red_a[tid >> 5] = (long long)acc; red_m[tid >> 5] = emax; }
        __syncthreads();
        if (tid == 0) {
            long long A = 0;
            int m = 0;
            for (int w = 0; w < SCAN_THREADS / 32; ++w) { A += red_a[w]; m = max(m, red_m[w]); }
            a.partA[(long)t * G + lb] = A;
            a.partM[(long)t * G + lb] = m;
            __threadfence();
            atomicAdd(&a.count[t], 1u);
        }
        __syncthreads();
    }

    // decision for the last frame, then close the open buffer
    if (!wait_and_decide(a, a.T - 1, G, st, &s_dec)) return;
    if (lb == 0 && tid == 0) {
        int nb = st.nb;
        if (st.n > 0) a.starts[nb++] = st.start;
        a.starts[nb] = a.T;
        *a.n_buffers = nb;
    }
}

}  // namespace

cudaError_t launch_energy_api(const uint8_t *rgb, int T, int H, int W, int wg, int wm,
                              int32_t *energy, cudaStream_t s) {
    long total = (long)T * H * W;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_energy_api<<<blocks, 256, 0, s>>>(rgb, T, H, W, wg, wm, energy);
    return cudaGetLastError();
}

// Co-resident CTAs for the cooperative scan: all SMs' worth, capped by the
// number of tiles of a frame.
int scan_grid_size(int H, int W, int *err_out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan, SCAN_THREADS, 0);
    if (e != cudaSuccess) { *err_out = (int)e; return 0; }
    *err_out = 0;
    long ntiles = (long)((H + TR - 1) / TR) * ((W + TC - 1) / TC);
    long g = (long)sms * per_sm;
    return (int)(g < ntiles ? g : ntiles);
}

cudaError_t launch_scan(const ScanArgs &a, int grid, cudaStream_t s) {
    ScanArgs copy = a;
    const ScanArgs *tab = nullptr;
    const int *bc = nullptr;
    void *args[] = {&copy, &tab, &bc};
    return cudaLaunchCooperativeKernel((const void *)k_scan, dim3(grid), dim3(SCAN_THREADS), args,
                                       0, s);
}

cudaError_t launch_scan_multi(const ScanArgs *tab, const int *block_clip, int grid,
                              cudaStream_t s) {
    ScanArgs none{};
    void *args[] = {&none, &tab, &block_clip};
    return cudaLaunchCooperativeKernel((const void *)k_scan, dim3(grid), dim3(SCAN_THREADS), args,
                                       0, s);
}

int scan_capacity(int *err_out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan, SCAN_THREADS, 0);
    if (e != cudaSuccess) { *err_out = (int)e; return 0; }
    *err_out = 0;
    return sms * per_sm;
}

int scan_tiles(int H, int W) { return ((H + TR - 1) / TR) * ((W + TC - 1) / TC); }

}  // namespace scpl
