// Energy of the frames (Sec. 3.3) and the dynamic spatiotemporal buffer scan
// (Sec. 3.2, Eq. 7-9).
//
// k_scan is one persistent cooperative launch over the whole clip.  Each CTA
// owns a fixed set of 8x128 pixel tiles for the whole clip, and each thread a
// quad of 4 pixels in every tile.  For every frame t it
//   (1) computes luma, the Sobel gradient (4 pixels at once in u16x2 lanes),
//       the frame difference and the energy e_t of its tiles (independent of
//       any buffer decision) and writes Y_t and D_t; e_t stays in registers
//       when the CTA owns at most MAXT tiles;
//   (2) waits until every CTA has published its partial sums for frame t-1,
//       reduces them and takes the buffer decision for t-1 (every CTA takes
//       the same decision from the same integers);
//   (3) folds e_{t-1} into its running sums S1, S2 as that decision says, and
//       publishes its partial A_t = sum floor(sqrt(65536 (n S2 - S1^2))) with
//       frame t added, plus the partial maximum of e_t.  When the decision
//       closes a buffer, S1 (its summed energy, the uniform energy map of
//       Sec. 3.2) is written out for the carving stage.
// Step (1) of frame t overlaps the device-wide reduction of frame t-1.
//
// Several clips can share one launch: a table gives each clip its own range
// of CTAs, and the waits and reductions above then run among that range only.
#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int TR = 8, TC = 128, SCAN_THREADS = 256;
constexpr int LUMW = TC + 8;   // luma tile row: TC + 2 columns, padded to whole words
enum { DEC_JOIN = 0, DEC_FLUSH = 1, DEC_CLOSE = 2 };

__device__ __forceinline__ int luma_px(const uint8_t *p) {
    return (77 * (int)p[0] + 150 * (int)p[1] + 29 * (int)p[2] + 128) >> 8;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

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

// Warp 0 waits until every CTA of the clip has added its partial sums of frame
// t to the clip's accumulators, then decides.  Returns false (and sets the
// status word) if the wait ran out of time or another CTA gave up.
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
        if (ok && lane == 0) {
            __threadfence();
            const long long A = (long long)__ldcg(
                reinterpret_cast<const unsigned long long *>(&a.partA[t]));
            const int m = __ldcg(&a.partM[t]);
            const bool first = blockIdx.x == (unsigned)a.cta0;
            if (first && a.A_out) {
                a.A_out[t] = A;
                a.M_out[t] = m;
            }
            *dec_out = decide(s, A, m, t, a, first);
        }
        if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// floor(sqrt(x)) for x < 2^53 without loops: a single-precision estimate
// (off by a few units at most), one Newton step on the exact integer residual,
// then a final correction by one.  Every float operation is correctly rounded.
__device__ __forceinline__ uint32_t isqrt53(unsigned long long x) {
    const float sf = __fsqrt_rn(__ull2float_rn(x));
    const uint32_t r0 = __float2uint_rz(sf);
    const long long R = (long long)x - (long long)r0 * (long long)r0;
    const float d = __fmul_rn(__ll2float_rn(R), __fdiv_rn(0.5f, __uint2float_rn(r0 > 0 ? r0 : 1)));
    unsigned long long r = (unsigned long long)((long long)r0 + __float2ll_rd(d));
    r -= (r * r > x) ? 1ull : 0ull;
    r += ((r + 1) * (r + 1) <= x) ? 1ull : 0ull;
    return (uint32_t)r;
}

// Packed u16x2 helpers for the 4 pixels of a thread: lane 0 = pixels 0 and 2,
// lane 1 = pixels 1 and 3 of a luma quad.
__device__ __forceinline__ uint32_t even16(uint32_t q) { return __byte_perm(q, 0, 0x4240); }
__device__ __forceinline__ uint32_t odd16(uint32_t q) { return __byte_perm(q, 0, 0x4341); }

// Sobel |Gx| + |Gy| of 4 consecutive pixels from three luma rows.  Each row is
// two aligned words holding the columns c-1 .. c+6 (bytes 0..7); the pixels
// are columns c .. c+3.  Returns (G of pixels 0, 2) and (G of pixels 1, 3).
__device__ __forceinline__ void sobel4(uint32_t u0, uint32_t u1, uint32_t m0, uint32_t m1,
                                       uint32_t d0, uint32_t d1, uint32_t &g02, uint32_t &g13) {
    // left, centre and right neighbours of the 4 pixels in each row
    const uint32_t uL = u0, uC = __funnelshift_r(u0, u1, 8), uR = __funnelshift_r(u0, u1, 16);
    const uint32_t mL = m0, mR = __funnelshift_r(m0, m1, 16);
    const uint32_t dL = d0, dC = __funnelshift_r(d0, d1, 8), dR = __funnelshift_r(d0, d1, 16);
    // the per-lane sums stay below 2^16, so packed adds cannot carry across lanes
    const uint32_t lE = even16(uL) + 2 * even16(mL) + even16(dL);
    const uint32_t rE = even16(uR) + 2 * even16(mR) + even16(dR);
    const uint32_t tE = even16(uL) + 2 * even16(uC) + even16(uR);
    const uint32_t bE = even16(dL) + 2 * even16(dC) + even16(dR);
    g02 = __vabsdiffu2(rE, lE) + __vabsdiffu2(bE, tE);
    const uint32_t lO = odd16(uL) + 2 * odd16(mL) + odd16(dL);
    const uint32_t rO = odd16(uR) + 2 * odd16(mR) + odd16(dR);
    const uint32_t tO = odd16(uL) + 2 * odd16(uC) + odd16(uR);
    const uint32_t bO = odd16(dL) + 2 * odd16(dC) + odd16(dR);
    g13 = __vabsdiffu2(rO, lO) + __vabsdiffu2(bO, tO);
}

// Tile ownership: CTA lb of a clip owns the contiguous tiles
// [lb * tpc, (lb + 1) * tpc) for the whole clip, tpc = ceil(tiles / G).  Up to
// MAXT tiles the CTA keeps S1 and S2 of its pixels in shared memory and the
// previous frame's energy and luma in registers; beyond that they live in
// global memory.
constexpr int MAXT = 4;
constexpr size_t SCAN_SMEM = (size_t)MAXT * SCAN_THREADS * 2 * sizeof(uint4);   // 32 KB

struct TileCtx {
    int r0, c0;      // tile origin
    int row, col;    // this thread's row and first column
    int nvalid;      // valid pixels of the quad (0..4)
};

__device__ __forceinline__ TileCtx tile_ctx(const ScanArgs &a, int tile, int tiles_x, int tid) {
    TileCtx c;
    c.r0 = (tile / tiles_x) * TR;
    c.c0 = (tile % tiles_x) * TC;
    c.row = c.r0 + (tid >> 5);
    c.col = c.c0 + 4 * (tid & 31);
    c.nvalid = c.row < a.H ? max(0, min(4, a.W - c.col)) : 0;
    return c;
}

__device__ __forceinline__ uint32_t luma4(uint32_t w0, uint32_t w1, uint32_t w2) {
    // 12 bytes = pixels p0..p3 as R G B R | G B R G | B R G B
    const uint32_t y0 = (77u * (w0 & 0xFF) + 150u * ((w0 >> 8) & 0xFF) + 29u * ((w0 >> 16) & 0xFF) + 128u) >> 8;
    const uint32_t y1 = (77u * (w0 >> 24) + 150u * (w1 & 0xFF) + 29u * ((w1 >> 8) & 0xFF) + 128u) >> 8;
    const uint32_t y2 = (77u * ((w1 >> 16) & 0xFF) + 150u * (w1 >> 24) + 29u * (w2 & 0xFF) + 128u) >> 8;
    const uint32_t y3 = (77u * ((w2 >> 8) & 0xFF) + 150u * ((w2 >> 16) & 0xFF) + 29u * (w2 >> 24) + 128u) >> 8;
    return y0 | (y1 << 8) | (y2 << 16) | (y3 << 24);
}

// Luma of the tile and its one-pixel frame (replicated at the image border)
// into lum[r][j] = Y(r0 - 1 + r, c0 - 1 + j).  With W a multiple of 4 every
// 4-pixel quad is three aligned words of RGB; otherwise pixel by pixel.
__device__ __forceinline__ void load_luma(const ScanArgs &a, const uint8_t *f, int r0, int c0,
                                          uint8_t (*lum)[LUMW]) {
    const int tid = threadIdx.x;
    if ((a.W & 3) == 0 && (reinterpret_cast<uintptr_t>(a.rgb) & 3) == 0) {
        // body and top/bottom frame rows: (TR + 2) rows x 32 quads
        for (int q = tid; q < (TR + 2) * 32; q += SCAN_THREADS) {
            const int r = q >> 5, x = q & 31;
            const int gi = clampi(r0 + r - 1, 0, a.H - 1);
            const int gj = c0 + 4 * x;
            uint32_t y = 0;
            if (gj < a.W) {
                const uint32_t *w =
                    reinterpret_cast<const uint32_t *>(f + ((long)gi * a.W + gj) * 3);
                y = luma4(__ldg(w), __ldg(w + 1), __ldg(w + 2));
            } else {   // past the right edge: replicate the last column
                y = luma_px(f + ((long)gi * a.W + a.W - 1) * 3) * 0x01010101u;
            }
            // columns c0 + 4x .. c0 + 4x + 3 sit at lum[r][1 + 4x ..]: unaligned by one
            lum[r][1 + 4 * x] = (uint8_t)y;
            lum[r][2 + 4 * x] = (uint8_t)(y >> 8);
            lum[r][3 + 4 * x] = (uint8_t)(y >> 16);
            lum[r][4 + 4 * x] = (uint8_t)(y >> 24);
        }
        // left and right frame columns
        if (tid < 2 * (TR + 2)) {
            const int r = tid >> 1, side = tid & 1;
            const int gi = clampi(r0 + r - 1, 0, a.H - 1);
            const int gj = clampi(side ? c0 + TC : c0 - 1, 0, a.W - 1);
            lum[r][side ? TC + 1 : 0] = (uint8_t)luma_px(f + ((long)gi * a.W + gj) * 3);
        }
    } else {
        for (int q = tid; q < (TR + 2) * (TC + 2); q += SCAN_THREADS) {
            const int r = q / (TC + 2), c = q - r * (TC + 2);
            const int gi = clampi(r0 + r - 1, 0, a.H - 1), gj = clampi(c0 + c - 1, 0, a.W - 1);
            lum[r][c] = (uint8_t)luma_px(f + ((long)gi * a.W + gj) * 3);
        }
    }
}

// One clip per launch (tab == NULL, every CTA works on a0) or one clip per
// range of CTAs (clip of CTA x = tab[block_clip[x]], CTAs [cta0, cta0 + G)).
__global__ void __launch_bounds__(SCAN_THREADS, 4)
k_scan(ScanArgs a0, const ScanArgs *__restrict__ tab, const int *__restrict__ block_clip) {
    extern __shared__ __align__(16) uint4 sstate[];   // [MAXT][2][SCAN_THREADS] S1, S2
    __shared__ ScanArgs a;
    __shared__ __align__(16) uint8_t lum[TR + 2][LUMW];
    __shared__ unsigned long long red_a[SCAN_THREADS / 32];
    __shared__ uint32_t red_m[SCAN_THREADS / 32];
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
        st.n = 0; st.M = 0; st.start = 0; st.nb = 0;
        s_dec = DEC_JOIN;
    }
    __syncthreads();
    const int G = a.G;
    const int lb = blockIdx.x - a.cta0;   // CTA index within the clip's range
    const int tiles_x = (a.W + TC - 1) / TC;
    const int ntiles = ((a.H + TR - 1) / TR) * tiles_x;
    const int tpc = (ntiles + G - 1) / G;
    const int first = lb * tpc;
    const int mine = max(0, min(tpc, ntiles - first));
    const bool resident = tpc <= MAXT;
    const long hw3 = (long)a.H * a.W * 3;
    const long yplane = (long)a.H * a.ypitch;

    // registers of the resident path: energy (u16x2 pairs) and luma quad of the
    // previous and the current frame for each owned tile
    uint32_t ep02[MAXT], ep13[MAXT], yp[MAXT], ec02[MAXT], ec13[MAXT];
#pragma unroll
    for (int k = 0; k < MAXT; ++k) ep02[k] = ep13[k] = yp[k] = ec02[k] = ec13[k] = 0;

    // phase A of one tile: energy of frame t, luma and motion written out
    auto phase_a = [&](int t, int tile, uint32_t &e02, uint32_t &e13, uint32_t &yprev,
                       uint32_t &emax2) {
        const TileCtx c = tile_ctx(a, tile, tiles_x, tid);
        const uint8_t *f = a.rgb + (long)t * hw3;
        load_luma(a, f, c.r0, c.c0, lum);
        __syncthreads();
        const int rr = tid >> 5, cc = 4 * (tid & 31);
        const uint32_t *L0 = reinterpret_cast<const uint32_t *>(&lum[rr][cc]);
        const uint32_t *L1 = reinterpret_cast<const uint32_t *>(&lum[rr + 1][cc]);
        const uint32_t *L2 = reinterpret_cast<const uint32_t *>(&lum[rr + 2][cc]);
        uint32_t g02, g13;
        sobel4(L0[0], L0[1], L1[0], L1[1], L2[0], L2[1], g02, g13);
        const uint32_t ycur = __funnelshift_r(L1[0], L1[1], 8);
        uint32_t yprv = yprev;
        if (!resident && t > 0 && c.nvalid > 0)
            yprv = *reinterpret_cast<const uint32_t *>(a.Y + (long)(t - 1) * yplane +
                                                       (long)c.row * a.ypitch + c.col);
        const uint32_t dq = t > 0 ? __vabsdiffu4(ycur, yprv) : 0u;
        e02 = (uint32_t)a.wg * g02 + (uint32_t)a.wm * even16(dq);
        e13 = (uint32_t)a.wg * g13 + (uint32_t)a.wm * odd16(dq);
        if (c.nvalid > 0) {
            // invalid pixels of a ragged quad do not count towards the maximum
            const uint32_t m02 = c.nvalid >= 3 ? e02 : (e02 & 0xFFFFu);
            const uint32_t m13 = c.nvalid >= 4 ? e13 : (c.nvalid >= 2 ? (e13 & 0xFFFFu) : 0u);
            emax2 = __vmaxu2(emax2, __vmaxu2(m02, m13));
            const long yo = (long)t * yplane + (long)c.row * a.ypitch + c.col;
            *reinterpret_cast<uint32_t *>(a.Y + yo) = ycur;
            *reinterpret_cast<uint32_t *>(a.D + yo) = dq;
        }
        yprev = ycur;
        __syncthreads();   // lum is reused by the next tile
    };

    // phase B of one tile: fold e_{t-1} into S1/S2 as the decision says, add
    // e_t, accumulate floor(sqrt(65536 (n S2 - S1^2))) of the valid pixels
    auto phase_b = [&](int t, int tile, int slot, int dec, int n1, int nb_closed, uint32_t pe02,
                       uint32_t pe13, uint32_t ce02, uint32_t ce13, unsigned long long &acc) {
        const TileCtx c = tile_ctx(a, tile, tiles_x, tid);
        uint4 *S1p, *S2p;
        if (resident) {
            S1p = &sstate[(slot * 2) * SCAN_THREADS + tid];
            S2p = &sstate[(slot * 2 + 1) * SCAN_THREADS + tid];
        } else {
            const long sidx = (long)tile * SCAN_THREADS + tid;
            S1p = reinterpret_cast<uint4 *>(a.S1) + sidx;
            S2p = reinterpret_cast<uint4 *>(a.S2) + sidx;
        }
        uint4 s1 = make_uint4(0, 0, 0, 0), s2 = make_uint4(0, 0, 0, 0);
        if (t > 0) {
            s1 = *S1p;
            s2 = *S2p;
            const uint32_t ep[4] = {pe02 & 0xFFFFu, pe13 & 0xFFFFu, pe02 >> 16, pe13 >> 16};
            uint32_t *S1v = &s1.x, *S2v = &s2.x;
            // the buffer that the decision closed: its summed energy
            const bool closing = dec != DEC_JOIN && a.E0 && nb_closed - 1 < a.nbcap;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (closing && v < c.nvalid)
                    a.E0[(long)(nb_closed - 1) * a.e0_plane + (long)c.row * a.W + c.col + v] =
                        (int32_t)(dec == DEC_CLOSE ? S1v[v] + ep[v] : S1v[v]);
                if (dec == DEC_JOIN) { S1v[v] += ep[v]; S2v[v] += ep[v] * ep[v]; }
                else if (dec == DEC_FLUSH) { S1v[v] = ep[v]; S2v[v] = ep[v] * ep[v]; }
                else { S1v[v] = 0; S2v[v] = 0; }
            }
        }
        *S1p = s1;
        *S2p = s2;
        const uint32_t ec[4] = {ce02 & 0xFFFFu, ce13 & 0xFFFFu, ce02 >> 16, ce13 >> 16};
        const uint32_t *S1v = &s1.x, *S2v = &s2.x;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (v < c.nvalid) {
                const unsigned long long a1 = S1v[v] + ec[v];
                const unsigned long long a2 = (unsigned long long)S2v[v] + ec[v] * ec[v];
                const unsigned long long Q = (unsigned long long)n1 * a2 - a1 * a1;
                acc += isqrt53(Q << 16);
            }
        }
    };

    // the CTA's partial sums of frame t into the clip's accumulators
    auto publish = [&](int t, unsigned long long acc, uint32_t emax2) {
        uint32_t em = max(emax2 & 0xFFFFu, emax2 >> 16);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        }
        if ((tid & 31) == 0) { red_a[tid >> 5] = acc; red_m[tid >> 5] = em; }
        __syncthreads();
        if (tid == 0) {
            unsigned long long A = 0;
            uint32_t m = 0;
            for (int w = 0; w < SCAN_THREADS / 32; ++w) { A += red_a[w]; m = max(m, red_m[w]); }
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.partA[t]), A);
            atomicMax(&a.partM[t], (int)m);
            __threadfence();
            atomicAdd(&a.count[t], 1u);
        }
        __syncthreads();
    };

    uint16_t *ering = a.ering;   // non-resident path: [2][ntiles][256][4]
    const long eslot = (long)ntiles * SCAN_THREADS * 4;

    for (int t = 0; t < a.T; ++t) {
        // ---- (1) energy of frame t on this CTA's tiles ----------------------
        uint32_t emax2 = 0;
        if (resident) {
#pragma unroll
            for (int k = 0; k < MAXT; ++k)
                if (k < mine) phase_a(t, first + k, ec02[k], ec13[k], yp[k], emax2);
        } else {
            for (int k = 0; k < mine; ++k) {
                uint32_t e02, e13, ydummy = 0;
                phase_a(t, first + k, e02, e13, ydummy, emax2);
                const long sidx = (long)(first + k) * SCAN_THREADS + tid;
                reinterpret_cast<uint2 *>(ering + (long)(t & 1) * eslot)[sidx] = make_uint2(e02, e13);
            }
        }

        // ---- (2) buffer decision for frame t-1 -------------------------------
        if (t > 0) {
            if (!wait_and_decide(a, t - 1, G, st, &s_dec)) return;
        }
        const int dec = s_dec;
        const int n1 = st.n + 1;
        const int nbc = st.nb;

        // ---- (3) fold e_{t-1} into S1/S2, partial A_t ------------------------
        unsigned long long acc = 0;
        if (resident) {
#pragma unroll
            for (int k = 0; k < MAXT; ++k)
                if (k < mine) {
                    phase_b(t, first + k, k, dec, n1, nbc, ep02[k], ep13[k], ec02[k], ec13[k], acc);
                    ep02[k] = ec02[k];
                    ep13[k] = ec13[k];
                }
        } else {
            for (int k = 0; k < mine; ++k) {
                const long sidx = (long)(first + k) * SCAN_THREADS + tid;
                const uint2 cur = reinterpret_cast<const uint2 *>(ering + (long)(t & 1) * eslot)[sidx];
                uint2 prv = make_uint2(0, 0);
                if (t > 0)
                    prv = reinterpret_cast<const uint2 *>(ering + (long)((t + 1) & 1) * eslot)[sidx];
                phase_b(t, first + k, 0, dec, n1, nbc, prv.x, prv.y, cur.x, cur.y, acc);
            }
        }
        publish(t, acc, emax2);
    }

    // decision for the last frame, then close the open buffer
    if (!wait_and_decide(a, a.T - 1, G, st, &s_dec)) return;
    const int dec = s_dec;
    // summed energy of the buffers this last decision closed or left open
    if (a.E0) {
        const int nb = st.nb;   // buffers closed so far (after this decision)
        for (int k = 0; k < mine; ++k) {
            const int tile = first + k;
            const TileCtx c = tile_ctx(a, tile, tiles_x, tid);
            if (c.nvalid == 0) continue;
            uint32_t pe02 = 0, pe13 = 0;
            uint4 s1;
            if (resident) {
                // registers hold e_{T-1}; pick the tile's entry without dynamic indexing
#pragma unroll
                for (int q = 0; q < MAXT; ++q)
                    if (q == k) { pe02 = ep02[q]; pe13 = ep13[q]; }
                s1 = sstate[(k * 2) * SCAN_THREADS + tid];
            } else {
                const long sidx = (long)tile * SCAN_THREADS + tid;
                const uint2 v = reinterpret_cast<const uint2 *>(
                    ering + (long)((a.T - 1) & 1) * eslot)[sidx];
                pe02 = v.x; pe13 = v.y;
                s1 = reinterpret_cast<const uint4 *>(a.S1)[sidx];
            }
            const uint32_t ep[4] = {pe02 & 0xFFFFu, pe13 & 0xFFFFu, pe02 >> 16, pe13 >> 16};
            const uint32_t S1v[4] = {s1.x, s1.y, s1.z, s1.w};
            // JOIN: the open buffer ends with frame T-1.  FLUSH: the previous
            // buffer closed before T-1, which is a buffer of its own.  CLOSE:
            // the buffer ending with T-1 closed at t_max.
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (v >= c.nvalid) continue;
                const long px = (long)c.row * a.W + c.col + v;
                if (dec == DEC_JOIN) {
                    if (nb < a.nbcap) a.E0[(long)nb * a.e0_plane + px] = (int32_t)(S1v[v] + ep[v]);
                } else if (dec == DEC_FLUSH) {
                    if (nb - 1 < a.nbcap) a.E0[(long)(nb - 1) * a.e0_plane + px] = (int32_t)S1v[v];
                    if (nb < a.nbcap) a.E0[(long)nb * a.e0_plane + px] = (int32_t)ep[v];
                } else {
                    if (nb - 1 < a.nbcap)
                        a.E0[(long)(nb - 1) * a.e0_plane + px] = (int32_t)(S1v[v] + ep[v]);
                }
            }
        }
    }
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

// Co-resident CTAs for the cooperative scan: all SMs' worth, lowered so that
// every CTA owns the same number of tiles.
int scan_grid_size(int H, int W, int *err_out) {
    const int cap = scan_capacity(err_out);
    if (*err_out || cap < 1) return 0;
    const long ntiles = (long)((H + TR - 1) / TR) * ((W + TC - 1) / TC);
    const long tpc = (ntiles + cap - 1) / cap;
    return (int)((ntiles + tpc - 1) / tpc);
}

cudaError_t launch_scan(const ScanArgs &a, int grid, cudaStream_t s) {
    ScanArgs copy = a;
    const ScanArgs *tab = nullptr;
    const int *bc = nullptr;
    void *args[] = {&copy, &tab, &bc};
    cudaError_t e = cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SCAN_SMEM);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)k_scan, dim3(grid), dim3(SCAN_THREADS), args,
                                       SCAN_SMEM, s);
}

cudaError_t launch_scan_multi(const ScanArgs *tab, const int *block_clip, int grid,
                              cudaStream_t s) {
    ScanArgs none{};
    void *args[] = {&none, &tab, &block_clip};
    cudaError_t e = cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SCAN_SMEM);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)k_scan, dim3(grid), dim3(SCAN_THREADS), args,
                                       SCAN_SMEM, s);
}

int scan_capacity(int *err_out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SCAN_SMEM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan, SCAN_THREADS,
                                                          SCAN_SMEM);
    if (e != cudaSuccess) { *err_out = (int)e; return 0; }
    *err_out = 0;
    return sms * per_sm;
}

int scan_tiles(int H, int W) { return ((H + TR - 1) / TR) * ((W + TC - 1) / TC); }

long scan_state_px(int H, int W) { return (long)scan_tiles(H, W) * TR * TC; }

}  // namespace scpl
