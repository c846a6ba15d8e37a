// Energy of the frames (Sec. 3.3) and the dynamic spatiotemporal buffer scan
// (Sec. 3.2, Eq. 7-9).
//
// k_scan is one persistent cooperative launch over the whole clip.  Each CTA
// owns a fixed block of 8x128 pixel tiles for the whole clip, and each thread
// a quad of 4 pixels in every tile.  For every frame it computes luma, the
// Sobel gradient (4 pixels at once in u16x2 lanes), the frame difference and
// the energy e_t (written out as Y_t and D_t), folds e_t into the running sums
// S1, S2 of the open buffer and adds its share of
// A_t = sum floor(sqrt(65536 (n S2 - S1^2))) to the clip's accumulator.  The
// decisions of Eq. 9 need every CTA's share, so frames are taken in rounds
// with one device-wide wait per round (see k_scan below).  When a decision
// closes a buffer, its S1 (the summed energy, the uniform energy map of
// Sec. 3.2) is written out for the carving stage.
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

// Thread 0 waits until every CTA of the clip has published round r.  Returns
// false (and sets the status word) if the wait ran out of time or another CTA
// gave up.
__device__ bool wait_round(const ScanArgs &a, int r, int G) {
    if (ld_acquire_u32(&a.count[r]) >= (unsigned)G) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (ld_acquire_u32(&a.count[r]) < (unsigned)G) {
        if (*(volatile int *)a.err != DEV_OK) return false;
        if (globaltimer_ns() - t0 > a.spin_limit_ns) {
            atomicCAS(a.err, DEV_OK, DEV_ETIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// floor(sqrt(x)) for x < 2^53 without loops.  A hardware square-root
// estimate (relative error below 2^-22) is off by a few units at most; one
// Newton step on the exact integer residual, with an approximate reciprocal,
// lands within one of the answer, and a final exact correction by one each
// way settles it.  Only the correction decides the result, so the estimates
// need no particular rounding.
__device__ __forceinline__ uint32_t isqrt53(unsigned long long x) {
    const float xf = __ull2float_rz(x);
    const float r0f = xf > 0.0f ? xf * rsqrtf(xf) : 0.0f;
    const uint32_t r0 = __float2uint_rz(r0f);
    const long long R = (long long)x - (long long)((unsigned long long)r0 * r0);
    const float d = __ll2float_rz(R) * __frcp_rz(2.0f * fmaxf(r0f, 1.0f));
    uint32_t r = r0 + (uint32_t)__float2int_rd(d);
    r -= ((unsigned long long)r * r > x) ? 1u : 0u;
    r += ((unsigned long long)(r + 1) * (r + 1) <= x) ? 1u : 0u;
    return r;
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
    const int ty = tile / tiles_x;
    c.r0 = ty * TR;
    c.c0 = (tile - ty * tiles_x) * TC;
    c.row = c.r0 + (tid >> 5);
    c.col = c.c0 + 4 * (tid & 31);
    c.nvalid = c.row < a.H ? max(0, min(4, a.W - c.col)) : 0;
    return c;
}

// Luma of 4 pixels from their 12 RGB bytes (R G B R | G B R G | B R G B):
// one byte dot product per pixel with the weights (77, 150, 29, 0).
__device__ __forceinline__ uint32_t luma4(uint32_t w0, uint32_t w1, uint32_t w2) {
    constexpr uint32_t K = 77u | (150u << 8) | (29u << 16);
    const uint32_t y0 = __dp4a(w0, K, 128u) >> 8;
    const uint32_t y1 = __dp4a(__byte_perm(w0, w1, 0x0543), K, 128u) >> 8;
    const uint32_t y2 = __dp4a(__byte_perm(w1, w2, 0x0432), K, 128u) >> 8;
    const uint32_t y3 = __dp4a(w2 >> 8, K, 128u) >> 8;
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
//
// Rounds: a round takes the next frames [t, w] (at most SCAN_FW, never past
// the frame where the open buffer reaches t_max, never past T - 1) and folds
// each into S1/S2 as if it joined the open buffer, publishing every frame's
// A_t.  After one device-wide wait every CTA replays the decisions of Eq. 9 in
// frame order on the same integers.  Up to the first frame that exceeds the
// threshold the guess was right.  At that frame f a new buffer starts: the
// closed buffer's sum is S1 minus the energies of frames f..w, S1/S2 restart
// from e_f, and the next round re-evaluates frames f+1..w from their stored
// energies.
__global__ void __launch_bounds__(SCAN_THREADS, 4)
k_scan(ScanArgs a0, const ScanArgs *__restrict__ tab, const int *__restrict__ block_clip) {
    extern __shared__ __align__(16) uint4 sstate[];   // [MAXT][2][SCAN_THREADS] S1, S2
    __shared__ ScanArgs a;
    __shared__ __align__(16) uint8_t lum[TR + 2][LUMW];
    __shared__ unsigned long long red_a[SCAN_THREADS / 32];
    __shared__ uint32_t red_m[SCAN_THREADS / 32];
    __shared__ DecState st;
    __shared__ int s_ok, s_ndec, s_last;
    __shared__ uint32_t s_rc[64];   // origins (r0 << 16 | c0) of the CTA's first 64 tiles

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
    const long eslot = (long)ntiles * SCAN_THREADS;   // uint2 entries per ring slot
    uint2 *ering = reinterpret_cast<uint2 *>(a.ering);  // [SCAN_FW][ntiles][256] e quads
    for (int k = tid; k < min(mine, 64); k += SCAN_THREADS) {
        const int ty = (first + k) / tiles_x;
        s_rc[k] = ((uint32_t)(ty * TR) << 16) | (uint32_t)((first + k - ty * tiles_x) * TC);
    }
    __syncthreads();
    // the geometry of the CTA's k-th tile for this thread
    auto ctx = [&](int k) {
        if (k >= 64) return tile_ctx(a, first + k, tiles_x, tid);
        TileCtx c;
        c.r0 = (int)(s_rc[k] >> 16);
        c.c0 = (int)(s_rc[k] & 0xFFFFu);
        c.row = c.r0 + (tid >> 5);
        c.col = c.c0 + 4 * (tid & 31);
        c.nvalid = c.row < a.H ? max(0, min(4, a.W - c.col)) : 0;
        return c;
    };
    uint32_t yp[MAXT];   // resident path: previous frame's luma quad per tile
#pragma unroll
    for (int k = 0; k < MAXT; ++k) yp[k] = 0;

    // energy of frame t on one tile: luma and motion written out, the e quad
    // (u16x2 pairs) stored in the ring
    auto phase_a = [&](int t, int k, uint32_t &yprev, uint32_t &emax2) {
        const int tile = first + k;
        const TileCtx c = ctx(k);
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
        const uint32_t e02 = (uint32_t)a.wg * g02 + (uint32_t)a.wm * even16(dq);
        const uint32_t e13 = (uint32_t)a.wg * g13 + (uint32_t)a.wm * odd16(dq);
        if (c.nvalid > 0) {
            // invalid pixels of a ragged quad do not count towards the maximum
            const uint32_t m02 = c.nvalid >= 3 ? e02 : (e02 & 0xFFFFu);
            const uint32_t m13 = c.nvalid >= 4 ? e13 : (c.nvalid >= 2 ? (e13 & 0xFFFFu) : 0u);
            emax2 = __vmaxu2(emax2, __vmaxu2(m02, m13));
            const long yo = (long)t * yplane + (long)c.row * a.ypitch + c.col;
            *reinterpret_cast<uint32_t *>(a.Y + yo) = ycur;
            *reinterpret_cast<uint32_t *>(a.D + yo) = dq;
        }
        ering[(long)(t % SCAN_FW) * eslot + (long)tile * SCAN_THREADS + tid] = make_uint2(e02, e13);
        yprev = ycur;
        __syncthreads();   // lum is reused by the next tile
    };

    auto state_ptrs = [&](int k, int tile, uint4 *&S1p, uint4 *&S2p) {
        if (resident) {
            S1p = &sstate[(k * 2) * SCAN_THREADS + tid];
            S2p = &sstate[(k * 2 + 1) * SCAN_THREADS + tid];
        } else {
            const long sidx = (long)tile * SCAN_THREADS + tid;
            S1p = reinterpret_cast<uint4 *>(a.S1) + sidx;
            S2p = reinterpret_cast<uint4 *>(a.S2) + sidx;
        }
    };

    // fold frame t into S1/S2 of one tile (restart when `fresh`) and add its
    // floor(sqrt(65536 (n S2 - S1^2))) over the valid pixels to acc
    auto fold = [&](int t, int k, int tile, bool fresh, int n1, unsigned long long &acc) {
        const TileCtx c = ctx(k);
        uint4 *S1p, *S2p;
        state_ptrs(k, tile, S1p, S2p);
        const uint2 e = ering[(long)(t % SCAN_FW) * eslot + (long)tile * SCAN_THREADS + tid];
        const uint32_t ev[4] = {e.x & 0xFFFFu, e.y & 0xFFFFu, e.x >> 16, e.y >> 16};
        uint4 s1 = make_uint4(0, 0, 0, 0), s2 = make_uint4(0, 0, 0, 0);
        if (!fresh) {
            s1 = *S1p;
            s2 = *S2p;
        }
        uint32_t *S1v = &s1.x, *S2v = &s2.x;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            S1v[v] += ev[v];
            S2v[v] += ev[v] * ev[v];
            if (v < c.nvalid) {
                const unsigned long long Q =
                    (unsigned long long)n1 * S2v[v] - (unsigned long long)S1v[v] * S1v[v];
                acc += isqrt53(Q << 16);
            }
        }
        *S1p = s1;
        *S2p = s2;
    };

    // block sum of acc and maximum of emax2 (thread 0 receives them)
    auto block_reduce = [&](unsigned long long &acc, uint32_t &em) {
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
            acc = A;
            em = m;
        }
        __syncthreads();
    };

    // summed energy of buffer bi (the E0 plane) for the valid pixels of my tiles:
    // S1 minus the ring energies of frames [g0, g1)
    auto write_e0 = [&](int bi, int g0, int g1) {
        if (!a.E0 || bi >= a.nbcap) return;
        for (int k = 0; k < mine; ++k) {
            const int tile = first + k;
            const TileCtx c = ctx(k);
            if (c.nvalid == 0) continue;
            uint4 *S1p, *S2p;
            state_ptrs(k, tile, S1p, S2p);
            uint4 s1 = *S1p;
            uint32_t *S1v = &s1.x;
            for (int g = g0; g < g1; ++g) {
                const uint2 e = ering[(long)(g % SCAN_FW) * eslot + (long)tile * SCAN_THREADS + tid];
                S1v[0] -= e.x & 0xFFFFu;
                S1v[1] -= e.y & 0xFFFFu;
                S1v[2] -= e.x >> 16;
                S1v[3] -= e.y >> 16;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (v < c.nvalid)
                    a.E0[(long)bi * a.e0_plane + (long)c.row * a.W + c.col + v] = (int32_t)S1v[v];
        }
    };

    int t = 0, horizon = 0, r = 0;
    while (t < a.T) {
        // the round's frames: up to SCAN_FW, ending where the open buffer
        // would reach t_max, and at the clip end
        const int n0 = st.n;
        int w = min(t + SCAN_FW - 1, a.T - 1);
        w = min(w, t + (a.t_max - n0) - 1);
        for (int f = t; f <= w; ++f) {
            uint32_t emax2 = 0;
            const bool fresh_frame = f >= horizon;
            if (fresh_frame && a.ready) {
                // frame f may still be on its way from the host: wait (bounded)
                // until the copy stream has raised the counter past its chunk
                if (tid == 0) {
                    const unsigned need = (unsigned)(f / a.ready_frames) + 1u;
                    int ok = 1;
                    if (ld_acquire_u32(a.ready) < need) {
                        const unsigned long long t0 = globaltimer_ns();
                        while (ld_acquire_u32(a.ready) < need) {
                            if (*(volatile int *)a.err != DEV_OK) { ok = 0; break; }
                            if (globaltimer_ns() - t0 > a.spin_limit_ns) {
                                atomicCAS(a.err, DEV_OK, DEV_ETIMEOUT);
                                ok = 0;
                                break;
                            }
                            __nanosleep(256);
                        }
                    }
                    s_ok = ok;
                }
                __syncthreads();
                if (!s_ok) return;
            }
            if (fresh_frame) {
                if (resident) {
#pragma unroll
                    for (int k = 0; k < MAXT; ++k)
                        if (k < mine) phase_a(f, k, yp[k], emax2);
                } else {
                    for (int k = 0; k < mine; ++k) {
                        uint32_t ydummy = 0;
                        phase_a(f, k, ydummy, emax2);
                    }
                }
            }
            unsigned long long acc = 0;
            const bool fresh = n0 == 0 && f == t;   // the open buffer starts here
            const int n1 = n0 + (f - t) + 1;
            if (resident) {
#pragma unroll
                for (int k = 0; k < MAXT; ++k)
                    if (k < mine) fold(f, k, first + k, fresh, n1, acc);
            } else {
                for (int k = 0; k < mine; ++k) fold(f, k, first + k, fresh, n1, acc);
            }
            uint32_t em = max(emax2 & 0xFFFFu, emax2 >> 16);
            block_reduce(acc, em);
            if (tid == 0) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.partA[(long)r * SCAN_FW + (f - t)]),
                          acc);
                if (fresh_frame) atomicMax(&a.partM[f], (int)em);
            }
        }
        horizon = max(horizon, w + 1);
        // publish the round, wait for the clip's other CTAs, replay decisions
        if (tid == 0) {
            __threadfence();
            atomicAdd(&a.count[r], 1u);
            int ok = wait_round(a, r, G) ? 1 : 0;
            int ndec = 0, last = DEC_JOIN;
            if (ok) {
                __threadfence();
                const bool lead = lb == 0;
                for (int f = t; f <= w; ++f) {
                    const long long A = (long long)__ldcg(reinterpret_cast<const unsigned long long *>(
                        &a.partA[(long)r * SCAN_FW + (f - t)]));
                    const int m = __ldcg(&a.partM[f]);
                    if (lead && a.A_out) {
                        a.A_out[f] = A;
                        a.M_out[f] = m;
                    }
                    last = decide(st, A, m, f, a, lead);
                    ++ndec;
                    if (last == DEC_FLUSH) break;
                }
            }
            s_ok = ok;
            s_ndec = ndec;
            s_last = last;
        }
        __syncthreads();
        if (!s_ok) return;
        const int fend = t + s_ndec;   // first frame not yet decided
        if (s_last == DEC_FLUSH) {
            // frame fend-1 starts a new buffer: the closed one is S1 minus the
            // energies of frames fend-1..w; S1/S2 restart from e_{fend-1}
            const int f = fend - 1;
            write_e0(st.nb - 1, f, w + 1);
            for (int k = 0; k < mine; ++k) {
                const int tile = first + k;
                uint4 *S1p, *S2p;
                state_ptrs(k, tile, S1p, S2p);
                const uint2 e = ering[(long)(f % SCAN_FW) * eslot + (long)tile * SCAN_THREADS + tid];
                const uint32_t ev[4] = {e.x & 0xFFFFu, e.y & 0xFFFFu, e.x >> 16, e.y >> 16};
                *S1p = make_uint4(ev[0], ev[1], ev[2], ev[3]);
                *S2p = make_uint4(ev[0] * ev[0], ev[1] * ev[1], ev[2] * ev[2], ev[3] * ev[3]);
            }
        } else if (s_last == DEC_CLOSE) {
            write_e0(st.nb - 1, w + 1, w + 1);   // the buffer ending with frame w
        }
        __syncthreads();
        t = fend;
        ++r;
    }
    // the buffer still open at the clip end
    if (st.n > 0) write_e0(st.nb, a.T, a.T);
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
