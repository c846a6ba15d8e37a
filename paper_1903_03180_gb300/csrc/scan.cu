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
#include <algorithm>

#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int TR = 8, TC = 128, SCAN_THREADS = 256;
constexpr int LUMW = TC + 8;   // luma tile row: TC + 2 columns, padded to whole words
enum { DEC_JOIN = 0, DEC_FLUSH = 1, DEC_CLOSE = 2, DEC_UNSURE = 3 };

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
// The threshold of Eq. 9 for a buffer of n1 frames with maxval M1, scaled:
// 256*alpha*M1*sqrt(n1-1)*H*W, products left to right.
__device__ double threshold(const ScanArgs &a, long long M1, int n1) {
    double thr = __dmul_rn(256.0, a.alpha);
    thr = __dmul_rn(thr, __ll2double_rn(M1));
    thr = __dmul_rn(thr, __dsqrt_rn(__int2double_rn(n1 - 1)));
    thr = __dmul_rn(thr, __int2double_rn(a.H));
    thr = __dmul_rn(thr, __int2double_rn(a.W));
    return thr;
}

// maxval of the open buffer once frame t (maximum emax) joins it
__device__ long long next_maxval(const DecState &s, long long emax, const ScanArgs &a) {
    return a.maxval_mode == 1 ? a.maxval_theory : (emax > s.M ? emax : s.M);
}

__device__ int decide(DecState &s, long long A, long long emax, int t, const ScanArgs &a,
                      bool write) {
    int n1 = s.n + 1;
    long long M1 = next_maxval(s, emax, a);
    bool exceeds = false;
    if (n1 >= 2) exceeds = __ll2double_rn(A) > threshold(a, M1, n1);
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
    const float d = __fdividef(__ll2float_rz(R), 2.0f * fmaxf(r0f, 1.0f));   // approximate
    uint32_t r = r0 + (uint32_t)__float2int_rd(d);
    r -= ((unsigned long long)r * r > x) ? 1u : 0u;
    r += ((unsigned long long)(r + 1) * (r + 1) <= x) ? 1u : 0u;
    return r;
}

// Packed u16x2 helpers for the 4 pixels of a thread: lane 0 = pixels 0 and 2,
// lane 1 = pixels 1 and 3 of a luma quad.
__device__ __forceinline__ uint32_t even16(uint32_t q) { return __byte_perm(q, 0, 0x4240); }
__device__ __forceinline__ uint32_t odd16(uint32_t q) { return __byte_perm(q, 0, 0x4341); }
// |x - y| and max(x, y, z) per 16-bit lane with the DPX three-way max/min (the
// per-lane difference max - min is never negative, so no borrow crosses lanes)
__device__ __forceinline__ uint32_t absdiff16(uint32_t x, uint32_t y) {
    return __vimax3_u16x2(x, y, 0u) - __vimin3_u16x2(x, y, 0xFFFFFFFFu);
}
__device__ __forceinline__ uint32_t max16(uint32_t x, uint32_t y, uint32_t z) {
    return __vimax3_u16x2(x, y, z);
}

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

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
    g02 = absdiff16(rE, lE) + absdiff16(bE, tE);
    const uint32_t lO = odd16(uL) + 2 * odd16(mL) + odd16(dL);
    const uint32_t rO = odd16(uR) + 2 * odd16(mR) + odd16(dR);
    const uint32_t tO = odd16(uL) + 2 * odd16(uC) + odd16(uR);
    const uint32_t bO = odd16(dL) + 2 * odd16(dC) + odd16(dR);
    g13 = absdiff16(rO, lO) + absdiff16(bO, tO);
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

__device__ __forceinline__ TileCtx tile_ctx(int H, int W, int tile, int tiles_x, int tid) {
    TileCtx c;
    const int ty = tile / tiles_x;
    c.r0 = ty * TR;
    c.c0 = (tile - ty * tiles_x) * TC;
    c.row = c.r0 + (tid >> 5);
    c.col = c.c0 + 4 * (tid & 31);
    c.nvalid = c.row < H ? max(0, min(4, W - c.col)) : 0;
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
__device__ __forceinline__ void load_luma(int H, int W, bool words, const uint8_t *f, int r0,
                                          int c0, uint8_t (*lum)[LUMW]) {
    const int tid = threadIdx.x;
    if (words) {
        // body and top/bottom frame rows: (TR + 2) rows x 32 quads
        for (int q = tid; q < (TR + 2) * 32; q += SCAN_THREADS) {
            const int r = q >> 5, x = q & 31;
            const int gi = clampi(r0 + r - 1, 0, H - 1);
            const int gj = c0 + 4 * x;
            uint32_t y = 0;
            if (gj < W) {
                const uint32_t *w =
                    reinterpret_cast<const uint32_t *>(f + ((long)gi * W + gj) * 3);
                y = luma4(__ldg(w), __ldg(w + 1), __ldg(w + 2));
            } else {   // past the right edge: replicate the last column
                y = luma_px(f + ((long)gi * W + W - 1) * 3) * 0x01010101u;
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
            const int gi = clampi(r0 + r - 1, 0, H - 1);
            const int gj = clampi(side ? c0 + TC : c0 - 1, 0, W - 1);
            lum[r][side ? TC + 1 : 0] = (uint8_t)luma_px(f + ((long)gi * W + gj) * 3);
        }
    } else {
        for (int q = tid; q < (TR + 2) * (TC + 2); q += SCAN_THREADS) {
            const int r = q / (TC + 2), c = q - r * (TC + 2);
            const int gi = clampi(r0 + r - 1, 0, H - 1), gj = clampi(c0 + c - 1, 0, W - 1);
            lum[r][c] = (uint8_t)luma_px(f + ((long)gi * W + gj) * 3);
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
    // the clip's arguments live in shared memory; the hot loops use register
    // copies (shared loads there could not be hoisted past the tile stores)
    const int H = a.H, W = a.W, T = a.T;
    const uint32_t wg = (uint32_t)a.wg, wm = (uint32_t)a.wm;
    const long ypitch = a.ypitch;
    const uint8_t *__restrict__ rgb = a.rgb;
    uint8_t *__restrict__ Yo = a.Y;
    uint8_t *__restrict__ Do = a.D;
    uint32_t *S1g = a.S1, *S2g = a.S2;
    int32_t *E0 = a.E0;
    const int nbcap = a.nbcap;
    const long e0_plane = a.e0_plane;
    const unsigned *ready = a.ready;
    const int ready_frames = a.ready_frames;
    const uint8_t *__restrict__ Yprev = a.Yprev;
    const bool words = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(rgb) & 3) == 0;
    const int G = a.G;
    const int lb = blockIdx.x - a.cta0;   // CTA index within the clip's range
    const int tiles_x = (W + TC - 1) / TC;
    const int ntiles = ((H + TR - 1) / TR) * tiles_x;
    const int tpc = (ntiles + G - 1) / G;
    const int first = lb * tpc;
    const int mine = max(0, min(tpc, ntiles - first));
    const bool resident = tpc <= MAXT;
    const long hw3 = (long)H * W * 3;
    const long yplane = (long)H * ypitch;
    const bool pf_ok = (reinterpret_cast<uintptr_t>(rgb) & 15) == 0;   // prefetch needs 16-byte bases
    const long eslot = (long)ntiles * SCAN_THREADS;   // uint2 entries per ring slot
    uint2 *ering = reinterpret_cast<uint2 *>(a.ering);  // [SCAN_FW][ntiles][256] e quads
    for (int k = tid; k < min(mine, 64); k += SCAN_THREADS) {
        const int ty = (first + k) / tiles_x;
        s_rc[k] = ((uint32_t)(ty * TR) << 16) | (uint32_t)((first + k - ty * tiles_x) * TC);
    }
    __syncthreads();
    // the geometry of the CTA's k-th tile for this thread
    auto ctx = [&](int k) {
        if (k >= 64) return tile_ctx(H, W, first + k, tiles_x, tid);
        TileCtx c;
        c.r0 = (int)(s_rc[k] >> 16);
        c.c0 = (int)(s_rc[k] & 0xFFFFu);
        c.row = c.r0 + (tid >> 5);
        c.col = c.c0 + 4 * (tid & 31);
        c.nvalid = c.row < H ? max(0, min(4, W - c.col)) : 0;
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
        const uint8_t *f = rgb + (long)t * hw3;
        // the tile's rows of the next frame into L2 now, so that its loads
        // wait for L2 instead of DRAM; ranges rounded inwards to 16 bytes
        // and kept inside the clip
        if (pf_ok && tid < TR + 2 && t + 1 < T) {
            const int row = clampi(c.r0 - 1 + tid, 0, H - 1);
            const long base = ((long)(t + 1) * H + row) * W * 3;
            const long lo = (base + 3L * max(c.c0 - 1, 0)) & ~15L;
            const long hi = (base + 3L * min(c.c0 + TC + 1, W)) & ~15L;
            if (hi > lo) prefetch_l2(rgb + lo, (unsigned)(hi - lo));
        }
        load_luma(H, W, words, f, c.r0, c.c0, lum);
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
            yprv = *reinterpret_cast<const uint32_t *>(Yo + (long)(t - 1) * yplane +
                                                       (long)c.row * ypitch + c.col);
        if (t == 0 && Yprev && c.nvalid > 0)
            yprv = *reinterpret_cast<const uint32_t *>(Yprev + (long)c.row * ypitch + c.col);
        // motion |Y_t - Y_{t-1}| on the u16 halves the energy uses
        const bool moves = t > 0 || Yprev;
        const uint32_t d02 = moves ? absdiff16(even16(ycur), even16(yprv)) : 0u;
        const uint32_t d13 = moves ? absdiff16(odd16(ycur), odd16(yprv)) : 0u;
        const uint32_t dq = __byte_perm(d02, d13, 0x6240);   // back to 4 bytes
        const uint32_t e02 = wg * g02 + wm * d02;
        const uint32_t e13 = wg * g13 + wm * d13;
        if (c.nvalid > 0) {
            // invalid pixels of a ragged quad do not count towards the maximum
            const uint32_t m02 = c.nvalid >= 3 ? e02 : (e02 & 0xFFFFu);
            const uint32_t m13 = c.nvalid >= 4 ? e13 : (c.nvalid >= 2 ? (e13 & 0xFFFFu) : 0u);
            emax2 = max16(emax2, m02, m13);
            const long yo = (long)t * yplane + (long)c.row * ypitch + c.col;
            *reinterpret_cast<uint32_t *>(Yo + yo) = ycur;
            *reinterpret_cast<uint32_t *>(Do + yo) = dq;
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
            S1p = reinterpret_cast<uint4 *>(S1g) + sidx;
            S2p = reinterpret_cast<uint4 *>(S2g) + sidx;
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
        if (!E0 || bi >= nbcap) return;
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
                    E0[(long)bi * e0_plane + (long)c.row * W + c.col + v] = (int32_t)S1v[v];
        }
    };

    int t = 0, horizon = 0, r = 0;
    while (t < T) {
        // the round's frames: up to SCAN_FW, ending where the open buffer
        // would reach t_max, and at the clip end
        const int n0 = st.n;
        int w = min(t + SCAN_FW - 1, T - 1);
        w = min(w, t + (a.t_max - n0) - 1);
        for (int f = t; f <= w; ++f) {
            uint32_t emax2 = 0;
            const bool fresh_frame = f >= horizon;
            if (fresh_frame && ready) {
                // frame f may still be on its way from the host: wait (bounded)
                // until the copy stream has raised the counter past its chunk
                if (tid == 0) {
                    const unsigned need = (unsigned)(f / ready_frames) + 1u;
                    int ok = 1;
                    if (ld_acquire_u32(ready) < need) {
                        const unsigned long long t0 = globaltimer_ns();
                        while (ld_acquire_u32(ready) < need) {
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
    if (st.n > 0) write_e0(st.nb, T, T);
    if (lb == 0 && tid == 0) {
        int nb = st.nb;
        if (st.n > 0) a.starts[nb++] = st.start;
        a.starts[nb] = T;
        *a.n_buffers = nb;
    }
}

// ---------------------------------------------------------------------------
// k_scan_wt, the warp-tile variant for one clip whose state stays on chip.
// Tile ownership: a tile is WT_TR rows x 128 columns and belongs to one warp for
// the whole clip; lane l holds columns 4l .. 4l+3 of every row of it.  Warp gw
// of a clip (CTA lb, warp w: gw = lb * WT_WARPS + w) owns the tiles
// [gw * tpw, (gw + 1) * tpw), tpw = ceil(tiles / warps).  With one tile a warp
// the running sums S1, S2 of its pixels stay in shared memory and the previous
// frame's luma in registers ("resident"); with more they live in global memory.
// Tiles of 6 rows: at 1080p that is 2700 tiles, so that 675 of the 760
// co-resident CTAs have work (8-row tiles left a third of them idle) and each
// warp's chain of rows per frame is a quarter shorter.
constexpr int WT_TR = 6;
constexpr int WT_THREADS = 128;
constexpr int WT_WARPS = WT_THREADS / 32;
constexpr size_t WT_SMEM = (size_t)WT_WARPS * WT_TR * 2 * 32 * sizeof(uint4);   // 24 KB

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
__global__ void __launch_bounds__(WT_THREADS, 5)
k_scan_wt(ScanArgs a0, const ScanArgs *__restrict__ tab, const int *__restrict__ block_clip) {
    extern __shared__ __align__(16) uint4 sstate[];   // [WT_WARPS][WT_TR][2][32] S1, S2
    __shared__ ScanArgs a;
    __shared__ unsigned long long red_a[SCAN_FW][WT_WARPS];   // per frame of the round
    __shared__ double red_f[SCAN_FW][WT_WARPS];               // (bounded rounds)
    __shared__ uint32_t red_m[SCAN_FW][WT_WARPS];
    __shared__ int s_exact;   // this round sums the exact floor(sqrt) (else a bounded float)
    __shared__ DecState st;
    __shared__ int s_ok, s_ndec, s_last;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        if (tab) {
            a = tab[block_clip[blockIdx.x]];
        } else {
            a = a0;
            a.cta0 = 0;
            a.G = gridDim.x;
        }
        st.n = 0; st.M = 0; st.start = 0; st.nb = 0;
        s_exact = a.A_out != nullptr;   // the diagnostics report every exact A_t
    }
    __syncthreads();
    // the clip's arguments live in shared memory; the hot loops use register
    // copies (shared loads there could not be hoisted past the state stores)
    const int H = a.H, W = a.W, T = a.T;
    const uint32_t wg = (uint32_t)a.wg, wm = (uint32_t)a.wm;
    const long ypitch = a.ypitch;
    const uint8_t *__restrict__ rgb = a.rgb;
    uint8_t *__restrict__ Yo = a.Y;
    uint8_t *__restrict__ Do = a.D;
    uint32_t *S1g = a.S1, *S2g = a.S2;
    int32_t *E0 = a.E0;
    const int nbcap = a.nbcap;
    const long e0_plane = a.e0_plane;
    const unsigned *ready = a.ready;
    const int ready_frames = a.ready_frames;
    const uint8_t *__restrict__ Yprev = a.Yprev;
    const int G = a.G;
    const int lb = blockIdx.x - a.cta0;   // CTA index within the clip's range
    const int tiles_x = (W + TC - 1) / TC;
    const int ntiles = ((H + WT_TR - 1) / WT_TR) * tiles_x;
    const int nwarps = G * WT_WARPS;
    const int tpw = (ntiles + nwarps - 1) / nwarps;
    const int gw = lb * WT_WARPS + w;
    const int first = gw * tpw;
    const int mine = max(0, min(tpw, ntiles - first));
    const bool resident = tpw <= 1;
    const bool words = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(rgb) & 3) == 0;
    const bool pf_ok = (reinterpret_cast<uintptr_t>(rgb) & 15) == 0;   // prefetch needs 16-byte bases
    const long hw3 = (long)H * W * 3;
    const long yplane = (long)H * ypitch;
    const long eslot = (long)ntiles * WT_TR * 32;           // uint2 entries per ring slot
    uint2 *ering = reinterpret_cast<uint2 *>(a.ering);  // [SCAN_FW][ntiles][WT_TR][32] e quads
    uint32_t yp[WT_TR];   // resident path: previous frame's luma quad of every row
#pragma unroll
    for (int r = 0; r < WT_TR; ++r) yp[r] = 0;

    auto state_ptrs = [&](int tile, int r, uint4 *&S1p, uint4 *&S2p) {
        if (resident) {
            S1p = &sstate[((w * WT_TR + r) * 2) * 32 + lane];
            S2p = &sstate[((w * WT_TR + r) * 2 + 1) * 32 + lane];
        } else {
            const long sidx = ((long)tile * WT_TR + r) * 32 + lane;
            S1p = reinterpret_cast<uint4 *>(S1g) + sidx;
            S2p = reinterpret_cast<uint4 *>(S2g) + sidx;
        }
    };
    auto ering_at = [&](int f, int tile, int r) -> uint2 & {
        return ering[(long)(f % SCAN_FW) * eslot + ((long)tile * WT_TR + r) * 32 + lane];
    };

    // fold one row's energy quad into S1/S2 (restart when `fresh`) and add
    // floor(sqrt(65536 (n S2 - S1^2))) of its valid pixels to acc
    // exact: acc += floor(sqrt(65536 Q)) per pixel, the integers Eq. 7-8 define;
    // otherwise accf += sqrt(Q) in single precision, an estimate whose error is
    // bounded (see the decisions below)
    auto fold = [&](int tile, int r, uint32_t e02, uint32_t e13, int nv, bool fresh, int n1,
                    bool exact, unsigned long long &acc, float &accf) {
        uint4 *S1p, *S2p;
        state_ptrs(tile, r, S1p, S2p);
        const uint32_t ev[4] = {e02 & 0xFFFFu, e13 & 0xFFFFu, e02 >> 16, e13 >> 16};
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
            if (v < nv) {
                const unsigned long long Q =
                    (unsigned long long)n1 * S2v[v] - (unsigned long long)S1v[v] * S1v[v];
                if (exact) {
                    acc += isqrt53(Q << 16);
                } else {
                    const float qf = __ull2float_rz(Q);
                    accf += qf > 0.0f ? qf * rsqrtf(qf) : 0.0f;
                }
            }
        }
        *S1p = s1;
        *S2p = s2;
    };

    // frame f on one tile: (fresh_frame) the energy of every row from the RGB
    // frame, luma and motion written out, the energy kept in the ring; then
    // every row folded into the running sums.  Rows are software-pipelined:
    // the raw bytes of row i+2 are loaded while row i is computed.
    auto tile_frame = [&](int f, int tile, bool fresh_frame, bool fresh, int n1, bool exact,
                          unsigned long long &acc, float &accf, uint32_t &emax2) {
        const int ty = tile / tiles_x;
        const int r0 = ty * WT_TR, c0 = (tile - ty * tiles_x) * TC;
        const int col = c0 + 4 * lane;
        const int nvq = max(0, min(4, W - col));
        if (!fresh_frame) {
#pragma unroll
            for (int r = 0; r < WT_TR; ++r) {
                const int nv = r0 + r < H ? nvq : 0;
                const uint2 e = ering_at(f, tile, r);
                fold(tile, r, e.x, e.y, nv, fresh, n1, exact, acc, accf);
            }
            return;
        }
        const uint8_t *fr = rgb + (long)f * hw3;
        // the tile's rows of the next frame into L2 now, so that its loads
        // wait for L2 instead of DRAM; ranges rounded inwards to 16 bytes
        // and kept inside the clip
        if (pf_ok && lane < WT_TR + 2 && f + 1 < T) {
            const int row = clampi(r0 - 1 + lane, 0, H - 1);
            const long base = ((long)(f + 1) * H + row) * W * 3;
            const long lo = (base + 3L * max(c0 - 1, 0)) & ~15L;
            const long hi = (base + 3L * min(c0 + TC + 1, W)) & ~15L;
            if (hi > lo) prefetch_l2(rgb + lo, (unsigned)(hi - lo));
        }
        const bool fastq = words && col + 3 < W;
        const int ecol = lane == 0 ? max(c0 - 1, 0) : min(c0 + TC, W - 1);
        // raw bytes of one row: the quad's 3 RGB words (or, off the fast path,
        // its luma already packed in w0) and the edge pixel of lanes 0 and 31
        struct Raw { uint32_t w0, w1, w2, e0, e1, e2; };
        auto fetch = [&](int row) {
            Raw x;
            const uint8_t *rp = fr + (long)clampi(row, 0, H - 1) * W * 3;
            if (fastq) {
                const uint32_t *w = reinterpret_cast<const uint32_t *>(rp + col * 3);
                x.w0 = __ldg(w);
                x.w1 = __ldg(w + 1);
                x.w2 = __ldg(w + 2);
            } else {
                x.w0 = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    x.w0 |= (uint32_t)luma_px(rp + min(col + j, W - 1) * 3) << (8 * j);
                x.w1 = x.w2 = 0;
            }
            x.e0 = x.e1 = x.e2 = 0;
            if (lane == 0 || lane == 31) {
                const uint8_t *ep = rp + ecol * 3;
                x.e0 = __ldg(ep);
                x.e1 = __ldg(ep + 1);
                x.e2 = __ldg(ep + 2);
            }
            return x;
        };
        // luma quad and its 8-byte window from raw bytes (shuffles: all lanes)
        auto window = [&](const Raw &x, uint32_t &q, uint32_t &u0, uint32_t &u1) {
            q = fastq ? luma4(x.w0, x.w1, x.w2) : x.w0;
            const uint32_t ey = (77u * x.e0 + 150u * x.e1 + 29u * x.e2 + 128u) >> 8;
            uint32_t lq = __shfl_up_sync(0xffffffffu, q, 1);
            uint32_t rq = __shfl_down_sync(0xffffffffu, q, 1);
            if (lane == 0) lq = ey << 24;
            if (lane == 31) rq = ey;
            u0 = __byte_perm(lq, q, 0x6543);
            u1 = __byte_perm(q, rq, 0x0043);
        };
        uint32_t qa, qb, a0, a1, b0, b1;
        {
            const Raw xa = fetch(r0 - 1), xb = fetch(r0);
            Raw xc = fetch(r0 + 1);
            window(xa, qa, a0, a1);
            window(xb, qb, b0, b1);
#pragma unroll
            for (int r = 0; r < WT_TR; ++r) {
                const int i = r0 + r;
                const Raw xn = fetch(i + 2);   // two rows ahead
                uint32_t qc, c0w, c1w;
                window(xc, qc, c0w, c1w);
                uint32_t g02, g13;
                sobel4(a0, a1, b0, b1, c0w, c1w, g02, g13);
                uint32_t yprv = yp[r];
                const int nv = i < H ? nvq : 0;
                if (!resident && f > 0 && nv > 0)
                    yprv = *reinterpret_cast<const uint32_t *>(Yo + (long)(f - 1) * yplane +
                                                               (long)i * ypitch + col);
                if (f == 0 && Yprev && nv > 0)
                    yprv = *reinterpret_cast<const uint32_t *>(Yprev + (long)i * ypitch + col);
                // motion |Y_t - Y_{t-1}| on the u16 halves the energy uses
                const bool moves = f > 0 || Yprev;
                const uint32_t d02 = moves ? absdiff16(even16(qb), even16(yprv)) : 0u;
                const uint32_t d13 = moves ? absdiff16(odd16(qb), odd16(yprv)) : 0u;
                const uint32_t dq = __byte_perm(d02, d13, 0x6240);   // back to 4 bytes
                const uint32_t e02 = wg * g02 + wm * d02;
                const uint32_t e13 = wg * g13 + wm * d13;
                if (nv > 0) {
                    // invalid pixels of a ragged quad do not count towards the maximum
                    const uint32_t m02 = nv >= 3 ? e02 : (e02 & 0xFFFFu);
                    const uint32_t m13 = nv >= 4 ? e13 : (nv >= 2 ? (e13 & 0xFFFFu) : 0u);
                    emax2 = max16(emax2, m02, m13);
                    const long yo = (long)f * yplane + (long)i * ypitch + col;
                    *reinterpret_cast<uint32_t *>(Yo + yo) = qb;
                    *reinterpret_cast<uint32_t *>(Do + yo) = dq;
                }
                ering_at(f, tile, r) = make_uint2(e02, e13);
                yp[r] = qb;
                fold(tile, r, e02, e13, nv, fresh, n1, exact, acc, accf);
                a0 = b0; a1 = b1; b0 = c0w; b1 = c1w; qb = qc;
                xc = xn;
            }
        }
    };

    // warp sum of acc and maximum of em into the round's slot i of this warp
    // (thread 0 adds the warps up once the round's frames are done)
    auto warp_reduce = [&](int i, bool exact, unsigned long long acc, float accf, uint32_t em) {
        double accd = accf;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (exact) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            else accd += __shfl_xor_sync(0xffffffffu, accd, o);
            em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        }
        if (lane == 0) {
            red_a[i][w] = acc;
            red_f[i][w] = accd;
            red_m[i][w] = em;
        }
    };

    // summed energy of buffer bi (the E0 plane) for the valid pixels of my tiles:
    // S1 minus the ring energies of frames [g0, g1)
    auto write_e0 = [&](int bi, int g0, int g1) {
        if (!E0 || bi >= nbcap) return;
        for (int k = 0; k < mine; ++k) {
            const int tile = first + k;
            const int ty = tile / tiles_x;
            const int r0 = ty * WT_TR, col = (tile - ty * tiles_x) * TC + 4 * lane;
            const int nvq = max(0, min(4, W - col));
            for (int r = 0; r < WT_TR; ++r) {
                if (r0 + r >= H || nvq == 0) continue;
                uint4 *S1p, *S2p;
                state_ptrs(tile, r, S1p, S2p);
                uint4 s1 = *S1p;
                uint32_t *S1v = &s1.x;
                for (int g = g0; g < g1; ++g) {
                    const uint2 e = ering_at(g, tile, r);
                    S1v[0] -= e.x & 0xFFFFu;
                    S1v[1] -= e.y & 0xFFFFu;
                    S1v[2] -= e.x >> 16;
                    S1v[3] -= e.y >> 16;
                }
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (v < nvq)
                        E0[(long)bi * e0_plane + (long)(r0 + r) * W + col + v] =
                            (int32_t)S1v[v];
            }
        }
    };

    int t = 0, horizon = 0, rnd = 0;
    while (t < T) {
        // the round's frames: up to SCAN_FW, ending where the open buffer
        // would reach t_max, and at the clip end
        const int n0 = st.n;
        const bool exact = s_exact;
        int wend = min(t + SCAN_FW - 1, T - 1);
        wend = min(wend, t + (a.t_max - n0) - 1);
        for (int f = t; f <= wend; ++f) {
            const bool fresh_frame = f >= horizon;
            if (fresh_frame && ready) {
                // frame f may still be on its way from the host: wait (bounded)
                // until the copy stream has raised the counter past its chunk
                if (tid == 0) {
                    const unsigned need = (unsigned)(f / ready_frames) + 1u;
                    int ok = 1;
                    if (ld_acquire_u32(ready) < need) {
                        const unsigned long long t0 = globaltimer_ns();
                        while (ld_acquire_u32(ready) < need) {
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
            unsigned long long acc = 0;
            float accf = 0.0f;
            uint32_t emax2 = 0;
            const bool fresh = n0 == 0 && f == t;   // the open buffer starts here
            const int n1 = n0 + (f - t) + 1;
            for (int k = 0; k < mine; ++k)
                tile_frame(f, first + k, fresh_frame, fresh, n1, exact, acc, accf, emax2);
            warp_reduce(f - t, exact, acc, accf, max(emax2 & 0xFFFFu, emax2 >> 16));
        }
        // the CTA's share of every frame of the round: one barrier per round
        __syncthreads();
        if (tid == 0) {
            for (int f = t; f <= wend; ++f) {
                unsigned long long A = 0;
                double Af = 0.0;
                uint32_t m = 0;
                for (int q = 0; q < WT_WARPS; ++q) {
                    A += red_a[f - t][q];
                    Af += red_f[f - t][q];
                    m = max(m, red_m[f - t][q]);
                }
                long long *slot = &a.partA[(long)rnd * SCAN_FW + (f - t)];
                if (exact)
                    atomicAdd(reinterpret_cast<unsigned long long *>(slot), A);
                else   // the slot (zeroed) holds a double in a bounded round
                    atomicAdd(reinterpret_cast<double *>(slot), Af);
                if (f >= horizon) atomicMax(&a.partM[f], (int)m);
            }
        }
        horizon = max(horizon, wend + 1);
        // publish the round, wait for the clip's other CTAs, replay decisions
        if (tid == 0) {
            __threadfence();
            atomicAdd(&a.count[rnd], 1u);
            int ok = wait_round(a, rnd, G) ? 1 : 0;
            int ndec = 0, last = DEC_JOIN;
            if (ok) {
                __threadfence();
                const bool lead = lb == 0;
                for (int f = t; f <= wend; ++f) {
                    const long long *slot = &a.partA[(long)rnd * SCAN_FW + (f - t)];
                    const int m = __ldcg(&a.partM[f]);
                    long long A;
                    if (exact) {
                        A = (long long)__ldcg(reinterpret_cast<const unsigned long long *>(slot));
                        if (lead && a.A_out) {
                            a.A_out[f] = A;
                            a.M_out[f] = m;
                        }
                    } else {
                        // S = 256 sum sqrt(Q) in floats: each sqrt within 2^-21.4 of
                        // its value, a thread's sum of at most 24 of them within
                        // 2^-19.5, the double sums beyond that within 2^-32.  So
                        // the exact A = sum floor(256 sqrt(Q)) lies in
                        // [S (1 - e) - H W, S (1 + e)] with e = 2^-16 (about
                        // 6x the bound).  A threshold outside that range is
                        // decided as the exact A would decide it; one inside it
                        // sends the frame back to be summed exactly.
                        const double S = 256.0 * __ldcg(reinterpret_cast<const double *>(slot));
                        constexpr double EPS = 1.52587890625e-05;   // 2^-16
                        A = 0;
                        const int n1 = st.n + 1;
                        if (n1 >= 2) {
                            const double thr = threshold(a, next_maxval(st, m, a), n1);
                            const double lo = S * (1.0 - EPS) - (double)a.H * (double)a.W;
                            const double hi = S * (1.0 + EPS);
                            if (lo > thr) {
                                A = 0x7FFFFFFFFFFFFFFFll;   // certainly above the threshold
                            } else if (!(hi <= thr)) {
                                last = DEC_UNSURE;
                                break;
                            }
                        }
                    }
                    last = decide(st, A, m, f, a, lead);
                    ++ndec;
                    if (last == DEC_FLUSH) break;
                }
            }
            s_ok = ok;
            s_ndec = ndec;
            s_last = last;
            // a frame too close to call is summed exactly in the next round
            s_exact = last == DEC_UNSURE || a.A_out != nullptr;
        }
        __syncthreads();
        if (!s_ok) return;
        const int fend = t + s_ndec;   // first frame not yet decided
        if (s_last == DEC_FLUSH) {
            // frame fend-1 starts a new buffer: the closed one is S1 minus the
            // energies of frames fend-1..wend; S1/S2 restart from e_{fend-1}
            const int f = fend - 1;
            write_e0(st.nb - 1, f, wend + 1);
            for (int k = 0; k < mine; ++k) {
                const int tile = first + k;
                for (int r = 0; r < WT_TR; ++r) {
                    uint4 *S1p, *S2p;
                    state_ptrs(tile, r, S1p, S2p);
                    const uint2 e = ering_at(f, tile, r);
                    const uint32_t ev[4] = {e.x & 0xFFFFu, e.y & 0xFFFFu, e.x >> 16, e.y >> 16};
                    *S1p = make_uint4(ev[0], ev[1], ev[2], ev[3]);
                    *S2p = make_uint4(ev[0] * ev[0], ev[1] * ev[1], ev[2] * ev[2], ev[3] * ev[3]);
                }
            }
        } else if (s_last == DEC_CLOSE) {
            write_e0(st.nb - 1, wend + 1, wend + 1);   // the buffer ending with frame wend
        } else if (s_last == DEC_UNSURE) {
            // frames fend..wend leave S1/S2 again (the open buffer as it was
            // before frame fend); the next round folds them back in from the
            // ring and sums their spread exactly
            for (int k = 0; k < mine; ++k) {
                const int tile = first + k;
                for (int r = 0; r < WT_TR; ++r) {
                    uint4 *S1p, *S2p;
                    state_ptrs(tile, r, S1p, S2p);
                    uint4 s1 = *S1p, s2 = *S2p;
                    for (int g = fend; g <= wend; ++g) {
                        const uint2 e = ering_at(g, tile, r);
                        const uint32_t ev[4] = {e.x & 0xFFFFu, e.y & 0xFFFFu, e.x >> 16,
                                                e.y >> 16};
                        s1.x -= ev[0]; s1.y -= ev[1]; s1.z -= ev[2]; s1.w -= ev[3];
                        s2.x -= ev[0] * ev[0]; s2.y -= ev[1] * ev[1];
                        s2.z -= ev[2] * ev[2]; s2.w -= ev[3] * ev[3];
                    }
                    *S1p = s1;
                    *S2p = s2;
                }
            }
        }
        __syncthreads();
        t = fend;
        ++rnd;
    }
    // the buffer still open at the clip end
    if (st.n > 0) write_e0(st.nb, T, T);
    if (lb == 0 && tid == 0) {
        int nb = st.nb;
        if (st.n > 0) a.starts[nb++] = st.start;
        a.starts[nb] = T;
        *a.n_buffers = nb;
    }
}

// out[i][j] = luma of pixel (i, j) of one frame, rows ypitch apart; the
// padding past W is left as it is (the scan reads it only for pixels that do
// not exist, whose energy counts nowhere)
__global__ void k_luma_plane(const uint8_t *rgb, int H, int W, long ypitch, uint8_t *out) {
    const long n = (long)H * W;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x) {
        const long i = q / W, j = q - i * W;
        out[i * ypitch + j] = (uint8_t)luma_px(rgb + q * 3);
    }
}

// r[i] = floor(sqrt(x[i])) by the routine the scan applies to 65536 Q of
// every pixel (Eq. 7-8); exposed so that it can be checked at its edges.
__global__ void k_isqrt_check(const unsigned long long *x, uint32_t *r, long n) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += stride)
        r[i] = isqrt53(x[i]);
}

}  // namespace

cudaError_t launch_luma_plane(const uint8_t *rgb, int H, int W, long ypitch, uint8_t *out,
                              cudaStream_t s) {
    const long n = (long)H * W;
    if (n <= 0) return cudaSuccess;
    const long blocks = (n + 255) / 256;
    k_luma_plane<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(rgb, H, W, ypitch, out);
    return cudaGetLastError();
}

cudaError_t launch_isqrt_check(const unsigned long long *x, uint32_t *r, long n,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long blocks = (n + 255) / 256;
    k_isqrt_check<<<(int)(blocks < 1216 ? blocks : 1216), 256, 0, s>>>(x, r, n);
    return cudaGetLastError();
}

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

namespace {

// Co-resident CTAs of the warp-tile variant, and whether a clip's tiles fit
// one per warp (so that its running sums stay in shared memory).
int scan_capacity_wt(int *err_out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scan_wt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)WT_SMEM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_wt, WT_THREADS, WT_SMEM);
    if (e != cudaSuccess) { *err_out = (int)e; return 0; }
    *err_out = 0;
    return sms * per_sm;
}

}  // namespace

cudaError_t launch_scan(const ScanArgs &a, int grid, cudaStream_t s) {
    ScanArgs copy = a;
    const ScanArgs *tab = nullptr;
    const int *bc = nullptr;
    void *args[] = {&copy, &tab, &bc};
    // one clip alone: the warp-tile variant when every warp can own a single
    // tile (each warp walks its tile's rows; its state stays on chip)
    int err = 0;
    const long ntiles = (long)scan_tiles_wt(a.H, a.W);
    const int cap_wt = scan_capacity_wt(&err);
    if (!err && (long)cap_wt * WT_WARPS >= ntiles) {
        const int g = (int)((ntiles + WT_WARPS - 1) / WT_WARPS);
        return cudaLaunchCooperativeKernel((const void *)k_scan_wt, dim3(g), dim3(WT_THREADS),
                                           args, WT_SMEM, s);
    }
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
int scan_tiles_wt(int H, int W) { return ((H + WT_TR - 1) / WT_TR) * ((W + TC - 1) / TC); }
int scan_tile_warps() { return 1; }   // a CTA works on one tile at a time

// pixels of the tile-major state, enough for either layout's tiles
long scan_state_px(int H, int W) {
    const long rows = std::max((long)((H + TR - 1) / TR) * TR, (long)((H + WT_TR - 1) / WT_TR) * WT_TR);
    return rows * ((W + TC - 1) / TC) * TC;
}

}  // namespace scpl
