// SCPL carving of fixed spatiotemporal buffers (Sec. 3.1 and 3.2).
//
// Per buffer:
//   k_energy_init  first iteration: E = sum_t wg*Sobel(Y_t) + SDo, with
//                  SDo = wm * sum_t D_t kept at original coordinates, O = id.
// Per buffer and iteration:
//   k_dp           one CTA per buffer: the cumulative-energy DP of Eq. 4 with
//                  each lane holding 4 (or 8) consecutive columns in
//                  registers, the parent label carried along (Eq. 5), the
//                  per-parent argmin of Eq. 6, the k_eff lowest children and
//                  the trace back through the recorded directions into
//                  per-row sorted removal lists.
//   k_update       many CTAs per buffer: O and E are compacted by the removal
//                  lists; only carved pixels whose 3x3 neighbourhood changed
//                  get their summed gradient recomputed from the frames'
//                  original luma (gathered through O).  A pixel whose old
//                  column q has no removed pixel within columns q-2..q+2 in
//                  rows i-1..i+1 keeps exactly its old neighbourhood (every
//                  seam moves at most one column per row), so its summed
//                  energy is the old one.
// After the last iteration k_gather copies every output pixel's colour from
// its original column.
#include <map>
#include <mutex>

#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int EN_QT = 128;     // threads (4-column quads) per k_energy_init CTA
constexpr int UP_THREADS = 256;
constexpr int DP_MAX_WARPS = 32;
constexpr int DP_PF = 4;       // rows of energy prefetched ahead of the DP
constexpr uint32_t INF32 = 0xFFFFFFFFu;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// #{m : r[m] < q} for an ascending list.
__device__ __forceinline__ int count_less(const uint16_t *__restrict__ r, int k, int q) {
    int lo = 0, hi = k;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int)r[mid] < q) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int sobel_l1(int a00, int a01, int a02, int a10, int a12, int a20,
                                        int a21, int a22) {
    int gx = (a02 + 2 * a12 + a22) - (a00 + 2 * a10 + a20);
    int gy = (a20 + 2 * a21 + a22) - (a00 + 2 * a01 + a02);
    return abs(gx) + abs(gy);
}

// ---------------------------------------------------------------------------
// k_energy_init: grid (ceil(W0 / (4 * EN_QT)), H, nb), EN_QT threads; every
// thread owns a quad of 4 columns of one row of one buffer.  It writes the
// identity origin map, SDo = wm * sum_t D_t, the frame-minor luma copy (16
// frames per uint4 and pixel, frames past the buffer zero) and E = sum_t e_t.
// The scan hands over E for most buffers (st.e0 >= 0); for the others the
// gradient of every frame is summed here.
__device__ __forceinline__ void transpose4x4(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                             uint32_t &p0, uint32_t &p1, uint32_t &p2,
                                             uint32_t &p3) {
    // w_f = (pixel 0..3 of frame f)  ->  p_j = (frames 0..3 of pixel j)
    const uint32_t t0 = __byte_perm(w0, w1, 0x5140), t1 = __byte_perm(w2, w3, 0x5140);
    const uint32_t t2 = __byte_perm(w0, w1, 0x7362), t3 = __byte_perm(w2, w3, 0x7362);
    p0 = __byte_perm(t0, t1, 0x5410);
    p1 = __byte_perm(t0, t1, 0x7632);
    p2 = __byte_perm(t2, t3, 0x5410);
    p3 = __byte_perm(t2, t3, 0x7632);
}

__global__ void __launch_bounds__(EN_QT) k_energy_init(CarveWs ws) {
    const int b = blockIdx.z;
    const BufState st = ws.st[b];
    const int W0 = ws.W0, H = ws.H;
    const int i = blockIdx.y;
    const int c = 4 * (blockIdx.x * EN_QT + threadIdx.x);
    if (c >= W0) return;
    const int nv = min(4, W0 - c);   // valid columns of the quad
    const long pitch = ws.pitch, plane = ws.plane;
    const long yrow = (long)i * ws.ypitch + c;
    const long fstride = (long)H * ws.ypitch;
    const uint8_t *Yb = ws.Y + (long)st.t0 * fstride + yrow;
    const uint8_t *Db = ws.D + (long)st.t0 * fstride + yrow;
    uint8_t *yfm = ws.Yfm + st.yfm + ((long)i * W0 + c) * st.tp;
    uint32_t sd02 = 0, sd13 = 0;   // sum of D, pixels (0, 2) and (1, 3) in u16 lanes
    for (int tb = 0; tb < st.tp; tb += 16) {
        uint32_t q[4][4];   // q[j][g]: frames tb + 4g .. tb + 4g + 3 of pixel j
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint32_t w[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const int t = tb + 4 * g + f;
                w[f] = 0;
                if (t < st.nt) {
                    w[f] = __ldg(reinterpret_cast<const uint32_t *>(Yb + (long)t * fstride));
                    const uint32_t d = __ldg(reinterpret_cast<const uint32_t *>(Db + (long)t * fstride));
                    sd02 += __byte_perm(d, 0, 0x4240);
                    sd13 += __byte_perm(d, 0, 0x4341);
                }
            }
            transpose4x4(w[0], w[1], w[2], w[3], q[0][g], q[1][g], q[2][g], q[3][g]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nv)
                *reinterpret_cast<uint4 *>(yfm + (long)j * st.tp + tb) =
                    make_uint4(q[j][0], q[j][1], q[j][2], q[j][3]);
    }
    const int sd[4] = {(int)(sd02 & 0xFFFFu) * ws.wm, (int)(sd13 & 0xFFFFu) * ws.wm,
                       (int)(sd02 >> 16) * ws.wm, (int)(sd13 >> 16) * ws.wm};
    int e[4] = {sd[0], sd[1], sd[2], sd[3]};
    if (st.e0 >= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nv) e[j] = __ldg(ws.E0 + st.e0 + (long)i * W0 + c + j);
    } else {
        // no sum from the scan: add the gradient of every frame
        for (int t = 0; t < st.nt; ++t) {
            const uint8_t *Yt = ws.Y + (long)(st.t0 + t) * fstride;
            const uint8_t *ru = Yt + (long)clampi(i - 1, 0, H - 1) * ws.ypitch;
            const uint8_t *rc = Yt + (long)i * ws.ypitch;
            const uint8_t *rd = Yt + (long)clampi(i + 1, 0, H - 1) * ws.ypitch;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= nv) continue;
                const int p = c + j, pl = max(p - 1, 0), pr = min(p + 1, W0 - 1);
                e[j] += ws.wg * sobel_l1(__ldg(ru + pl), __ldg(ru + p), __ldg(ru + pr),
                                         __ldg(rc + pl), __ldg(rc + pr), __ldg(rd + pl),
                                         __ldg(rd + p), __ldg(rd + pr));
            }
        }
    }
    uint16_t *O = ws.O + (long)b * 2 * plane + (long)i * pitch + c;
    int32_t *SDo = ws.SD + (long)b * plane + (long)i * pitch + c;
    int32_t *E = ws.E + (long)b * 2 * plane + (long)i * pitch + c;
    // pitch is a multiple of 32 and c of 4: whole quads are aligned vectors
    *reinterpret_cast<uint2 *>(O) = make_uint2((uint32_t)c | ((uint32_t)(c + 1) << 16),
                                               (uint32_t)(c + 2) | ((uint32_t)(c + 3) << 16));
    *reinterpret_cast<int4 *>(SDo) = make_int4(sd[0], sd[1], sd[2], sd[3]);
    *reinterpret_cast<int4 *>(E) = make_int4(e[0], e[1], e[2], e[3]);
}

// ---------------------------------------------------------------------------
// k_update: grid (ceil(H/RB), nb), UP_THREADS threads, dynamic shared memory
// (see update_smem_bytes).
//   0. One thread stages the CTA's rows into shared memory with bulk copies:
//      the origin map of rows i0-1 .. i0+RB and the summed energy of rows
//      i0 .. i0+RB-1, at the committed width.
//   2. Meanwhile the changed pixels of the rows are marked in a bitmap and
//      listed.
//   1. O and E are compacted: each thread gathers 8 consecutive output pixels
//      from the staged rows and writes them as vectors.
//   3. Each changed pixel's summed gradient is recomputed from the frame-minor
//      luma copy written by k_energy_init (its neighbours' origins come from
//      the staged rows), 16 frames per work item.
constexpr unsigned long long UP_WAIT_NS = 2000000000ull;   // bound of the staging wait

template <bool FWD>
__global__ void __launch_bounds__(UP_THREADS) k_update(CarveWs ws, int RB) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_cnt;
    __shared__ __align__(8) uint64_t s_mbar;
    pdl_launch_dependents();
    pdl_wait();   // the DP's selection and removal lists
    const int b = blockIdx.y;
    const BufState st = ws.st[b];
    const int keff = st.k_eff;
    if (keff == 0) return;
    const int Wc = st.W, Wn = Wc - keff;
    const int s_in = st.slot, s_out = s_in ^ 1;
    const bool need_e = Wn > st.target;
    const int H = ws.H, i0 = blockIdx.x * RB;
    if (i0 >= H) return;
    const int nrows = min(RB, H - i0);
    const int tid = threadIdx.x;
    const long pitch = ws.pitch, plane = ws.plane;
    const int kcap = ws.kcap;
    const int nwords0 = (ws.W0 + 31) >> 5;
    const int list_cap = RB * min(ws.W0, 9 * kcap);
    uint16_t *rl = reinterpret_cast<uint16_t *>(smraw);   // [RB+2][kcap] lists of rows i0-1..i0+RB
    size_t off = ((size_t)(RB + 2) * kcap * 2 + 15) & ~(size_t)15;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smraw + off);   // [RB][nwords0]
    off += (size_t)RB * nwords0 * 4;
    uint32_t *list = reinterpret_cast<uint32_t *>(smraw + off);  // [list_cap] (row << 16 | old column)
    off = (off + (size_t)list_cap * 4 + 15) & ~(size_t)15;
    const int W8 = (ws.W0 + 7) & ~7, W4 = (ws.W0 + 3) & ~3;     // staged row strides
    uint16_t *Os = reinterpret_cast<uint16_t *>(smraw + off);    // [RB+2][W8] O of rows i0-1..
    off += (size_t)(RB + 2) * W8 * 2;
    int32_t *Es = reinterpret_cast<int32_t *>(smraw + off);      // [RB][W4] E of rows i0..
    off += (size_t)RB * W4 * 4;
    int *acc = reinterpret_cast<int *>(smraw + off);             // [list_cap] recomputed sums
    // forward terms: the listed pixels' recomputed row terms and diagonal sums
    constexpr bool fwd = FWD;
    int *accu = acc + list_cap;                                  // [list_cap] (fwd only)
    uint32_t *accp = reinterpret_cast<uint32_t *>(accu + list_cap);   // [list_cap] (fwd only)
    const uint16_t *rem = ws.rem + (long)b * H * kcap;
    const uint16_t *__restrict__ Oin = ws.O + ((long)b * 2 + s_in) * plane;
    const int32_t *__restrict__ Ein = ws.E + ((long)b * 2 + s_in) * plane;
    if (tid == 0) {
        // rows start 64-byte aligned (pitch is a multiple of 32) and the
        // rounded widths stay within the pitch
        const unsigned obytes = (unsigned)((Wc + 7) & ~7) * 2u;
        const unsigned ebytes = (unsigned)((Wc + 3) & ~3) * 4u;
        mbar_init(&s_mbar, 1);
        fence_mbar_init();
        mbar_expect_tx(&s_mbar, (unsigned)(nrows + 2) * obytes + (need_e ? (unsigned)nrows * ebytes : 0u));
        for (int r = 0; r < nrows + 2; ++r)
            bulk_g2s(Os + (size_t)r * W8, Oin + (long)clampi(i0 + r - 1, 0, H - 1) * pitch, obytes,
                     &s_mbar);
        if (need_e)
            for (int r = 0; r < nrows; ++r)
                bulk_g2s(Es + (size_t)r * W4, Ein + (long)(i0 + r) * pitch, ebytes, &s_mbar);
    }

    for (int x = tid; x < (RB + 2) * keff; x += UP_THREADS) {
        const int r = x / keff, m = x - r * keff;
        const int gi = clampi(i0 + r - 1, 0, H - 1);
        rl[r * kcap + m] = rem[(long)gi * kcap + m];
    }
    for (int x = tid; x < nrows * nwords0; x += UP_THREADS) bm[x] = 0;
    if (tid == 0) s_cnt = 0;
    __syncthreads();   // lists loaded; the staging barrier is initialised

    // 2. while the rows arrive: old columns within 1 of a removed pixel in
    //    rows i-1, i, i+1, marked in a bitmap and listed.  No other pixel
    //    changes: seams move at most one column a row, so the new 3x3
    //    neighbourhood of a pixel x (and so its gradient and forward terms)
    //    holds the same original pixels unless some row i-1 .. i+1 lost a
    //    pixel in x-1 .. x+1
    int cnt = 0;
    if (need_e) {
        const int per_row = 9 * keff;
        for (int x = tid; x < nrows * per_row; x += UP_THREADS) {
            const int r = x / per_row, y = x - r * per_row;
            const int a = y / (3 * keff), z = y - a * 3 * keff;
            const int mm = z / 3, d = z - mm * 3 - 1;
            const int c = (int)rl[(r + a) * kcap + mm] + d;
            if (c >= 0 && c < Wc) atomicOr(&bm[r * nwords0 + (c >> 5)], 1u << (c & 31));
        }
        __syncthreads();
        for (int x = tid; x < nrows * keff; x += UP_THREADS) {
            const int r = x / keff, mm = x - r * keff;
            const int c = rl[(r + 1) * kcap + mm];
            atomicAnd(&bm[r * nwords0 + (c >> 5)], ~(1u << (c & 31)));
        }
        __syncthreads();
        const int nwords = (Wc + 31) >> 5;
        const int lane = tid & 31;
        // every warp reserves room for all its words' bits with one atomic
        for (int x0 = tid - lane; x0 < nrows * nwords; x0 += UP_THREADS) {
            const int x = x0 + lane;
            uint32_t bits = 0;
            int r = 0, wd = 0;
            if (x < nrows * nwords) {
                r = x / nwords;
                wd = x - r * nwords;
                bits = bm[r * nwords0 + wd];
            }
            const int n = __popc(bits);
            int pre = n;   // inclusive prefix over the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += y;
            }
            int base = 0;
            if (lane == 31) base = atomicAdd(&s_cnt, pre);
            base = __shfl_sync(0xffffffffu, base, 31);
            int pos = base + pre - n;
            while (bits) {
                const int bit = __ffs(bits) - 1;
                bits &= bits - 1;
                list[pos++] = ((uint32_t)r << 16) | (uint32_t)(wd * 32 + bit);
            }
        }
        __syncthreads();
        cnt = s_cnt;
        for (int e = tid; e < cnt; e += UP_THREADS) acc[e] = 0;
        if constexpr (fwd)
            for (int e = tid; e < cnt; e += UP_THREADS) {
                accu[e] = 0;
                accp[e] = 0;
            }
        if (tid == 0 && ws.dirty_count) atomicAdd(ws.dirty_count + b, (unsigned long long)cnt);
    }
    mbar_wait(&s_mbar, 0u, ws.err, UP_WAIT_NS);

    // 1. compaction of the origin map and of the summed energy
    uint16_t *__restrict__ Oout = ws.O + ((long)b * 2 + s_out) * plane;
    int32_t *__restrict__ Eout = ws.E + ((long)b * 2 + s_out) * plane;
    const int chunks = (Wn + 7) >> 3;
    for (int x = tid; x < nrows * chunks; x += UP_THREADS) {
        const int r = x / chunks, p0 = (x - r * chunks) * 8;
        const long roff = (long)(i0 + r) * pitch;
        const uint16_t *rr = rl + (r + 1) * kcap;
        int m = 0;
        {   // removals at or before the source of p0
            int lo = 0, hi = keff;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int)rr[mid] - mid <= p0) lo = mid + 1; else hi = mid;
            }
            m = lo;
        }
        int src[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int p = p0 + j;
            while (m < keff && (int)rr[m] - m <= p) ++m;
            src[j] = min(p + m, Wc - 1);
        }
        uint16_t ov[8];
        int ev[8];
        const uint16_t *orow = Os + (size_t)(r + 1) * W8;
        const int32_t *erow = Es + (size_t)r * W4;
#pragma unroll
        for (int j = 0; j < 8; ++j) ov[j] = orow[src[j]];
        if (need_e) {
#pragma unroll
            for (int j = 0; j < 8; ++j) ev[j] = erow[src[j]];
        }
        if (fwd && need_e) {   // the diagonal sums move with their pixels
            const uint32_t *prow = ws.P + ((long)b * 2 + s_in) * plane + roff;
            uint32_t *pout = ws.P + ((long)b * 2 + s_out) * plane + roff;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (p0 + j < Wn) pout[p0 + j] = __ldg(prow + src[j]);
        }
        if (p0 + 8 <= Wn) {
            uint4 o4;
            o4.x = (uint32_t)ov[0] | ((uint32_t)ov[1] << 16);
            o4.y = (uint32_t)ov[2] | ((uint32_t)ov[3] << 16);
            o4.z = (uint32_t)ov[4] | ((uint32_t)ov[5] << 16);
            o4.w = (uint32_t)ov[6] | ((uint32_t)ov[7] << 16);
            *reinterpret_cast<uint4 *>(Oout + roff + p0) = o4;
            if (need_e) {
                *reinterpret_cast<int4 *>(Eout + roff + p0) = make_int4(ev[0], ev[1], ev[2], ev[3]);
                *reinterpret_cast<int4 *>(Eout + roff + p0 + 4) =
                    make_int4(ev[4], ev[5], ev[6], ev[7]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (p0 + j < Wn) {
                    Oout[roff + p0 + j] = ov[j];
                    if (need_e) Eout[roff + p0 + j] = ev[j];
                }
            }
        }
    }
    if (!need_e) return;
    __syncthreads();   // the compacted energy is written before the changed pixels

    // 3. exact recompute of the changed pixels: every frame's Sobel gradient
    //    from the frame-minor luma copy, one work item per changed pixel and
    //    16-frame group (one vector load per neighbour), bytes widened to
    //    16-bit lanes and |P - N| taken with packed max/min; the groups' sums
    //    meet in shared memory
    const int32_t *SDo = ws.SD + (long)b * plane;
    const uint8_t *yfm = ws.Yfm + st.yfm;
    const int tp = st.tp, ng = tp >> 4;
    for (int x = tid; x < cnt * ng; x += UP_THREADS) {
        const int e = x / ng, f = x - e * ng;
        const int r = (int)(list[e] >> 16), q = (int)(list[e] & 0xFFFFu);
        const int i = i0 + r;
        const int p = q - count_less(rl + (r + 1) * kcap, keff, q);
        const uint4 *nb[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int gi = clampi(i + a - 1, 0, H - 1);
            const uint16_t *rr = rl + (r + a) * kcap;
            // source columns of x-1, x, x+1 (clamped): one search, then steps
            // over the removals that fall between consecutive columns
            const int xl = max(p - 1, 0), xr = min(p + 1, Wn - 1);
            int m = 0;
            {
                int lo = 0, hi = keff;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if ((int)rr[mid] - mid <= xl) lo = mid + 1; else hi = mid;
                }
                m = lo;
            }
            int src[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int x = c == 0 ? xl : (c == 1 ? min(p, Wn - 1) : xr);
                while (m < keff && (int)rr[m] - m <= x) ++m;
                src[c] = x + m;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int o = Os[(size_t)(r + a) * W8 + src[c]];
                nb[a][c] = reinterpret_cast<const uint4 *>(yfm + ((long)gi * ws.W0 + o) * tp);
            }
        }
        const uint4 v00 = __ldg(nb[0][0] + f), v01 = __ldg(nb[0][1] + f), v02 = __ldg(nb[0][2] + f);
        const uint4 v10 = __ldg(nb[1][0] + f), v12 = __ldg(nb[1][2] + f);
        const uint4 v20 = __ldg(nb[2][0] + f), v21 = __ldg(nb[2][1] + f), v22 = __ldg(nb[2][2] + f);
        const uint32_t w00[4] = {v00.x, v00.y, v00.z, v00.w}, w01[4] = {v01.x, v01.y, v01.z, v01.w};
        const uint32_t w02[4] = {v02.x, v02.y, v02.z, v02.w}, w10[4] = {v10.x, v10.y, v10.z, v10.w};
        const uint32_t w12[4] = {v12.x, v12.y, v12.z, v12.w}, w20[4] = {v20.x, v20.y, v20.z, v20.w};
        const uint32_t w21[4] = {v21.x, v21.y, v21.z, v21.w}, w22[4] = {v22.x, v22.y, v22.z, v22.w};
        uint32_t packed = 0;   // two 16-bit lane sums, at most 8 * 2040 each
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t sel = h ? 0x4342u : 0x4140u;   // bytes (2,3) or (0,1) -> u16 lanes
                const uint32_t a00 = __byte_perm(w00[k], 0, sel), a01 = __byte_perm(w01[k], 0, sel);
                const uint32_t a02 = __byte_perm(w02[k], 0, sel), a10 = __byte_perm(w10[k], 0, sel);
                const uint32_t a12 = __byte_perm(w12[k], 0, sel), a20 = __byte_perm(w20[k], 0, sel);
                const uint32_t a21 = __byte_perm(w21[k], 0, sel), a22 = __byte_perm(w22[k], 0, sel);
                const uint32_t gxp = a02 + 2u * a12 + a22, gxn = a00 + 2u * a10 + a20;
                const uint32_t gyp = a20 + 2u * a21 + a22, gyn = a00 + 2u * a01 + a02;
                const uint32_t gx = __vimax3_u16x2(gxp, gxn, 0u) - __vimin3_u16x2(gxp, gxn, 0xFFFFFFFFu);
                const uint32_t gy = __vimax3_u16x2(gyp, gyn, 0u) - __vimin3_u16x2(gyp, gyn, 0xFFFFFFFFu);
                packed += gx + gy;
            }
        }
        atomicAdd(&acc[e], (int)(packed & 0xFFFFu) + (int)(packed >> 16));
        if (fwd) {
            // forward terms of the group's 16 frames: left L = (i, p-1), right
            // R = (i, p+1), above U = (i-1, p); the row term is 0 in the first
            // and last column, the diagonal sums stay below 2^16 a pixel
            const uint32_t *wL = w10, *wR = w12, *wU = w01;
            uint32_t cu = 0, da = 0, db = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cu += __vsadu4(wR[k], wL[k]);
                da += __vsadu4(wU[k], wL[k]);
                db += __vsadu4(wU[k], wR[k]);
            }
            if (p > 0 && p < Wn - 1) atomicAdd(&accu[e], (int)cu);
            atomicAdd(&accp[e], da | (db << 16));
        }
    }
    __syncthreads();
    for (int e = tid; e < cnt; e += UP_THREADS) {
        const int r = (int)(list[e] >> 16), q = (int)(list[e] & 0xFFFFu);
        const int i = i0 + r;
        const int p = q - count_less(rl + (r + 1) * kcap, keff, q);
        const int ocenter = Os[(size_t)(r + 1) * W8 + q];   // the pixel's own origin
        int ev = ws.wg * acc[e] + SDo[(long)i * pitch + ocenter];
        if (fwd) {
            ev += ws.wf * accu[e];
            ws.P[((long)b * 2 + s_out) * plane + (long)i * pitch + p] = accp[e];
        }
        Eout[(long)i * pitch + p] = ev;
    }
}

// ---------------------------------------------------------------------------
// k_forward_init: grid (ceil(W0 / FW_T), H, nb), FW_T threads, one pixel
// each.  The forward terms of a buffer at its original width, summed over its
// frames from the frame-minor luma copy, 16 frames per vector (per-byte
// absolute differences added by __vsadu4; frames past the buffer are zero in
// every pixel and add nothing): the row term CU = |Y(i,j+1) - Y(i,j-1)| (0 in
// the first and last column) goes into E with weight wf, the diagonal terms
// A = |Y(i-1,j) - Y(i,j-1)| and B = |Y(i-1,j) - Y(i,j+1)| into P.  Terms that
// no move reads (A in column 0, B in the last column, both in row 0) come from
// clamped neighbours.
constexpr int FW_T = 128;

__global__ void __launch_bounds__(FW_T) k_forward_init(CarveWs ws) {
    const int b = blockIdx.z, i = blockIdx.y;
    const int j = blockIdx.x * FW_T + threadIdx.x;
    const int W0 = ws.W0;
    if (j >= W0) return;
    const BufState st = ws.st[b];
    const int tp = st.tp;
    const uint8_t *yfm = ws.Yfm + st.yfm;
    const uint4 *L = reinterpret_cast<const uint4 *>(yfm + ((long)i * W0 + max(j - 1, 0)) * tp);
    const uint4 *R = reinterpret_cast<const uint4 *>(yfm + ((long)i * W0 + min(j + 1, W0 - 1)) * tp);
    const uint4 *U = reinterpret_cast<const uint4 *>(yfm + ((long)max(i - 1, 0) * W0 + j) * tp);
    uint32_t cu = 0, da = 0, db = 0;
    for (int g = 0; g < (tp >> 4); ++g) {
        const uint4 l = __ldg(L + g), r = __ldg(R + g), u = __ldg(U + g);
        cu += __vsadu4(r.x, l.x) + __vsadu4(r.y, l.y) + __vsadu4(r.z, l.z) + __vsadu4(r.w, l.w);
        da += __vsadu4(u.x, l.x) + __vsadu4(u.y, l.y) + __vsadu4(u.z, l.z) + __vsadu4(u.w, l.w);
        db += __vsadu4(u.x, r.x) + __vsadu4(u.y, r.y) + __vsadu4(u.z, r.z) + __vsadu4(u.w, r.w);
    }
    if (j == 0 || j == W0 - 1) cu = 0;
    const long o = (long)b * 2 * ws.plane + (long)i * ws.pitch + j;   // slot 0
    ws.E[o] += ws.wf * (int)cu;
    ws.P[o] = da | (db << 16);
}

// ---------------------------------------------------------------------------
// k_dp: one CTA of 32*NW threads per buffer.  Lane l of warp w holds the V
// consecutive columns base = (32w + l)*V .. base+V-1 of the current DP row:
// their cumulative energy (u32) and parent label.  A row step takes the left
// and right neighbours from the adjacent lanes (shuffles) or, at a warp's
// edge, from the neighbouring warp's boundary slot of the previous row.
//
// Ties: the candidates are compared j-1, j, j+1 with a strict "<", so the
// lowest column wins among equal cumulative energies (the tie reading of
// Eq. 4 that makes paths non-crossing).
//
// Directions: 2 bits per pixel, one u32 word per 4 rows x 4 columns:
// word [i/4][j/4], bits 8*(i%4) + 2*(j%4).
//
// FWD (forward terms): the move from the upper left also costs wf * A and
// the move from the upper right wf * B, both read from the P plane of the
// pixel; a neighbour outside the row (cost INF32) stays INF32.
template <int V, bool FWD>
__global__ void __launch_bounds__(DP_MAX_WARPS * 32, 1)
k_dp(CarveWs ws, int k, int16_t *seams, long seam_stride, int band_blocks) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint32_t bnd_c[2][DP_MAX_WARPS][2], bnd_l[2][DP_MAX_WARPS][2];
    __shared__ int s_W, s_slot, s_removed, s_target, s_active, s_cnt, s_k;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int NT = blockDim.x, NW = NT >> 5;
    const int H = ws.H;
    if (tid == 0) {
        BufState st = ws.st[b];
        committed(st, st.W, st.slot, st.removed);
        st.k_eff = 0;
        ws.st[b] = st;
        s_W = st.W; s_slot = st.slot; s_removed = st.removed; s_target = st.target;
        s_active = st.W > st.target;
        s_k = st.k > 0 ? st.k : k;
        s_cnt = 0;
    }
    __syncthreads();
    if (!s_active) return;
    const int W = s_W;
    const int32_t *E = ws.E + ((long)b * 2 + s_slot) * ws.plane;
    const long pitch = ws.pitch;
    const int base = (w * 32 + lane) * V;
    const int dstride = ws.dstride;
    uint32_t *dirs = ws.dirs + (long)b * ws.dbuf;
    const bool vec = ((pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(E) & 15) == 0);
    const uint32_t *Pd = FWD ? ws.P + ((long)b * 2 + s_slot) * ws.plane : nullptr;
    const uint32_t wf = FWD ? (uint32_t)ws.wf : 0u;
    auto loadP = [&](int i, uint32_t (&dst)[V]) {   // the diagonal sums of row i
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v] = 0;
        if (FWD && i < H && base < W) {
            const uint32_t *row = Pd + (long)i * pitch + base;
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (base + v < W) dst[v] = __ldcg(row + v);
        }
    };

    auto loadE = [&](int i, int (&dst)[V]) {
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v] = 0;
        if (i < H && base < W) {
            const int32_t *row = E + (long)i * pitch + base;
            if (vec && base + V <= pitch) {
#pragma unroll
                for (int v4 = 0; v4 < V; v4 += 4) {
                    const int4 q = __ldcg(reinterpret_cast<const int4 *>(row + v4));
                    dst[v4] = q.x; dst[v4 + 1] = q.y; dst[v4 + 2] = q.z; dst[v4 + 3] = q.w;
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (base + v < W) dst[v] = __ldcg(row + v);
            }
        }
    };

    uint32_t cost[V], lab[V];
    bool valid[V];
    {
        int e0[V];
        loadE(0, e0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            valid[v] = base + v < W;
            cost[v] = valid[v] ? (uint32_t)e0[v] : INF32;
            lab[v] = (uint32_t)(base + v);
        }
    }
    if (lane == 0) { bnd_c[0][w][0] = cost[0]; bnd_l[0][w][0] = lab[0]; }
    if (lane == 31) { bnd_c[0][w][1] = cost[V - 1]; bnd_l[0][w][1] = lab[V - 1]; }
    int ering[DP_PF][V];
#pragma unroll
    for (int u = 0; u < DP_PF; ++u) loadE(1 + u, ering[u]);
    uint32_t pring[FWD ? DP_PF : 1][V];
    if constexpr (FWD) {
#pragma unroll
        for (int u = 0; u < DP_PF; ++u) loadP(1 + u, pring[u]);
    }
    uint32_t dw[V / 4];
#pragma unroll
    for (int g = 0; g < V / 4; ++g) dw[g] = 0;
    const bool store_dirs = base < ws.W0;
    __syncthreads();

    for (int ib = 1; ib < H; ib += DP_PF) {
#pragma unroll
        for (int u = 0; u < DP_PF; ++u) {
            const int i = ib + u;
            if (i < H) {
                const int sp = (i - 1) & 1;
                uint32_t lc = __shfl_up_sync(0xffffffffu, cost[V - 1], 1);
                uint32_t ll = __shfl_up_sync(0xffffffffu, lab[V - 1], 1);
                uint32_t rc = __shfl_down_sync(0xffffffffu, cost[0], 1);
                uint32_t rl = __shfl_down_sync(0xffffffffu, lab[0], 1);
                if (lane == 0) {
                    lc = w > 0 ? bnd_c[sp][w - 1][1] : INF32;
                    ll = w > 0 ? bnd_l[sp][w - 1][1] : 0u;
                }
                if (lane == 31) {
                    rc = w < NW - 1 ? bnd_c[sp][w + 1][0] : INF32;
                    rl = w < NW - 1 ? bnd_l[sp][w + 1][0] : 0u;
                }
                uint32_t nc[V], nl[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    uint32_t c0 = v == 0 ? lc : cost[v - 1];
                    const uint32_t l0 = v == 0 ? ll : lab[v - 1];
                    uint32_t c2 = v == V - 1 ? rc : cost[v + 1];
                    const uint32_t l2 = v == V - 1 ? rl : lab[v + 1];
                    if constexpr (FWD) {
                        // real cumulative costs stay below 2^31 (checked on the host)
                        const uint32_t pw = pring[u][v];
                        if (c0 < 0x80000000u) c0 += wf * (pw & 0xFFFFu);
                        if (c2 < 0x80000000u) c2 += wf * (pw >> 16);
                    }
                    uint32_t m = c0, l = l0, d = 0;
                    if (cost[v] < m) { m = cost[v]; l = lab[v]; d = 1; }
                    if (c2 < m) { m = c2; l = l2; d = 2; }
                    nc[v] = valid[v] ? m + (uint32_t)ering[u][v] : INF32;
                    nl[v] = l;
                    dw[v >> 2] |= d << (8 * (i & 3) + 2 * (v & 3));
                }
#pragma unroll
                for (int v = 0; v < V; ++v) { cost[v] = nc[v]; lab[v] = nl[v]; }
                if ((i & 3) == 3 || i == H - 1) {
                    if (store_dirs) {
#pragma unroll
                        for (int g = 0; g < V / 4; ++g)
                            if (base + 4 * g < ws.W0)
                                dirs[(long)(i >> 2) * dstride + (base >> 2) + g] = dw[g];
                    }
#pragma unroll
                    for (int g = 0; g < V / 4; ++g) dw[g] = 0;
                }
                if (lane == 0) { bnd_c[i & 1][w][0] = cost[0]; bnd_l[i & 1][w][0] = lab[0]; }
                if (lane == 31) { bnd_c[i & 1][w][1] = cost[V - 1]; bnd_l[i & 1][w][1] = lab[V - 1]; }
                loadE(i + DP_PF, ering[u]);
                if constexpr (FWD) loadP(i + DP_PF, pring[u]);
                __syncthreads();
            }
        }
    }

    // ---- Eq. 6: least (CE, column) child of every parent --------------------
    const int W0 = ws.W0;
    uint64_t *segmin = reinterpret_cast<uint64_t *>(smraw);   // [W0]
    uint64_t *cand = segmin + W0;                             // [W0]
    int *sel = reinterpret_cast<int *>(cand + W0);            // [W0]
    int *pos = sel + W0;                                      // [W0]
    uint32_t *band = reinterpret_cast<uint32_t *>(pos + W0);  // [2][band_blocks*dstride]
    for (int j = tid; j < W; j += NT) segmin[j] = ~0ull;
    __syncthreads();
    {
        // runs of equal labels inside the lane's columns, one atomic per run
        uint64_t run = ~0ull;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (valid[v]) {
                const uint64_t key = ((uint64_t)cost[v] << 32) | (uint32_t)(base + v);
                run = key < run ? key : run;
                const bool last_of_run = (v == V - 1) || !valid[v + 1] || lab[v + 1] != lab[v];
                if (last_of_run) {
                    atomicMin(reinterpret_cast<unsigned long long *>(&segmin[lab[v]]),
                              (unsigned long long)run);
                    run = ~0ull;
                }
            }
        }
    }
    __syncthreads();
    for (int a = tid; a < W; a += NT) {
        const uint64_t v = segmin[a];
        if (v != ~0ull) cand[atomicAdd(&s_cnt, 1)] = v;
    }
    __syncthreads();
    const int n = s_cnt;
    int keff = min(s_k, W - s_target);
    keff = min(keff, n);
    for (int c = tid; c < n; c += NT) {
        const uint64_t v = cand[c];
        int r = 0;
        for (int c2 = 0; c2 < n; ++c2) r += cand[c2] < v;
        if (r < keff) sel[r] = (int)(uint32_t)v;
    }
    __syncthreads();
    for (int r = tid; r < keff; r += NT) {
        const int c = sel[r];
        int q = 0;
        for (int r2 = 0; r2 < keff; ++r2) q += sel[r2] < c;
        pos[r] = q;
    }
    __syncthreads();

    // ---- trace back (Sec. 3.1): bands of direction rows staged in shared
    // memory, the next band loaded by the non-walking warps meanwhile --------
    const int nblk = (H + 3) >> 2;
    const int nbands = (nblk + band_blocks - 1) / band_blocks;
    const int band_words = band_blocks * dstride;
    const int wt = min(((keff + 31) >> 5) << 5, NT);   // walker threads, whole warps
    const bool loaders = wt < NT;
    const uint16_t *Ocur = ws.O + ((long)b * 2 + s_slot) * ws.plane;
    uint16_t *rem = ws.rem + (long)b * H * ws.kcap;
    auto load_band = [&](int q, int t_begin, int t_step) {
        const int bhi = nblk - q * band_blocks;
        const int blo = max(bhi - band_blocks, 0);
        const int nwd = (bhi - blo) * dstride;
        const uint32_t *src = dirs + (long)blo * dstride;
        uint32_t *dst = band + (q & 1) * band_words;
        for (int x = t_begin; x < nwd; x += t_step) dst[x] = __ldcg(src + x);
    };
    load_band(0, tid, NT);
    __syncthreads();
    // sel[s] holds seam s's column at the current row while it is traced
    for (int q = 0; q < nbands; ++q) {
        if (q + 1 < nbands && loaders && tid >= wt) load_band(q + 1, tid - wt, NT - wt);
        const int bhi = nblk - q * band_blocks;
        const int blo = max(bhi - band_blocks, 0);
        const uint32_t *cur = band + (q & 1) * band_words;
        const int top = min(bhi * 4, H);
        for (int sidx = tid; sidx < keff; sidx += NT) {
            int col = sel[sidx];
            const int mypos = pos[sidx];
            for (int i = top - 1; i >= blo * 4; --i) {
                rem[(long)i * ws.kcap + mypos] = (uint16_t)col;
                if (seams)
                    seams[(long)b * seam_stride + (long)(s_removed + sidx) * H + i] =
                        (int16_t)Ocur[(long)i * pitch + col];
                if (i > 0) {
                    const uint32_t word = cur[((i >> 2) - blo) * dstride + (col >> 2)];
                    const int d = (int)((word >> (8 * (i & 3) + 2 * (col & 3))) & 3u);
                    col += d - 1;
                }
            }
            sel[sidx] = col;
        }
        if (q + 1 < nbands && !loaders) load_band(q + 1, tid, NT);
        __syncthreads();
    }
    if (tid == 0) {
        const int it = ws.st[b].iters;
        if (it < ws.klog_stride) ws.klog[(long)b * ws.klog_stride + it] = keff;
        ws.st[b].iters = it + 1;
        ws.st[b].k_eff = keff;
    }
}

// O = identity in slot 0 (used before a standalone DP on a caller's map).
__global__ void k_identity_O(CarveWs ws) {
    const int b = blockIdx.y;
    uint16_t *O = ws.O + (long)b * 2 * ws.plane;
    long total = (long)ws.H * ws.W0;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x) {
        int i = (int)(q / ws.W0), j = (int)(q % ws.W0);
        O[(long)i * ws.pitch + j] = (uint16_t)j;
    }
}

// One output row of the colour gather: dst[p] = src[O[p]] for p < target.
// Every thread moves quads of 4 pixels: 4 origins in one load, 12 bytes out as
// three words when the row is word-aligned.
__device__ __forceinline__ void gather_row(const uint16_t *__restrict__ O,
                                           const uint8_t *__restrict__ src,
                                           uint8_t *__restrict__ dst, int target) {
    const bool words = ((reinterpret_cast<uintptr_t>(dst) & 3) == 0);
    for (int p = 4 * threadIdx.x; p < target; p += 4 * blockDim.x) {
        const uint2 o4 = *reinterpret_cast<const uint2 *>(O + p);   // O rows are 8-byte aligned
        const int o[4] = {(int)(o4.x & 0xFFFF), (int)(o4.x >> 16), (int)(o4.y & 0xFFFF),
                          (int)(o4.y >> 16)};
        const int n = min(4, target - p);
        if (n == 4 && words) {
            uint32_t b[12];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                b[3 * j + 0] = src[o[j] * 3 + 0];
                b[3 * j + 1] = src[o[j] * 3 + 1];
                b[3 * j + 2] = src[o[j] * 3 + 2];
            }
            uint32_t *d = reinterpret_cast<uint32_t *>(dst + p * 3);
            d[0] = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
            d[1] = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
            d[2] = b[8] | (b[9] << 8) | (b[10] << 16) | (b[11] << 24);
        } else {
            for (int j = 0; j < n; ++j) {
                dst[(p + j) * 3 + 0] = src[o[j] * 3 + 0];
                dst[(p + j) * 3 + 1] = src[o[j] * 3 + 1];
                dst[(p + j) * 3 + 2] = src[o[j] * 3 + 2];
            }
        }
    }
}

// One output row of two frames at once: dst_u[p] = src_u[O_u[p]] for p <
// target (u = a, b).  Each thread's origin quad is read once when both frames
// share their origin row (frames of one buffer), and the source bytes of both
// frames are in flight together.  NT: threads of the CTA.
template <int NT>
__device__ __forceinline__ void gather_pair(const uint16_t *__restrict__ Oa,
                                            const uint16_t *__restrict__ Ob,
                                            const uint8_t *__restrict__ srca,
                                            const uint8_t *__restrict__ srcb,
                                            uint8_t *__restrict__ dsta, uint8_t *__restrict__ dstb,
                                            int target) {
    const bool words = ((reinterpret_cast<uintptr_t>(dsta) & 3) == 0) &&
                       ((reinterpret_cast<uintptr_t>(dstb) & 3) == 0);
    for (int p = 4 * threadIdx.x; p < target; p += 4 * NT) {
        const int n = min(4, target - p);
        const uint2 qa = *reinterpret_cast<const uint2 *>(Oa + p);   // O rows are 8-byte aligned
        const uint2 qb = Oa == Ob ? qa : *reinterpret_cast<const uint2 *>(Ob + p);
        const int oa[4] = {(int)(qa.x & 0xFFFF), (int)(qa.x >> 16), (int)(qa.y & 0xFFFF),
                           (int)(qa.y >> 16)};
        const int ob[4] = {(int)(qb.x & 0xFFFF), (int)(qb.x >> 16), (int)(qb.y & 0xFFFF),
                           (int)(qb.y >> 16)};
        if (n == 4 && words) {
            uint32_t x[12], y[12];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    x[3 * j + c] = srca[oa[j] * 3 + c];
                    y[3 * j + c] = srcb[ob[j] * 3 + c];
                }
            uint32_t *da = reinterpret_cast<uint32_t *>(dsta + p * 3);
            uint32_t *db = reinterpret_cast<uint32_t *>(dstb + p * 3);
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                da[w] = x[4 * w] | (x[4 * w + 1] << 8) | (x[4 * w + 2] << 16) | (x[4 * w + 3] << 24);
                db[w] = y[4 * w] | (y[4 * w + 1] << 8) | (y[4 * w + 2] << 16) | (y[4 * w + 3] << 24);
            }
        } else {
            for (int j = 0; j < n; ++j)
                for (int c = 0; c < 3; ++c) {
                    dsta[(p + j) * 3 + c] = srca[oa[j] * 3 + c];
                    dstb[(p + j) * 3 + c] = srcb[ob[j] * 3 + c];
                }
        }
    }
}

// Final colour gather: out[t][i][p] = rgb[t][i][O[i][p]].  grid (H, ceil(nt /
// GA_FRAMES)), GA_THREADS threads: the CTA takes row i of GA_FRAMES
// consecutive frames [t0 + GA_FRAMES * blockIdx.y, ...), two at a time
// (gather_pair; a lone last frame through gather_row).
constexpr int GA_FRAMES = 8;
constexpr int GA_THREADS = 128;
__global__ void __launch_bounds__(GA_THREADS) k_gather(CarveWs ws, const uint8_t *__restrict__ rgb,
                                                      const int *buf_of_frame, int target,
                                                      uint8_t *__restrict__ out, int t0, int nt) {
    const int i = blockIdx.x;
    const int fa = t0 + GA_FRAMES * blockIdx.y, fb = min(fa + GA_FRAMES, t0 + nt);
    const long rowb = (long)ws.W0 * 3, outb = (long)target * 3;
    auto orow = [&](int t) {
        const int b = buf_of_frame[t];
        int W, slot, removed;
        committed(ws.st[b], W, slot, removed);
        return ws.O + ((long)b * 2 + slot) * ws.plane + (long)i * ws.pitch;
    };
    for (int t = fa; t < fb; t += 2) {
        const uint8_t *src = rgb + ((long)t * ws.H + i) * rowb;
        uint8_t *dst = out + ((long)t * ws.H + i) * outb;
        if (t + 1 < fb)
            gather_pair<GA_THREADS>(orow(t), orow(t + 1), src, src + (long)ws.H * rowb, dst,
                        dst + (long)ws.H * outb, target);
        else
            gather_row(orow(t), src, dst, target);
    }
}

// Final colour gather of frames listed in a table (frames of several clips
// that share one (H, W0) workspace).  grid (H, ceil(nframes / GA_FRAMES)),
// GA_THREADS threads: entries [GA_FRAMES * blockIdx.y, ...), two at a time
// when both have the same target width.
__global__ void __launch_bounds__(GA_THREADS) k_gather_frames(CarveWs ws,
                                                             const GatherFrame *__restrict__ tab,
                                                             int nframes) {
    const int i = blockIdx.x;
    const int fa = GA_FRAMES * blockIdx.y, fb = min(fa + GA_FRAMES, nframes);
    // the entry's origin row, or NULL (reported) if its buffer missed its target
    auto orow = [&](const GatherFrame &g) -> const uint16_t * {
        int W, slot, removed;
        committed(ws.st[g.b], W, slot, removed);
        if (W != g.target) {   // carving did not reach the target: report, copy nothing
            if (i == 0 && threadIdx.x == 0) atomicExch(ws.err, DEV_EINTERNAL);
            return nullptr;
        }
        return ws.O + ((long)g.b * 2 + slot) * ws.plane + (long)i * ws.pitch;
    };
    for (int e = fa; e < fb;) {
        const GatherFrame g = tab[e];
        const uint16_t *O = orow(g);
        if (e + 1 < fb && tab[e + 1].target == g.target) {
            const GatherFrame h = tab[e + 1];
            const uint16_t *O2 = orow(h);
            if (O && O2)
                gather_pair<GA_THREADS>(O, O2, g.src + (long)i * ws.W0 * 3, h.src + (long)i * ws.W0 * 3,
                            g.dst + (long)i * g.target * 3, h.dst + (long)i * h.target * 3,
                            g.target);
            else if (O)
                gather_row(O, g.src + (long)i * ws.W0 * 3, g.dst + (long)i * g.target * 3,
                           g.target);
            else if (O2)
                gather_row(O2, h.src + (long)i * ws.W0 * 3, h.dst + (long)i * h.target * 3,
                           h.target);
            e += 2;
        } else {
            if (O)
                gather_row(O, g.src + (long)i * ws.W0 * 3, g.dst + (long)i * g.target * 3,
                           g.target);
            e += 1;
        }
    }
}

// dst[t][j][i] = src[t][i][j] for RGB pixels: [T][H][W][3] -> [T][W][H][3].
// 32x32 pixel tiles through shared memory, grid (ceil(W/32), ceil(H/32), T).
__global__ void __launch_bounds__(256) k_transpose_rgb(const uint8_t *__restrict__ src, int H,
                                                       int W, uint8_t *__restrict__ dst) {
    __shared__ uint8_t tile[32][32 * 3 + 4];
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const long frame = (long)blockIdx.z * H * W * 3;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + tx;
        if (i < H && j < W) {
            const uint8_t *p = src + frame + ((long)i * W + j) * 3;
            tile[r][tx * 3 + 0] = p[0];
            tile[r][tx * 3 + 1] = p[1];
            tile[r][tx * 3 + 2] = p[2];
        }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r, i = i0 + tx;   // output row j, column i
        if (i < H && j < W) {
            uint8_t *q = dst + frame + ((long)j * H + i) * 3;
            q[0] = tile[tx][r * 3 + 0];
            q[1] = tile[tx][r * 3 + 1];
            q[2] = tile[tx][r * 3 + 2];
        }
    }
}

int dp_lanes_cols(int W0) { return W0 <= 4096 ? 4 : 8; }

template <int V>
cudaError_t launch_dp_t(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                        cudaStream_t s) {
    int band_blocks = 0;
    size_t smem = dp_smem_bytes(ws.W0, ws.H, &band_blocks);
    const int nw = (ws.W0 + 32 * V - 1) / (32 * V);
    if (ws.wf > 0) {
        if (!ws.P) return cudaErrorInvalidValue;
        cudaError_t e = raise_dyn_smem((const void *)k_dp<V, true>, smem);
        if (e != cudaSuccess) return e;
        k_dp<V, true><<<nb, 32 * nw, smem, s>>>(ws, k, seams, seam_stride, band_blocks);
        return cudaGetLastError();
    }
    cudaError_t e = raise_dyn_smem((const void *)k_dp<V, false>, smem);
    if (e != cudaSuccess) return e;
    k_dp<V, false><<<nb, 32 * nw, smem, s>>>(ws, k, seams, seam_stride, band_blocks);
    return cudaGetLastError();
}

}  // namespace

// Dynamic shared memory of k_dp: segmin, cand (u64), sel, pos (int) over W0
// columns, plus two bands of direction words, as many 4-row blocks as fit.
size_t dp_smem_bytes(int W0, int H, int *band_blocks) {
    const size_t fixed = (size_t)W0 * 24;
    const size_t limit = 227 * 1024 - 4096;   // minus the static shared memory
    const size_t dstride = (((size_t)(W0 + 3) / 4) + 3) & ~(size_t)3;   // as CarveWs::dstride
    size_t budget = limit > fixed ? limit - fixed : 0;
    if (budget > 64 * 1024) budget = 64 * 1024;
    int bb = (int)(budget / (2 * dstride * 4));
    const int nblk = (H + 3) / 4;
    if (bb > nblk) bb = nblk;
    if (bb < 1) bb = 1;
    *band_blocks = bb;
    return fixed + 2 * (size_t)bb * dstride * 4;
}

// Dynamic shared memory of a k_update CTA of `rb` rows: removal lists, the
// changed-pixel bitmap and list, the staged origin and energy rows, and the
// recomputed sums of the listed pixels.
size_t update_smem_bytes_rows(int W0, int kcap, int rb, bool fwd) {
    const size_t per_row_list = (size_t)(W0 < 9 * kcap ? W0 : 9 * kcap);
    const size_t nwords0 = (size_t)(W0 + 31) / 32;
    size_t off = (((size_t)(rb + 2) * kcap * 2 + 15) & ~(size_t)15) + (size_t)rb * nwords0 * 4;
    off = (off + (size_t)rb * per_row_list * 4 + 15) & ~(size_t)15;
    const size_t w8 = (size_t)(W0 + 7) & ~(size_t)7, w4 = (size_t)(W0 + 3) & ~(size_t)3;
    return off + (size_t)(rb + 2) * w8 * 2 + (size_t)rb * w4 * 4 +
           (size_t)rb * per_row_list * 4 * (fwd ? 3 : 1);
}

// Rows per k_update CTA (the most, up to 4, that keep five CTAs on an SM,
// as many as its registers allow, so that the recompute's gathers keep the
// L1 that shared memory would take; at least 1) and its dynamic shared
// memory.
size_t update_smem_bytes(int W0, int kcap, int *rows, bool fwd) {
    int rb = 4;
    size_t bytes = update_smem_bytes_rows(W0, kcap, rb, fwd);
    while (rb > 1 && bytes > 44 * 1024) bytes = update_smem_bytes_rows(W0, kcap, --rb, fwd);
    *rows = rb;
    return bytes;
}

cudaError_t launch_energy_init(const CarveWs &ws, int nb, cudaStream_t s) {
    dim3 grid((ws.W0 + 4 * EN_QT - 1) / (4 * EN_QT), ws.H, nb);
    k_energy_init<<<grid, EN_QT, 0, s>>>(ws);
    if (ws.wf > 0) {
        if (!ws.P) return cudaErrorInvalidValue;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_forward_init<<<dim3((ws.W0 + FW_T - 1) / FW_T, ws.H, nb), FW_T, 0, s>>>(ws);
    }
    return cudaGetLastError();
}

cudaError_t launch_update(const CarveWs &ws, int nb, cudaStream_t s) {
    int rb = 8;
    const bool fwd = ws.wf > 0;
    if (fwd && !ws.P) return cudaErrorInvalidValue;
    size_t smem = update_smem_bytes(ws.W0, ws.kcap, &rb, fwd);
    if (ws.up_rows >= 1 && ws.up_rows < rb) {
        rb = ws.up_rows;
        smem = update_smem_bytes_rows(ws.W0, ws.kcap, rb, fwd);
    }
    const void *fn = fwd ? (const void *)k_update<true> : (const void *)k_update<false>;
    cudaError_t e = raise_dyn_smem(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((ws.H + rb - 1) / rb, nb);
    cfg.blockDim = dim3(UP_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = fwd ? cudaLaunchKernelEx(&cfg, k_update<true>, ws, rb)
            : cudaLaunchKernelEx(&cfg, k_update<false>, ws, rb);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

namespace {
// Condition of the device-side carving loop: 1 while some buffer is still
// wider than its target after the body's iterations and no device wait or
// check has failed, else 0.  One thread, launched inside the loop's body.
__global__ void k_loop_more(cudaGraphConditionalHandle h, const BufState *st, int nb,
                            const int *err) {
    unsigned more = 0;
    if (*(volatile const int *)err == DEV_OK)
        for (int b = 0; b < nb; ++b)
            if (st[b].W - st[b].k_eff > st[b].target) {
                more = 1;
                break;
            }
    cudaGraphSetConditional(h, more);
}
}  // namespace

cudaError_t build_carve_loop(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                             int per_body, cudaStream_t s, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node = nullptr;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(s, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        for (int i = 0; i < per_body && e == cudaSuccess; ++i) {
            e = ws.J ? launch_dpc(ws, nb, k, seams, seam_stride, s)
                     : launch_dp_select(ws, nb, k, seams, seam_stride, s);
            if (e == cudaSuccess) e = launch_update(ws, nb, s);
        }
        if (e == cudaSuccess) {
            k_loop_more<<<1, 1, 0, s>>>(h, ws.st, nb, ws.err);
            e = cudaGetLastError();
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &captured);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

cudaError_t launch_dp_select(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                             cudaStream_t s) {
    if (dp_lanes_cols(ws.W0) == 4) return launch_dp_t<4>(ws, nb, k, seams, seam_stride, s);
    return launch_dp_t<8>(ws, nb, k, seams, seam_stride, s);
}

cudaError_t launch_identity_O(const CarveWs &ws, int nb, cudaStream_t s) {
    k_identity_O<<<dim3(152, nb), 256, 0, s>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_gather_range(const CarveWs &ws, const uint8_t *rgb, int t0, int nt,
                                const int *buf_of_frame, int target, uint8_t *out,
                                cudaStream_t s) {
    for (int f = 0; f < nt; f += 65535) {
        const int n = nt - f < 65535 ? nt - f : 65535;
        k_gather<<<dim3(ws.H, (n + GA_FRAMES - 1) / GA_FRAMES), GA_THREADS, 0, s>>>(
            ws, rgb, buf_of_frame, target, out, t0 + f, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const CarveWs &ws, const uint8_t *rgb, int T, const int *buf_of_frame,
                          int target, uint8_t *out, cudaStream_t s) {
    return launch_gather_range(ws, rgb, 0, T, buf_of_frame, target, out, s);
}

cudaError_t launch_gather_frames(const CarveWs &ws, const GatherFrame *tab, int nframes,
                                 cudaStream_t s) {
    for (int f0 = 0; f0 < nframes; f0 += 65535) {
        const int n = nframes - f0 < 65535 ? nframes - f0 : 65535;
        k_gather_frames<<<dim3(ws.H, (n + GA_FRAMES - 1) / GA_FRAMES), GA_THREADS, 0, s>>>(
            ws, tab + f0, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_transpose_rgb(const uint8_t *src, int T, int H, int W, uint8_t *dst,
                                 cudaStream_t s) {
    for (int t0 = 0; t0 < T; t0 += 65535) {
        const int n = T - t0 < 65535 ? T - t0 : 65535;
        const long off = (long)t0 * H * W * 3;
        k_transpose_rgb<<<dim3((W + 31) / 32, (H + 31) / 32, n), 256, 0, s>>>(src + off, H, W,
                                                                              dst + off);
    }
    return cudaGetLastError();
}

namespace {
size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
}  // namespace

cudaError_t raise_dyn_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = limit[std::make_pair(dev, func)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

size_t carve_ws_assign(CarveWs &ws, int nb, int klog_stride, bool dpc, char *base) {
    const int H = ws.H, W0 = ws.W0;
    ws.pitch = (W0 + 31) / 32 * 32;
    ws.plane = (long)H * ws.pitch;
    ws.dstride = (((W0 + 3) / 4) + 3) & ~3;
    ws.dbuf = (long)((H + 15) / 16) * 4 * ws.dstride;
    ws.jstride = (W0 + 7) & ~7;
    ws.kcap = ws.kcap < 1 ? 1 : ws.kcap;
    ws.klog_stride = klog_stride < 1 ? 1 : klog_stride;
    ws.rj = 0;
    ws.nbands = 0;
    if (dpc) {
        int C = 0, rj = 0;
        size_t smem = 0;
        if (ws.dpc_r != 16 && ws.dpc_r != 32) ws.dpc_r = 32;
        if (ws.dpc_wpc != 8) ws.dpc_wpc = 4;
        if (ws.dpc_v != 2 || ws.dpc_r != 16) ws.dpc_v = 4;
        if (!dpc_plan(W0, H, ws.dpc_r, ws.dpc_wpc, ws.dpc_v, &C, &rj, &smem, ws.wf > 0))
            dpc = false;
        else {
            ws.rj = rj;
            ws.nbands = (H + rj - 1) / rj;
        }
    }
    if (!dpc) ws.dpc_r = 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += al256(bytes < 1 ? 1 : bytes);
        return base ? base + o : nullptr;
    };
    ws.E = reinterpret_cast<int32_t *>(take((size_t)nb * 2 * ws.plane * 4));
    ws.SD = reinterpret_cast<int32_t *>(take((size_t)nb * ws.plane * 4));
    ws.O = reinterpret_cast<uint16_t *>(take((size_t)nb * 2 * ws.plane * 2));
    ws.dirs = reinterpret_cast<uint32_t *>(take((size_t)nb * ws.dbuf * 4));
    ws.dirty_count = reinterpret_cast<unsigned long long *>(take((size_t)nb * 8));
    ws.rem = reinterpret_cast<uint16_t *>(take((size_t)nb * H * ws.kcap * 2));
    ws.st = reinterpret_cast<BufState *>(take((size_t)nb * sizeof(BufState)));
    ws.klog = reinterpret_cast<int *>(take((size_t)nb * ws.klog_stride * 4));
    ws.J = nullptr;
    ws.colbot = nullptr;
    ws.dpx = nullptr;
    if (dpc) {
        ws.J = reinterpret_cast<uint16_t *>(take((size_t)nb * ws.nbands * ws.jstride * 2));
        ws.colbot = reinterpret_cast<uint16_t *>(take((size_t)nb * ws.nbands * ws.kcap * 2));
        ws.dpx = reinterpret_cast<int *>(take((size_t)nb * (1 + ws.kcap) * 4));
    }
    ws.P = ws.wf > 0 ? reinterpret_cast<uint32_t *>(take((size_t)nb * 2 * ws.plane * 4)) : nullptr;
    return off;
}

}  // namespace scpl
