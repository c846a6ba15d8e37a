// SCPL carving of fixed spatiotemporal buffers (Sec. 3.1 and 3.2).
//
// Per buffer and iteration:
//   k_dp_select  one CTA per buffer: the cumulative-energy DP of Eq. 4 with
//                packed keys (CE << 32 | dir << 24 | parent label), the
//                per-parent argmin of Eq. 6, the k_eff lowest children, and
//                the trace back through the recorded directions into per-row
//                sorted removal lists.
//   k_energy     many CTAs per buffer: the origin map O and the summed motion
//                energy SD are compacted by the removal lists, and the summed
//                energy of the next iteration, E = sum_t wg*Sobel(carved Y_t) +
//                SD, is rebuilt by gathering every frame's original luma
//                through O (the luma itself is never rewritten).
// After the last iteration k_gather copies every output pixel's colour from
// its original column.
#include "scpl_internal.cuh"

namespace scpl {

namespace {

constexpr int EN_RB = 8;      // rows per k_energy CTA
constexpr int EN_CW = 256;    // carved columns per k_energy CTA (= threads)
constexpr int DP_THREADS = 1024;
constexpr int DP_PF = 8;      // rows of energy prefetched ahead of the DP

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Committed view of a buffer's state (applies a pending iteration).
__device__ __forceinline__ void committed(const BufState &s, int &W, int &slot, int &removed) {
    if (s.k_eff > 0) {
        W = s.W - s.k_eff;
        slot = s.slot ^ 1;
        removed = s.removed + s.k_eff;
    } else {
        W = s.W;
        slot = s.slot;
        removed = s.removed;
    }
}

// Source column (at the old width) of carved column p, given the ascending
// removal list r[0..k) of the row: p + #{m : r[m] - m <= p}.
__device__ __forceinline__ int src_col(const uint16_t *__restrict__ r, int k, int p) {
    int lo = 0, hi = k;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int)r[mid] - mid <= p) lo = mid + 1; else hi = mid;
    }
    return p + lo;
}

// ---------------------------------------------------------------------------
// k_energy: grid (ceil(W0/EN_CW), ceil(H/EN_RB), nb), EN_CW threads.
// init = 1: first iteration (O = identity, SD = wm * sum_t D_t), writes slot 0.
// init = 0: applies the pending removal lists, writes slot ^ 1.
template <bool INIT>
__global__ void __launch_bounds__(EN_CW) k_energy(CarveWs ws) {
    const int b = blockIdx.z;
    const BufState st = ws.st[b];
    int Wn, s_in = 0, s_out = 0, keff = 0;
    if (INIT) {
        Wn = ws.W0;
    } else {
        keff = st.k_eff;
        if (keff == 0) return;
        Wn = st.W - keff;
        s_in = st.slot;
        s_out = s_in ^ 1;
    }
    const bool need_e = INIT || Wn > st.target;
    const int p0 = blockIdx.x * EN_CW;
    const int i0 = blockIdx.y * EN_RB;
    if (p0 >= Wn || i0 >= ws.H) return;

    __shared__ uint16_t Os[EN_RB + 2][EN_CW + 2];
    const int tid = threadIdx.x;
    const int H = ws.H;
    const long plane = ws.plane, pitch = ws.pitch;
    const uint16_t *Oin = ws.O + ((long)b * 2 + s_in) * plane;
    uint16_t *Oout = ws.O + ((long)b * 2 + s_out) * plane;
    const uint16_t *rem = ws.rem + (long)b * H * ws.kcap;

    for (int q = tid; q < (EN_RB + 2) * (EN_CW + 2); q += EN_CW) {
        int r = q / (EN_CW + 2), c = q % (EN_CW + 2);
        int gi = clampi(i0 + r - 1, 0, H - 1);
        int pc = clampi(p0 + c - 1, 0, Wn - 1);
        uint16_t o;
        if (INIT) o = (uint16_t)pc;
        else o = Oin[(long)gi * pitch + src_col(rem + (long)gi * ws.kcap, keff, pc)];
        Os[r][c] = o;
    }
    __syncthreads();

    const int p = p0 + tid;
    const bool col_ok = p < Wn;
    const int32_t *SDin = ws.SD + ((long)b * 2 + s_in) * plane;
    int32_t *SDout = ws.SD + ((long)b * 2 + s_out) * plane;
    int32_t eacc[EN_RB];
#pragma unroll
    for (int r = 0; r < EN_RB; ++r) {
        eacc[r] = 0;
        int i = i0 + r;
        if (col_ok && i < H) {
            Oout[(long)i * pitch + p] = Os[r + 1][tid + 1];
            if (need_e) {
                int sd = 0;
                if (INIT) {
                    for (int t = st.t0; t < st.t0 + st.nt; ++t)
                        sd += ws.D[((long)t * H + i) * ws.ypitch + p];
                    sd *= ws.wm;
                } else {
                    sd = SDin[(long)i * pitch + src_col(rem + (long)i * ws.kcap, keff, p)];
                }
                SDout[(long)i * pitch + p] = sd;
                eacc[r] = sd;
            }
        }
    }
    if (!need_e || !col_ok) return;

    for (int t = st.t0; t < st.t0 + st.nt; ++t) {
        const uint8_t *Yt = ws.Y + (long)t * H * ws.ypitch;
#pragma unroll
        for (int r = 0; r < EN_RB; ++r) {
            int i = i0 + r;
            if (i < H) {
                const uint8_t *ru = Yt + (long)clampi(i - 1, 0, H - 1) * ws.ypitch;
                const uint8_t *rc = Yt + (long)i * ws.ypitch;
                const uint8_t *rd = Yt + (long)clampi(i + 1, 0, H - 1) * ws.ypitch;
                int a00 = __ldg(ru + Os[r][tid]), a01 = __ldg(ru + Os[r][tid + 1]),
                    a02 = __ldg(ru + Os[r][tid + 2]);
                int a10 = __ldg(rc + Os[r + 1][tid]), a12 = __ldg(rc + Os[r + 1][tid + 2]);
                int a20 = __ldg(rd + Os[r + 2][tid]), a21 = __ldg(rd + Os[r + 2][tid + 1]),
                    a22 = __ldg(rd + Os[r + 2][tid + 2]);
                int gx = (a02 + 2 * a12 + a22) - (a00 + 2 * a10 + a20);
                int gy = (a20 + 2 * a21 + a22) - (a00 + 2 * a01 + a02);
                eacc[r] += ws.wg * (abs(gx) + abs(gy));
            }
        }
    }
    int32_t *Eout = ws.E + ((long)b * 2 + s_out) * plane;
#pragma unroll
    for (int r = 0; r < EN_RB; ++r) {
        int i = i0 + r;
        if (i < H) Eout[(long)i * pitch + p] = eacc[r];
    }
}

// ---------------------------------------------------------------------------
// k_dp_select: one CTA of DP_THREADS per buffer; thread tid owns the columns
// tid + m*DP_THREADS, m < MPT.
//
// Shared memory: keys[2][W0 + 2] (sentinels at both ends) and cand[W0], all
// uint64; the same bytes are reused by the selection and the trace back.
template <int MPT>
__global__ void __launch_bounds__(DP_THREADS, 1)
k_dp_select(CarveWs ws, int k, int16_t *seams, long seam_stride) {
    extern __shared__ uint64_t sm[];
    __shared__ int s_W, s_slot, s_removed, s_target, s_active, s_cnt;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int H = ws.H;
    if (tid == 0) {
        BufState st = ws.st[b];
        committed(st, st.W, st.slot, st.removed);
        st.k_eff = 0;
        ws.st[b] = st;
        s_W = st.W; s_slot = st.slot; s_removed = st.removed; s_target = st.target;
        s_active = st.W > st.target;
        s_cnt = 0;
    }
    __syncthreads();
    if (!s_active) return;
    const int W = s_W;
    const int32_t *E = ws.E + ((long)b * 2 + s_slot) * ws.plane;
    uint32_t *dirs = ws.dirs + (long)b * H * ws.ngroups * 2;
    uint64_t *keysA = sm, *keysB = sm + (ws.W0 + 2), *cand = sm + 2 * (ws.W0 + 2);
    const long pitch = ws.pitch;
    const int lane = tid & 31;

    // row 0: CE = E, label = column, direction byte 0
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        int j = tid + m * DP_THREADS;
        if (j < W) keysA[j + 1] = ((uint64_t)(uint32_t)E[j] << 32) | (uint32_t)j;
    }
    if (tid == 0) { keysA[0] = keysA[W + 1] = keysB[0] = keysB[W + 1] = KEY_INF; }

    int ereg[DP_PF][MPT];
#pragma unroll
    for (int u = 0; u < DP_PF; ++u)
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            int j = tid + m * DP_THREADS, i = 1 + u;
            ereg[u][m] = (i < H && j < W) ? E[(long)i * pitch + j] : 0;
        }
    __syncthreads();

    // rows 1..H-1 (Eq. 4); among equal CE the lowest column wins because the
    // direction byte (0 = j-1, 1 = j, 2 = j+1) is the next key field
    for (int ib = 1; ib < H; ib += DP_PF) {
#pragma unroll
        for (int u = 0; u < DP_PF; ++u) {
            const int i = ib + u;
            if (i < H) {
                const uint64_t *cur = ((i - 1) & 1) ? keysB : keysA;
                uint64_t *nxt = (i & 1) ? keysB : keysA;
#pragma unroll
                for (int m = 0; m < MPT; ++m) {
                    const int j = tid + m * DP_THREADS;
                    uint32_t d = 0;
                    if (j < W) {
                        uint64_t k0 = cur[j], k1 = cur[j + 1] | (1ull << 24),
                                 k2 = cur[j + 2] | (2ull << 24);
                        uint64_t mn = k0 < k1 ? k0 : k1;
                        mn = mn < k2 ? mn : k2;
                        d = (uint32_t)(mn >> 24) & 3u;
                        nxt[j + 1] = (mn & ~KEY_DIR_MASK) + ((uint64_t)(uint32_t)ereg[u][m] << 32);
                    }
                    // direction bit planes of this warp's 32 columns
                    unsigned lo = __ballot_sync(0xffffffffu, d & 1u);
                    unsigned hi = __ballot_sync(0xffffffffu, (d >> 1) & 1u);
                    const int g = (tid >> 5) + m * (DP_THREADS / 32);
                    if (lane == 0 && g * 32 < W) {
                        uint32_t *dst = dirs + ((long)i * ws.ngroups + g) * 2;
                        dst[0] = lo;
                        dst[1] = hi;
                    }
                    const int ip = i + DP_PF;
                    ereg[u][m] = (ip < H && j < W) ? E[(long)ip * pitch + j] : 0;
                }
                __syncthreads();
            }
        }
    }
    const uint64_t *last = ((H - 1) & 1) ? keysB : keysA;
    uint64_t *segmin = ((H - 1) & 1) ? keysA : keysB;   // the other row buffer

    // ---- Eq. 6: least (CE, column) child of every parent --------------------
    for (int j = tid; j < W; j += DP_THREADS) segmin[j] = KEY_INF;
    __syncthreads();
    for (int j = tid; j < W; j += DP_THREADS) {
        uint64_t key = last[j + 1];
        uint32_t lab = (uint32_t)key & LABEL_MASK;
        atomicMin((unsigned long long *)&segmin[lab],
                  (unsigned long long)((key & 0xFFFFFFFF00000000ull) | (uint32_t)j));
    }
    __syncthreads();
    for (int a = tid; a < W; a += DP_THREADS) {
        uint64_t v = segmin[a];
        if (v != KEY_INF) cand[atomicAdd(&s_cnt, 1)] = v;
    }
    __syncthreads();
    const int n = s_cnt;
    int keff = min(k, W - s_target);
    keff = min(keff, n);
    // rank by (CE, column): keys are distinct because the columns are.  The
    // row buffers (`last`, `segmin`) are dead now; sel/pos reuse keysA.
    int *sel = (int *)keysA;            // [keff] end columns in rank order
    int *pos = sel + W;                 // [keff] rank among the seams by column
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        const int c = tid + m * DP_THREADS;
        if (c < n) {
            const uint64_t v = cand[c];
            int r = 0;
            for (int c2 = 0; c2 < n; ++c2) r += cand[c2] < v;
            if (r < keff) sel[r] = (int)(uint32_t)v;
        }
    }
    __syncthreads();
    for (int r = tid; r < keff; r += DP_THREADS) {
        int c = sel[r], q = 0;
        for (int r2 = 0; r2 < keff; ++r2) q += sel[r2] < c;
        pos[r] = q;
    }
    __syncthreads();

    // ---- trace back (Sec. 3.1), bands of direction rows staged in smem ------
    // staging area: keysB + cand region, (W0 + 2 + W0) * 8 bytes
    uint32_t *band = (uint32_t *)keysB;
    const long band_words = ((long)(ws.W0 + 2) + ws.W0) * 2;   // uint32 words available
    const int row_words = ws.ngroups * 2;
    int BR = (int)(band_words / row_words);
    if (BR > H) BR = H;
    const uint16_t *Ocur = ws.O + ((long)b * 2 + s_slot) * ws.plane;
    uint16_t *rem = ws.rem + (long)b * H * ws.kcap;
    int col = 0, mypos = 0;
    if (tid < keff) { col = sel[tid]; mypos = pos[tid]; }
    for (int top = H; top > 0; top -= BR) {
        const int lo = max(top - BR, 0);
        __syncthreads();
        const long nw = (long)(top - lo) * row_words;
        const uint32_t *srcw = dirs + (long)lo * row_words;
        for (long w = tid; w < nw; w += DP_THREADS) band[w] = __ldcg(srcw + w);
        __syncthreads();
        if (tid < keff) {
            for (int i = top - 1; i >= lo; --i) {
                rem[(long)i * ws.kcap + mypos] = (uint16_t)col;
                if (seams)
                    seams[(long)b * seam_stride + (long)(s_removed + tid) * H + i] =
                        (int16_t)Ocur[(long)i * pitch + col];
                if (i > 0 && i > lo) {
                    const uint32_t *wrow = band + (long)(i - lo) * row_words + (col >> 5) * 2;
                    int d = (int)((wrow[0] >> (col & 31)) & 1u) |
                            (int)(((wrow[1] >> (col & 31)) & 1u) << 1);
                    col += d - 1;
                }
            }
            if (lo > 0) {
                // the step from row lo to row lo-1 needs row lo's directions,
                // which are in this band (row index 0)
                const uint32_t *wrow = band + (col >> 5) * 2;
                int d = (int)((wrow[0] >> (col & 31)) & 1u) |
                        (int)(((wrow[1] >> (col & 31)) & 1u) << 1);
                col += d - 1;
            }
        }
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

// Final colour gather: out[t][i][p] = rgb[t][i][O[i][p]].  grid (H, T).
__global__ void k_gather(CarveWs ws, const uint8_t *__restrict__ rgb, const int *buf_of_frame,
                         int target, uint8_t *__restrict__ out) {
    const int i = blockIdx.x, t = blockIdx.y;
    const int b = buf_of_frame[t];
    int W, slot, removed;
    committed(ws.st[b], W, slot, removed);
    const uint16_t *O = ws.O + ((long)b * 2 + slot) * ws.plane + (long)i * ws.pitch;
    const uint8_t *src = rgb + ((long)t * ws.H + i) * ws.W0 * 3;
    uint8_t *dst = out + ((long)t * ws.H + i) * (long)target * 3;
    for (int p = threadIdx.x; p < target; p += blockDim.x) {
        int o = O[p];
        dst[p * 3 + 0] = src[o * 3 + 0];
        dst[p * 3 + 1] = src[o * 3 + 1];
        dst[p * 3 + 2] = src[o * 3 + 2];
    }
}

template <int MPT>
cudaError_t launch_dp_t(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                        cudaStream_t s) {
    size_t smem = dp_select_smem_bytes(ws.W0);
    cudaError_t e = cudaFuncSetAttribute(k_dp_select<MPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dp_select<MPT><<<nb, DP_THREADS, smem, s>>>(ws, k, seams, seam_stride);
    return cudaGetLastError();
}

}  // namespace

size_t dp_select_smem_bytes(int W0) { return ((size_t)(W0 + 2) * 2 + W0) * sizeof(uint64_t); }

cudaError_t launch_energy_init(const CarveWs &ws, int nb, cudaStream_t s) {
    dim3 grid((ws.W0 + EN_CW - 1) / EN_CW, (ws.H + EN_RB - 1) / EN_RB, nb);
    k_energy<true><<<grid, EN_CW, 0, s>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_energy_iter(const CarveWs &ws, int nb, cudaStream_t s) {
    dim3 grid((ws.W0 + EN_CW - 1) / EN_CW, (ws.H + EN_RB - 1) / EN_RB, nb);
    k_energy<false><<<grid, EN_CW, 0, s>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_dp_select(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                             cudaStream_t s) {
    int mpt = (ws.W0 + DP_THREADS - 1) / DP_THREADS;
    if (mpt <= 1) return launch_dp_t<1>(ws, nb, k, seams, seam_stride, s);
    if (mpt <= 2) return launch_dp_t<2>(ws, nb, k, seams, seam_stride, s);
    if (mpt <= 4) return launch_dp_t<4>(ws, nb, k, seams, seam_stride, s);
    return launch_dp_t<8>(ws, nb, k, seams, seam_stride, s);
}

cudaError_t launch_identity_O(const CarveWs &ws, int nb, cudaStream_t s) {
    k_identity_O<<<dim3(152, nb), 256, 0, s>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_gather(const CarveWs &ws, const uint8_t *rgb, int T, const int *buf_of_frame,
                          int target, uint8_t *out, cudaStream_t s) {
    k_gather<<<dim3(ws.H, T), 256, 0, s>>>(ws, rgb, buf_of_frame, target, out);
    return cudaGetLastError();
}

}  // namespace scpl
