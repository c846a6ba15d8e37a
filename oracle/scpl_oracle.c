/*
 * scpl_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded CPU statement of what "Fast Video Retargeting
 * Based on Seam Carving with Parental Labeling" (arXiv 1903.03180) computes on
 * its hot path.  It exists only so that tests and the benchmark's CPU baseline
 * can check the CUDA library against something obviously correct.  It shares no
 * code, header, table or helper with the CUDA library, and nothing in the
 * product imports or links it.
 *
 * Every function names the passage of the paper it follows.  Where the paper is
 * silent or ambiguous, the reading taken is stated beside the code:
 *   R1  luma: integer BT.601, Y = (77 R + 150 G + 29 B + 128) >> 8.
 *   R2  gradient: 3x3 Sobel, G = |Gx| + |Gy| (L1), replicate border (Sec. 3.3).
 *   R3  motion: D_t = |Y_t - Y_{t-1}| on the original luma, D_0 = 0;
 *       e = wg * G + wm * D with integer weights (Sec. 3.3).
 *   R4  DP: Eq. 4 with out-of-range neighbours skipped; among equal cumulative
 *       energies the lowest column wins (the paper is silent on ties).
 *   R5  labels: the parent of a pixel is the row-0 column its path starts from
 *       (Sec. 3.1, Eq. 5).
 *   R6  selection: per parent the child of least (CE, column) (Eq. 6); the
 *       k_eff = min(k, seams still to remove, #parents) lowest of those by
 *       (CE, column) are removed in one iteration.
 *   R7  buffer: Eq. 7-9 evaluated exactly in integers as
 *       A = sum_ij floor(sqrt(65536 * (n*S2 - S1^2))) and the frame that makes
 *       (double)A > 256*alpha*M*sqrt(n-1)*H*W (n >= 2) starts the next buffer;
 *       a buffer also closes when it reaches t_max frames and at the clip end.
 *       M is the running maximum energy of the buffered frames (mode 0) or the
 *       energy function's theoretical maximum (mode 1).
 *   R8  uniform energy: the sum of the buffered energy maps (the average of
 *       Sec. 3.2 up to a positive factor, which changes no comparison).
 *   R9  carving: per iteration the gradient is recomputed on the carved frames,
 *       the motion term is carved along with the frames (Sec. 3.2, 3.3).
 *   R14 forward energy (Sec. 2, the forward energy of the related work): the
 *       cost of a seam is also charged, with integer weight wf, the luma
 *       differences its removal creates between pixels that become neighbours,
 *       summed over the buffer's frames.  Entering (i,j) costs the horizontal
 *       term CU = |Y(i,j+1) - Y(i,j-1)| (0 in the first and last column, where
 *       no pair is created); coming from (i-1,j-1) adds |Y(i-1,j) - Y(i,j-1)|,
 *       from (i-1,j+1) adds |Y(i-1,j) - Y(i,j+1)|, from (i-1,j) nothing.  The
 *       buffer scan keeps the backward energy e of Sec. 3.3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------- */
/* R1: luma of one RGB pixel (Sec. 3.3 computes energy on the frame; the
 * frame's intensity is taken as integer BT.601 luma).                        */
static int luma_of(const uint8_t *px) {
    return (77 * (int)px[0] + 150 * (int)px[1] + 29 * (int)px[2] + 128) >> 8;
}

int orc_luma(const uint8_t *rgb, int H, int W, uint8_t *Y) {
    if (H < 1 || W < 1) return ORC_EINVAL;
    for (long p = 0; p < (long)H * W; ++p) Y[p] = (uint8_t)luma_of(rgb + 3 * p);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R2: Sobel gradient energy (Sec. 3.3, "Sobel gradient energy").
 * Gx = [-1 0 1; -2 0 2; -1 0 1] correlated with Y, Gy = its transpose,
 * G = |Gx| + |Gy|, pixels outside the frame take the value of the nearest
 * pixel inside it.                                                           */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int orc_sobel(const uint8_t *Y, int H, int W, int32_t *G) {
    if (H < 1 || W < 1) return ORC_EINVAL;
    for (int i = 0; i < H; ++i) {
        for (int j = 0; j < W; ++j) {
            int y[3][3];
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b)
                    y[a + 1][b + 1] = Y[(long)clampi(i + a, 0, H - 1) * W + clampi(j + b, 0, W - 1)];
            int gx = (y[0][2] + 2 * y[1][2] + y[2][2]) - (y[0][0] + 2 * y[1][0] + y[2][0]);
            int gy = (y[2][0] + 2 * y[2][1] + y[2][2]) - (y[0][0] + 2 * y[0][1] + y[0][2]);
            G[(long)i * W + j] = abs(gx) + abs(gy);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R3: frame difference of the original luma (Sec. 3.3): D_0 = 0,
 * D_t = |Y_t - Y_{t-1}|.  frames: [T][H][W][3], D: [T][H][W].                */
int orc_motion(const uint8_t *frames, int T, int H, int W, uint8_t *D) {
    if (T < 1 || H < 1 || W < 1) return ORC_EINVAL;
    long hw = (long)H * W;
    for (int t = 0; t < T; ++t) {
        for (long p = 0; p < hw; ++p) {
            if (t == 0) {
                D[p] = 0;
            } else {
                int a = luma_of(frames + 3 * ((long)t * hw + p));
                int b = luma_of(frames + 3 * ((long)(t - 1) * hw + p));
                D[(long)t * hw + p] = (uint8_t)abs(a - b);
            }
        }
    }
    return ORC_OK;
}

/* R3: motion-aware energy of every frame of a clip (Sec. 3.3):
 * e_t = wg * Sobel(Y_t) + wm * D_t.  e: [T][H][W] int32.                    */
int orc_energy(const uint8_t *frames, int T, int H, int W, int wg, int wm, int32_t *e) {
    if (T < 1 || H < 1 || W < 1 || wg < 0 || wm < 0) return ORC_EINVAL;
    long hw = (long)H * W;
    uint8_t *Y = (uint8_t *)malloc(hw);
    int32_t *G = (int32_t *)malloc(hw * sizeof(int32_t));
    uint8_t *D = (uint8_t *)malloc(hw * T);
    if (!Y || !G || !D) { free(Y); free(G); free(D); return ORC_ENOMEM; }
    orc_motion(frames, T, H, W, D);
    for (int t = 0; t < T; ++t) {
        orc_luma(frames + 3 * (long)t * hw, H, W, Y);
        orc_sobel(Y, H, W, G);
        for (long p = 0; p < hw; ++p) e[(long)t * hw + p] = wg * G[p] + wm * (int)D[(long)t * hw + p];
    }
    free(Y); free(G); free(D);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R4/R5: the cumulative-energy DP of Eq. 4 with parental labels (Sec. 3.1).
 *   CE(0,j) = E(0,j), L(0,j) = j
 *   CE(i,j) = E(i,j) + min_{j' in {j-1,j,j+1}, 0<=j'<W} CE(i-1,j')
 *   L(i,j)  = L(i-1, j*) with j* the minimising j' (lowest j' on ties)
 *   dir(i,j) = j* - j + 1 in {0,1,2} (the "indicator" the paper records to
 *   trace a seam back); dir(0,j) = 1.
 * CE, L, dir: [H][W].                                                        */
int orc_dp(const int32_t *E, int H, int W, int64_t *CE, int32_t *L, uint8_t *dir) {
    if (H < 1 || W < 1) return ORC_EINVAL;
    for (int j = 0; j < W; ++j) { CE[j] = E[j]; L[j] = j; dir[j] = 1; }
    for (int i = 1; i < H; ++i) {
        const int64_t *up = CE + (long)(i - 1) * W;
        for (int j = 0; j < W; ++j) {
            int best_j = -1;
            for (int jj = j - 1; jj <= j + 1; ++jj) {
                if (jj < 0 || jj >= W) continue;
                if (best_j < 0 || up[jj] < up[best_j]) best_j = jj; /* strict: lowest column on ties */
            }
            long p = (long)i * W + j;
            CE[p] = (int64_t)E[p] + up[best_j];
            L[p] = L[(long)(i - 1) * W + best_j];
            dir[p] = (uint8_t)(best_j - j + 1);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R14: forward terms of one luma frame [H][W]:
 *   CU(i,j) = |Y(i,j+1) - Y(i,j-1)| for 0 < j < W-1, else 0
 *   A(i,j)  = |Y(i-1,j) - Y(i,j-1)| for i >= 1 and j >= 1, else 0
 *   B(i,j)  = |Y(i-1,j) - Y(i,j+1)| for i >= 1 and j <= W-2, else 0
 * CU is the pair a seam through (i,j) joins in row i; A (B) the pair it joins
 * between rows i-1 and i when it arrives from the upper left (right).        */
int orc_forward_terms(const uint8_t *Y, int H, int W, int32_t *CU, int32_t *A, int32_t *B) {
    if (H < 1 || W < 1) return ORC_EINVAL;
    for (int i = 0; i < H; ++i) {
        const uint8_t *r = Y + (long)i * W;
        const uint8_t *u = i > 0 ? Y + (long)(i - 1) * W : NULL;
        for (int j = 0; j < W; ++j) {
            long p = (long)i * W + j;
            CU[p] = (j > 0 && j < W - 1) ? abs((int)r[j + 1] - (int)r[j - 1]) : 0;
            A[p] = (u && j >= 1) ? abs((int)u[j] - (int)r[j - 1]) : 0;
            B[p] = (u && j <= W - 2) ? abs((int)u[j] - (int)r[j + 1]) : 0;
        }
    }
    return ORC_OK;
}

/* R4/R5 with R14: the DP of Eq. 4 with parental labels where the move from
 * (i-1,j-1) costs wf*A(i,j) extra and the move from (i-1,j+1) wf*B(i,j); E
 * already holds the per-pixel part (backward energy + wf*CU).
 *   CE(i,j) = E(i,j) + min( CE(i-1,j-1) + wf*A(i,j), CE(i-1,j), CE(i-1,j+1) + wf*B(i,j) )
 * over the neighbours inside the row, lowest j' on ties, labels and
 * indicators as in orc_dp.  With wf = 0 this is orc_dp.                      */
int orc_dp_fwd(const int32_t *E, const int32_t *A, const int32_t *B, int wf, int H, int W,
               int64_t *CE, int32_t *L, uint8_t *dir) {
    if (H < 1 || W < 1) return ORC_EINVAL;
    for (int j = 0; j < W; ++j) { CE[j] = E[j]; L[j] = j; dir[j] = 1; }
    for (int i = 1; i < H; ++i) {
        const int64_t *up = CE + (long)(i - 1) * W;
        for (int j = 0; j < W; ++j) {
            long p = (long)i * W + j;
            int best_j = -1;
            int64_t best = 0;
            for (int jj = j - 1; jj <= j + 1; ++jj) {
                if (jj < 0 || jj >= W) continue;
                int64_t c = up[jj];
                if (jj == j - 1) c += (int64_t)wf * A[p];
                if (jj == j + 1) c += (int64_t)wf * B[p];
                if (best_j < 0 || c < best) { best_j = jj; best = c; } /* lowest column on ties */
            }
            CE[p] = (int64_t)E[p] + best;
            L[p] = L[(long)(i - 1) * W + best_j];
            dir[p] = (uint8_t)(best_j - j + 1);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R6: Eq. 6 -- for every parent present in the last row, its child of least
 * (CE, column); then the `cap` lowest of those by (CE, column).  Writes the
 * chosen end columns in that order to cols[] and returns how many (k_eff).  */
typedef struct { int64_t ce; int32_t col; } orc_cand;

static int cand_less(const orc_cand *a, const orc_cand *b) {
    return a->ce < b->ce || (a->ce == b->ce && a->col < b->col);
}

int orc_select(const int64_t *ce_last, const int32_t *lab_last, int W, int cap, int32_t *cols) {
    if (W < 1 || cap < 0) return -ORC_EINVAL;
    /* best child per parent label; parents are row-0 columns, so 0 <= label < W */
    orc_cand *best = (orc_cand *)malloc(sizeof(orc_cand) * W);
    orc_cand *list = (orc_cand *)malloc(sizeof(orc_cand) * W);
    if (!best || !list) { free(best); free(list); return -ORC_ENOMEM; }
    for (int a = 0; a < W; ++a) best[a].col = -1;
    for (int j = 0; j < W; ++j) {
        orc_cand c = { ce_last[j], j };
        int a = lab_last[j];
        if (best[a].col < 0 || cand_less(&c, &best[a])) best[a] = c;
    }
    int n = 0;
    for (int a = 0; a < W; ++a) if (best[a].col >= 0) list[n++] = best[a];
    /* plain insertion sort by (CE, column) */
    for (int x = 1; x < n; ++x) {
        orc_cand v = list[x];
        int y = x - 1;
        while (y >= 0 && cand_less(&v, &list[y])) { list[y + 1] = list[y]; --y; }
        list[y + 1] = v;
    }
    int k_eff = n < cap ? n : cap;
    for (int s = 0; s < k_eff; ++s) cols[s] = list[s].col;
    free(best); free(list);
    return k_eff;
}

/* Trace one seam back from (H-1, end_col) through the recorded indicators
 * (Sec. 3.1: "Seam removal can thus be done through tracing back the
 * indicators").  path: [H], path[i] = column of the seam in row i.           */
int orc_backtrack(const uint8_t *dir, int H, int W, int end_col, int32_t *path) {
    if (H < 1 || end_col < 0 || end_col >= W) return ORC_EINVAL;
    path[H - 1] = end_col;
    for (int i = H - 1; i >= 1; --i) path[i - 1] = path[i] + (int)dir[(long)i * W + path[i]] - 1;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R7: ASDE (Eq. 7-8) in exact integers.  For a buffer of n energy maps,
 * Std(i,j) = sqrt(n*S2 - S1^2) / n with S1 = sum_t e, S2 = sum_t e^2, so
 * ASDE = sum_ij sqrt(Q_ij) / (n*H*W), Q = n*S2 - S1^2.  The sum is kept as
 * A = sum_ij floor(sqrt(65536 * Q_ij)) ~= 256 * sum_ij sqrt(Q_ij).           */
static uint64_t isqrt_floor(uint64_t x) {
    uint64_t s = (uint64_t)sqrt((double)x);
    while (s > 0 && s * s > x) --s;            /* enforce s^2 <= x            */
    while ((s + 1) * (s + 1) <= x) ++s;        /* enforce x < (s+1)^2         */
    return s;
}

uint64_t orc_isqrt(uint64_t x) { return isqrt_floor(x); }

int orc_asde_sum(const int32_t *e, int n, int H, int W, int64_t *A_out) {
    if (n < 1 || H < 1 || W < 1) return ORC_EINVAL;
    long hw = (long)H * W;
    int64_t A = 0;
    for (long p = 0; p < hw; ++p) {
        int64_t s1 = 0, s2 = 0;
        for (int t = 0; t < n; ++t) {
            int64_t v = e[(long)t * hw + p];
            s1 += v;
            s2 += v * v;
        }
        int64_t Q = (int64_t)n * s2 - s1 * s1;
        A += (int64_t)isqrt_floor((uint64_t)Q << 16);
    }
    *A_out = A;
    return ORC_OK;
}

/* Eq. 9: phi(n) = alpha*sqrt(((M - M/n)^2 + (n-1)(M/n)^2)/n), which equals
 * alpha*M*sqrt(n-1)/n.  ASDE > phi(n)  <=>  sum sqrt(Q) > alpha*M*sqrt(n-1)*H*W,
 * decided here as (double)A > 256*alpha*M*sqrt(n-1)*H*W, the product taken
 * left to right in IEEE double.                                               */
double orc_threshold(int n, int64_t M, int H, int W, double alpha) {
    double thr = 256.0 * alpha;
    thr = thr * (double)M;
    thr = thr * sqrt((double)(n - 1));
    thr = thr * (double)H;
    thr = thr * (double)W;
    return thr;
}

int orc_exceeds(int64_t A, int n, int64_t M, int H, int W, double alpha) {
    if (n < 2) return 0;
    return (double)A > orc_threshold(n, M, H, W, alpha);
}

/* R7: the dynamic spatiotemporal buffer of Sec. 3.2.  Frames join one at a
 * time; after frame f joins a buffer of n frames the ASDE is tested against
 * phi(n).  If it exceeds, the buffer is fixed without f and f starts the next
 * buffer.  starts[] receives the first frame of every buffer plus a final
 * starts[n_buffers] = T.  e: [T][H][W].                                      */
int orc_scan(const int32_t *e, int T, int H, int W, double alpha, int t_max, int maxval_mode,
             int64_t maxval_theory, int32_t *starts, int *n_buffers) {
    if (T < 1 || H < 1 || W < 1 || t_max < 1) return ORC_EINVAL;
    long hw = (long)H * W;
    int64_t *S1 = (int64_t *)calloc(hw, sizeof(int64_t));
    int64_t *S2 = (int64_t *)calloc(hw, sizeof(int64_t));
    if (!S1 || !S2) { free(S1); free(S2); return ORC_ENOMEM; }
    int nb = 0, start = 0, n = 0;
    int64_t M = 0;
    for (int f = 0; f < T; ++f) {
        const int32_t *ef = e + (long)f * hw;
        int64_t emax = 0;
        for (long p = 0; p < hw; ++p) if (ef[p] > emax) emax = ef[p];
        /* candidate buffer = current buffer + frame f */
        int n1 = n + 1;
        int64_t M1 = maxval_mode == 1 ? maxval_theory : (emax > M ? emax : M);
        int64_t A = 0;
        for (long p = 0; p < hw; ++p) {
            int64_t a1 = S1[p] + ef[p];
            int64_t a2 = S2[p] + (int64_t)ef[p] * ef[p];
            int64_t Q = (int64_t)n1 * a2 - a1 * a1;
            A += (int64_t)isqrt_floor((uint64_t)Q << 16);
        }
        if (orc_exceeds(A, n1, M1, H, W, alpha)) {
            /* buffer [start, f) is fixed; f starts the next one */
            starts[nb++] = start;
            start = f;
            n = 1;
            M = maxval_mode == 1 ? maxval_theory : emax;
            for (long p = 0; p < hw; ++p) { S1[p] = ef[p]; S2[p] = (int64_t)ef[p] * ef[p]; }
        } else {
            n = n1;
            M = M1;
            for (long p = 0; p < hw; ++p) { S1[p] += ef[p]; S2[p] += (int64_t)ef[p] * ef[p]; }
            if (n == t_max) {
                starts[nb++] = start;
                start = f + 1;
                n = 0;
                M = 0;
                memset(S1, 0, hw * sizeof(int64_t));
                memset(S2, 0, hw * sizeof(int64_t));
            }
        }
    }
    if (n > 0) starts[nb++] = start;
    starts[nb] = T;
    *n_buffers = nb;
    free(S1); free(S2);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R8/R9: carve one fixed buffer of Tb frames to width `target` (Sec. 3.1 and
 * 3.2: the same seams are removed from every frame of the buffer).
 *   frames: [Tb][H][W0][3]   D: [Tb][H][W0] motion maps of these frames
 *   out:    [Tb][H][target][3]
 *   seams:  [W0-target][H] original column of every removed pixel, seams in
 *           removal order (iteration, then rank by (CE, column)); may be NULL
 *   k_eff:  per-iteration seam counts (up to W0-target entries); may be NULL
 * Returns the number of iterations, or a negative error.                    */
int orc_carve_buffer(const uint8_t *frames, const uint8_t *D, int Tb, int H, int W0, int target,
                     int k, int wg, int wm, int wf, uint8_t *out, int16_t *seams,
                     int32_t *k_eff_out) {
    if (Tb < 1 || H < 1 || W0 < 1 || target < 1 || target > W0 || k < 1 || wf < 0)
        return -ORC_EINVAL;
    long hw0 = (long)H * W0;
    uint8_t *rgb = (uint8_t *)malloc(3 * hw0 * Tb);   /* carved colour frames  */
    uint8_t *dm = (uint8_t *)malloc(hw0 * Tb);        /* carved motion maps    */
    int32_t *orig = (int32_t *)malloc(sizeof(int32_t) * hw0); /* original column */
    int32_t *E = (int32_t *)malloc(sizeof(int32_t) * hw0);
    int32_t *G = (int32_t *)malloc(sizeof(int32_t) * hw0);
    uint8_t *Y = (uint8_t *)malloc(hw0);
    int64_t *CE = (int64_t *)malloc(sizeof(int64_t) * hw0);
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * hw0);
    uint8_t *dir = (uint8_t *)malloc(hw0);
    uint8_t *kill = (uint8_t *)malloc(hw0);
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * W0);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * H);
    /* R14: one frame's forward terms, and the buffer's sums of A and B */
    int32_t *fcu = (int32_t *)malloc(sizeof(int32_t) * hw0);
    int32_t *fa = (int32_t *)malloc(sizeof(int32_t) * hw0);
    int32_t *fb = (int32_t *)malloc(sizeof(int32_t) * hw0);
    int32_t *sa = (int32_t *)malloc(sizeof(int32_t) * hw0);
    int32_t *sb = (int32_t *)malloc(sizeof(int32_t) * hw0);
    int rc = 0;
    if (!rgb || !dm || !orig || !E || !G || !Y || !CE || !L || !dir || !kill || !cols || !path ||
        !fcu || !fa || !fb || !sa || !sb) {
        rc = -ORC_ENOMEM;
        goto done;
    }
    memcpy(rgb, frames, 3 * hw0 * Tb);
    memcpy(dm, D, hw0 * Tb);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W0; ++j) orig[(long)i * W0 + j] = j;

    int W = W0, removed = 0, iters = 0;
    while (W > target) {
        long hw = (long)H * W;
        /* uniform energy of the buffer at the current width (R8, R9) */
        memset(E, 0, sizeof(int32_t) * hw);
        memset(sa, 0, sizeof(int32_t) * hw);
        memset(sb, 0, sizeof(int32_t) * hw);
        for (int t = 0; t < Tb; ++t) {
            orc_luma(rgb + 3 * (long)t * hw, H, W, Y);
            orc_sobel(Y, H, W, G);
            for (long p = 0; p < hw; ++p) E[p] += wg * G[p] + wm * (int)dm[(long)t * hw + p];
            if (wf > 0) {   /* R14, summed over the buffer like the energy (R8) */
                orc_forward_terms(Y, H, W, fcu, fa, fb);
                for (long p = 0; p < hw; ++p) {
                    E[p] += wf * fcu[p];
                    sa[p] += fa[p];
                    sb[p] += fb[p];
                }
            }
        }
        if (wf > 0) orc_dp_fwd(E, sa, sb, wf, H, W, CE, L, dir);
        else orc_dp(E, H, W, CE, L, dir);
        int cap = k < W - target ? k : W - target;
        int k_eff = orc_select(CE + (long)(H - 1) * W, L + (long)(H - 1) * W, W, cap, cols);
        if (k_eff < 1) { rc = -ORC_EINVAL; goto done; }
        memset(kill, 0, hw);
        for (int s = 0; s < k_eff; ++s) {
            orc_backtrack(dir, H, W, cols[s], path);
            for (int i = 0; i < H; ++i) {
                long p = (long)i * W + path[i];
                kill[p] = 1;
                if (seams) seams[(long)(removed + s) * H + i] = (int16_t)orig[p];
            }
        }
        /* delete the marked pixels row by row from every carved array; the
         * arrays are compacted in place, frame by frame in storage order, so
         * no write ever lands ahead of the next read */
        int Wn = W - k_eff;
        for (int i = 0; i < H; ++i) {
            int q = 0;
            for (int j = 0; j < W; ++j) {
                long p = (long)i * W + j;
                if (kill[p]) continue;
                orig[(long)i * Wn + q] = orig[p];
                ++q;
            }
            if (q != Wn) { rc = -ORC_EINVAL; goto done; } /* every row narrows by k_eff */
        }
        for (int t = 0; t < Tb; ++t) {
            for (int i = 0; i < H; ++i) {
                int q = 0;
                for (int j = 0; j < W; ++j) {
                    long p = (long)i * W + j;
                    if (kill[p]) continue;
                    long pn = (long)i * Wn + q;
                    const uint8_t *src = rgb + 3 * ((long)t * hw + p);
                    uint8_t *dst = rgb + 3 * ((long)t * H * Wn + pn);
                    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2];
                    dm[(long)t * H * Wn + pn] = dm[(long)t * hw + p];
                    ++q;
                }
            }
        }
        if (k_eff_out) k_eff_out[iters] = k_eff;
        W = Wn;
        removed += k_eff;
        ++iters;
    }
    memcpy(out, rgb, 3 * (long)Tb * H * target);
    rc = iters;
done:
    free(rgb); free(dm); free(orig); free(E); free(G); free(Y); free(CE); free(L);
    free(dir); free(kill); free(cols); free(path); free(fcu); free(fa); free(fb); free(sa);
    free(sb);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* The whole clip: energy (Sec. 3.3), buffer scan (Sec. 3.2), then every fixed
 * buffer carved to `target` (Sec. 3.1/3.2), with forward terms of weight wf
 * in the seam cost when wf > 0 (R14).  use_buffer = 0 gives per-frame
 * SCPL (every frame its own buffer); with k = 1 that is classic seam carving
 * applied frame by frame (the paper's "raw" comparison).
 *   out:   [T][H][target][3]
 *   starts: [T+1] buffer starts, n_buffers receives the count
 *   seams: [n_buffers][W0-target][H] or NULL                                 */
int orc_carve(const uint8_t *frames, int T, int H, int W0, int target, int k, int wg, int wm,
              int wf, double alpha, int t_max, int use_buffer, int maxval_mode, uint8_t *out,
              int32_t *starts, int *n_buffers, int16_t *seams) {
    if (T < 1 || H < 1 || W0 < 1 || target < 1 || target > W0 || k < 1) return ORC_EINVAL;
    long hw = (long)H * W0;
    int32_t *e = (int32_t *)malloc(sizeof(int32_t) * hw * T);
    uint8_t *D = (uint8_t *)malloc(hw * T);
    if (!e || !D) { free(e); free(D); return ORC_ENOMEM; }
    int rc = orc_energy(frames, T, H, W0, wg, wm, e);
    if (rc == ORC_OK) rc = orc_motion(frames, T, H, W0, D);
    if (rc == ORC_OK) {
        int64_t theory = (int64_t)255 * (8 * wg + wm);
        rc = orc_scan(e, T, H, W0, alpha, use_buffer ? t_max : 1, maxval_mode, theory, starts,
                      n_buffers);
    }
    for (int b = 0; rc == ORC_OK && b < *n_buffers; ++b) {
        int t0 = starts[b], tb = starts[b + 1] - starts[b];
        int it = orc_carve_buffer(frames + 3 * (long)t0 * hw, D + (long)t0 * hw, tb, H, W0, target,
                                  k, wg, wm, wf, out + 3 * (long)t0 * H * target,
                                  seams ? seams + (long)b * (W0 - target) * H : NULL, NULL);
        if (it < 0) rc = -it;
    }
    free(e); free(D);
    return rc;
}
