/*
 * scpl.h -- C ABI of libscpl, GB300 (sm_103a) video retargeting by Seam
 * Carving with Parental Labeling (SCPL), arXiv 1903.03180.
 *
 * Conventions shared by every entry point:
 *  - Pointers marked [device] are CUDA device pointers owned by the caller;
 *    pointers marked [host] are ordinary host memory owned by the caller.
 *    The library never frees caller memory.  The library owns its own
 *    workspaces, grows them on demand and frees them in scpl_destroy.
 *  - Frames are uint8 RGB, layout [T][H][W][3], contiguous (HWC).
 *  - Work is issued on the handle's stream.  Entry points that return results
 *    to [host] pointers synchronise that stream before returning; the others
 *    return as soon as the work is queued.
 *  - Every entry point returns an scpl_status; nothing throws.  On a non-zero
 *    status scpl_last_error() describes it.  After SCPL_EINVAL, SCPL_ENOMEM,
 *    SCPL_EOVERFLOW, SCPL_ETIMEOUT or SCPL_ECANCELED the handle stays usable.  After
 *    SCPL_ECUDA it is usable unless the CUDA context itself was lost.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef SCPL_H
#define SCPL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scpl_ctx *scpl_handle;

typedef enum {
    SCPL_OK = 0,
    SCPL_EINVAL = 1,    /* bad argument (sizes, pointers, parameters)          */
    SCPL_ENOMEM = 2,    /* a workspace could not be allocated                  */
    SCPL_ECUDA = 3,     /* a CUDA call failed                                  */
    SCPL_ETIMEOUT = 4,  /* a bounded device-side wait ran out                  */
    SCPL_EOVERFLOW = 5, /* the sizes could overflow the exact integer sums     */
    SCPL_ECANCELED = 6  /* a server job was cancelled (scpl_server_cancel)     */
} scpl_status;

/* Parameters of the method.
 *  alpha        Eq. 9's alpha (the paper's useful range is [0.15, 0.25]).
 *  wg, wm       integer weights of the gradient and motion energies,
 *               e = wg*|Sobel(Y)|_1 + wm*|Y_t - Y_{t-1}| (Sec. 3.3).
 *  t_max        cap on frames per spatiotemporal buffer (1 <= t_max <= 1024).
 *  use_buffer   0: every frame is its own buffer (per-frame SCPL; with k = 1
 *               this is classic seam carving frame by frame).
 *  maxval_mode  Eq. 9's maxval: 0 = running maximum of the buffered energy
 *               maps, 1 = the energy function's maximum 255*(8*wg + wm).
 *  wf           weight of the forward terms in the seam cost (0..255; 0 =
 *               the paper's backward energy only).  With wf > 0 a seam also
 *               pays, per frame of its buffer, wf times the luma differences
 *               its removal creates between pixels that become neighbours
 *               (the forward energy the paper's Sec. 2 names): in its own
 *               row |Y(i,j+1) - Y(i,j-1)| (nothing in the first and last
 *               column), and between rows i-1 and i |Y(i-1,j) - Y(i,j-1)|
 *               when it arrives from the upper left, |Y(i-1,j) - Y(i,j+1)|
 *               from the upper right.  The buffer scan (Eq. 7-9) keeps the
 *               backward energy.  wf > 0 needs buffers of at most 256 frames
 *               (t_max <= 256, or use_buffer 0); widths up to 4096 carve
 *               with the cluster DP, wider ones with the single-CTA DP.
 *               scpl_seams and scpl_seams_noalloc take a caller's energy map
 *               and charge no forward terms.                                */
typedef struct {
    double alpha;
    int wg, wm;
    int t_max;
    int use_buffer;
    int maxval_mode;
    int wf;
} scpl_params;

/* Fill p with the defaults: alpha 0.20, wg 1, wm 2, t_max 128, buffer on,
 * maxval_mode 0, wf 0. */
void scpl_default_params(scpl_params *p);

/* Create a handle bound to the current CUDA device and to `stream`
 * (a cudaStream_t passed as void*; NULL = the legacy default stream).
 * Returns SCPL_EINVAL for a NULL out or invalid parameters. */
scpl_status scpl_create(const scpl_params *p, void *stream, scpl_handle *out);

/* Rebind the handle to another stream of the same device. */
scpl_status scpl_set_stream(scpl_handle h, void *stream);

/* Release every workspace of the handle.  NULL is accepted. */
void scpl_destroy(scpl_handle h);

/* Text of the last error on this handle ("" if none).  The string lives until
 * the next call on the handle. */
const char *scpl_last_error(scpl_handle h);

/* Per-frame energy of a clip (Sec. 3.3): integer BT.601 luma
 * Y = (77R + 150G + 29B + 128) >> 8, Sobel gradient |Gx| + |Gy| with a
 * replicate border, frame difference D_t = |Y_t - Y_{t-1}| with D_0 = 0,
 * e_t = wg*G_t + wm*D_t.
 *   frames  [device] uint8 [T][H][W][3]
 *   energy  [device] int32 [T][H][W], written
 * Asynchronous.  SCPL_EINVAL if T, H or W < 1 or a pointer is NULL. */
scpl_status scpl_energy(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                        int32_t *energy);

/* Spatiotemporal buffer boundaries of a clip (Sec. 3.2, Eq. 7-9).  Frames
 * join the open buffer one by one; a frame whose joining would make the
 * buffer's ASDE exceed phi(n) starts the next buffer instead; a buffer is also
 * closed at t_max frames and at the end of the clip.  The comparison is made
 * exactly: A = sum_ij floor(256*sqrt(n*S2_ij - S1_ij^2)) (S1, S2 the sums of
 * e and e^2 over the buffer) against 256*alpha*M*sqrt(n-1)*H*W in IEEE double.
 *   frames        [device] uint8 [T][H][W][3]
 *   buffer_starts [host] int32 [T+1]: first frame of each buffer, then T
 *   n_buffers     [host] receives the number of buffers
 * Synchronises the stream.  SCPL_ETIMEOUT if the device-wide per-frame
 * reduction waited longer than its limit (the handle stays usable). */
scpl_status scpl_scan(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                      int32_t *buffer_starts, int *n_buffers);

/* scpl_scan plus the integers each decision used (diagnostic): for every
 * frame t, A[t] = sum over pixels of floor(sqrt(65536 (n S2 - S1^2))) with
 * frame t added to the open buffer (Eq. 7-8 scaled by 256 n), and emax[t] =
 * the maximum energy of frame t (Eq. 9's maxval is the running maximum of
 * these, or the theoretical one).
 *   A     [host] int64 [T]
 *   emax  [host] int32 [T]
 * Synchronises the stream. */
scpl_status scpl_scan_stats(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                            int32_t *buffer_starts, int *n_buffers, int64_t *A, int32_t *emax);

/* scpl_scan on frames that are still arriving (streaming ingest): the buffer
 * decisions start while a producer is still copying later frames in.  The
 * producer announces each chunk of `chunk` frames by raising a device counter
 * to the number of chunks complete; the scan reads frame t only once
 * *arrived >= t / chunk + 1.
 *   arrived  [device] uint32, raised by the producer on another stream with
 *            scpl_signal_arrival after each chunk's copy.  (A stream memory
 *            operation needs no SM; a kernel on another stream may not be
 *            scheduled while the scan's persistent grid holds every SM.)
 *   chunk    frames per announcement, >= 1
 * The result equals scpl_scan's on the complete frames.  A wait for a frame
 * is bounded by the handle's wait limit (scpl_set_wait_limit): a counter that
 * stops short ends the call with SCPL_ETIMEOUT, buffer_starts unwritten, and
 * the handle stays usable.  Synchronises the stream. */
scpl_status scpl_scan_arrivals(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                               const uint32_t *arrived, int chunk, int32_t *buffer_starts,
                               int *n_buffers);

/* Enqueue on `stream` (a cudaStream_t, NULL = the legacy default stream) a
 * write of `value` to the device word *counter, after the stream's earlier
 * work and a memory fence: the announcement scpl_scan_arrivals waits for.
 * Needs no handle.  SCPL_EINVAL for a NULL counter, SCPL_ECUDA if the driver
 * lacks stream memory operations. */
scpl_status scpl_signal_arrival(void *stream, uint32_t *counter, uint32_t value);

/* Widen a clip by seam insertion (the inverse use of seam carving; the
 * insertion rule is Avidan & Shamir's).  To add m = target_W - W columns the
 * clip is carved to W - m by SCPL (as scpl_carve does, on a scratch copy);
 * the m seams removed from each spatiotemporal buffer, in original columns,
 * are inserted into every frame of that buffer.  Each row keeps its original
 * pixels in order and, after each seam pixel x, gets a new pixel that is the
 * rounded mean (a + b + 1) >> 1, per channel, of pixels x and x+1 (x itself
 * at the last column).
 *   frames        [device] uint8 [T][H][W][3]
 *   out           [device] uint8 [T][H][target_W][3]
 *   buffer_starts [host] int32 [T+1] or NULL; n_buffers [host] or NULL
 * W <= target_W <= 2W-2 and W <= 8192 (else SCPL_EINVAL); k >= 1.
 * Synchronises the stream. */
scpl_status scpl_enlarge(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                         int target_W, int k, uint8_t *out, int32_t *buffer_starts,
                         int *n_buffers);

/* Enlarge a clip along both axes (Sec. 2 retargets either way): the width
 * grows first, exactly as scpl_enlarge does; the height then grows as the
 * width of the transposed result (its horizontal seams are the vertical seams
 * of the transposed frames, found by the same SCPL carving with its own buffer
 * scan), and the result is transposed back.  A target equal to its size adds
 * nothing along that axis.
 *   frames [device] uint8 [T][H][W][3]
 *   out    [device] uint8 [T][target_H][target_W][3]
 * W <= target_W <= max(W, 2W-2), H <= target_H <= max(H, 2H-2), W <= 8192,
 * and H <= 8192 when the height grows (else SCPL_EINVAL); k >= 1.  Scratch
 * copies of the intermediate clips are the handle's.  Synchronises the
 * stream. */
scpl_status scpl_enlarge_job(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                             int target_W, int target_H, int k, uint8_t *out);

/* Sharpness of blends of consecutive frames (a measure of temporal
 * consistency; a numeric stand-in for Fig. 9 of Sec. 4): on a nearly static
 * clip, frames carved with the same seams blend into a sharp image, frames
 * carved independently into a blurred one.  For every run of `window`
 * consecutive frames t .. t+window-1 (t = 0 .. T-window), the blend B is the
 * sum of their integer BT.601 luma maps; *num adds the L1 Sobel magnitude
 * |Gx|+|Gy| (3x3, replicate border) of B, and *den the same magnitude of each
 * frame of the run.  num <= den; num / den is 1 for static content.
 *   frames   [device] uint8 [T][H][W][3]
 *   num, den [host] exact sums (0 and 0 when T < window)
 * SCPL_EINVAL for window outside [1, 64].  Synchronises the stream. */
scpl_status scpl_blend_sharpness(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                                 int window, int64_t *num, int64_t *den);

/* The integer square root of the buffer decision (Sec. 3.2, Eq. 7-8): the
 * scan adds floor(sqrt(65536 * Q)) over the pixels, with Q = n*S2 - S1^2 the
 * scaled spread of a pixel's energy over the n buffered frames.  This runs the
 * scan's own device routine on caller values, so that it can be checked
 * against an exact integer square root at its edges.
 *   x [device] uint64 [n], each below 2^53 (the scan's values stay below
 *     2^51; larger values give an unspecified result, never a fault)
 *   r [device] uint32 [n], written: r[i] = floor(sqrt(x[i]))
 *   stream cudaStream_t as void* (NULL = legacy default stream); asynchronous
 * SCPL_EINVAL for n < 0 or NULL arrays with n > 0; SCPL_ECUDA if the launch
 * fails. */
scpl_status scpl_isqrt(const uint64_t *x, uint32_t *r, long n, void *stream);

/* Bound, in nanoseconds, of each device-wide wait of the handle's buffer
 * scans: the per-round reduction across the scan's CTAs and the waits for
 * arriving frames (default 2e9).  A wait that runs out makes its call return
 * SCPL_ETIMEOUT instead of hanging.  (The carving kernels wait only within a
 * thread-block cluster, under a fixed 2 s bound.)  SCPL_EINVAL outside
 * [1e5, 6e10]. */
scpl_status scpl_set_wait_limit(scpl_handle h, uint64_t ns);

/* One SCPL iteration on an energy map (Sec. 3.1, Eq. 4-6): the cumulative
 * energy DP carrying each pixel's row-0 parent (lowest column on ties), the
 * least-(CE, column) child of every parent, the k_eff = min(k, #parents)
 * lowest of those by (CE, column), traced back through the recorded
 * directions.
 *   energy  [device] int32 [H][W], values >= 0, column sums < 2^31
 *   cols    [device] int16 [k][H]: cols[s][i] = column of seam s in row i,
 *           seams in rank order; rows s >= k_eff are left untouched
 *   k_eff   [host] receives the number of seams found
 * Synchronises the stream. */
scpl_status scpl_seams(scpl_handle h, const int32_t *energy, int H, int W, int k,
                       int16_t *cols, int *k_eff);

/* Retarget a clip to width target_W (Sec. 3): energy, buffer scan, then for
 * every buffer repeated SCPL iterations on the summed energy of its frames
 * (the gradient recomputed on the carved frames, the motion term carved
 * along), each removing k_eff = min(k, W - target_W, #parents) disjoint seams
 * from every frame of the buffer, until the width is target_W.
 *   frames         [device] uint8 [T][H][W][3]
 *   out            [device] uint8 [T][H][target_W][3], written
 *   buffer_starts  [host] int32 [T+1] or NULL
 *   n_buffers      [host] or NULL
 *   seams          [device] int16 [n_buffers][W - target_W][H] or NULL: for
 *                  every buffer, the original column of every removed pixel,
 *                  seams in removal order (iteration, then rank)
 * Limits: 1 <= T, 1 <= H <= 65535, 2 <= target_W <= W <= 8192, 1 <= k;
 * 255*(8*wg + wm)*min(T, t_max)*H < 2^31 and t_max*(255*(8*wg+wm))^2 < 2^32
 * (else SCPL_EOVERFLOW).  Synchronises the stream (the buffer count decides
 * the launch shapes).  The iterations run as one CUDA graph that loops on the
 * device until every buffer is carved (a conditional WHILE node); the handle
 * keeps that graph and builds a new one when the workspace, the buffer count,
 * k or the seam output changes.  With profiling on (scpl_set_profiling) the
 * iterations are launched from the host instead, each bracketed by events. */
scpl_status scpl_carve(scpl_handle h, const uint8_t *frames, int T, int H, int W, int target_W,
                       int k, uint8_t *out, int32_t *buffer_starts, int *n_buffers,
                       int16_t *seams);

/* Carve one fixed spatiotemporal buffer on its own (Sec. 3.2: once a buffer
 * is fixed, its seams depend on its own frames only, and the same seams are
 * removed from every frame of it).  This is how a clip's buffers are dealt to
 * several GPUs after one scan: a rank carves the frames [t0, t1) of buffer b
 * and gets exactly what scpl_carve gives for those frames of the whole clip.
 * No flush decision is taken: the T frames are one buffer.
 *   frames     [device] uint8 [T][H][W][3]: the buffer's frames
 *   prev_frame [device] uint8 [H][W][3]: the clip's frame t0 - 1, from which
 *              the motion term of the buffer's first frame is taken (R3:
 *              D_t = |Y_t - Y_{t-1}|), or NULL when the buffer starts the clip
 *              (D = 0 there)
 *   out        [device] uint8 [T][H][target_W][3], written
 *   seams      [device] int16 [1][W - target_W][H] or NULL
 * T <= t_max of the handle's parameters (a buffer never holds more; else
 * SCPL_EINVAL); the other limits and errors are scpl_carve's.  Synchronises
 * the stream. */
scpl_status scpl_carve_buffer(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                              const uint8_t *prev_frame, int target_W, int k, uint8_t *out,
                              int16_t *seams);

/* scpl_carve on host memory, through library-owned device buffers.  The
 * frames go up by scpl_copy before the buffer scan reads them; every
 * spatiotemporal buffer is gathered and copied back (scpl_copy, on a copy
 * stream) as soon as it is carved, while the others carve on.  Page-locked
 * host memory is read and written by the copy kernel; pageable memory works
 * too, through the copy engines.
 *   frames [host] uint8 [T][H][W][3]   out [host] uint8 [T][H][target_W][3]
 *   seams  [host] int16 [n_buffers][W - target_W][H] or NULL (size it for T
 *          buffers when the count is not known in advance)
 * Synchronises before returning. */
scpl_status scpl_carve_host(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                            int target_W, int k, uint8_t *out, int32_t *buffer_starts,
                            int *n_buffers, int16_t *seams);

/* scpl_carve_host for n clips of one shape, streamed through two device
 * slots: clip i+1's frames go up on an input stream once clip i's buffer scan
 * has finished, so the upload runs beside clip i's carving; clip i's carved
 * buffers come back on the copy stream while the rest of clip i and then clip
 * i+1 run.  Both directions use scpl_copy.  Clip i+1's scan waits for its
 * upload through stream order only.  Every clip's result equals
 * scpl_carve_host's.
 *   frames    [host] n pointers to uint8 [T][H][W][3] (page-locked)
 *   out       [host] n pointers to uint8 [T][H][target_W][3] (page-locked)
 *   n_buffers [host] int [n] or NULL: each clip's buffer count
 * Synchronises before returning; on an error the clips before the failing
 * one are complete. */
scpl_status scpl_carve_host_many(scpl_handle h, int n, const uint8_t *const *frames, int T,
                                 int H, int W, int target_W, int k, uint8_t *const *out,
                                 int *n_buffers);

/* The bulk transfer of the host-memory entry points (the paper has no
 * counterpart: it moves frames between host and device memory).  Copies
 * `bytes` from src to dst, asynchronously on `stream` (a cudaStream_t as
 * void*, NULL = legacy default stream), where either side may be device
 * memory or page-locked host memory.  When both are addressable by the device
 * and share their offset within 16 bytes, a kernel of 16 CTAs reads or writes
 * the host side over the CPU-GPU link with 16-byte accesses (on a
 * Grace-attached GB300 that holds about 210 GB/s up and 192 GB/s down, where
 * the copy engines were seen to fall to 25-60 GB/s for seconds at a time);
 * otherwise it is cudaMemcpyAsync.  The caller keeps both buffers alive and
 * unchanged until the stream has passed the copy.
 * SCPL_EINVAL for a NULL pointer with bytes > 0; SCPL_ECUDA if the launch or
 * the copy fails. */
scpl_status scpl_copy(void *dst, const void *src, size_t bytes, void *stream);

/* scpl_seams without any memory allocation.  The paper has no counterpart:
 * this exists for callers that must not allocate device memory -- a real-time
 * frame loop that cannot take cudaMalloc's implicit synchronisation of the
 * device, or a host application that hands out all device memory from its
 * own fixed pool and lets no library allocate after start-up.  It computes
 * exactly what scpl_seams computes (one SCPL
 * iteration: Eq. 4 DP with parental labels, Eq. 6 per-parent argmin, the
 * k_eff lowest children traced back), needs no handle, and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   energy  [device] int32 [H][W], read in place
 *   cols    [device] int16 [k][H], written as by scpl_seams
 *   k_eff   [host] receives the number of seams found
 *   stream  cudaStream_t as void* (NULL = legacy default stream)
 * Its scratch is one fixed array of about 9 MiB in device memory, reserved on
 * every GPU that loads the library and held until the process exits.  Limits
 * (else SCPL_EINVAL): H*W <= 2^21, W <= 4096, H <= 65535, k <= 64.  The first call on a
 * device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.  All calls
 * share the one array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and give wrong seams, so serialise them.  Synchronises
 * `stream` before returning.  SCPL_ECUDA if a CUDA call fails. */
scpl_status scpl_seams_noalloc(const int32_t *energy, int H, int W, int k, int16_t *cols,
                               int *k_eff, void *stream);

/* Per-kernel accounting of the handle's launches (not part of the paper: a
 * measurement aid).  While profiling is on, every kernel launch of the handle
 * is bracketed by CUDA events on the handle's stream, and every scpl_carve
 * call adds its kernels' algorithmic bytes, the bytes the method has to move.
 * Per launch, with H rows, W_c the width a buffer is carved at, W_n the width
 * after the iteration, k_e its seam count and T_b its frames:
 *   k_scan        28 per pixel and frame (RGB 3, luma and motion out 2, the
 *                 previous luma 1, S1 and S2 read and written 16, energy 6)
 *   k_energy_init H*(2*T_b*W + 10*W) per buffer (luma and motion of every
 *                 frame, origin map, summed and per-pixel energy out)
 *   k_dp          H*(4.5*W_c + 2*k_e) per buffer (energy read, directions
 *                 written and read back, removal lists)
 *   k_update      H*(12*W_n + 6*k_e) per buffer (origin map and energy read
 *                 and written at the new width, the lists of a row and its
 *                 neighbours; 4*W_n in a buffer's last iteration, which
 *                 compacts only the origin map), plus (3*T_b + 8) per
 *                 recomputed pixel
 *   k_gather      H*target_W*(6*T + 2*n_buffers) per clip (colour in and
 *                 out, the origin map of each buffer)
 * With forward terms (wf > 0) the DP adds 4*W_c per row, the update 8*W_n
 * per row and 4 per recomputed pixel, the initialisation H*(T_b*W + 12*W).
 *   scpl_set_profiling(h, 1) clears the counters and turns accounting on;
 *   scpl_set_profiling(h, 0) turns it off.
 *   scpl_get_stats synchronises the stream and fills *out. */
typedef struct {
    char name[32];
    long long launches;
    double ms;       /* summed event-timed duration of those launches       */
    double bytes;    /* summed algorithmic bytes of those launches          */
} scpl_kernel_stat;

typedef struct {
    int n_buffers;              /* of the last scpl_carve call              */
    int iterations_max;         /* most SCPL iterations of any of its buffers */
    long long iterations_total; /* summed over its buffers                   */
    double carved_px;           /* sum over its buffers and iterations of
                                   H * (width before the iteration)         */
    int n_kernels;
    scpl_kernel_stat kernel[8];
    long long launches;         /* kernel launches of the last scpl_carve call,
                                   every iteration of its device-side loop
                                   included (profiled or not)               */
} scpl_stats;

scpl_status scpl_set_profiling(scpl_handle h, int on);
/* The seams removed in every SCPL iteration of the last scpl_carve (or
 * scpl_carve_host) on the handle: k_eff of buffer 0's iterations in order,
 * then buffer 1's, and so on (Eq. 6: min(k, parents, remaining)).  Writes up
 * to max entries to keff and, if iters is not NULL, each buffer's iteration
 * count to iters [n_buffers]; returns the number of entries (-1 for a NULL
 * handle). */
int scpl_keff_log(scpl_handle h, int32_t *keff, int max, int32_t *iters);
scpl_status scpl_get_stats(scpl_handle h, scpl_stats *out);

/* ------------------------------------------------------------------------
 * Autotuning (no counterpart in the paper).  Per frame size (H, W, in carving
 * orientation) the carving kernels have choices that change only the time.
 * The cluster DP holds V columns per lane, so a warp holds 32V columns, and
 * owns 32V - 2R of them with halo depth R (the rows between halo exchanges):
 * V = 4, R = 32 owns 64; V = 4, R = 16 owns 96; V = 2, R = 16 owns 32 with
 * half the instructions per row and warp.  Its CTAs have 4 or 8 warps (how
 * many CTAs carve one frame, and whether two warps share an SM
 * sub-partition).  The single-CTA DP can replace the cluster, and the update
 * takes 1, 2 or 4 rows per CTA.  A process-wide table holds one choice per
 * size; scpl_carve, scpl_carve_batch and servers use it when an entry exists,
 * and the defaults (R = 32, V = 4, 4 warps, the most update rows that fit)
 * otherwise. */
typedef struct {
    int H, W;
    int dpc_halo;        /* 16 or 32: the cluster DP's R; 0: the single-CTA DP        */
    int dpc_warps;       /* warps per cluster-DP CTA: 4 or 8                            */
    int dpc_lane_cols;   /* columns per lane of the cluster DP: 4, or 2 with R = 16     */
    int update_rows;     /* rows per update CTA: 1, 2 or 4                              */
    float dp_us[7];      /* measured DP times, us (< 0: unusable): R32 x 4 warps, R16 x 4,
                            R32 x 8, R16 x 8 (4 columns a lane), the single-CTA DP,
                            R16 x 4 warps and R16 x 8 warps with 2 columns a lane      */
    float up_us[3];      /* measured update times with 1, 2 and 4 rows, us              */
} scpl_tuning;

/* Measure every choice for (H, W) with k seams per iteration on a scratch
 * workspace (synthetic energy, allocated and freed here) on the handle's
 * stream, record the fastest in the table and return the measurements in
 * *out (may be NULL).  Synchronises the stream. */
scpl_status scpl_tune(scpl_handle h, int H, int W, int k, scpl_tuning *out);
/* Record a known choice (e.g. from a file the caller keeps); the measured
 * fields are not used.  SCPL_EINVAL for an unknown halo or row count. */
scpl_status scpl_tuning_set(const scpl_tuning *t);
/* The recorded choice for (H, W): SCPL_OK, or SCPL_EINVAL if there is none. */
scpl_status scpl_tuning_get(int H, int W, scpl_tuning *out);
void scpl_tuning_clear(void);
/* Copy up to max recorded choices into out (ordered by H, then W); returns
 * how many the table holds (a caller can save them and restore them with
 * scpl_tuning_set, e.g. as a tuning cache kept between processes). */
int scpl_tuning_list(scpl_tuning *out, int max);
/* on != 0: scpl_carve and scpl_carve_batch tune every size they meet for the
 * first time (once per process) before carving it. */
scpl_status scpl_set_autotune(scpl_handle h, int on);

/* ------------------------------------------------------------------------
 * Many clips at once: batching and serving.  The paper carves one video at a
 * time (Sec. 3, 4); it has no counterpart for these entry points.  They run
 * the same kernels as scpl_carve, with every stage launched once for all the
 * clips that are at that stage, and give each clip the same result as
 * scpl_carve gives it alone.
 *
 * A job retargets one clip of T frames from H x W to target_H x target_W.
 * A smaller width is reached by vertical seams (Sec. 3.1); a smaller height
 * by horizontal seams, i.e. the same method on the transposed frames
 * (Sec. 2: seams are vertical or horizontal).  When both shrink the width is
 * carved first.  k is the cap on seams per iteration, as in scpl_carve.
 *  frames  [T][H][W][3]                 device, or host when on_host != 0
 *  out     [T][target_H][target_W][3]   device, or host when on_host != 0
 *  buffer_starts  [host] or NULL, T+1 entries: the spatiotemporal buffers of
 *          the first pass (as scpl_carve returns them), written when that
 *          pass's scan completes
 *  n_buffers, status  written by the library (status = this job's result)
 * The caller keeps frames, out and buffer_starts valid and unchanged until
 * the job has completed.  Host frames should be page-locked for the copies
 * to overlap other work (pageable memory works, synchronously). */
typedef struct {
    const uint8_t *frames;
    int T, H, W;
    int target_W, target_H;
    int k;
    int on_host;
    uint8_t *out;
    int32_t *buffer_starts;
    int n_buffers;
    int status;
} scpl_job;

/* Carve every job; returns when all have completed (host-synchronous).  The
 * work starts after everything queued before on the handle's stream.  The
 * handle keeps the engine and its device memory pool between calls (freed by
 * scpl_destroy).  Each group of same-size passes carves in one launch of a
 * CUDA graph that loops on the device until all of the group's buffers reach
 * their targets (servers carve in chunks with a read-back between them).
 * Returns SCPL_OK if every job succeeded, else the first failing job's status
 * (each job's own result is in jobs[i].status; a job with bad arguments
 * fails alone with SCPL_EINVAL). */
scpl_status scpl_carve_batch(scpl_handle h, scpl_job *jobs, int n_jobs);

/* Device memory one job holds while it runs, as admission counts it: the
 * copies of host frames and outputs, the transposed frames of a horizontal
 * pass, the luma and motion maps, the scan state and the carving workspace of
 * one spatiotemporal buffer.  Each further buffer the scan finds adds
 * scpl_job_footprint_per_buffer bytes when it is found (with forward terms,
 * p->wf > 0, also two 32-bit planes of the pass's padded frame size).  0 for
 * an invalid job. */
size_t scpl_job_footprint(const scpl_params *p, const scpl_job *job);
size_t scpl_job_footprint_per_buffer(const scpl_job *job);

/* A server: continuous batching of retarget jobs on one GPU.
 *  scpl_server_create   hbm_budget = bytes of device memory the admitted jobs
 *                       may hold (0: 90 % of the free memory at creation).
 *  scpl_server_submit   queue a job (the struct is copied; its buffers must
 *                       stay valid until completion).  *ticket identifies it.
 *  scpl_server_progress admit queued jobs in arrival order while their
 *                       footprint fits the budget, and launch the next stage
 *                       of every admitted job whose previous stage finished.
 *                       Jobs admitted while others run share the GPU with
 *                       them.  wait != 0: if nothing could be launched, block
 *                       until some work in flight finishes.
 *  scpl_server_poll     up to max completed jobs since the last poll: their
 *                       tickets and statuses; returns how many.
 *  scpl_server_drain    progress until every submitted job has completed.
 *  scpl_server_cancel   a queued job completes at once with SCPL_ECANCELED;
 *                       an admitted job takes no further stage and completes
 *                       with SCPL_ECANCELED once the launches already made
 *                       for it have finished (its out buffer is then
 *                       unspecified, and may be written until it completes).
 *                       SCPL_EINVAL if the ticket is unknown or the job has
 *                       already finished or failed.
 * Faults are contained per job: a job that cannot fit the budget, or whose
 * device memory the allocator refuses while nothing else runs, completes with
 * SCPL_ENOMEM (a refusal while other jobs run delays it until they release
 * memory); a device-side wait that runs out fails the jobs of that launch with
 * SCPL_ETIMEOUT.  The server stays usable after each.
 * A server is not thread-safe: one host thread drives it. */
typedef struct scpl_server_s *scpl_server;

typedef struct {
    long long submitted, completed, failed;
    int queued, active;
    long long scan_waves;        /* multi-clip scan launches                   */
    long long groups;            /* carving groups (clips of one size per wave) */
    long long chunks;            /* DP + update chunks launched as CUDA graphs */
    long long graphs_built;
    long long kernel_launches;   /* kernels of this library, graph nodes included */
    size_t reserved_bytes, peak_reserved_bytes, budget_bytes;
    long long cancelled;         /* jobs that ended with SCPL_ECANCELED         */
} scpl_server_stats;

/* Counters of the handle's batch engine (zeros before the first
 * scpl_carve_batch): scan waves, groups, graph chunks, kernel launches. */
scpl_status scpl_batch_stats(scpl_handle h, scpl_server_stats *out);

scpl_status scpl_server_create(const scpl_params *p, size_t hbm_budget, void *stream,
                               scpl_server *out);
scpl_status scpl_server_submit(scpl_server s, const scpl_job *job, long long *ticket);
/* on != 0: tune every frame size the first time a job of that size is carved. */
scpl_status scpl_server_set_autotune(scpl_server s, int on);
scpl_status scpl_server_progress(scpl_server s, int wait, int *n_active, int *n_queued);
int scpl_server_poll(scpl_server s, long long *tickets, int *statuses, int max);
scpl_status scpl_server_drain(scpl_server s);
scpl_status scpl_server_cancel(scpl_server s, long long ticket);
/* Fault injection for testing the paths above: after `skip` more device
 * allocations of the server succeed, the next `count` are refused as if the
 * device were out of memory (count = 0 turns it off).  Host-side only: no
 * device work is affected. */
scpl_status scpl_server_refuse_allocations(scpl_server s, long long skip, int count);
scpl_status scpl_server_get_stats(scpl_server s, scpl_server_stats *out);
const char *scpl_server_last_error(scpl_server s);
void scpl_server_destroy(scpl_server s);

#ifdef __cplusplus
}
#endif

#endif /* SCPL_H */
