// Internal declarations of libscpl: device-side data layout and the launchers
// that the C ABI (scpl_api.cu) calls.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace scpl {

constexpr uint64_t KEY_INF = ~0ull;
constexpr uint64_t KEY_DIR_MASK = 0xFFull << 24;   // tie-break / direction byte of a DP key
constexpr uint32_t LABEL_MASK = 0xFFFFFFu;         // 24-bit parent label of a DP key

// Status words written by kernels (DEV_OK and DEV_ETIMEOUT have the values of
// the matching scpl_status; the host maps DEV_EINTERNAL to SCPL_ECUDA).
constexpr int DEV_OK = 0;
constexpr int DEV_ETIMEOUT = 4;
constexpr int DEV_EINTERNAL = 6;   // an internal table held an out-of-range column

// A named NVTX range over a host scope: the library's stages on a profiler's
// timeline (scan, carve, gather, server waves, groups and chunks, tuning).
// Without an attached tool the push and pop return at once.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Per-buffer carving state, one per spatiotemporal buffer, in device memory.
// An iteration's seams are selected by k_dp_select (k_eff > 0 = "pending");
// k_energy then writes the carved arrays to slot ^ 1; the next k_dp_select
// (or the final gather) commits the pending iteration.
struct BufState {
    int t0, nt;      // frames [t0, t0 + nt) of the clip
    int W;           // committed width
    int k_eff;       // seams selected in the pending iteration (0 = none)
    int removed;     // seams committed so far
    int slot;        // slot of E / SD / O that holds width W
    int target;      // target width
    int iters;       // iterations selected so far
    int tp;          // frames of the frame-minor luma copy (nt rounded up to 16)
    int k;           // seams per iteration of this buffer (0: the launch's k)
    long long yfm;   // byte offset of this buffer's frame-minor luma copy
    long long e0;    // element offset in CarveWs::E0 of the summed energy the
                     // scan wrote for this buffer, -1: none (k_energy_init sums)
};

#ifdef __CUDACC__
// ---- TMA bulk copies and mbarriers (inline PTX) ------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"(bytes)
                 : "memory");
}
// Global -> this CTA's shared memory; bytes and both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for an mbarrier phase: after `limit_ns` the status word gets
// DEV_ETIMEOUT and the caller continues (its data is then invalid; the host
// reports the error), so no wait can hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, unsigned parity, int *err,
                                          unsigned long long limit_ns) {
    if (mbar_try_wait(mbar, parity)) return true;
    if (err && *(volatile int *)err != DEV_OK) return false;   // an earlier wait gave up
    const unsigned long long t0 = globaltimer_now();
    while (!mbar_try_wait(mbar, parity)) {
        if (globaltimer_now() - t0 > limit_ns) {
            if (err) atomicExch(err, DEV_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// Programmatic dependent launch (the DP and update kernels of a carving loop
// are launched with programmatic stream serialisation): a kernel lets its
// dependent start launching at once, and waits for its predecessor's results
// before its first read of them.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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
#endif

// Arrays of one clip's carving, all in device memory.
struct CarveWs {
    int H, W0;          // clip height and original width
    long pitch;         // elements per row of E / SD / O (>= W0)
    long plane;         // H * pitch
    int dstride;        // direction words per 4-row block: ceil(W0 / 4) rounded up to 4
    long dbuf;          // direction words per buffer: ceil(H / 16) * 4 * dstride
    int kcap;           // capacity of a row's removal list
    int32_t *E;         // [nb][2][plane]  summed energy of the buffer
    int32_t *SD;        // [nb][plane]     wm * sum_t D_t at original coordinates
    uint16_t *O;        // [nb][2][plane]  original column of each carved pixel
    uint32_t *dirs;     // [nb][dbuf] DP directions, 2 bits per pixel, one word per 4x4 block
    uint16_t *rem;      // [nb][H][kcap]   columns removed in a row, ascending
    BufState *st;       // [nb]
    int *klog;          // [nb][klog_stride] k_eff of every iteration
    int klog_stride;
    const uint8_t *Y;   // [T][H][ypitch]  original luma of every frame
    const uint8_t *D;   // [T][H][ypitch]  motion map of every frame
    long ypitch;
    int wg, wm;
    unsigned long long *dirty_count;   // [nb] pixels recomputed by k_update (or NULL)
    uint8_t *Yfm;       // per buffer [H][W0][tp] original luma, frames innermost
    // cluster DP (k_dpc) only
    int rj;             // rows per trace-back band
    int nbands;         // ceil(H / rj)
    uint16_t *J;        // [nb][nbands][W0]  column, at the last row of the band above, of
                        //                   the path through (band's last row, j); band
                        //                   0: the path's row-0 column
    uint16_t *colbot;   // [nb][nbands][kcap] column of each seam at each band's last row
    int *dpx;           // [nb][1 + kcap]     k_eff, then each seam's rank by column
    int jstride;        // row stride of J (W0 rounded up to 8)
    int dpc_r;          // halo depth of the cluster DP (16 or 32); 0: the single-CTA DP
    int dpc_wpc;        // warps per cluster-DP CTA (4 or 8; 0 means 4)
    int dpc_v;          // columns per lane of the cluster DP (4 or 2, 2 with R = 16; 0 means 4)
    int up_rows;        // rows per k_update CTA (1, 2 or 4); 0: the largest that fits
    int *err;           // device status word (bounded waits)
    const int32_t *E0;  // summed energy planes [H][W0] from the scan (see BufState::e0)
    // forward terms (wf > 0): E then also holds wf * sum_t CU, and P holds the
    // buffer's sums of the two diagonal terms, A in the low and B in the high
    // 16 bits; the DP charges wf * A (wf * B) for a move from the upper left
    // (right)
    int wf = 0;
    uint32_t *P = nullptr;   // [nb][2][plane], slots as in E
};

constexpr int SCAN_FW = 8;   // frames per round of the buffer scan

// Scan (Sec. 3.2) arguments.
struct ScanArgs {
    const uint8_t *rgb;     // [T][H][W][3]
    int T, H, W;
    long ypitch;
    uint8_t *Y, *D;         // [T][H][ypitch]
    uint16_t *ering;        // [SCAN_FW][scan_state_px] energy of the frames of a round (tile-major)
    uint32_t *S1, *S2;      // [scan_state_px] sums of e and e^2 over the open buffer (tile-major)
    long long *partA;       // [T][SCAN_FW] A_t of each round's frames over the clip's CTAs (zeroed)
    int *partM;             // [T] maximum e_t over the clip's CTAs (zeroed)
    unsigned *count;        // [T] CTAs that published round r (zeroed)
    int *starts;            // [T+1] buffer starts (device)
    int *n_buffers;         // device scalar
    int *err;               // device status word
    int wg, wm;
    double alpha;
    int t_max, maxval_mode;
    long long maxval_theory;
    unsigned long long spin_limit_ns;
    int cta0, G;            // the clip's CTAs in a multi-clip launch
    int32_t *E0;            // [nbcap][H][W] summed energy of each closed buffer (or NULL)
    int nbcap;
    long e0_plane;          // H * W
    long long *A_out;       // [T] A_t of every frame (diagnostic, or NULL)
    int *M_out;             // [T] maximum e_t of every frame (diagnostic)
    // frames still arriving (or NULL): frame f may be read once *ready exceeds
    // f / ready_frames; a copy stream raises it after every chunk it copies
    const unsigned *ready;
    int ready_frames;
    // luma of the frame just before frame 0 ([H][ypitch], or NULL): frame 0's
    // motion term is taken against it instead of being 0 (a buffer carved on
    // its own, away from the start of its clip)
    const uint8_t *Yprev;
};

// Launchers (return the CUDA error of the launch).
cudaError_t launch_energy_api(const uint8_t *rgb, int T, int H, int W, int wg, int wm,
                              int32_t *energy, cudaStream_t s);
int scan_grid_size(int H, int W, int *err_out);
cudaError_t launch_scan(const ScanArgs &a, int grid, cudaStream_t s);
// Integer BT.601 luma of one RGB frame [H][W][3] into out [H][ypitch].
cudaError_t launch_luma_plane(const uint8_t *rgb, int H, int W, long ypitch, uint8_t *out,
                              cudaStream_t s);
// floor(sqrt(x)) of n values (device arrays) by the scan's own routine.
cudaError_t launch_isqrt_check(const unsigned long long *x, uint32_t *r, long n,
                               cudaStream_t s);
// Several clips in one cooperative launch: tab (device) holds each clip's
// arguments with its CTA range, block_clip (device) the clip of every CTA.
cudaError_t launch_scan_multi(const ScanArgs *tab, const int *block_clip, int grid,
                              cudaStream_t s);
int scan_capacity(int *err_out);   // co-resident scan CTAs on this GPU
int scan_tiles(int H, int W);      // 8x128 tiles of one frame
int scan_tiles_wt(int H, int W);   // 6x128 tiles of the single-clip warp-tile layout
int scan_tile_warps();             // tile-owning warps per scan CTA
long scan_state_px(int H, int W);  // pixels of the tile-major scan state

cudaError_t launch_energy_init(const CarveWs &ws, int nb, cudaStream_t s);
cudaError_t launch_update(const CarveWs &ws, int nb, cudaStream_t s);
cudaError_t launch_dp_select(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                             cudaStream_t s);
// Cluster DP with halo depth R (16 or 32), WPC warps per CTA (4 or 8) and V
// columns per lane (4, or 2 with R = 16): plan (CTAs per cluster, band rows,
// shared memory) for a width and height; returns false if this GPU cannot
// run it (then use launch_dp_select).  launch_dpc uses ws.dpc_r, ws.dpc_wpc
// and ws.dpc_v.
bool dpc_plan(int W0, int H, int R, int WPC, int V, int *ctas, int *rj, size_t *smem,
              bool fwd = false);
bool dpc_available(int W0, int H, int R, int WPC, int V, bool fwd = false);
// Sets ws.dpc_r / dpc_wpc / dpc_v to the requested layout (requested = the
// fields hold a tuned choice) if available, else to the default for the size;
// false if no cluster layout runs here.
bool dpc_select(int W0, int H, CarveWs &ws, bool requested);
cudaError_t launch_dpc(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                       cudaStream_t s);
cudaError_t launch_identity_O(const CarveWs &ws, int nb, cudaStream_t s);
// The carving iterations as one graph that runs on its own until every
// buffer reaches its target: a conditional WHILE node around `per_body` DP +
// update launches (the cluster DP when ws.J is set) and a one-thread kernel
// that sets the loop's condition from the buffer states and the status word.
// The graph's kernels get exactly these arguments.
cudaError_t build_carve_loop(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                             int per_body, cudaStream_t s, cudaGraphExec_t *out);
cudaError_t launch_gather(const CarveWs &ws, const uint8_t *rgb, int T, const int *buf_of_frame,
                          int target, uint8_t *out, cudaStream_t s);
// The colour gather of frames [t0, t0 + nt) only.
cudaError_t launch_gather_range(const CarveWs &ws, const uint8_t *rgb, int t0, int nt,
                                const int *buf_of_frame, int target, uint8_t *out,
                                cudaStream_t s);
// One frame of a batched colour gather: out rows of frame `dst` from `src`
// (both [H][*][3], device) through the origin map of buffer b.
struct GatherFrame {
    const uint8_t *src;
    uint8_t *dst;
    int b;
    int target;
};
cudaError_t launch_gather_frames(const CarveWs &ws, const GatherFrame *tab, int nframes,
                                 cudaStream_t s);
// [T][H][W][3] -> [T][W][H][3]
cudaError_t launch_transpose_rgb(const uint8_t *src, int T, int H, int W, uint8_t *dst,
                                 cudaStream_t s);
// Bulk copy between page-locked host memory and device memory (either way) by
// a kernel of a few dozen CTAs that reads or writes the host side over the
// CPU-GPU link (hostcopy.cu); memory the device cannot address goes through
// cudaMemcpyAsync instead.
cudaError_t link_copy(void *dst, const void *src, size_t bytes, cudaStream_t s);
// Carving workspace of nb buffers in one slab: sets ws's geometry (from ws.H,
// ws.W0, ws.kcap) and, when base is not NULL, its array pointers into base.
// Returns the slab size in bytes.  dpc: also the cluster-DP tables.
size_t carve_ws_assign(CarveWs &ws, int nb, int klog_stride, bool dpc, char *base);
}  // namespace scpl

#include <string>
#include "scpl.h"

namespace scpl {
// Autotuning table (tune.cu): the measured choice per (H, W).
bool tuning_lookup(int H, int W, scpl_tuning *out);
void tuning_store(const scpl_tuning &t);
void tuning_clear();
// Blend sharpness of a retargeted clip (quality.cu): luma of every frame into
// Y [T][H][W], then acc[0] += num, acc[1] += den over the runs of `window`.
cudaError_t launch_blend_sharpness(const uint8_t *frames, int T, int H, int W, int window,
                                   uint8_t *Y, unsigned long long *acc, cudaStream_t s);

// Seam insertion (insert.cu): every frame of buffer b (frames starts[b] ..
// starts[b+1]-1) widened from W to target by the m seams of
// seams[b * seam_stride + s * H + i] (original columns).
cudaError_t launch_insert_seams(const uint8_t *frames, int H, int W, int target,
                                const int16_t *seams, long seam_stride, int m,
                                const int *starts, int nb, uint8_t *out, cudaStream_t s);

int tuning_list(scpl_tuning *out, int max);

// true if the table held a choice for (H, W) (then applied to ws)
bool tuning_apply(int H, int W, CarveWs &ws, bool *use_dpc);
scpl_status tune_class(int H, int W, int k, cudaStream_t s, scpl_tuning *out);

// scpl_carve_batch's engine (engine.cu), owned by a handle.
scpl_status engine_run_batch(scpl_server_s **eng, const scpl_params &p, cudaStream_t stream,
                             bool autotune, scpl_job *jobs, int n_jobs, std::string &err);
void engine_destroy(scpl_server_s *eng);
scpl_status engine_stats(scpl_server_s *eng, scpl_server_stats *out);
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  It never lowers the limit, so a CUDA graph captured earlier
// with a larger launch of the same kernel stays launchable.
cudaError_t raise_dyn_smem(const void *func, size_t bytes);
size_t dp_smem_bytes(int W0, int H, int *band_blocks);
size_t update_smem_bytes(int W0, int kcap, int *rows, bool fwd = false);

// Forward terms: wf in [0, 255]; with wf > 0 a buffer holds at most 256
// frames, so a pixel's sums of the diagonal terms (255 a frame) fit 16 bits.
inline bool forward_params_ok(const scpl_params &p) {
    if (p.wf < 0 || p.wf > 255) return false;
    return p.wf == 0 || (p.use_buffer ? p.t_max : 1) <= 256;
}
// Largest step of a column's cumulative energy from one row to the next:
// the summed energy of tb frames plus, with forward terms, wf times the row's
// term and a diagonal term (255 each a frame).
inline long long dp_row_max(long long emax, long long tb, int wf) {
    return emax * tb + 2LL * 255 * wf * tb;
}

}  // namespace scpl
