// Internal declarations of libscpl: device-side data layout and the launchers
// that the C ABI (scpl_api.cu) calls.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace scpl {

constexpr uint64_t KEY_INF = ~0ull;
constexpr uint64_t KEY_DIR_MASK = 0xFFull << 24;   // tie-break / direction byte of a DP key
constexpr uint32_t LABEL_MASK = 0xFFFFFFu;         // 24-bit parent label of a DP key

// Status words written by kernels (mirror scpl_status).
constexpr int DEV_OK = 0;
constexpr int DEV_ETIMEOUT = 4;

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
};

// Arrays of one clip's carving, all in device memory.
struct CarveWs {
    int H, W0;          // clip height and original width
    long pitch;         // elements per row of E / SD / O (>= W0)
    long plane;         // H * pitch
    int ngroups;        // ceil(W0 / 32): 32-column groups of the direction bit planes
    int kcap;           // capacity of a row's removal list
    int32_t *E;         // [nb][2][plane]  summed energy of the buffer
    int32_t *SD;        // [nb][2][plane]  summed, carved motion energy wm * sum_t D_t
    uint16_t *O;        // [nb][2][plane]  original column of each carved pixel
    uint32_t *dirs;     // [nb][H][ngroups][2] DP directions as two bit planes
    uint16_t *rem;      // [nb][H][kcap]   columns removed in a row, ascending
    BufState *st;       // [nb]
    int *klog;          // [nb][klog_stride] k_eff of every iteration
    int klog_stride;
    const uint8_t *Y;   // [T][H][ypitch]  original luma of every frame
    const uint8_t *D;   // [T][H][ypitch]  motion map of every frame
    long ypitch;
    int wg, wm;
};

// Scan (Sec. 3.2) arguments.
struct ScanArgs {
    const uint8_t *rgb;     // [T][H][W][3]
    int T, H, W;
    long ypitch;
    uint8_t *Y, *D;         // [T][H][ypitch]
    uint16_t *ering;        // [2][H*W] energy of the last two frames
    uint32_t *S1, *S2;      // [H*W] sums of e and e^2 over the open buffer
    long long *partA;       // [T][G] per-CTA partial ASDE sums
    int *partM;             // [T][G] per-CTA partial energy maxima
    unsigned *count;        // [T] CTAs that published frame t
    int *starts;            // [T+1] buffer starts (device)
    int *n_buffers;         // device scalar
    int *err;               // device status word
    int wg, wm;
    double alpha;
    int t_max, maxval_mode;
    long long maxval_theory;
    unsigned long long spin_limit_ns;
};

// Launchers (return the CUDA error of the launch).
cudaError_t launch_energy_api(const uint8_t *rgb, int T, int H, int W, int wg, int wm,
                              int32_t *energy, cudaStream_t s);
int scan_grid_size(int H, int W, int *err_out);
cudaError_t launch_scan(const ScanArgs &a, int grid, cudaStream_t s);

cudaError_t launch_energy_init(const CarveWs &ws, int nb, cudaStream_t s);
cudaError_t launch_energy_iter(const CarveWs &ws, int nb, cudaStream_t s);
cudaError_t launch_dp_select(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                             cudaStream_t s);
cudaError_t launch_identity_O(const CarveWs &ws, int nb, cudaStream_t s);
cudaError_t launch_gather(const CarveWs &ws, const uint8_t *rgb, int T, const int *buf_of_frame,
                          int target, uint8_t *out, cudaStream_t s);
size_t dp_select_smem_bytes(int W0);

}  // namespace scpl
