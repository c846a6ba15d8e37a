// scpl_seams_noalloc: one SCPL iteration on a caller's energy map that
// allocates no memory at all.
//
// Who needs it: code that may not call cudaMalloc -- a real-time frame loop
// that cannot afford cudaMalloc's implicit device-wide synchronisation (it
// stalls every stream of the device until the allocation is done), or a host
// application that owns all device memory through its own fixed pool and
// forbids libraries from allocating after start-up, so that a long-running
// process can never fail half-way for lack of memory.  scpl_seams grows
// handle-owned workspaces with cudaMalloc; this entry point instead works in
// one fixed scratch array that the library reserves in device memory when it
// is loaded.
//
// The scratch is the file-scope __device__ array below.  Every GPU that loads
// the library holds it until the process exits.  In host code `g_scratch` is
// only a host-side stand-in for the symbol, so its device address is looked up
// with cudaGetSymbolAddress once per device (with that device current) and
// cached.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "scpl.h"
#include "scpl_internal.cuh"

using namespace scpl;

namespace {

// Size limits of the fixed scratch (H*W pixels, width, seams per call).
constexpr long NA_MAX_PIXELS = 1L << 21;   // 2,097,152 (1920 x 1080 fits)
constexpr int NA_MAX_W = 4096;
constexpr int NA_MAX_H = 65535;
constexpr int NA_MAX_K = 64;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Scratch layout: origin map O (u16 per pixel), DP directions (one u32 per
// 4x4 pixel block, rows of ceil(W/4) words padded to a multiple of 4),
// removal lists (u16 [H][k]),
// buffer state and the k_eff log.
constexpr size_t NA_O_BYTES = align256(NA_MAX_PIXELS * sizeof(uint16_t));
constexpr size_t NA_DIRS_BYTES =
    align256((size_t)(NA_MAX_PIXELS / 16 + NA_MAX_H + NA_MAX_W / 4 + 4) * sizeof(uint32_t));
constexpr size_t NA_REM_BYTES = align256((size_t)NA_MAX_PIXELS * sizeof(uint16_t));
constexpr size_t NA_ST_BYTES = align256(sizeof(BufState) + sizeof(int));
constexpr size_t NA_OFF_DIRS = NA_O_BYTES;
constexpr size_t NA_OFF_REM = NA_OFF_DIRS + NA_DIRS_BYTES;
constexpr size_t NA_OFF_ST = NA_OFF_REM + NA_REM_BYTES;
constexpr size_t NA_SCRATCH_BYTES = NA_OFF_ST + NA_ST_BYTES;   // about 9 MiB

__device__ __align__(256) unsigned char g_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch on the current device (set up on first use).
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Every call starts from a fresh buffer state (the scratch keeps whatever the
// previous call left there).
__global__ void k_noalloc_reset(BufState *st, int *klog, int W, int target) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        BufState s;
        s.t0 = 0; s.nt = 1; s.W = W; s.k_eff = 0; s.removed = 0; s.slot = 0;
        s.target = target; s.iters = 0; s.tp = 0; s.k = 0; s.yfm = 0; s.e0 = -1;
        *st = s;
        *klog = 0;
    }
}

}  // namespace

extern "C" scpl_status scpl_seams_noalloc(const int32_t *energy, int H, int W, int k,
                                          int16_t *cols, int *k_eff, void *stream) {
    if (!energy || !cols || !k_eff) return SCPL_EINVAL;
    if (H < 1 || W < 1 || k < 1) return SCPL_EINVAL;
    if (W > NA_MAX_W || H > NA_MAX_H || (long)H * W > NA_MAX_PIXELS || k > NA_MAX_K)
        return SCPL_EINVAL;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SCPL_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int kc = k < W ? k : W;

    CarveWs ws;
    ws.H = H;
    ws.W0 = W;
    ws.pitch = W;                       // the caller's map is read in place
    ws.plane = (long)H * W;
    ws.dstride = (((W + 3) / 4) + 3) & ~3;
    ws.dbuf = (long)((H + 3) / 4) * ws.dstride;
    ws.dirty_count = nullptr;
    ws.Yfm = nullptr;
    ws.E0 = nullptr;
    ws.err = nullptr;
    ws.J = nullptr;
    ws.colbot = nullptr;
    ws.dpx = nullptr;
    ws.rj = 0;
    ws.nbands = 0;
    ws.jstride = 0;
    ws.kcap = kc;
    ws.E = const_cast<int32_t *>(energy);
    ws.SD = nullptr;
    ws.O = reinterpret_cast<uint16_t *>(base);
    ws.dirs = reinterpret_cast<uint32_t *>(base + NA_OFF_DIRS);
    ws.rem = reinterpret_cast<uint16_t *>(base + NA_OFF_REM);
    ws.st = reinterpret_cast<BufState *>(base + NA_OFF_ST);
    ws.klog = reinterpret_cast<int *>(base + NA_OFF_ST + sizeof(BufState));
    ws.klog_stride = 1;
    ws.Y = nullptr;
    ws.D = nullptr;
    ws.ypitch = 0;
    ws.wg = 0;
    ws.wm = 0;

    k_noalloc_reset<<<1, 32, 0, s>>>(ws.st, ws.klog, W, W - kc);
    if (cudaGetLastError() != cudaSuccess) return SCPL_ECUDA;
    if (launch_identity_O(ws, 1, s) != cudaSuccess) return SCPL_ECUDA;
    if (launch_dp_select(ws, 1, k, cols, 0, s) != cudaSuccess) return SCPL_ECUDA;
    int ke = 0;
    if (cudaMemcpyAsync(&ke, &ws.st->k_eff, sizeof(int), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return SCPL_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SCPL_ECUDA;
    *k_eff = ke;
    return SCPL_OK;
}
