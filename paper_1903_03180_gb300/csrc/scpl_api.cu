// C ABI of libscpl (declared in include/scpl.h): argument checks, workspace
// management and the host-side order of launches.  All arithmetic of the
// method runs in the kernels of scan.cu and carve.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "scpl.h"
#include "scpl_internal.cuh"

using namespace scpl;

namespace {

// A grow-only device allocation.
struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// A grow-only page-locked host allocation.
struct HostBuf {
    void *p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMallocHost(&p, bytes);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

constexpr unsigned long long SPIN_LIMIT_NS = 2000000000ull;   // 2 s per device-wide wait

// Kernel kinds for the per-kernel accounting.
enum KernelId { K_SCAN, K_ENERGY_INIT, K_ENERGY_ITER, K_DP_SELECT, K_GATHER, K_IDENTITY,
                K_ENERGY_API, K_COUNT };
const char *const kKernelNames[K_COUNT] = {"k_scan", "k_energy_init", "k_update",
                                           "k_dp", "k_gather", "k_identity_O",
                                           "k_energy_api"};

// Event-bracketed launches while profiling is on.
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<int, size_t>> marks;   // kernel id, index of its start event
    double ms[K_COUNT] = {};
    long long launches[K_COUNT] = {};
    double bytes[K_COUNT] = {};
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void clear() {
        used = 0;
        marks.clear();
        for (int i = 0; i < K_COUNT; ++i) { ms[i] = 0; launches[i] = 0; bytes[i] = 0; }
    }
};

long round_up(long v, long m) { return (v + m - 1) / m * m; }

constexpr int CARVE_LOOP_ITERS = 8;   // DP + update pairs per body of the device-side loop

}  // namespace

struct scpl_ctx {
    scpl_params p;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    // scan
    DevBuf Y, D, ering, S1, S2, partA, partM, count, starts, nbuf, errw, E0;
    int e0cap = 0;   // summed-energy planes the last scan could write
    // carving: one slab for every array of the carving workspace
    DevBuf cws, bof;
    // host-memory entry point staging
    DevBuf in_frames, out_frames, seams_dev;
    DevBuf qY, qacc;   // blend sharpness: luma of every frame, the two sums
    DevBuf ej_mid, ej_tin, ej_tout;   // scpl_enlarge_job: widened, transposed, enlarged
    // scpl_carve_host_many: a second input and output slot and the input copy
    // stream
    DevBuf in2, out2;
    DevBuf Yprev;   // scpl_carve_buffer: luma of the frame before the buffer
    cudaStream_t istream = nullptr;
    DevBuf Yfm;
    bool autotune = false;
    unsigned long long wait_ns = SPIN_LIMIT_NS;   // bound of the scan's device-wide waits
    // host-memory path: copy stream and side stream for early gathers
    cudaStream_t cstream = nullptr, gstream = nullptr;
    HostBuf h_small;   // starts + n_buffers + states readback
    Profiler prof;
    // the carving loop as a graph that runs on the device until every buffer
    // reaches its target, kept for the next call with the same workspace and
    // arguments (the key: the workspace's bytes, nb, k, seams, their stride)
    cudaGraphExec_t loop = nullptr;
    unsigned char loop_ws[sizeof(CarveWs)] = {};
    int loop_nb = 0, loop_k = 0;
    int16_t *loop_seams = nullptr;
    long loop_stride = 0;
    bool loop_unavailable = false;   // conditional graph nodes cannot be built here
    cudaStream_t lstream = nullptr;  // capture stream of the loop (the handle's may be the
                                     // legacy default stream, which cannot be captured)
    scpl_server_s *engine = nullptr;   // scpl_carve_batch's engine (created on first use)
    // summary of the last scpl_carve call
    int last_nb = 0, last_iter_max = 0;
    long long last_launches = 0;   // kernel launches of the last scpl_carve call
    std::vector<int> last_keff, last_iters;   // k_eff of every iteration, per buffer
    long long last_iter_total = 0;
    double last_carved_px = 0;
};

namespace {

scpl_status fail(scpl_ctx *h, scpl_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return s;
}

#define SCPL_CUDA(h, call)                                                                 \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            scpl_status s_ = (e_ == cudaErrorMemoryAllocation) ? SCPL_ENOMEM : SCPL_ECUDA; \
            return fail(h, s_, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                        __LINE__);                                                         \
        }                                                                                  \
    } while (0)

// Runs `launch` (issued on stream s) bracketed by events when profiling is on.
template <class F>
cudaError_t timed_on(scpl_ctx *h, int id, cudaStream_t s, F launch) {
    if (!h->prof.on) return launch();
    cudaEvent_t a = h->prof.next(), b = h->prof.next();
    if (!a || !b) return launch();
    cudaEventRecord(a, s);
    cudaError_t e = launch();
    cudaEventRecord(b, s);
    h->prof.marks.push_back({id, h->prof.used - 2});
    return e;
}
template <class F>
cudaError_t timed(scpl_ctx *h, int id, F launch) {
    return timed_on(h, id, h->stream, launch);
}

scpl_status check_params(const scpl_params *p) {
    if (!p) return SCPL_EINVAL;
    if (!(p->alpha >= 0.0) || p->alpha > 1e6) return SCPL_EINVAL;
    if (p->wg < 0 || p->wm < 0 || p->wg + p->wm == 0) return SCPL_EINVAL;
    if (p->t_max < 1 || p->t_max > 1024) return SCPL_EINVAL;
    if (p->maxval_mode != 0 && p->maxval_mode != 1) return SCPL_EINVAL;
    if (!forward_params_ok(*p)) return SCPL_EINVAL;
    return SCPL_OK;
}

long long energy_max(const scpl_params &p) { return 255LL * (8LL * p.wg + p.wm); }

int effective_tmax(const scpl_params &p) { return p.use_buffer ? p.t_max : 1; }

// Overflow limits of the exact integer arithmetic: the DP keys hold a
// column's cumulative energy in 32 bits, S2 holds t_max * e^2 in 32 bits and
// the scan keeps e in 16 bits.
scpl_status check_overflow(scpl_ctx *h, int T, int H) {
    long long em = energy_max(h->p);
    long long tb = std::min<long long>(T, effective_tmax(h->p));
    if (em >= 65536) return fail(h, SCPL_EOVERFLOW, "energy maximum %lld exceeds 16 bits", em);
    if (dp_row_max(em, tb, h->p.wf) * H >= (1LL << 31))
        return fail(h, SCPL_EOVERFLOW, "cumulative energy %lld*%d can exceed 2^31",
                    dp_row_max(em, tb, h->p.wf), H);
    if ((long long)effective_tmax(h->p) * em * em >= (1LL << 32))
        return fail(h, SCPL_EOVERFLOW, "t_max*emax^2 can exceed 2^32");
    return SCPL_OK;
}

constexpr int E0_PLANES = 16;   // buffers whose summed energy the scan keeps

// Runs the buffer scan; leaves Y, D (original luma / motion) and the summed
// energy of the first E0_PLANES buffers in the handle and the starts on the
// host.  A and M (host, or NULL) receive every frame's A_t and maximum e_t.
// prev_rgb (device [H][W][3], or NULL) is the frame before frame 0, for frame
// 0's motion term; `fixed` makes the T frames one buffer (no flush decision).
scpl_status run_scan(scpl_ctx *h, const uint8_t *frames, int T, int H, int W,
                     std::vector<int> &starts, bool keep_e0, long long *A = nullptr,
                     int *M = nullptr, const unsigned *ready = nullptr, int ready_frames = 1,
                     const uint8_t *prev_rgb = nullptr, bool fixed = false) {
    TraceRange trace("scpl.scan");
    const long ypitch = round_up(W, 16);
    const long hw = (long)H * W;
    int gerr = 0;
    int G = scan_grid_size(H, W, &gerr);
    if (gerr || G < 1) return fail(h, SCPL_ECUDA, "scan occupancy query failed (%d)", gerr);
    SCPL_CUDA(h, h->Y.ensure((size_t)T * H * ypitch));
    SCPL_CUDA(h, h->D.ensure((size_t)T * H * ypitch));
    const size_t spx = (size_t)scan_state_px(H, W);
    SCPL_CUDA(h, h->ering.ensure((size_t)SCAN_FW * spx * sizeof(uint16_t)));
    SCPL_CUDA(h, h->S1.ensure(spx * sizeof(uint32_t)));
    SCPL_CUDA(h, h->S2.ensure(spx * sizeof(uint32_t)));
    h->e0cap = keep_e0 ? std::min(T, E0_PLANES) : 0;
    if (h->e0cap) SCPL_CUDA(h, h->E0.ensure((size_t)h->e0cap * hw * sizeof(int32_t)));
    // per-round A_t [rounds][SCAN_FW], frame maxima [T], then the diagnostics
    // M_t, A_t.  A round decides at least one frame, except a round whose
    // first frame is too close to call on its bounded sum; the round after it
    // is exact and decides at least one: 2T rounds at most.
    const size_t rounds = 2 * (size_t)T;
    const size_t accb = rounds * SCAN_FW * 8;
    SCPL_CUDA(h, h->partA.ensure(accb + (size_t)T * 16));
    SCPL_CUDA(h, h->count.ensure(rounds * sizeof(unsigned)));
    SCPL_CUDA(h, h->starts.ensure((size_t)(T + 1) * sizeof(int)));
    SCPL_CUDA(h, h->nbuf.ensure(sizeof(int)));
    SCPL_CUDA(h, h->errw.ensure(sizeof(int)));
    SCPL_CUDA(h, h->h_small.ensure((size_t)(T + 4) * sizeof(int)));
    cudaStream_t s = h->stream;
    SCPL_CUDA(h, cudaMemsetAsync(h->count.p, 0, rounds * sizeof(unsigned), s));
    SCPL_CUDA(h, cudaMemsetAsync(h->partA.p, 0, accb + (size_t)T * 4, s));
    SCPL_CUDA(h, cudaMemsetAsync(h->errw.p, 0, sizeof(int), s));
    if (prev_rgb) {
        SCPL_CUDA(h, h->Yprev.ensure((size_t)H * ypitch));
        SCPL_CUDA(h, launch_luma_plane(prev_rgb, H, W, ypitch, h->Yprev.as<uint8_t>(), s));
    }
    ScanArgs a;
    a.rgb = frames; a.T = T; a.H = H; a.W = W; a.ypitch = ypitch;
    a.Y = h->Y.as<uint8_t>(); a.D = h->D.as<uint8_t>();
    a.ering = h->ering.as<uint16_t>();
    a.S1 = h->S1.as<uint32_t>(); a.S2 = h->S2.as<uint32_t>();
    a.partA = h->partA.as<long long>();
    a.partM = reinterpret_cast<int *>(h->partA.as<char>() + accb);
    a.count = h->count.as<unsigned>();
    a.starts = h->starts.as<int>(); a.n_buffers = h->nbuf.as<int>();
    a.err = h->errw.as<int>();
    a.wg = h->p.wg; a.wm = h->p.wm; a.alpha = h->p.alpha;
    a.t_max = effective_tmax(h->p); a.maxval_mode = h->p.maxval_mode;
    a.maxval_theory = energy_max(h->p);
    a.spin_limit_ns = h->wait_ns;
    a.E0 = h->e0cap ? h->E0.as<int32_t>() : nullptr;
    a.nbcap = h->e0cap;
    a.e0_plane = hw;
    a.A_out = nullptr;
    a.M_out = nullptr;
    a.ready = ready;
    a.ready_frames = ready_frames;
    a.Yprev = prev_rgb ? h->Yprev.as<uint8_t>() : nullptr;
    if (fixed) {
        // one buffer of all T frames: the cap at T closes it at the end, and
        // with alpha = 1e6 no spread can exceed the threshold (A is at most
        // 128 n M H W, the threshold 2.56e8 M sqrt(n-1) H W)
        a.alpha = 1e6;
        a.t_max = T;
    }
    if (A) {   // diagnostics after the accumulators in the same allocation
        a.M_out = reinterpret_cast<int *>(h->partA.as<char>() + accb + (size_t)T * 4);
        a.A_out = reinterpret_cast<long long *>(h->partA.as<char>() + accb + (size_t)T * 8);
    }
    SCPL_CUDA(h, timed(h, K_SCAN, [&] { return launch_scan(a, G, s); }));
    if (h->prof.on) h->prof.bytes[K_SCAN] += 28.0 * hw * T;
    int *hs = h->h_small.as<int>();
    SCPL_CUDA(h, cudaMemcpyAsync(hs, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCPL_CUDA(h, cudaMemcpyAsync(hs + 1, h->nbuf.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCPL_CUDA(h, cudaMemcpyAsync(hs + 2, h->starts.p, (size_t)(T + 1) * sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
    SCPL_CUDA(h, cudaStreamSynchronize(s));
    if (hs[0] == DEV_ETIMEOUT)
        return fail(h, SCPL_ETIMEOUT, "buffer scan: a device-wide wait exceeded %llu ns",
                    h->wait_ns);
    int nb = hs[1];
    if (nb < 1 || nb > T) return fail(h, SCPL_ECUDA, "buffer scan returned %d buffers", nb);
    starts.assign(hs + 2, hs + 2 + nb + 1);
    if (A) {
        SCPL_CUDA(h, cudaMemcpyAsync(A, a.A_out, (size_t)T * 8, cudaMemcpyDeviceToHost, s));
        SCPL_CUDA(h, cudaMemcpyAsync(M, a.M_out, (size_t)T * 4, cudaMemcpyDeviceToHost, s));
        SCPL_CUDA(h, cudaStreamSynchronize(s));
    }
    return SCPL_OK;
}

// Workspace of the carving stage for nb buffers (one grow-only slab).
scpl_status carve_ws(scpl_ctx *h, int nb, int H, int W0, int kcap, CarveWs &ws,
                     int klog_stride = 1) {
    std::memset(&ws, 0, sizeof ws);   // every byte set: the device loop compares workspaces
    ws.H = H;
    ws.W0 = W0;
    ws.kcap = std::max(kcap, 1);
    SCPL_CUDA(h, h->errw.ensure(sizeof(int)));
    ws.err = h->errw.as<int>();
    int bb = 0, rb = 0;
    if (dp_smem_bytes(W0, H, &bb) > 227 * 1024 - 4096 ||
        update_smem_bytes(W0, ws.kcap, &rb, h->p.wf > 0) > 200 * 1024)
        return fail(h, SCPL_EINVAL, "width %d exceeds the shared-memory limits", W0);
    // the tuned choice for this size (cluster-DP layout or the single-CTA DP,
    // update rows), measured first if autotuning is on; the default layout
    // for the size otherwise
    ws.dpc_r = 32;
    ws.dpc_wpc = 4;
    ws.dpc_v = 4;
    ws.up_rows = 0;
    bool use_dpc = true;
    if (h->autotune && !tuning_lookup(H, W0, nullptr))
        tune_class(H, W0, ws.kcap, h->stream, nullptr);   // on failure: the defaults
    const bool tuned = tuning_apply(H, W0, ws, &use_dpc);
    // forward terms: their planes, and the cluster-DP layouts built with them
    ws.wf = h->p.wf;
    if (ws.wf > 0) use_dpc = true;
    // cluster DP (used when the GPU can co-schedule the cluster)
    const bool dpc = use_dpc && dpc_select(W0, H, ws, tuned);
    const size_t bytes = carve_ws_assign(ws, nb, klog_stride, dpc, nullptr);
    SCPL_CUDA(h, h->cws.ensure(bytes));
    carve_ws_assign(ws, nb, klog_stride, dpc, h->cws.as<char>());
    ws.Y = h->Y.as<uint8_t>();
    ws.D = h->D.as<uint8_t>();
    ws.ypitch = round_up(W0, 16);
    ws.wg = h->p.wg;
    ws.wm = h->p.wm;
    return SCPL_OK;
}

scpl_status check_frames(scpl_ctx *h, const void *frames, int T, int H, int W) {
    if (!h) return SCPL_EINVAL;
    if (!frames) return fail(h, SCPL_EINVAL, "frames is NULL");
    if (T < 1 || H < 1 || W < 1) return fail(h, SCPL_EINVAL, "T=%d H=%d W=%d must be >= 1", T, H, W);
    if (H > 65535) return fail(h, SCPL_EINVAL, "H=%d exceeds 65535", H);
    if (W > 8192) return fail(h, SCPL_EINVAL, "W=%d exceeds 8192", W);
    return SCPL_OK;
}

}  // namespace

namespace {

// cuStreamWriteValue32 from the driver, looked up once (NULL if unavailable).
PFN_cuStreamWriteValue32_v11070 stream_write_value() {
    static PFN_cuStreamWriteValue32_v11070 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuStreamWriteValue32_v11070>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// scpl_carve with the options of the host-memory paths: `ready` (frames still
// arriving, see ScanArgs::ready), `host_out` (every buffer's output frames
// are gathered as soon as the buffer is carved and copied to host_out on the
// copy stream while the other buffers carve on) and `after_scan` (called
// once the scan has finished, before the carving is issued).
scpl_status carve_run(scpl_ctx *h, const uint8_t *frames, int T, int H, int W, int target_W,
                      int k, uint8_t *out, int32_t *buffer_starts, int *n_buffers,
                      int16_t *seams, const unsigned *ready, int ready_frames,
                      uint8_t *host_out,
                      const std::function<scpl_status()> &after_scan = nullptr,
                      const uint8_t *prev_rgb = nullptr, bool fixed = false) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!out) return fail(h, SCPL_EINVAL, "out is NULL");
    if (target_W < 2 || target_W > W)
        return fail(h, SCPL_EINVAL, "target_W=%d must be in [2, W=%d]", target_W, W);
    if (k < 1) return fail(h, SCPL_EINVAL, "k=%d must be >= 1", k);
    if ((s = check_overflow(h, T, H)) != SCPL_OK) return s;

    // kernel launches of this call: the scan (with the luma of the frame
    // before a lone buffer), the initialisation, the iterations, the gathers
    long long launched = 1 + (prev_rgb ? 1 : 0);
    bool carve_looped = false;
    int loop_iters = 0;
    std::vector<int> starts;
    if ((s = run_scan(h, frames, T, H, W, starts, true, nullptr, nullptr, ready, ready_frames,
                      prev_rgb, fixed)) != SCPL_OK)
        return s;
    // the scan has finished (its starts are on the host): work that must not
    // share the GPU with the scan's device-wide waits may be issued now
    if (after_scan && (s = after_scan()) != SCPL_OK) return s;
    const int nb = (int)starts.size() - 1;
    const int remove = W - target_W;
    TraceRange trace("scpl.carve");
    CarveWs ws;
    if ((s = carve_ws(h, nb, H, W, std::min(k, std::max(remove, 1)), ws, remove)) != SCPL_OK)
        return s;
    cudaStream_t st = h->stream;

    // per-buffer states and the frame -> buffer map
    SCPL_CUDA(h, h->bof.ensure((size_t)T * sizeof(int)));
    size_t need = 64 + (size_t)nb * sizeof(BufState) + (size_t)T * sizeof(int) +
                  (size_t)nb * std::max(remove, 1) * sizeof(int) + 8 +
                  (size_t)nb * sizeof(unsigned long long);
    SCPL_CUDA(h, h->h_small.ensure(need));
    BufState *hb = reinterpret_cast<BufState *>(h->h_small.as<char>() + 64);
    int *hbof = reinterpret_cast<int *>(hb + nb);
    int *hklog = hbof + T;
    long long yfm_total = 0;
    for (int b = 0; b < nb; ++b) {
        const int nt = starts[b + 1] - starts[b];
        const int tp = (nt + 15) & ~15;
        const long long e0 = b < h->e0cap ? (long long)b * H * W : -1;
        hb[b] = BufState{starts[b], nt, W, 0, 0, 0, target_W, 0, tp, 0, yfm_total, e0};
        yfm_total += (long long)H * W * tp;
        for (int t = starts[b]; t < starts[b + 1]; ++t) hbof[t] = b;
    }
    SCPL_CUDA(h, h->Yfm.ensure((size_t)std::max<long long>(yfm_total, 16)));
    ws.Yfm = h->Yfm.as<uint8_t>();
    ws.E0 = h->E0.as<int32_t>();
    SCPL_CUDA(h, cudaMemcpyAsync(ws.st, hb, (size_t)nb * sizeof(BufState),
                                 cudaMemcpyHostToDevice, st));
    SCPL_CUDA(h, cudaMemcpyAsync(h->bof.p, hbof, (size_t)T * sizeof(int), cudaMemcpyHostToDevice,
                                 st));
    const long seam_stride = (long)remove * H;

    SCPL_CUDA(h, cudaMemsetAsync(ws.dirty_count, 0, (size_t)nb * sizeof(unsigned long long), st));
    // host path: gather buffer b on the side stream once carved, then copy its
    // frames to the host on the copy stream
    std::vector<char> gathered(nb, 0);
    cudaEvent_t ev_carved = nullptr, ev_gathered = nullptr;
    if (host_out) {
        SCPL_CUDA(h, cudaEventCreateWithFlags(&ev_carved, cudaEventDisableTiming));
        SCPL_CUDA(h, cudaEventCreateWithFlags(&ev_gathered, cudaEventDisableTiming));
    }
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev_guard{ev_carved, ev_gathered};
    const size_t frame_out = (size_t)H * target_W * 3;
    auto gather_out = [&](int b) -> scpl_status {
        const int t0 = starts[b], nt = starts[b + 1] - starts[b];
        TraceRange gtrace("scpl.gather");
        SCPL_CUDA(h, cudaEventRecord(ev_carved, st));
        SCPL_CUDA(h, cudaStreamWaitEvent(h->gstream, ev_carved, 0));
        SCPL_CUDA(h, timed_on(h, K_GATHER, h->gstream, [&] {
                      return launch_gather_range(ws, frames, t0, nt, h->bof.as<int>(), target_W,
                                                 out, h->gstream);
                  }));
        SCPL_CUDA(h, cudaEventRecord(ev_gathered, h->gstream));
        SCPL_CUDA(h, cudaStreamWaitEvent(h->cstream, ev_gathered, 0));
        SCPL_CUDA(h, link_copy(host_out + (size_t)t0 * frame_out, out + (size_t)t0 * frame_out,
                               (size_t)nt * frame_out, h->cstream));
        gathered[b] = 1;
        return SCPL_OK;
    };
    if (remove == 0) {
        SCPL_CUDA(h, timed(h, K_IDENTITY, [&] { return launch_identity_O(ws, nb, st); }));
    } else {
        SCPL_CUDA(h, timed(h, K_ENERGY_INIT, [&] { return launch_energy_init(ws, nb, st); }));
        int iters = (remove + k - 1) / k;
        launched += 1 + (h->p.wf > 0 ? 1 : 0);   // k_energy_init (+ k_forward_init)
        // device-resident clips (not profiled per kernel): the iterations as
        // one graph that loops on the device until every buffer is carved
        bool looped = false;
        if (!host_out && !h->prof.on && !h->loop_unavailable) {
            const bool same = h->loop && h->loop_nb == nb && h->loop_k == k &&
                              h->loop_seams == seams && h->loop_stride == seam_stride &&
                              std::memcmp(h->loop_ws, &ws, sizeof ws) == 0;
            if (!same) {
                if (h->loop) SCPL_CUDA(h, cudaGraphExecDestroy(h->loop));
                h->loop = nullptr;
                cudaGraphExec_t ge = nullptr;
                if (!h->lstream)
                    SCPL_CUDA(h, cudaStreamCreateWithFlags(&h->lstream, cudaStreamNonBlocking));
                if (build_carve_loop(ws, nb, k, seams, seam_stride, CARVE_LOOP_ITERS, h->lstream,
                                     &ge) == cudaSuccess) {
                    h->loop = ge;
                    h->loop_nb = nb;
                    h->loop_k = k;
                    h->loop_seams = seams;
                    h->loop_stride = seam_stride;
                    std::memcpy(h->loop_ws, &ws, sizeof ws);
                } else {
                    cudaGetLastError();
                    h->loop_unavailable = true;   // conditional nodes unavailable: chunks
                }
            }
            if (h->loop) {
                SCPL_CUDA(h, cudaGraphLaunch(h->loop, st));
                looped = true;
            }
        }
        carve_looped = looped;
        for (int guard = 0; guard <= remove && !looped; ++guard) {
            launched += 2LL * iters;
            for (int q = 0; q < iters; ++q) {
                SCPL_CUDA(h, timed(h, K_DP_SELECT, [&] {
                              return ws.J ? launch_dpc(ws, nb, k, seams, seam_stride, st)
                                          : launch_dp_select(ws, nb, k, seams, seam_stride, st);
                          }));
                SCPL_CUDA(h, timed(h, K_ENERGY_ITER, [&] { return launch_update(ws, nb, st); }));
            }
            SCPL_CUDA(h, cudaMemcpyAsync(hb, ws.st, (size_t)nb * sizeof(BufState),
                                         cudaMemcpyDeviceToHost, st));
            SCPL_CUDA(h, cudaStreamSynchronize(st));
            if (host_out)   // buffers that reached the target: gather and send them now
                for (int b = 0; b < nb; ++b)
                    if (!gathered[b] && hb[b].W - hb[b].k_eff <= target_W) {
                        if ((s = gather_out(b)) != SCPL_OK) return s;
                    }
            // the next chunk: enough iterations for every buffer at the mean
            // number of seams it has removed per iteration so far, at most 32
            // (a buffer's last k_eff swings from 2 to 16 and overshot by a
            // fifth of the launches; a launch past a buffer's target costs a
            // few microseconds, a read-back between chunks a few tens)
            int next = 0;
            for (int b = 0; b < nb; ++b) {
                const int Wc = hb[b].W - hb[b].k_eff;
                const int r = Wc - target_W;
                if (r > 0) {
                    const double mean = std::max(1.0, (double)(W - Wc) / std::max(hb[b].iters, 1));
                    next = std::max(next, (int)std::ceil(r / mean));
                }
            }
            if (next == 0) break;
            iters = std::min(std::max(next, 1), 32);
            // host path: look again after a few iterations, so that buffers
            // that finish early are gathered and copied out while the others
            // carve on
            if (host_out) iters = std::min(iters, 8);
        }
    }
    if (host_out) {
        for (int b = 0; b < nb; ++b)
            if (!gathered[b] && (s = gather_out(b)) != SCPL_OK) return s;
    } else {
        SCPL_CUDA(h, timed(h, K_GATHER, [&] {
                      return launch_gather(ws, frames, T, h->bof.as<int>(), target_W, out, st);
                  }));
    }

    // iteration summary (and the algorithmic bytes while profiling)
    h->last_nb = nb;
    launched += remove == 0 ? 1 : (host_out ? nb : 1);   // identity O or the colour gathers
    h->last_iter_max = 0;
    h->last_iter_total = 0;
    h->last_carved_px = 0;
    h->last_keff.clear();
    h->last_iters.assign(nb, 0);
    if (remove > 0) {
        unsigned long long *hdirty = reinterpret_cast<unsigned long long *>(
            h->h_small.as<char>() + 64 + (((size_t)nb * sizeof(BufState) + (size_t)T * sizeof(int) +
                                           (size_t)nb * remove * sizeof(int) + 7) & ~(size_t)7));
        SCPL_CUDA(h, cudaMemcpyAsync(hklog, ws.klog, (size_t)nb * remove * sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
        SCPL_CUDA(h, cudaMemcpyAsync(hdirty, ws.dirty_count, (size_t)nb * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, st));
        SCPL_CUDA(h, cudaStreamSynchronize(st));
        const bool fwd = h->p.wf > 0;
        for (int b = 0; b < nb; ++b) {
            const double Tb = hb[b].nt;
            int Wc = W, it = 0;
            while (Wc > target_W && it < remove) {
                const int ke = hklog[(long)b * remove + it];
                const int Wn = Wc - ke;
                h->last_carved_px += (double)H * Wc;
                h->last_keff.push_back(ke);
                if (h->prof.on) {
                    // DP: E read, directions written and read back, lists written
                    // (forward terms: the diagonal sums read too)
                    h->prof.bytes[K_DP_SELECT] += H * ((fwd ? 8.5 : 4.5) * Wc + 2.0 * ke);
                    // update: O and E read (gathered) and written at the new width,
                    // the removal lists of each row and its two neighbours
                    // (forward terms: the diagonal sums as well)
                    if (Wn > target_W)
                        h->prof.bytes[K_ENERGY_ITER] += H * ((fwd ? 20.0 : 12.0) * Wn + 6.0 * ke);
                    else
                        h->prof.bytes[K_ENERGY_ITER] += H * (4.0 * Wn + 6.0 * ke);
                }
                Wc = Wn;
                ++it;
            }
            h->last_iter_max = std::max(h->last_iter_max, it);
            h->last_iter_total += it;
            h->last_iters[b] = it;
            loop_iters = std::max(loop_iters, it);
            if (h->prof.on) {
                // first iteration: luma and motion of every frame, O, SDo, E out
                // (forward terms: the frame-minor luma read back, E read and
                // written again, the diagonal sums written)
                h->prof.bytes[K_ENERGY_INIT] +=
                    H * (2.0 * Tb * W + 10.0 * W) + (fwd ? H * (Tb * W + 12.0 * W) : 0.0);
                // recomputed pixels: 3 luma bytes of every frame, SDo read, E
                // write (and the diagonal sums)
                h->prof.bytes[K_ENERGY_ITER] += (double)hdirty[b] * (3.0 * Tb + (fwd ? 12.0 : 8.0));
            }
        }
    }
    if (h->prof.on) {
        h->prof.bytes[K_GATHER] += (double)H * target_W * (6.0 * T + 2.0 * nb);
        if (remove == 0) h->prof.bytes[K_IDENTITY] += 2.0 * H * W * nb;
    }
    // the device-side loop ran whole bodies of CARVE_LOOP_ITERS DP + update
    // launches and one condition kernel, up to the longest buffer's iterations
    if (carve_looped)
        launched += (long long)std::max(1, (loop_iters + CARVE_LOOP_ITERS - 1) / CARVE_LOOP_ITERS) *
                    (2LL * CARVE_LOOP_ITERS + 1);
    h->last_launches = launched;
    int *herr = reinterpret_cast<int *>(h->h_small.as<char>());
    SCPL_CUDA(h, cudaMemcpyAsync(herr, ws.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCPL_CUDA(h, cudaStreamSynchronize(st));
    if (*herr == DEV_ETIMEOUT)
        return fail(h, SCPL_ETIMEOUT, "a bounded device-side wait ran out while carving");
    if (*herr != DEV_OK)
        return fail(h, SCPL_ECUDA, "internal consistency check failed on the device (%d)", *herr);
    if (buffer_starts) std::copy(starts.begin(), starts.end(), buffer_starts);
    if (n_buffers) *n_buffers = nb;
    return SCPL_OK;
}

}  // namespace

extern "C" {

void scpl_default_params(scpl_params *p) {
    if (!p) return;
    p->alpha = 0.20;
    p->wg = 1;
    p->wm = 2;
    p->t_max = 128;
    p->use_buffer = 1;
    p->maxval_mode = 0;
    p->wf = 0;
}

scpl_status scpl_create(const scpl_params *p, void *stream, scpl_handle *out) {
    if (!out) return SCPL_EINVAL;
    *out = nullptr;
    scpl_params def;
    scpl_default_params(&def);
    if (!p) p = &def;
    if (check_params(p) != SCPL_OK) return SCPL_EINVAL;
    scpl_ctx *h = new (std::nothrow) scpl_ctx();
    if (!h) return SCPL_ENOMEM;
    h->p = *p;
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return SCPL_ECUDA;
    }
    *out = h;
    return SCPL_OK;
}

scpl_status scpl_set_stream(scpl_handle h, void *stream) {
    if (!h) return SCPL_EINVAL;
    h->stream = (cudaStream_t)stream;
    return SCPL_OK;
}

void scpl_destroy(scpl_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    DevBuf *bufs[] = {&h->Y, &h->D, &h->ering, &h->S1, &h->S2, &h->partA, &h->partM,
                      &h->count, &h->starts, &h->nbuf, &h->errw, &h->E0, &h->cws, &h->bof,
                      &h->in_frames, &h->out_frames, &h->seams_dev, &h->Yfm, &h->qY,
                      &h->qacc, &h->in2, &h->out2, &h->Yprev, &h->ej_mid, &h->ej_tin,
                      &h->ej_tout};
    if (h->istream) cudaStreamSynchronize(h->istream);
    if (h->cstream) cudaStreamSynchronize(h->cstream);
    if (h->gstream) cudaStreamSynchronize(h->gstream);
    for (DevBuf *b : bufs) b->release();
    engine_destroy(h->engine);
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    if (h->istream) cudaStreamDestroy(h->istream);
    for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
    if (h->loop) cudaGraphExecDestroy(h->loop);
    if (h->lstream) cudaStreamDestroy(h->lstream);
    h->h_small.release();
    delete h;
}

const char *scpl_last_error(scpl_handle h) { return h ? h->err.c_str() : "null handle"; }

scpl_status scpl_energy(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                        int32_t *energy) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!energy) return fail(h, SCPL_EINVAL, "energy is NULL");
    SCPL_CUDA(h, timed(h, K_ENERGY_API, [&] {
                  return launch_energy_api(frames, T, H, W, h->p.wg, h->p.wm, energy, h->stream);
              }));
    if (h->prof.on) h->prof.bytes[K_ENERGY_API] += 7.0 * T * H * W;
    return SCPL_OK;
}

scpl_status scpl_scan(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                      int32_t *buffer_starts, int *n_buffers) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if ((s = check_overflow(h, T, H)) != SCPL_OK) return s;
    std::vector<int> starts;
    if ((s = run_scan(h, frames, T, H, W, starts, false)) != SCPL_OK) return s;
    if (buffer_starts) std::copy(starts.begin(), starts.end(), buffer_starts);
    if (n_buffers) *n_buffers = (int)starts.size() - 1;
    return SCPL_OK;
}

scpl_status scpl_scan_arrivals(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                               const uint32_t *arrived, int chunk, int32_t *buffer_starts,
                               int *n_buffers) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!arrived) return fail(h, SCPL_EINVAL, "arrived is NULL");
    if (chunk < 1) return fail(h, SCPL_EINVAL, "chunk=%d must be >= 1", chunk);
    if ((s = check_overflow(h, T, H)) != SCPL_OK) return s;
    std::vector<int> starts;
    if ((s = run_scan(h, frames, T, H, W, starts, false, nullptr, nullptr, arrived, chunk)) !=
        SCPL_OK)
        return s;
    if (buffer_starts) std::copy(starts.begin(), starts.end(), buffer_starts);
    if (n_buffers) *n_buffers = (int)starts.size() - 1;
    return SCPL_OK;
}

scpl_status scpl_signal_arrival(void *stream, uint32_t *counter, uint32_t value) {
    if (!counter) return SCPL_EINVAL;
    PFN_cuStreamWriteValue32_v11070 write_value = stream_write_value();
    if (!write_value) return SCPL_ECUDA;
    return write_value(reinterpret_cast<CUstream>(stream), reinterpret_cast<CUdeviceptr>(counter),
                       (cuuint32_t)value, CU_STREAM_WRITE_VALUE_DEFAULT) == CUDA_SUCCESS
               ? SCPL_OK
               : SCPL_ECUDA;
}

scpl_status scpl_enlarge(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                         int target_W, int k, uint8_t *out, int32_t *buffer_starts,
                         int *n_buffers) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!out) return fail(h, SCPL_EINVAL, "out is NULL");
    if (k < 1) return fail(h, SCPL_EINVAL, "k=%d must be >= 1", k);
    const int m = target_W - W;
    if (m < 0 || m > W - 2)
        return fail(h, SCPL_EINVAL, "target_W=%d must be in [W, 2W-2] for W=%d", target_W, W);
    cudaStream_t st = h->stream;
    if (m == 0) {
        SCPL_CUDA(h, cudaMemcpyAsync(out, frames, (size_t)T * H * W * 3, cudaMemcpyDeviceToDevice,
                                     st));
        SCPL_CUDA(h, cudaStreamSynchronize(st));
        if (buffer_starts) {
            buffer_starts[0] = 0;
            buffer_starts[1] = T;
        }
        if (n_buffers) *n_buffers = 1;
        return SCPL_OK;
    }
    // the seams carving removes, from a scratch copy carved to W - m
    SCPL_CUDA(h, h->out_frames.ensure((size_t)T * H * (W - m) * 3));
    SCPL_CUDA(h, h->seams_dev.ensure((size_t)T * m * H * sizeof(int16_t)));
    std::vector<int> starts(T + 1);
    int nb = 0;
    if ((s = carve_run(h, frames, T, H, W, W - m, k, h->out_frames.as<uint8_t>(), starts.data(),
                       &nb, h->seams_dev.as<int16_t>(), nullptr, 1, nullptr)) != SCPL_OK)
        return s;
    // h->starts still holds the scan's buffer starts on the device
    SCPL_CUDA(h, launch_insert_seams(frames, H, W, target_W, h->seams_dev.as<int16_t>(),
                                     (long)m * H, m, h->starts.as<int>(), nb, out, st));
    SCPL_CUDA(h, cudaStreamSynchronize(st));
    if (buffer_starts) std::copy(starts.begin(), starts.begin() + nb + 1, buffer_starts);
    if (n_buffers) *n_buffers = nb;
    return SCPL_OK;
}

scpl_status scpl_enlarge_job(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                             int target_W, int target_H, int k, uint8_t *out) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!out) return fail(h, SCPL_EINVAL, "out is NULL");
    if (k < 1) return fail(h, SCPL_EINVAL, "k=%d must be >= 1", k);
    if (target_W < W || target_W > std::max(W, 2 * W - 2))
        return fail(h, SCPL_EINVAL, "target_W=%d must be in [W, 2W-2] for W=%d", target_W, W);
    if (target_H < H || target_H > std::max(H, 2 * H - 2))
        return fail(h, SCPL_EINVAL, "target_H=%d must be in [H, 2H-2] for H=%d", target_H, H);
    if (target_H == H) return scpl_enlarge(h, frames, T, H, W, target_W, k, out, nullptr, nullptr);
    if (H > 8192) return fail(h, SCPL_EINVAL, "H=%d exceeds 8192 for a height enlargement", H);
    cudaStream_t st = h->stream;
    // the width first, into a scratch clip
    const uint8_t *mid = frames;
    if (target_W > W) {
        SCPL_CUDA(h, h->ej_mid.ensure((size_t)T * H * target_W * 3));
        if ((s = scpl_enlarge(h, frames, T, H, W, target_W, k, h->ej_mid.as<uint8_t>(), nullptr,
                              nullptr)) != SCPL_OK)
            return s;
        mid = h->ej_mid.as<uint8_t>();
    }
    // the height as the width of the transposed clip, then back
    SCPL_CUDA(h, h->ej_tin.ensure((size_t)T * target_W * H * 3));
    SCPL_CUDA(h, h->ej_tout.ensure((size_t)T * target_W * target_H * 3));
    SCPL_CUDA(h, launch_transpose_rgb(mid, T, H, target_W, h->ej_tin.as<uint8_t>(), st));
    if ((s = scpl_enlarge(h, h->ej_tin.as<uint8_t>(), T, target_W, H, target_H, k,
                          h->ej_tout.as<uint8_t>(), nullptr, nullptr)) != SCPL_OK)
        return s;
    SCPL_CUDA(h, launch_transpose_rgb(h->ej_tout.as<uint8_t>(), T, target_W, target_H, out, st));
    SCPL_CUDA(h, cudaStreamSynchronize(st));
    return SCPL_OK;
}

scpl_status scpl_blend_sharpness(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                                 int window, int64_t *num, int64_t *den) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!num || !den) return fail(h, SCPL_EINVAL, "num and den must not be NULL");
    if (window < 1 || window > 64) return fail(h, SCPL_EINVAL, "window=%d outside [1, 64]", window);
    *num = *den = 0;
    if (T < window) return SCPL_OK;
    cudaStream_t st = h->stream;
    SCPL_CUDA(h, h->qY.ensure((size_t)T * H * W));
    SCPL_CUDA(h, h->qacc.ensure(16));
    SCPL_CUDA(h, h->h_small.ensure(16));
    SCPL_CUDA(h, cudaMemsetAsync(h->qacc.p, 0, 16, st));
    SCPL_CUDA(h, launch_blend_sharpness(frames, T, H, W, window, h->qY.as<uint8_t>(),
                                        h->qacc.as<unsigned long long>(), st));
    unsigned long long *hs = h->h_small.as<unsigned long long>();
    SCPL_CUDA(h, cudaMemcpyAsync(hs, h->qacc.p, 16, cudaMemcpyDeviceToHost, st));
    SCPL_CUDA(h, cudaStreamSynchronize(st));
    *num = (int64_t)hs[0];
    *den = (int64_t)hs[1];
    return SCPL_OK;
}

scpl_status scpl_isqrt(const uint64_t *x, uint32_t *r, long n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !r))) return SCPL_EINVAL;
    if (launch_isqrt_check(reinterpret_cast<const unsigned long long *>(x), r, n,
                           static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SCPL_ECUDA;
    return SCPL_OK;
}

scpl_status scpl_set_wait_limit(scpl_handle h, uint64_t ns) {
    if (!h) return SCPL_EINVAL;
    if (ns < 100000ull || ns > 60000000000ull)
        return fail(h, SCPL_EINVAL, "wait limit %llu ns outside [1e5, 6e10]",
                    (unsigned long long)ns);
    h->wait_ns = ns;
    return SCPL_OK;
}

scpl_status scpl_scan_stats(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                            int32_t *buffer_starts, int *n_buffers, int64_t *A, int32_t *emax) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!A || !emax) return fail(h, SCPL_EINVAL, "A and emax must not be NULL");
    if ((s = check_overflow(h, T, H)) != SCPL_OK) return s;
    std::vector<int> starts;
    std::vector<long long> a(T);
    if ((s = run_scan(h, frames, T, H, W, starts, false, a.data(), emax)) != SCPL_OK) return s;
    for (int t = 0; t < T; ++t) A[t] = a[t];
    if (buffer_starts) std::copy(starts.begin(), starts.end(), buffer_starts);
    if (n_buffers) *n_buffers = (int)starts.size() - 1;
    return SCPL_OK;
}

scpl_status scpl_seams(scpl_handle h, const int32_t *energy, int H, int W, int k, int16_t *cols,
                       int *k_eff) {
    scpl_status s = check_frames(h, energy, 1, H, W);
    if (s != SCPL_OK) return s;
    if (!cols || !k_eff) return fail(h, SCPL_EINVAL, "cols and k_eff must not be NULL");
    if (k < 1) return fail(h, SCPL_EINVAL, "k=%d must be >= 1", k);
    CarveWs ws;
    int kc = std::min(k, W);
    if ((s = carve_ws(h, 1, H, W, kc, ws)) != SCPL_OK) return s;
    ws.wf = 0;   // a caller's energy map comes without frames: no forward terms
    cudaStream_t st = h->stream;
    SCPL_CUDA(h, cudaMemsetAsync(ws.err, 0, sizeof(int), st));
    SCPL_CUDA(h, cudaMemcpy2DAsync(ws.E, ws.pitch * sizeof(int32_t), energy,
                                   (size_t)W * sizeof(int32_t), (size_t)W * sizeof(int32_t), H,
                                   cudaMemcpyDeviceToDevice, st));
    SCPL_CUDA(h, timed(h, K_IDENTITY, [&] { return launch_identity_O(ws, 1, st); }));
    SCPL_CUDA(h, h->h_small.ensure(64 + sizeof(BufState)));
    BufState *hb = reinterpret_cast<BufState *>(h->h_small.as<char>() + 64);
    SCPL_CUDA(h, cudaStreamSynchronize(st));   // the staging area is reused below
    *hb = BufState{0, 1, W, 0, 0, 0, W - kc, 0, 0, 0, 0, -1};
    SCPL_CUDA(h, cudaMemcpyAsync(ws.st, hb, sizeof(BufState), cudaMemcpyHostToDevice, st));
    SCPL_CUDA(h, timed(h, K_DP_SELECT, [&] {
                  return ws.J ? launch_dpc(ws, 1, k, cols, 0, st)
                              : launch_dp_select(ws, 1, k, cols, 0, st);
              }));
    SCPL_CUDA(h, cudaMemcpyAsync(hb, ws.st, sizeof(BufState), cudaMemcpyDeviceToHost, st));
    int *herr = reinterpret_cast<int *>(h->h_small.as<char>());
    SCPL_CUDA(h, cudaMemcpyAsync(herr, ws.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCPL_CUDA(h, cudaStreamSynchronize(st));
    if (*herr == DEV_ETIMEOUT)
        return fail(h, SCPL_ETIMEOUT, "a bounded device-side wait ran out in the DP");
    if (*herr != DEV_OK)
        return fail(h, SCPL_ECUDA, "internal consistency check failed on the device (%d)", *herr);
    *k_eff = hb->k_eff;
    return SCPL_OK;
}

scpl_status scpl_carve(scpl_handle h, const uint8_t *frames, int T, int H, int W, int target_W,
                       int k, uint8_t *out, int32_t *buffer_starts, int *n_buffers,
                       int16_t *seams) {
    return carve_run(h, frames, T, H, W, target_W, k, out, buffer_starts, n_buffers, seams,
                     nullptr, 1, nullptr);
}

scpl_status scpl_carve_buffer(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                              const uint8_t *prev_frame, int target_W, int k, uint8_t *out,
                              int16_t *seams) {
    if (!h) return SCPL_EINVAL;
    if (T > effective_tmax(h->p))
        return fail(h, SCPL_EINVAL, "a fixed buffer holds at most t_max = %d frames, not %d",
                    effective_tmax(h->p), T);
    return carve_run(h, frames, T, H, W, target_W, k, out, nullptr, nullptr, seams, nullptr, 1,
                     nullptr, nullptr, prev_frame, true);
}

scpl_status scpl_carve_host(scpl_handle h, const uint8_t *frames, int T, int H, int W,
                            int target_W, int k, uint8_t *out, int32_t *buffer_starts,
                            int *n_buffers, int16_t *seams) {
    scpl_status s = check_frames(h, frames, T, H, W);
    if (s != SCPL_OK) return s;
    if (!out) return fail(h, SCPL_EINVAL, "out is NULL");
    if (target_W < 2 || target_W > W)
        return fail(h, SCPL_EINVAL, "target_W=%d must be in [2, W=%d]", target_W, W);
    const size_t frame_in = (size_t)H * W * 3;
    const size_t in_bytes = (size_t)T * frame_in;
    const size_t seam_bytes = (size_t)T * (W - target_W) * H * sizeof(int16_t);
    SCPL_CUDA(h, h->in_frames.ensure(in_bytes));
    SCPL_CUDA(h, h->out_frames.ensure((size_t)T * H * target_W * 3));
    if (seams) SCPL_CUDA(h, h->seams_dev.ensure(std::max<size_t>(seam_bytes, 2)));
    if (!h->cstream) SCPL_CUDA(h, cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    if (!h->gstream) SCPL_CUDA(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    cudaStream_t st = h->stream;
    // The frames go up by the link-copy kernel before the scan reads them (no
    // kernel here waits on another); the carved frames come back per buffer as
    // the buffers finish, by the same kernel on the copy stream.
    SCPL_CUDA(h, link_copy(h->in_frames.p, frames, in_bytes, st));
    int nb = 0;
    std::vector<int> starts(T + 1);
    s = carve_run(h, h->in_frames.as<uint8_t>(), T, H, W, target_W, k,
                  h->out_frames.as<uint8_t>(), starts.data(), &nb,
                  seams ? h->seams_dev.as<int16_t>() : nullptr, nullptr, 1, out);
    cudaError_t e1 = cudaStreamSynchronize(h->cstream);
    cudaError_t e2 = cudaStreamSynchronize(h->gstream);
    if (s != SCPL_OK) return s;
    SCPL_CUDA(h, e1);
    SCPL_CUDA(h, e2);
    if (seams)
        SCPL_CUDA(h, cudaMemcpyAsync(seams, h->seams_dev.p,
                                     (size_t)nb * (W - target_W) * H * sizeof(int16_t),
                                     cudaMemcpyDeviceToHost, st));
    SCPL_CUDA(h, cudaStreamSynchronize(st));
    if (buffer_starts) std::copy(starts.begin(), starts.begin() + nb + 1, buffer_starts);
    if (n_buffers) *n_buffers = nb;
    return SCPL_OK;
}

scpl_status scpl_carve_host_many(scpl_handle h, int n, const uint8_t *const *frames, int T,
                                 int H, int W, int target_W, int k, uint8_t *const *out,
                                 int *n_buffers) {
    if (!h) return SCPL_EINVAL;
    if (n < 0 || (n > 0 && (!frames || !out))) return fail(h, SCPL_EINVAL, "bad clip lists");
    if (n == 0) return SCPL_OK;
    for (int i = 0; i < n; ++i) {
        scpl_status s = check_frames(h, frames[i], T, H, W);
        if (s != SCPL_OK) return s;
        if (!out[i]) return fail(h, SCPL_EINVAL, "out[%d] is NULL", i);
    }
    if (target_W < 2 || target_W > W)
        return fail(h, SCPL_EINVAL, "target_W=%d must be in [2, W=%d]", target_W, W);
    const size_t frame_in = (size_t)H * W * 3;
    const size_t in_bytes = (size_t)T * frame_in, out_bytes = (size_t)T * H * target_W * 3;
    SCPL_CUDA(h, h->in_frames.ensure(in_bytes));
    SCPL_CUDA(h, h->in2.ensure(in_bytes));
    SCPL_CUDA(h, h->out_frames.ensure(out_bytes));
    SCPL_CUDA(h, h->out2.ensure(out_bytes));
    if (!h->cstream) SCPL_CUDA(h, cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    if (!h->gstream) SCPL_CUDA(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    if (!h->istream) SCPL_CUDA(h, cudaStreamCreateWithFlags(&h->istream, cudaStreamNonBlocking));
    cudaStream_t st = h->stream;
    uint8_t *in_slot[2] = {h->in_frames.as<uint8_t>(), h->in2.as<uint8_t>()};
    uint8_t *out_slot[2] = {h->out_frames.as<uint8_t>(), h->out2.as<uint8_t>()};
    // up[s]: the clip in slot s is on the device; done[s]: every read of the
    // slot's input (the gathers) and of its output (the copies back) has
    // finished, so the slot may take the next clip
    cudaEvent_t up[2] = {}, done[2] = {};
    struct Guard {
        cudaEvent_t *a, *b;
        ~Guard() {
            for (int s = 0; s < 2; ++s) {
                if (a[s]) cudaEventDestroy(a[s]);
                if (b[s]) cudaEventDestroy(b[s]);
            }
        }
    } guard{up, done};
    for (int s = 0; s < 2; ++s) {
        SCPL_CUDA(h, cudaEventCreateWithFlags(&up[s], cudaEventDisableTiming));
        SCPL_CUDA(h, cudaEventCreateWithFlags(&done[s], cudaEventDisableTiming));
    }
    // the caller's earlier work on the handle's stream comes first
    SCPL_CUDA(h, cudaEventRecord(done[0], st));
    SCPL_CUDA(h, cudaEventRecord(done[1], st));
    // Clip i's frames go up into slot i & 1 by the link-copy kernel on the
    // input stream.  Clip i+1's upload is issued once clip i's scan has
    // finished, so it runs beside clip i's carving and never beside a scan;
    // clip i+1's scan waits for it by an event.  No kernel waits on another.
    auto upload = [&](int i) -> scpl_status {
        const int s = i & 1;
        SCPL_CUDA(h, cudaStreamWaitEvent(h->istream, done[s], 0));
        SCPL_CUDA(h, link_copy(in_slot[s], frames[i], in_bytes, h->istream));
        SCPL_CUDA(h, cudaEventRecord(up[s], h->istream));
        return SCPL_OK;
    };
    scpl_status s = upload(0);
    std::vector<int> starts(T + 1);
    for (int i = 0; i < n && s == SCPL_OK; ++i) {
        const int sl = i & 1;
        SCPL_CUDA(h, cudaStreamWaitEvent(st, up[sl], 0));
        int nb = 0;
        const std::function<scpl_status()> next = [&]() -> scpl_status {
            return i + 1 < n ? upload(i + 1) : SCPL_OK;
        };
        s = carve_run(h, in_slot[sl], T, H, W, target_W, k, out_slot[sl], starts.data(), &nb,
                      nullptr, nullptr, 1, out[i], next);
        if (s != SCPL_OK) break;
        if (n_buffers) n_buffers[i] = nb;
        // every gather is followed on the copy stream by its buffer's copy
        // back, which waits for it: the slot is free once the copy stream
        // reaches this point
        SCPL_CUDA(h, cudaEventRecord(done[sl], h->cstream));
    }
    cudaError_t e1 = cudaStreamSynchronize(h->istream);
    cudaError_t e2 = cudaStreamSynchronize(h->gstream);
    cudaError_t e3 = cudaStreamSynchronize(h->cstream);
    if (s != SCPL_OK) return s;
    SCPL_CUDA(h, e1);
    SCPL_CUDA(h, e2);
    SCPL_CUDA(h, e3);
    return SCPL_OK;
}

scpl_status scpl_carve_batch(scpl_handle h, scpl_job *jobs, int n_jobs) {
    if (!h) return SCPL_EINVAL;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(h, SCPL_EINVAL, "bad job list");
    if (n_jobs == 0) return SCPL_OK;
    std::string err;
    scpl_status s = engine_run_batch(&h->engine, h->p, h->stream, h->autotune, jobs, n_jobs, err);
    if (s != SCPL_OK) return fail(h, s, "%s", err.c_str());
    return SCPL_OK;
}

scpl_status scpl_batch_stats(scpl_handle h, scpl_server_stats *out) {
    if (!h || !out) return SCPL_EINVAL;
    return engine_stats(h->engine, out);
}

scpl_status scpl_tune(scpl_handle h, int H, int W, int k, scpl_tuning *out) {
    if (!h) return SCPL_EINVAL;
    if (H < 1 || H > 65535 || W < 4 || W > 8192 || k < 1)
        return fail(h, SCPL_EINVAL, "cannot tune H=%d W=%d k=%d", H, W, k);
    scpl_status s = tune_class(H, W, k, h->stream, out);
    if (s != SCPL_OK) return fail(h, s, "tuning H=%d W=%d failed", H, W);
    return SCPL_OK;
}

scpl_status scpl_tuning_set(const scpl_tuning *t) {
    if (!t || t->H < 1 || t->W < 1) return SCPL_EINVAL;
    if (t->dpc_halo != 0 && t->dpc_halo != 16 && t->dpc_halo != 32) return SCPL_EINVAL;
    if (t->dpc_halo != 0 && t->dpc_warps != 4 && t->dpc_warps != 8) return SCPL_EINVAL;
    if (t->dpc_halo != 0 && t->dpc_lane_cols != 4 &&
        !(t->dpc_lane_cols == 2 && t->dpc_halo == 16))
        return SCPL_EINVAL;
    if (t->update_rows != 1 && t->update_rows != 2 && t->update_rows != 4) return SCPL_EINVAL;
    tuning_store(*t);
    return SCPL_OK;
}

scpl_status scpl_tuning_get(int H, int W, scpl_tuning *out) {
    if (!out) return SCPL_EINVAL;
    return tuning_lookup(H, W, out) ? SCPL_OK : SCPL_EINVAL;
}

void scpl_tuning_clear(void) { tuning_clear(); }

int scpl_keff_log(scpl_handle h, int32_t *keff, int max, int32_t *iters) {
    if (!h) return -1;
    const int n = (int)h->last_keff.size();
    for (int i = 0; keff && i < n && i < max; ++i) keff[i] = h->last_keff[i];
    if (iters)
        for (int b = 0; b < (int)h->last_iters.size(); ++b) iters[b] = h->last_iters[b];
    return n;
}

int scpl_tuning_list(scpl_tuning *out, int max) { return tuning_list(out, max < 0 ? 0 : max); }

scpl_status scpl_set_autotune(scpl_handle h, int on) {
    if (!h) return SCPL_EINVAL;
    h->autotune = on != 0;
    return SCPL_OK;
}

scpl_status scpl_set_profiling(scpl_handle h, int on) {
    if (!h) return SCPL_EINVAL;
    if (on) {
        SCPL_CUDA(h, cudaStreamSynchronize(h->stream));
        h->prof.clear();
    }
    h->prof.on = on != 0;
    return SCPL_OK;
}

scpl_status scpl_get_stats(scpl_handle h, scpl_stats *out) {
    if (!h || !out) return SCPL_EINVAL;
    SCPL_CUDA(h, cudaStreamSynchronize(h->stream));
    Profiler &pr = h->prof;
    for (auto &m : pr.marks) {
        float ms = 0.f;
        SCPL_CUDA(h, cudaEventElapsedTime(&ms, pr.pool[m.second], pr.pool[m.second + 1]));
        pr.ms[m.first] += ms;
        pr.launches[m.first] += 1;
    }
    pr.marks.clear();
    pr.used = 0;
    std::memset(out, 0, sizeof *out);
    out->n_buffers = h->last_nb;
    out->iterations_max = h->last_iter_max;
    out->iterations_total = h->last_iter_total;
    out->carved_px = h->last_carved_px;
    out->launches = h->last_launches;
    int n = 0;
    for (int i = 0; i < K_COUNT && n < 8; ++i) {
        if (pr.launches[i] == 0 && pr.bytes[i] == 0) continue;
        scpl_kernel_stat &ks = out->kernel[n++];
        std::snprintf(ks.name, sizeof ks.name, "%s", kKernelNames[i]);
        ks.launches = pr.launches[i];
        ks.ms = pr.ms[i];
        ks.bytes = pr.bytes[i];
    }
    out->n_kernels = n;
    return SCPL_OK;
}

}  // extern "C"
