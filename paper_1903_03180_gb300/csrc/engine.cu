// Batching and serving: many retarget jobs carved together on one GPU.
//
// The paper carves one video at a time (Sec. 3, 4).  This engine runs the same
// kernels over many clips at once and gives every clip the result that
// scpl_carve gives it alone.
//
// A job is split into passes.  A pass carves vertical seams out of a
// [T][H][W][3] clip down to a target width.  A job that shrinks the height has
// a pass on the transposed frames; a job that shrinks both has two passes.
// A pass goes through:
//   scan   one cooperative launch (k_scan) for every pass waiting to be
//          scanned; each clip gets its own range of CTAs and its own device-wide
//          waits, so clips of any size share the launch.  The luma and motion
//          maps land in the pool of the pass's group.
//   group  passes of the same (H, W) scanned in the same wave form a group.
//          Their spatiotemporal buffers become the items of one carving
//          workspace, so one k_energy_init, one DP launch and one k_update
//          launch per iteration serve every buffer of every clip in the group.
//   carve  for scpl_carve_batch, one launch of a CUDA graph whose
//          conditional WHILE node repeats a body of LOOP_ITERS DP + update
//          launches followed by a one-thread kernel that reads the item
//          states and sets the loop's condition (some item still above its
//          target, no device error), so the GPU runs the group's iterations
//          to the end with no host in the loop.  Servers, whose groups are
//          small and many, and builds where conditional nodes are
//          unavailable carve in chunks of q iterations captured once per
//          (group, q), with the item states read back after each chunk to
//          size the next (measured: serving at 100 requests/s gave 6,681
//          frames/s with chunks against 5,828 with the loop).  Items that
//          reach their target width become no-ops in later launches.
//   gather one launch per group for the colour frames of all its passes, then
//          transposes for horizontal passes and the copy back for host jobs.
// Each group runs on one of 16 streams, so groups of different sizes, and jobs
// admitted while others are carving, overlap on the GPU.
//
// Memory: every allocation is stream-ordered from the engine's own pool.  A
// job is admitted only when its footprint fits the budget.  The footprint
// counts one buffer per pass, and more buffers are added when the scan finds
// them.  Admission pauses while a group waits for memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "scpl.h"
#include "scpl_internal.cuh"

using namespace scpl;

namespace {

constexpr int N_STREAMS = 16;
constexpr int MAX_CHUNK = 16;
constexpr int LOOP_ITERS = 4;   // DP + update pairs per body of the device-side loop
constexpr unsigned long long SPIN_NS = 2000000000ull;   // bounded device-wide waits

long rup(long v, long m) { return (v + m - 1) / m * m; }
size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

long long emax_of(const scpl_params &p) { return 255LL * (8LL * p.wg + p.wm); }
int tmax_of(const scpl_params &p) { return p.use_buffer ? p.t_max : 1; }

// Page-locked host blocks, reused between waves and groups.
struct Pinned {
    void *p = nullptr;
    size_t n = 0;
};
struct PinnedPool {
    std::vector<Pinned> free_, all_;
    cudaError_t get(size_t bytes, Pinned &out) {
        for (size_t i = 0; i < free_.size(); ++i)
            if (free_[i].n >= bytes) {
                out = free_[i];
                free_.erase(free_.begin() + i);
                return cudaSuccess;
            }
        bytes = std::max<size_t>(a256(bytes), 4096);
        void *p = nullptr;
        cudaError_t e = cudaMallocHost(&p, bytes);
        if (e != cudaSuccess) return e;
        out = Pinned{p, bytes};
        all_.push_back(out);
        return cudaSuccess;
    }
    void put(Pinned b) {
        if (b.p) free_.push_back(b);
    }
    ~PinnedPool() {
        for (auto &b : all_) cudaFreeHost(b.p);
    }
};

// Geometry of one pass in carving orientation.
struct PassDims {
    int T, H, W, target;
};

// Bytes of one pass's scan state (freed with its wave) and of one carving
// buffer (item) of the pass.
size_t scan_state_bytes(const PassDims &d) {
    const size_t spx = (size_t)scan_state_px(d.H, d.W);
    const size_t G = (size_t)scan_tiles(d.H, d.W);
    (void)G;
    return a256((size_t)SCAN_FW * spx * 2) + 2 * a256(spx * 4) + a256((size_t)(d.T + 1) * 4) +
           a256((size_t)d.T * (8 * SCAN_FW + 8) + 8);
}
// Buffers of a pass whose summed energy the scan keeps (more are summed by
// k_energy_init from the luma and motion maps).
int e0_planes(const PassDims &d) { return std::min(d.T, 4); }
size_t e0_bytes(const PassDims &d) { return a256((size_t)e0_planes(d) * d.H * d.W * 4); }
size_t item_bytes(const PassDims &d, int kcap, int wf) {
    CarveWs ws{};
    ws.H = d.H;
    ws.W0 = d.W;
    ws.kcap = kcap;
    ws.wf = wf;
    return carve_ws_assign(ws, 1, d.W - d.target, true, nullptr);
}
size_t pass_bytes(const PassDims &d, int k, int wf) {
    const size_t yp = (size_t)rup(d.W, 16);
    const size_t ypool = 2 * (size_t)d.T * d.H * yp;
    const size_t yfm = (size_t)d.H * d.W * rup(d.T, 16);
    const int kcap = std::max(1, std::min(k, d.W - d.target));
    return ypool + e0_bytes(d) + scan_state_bytes(d) + item_bytes(d, kcap, wf) + yfm +
           (size_t)d.T * 32;
}

// The passes of a job: width first, then height on the transposed frames.
int job_passes(const scpl_job &j, PassDims out[2]) {
    int n = 0;
    int Wc = j.W;
    if (j.target_W < j.W) {
        out[n++] = PassDims{j.T, j.H, j.W, j.target_W};
        Wc = j.target_W;
    }
    if (j.target_H < j.H) out[n++] = PassDims{j.T, Wc, j.H, j.target_H};
    return n;
}

size_t rgb_bytes(int T, int H, int W) { return (size_t)T * H * W * 3; }

// Device memory the job owns outside its groups.
size_t job_own_bytes(const scpl_job &j) {
    size_t b = 0;
    const int Wc = j.target_W;
    if (j.on_host) b += rgb_bytes(j.T, j.H, j.W) + rgb_bytes(j.T, j.target_H, j.target_W);
    if (j.target_H < j.H) {
        if (j.target_W < j.W) b += rgb_bytes(j.T, j.H, Wc);   // width pass output
        b += rgb_bytes(j.T, Wc, j.H);                          // transposed input
        b += rgb_bytes(j.T, Wc, j.target_H);                   // transposed output
    }
    return b;
}

scpl_status check_job(const scpl_params &p, const scpl_job &j) {
    if (!j.frames || !j.out) return SCPL_EINVAL;
    if (j.T < 1 || j.H < 1 || j.W < 1 || j.k < 1) return SCPL_EINVAL;
    if (j.H > 8192 || j.W > 8192) return SCPL_EINVAL;
    if (j.target_W < 2 || j.target_W > j.W || j.target_H < 2 || j.target_H > j.H)
        return SCPL_EINVAL;
    PassDims d[2];
    const int n = job_passes(j, d);
    const long long em = emax_of(p);
    const long long tb = std::min<long long>(j.T, tmax_of(p));
    if (em >= 65536 || (long long)tmax_of(p) * em * em >= (1LL << 32)) return SCPL_EOVERFLOW;
    for (int i = 0; i < n; ++i) {
        if (dp_row_max(em, tb, p.wf) * d[i].H >= (1LL << 31)) return SCPL_EOVERFLOW;
        int bb = 0, rb = 0;
        const int kcap = std::max(1, std::min(j.k, d[i].W - d[i].target));
        if (dp_smem_bytes(d[i].W, d[i].H, &bb) > 227 * 1024 - 4096 ||
            update_smem_bytes(d[i].W, kcap, &rb, p.wf > 0) > 200 * 1024)
            return SCPL_EINVAL;
    }
    return SCPL_OK;
}

size_t footprint(const scpl_params &p, const scpl_job &j) {
    if (check_job(p, j) != SCPL_OK) return 0;
    PassDims d[2];
    const int n = job_passes(j, d);
    size_t b = job_own_bytes(j);
    for (int i = 0; i < n; ++i) b += pass_bytes(d[i], j.k, p.wf);
    return b;
}

enum JobState { J_QUEUED, J_ACTIVE, J_FINISHING, J_DONE };

struct Job {
    scpl_job spec;
    scpl_job *user = nullptr;   // batch mode: results are written back here
    long long ticket = 0;
    int state = J_QUEUED;
    int status = SCPL_OK;
    size_t reserved = 0;
    std::vector<void *> owned;  // device allocations of the job itself
    const uint8_t *in_dev = nullptr;
    uint8_t *out_dev = nullptr;
    uint8_t *mid = nullptr, *tr_in = nullptr, *tr_out = nullptr;
    cudaEvent_t done = nullptr;
    int npass = 0;
};

struct Pass {
    int job = -1;
    int index = 0;              // 0 or 1 within its job
    bool transposed = false;    // carving the transposed frames
    const uint8_t *src = nullptr;
    uint8_t *dst = nullptr;
    PassDims d{};
    int k = 1;
    cudaEvent_t ready = nullptr;   // src complete (null: ordered on the main stream)
    int group = -1;
    int frame_off = 0;
    bool item = false;          // its buffers are items of its carving group
    long long e0_off = 0;       // element offset of its summed-energy planes
    int nb = 0, item0 = 0;
    std::vector<int> starts;
    size_t group_share = 0;     // bytes of its group attributed to this pass
};

struct Group {
    int H = 0, W = 0;
    long ypitch = 0;
    int T_total = 0;
    uint8_t *ypool = nullptr;
    size_t ypool_bytes = 0;
    char *slab = nullptr;
    size_t slab_bytes = 0;
    CarveWs ws{};
    int nb = 0;
    bool dpc = false;
    std::vector<int> passes;
    cudaStream_t stream = nullptr;
    Pinned hb;                  // states + err readback / upload staging
    cudaEvent_t ev = nullptr;
    int phase = 0;              // 0 scanning, 1 waiting for memory, 2 carving, 3 finished
    std::map<int, cudaGraphExec_t> graphs;   // q > 0: chunks; 0: the device-side loop
    bool looped = false;        // the carving ran as the device-side loop
    size_t held_after = 0;      // bytes of completed jobs still held by this group
    int wave = -1;
    size_t gt_off = 0;          // gather table in the slab
    int nframes = 0;
};

struct Wave {
    std::vector<int> passes;
    std::vector<int> groups;
    char *slab = nullptr;
    Pinned h;
    size_t res_off = 0;
    std::vector<size_t> res_pos;
    cudaEvent_t ev = nullptr;
    bool done = false;
};

}  // namespace

struct scpl_server_s {
    scpl_params p{};
    cudaStream_t user = nullptr;
    cudaStream_t main = nullptr;
    cudaStream_t pool[N_STREAMS] = {};
    int next_stream = 0;
    cudaMemPool_t mpool = nullptr;
    int device = 0;
    size_t budget = 0, reserved = 0, peak = 0;
    int scan_cap = 0;
    std::vector<std::unique_ptr<Job>> jobs;
    std::deque<int> queue;
    std::vector<Pass> passes;
    std::vector<std::unique_ptr<Group>> groups;
    std::vector<std::unique_ptr<Wave>> waves;
    std::vector<int> pending_scan;
    std::vector<std::pair<long long, int>> completed;
    PinnedPool pinned;
    std::string err;
    bool broken = false;
    long long next_ticket = 1;
    scpl_server_stats st{};
    int active_jobs = 0;
    bool autotune = false;
    bool device_loop = false;   // groups carve as one device-side loop (scpl_carve_batch)
    bool hold = false;          // admission waits for running work after a refusal
    long long refuse_skip = 0;  // injected allocator refusals (testing)
    int refuse_n = 0;
};

namespace {

using Srv = scpl_server_s;

scpl_status sfail(Srv *s, scpl_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s->err = buf;
    return code;
}

#define SRV_CUDA(s, call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (s)->broken = true;                                                            \
            return sfail(s, e_ == cudaErrorMemoryAllocation ? SCPL_ENOMEM : SCPL_ECUDA,     \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                  \
    } while (0)

// An allocation: a refusal returns SCPL_ENOMEM and leaves the server usable.
#define SRV_ALLOC(s, call)                                                                  \
    do {                                                                                   \
        cudaError_t ea_ = (call);                                                          \
        if (ea_ == cudaErrorMemoryAllocation)                                              \
            return sfail(s, SCPL_ENOMEM, "%s: refused (%s:%d)", #call, __FILE__, __LINE__);  \
        SRV_CUDA(s, ea_);                                                                  \
    } while (0)

// Device allocation from the engine's pool.  A refusal (the pool or the
// device is out of memory, or an injected refusal) leaves the server usable:
// the callers below delay or fail only the jobs that needed the memory.
cudaError_t dalloc(Srv *s, void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (s->refuse_n > 0) {
        if (s->refuse_skip > 0) {
            --s->refuse_skip;
        } else {
            --s->refuse_n;
            return cudaErrorMemoryAllocation;
        }
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), s->mpool, st);
    if (e == cudaErrorMemoryAllocation) cudaGetLastError();   // not sticky
    return e;
}

// Work in flight whose completion releases memory (or reports a job).
bool in_flight(Srv *s);
struct Group;
scpl_status free_group(Srv *s, Group &G);

void add_reserved(Srv *s, long long delta) {
    s->reserved = (size_t)((long long)s->reserved + delta);
    s->peak = std::max(s->peak, s->reserved);
}

void count_launches(Srv *s, long long n) { s->st.kernel_launches += n; }

// ---- admission --------------------------------------------------------------
scpl_status start_job(Srv *s, int jid) {
    Job &J = *s->jobs[jid];
    const scpl_job &j = J.spec;
    cudaStream_t m = s->main;
    auto own = [&](size_t bytes, uint8_t **out) -> cudaError_t {
        void *p = nullptr;
        cudaError_t e = dalloc(s, &p, bytes, m);
        if (e == cudaSuccess) {
            J.owned.push_back(p);
            *out = static_cast<uint8_t *>(p);
        }
        return e;
    };
    if (j.on_host) {
        uint8_t *in = nullptr;
        SRV_ALLOC(s, own(rgb_bytes(j.T, j.H, j.W), &in));
        SRV_CUDA(s, link_copy(in, j.frames, rgb_bytes(j.T, j.H, j.W), m));
        J.in_dev = in;
        SRV_ALLOC(s, own(rgb_bytes(j.T, j.target_H, j.target_W), &J.out_dev));
    } else {
        J.in_dev = j.frames;
        J.out_dev = j.out;
    }
    SRV_CUDA(s, cudaEventCreateWithFlags(&J.done, cudaEventDisableTiming));
    PassDims d[2];
    J.npass = job_passes(j, d);
    if (J.npass == 0) {   // nothing to carve: the output is the input
        SRV_CUDA(s, cudaMemcpyAsync(J.out_dev, J.in_dev, rgb_bytes(j.T, j.H, j.W),
                                    cudaMemcpyDeviceToDevice, m));
        if (j.on_host)
            SRV_CUDA(s, link_copy(j.out, J.out_dev, rgb_bytes(j.T, j.H, j.W), m));
        if (j.buffer_starts) {
            j.buffer_starts[0] = 0;
            j.buffer_starts[1] = j.T;
        }
        J.spec.n_buffers = 0;
        SRV_CUDA(s, cudaEventRecord(J.done, m));
        J.state = J_FINISHING;
        return SCPL_OK;
    }
    const bool both = J.npass == 2;
    const bool height_only = !both && d[0].W == j.H && j.target_H < j.H;
    if (both) SRV_ALLOC(s, own(rgb_bytes(j.T, j.H, j.target_W), &J.mid));
    if (j.target_H < j.H) {
        SRV_ALLOC(s, own(rgb_bytes(j.T, j.target_W, j.H), &J.tr_in));
        SRV_ALLOC(s, own(rgb_bytes(j.T, j.target_W, j.target_H), &J.tr_out));
    }
    Pass P;
    P.job = jid;
    P.index = 0;
    P.d = d[0];
    P.k = j.k;
    if (height_only) {
        SRV_CUDA(s, launch_transpose_rgb(J.in_dev, j.T, j.H, j.W, J.tr_in, m));
        count_launches(s, 1);
        P.transposed = true;
        P.src = J.tr_in;
        P.dst = J.tr_out;
    } else {
        P.src = J.in_dev;
        P.dst = both ? J.mid : J.out_dev;
    }
    s->passes.push_back(P);
    s->pending_scan.push_back((int)s->passes.size() - 1);
    J.state = J_ACTIVE;
    return SCPL_OK;
}

// A job that ends without running (or without running further): reported at
// the next poll.
void complete_now(Srv *s, Job &J, int status) {
    J.status = status;
    J.state = J_DONE;
    s->completed.push_back({J.ticket, status});
    if (status == SCPL_ECANCELED) s->st.cancelled++;
    else s->st.failed++;
    if (J.user) J.user->status = status;
}

// Undo a start_job whose allocations were refused: the job is queued again.
void unstart_job(Srv *s, Job &J) {
    for (void *p : J.owned) cudaFreeAsync(p, s->main);   // after its queued copies
    J.owned.clear();
    J.in_dev = nullptr;
    J.out_dev = J.mid = J.tr_in = J.tr_out = nullptr;
    if (J.done) cudaEventDestroy(J.done);
    J.done = nullptr;
    add_reserved(s, -(long long)J.reserved);
    J.reserved = 0;
    J.state = J_QUEUED;
    s->active_jobs--;
}

// Admit queued jobs in arrival order while they fit.
scpl_status admit(Srv *s, bool *any) {
    for (auto &g : s->groups)
        if (g && g->phase == 1) return SCPL_OK;   // a group waits for memory
    if (s->hold) return SCPL_OK;                  // the allocator refused: wait
    while (!s->queue.empty()) {
        const int jid = s->queue.front();
        Job &J = *s->jobs[jid];
        const size_t fp = footprint(s->p, J.spec);
        if (s->reserved + fp > s->budget) {
            if (s->active_jobs > 0) break;   // wait for memory to free up
            if (fp > s->budget) {            // can never fit
                s->queue.pop_front();
                complete_now(s, J, SCPL_ENOMEM);
                *any = true;
                continue;
            }
        }
        s->queue.pop_front();
        J.reserved = fp;
        add_reserved(s, (long long)fp);
        s->active_jobs++;
        scpl_status st = start_job(s, jid);
        if (st == SCPL_ENOMEM && !s->broken) {
            // the allocator refused the job's own buffers: wait for running
            // work to release memory, or fail the job if nothing runs
            unstart_job(s, J);
            if (in_flight(s) || s->active_jobs > 0) {
                s->queue.push_front(jid);
                s->hold = true;
                return SCPL_OK;
            }
            complete_now(s, J, SCPL_ENOMEM);
            *any = true;
            continue;
        }
        if (st != SCPL_OK) return st;
        *any = true;
    }
    return SCPL_OK;
}

// ---- scan waves ---------------------------------------------------------------
scpl_status launch_wave(Srv *s, bool *launched) {
    *launched = false;
    if (s->pending_scan.empty()) return SCPL_OK;
    TraceRange trace("scpl.server.wave");
    std::unique_ptr<Wave> W(new Wave());
    const size_t g0 = s->groups.size();
    // a cooperative launch starts only when all its CTAs fit at once: while
    // groups are carving, a wave takes half the GPU so that it can start
    // beside them instead of waiting for the whole GPU to drain
    bool carving = false;
    for (auto &g : s->groups)
        if (g && g->phase == 2) carving = true;
    const int cap = carving ? std::max(1, s->scan_cap / 2) : s->scan_cap;
    std::vector<int> take, rest;
    for (int pid : s->pending_scan) ((int)take.size() < cap ? take : rest).push_back(pid);
    s->pending_scan = rest;
    W->passes = take;
    // the allocator refused the wave's memory: its passes go back to the
    // queue until running work releases memory, or fail if nothing runs
    auto refused = [&]() -> scpl_status {
        for (size_t g = g0; g < s->groups.size(); ++g)
            if (s->groups[g]->ypool) cudaFreeAsync(s->groups[g]->ypool, s->main);
        s->st.groups -= (long long)(s->groups.size() - g0);
        s->groups.resize(g0);
        for (int pid : take) {
            s->passes[pid].group = -1;
            s->passes[pid].frame_off = 0;
        }
        std::vector<int> back = take;
        back.insert(back.end(), rest.begin(), rest.end());
        s->pending_scan = back;
        if (in_flight(s)) return SCPL_OK;
        for (int pid : take) {
            Job &J = *s->jobs[s->passes[pid].job];
            if (J.status == SCPL_OK) J.status = SCPL_ENOMEM;
        }
        *launched = true;   // the failed jobs are reaped next
        return SCPL_OK;
    };
    const int wid = (int)s->waves.size();

    // groups: passes of one (H, W) in this wave
    std::map<std::pair<int, int>, int> gix;
    for (int pid : take) {
        Pass &P = s->passes[pid];
        auto key = std::make_pair(P.d.H, P.d.W);
        auto it = gix.find(key);
        int g;
        if (it == gix.end()) {
            std::unique_ptr<Group> G(new Group());
            G->H = P.d.H;
            G->W = P.d.W;
            G->ypitch = rup(P.d.W, 16);
            G->stream = s->pool[s->next_stream++ % N_STREAMS];
            G->wave = wid;
            s->groups.push_back(std::move(G));
            g = (int)s->groups.size() - 1;
            gix[key] = g;
            W->groups.push_back(g);
            s->st.groups++;
        } else {
            g = it->second;
        }
        Group &G = *s->groups[g];
        P.group = g;
        P.frame_off = G.T_total;
        G.T_total += P.d.T;
        G.passes.push_back(pid);
    }
    cudaStream_t m = s->main;
    for (int pid : take)
        if (s->passes[pid].ready) SRV_CUDA(s, cudaStreamWaitEvent(m, s->passes[pid].ready, 0));
    for (int g : W->groups) {
        Group &G = *s->groups[g];
        G.ypool_bytes = 2 * (size_t)G.T_total * G.H * G.ypitch;
        size_t e0 = 0;   // summed-energy planes follow the luma and motion maps
        for (int pid : G.passes) {
            Pass &P = s->passes[pid];
            P.e0_off = (long long)(e0 / 4);
            e0 += e0_bytes(P.d);
        }
        G.ypool_bytes += e0;
        void *p = nullptr;
        const cudaError_t ea = dalloc(s, &p, G.ypool_bytes, m);
        if (ea == cudaErrorMemoryAllocation) return refused();
        SRV_CUDA(s, ea);
        G.ypool = static_cast<uint8_t *>(p);
    }

    // CTAs per clip: one each, the rest in proportion to the work
    const int n = (int)take.size();
    std::vector<double> work(n);
    double wsum = 0;
    for (int i = 0; i < n; ++i) {
        const Pass &P = s->passes[take[i]];
        work[i] = (double)P.d.T * scan_tiles(P.d.H, P.d.W);
        wsum += work[i];
    }
    std::vector<int> G(n);
    int total = 0;
    for (int i = 0; i < n; ++i) {
        const Pass &P = s->passes[take[i]];
        int g = 1 + (int)((double)(cap - n) * work[i] / std::max(wsum, 1.0));
        const int tw = scan_tile_warps();
        g = std::min(g, (scan_tiles(P.d.H, P.d.W) + tw - 1) / tw);   // a tile per warp at most
        G[i] = std::max(g, 1);
        total += G[i];
    }

    // per-pass scan state in one slab: status words, then per frame the A_t
    // and maximum accumulators and the arrival counts (all zeroed)
    std::vector<size_t> off(n);
    size_t o = a256((size_t)n * 8);   // [n] err words
    std::vector<size_t> cnt_off(n);
    size_t cnt_bytes = 0;
    for (int i = 0; i < n; ++i) {
        cnt_off[i] = cnt_bytes;   // A [T][SCAN_FW] int64, M [T] int32, count [T] uint32
        cnt_bytes += (size_t)s->passes[take[i]].d.T * (8 * SCAN_FW + 8);
    }
    const size_t zero_bytes = a256(o + cnt_bytes);
    o = zero_bytes;
    for (int i = 0; i < n; ++i) {
        off[i] = o;
        o += scan_state_bytes(s->passes[take[i]].d);
    }
    const size_t tab_off = o;
    o = a256(o + (size_t)n * sizeof(ScanArgs));
    const size_t bc_off = o;
    o = a256(o + (size_t)total * 4);
    void *slab = nullptr;
    const cudaError_t ea = dalloc(s, &slab, o, m);
    if (ea == cudaErrorMemoryAllocation) return refused();
    SRV_CUDA(s, ea);
    W->slab = static_cast<char *>(slab);
    char *base = W->slab;

    // host staging: table, block map, then results [err, nb, starts[T+1]] per pass
    size_t res_ints = 0;
    W->res_pos.resize(n);
    for (int i = 0; i < n; ++i) {
        W->res_pos[i] = res_ints;
        res_ints += 2 + (size_t)s->passes[take[i]].d.T + 1;
    }
    const size_t up_bytes = (size_t)n * sizeof(ScanArgs) + (size_t)total * 4;
    W->res_off = a256(up_bytes);
    SRV_CUDA(s, s->pinned.get(W->res_off + res_ints * 4, W->h));
    ScanArgs *tab = static_cast<ScanArgs *>(W->h.p);
    int *bc = reinterpret_cast<int *>(static_cast<char *>(W->h.p) + (size_t)n * sizeof(ScanArgs));
    int cta = 0;
    for (int i = 0; i < n; ++i) {
        const Pass &P = s->passes[take[i]];
        const Group &Gr = *s->groups[P.group];
        const size_t hw = (size_t)P.d.H * P.d.W;
        char *q = base + off[i];
        ScanArgs a{};
        a.rgb = P.src;
        a.T = P.d.T;
        a.H = P.d.H;
        a.W = P.d.W;
        a.ypitch = Gr.ypitch;
        a.Y = Gr.ypool + (size_t)P.frame_off * P.d.H * Gr.ypitch;
        a.D = Gr.ypool + ((size_t)Gr.T_total + P.frame_off) * P.d.H * Gr.ypitch;
        const size_t spx = (size_t)scan_state_px(P.d.H, P.d.W);
        a.ering = reinterpret_cast<uint16_t *>(q);
        q += a256((size_t)SCAN_FW * spx * 2);
        a.S1 = reinterpret_cast<uint32_t *>(q);
        q += a256(spx * 4);
        a.S2 = reinterpret_cast<uint32_t *>(q);
        q += a256(spx * 4);
        char *acc = base + a256((size_t)n * 8) + cnt_off[i];
        a.partA = reinterpret_cast<long long *>(acc);
        a.partM = reinterpret_cast<int *>(acc + (size_t)P.d.T * 8 * SCAN_FW);
        a.count = reinterpret_cast<unsigned *>(acc + (size_t)P.d.T * (8 * SCAN_FW + 4));
        a.starts = reinterpret_cast<int *>(q);
        q += a256((size_t)(P.d.T + 1) * 4);
        a.n_buffers = reinterpret_cast<int *>(q);
        a.err = reinterpret_cast<int *>(base + (size_t)i * 8);
        a.wg = s->p.wg;
        a.wm = s->p.wm;
        a.alpha = s->p.alpha;
        a.t_max = tmax_of(s->p);
        a.maxval_mode = s->p.maxval_mode;
        a.maxval_theory = emax_of(s->p);
        a.spin_limit_ns = SPIN_NS;
        a.cta0 = cta;
        a.G = G[i];
        a.E0 = reinterpret_cast<int32_t *>(Gr.ypool + 2 * (size_t)Gr.T_total * Gr.H * Gr.ypitch) +
               P.e0_off;
        a.nbcap = e0_planes(P.d);
        a.e0_plane = (long)hw;
        a.A_out = nullptr;
        a.M_out = nullptr;
        tab[i] = a;
        for (int c = 0; c < G[i]; ++c) bc[cta + c] = i;
        cta += G[i];
    }
    SRV_CUDA(s, cudaMemsetAsync(base, 0, zero_bytes, m));
    SRV_CUDA(s, cudaMemcpyAsync(base + tab_off, tab, (size_t)n * sizeof(ScanArgs),
                                cudaMemcpyHostToDevice, m));
    SRV_CUDA(s, cudaMemcpyAsync(base + bc_off, bc, (size_t)total * 4, cudaMemcpyHostToDevice, m));
    SRV_CUDA(s, launch_scan_multi(reinterpret_cast<ScanArgs *>(base + tab_off),
                                  reinterpret_cast<int *>(base + bc_off), total, m));
    count_launches(s, 1);
    int *res = reinterpret_cast<int *>(static_cast<char *>(W->h.p) + W->res_off);
    for (int i = 0; i < n; ++i) {
        const ScanArgs &a = tab[i];
        int *r = res + W->res_pos[i];
        SRV_CUDA(s, cudaMemcpyAsync(r, a.err, 4, cudaMemcpyDeviceToHost, m));
        SRV_CUDA(s, cudaMemcpyAsync(r + 1, a.n_buffers, 4, cudaMemcpyDeviceToHost, m));
        SRV_CUDA(s, cudaMemcpyAsync(r + 2, a.starts, (size_t)(a.T + 1) * 4,
                                    cudaMemcpyDeviceToHost, m));
    }
    SRV_CUDA(s, cudaEventCreateWithFlags(&W->ev, cudaEventDisableTiming));
    SRV_CUDA(s, cudaEventRecord(W->ev, m));
    s->waves.push_back(std::move(W));
    s->st.scan_waves++;
    *launched = true;
    return SCPL_OK;
}

// ---- carving ------------------------------------------------------------------
// Largest power of two <= v, in [1, MAX_CHUNK].
int chunk_len(long v) {
    int q = 1;
    while (q * 2 <= v && q * 2 <= MAX_CHUNK) q *= 2;
    return q;
}

// Launches the group's device-side loop (built once per group) and queues the
// read-back of the item states and the error word behind it.  *used stays
// false (and nothing is launched) for servers and where the loop cannot be
// built; the caller then carves in chunks.
scpl_status launch_loop(Srv *s, Group &G, bool *used) {
    TraceRange trace("scpl.server.chunk");
    *used = false;
    if (!s->device_loop) return SCPL_OK;
    cudaGraphExec_t ge = nullptr;
    auto it = G.graphs.find(0);
    if (it != G.graphs.end()) {
        ge = it->second;
    } else {
        if (build_carve_loop(G.ws, G.nb, 1, nullptr, 0, LOOP_ITERS, G.stream, &ge) !=
            cudaSuccess) {
            cudaGetLastError();
            return SCPL_OK;   // conditional nodes unavailable: chunks
        }
        G.graphs[0] = ge;
        s->st.graphs_built++;
    }
    SRV_CUDA(s, cudaGraphLaunch(ge, G.stream));
    G.looped = true;
    *used = true;
    s->st.chunks++;
    BufState *hst = static_cast<BufState *>(G.hb.p);
    int *herr = reinterpret_cast<int *>(hst + G.nb);
    SRV_CUDA(s, cudaMemcpyAsync(hst, G.ws.st, (size_t)G.nb * sizeof(BufState),
                                cudaMemcpyDeviceToHost, G.stream));
    SRV_CUDA(s, cudaMemcpyAsync(herr, G.ws.err, 4, cudaMemcpyDeviceToHost, G.stream));
    SRV_CUDA(s, cudaEventRecord(G.ev, G.stream));
    return SCPL_OK;
}

scpl_status launch_chunk(Srv *s, Group &G, int q) {
    TraceRange trace("scpl.server.chunk");
    cudaGraphExec_t ge = nullptr;
    auto it = G.graphs.find(q);
    if (it != G.graphs.end()) {
        ge = it->second;
    } else {
        cudaGraph_t graph = nullptr;
        SRV_CUDA(s, cudaStreamBeginCapture(G.stream, cudaStreamCaptureModeRelaxed));
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < q && e == cudaSuccess; ++i) {
            e = G.dpc ? launch_dpc(G.ws, G.nb, 1, nullptr, 0, G.stream)
                      : launch_dp_select(G.ws, G.nb, 1, nullptr, 0, G.stream);
            if (e == cudaSuccess) e = launch_update(G.ws, G.nb, G.stream);
        }
        cudaError_t e2 = cudaStreamEndCapture(G.stream, &graph);
        SRV_CUDA(s, e);
        SRV_CUDA(s, e2);
        e = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        SRV_CUDA(s, e);
        G.graphs[q] = ge;
        s->st.graphs_built++;
    }
    SRV_CUDA(s, cudaGraphLaunch(ge, G.stream));
    count_launches(s, 2LL * q);
    s->st.chunks++;
    BufState *hst = static_cast<BufState *>(G.hb.p);
    int *herr = reinterpret_cast<int *>(hst + G.nb);
    SRV_CUDA(s, cudaMemcpyAsync(hst, G.ws.st, (size_t)G.nb * sizeof(BufState),
                                cudaMemcpyDeviceToHost, G.stream));
    SRV_CUDA(s, cudaMemcpyAsync(herr, G.ws.err, 4, cudaMemcpyDeviceToHost, G.stream));
    SRV_CUDA(s, cudaEventRecord(G.ev, G.stream));
    return SCPL_OK;
}

// Next chunk length from the item states, 0 when every item is done.
int next_chunk(const Group &G) {
    const BufState *hst = static_cast<const BufState *>(G.hb.p);
    long rem_max = 0;
    int kmin = 1 << 30;
    for (int b = 0; b < G.nb; ++b) {
        const int Wc = hst[b].W - hst[b].k_eff;
        const int r = Wc - hst[b].target;
        if (r > 0) {
            rem_max = std::max<long>(rem_max, r);
            const int ke = hst[b].k_eff > 0 ? hst[b].k_eff : std::max(hst[b].k, 1);
            kmin = std::min(kmin, ke);
        }
    }
    if (rem_max == 0) return 0;
    return chunk_len((rem_max + kmin - 1) / kmin);
}

// Items, workspace and the first launches of a group whose scan finished.
scpl_status setup_group(Srv *s, int gid) {
    TraceRange trace("scpl.server.group");
    Group &G = *s->groups[gid];
    std::vector<int> ok;
    for (int pid : G.passes)
        if (s->jobs[s->passes[pid].job]->status == SCPL_OK) ok.push_back(pid);
    int nb = 0, kcap = 1, klog = 1;
    for (int pid : ok) {
        Pass &P = s->passes[pid];
        P.item0 = nb;
        nb += P.nb;
        kcap = std::max(kcap, std::min(P.k, P.d.W - P.d.target));
        klog = std::max(klog, P.d.W - P.d.target);
    }
    G.nb = nb;
    if (nb == 0) return free_group(s, G);   // every pass failed or was cancelled
    CarveWs &ws = G.ws;
    ws = CarveWs{};
    ws.H = G.H;
    ws.W0 = G.W;
    ws.kcap = kcap;
    ws.dpc_r = 32;
    ws.dpc_wpc = 4;
    ws.dpc_v = 4;
    bool use_dpc = true;
    // sizes were tuned when their wave finished
    const bool tuned = tuning_apply(G.H, G.W, ws, &use_dpc);
    ws.wf = s->p.wf;   // forward terms: their planes and the cluster-DP layouts built with them
    if (ws.wf > 0) use_dpc = true;
    G.dpc = use_dpc && dpc_select(G.W, G.H, ws, tuned);
    const size_t ws_bytes = carve_ws_assign(ws, nb, klog, G.dpc, nullptr);
    // frames of every item, the gather table and the frame-minor luma
    long long yfm_total = 0;
    int nframes = 0;
    for (int pid : ok) {
        const Pass &P = s->passes[pid];
        for (int b = 0; b < P.nb; ++b) {
            const int nt = P.starts[b + 1] - P.starts[b];
            yfm_total += (long long)G.H * G.W * rup(nt, 16);
        }
        nframes += P.d.T;
    }
    const size_t err_off = a256(ws_bytes);
    const size_t gt_off = err_off + 256;
    const size_t yfm_off = a256(gt_off + (size_t)nframes * sizeof(GatherFrame));
    const size_t bytes = yfm_off + a256((size_t)std::max<long long>(yfm_total, 16));
    G.gt_off = gt_off;
    G.nframes = nframes;
    // memory: each pass reserved one item; add the others now
    long long extra = 0;
    for (int pid : ok) {
        Pass &P = s->passes[pid];
        const int kc = std::max(1, std::min(P.k, P.d.W - P.d.target));
        const long long add = (long long)(P.nb - 1) * (long long)item_bytes(P.d, kc, s->p.wf);
        extra += add;
    }
    // wait until memory frees up (admission pauses meanwhile), unless this
    // group's jobs are the only ones left
    if (extra > 0 && s->reserved + extra > s->budget && s->active_jobs > (int)ok.size()) {
        G.phase = 1;
        return SCPL_OK;
    }
    void *p = nullptr;
    SRV_CUDA(s, cudaStreamWaitEvent(G.stream, s->waves[G.wave]->ev, 0));
    const cudaError_t ea = dalloc(s, &p, bytes, G.stream);
    if (ea == cudaErrorMemoryAllocation) {
        // refused: wait for running work to release memory, or fail the
        // group's jobs if nothing else runs
        G.phase = 1;
        if (in_flight(s)) return SCPL_OK;
        for (int pid : ok) {
            Job &J = *s->jobs[s->passes[pid].job];
            if (J.status == SCPL_OK) J.status = SCPL_ENOMEM;
        }
        return free_group(s, G);
    }
    SRV_CUDA(s, ea);
    G.phase = 2;
    for (int pid : ok) {
        Pass &P = s->passes[pid];
        const int kc = std::max(1, std::min(P.k, P.d.W - P.d.target));
        const long long add = (long long)(P.nb - 1) * (long long)item_bytes(P.d, kc, s->p.wf);
        s->jobs[P.job]->reserved += add;
        add_reserved(s, add);
        P.item = true;
    }
    G.slab = static_cast<char *>(p);
    G.slab_bytes = bytes;
    carve_ws_assign(ws, nb, klog, G.dpc, G.slab);
    if (G.dpc && !ws.J) G.dpc = false;
    ws.err = reinterpret_cast<int *>(G.slab + err_off);
    ws.Y = G.ypool;
    ws.D = G.ypool + (size_t)G.T_total * G.H * G.ypitch;
    ws.ypitch = G.ypitch;
    ws.wg = s->p.wg;
    ws.wm = s->p.wm;
    ws.Yfm = reinterpret_cast<uint8_t *>(G.slab + yfm_off);
    ws.E0 = reinterpret_cast<const int32_t *>(G.ypool + 2 * (size_t)G.T_total * G.H * G.ypitch);
    // share of the group's memory per pass (by frames)
    for (int pid : ok) {
        Pass &P = s->passes[pid];
        P.group_share = (size_t)((double)(bytes + G.ypool_bytes) * P.d.T / std::max(nframes, 1));
    }

    // host staging: states (also the readback area), err word, gather table
    const size_t st_bytes = (size_t)nb * sizeof(BufState);
    SRV_CUDA(s, s->pinned.get(st_bytes + 256 + (size_t)nframes * sizeof(GatherFrame), G.hb));
    BufState *hst = static_cast<BufState *>(G.hb.p);
    GatherFrame *hgt =
        reinterpret_cast<GatherFrame *>(static_cast<char *>(G.hb.p) + st_bytes + 256);
    long long yfm = 0;
    int f = 0;
    for (int pid : ok) {
        const Pass &P = s->passes[pid];
        const int tgt = P.d.target;
        for (int b = 0; b < P.nb; ++b) {
            const int t0 = P.starts[b], nt = P.starts[b + 1] - t0;
            const int tp = (int)rup(nt, 16);
            const long long e0 =
                b < e0_planes(P.d) ? P.e0_off + (long long)b * G.H * G.W : -1;
            hst[P.item0 + b] =
                BufState{P.frame_off + t0, nt, G.W, 0, 0, 0, tgt, 0, tp, P.k, yfm, e0};
            yfm += (long long)G.H * G.W * tp;
            for (int t = t0; t < t0 + nt; ++t) {
                GatherFrame gf;
                gf.src = P.src + (size_t)t * G.H * G.W * 3;
                gf.dst = P.dst + (size_t)t * G.H * tgt * 3;
                gf.b = P.item0 + b;
                gf.target = tgt;
                hgt[f++] = gf;
            }
        }
    }
    cudaStream_t gs = G.stream;
    SRV_CUDA(s, cudaMemcpyAsync(ws.st, hst, st_bytes, cudaMemcpyHostToDevice, gs));
    SRV_CUDA(s, cudaMemcpyAsync(G.slab + gt_off, hgt, (size_t)nframes * sizeof(GatherFrame),
                                cudaMemcpyHostToDevice, gs));
    SRV_CUDA(s, cudaMemsetAsync(ws.err, 0, 4, gs));
    SRV_CUDA(s, cudaMemsetAsync(ws.dirty_count, 0, (size_t)nb * 8, gs));
    SRV_CUDA(s, launch_energy_init(ws, nb, gs));
    count_launches(s, 1);
    SRV_CUDA(s, cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming));
    // the first chunk from the largest removal and the largest k
    long rem_max = 0;
    int kmax = 1;
    for (int pid : ok) {
        const Pass &P = s->passes[pid];
        rem_max = std::max<long>(rem_max, P.d.W - P.d.target);
        kmax = std::max(kmax, std::min(P.k, P.d.W - P.d.target));
    }
    bool looped = false;
    scpl_status st = launch_loop(s, G, &looped);
    if (st != SCPL_OK || looped) return st;
    return launch_chunk(s, G, chunk_len((rem_max + kmax - 1) / kmax));
}

// Every item of the group reached its target: gather, then finish its passes.
scpl_status pass_done(Srv *s, int pid, cudaStream_t gs) {
    Pass P = s->passes[pid];   // a copy: s->passes may grow below
    Job &J = *s->jobs[P.job];
    const scpl_job &j = J.spec;
    if (J.status != SCPL_OK) {
        // failed or cancelled while the group carved: it ends after the
        // group's launches that read or write its frames
        if (J.state == J_ACTIVE && J.done) {
            SRV_CUDA(s, cudaEventRecord(J.done, gs));
            J.state = J_FINISHING;
        }
        return SCPL_OK;
    }
    if (P.index == 0 && J.npass == 2) {
        // the height pass works on the transposed output of the width pass
        SRV_CUDA(s, launch_transpose_rgb(J.mid, j.T, j.H, j.target_W, J.tr_in, gs));
        count_launches(s, 1);
        Pass N;
        N.job = P.job;
        N.index = 1;
        N.transposed = true;
        N.src = J.tr_in;
        N.dst = J.tr_out;
        N.d = PassDims{j.T, j.target_W, j.H, j.target_H};
        N.k = j.k;
        SRV_CUDA(s, cudaEventCreateWithFlags(&N.ready, cudaEventDisableTiming));
        SRV_CUDA(s, cudaEventRecord(N.ready, gs));
        s->passes.push_back(N);
        s->pending_scan.push_back((int)s->passes.size() - 1);
        return SCPL_OK;
    }
    if (P.transposed) {
        SRV_CUDA(s, launch_transpose_rgb(J.tr_out, j.T, j.target_W, j.target_H, J.out_dev, gs));
        count_launches(s, 1);
    }
    if (j.on_host)
        SRV_CUDA(s, link_copy(j.out, J.out_dev, rgb_bytes(j.T, j.target_H, j.target_W), gs));
    SRV_CUDA(s, cudaEventRecord(J.done, gs));
    J.state = J_FINISHING;
    return SCPL_OK;
}

scpl_status free_group(Srv *s, Group &G) {
    cudaStream_t gs = G.stream;
    if (G.slab) SRV_CUDA(s, cudaFreeAsync(G.slab, gs));
    if (G.ypool) SRV_CUDA(s, cudaFreeAsync(G.ypool, gs));
    G.slab = nullptr;
    G.ypool = nullptr;
    for (auto &kv : G.graphs) cudaGraphExecDestroy(kv.second);
    G.graphs.clear();
    s->pinned.put(G.hb);
    G.hb = Pinned{};
    add_reserved(s, -(long long)G.held_after);
    G.held_after = 0;
    G.phase = 3;
    s->hold = false;
    return SCPL_OK;
}

scpl_status finish_group(Srv *s, int gid) {
    TraceRange trace("scpl.server.finish");
    Group &G = *s->groups[gid];
    cudaStream_t gs = G.stream;
    if (G.nframes > 0) {
        SRV_CUDA(s, launch_gather_frames(G.ws, reinterpret_cast<GatherFrame *>(G.slab + G.gt_off),
                                         G.nframes, gs));
        count_launches(s, (G.nframes + 65534) / 65535);
    }
    const std::vector<int> mine = G.passes;
    for (int pid : mine) {
        scpl_status st = pass_done(s, pid, gs);
        if (st != SCPL_OK) return st;
    }
    // completed jobs hand their share of this group's memory to the group
    return free_group(s, G);
}

// A device-side status word of a group is set: every job in it fails.
void fail_group_jobs(Srv *s, Group &G, int dev_err) {
    const int code = dev_err == DEV_ETIMEOUT ? SCPL_ETIMEOUT : SCPL_ECUDA;
    for (int pid : G.passes) {
        Job &J = *s->jobs[s->passes[pid].job];
        if (J.status == SCPL_OK) J.status = code;
    }
}

// Jobs that failed or whose last work finished: release and report them.
scpl_status reap_jobs(Srv *s, bool *any) {
    for (size_t jid = 0; jid < s->jobs.size(); ++jid) {
        Job &J = *s->jobs[jid];
        if (J.state != J_ACTIVE && J.state != J_FINISHING) continue;
        bool finished = false;
        if (J.state == J_FINISHING) {
            cudaError_t e = cudaEventQuery(J.done);
            if (e == cudaErrorNotReady) continue;
            SRV_CUDA(s, e);
            finished = true;
        } else if (J.status != SCPL_OK) {
            // failed or cancelled: done once no scan wave still reads its
            // frames and no carving group still has its buffers as items (a
            // group that finishes records J.done after its last launch)
            bool busy = false;
            for (const Pass &P : s->passes) {
                if (P.job != (int)jid || P.group < 0) continue;
                const Group &G = *s->groups[P.group];
                if (!s->waves[G.wave]->done || (P.item && G.phase == 2)) busy = true;
            }
            if (busy) continue;
            std::vector<int> keep;   // a pass still queued for a scan is dropped
            for (int q : s->pending_scan)
                if (s->passes[q].job != (int)jid) keep.push_back(q);
            s->pending_scan = keep;
            finished = true;
        }
        if (!finished) continue;
        // release: own memory now; group memory stays with the group until it ends
        for (void *p : J.owned) SRV_CUDA(s, cudaFreeAsync(p, s->main));
        J.owned.clear();
        size_t in_groups = 0;
        for (const Pass &P : s->passes) {
            if (P.job != (int)jid || P.group < 0) continue;
            Group &G = *s->groups[P.group];
            if (G.phase != 3) {
                G.held_after += P.group_share;
                in_groups += P.group_share;
            }
        }
        const size_t release = J.reserved > in_groups ? J.reserved - in_groups : 0;
        add_reserved(s, -(long long)release);
        J.reserved = 0;
        if (J.done) cudaEventDestroy(J.done);
        J.done = nullptr;
        J.state = J_DONE;
        s->active_jobs--;
        s->completed.push_back({J.ticket, J.status});
        if (J.status == SCPL_OK) s->st.completed++;
        else if (J.status == SCPL_ECANCELED) s->st.cancelled++;
        else s->st.failed++;
        s->hold = false;   // memory was released
        if (J.user) {
            J.user->status = J.status;
            J.user->n_buffers = J.spec.n_buffers;
        }
        *any = true;
    }
    return SCPL_OK;
}

void compact(Srv *s);

// One scheduling round.  *any = something was launched or completed.
scpl_status round(Srv *s, bool *any) {
    scpl_status st;
    // scan waves that finished: items of their groups
    for (size_t wid = 0; wid < s->waves.size(); ++wid) {
        Wave &W = *s->waves[wid];
        if (W.done) continue;
        cudaError_t e = cudaEventQuery(W.ev);
        if (e == cudaErrorNotReady) continue;
        SRV_CUDA(s, e);
        W.done = true;
        *any = true;
        const int *res = reinterpret_cast<const int *>(static_cast<char *>(W.h.p) + W.res_off);
        for (size_t i = 0; i < W.passes.size(); ++i) {
            Pass &P = s->passes[W.passes[i]];
            Job &J = *s->jobs[P.job];
            const int *r = res + W.res_pos[i];
            const int nb = r[1];
            if (r[0] != DEV_OK || nb < 1 || nb > P.d.T) {
                if (J.status == SCPL_OK) J.status = r[0] == DEV_ETIMEOUT ? SCPL_ETIMEOUT : SCPL_ECUDA;
                P.nb = 0;
                continue;
            }
            P.nb = nb;
            P.starts.assign(r + 2, r + 2 + nb + 1);
            if (P.index == 0) {
                J.spec.n_buffers = nb;
                if (J.spec.buffer_starts)
                    std::copy(P.starts.begin(), P.starts.end(), J.spec.buffer_starts);
            }
        }
        SRV_CUDA(s, cudaFreeAsync(W.slab, s->main));
        W.slab = nullptr;
        s->pinned.put(W.h);
        W.h = Pinned{};
        // new sizes are tuned before this wave's groups start carving, so that
        // the measurements see only what was already running
        if (s->autotune)
            for (int g : W.groups) {
                const Group &G = *s->groups[g];
                if (tuning_lookup(G.H, G.W, nullptr)) continue;
                int kcap = 1;
                for (int pid : G.passes)
                    kcap = std::max(kcap, std::min(s->passes[pid].k,
                                                   s->passes[pid].d.W - s->passes[pid].d.target));
                tune_class(G.H, G.W, kcap, s->main, nullptr);   // on failure: the defaults
            }
        for (int g : W.groups)
            if ((st = setup_group(s, g)) != SCPL_OK) return st;
    }
    // groups waiting for memory
    for (size_t g = 0; g < s->groups.size(); ++g)
        if (s->groups[g]->phase == 1) {
            if ((st = setup_group(s, (int)g)) != SCPL_OK) return st;
            if (s->groups[g]->phase == 2) *any = true;
        }
    // carving chunks that finished
    for (size_t g = 0; g < s->groups.size(); ++g) {
        Group &G = *s->groups[g];
        if (G.phase != 2) continue;
        cudaError_t e = cudaEventQuery(G.ev);
        if (e == cudaErrorNotReady) continue;
        SRV_CUDA(s, e);
        *any = true;
        const int *herr =
            reinterpret_cast<const int *>(static_cast<BufState *>(G.hb.p) + G.nb);
        if (*herr != DEV_OK) {
            fail_group_jobs(s, G, *herr);
            if ((st = free_group(s, G)) != SCPL_OK) return st;
            continue;
        }
        const int q = next_chunk(G);
        if (q > 0) {
            if ((st = launch_chunk(s, G, q)) != SCPL_OK) return st;
        } else {
            if (G.looped) {
                // the loop ran bodies of LOOP_ITERS DP + update launches and
                // one condition kernel each, up to the longest item's
                // iterations (the items' selecting DP launches)
                const BufState *hst = static_cast<const BufState *>(G.hb.p);
                int it = 0;
                for (int b = 0; b < G.nb; ++b) it = std::max(it, hst[b].iters);
                const long long bodies = std::max(1, (it + LOOP_ITERS - 1) / LOOP_ITERS);
                count_launches(s, bodies * (2LL * LOOP_ITERS + 1));
                G.looped = false;
            }
            if ((st = finish_group(s, (int)g)) != SCPL_OK) return st;
        }
    }
    if ((st = reap_jobs(s, any)) != SCPL_OK) return st;
    if ((st = admit(s, any)) != SCPL_OK) return st;
    if (!s->pending_scan.empty()) {
        bool launched = false;
        if ((st = launch_wave(s, &launched)) != SCPL_OK) return st;
        if (launched) *any = true;
    }
    compact(s);
    return SCPL_OK;
}

// Blocks until some work in flight finishes (or returns at once if none).
scpl_status wait_some(Srv *s) {
    for (auto &W : s->waves)
        if (!W->done) {
            SRV_CUDA(s, cudaEventSynchronize(W->ev));
            return SCPL_OK;
        }
    for (auto &G : s->groups)
        if (G->phase == 2) {
            SRV_CUDA(s, cudaEventSynchronize(G->ev));
            return SCPL_OK;
        }
    for (auto &J : s->jobs)
        if (J->state == J_FINISHING) {
            SRV_CUDA(s, cudaEventSynchronize(J->done));
            return SCPL_OK;
        }
    return SCPL_OK;
}

int count_queued(Srv *s) { return (int)s->queue.size(); }

// With nothing queued, active or in flight, the records of finished jobs are
// dropped so that a long-running server does not grow (tickets stay unique).
void compact(Srv *s) {
    if (s->active_jobs != 0 || !s->queue.empty() || !s->pending_scan.empty()) return;
    for (auto &G : s->groups)
        if (G->phase != 3) return;
    for (auto &W : s->waves)
        if (!W->done) return;
    for (auto &G : s->groups)
        if (G->ev) cudaEventDestroy(G->ev);
    for (auto &W : s->waves)
        if (W->ev) cudaEventDestroy(W->ev);
    for (auto &P : s->passes)
        if (P.ready) cudaEventDestroy(P.ready);
    s->groups.clear();
    s->waves.clear();
    s->passes.clear();
    s->jobs.clear();
}

scpl_status create(const scpl_params *p, size_t budget, void *stream, Srv **out) {
    scpl_params def;
    scpl_default_params(&def);
    if (!p) p = &def;
    if (!(p->alpha >= 0.0) || p->alpha > 1e6 || p->wg < 0 || p->wm < 0 || p->wg + p->wm == 0 ||
        p->t_max < 1 || p->t_max > 1024 || (p->maxval_mode != 0 && p->maxval_mode != 1) ||
        !forward_params_ok(*p))
        return SCPL_EINVAL;
    std::unique_ptr<Srv> s(new Srv());
    s->p = *p;
    s->user = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&s->device) != cudaSuccess) return SCPL_ECUDA;
    if (cudaStreamCreateWithFlags(&s->main, cudaStreamNonBlocking) != cudaSuccess)
        return SCPL_ECUDA;
    for (int i = 0; i < N_STREAMS; ++i)
        if (cudaStreamCreateWithFlags(&s->pool[i], cudaStreamNonBlocking) != cudaSuccess)
            return SCPL_ECUDA;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->mpool, &props) != cudaSuccess) return SCPL_ECUDA;
    uint64_t keep = ~0ull;   // keep freed memory in the pool for reuse
    if (cudaMemPoolSetAttribute(s->mpool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
        return SCPL_ECUDA;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return SCPL_ECUDA;
    s->budget = budget ? budget : (size_t)(0.9 * (double)free_b);
    int err = 0;
    s->scan_cap = scan_capacity(&err);
    if (err || s->scan_cap < 1) return SCPL_ECUDA;
    *out = s.release();
    return SCPL_OK;
}

void destroy(Srv *s) {
    if (!s) return;
    if (s->main) cudaStreamSynchronize(s->main);
    for (int i = 0; i < N_STREAMS; ++i)
        if (s->pool[i]) cudaStreamSynchronize(s->pool[i]);
    for (auto &G : s->groups) {
        if (G->phase != 3) free_group(s, *G);
        if (G->ev) cudaEventDestroy(G->ev);
    }
    for (auto &W : s->waves) {
        if (W->slab) cudaFreeAsync(W->slab, s->main);
        if (W->ev) cudaEventDestroy(W->ev);
    }
    for (auto &J : s->jobs) {
        for (void *p : J->owned) cudaFreeAsync(p, s->main);
        if (J->done) cudaEventDestroy(J->done);
    }
    for (auto &P : s->passes)
        if (P.ready) cudaEventDestroy(P.ready);
    if (s->main) cudaStreamSynchronize(s->main);
    for (int i = 0; i < N_STREAMS; ++i)
        if (s->pool[i]) {
            cudaStreamSynchronize(s->pool[i]);
            cudaStreamDestroy(s->pool[i]);
        }
    if (s->mpool) cudaMemPoolDestroy(s->mpool);
    if (s->main) cudaStreamDestroy(s->main);
    delete s;
}

scpl_status submit(Srv *s, const scpl_job *job, scpl_job *user, long long *ticket) {
    if (!job) return sfail(s, SCPL_EINVAL, "job is NULL");
    std::unique_ptr<Job> J(new Job());
    J->spec = *job;
    J->spec.status = SCPL_OK;
    J->spec.n_buffers = 0;
    J->user = user;
    J->ticket = s->next_ticket++;
    if (ticket) *ticket = J->ticket;
    s->st.submitted++;
    const scpl_status v = check_job(s->p, J->spec);
    if (v != SCPL_OK) {   // fails alone, reported at the next poll
        complete_now(s, *J, v);
        s->jobs.push_back(std::move(J));
        return SCPL_OK;
    }
    {
        // the job's work starts after what the caller queued before on its
        // stream (the legacy default stream too: the engine's streams do not
        // synchronise with it implicitly)
        cudaEvent_t e;
        SRV_CUDA(s, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        SRV_CUDA(s, cudaEventRecord(e, s->user));
        SRV_CUDA(s, cudaStreamWaitEvent(s->main, e, 0));
        cudaEventDestroy(e);
    }
    s->queue.push_back((int)s->jobs.size());
    s->jobs.push_back(std::move(J));
    return SCPL_OK;
}

scpl_status progress(Srv *s, int wait) {
    if (s->broken) return sfail(s, SCPL_ECUDA, "the server hit a CUDA error earlier: %s",
                                s->err.c_str());
    bool any = false;
    scpl_status st = round(s, &any);
    if (st != SCPL_OK) return st;
    if (!any && wait) {
        if ((st = wait_some(s)) != SCPL_OK) return st;
        st = round(s, &any);
    }
    return st;
}

bool idle(Srv *s) { return s->active_jobs == 0 && s->queue.empty(); }

// Cancel a job: a queued job ends at once; an admitted one stops taking new
// stages and ends when the launches already made for it have finished.
scpl_status cancel(Srv *s, long long ticket) {
    for (size_t jid = 0; jid < s->jobs.size(); ++jid) {
        Job &J = *s->jobs[jid];
        if (J.ticket != ticket) continue;
        if (J.state == J_QUEUED) {
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
                if (*it == (int)jid) {
                    s->queue.erase(it);
                    break;
                }
            complete_now(s, J, SCPL_ECANCELED);
            return SCPL_OK;
        }
        if (J.state == J_ACTIVE && J.status == SCPL_OK) {
            J.status = SCPL_ECANCELED;
            return SCPL_OK;
        }
        return sfail(s, SCPL_EINVAL, "job %lld has already finished or failed", ticket);
    }
    return sfail(s, SCPL_EINVAL, "no job with ticket %lld", ticket);
}

bool in_flight(Srv *s) {
    for (auto &W : s->waves)
        if (!W->done) return true;
    for (auto &G : s->groups)
        if (G->phase == 2) return true;
    for (auto &J : s->jobs)
        if (J->state == J_FINISHING) return true;
    return false;
}

scpl_status drain(Srv *s) {
    int stalled = 0;
    while (!idle(s)) {
        const long long before = s->st.completed + s->st.failed + s->st.chunks + s->st.scan_waves;
        scpl_status st = progress(s, 1);
        if (st != SCPL_OK) return st;
        const long long after = s->st.completed + s->st.failed + s->st.chunks + s->st.scan_waves;
        stalled = (after == before && !in_flight(s)) ? stalled + 1 : 0;
        if (stalled > 1000)
            return sfail(s, SCPL_ECUDA, "engine stalled with %d active and %d queued jobs",
                         s->active_jobs, (int)s->queue.size());
    }
    return SCPL_OK;
}

}  // namespace

extern "C" scpl_status scpl_server_get_stats(scpl_server s, scpl_server_stats *out);

namespace scpl {

// scpl_carve_batch: the handle's engine (created on first use and kept, with
// its memory pool, until the handle is destroyed), every job submitted at once.
scpl_status engine_run_batch(scpl_server_s **eng, const scpl_params &p, cudaStream_t stream,
                             bool autotune, scpl_job *jobs, int n_jobs, std::string &err) {
    scpl_status st = SCPL_OK;
    if (!*eng) {
        st = create(&p, 0, stream, eng);
        if (st != SCPL_OK) {
            err = "could not create the batch engine";
            return st;
        }
    }
    Srv *s = *eng;
    s->user = stream;
    s->autotune = autotune;
    s->device_loop = true;
    if (s->broken) {
        err = "the batch engine hit a CUDA error earlier: " + s->err;
        return SCPL_ECUDA;
    }
    for (int i = 0; i < n_jobs && st == SCPL_OK; ++i) st = submit(s, &jobs[i], &jobs[i], nullptr);
    if (st == SCPL_OK) st = drain(s);
    s->completed.clear();
    if (st != SCPL_OK) {
        err = s->err;
        return st;
    }
    for (int i = 0; i < n_jobs; ++i)
        if (jobs[i].status != SCPL_OK) {
            err = "job " + std::to_string(i) + " failed";
            return (scpl_status)jobs[i].status;
        }
    return SCPL_OK;
}

void engine_destroy(scpl_server_s *eng) { destroy(eng); }

scpl_status engine_stats(scpl_server_s *eng, scpl_server_stats *out) {
    if (!eng) {
        std::memset(out, 0, sizeof *out);
        return SCPL_OK;
    }
    return scpl_server_get_stats(eng, out);
}

}  // namespace scpl

extern "C" {

size_t scpl_job_footprint(const scpl_params *p, const scpl_job *job) {
    scpl_params def;
    scpl_default_params(&def);
    if (!job) return 0;
    return footprint(p ? *p : def, *job);
}

size_t scpl_job_footprint_per_buffer(const scpl_job *job) {
    if (!job) return 0;
    PassDims d[2];
    const int n = job_passes(*job, d);
    size_t b = 0;
    for (int i = 0; i < n; ++i)
        b = std::max(b, item_bytes(d[i], std::max(1, std::min(job->k, d[i].W - d[i].target)), 0));
    return b;
}

scpl_status scpl_server_create(const scpl_params *p, size_t hbm_budget, void *stream,
                               scpl_server *out) {
    if (!out) return SCPL_EINVAL;
    *out = nullptr;
    return create(p, hbm_budget, stream, out);
}

scpl_status scpl_server_submit(scpl_server s, const scpl_job *job, long long *ticket) {
    if (!s) return SCPL_EINVAL;
    return submit(s, job, nullptr, ticket);
}

scpl_status scpl_server_set_autotune(scpl_server s, int on) {
    if (!s) return SCPL_EINVAL;
    s->autotune = on != 0;
    return SCPL_OK;
}

scpl_status scpl_server_progress(scpl_server s, int wait, int *n_active, int *n_queued) {
    if (!s) return SCPL_EINVAL;
    scpl_status st = progress(s, wait);
    if (n_active) *n_active = s->active_jobs;
    if (n_queued) *n_queued = count_queued(s);
    return st;
}

int scpl_server_poll(scpl_server s, long long *tickets, int *statuses, int max) {
    if (!s || max <= 0) return 0;
    const int n = std::min<int>(max, (int)s->completed.size());
    for (int i = 0; i < n; ++i) {
        if (tickets) tickets[i] = s->completed[i].first;
        if (statuses) statuses[i] = s->completed[i].second;
    }
    s->completed.erase(s->completed.begin(), s->completed.begin() + n);
    return n;
}

scpl_status scpl_server_drain(scpl_server s) {
    if (!s) return SCPL_EINVAL;
    return drain(s);
}

scpl_status scpl_server_cancel(scpl_server s, long long ticket) {
    if (!s) return SCPL_EINVAL;
    return cancel(s, ticket);
}

scpl_status scpl_server_refuse_allocations(scpl_server s, long long skip, int count) {
    if (!s || skip < 0 || count < 0) return SCPL_EINVAL;
    s->refuse_skip = skip;
    s->refuse_n = count;
    return SCPL_OK;
}

scpl_status scpl_server_get_stats(scpl_server s, scpl_server_stats *out) {
    if (!s || !out) return SCPL_EINVAL;
    *out = s->st;
    out->queued = count_queued(s);
    out->active = s->active_jobs;
    out->reserved_bytes = s->reserved;
    out->peak_reserved_bytes = s->peak;
    out->budget_bytes = s->budget;
    return SCPL_OK;
}

const char *scpl_server_last_error(scpl_server s) { return s ? s->err.c_str() : "null server"; }

void scpl_server_destroy(scpl_server s) { destroy(s); }

}  // extern "C"
