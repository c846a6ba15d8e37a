// Autotuning of the carving kernels per frame size (H, W).
//
// Every candidate is timed on a scratch workspace of four buffers carved in
// one launch, the regime of a clip's first iterations and of batches: a
// choice that wins on one buffer alone can lose once several run at once.
//
// The choices are the cluster DP's layout (halo depth R, warps per CTA and
// columns per lane: R32 x 4 warps, R16 x 4, R32 x 8, R16 x 8 with 4 columns a
// lane; R16 x 4 and R16 x 8 with 2), the single-CTA DP, and the rows per
// k_update CTA (1, 2 or 4).  The scratch buffers hold synthetic energy and
// luma of that size; each candidate is timed with CUDA events, and the
// fastest is recorded in a process-wide table.  Every choice computes the
// same result (the DP and the update are exact), so only the time differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "scpl.h"
#include "scpl_internal.cuh"

namespace scpl {

namespace {

std::mutex g_mu;
std::map<std::pair<int, int>, scpl_tuning> g_table;

// Synthetic energy (a smooth ramp plus hashed texture, like a natural frame's
// gradient) and luma for the scratch workspace.
__global__ void k_tune_fill(int32_t *E, long pitch, int H, int W, uint8_t *yfm, long yfm_bytes) {
    const long n = (long)H * W;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q / W), j = (int)(q - (long)i * W);
        uint32_t h = (uint32_t)q * 2654435761u;
        h ^= h >> 15;
        E[(long)i * pitch + j] = (int32_t)(((i + j) & 63) * 8 + (h & 511));
    }
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < yfm_bytes;
         q += (long)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)q * 2246822519u;
        h ^= h >> 13;
        yfm[q] = (uint8_t)h;
    }
}

__global__ void k_tune_identity(uint16_t *O, long pitch, int H, int W) {
    const long n = (long)H * W;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q / W), j = (int)(q - (long)i * W);
        O[(long)i * pitch + j] = (uint16_t)j;
    }
}

struct Scratch {
    void *slab = nullptr, *yfm = nullptr, *err = nullptr;
    ~Scratch() {
        if (slab) cudaFree(slab);
        if (yfm) cudaFree(yfm);
        if (err) cudaFree(err);
    }
};

}  // namespace

bool tuning_lookup(int H, int W, scpl_tuning *out) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(std::make_pair(H, W));
    if (it == g_table.end()) return false;
    if (out) *out = it->second;
    return true;
}

void tuning_store(const scpl_tuning &t) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[std::make_pair(t.H, t.W)] = t;
}

void tuning_clear() {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table.clear();
}

int tuning_list(scpl_tuning *out, int max) {
    std::lock_guard<std::mutex> lock(g_mu);
    int i = 0;
    for (const auto &kv : g_table) {   // std::map: ordered by (H, W)
        if (out && i < max) out[i] = kv.second;
        ++i;
    }
    return i;
}

// Apply the recorded choice for (H, W), if any, to a workspace about to be
// laid out: the cluster-DP layout (or the single-CTA DP) and the update rows.
bool tuning_apply(int H, int W, CarveWs &ws, bool *use_dpc) {
    scpl_tuning t;
    if (!tuning_lookup(H, W, &t)) return false;
    if (t.dpc_halo == 0) {
        *use_dpc = false;
    } else {
        ws.dpc_r = t.dpc_halo;
        ws.dpc_wpc = t.dpc_warps;
        ws.dpc_v = t.dpc_lane_cols;
    }
    ws.up_rows = t.update_rows;
    return true;
}

scpl_status tune_class(int H, int W, int k, cudaStream_t s, scpl_tuning *out) {
    if (H < 1 || W < 4 || k < 1) return SCPL_EINVAL;
    TraceRange trace("scpl.tune");
    const int remove = std::min(W - 2, 4 * k);
    const int kcap = std::max(1, std::min(k, remove));
    scpl_tuning t{};
    t.H = H;
    t.W = W;
    t.dpc_halo = 32;
    t.dpc_warps = 4;
    t.dpc_lane_cols = 4;
    t.update_rows = 0;
    const int tp = 16;   // frames of each scratch buffer
    constexpr int NBT = 4;   // scratch buffers
    CarveWs ws{};
    ws.H = H;
    ws.W0 = W;
    ws.kcap = kcap;
    ws.dpc_r = 32;
    ws.dpc_wpc = 4;
    ws.dpc_v = 4;
    Scratch sc;
    // one slab big enough for the layout of every candidate (E, SD and O come
    // first and sit at the same offsets in all of them)
    size_t bytes = 0;
    for (int R : {16, 32, 0})
        for (int wpc : {4, 8})
            for (int v : {4, 2}) {
                CarveWs c = ws;
                c.dpc_r = R;
                c.dpc_wpc = wpc;
                c.dpc_v = v;
                bytes = std::max(bytes, carve_ws_assign(c, NBT, remove, R != 0, nullptr));
            }
    if (cudaMalloc(&sc.slab, bytes) != cudaSuccess) return SCPL_ENOMEM;
    const long yfm_bytes = (long)H * W * tp * NBT;
    if (cudaMalloc(&sc.yfm, (size_t)yfm_bytes) != cudaSuccess) return SCPL_ENOMEM;
    if (cudaMalloc(&sc.err, 256) != cudaSuccess) return SCPL_ENOMEM;
    carve_ws_assign(ws, NBT, remove, true, static_cast<char *>(sc.slab));
    ws.Yfm = static_cast<uint8_t *>(sc.yfm);
    ws.err = static_cast<int *>(sc.err);
    ws.wg = 1;
    ws.wm = 2;
    ws.E0 = nullptr;
    ws.Y = nullptr;
    ws.D = nullptr;
    BufState st0[NBT];
    for (int b = 0; b < NBT; ++b)
        st0[b] = BufState{0, tp, W, 0, 0, 0, W - remove, 0, tp, k, (long long)b * H * W * tp, -1};
    if (cudaMemsetAsync(sc.err, 0, 256, s) != cudaSuccess) return SCPL_ECUDA;
    if (cudaMemsetAsync(ws.SD, 0, (size_t)NBT * ws.plane * 4, s) != cudaSuccess) return SCPL_ECUDA;
    for (int b = 0; b < NBT; ++b) {   // slot 0 of every buffer; the luma copy once
        k_tune_fill<<<304, 256, 0, s>>>(ws.E + (long)b * 2 * ws.plane, ws.pitch, H, W, ws.Yfm,
                                        b == 0 ? yfm_bytes : 0);
        k_tune_identity<<<304, 256, 0, s>>>(ws.O + (long)b * 2 * ws.plane, ws.pitch, H, W);
    }
    if (cudaGetLastError() != cudaSuccess) return SCPL_ECUDA;

    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return SCPL_ECUDA;
    }
    auto reset = [&]() {
        return cudaMemcpyAsync(ws.st, st0, sizeof st0, cudaMemcpyHostToDevice, s);
    };
    const int reps = 3;
    // time one DP candidate (the state is reset before every run)
    // kind 16, 32: cluster halo; 0: one CTA
    auto time_dp = [&](int kind, int wpc, int lane_cols) -> float {
        CarveWs v = ws;
        v.dpc_r = kind;
        v.dpc_wpc = wpc;
        v.dpc_v = lane_cols;
        if (kind != 0 && !dpc_available(W, H, kind, wpc, lane_cols)) return -1.0f;
        carve_ws_assign(v, NBT, remove, kind != 0, static_cast<char *>(sc.slab));
        if (kind != 0 && (v.dpc_r != kind || v.dpc_wpc != wpc || v.dpc_v != lane_cols))
            return -1.0f;
        if (kind == 0) {
            int bb = 0;
            if (dp_smem_bytes(W, H, &bb) > 227 * 1024 - 4096) return -1.0f;
        }
        float best = 1e30f;
        for (int r = 0; r <= reps; ++r) {
            if (reset() != cudaSuccess) return -1.0f;
            cudaEventRecord(a, s);
            cudaError_t e = kind ? launch_dpc(v, NBT, k, nullptr, 0, s)
                                 : launch_dp_select(v, NBT, k, nullptr, 0, s);
            cudaEventRecord(b, s);
            if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
                cudaGetLastError();
                return -1.0f;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            if (r > 0) best = std::min(best, ms);   // the first run warms up
        }
        return best * 1000.0f;
    };
    constexpr int NC = 7;
    const int kinds[NC] = {32, 16, 32, 16, 0, 16, 16}, warps[NC] = {4, 4, 8, 8, 4, 4, 8};
    const int cols[NC] = {4, 4, 4, 4, 4, 2, 2};
    for (int i = 0; i < NC; ++i) t.dp_us[i] = time_dp(kinds[i], warps[i], cols[i]);
    // the fastest DP; then leave one pending iteration for the update timing
    float best = 1e30f;
    for (int i = 0; i < NC; ++i)
        if (t.dp_us[i] > 0.0f && t.dp_us[i] < best) {
            best = t.dp_us[i];
            t.dpc_halo = kinds[i];
            t.dpc_warps = warps[i];
            t.dpc_lane_cols = cols[i];
        }
    scpl_status result = SCPL_OK;
    if (best >= 1e29f) {
        result = SCPL_ECUDA;
    } else {
        CarveWs v = ws;   // any exact DP leaves the same pending iteration
        v.dpc_r = t.dp_us[0] > 0 ? 32 : 0;
        v.dpc_wpc = 4;
        v.dpc_v = 4;
        carve_ws_assign(v, NBT, remove, v.dpc_r != 0, static_cast<char *>(sc.slab));
        cudaError_t e = reset();
        if (e == cudaSuccess)
            e = t.dp_us[0] > 0 ? launch_dpc(v, NBT, k, nullptr, 0, s)
                               : launch_dp_select(v, NBT, k, nullptr, 0, s);
        if (e != cudaSuccess) result = SCPL_ECUDA;
        const int rows[3] = {1, 2, 4};
        float ubest = 1e30f;
        for (int i = 0; i < 3 && result == SCPL_OK; ++i) {
            CarveWs u = v;
            u.up_rows = rows[i];
            float tb = 1e30f;
            for (int r = 0; r <= reps; ++r) {
                cudaEventRecord(a, s);
                e = launch_update(u, NBT, s);   // idempotent on a pending iteration
                cudaEventRecord(b, s);
                if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
                    result = SCPL_ECUDA;
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, a, b);
                if (r > 0) tb = std::min(tb, ms);
            }
            t.up_us[i] = tb * 1000.0f;
            if (tb < ubest) {
                ubest = tb;
                t.update_rows = rows[i];
            }
        }
    }
    int herr = 0;
    if (cudaMemcpy(&herr, sc.err, sizeof herr, cudaMemcpyDeviceToHost) != cudaSuccess || herr)
        result = herr == DEV_ETIMEOUT ? SCPL_ETIMEOUT : SCPL_ECUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaStreamSynchronize(s) != cudaSuccess) result = SCPL_ECUDA;
    if (result != SCPL_OK) return result;
    tuning_store(t);
    if (out) *out = t;
    return SCPL_OK;
}

}  // namespace scpl
