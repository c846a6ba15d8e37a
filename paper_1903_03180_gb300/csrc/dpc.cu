// k_dpc: one SCPL iteration (Sec. 3.1, Eq. 4-6) of a buffer on a thread-block
// cluster.
//
// DP (Eq. 4 with parental labels, Eq. 5).  Each lane holds V consecutive
// columns (V = 4 or 2), so a warp holds a window of 32V columns in registers.
// With halo depth R, warp g owns the 32V - 2R columns in the middle of its
// window, [g(32V-2R), (g+1)(32V-2R)), and the window starts R columns to the
// left of them.  (V = 4, R = 32: 64 owned of 128; V = 4, R = 16: 96 of 128;
// V = 2, R = 16: 32 of 64.)  A row step needs only the neighbours in the
// adjacent lanes (shuffles); the window's outer columns go stale one column
// per row (trapezoid), so after R rows exactly the owned columns are still
// exact.  Then every warp sends the R owned columns at each of its edges
// straight into its neighbours' inboxes with st.async (shared or distributed
// shared memory), which completes on the receiving warp's mbarrier, and
// refreshes its own R-column halos from its inbox.  Warps are coupled only to
// their two neighbours; the DP loop takes no CTA or cluster barrier.  Each
// warp's energy rows arrive by TMA tensor copies (one 16-row x 32V-column box
// per stage) into its own ring.  V = 2 halves a warp's instructions per row,
// so two warps can share an SM sub-partition and fill each other's dependency
// stalls.
//
// Forward terms (FWD): each stage also brings the 16 x 32V box of the P plane
// (the pixel's summed diagonal terms A | B << 16) by TMA on the same mbarrier,
// and the moves from the upper left and right cost wf * A and wf * B more.
// Outside [0, W) both are taken as 0, so a column next to a real one still
// ends up at 2^31 or more.
//
// Columns outside [0, W) carry energy 2^31: a real cumulative energy is below
// 2^31 (checked on the host), so the column next to a real one always ends up
// at 2^31 or more and is never chosen, whatever lies further out.  Among equal
// cumulative energies the lowest column wins (candidates compared j-1, j, j+1
// with a strict "<"), which keeps paths non-crossing.
//
// Every pixel carries (label << 16 | anchor): the label is the row-0 column of
// its path (Eq. 5); the anchor is the path's column in the row just above the
// current trace-back band of rj rows (the parent it took at the band's first
// row; in band 0 its row-0 column).  At each band's last row the anchors of
// the owned columns are stored (J): the column at the last row of the band
// above, so the trace back goes from band to band in one look-up.
//
// Selection (Eq. 6): each CTA min-reduces (CE << 32 | column) per label over
// its owned last-row columns and writes each parent's minimum, once, into its
// list in CTA 0 (distributed shared memory); CTA 0 merges the short lists,
// ranks the parents' minima and keeps the k_eff lowest.
//
// Trace back: CTA 0 follows every selected seam from band to band through J
// (bulk-copied into shared memory) and records the seam's column at every
// band's last row; then the other CTAs (CTA 0 alone in a one-CTA cluster)
// walk all seams through their share of the bands at once (one thread per
// seam and band), the bands' directions bulk-copied into shared memory while
// the selection runs, and write the per-row removal lists.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "scpl_internal.cuh"

namespace cg = cooperative_groups;

namespace scpl {

namespace {

constexpr int DPC_S = 16;                        // rows per TMA stage of the energy ring
// The template parameters of k_dpc: the halo depth R (16 or 32), which is also
// the number of rows between halo refreshes; the warps per CTA WPC (4 or 8:
// with 8 the cluster needs half the CTAs and two warps share an SM
// sub-partition); and the columns per lane V (4 or 2; 2 only with R = 16).
__host__ __device__ constexpr int dpc_ww(int V) { return 32 * V; }   // a warp's window
__host__ __device__ constexpr int dpc_oww(int R, int V) { return dpc_ww(V) - 2 * R; }
// energy stages in flight per warp (8 warps of 128-column windows, or 4 with
// the forward terms' second ring, keep 2 to fit shared memory)
__host__ __device__ constexpr int dpc_nst(int WPC, int V, bool FWD = false) {
    return V == 4 && (WPC == 8 || FWD) ? 2 : 4;
}
__host__ __device__ constexpr int dpc_lmax(int R, int WPC, int V) { return WPC * dpc_oww(R, V); }
__host__ __device__ constexpr size_t dpc_wslot(int V) {   // one warp's stage: 8 or 4 KB
    return (size_t)DPC_S * dpc_ww(V) * 4;
}
__host__ __device__ constexpr size_t dpc_ring(int WPC, int V, bool FWD = false) {
    return (size_t)WPC * dpc_nst(WPC, V, FWD) * dpc_wslot(V);   // per plane
}
constexpr size_t DPC_STAGE_BUDGET = 96 * 1024;   // trace-back staging
constexpr uint32_t BIG = 0x80000000u;            // energy of columns outside [0, W)
constexpr uint32_t INF32 = 0xFFFFFFFFu;
constexpr unsigned long long WAIT_NS = 2000000000ull;

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

// Shared-memory layout after the DP (aliases the energy ring).  segmin comes
// first in every CTA; the rest is CTA 0's: the other CTAs' lists of their
// parents' minima (keys, labels and counts per CTA), the candidates, the
// selection and the band anchors.
struct PostLayout {
    size_t segmin, cand, sel, pos, js, lkeys, llabs, lcnt, end;
    __host__ __device__ PostLayout(int W0, int C, int kcap, int nb, int jstride, int lmax) {
        size_t o = 0;
        segmin = o; o = al16(o + (size_t)W0 * 8);
        cand = o;   o = al16(o + (size_t)W0 * 8);
        sel = o;    o = al16(o + (size_t)kcap * 4);
        pos = o;    o = al16(o + (size_t)kcap * 4);
        js = o;     o = al16(o + (size_t)nb * jstride * 2);
        lkeys = o;  o = al16(o + (size_t)C * lmax * 8);
        llabs = o;  o = al16(o + (size_t)C * lmax * 4);
        lcnt = o;   o = al16(o + (size_t)C * 4);
        end = o;
    }
};

// Trace-back walk layout: after segmin, so that the walking CTAs can stage
// their bands' directions while the parents' minima are still being taken
// (it aliases the rest of CTA 0's layout, which a walk starts only after).
struct WalkLayout {
    size_t stage, cur, pos, end;
    __host__ __device__ WalkLayout(int W0, int kcap, int nbq_max) {
        stage = al16((size_t)W0 * 8);
        cur = al16(stage + DPC_STAGE_BUDGET);
        pos = al16(cur + (size_t)nbq_max * kcap * 4);
        end = al16(pos + (size_t)kcap * 4);
    }
};

__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// 16 or 8 bytes into (possibly another CTA's) shared memory, completing on
// that CTA's mbarrier.
__device__ __forceinline__ void st_async_v(uint32_t raddr, const uint32_t (&v)[4], uint32_t rmbar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::
            "r"(raddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(rmbar)
        : "memory");
}
__device__ __forceinline__ void st_async_v(uint32_t raddr, const uint32_t (&v)[2], uint32_t rmbar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(
            raddr),
        "r"(v[0]), "r"(v[1]), "r"(rmbar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z,
                                            uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
        : "memory");
}
// Bounded wait with cluster-scope acquire (data written by other CTAs).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *mbar, unsigned parity, int *err,
                                                  unsigned long long limit_ns) {
    auto try_once = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (try_once()) return true;
    if (err && *(volatile int *)err != DEV_OK) return false;   // an earlier wait gave up
    const unsigned long long t0 = globaltimer_now();
    while (!try_once()) {
        if (globaltimer_now() - t0 > limit_ns) {
            if (err) atomicExch(err, DEV_ETIMEOUT);
            return false;
        }
    }
    return true;
}

template <int R, int WPC, int V, bool FWD>
__global__ void __launch_bounds__(WPC * 32, 1)
k_dpc(const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmP,
      CarveWs ws, int k, int16_t *seams, long seam_stride) {
    static_assert((V == 4 && (R == 16 || R == 32)) || (V == 2 && R == 16), "window layout");
    constexpr int DPC_V = V;                      // columns per lane
    constexpr int DPC_WW = dpc_ww(V);             // columns of a warp's window
    constexpr size_t DPC_WSLOT = dpc_wslot(V);    // bytes of one warp's stage
    constexpr int DPC_WPC = WPC;                  // warps per CTA
    constexpr int DPC_NST = dpc_nst(WPC, V, FWD); // energy stages in flight per warp
    constexpr int DPC_R = R;                      // rows between halo refreshes (= halo width)
    constexpr int DPC_SPR = DPC_R / DPC_S;        // stages per refresh
    constexpr int DPC_HL = DPC_R / DPC_V;         // halo lanes on each side of a warp
    constexpr int DPC_OWW = dpc_oww(R, V);        // owned columns per warp
    constexpr int DPC_LMAX = dpc_lmax(R, WPC, V); // parents a CTA can report
    extern __shared__ __align__(128) unsigned char smraw[];
    // halo inboxes: [parity][warp][value], filled by the neighbouring warps
    __shared__ __align__(16) uint32_t inLc[2][DPC_WPC][DPC_R], inLl[2][DPC_WPC][DPC_R];
    __shared__ __align__(16) uint32_t inRc[2][DPC_WPC][DPC_R], inRl[2][DPC_WPC][DPC_R];
    __shared__ __align__(8) uint64_t mring[DPC_WPC][DPC_NST];   // per-warp energy stages
    __shared__ __align__(8) uint64_t minbox[DPC_WPC][2];        // per-warp halo inboxes
    __shared__ __align__(8) uint64_t mbar[2];                    // trace-back copies
    __shared__ int s_cnt, s_keff;

    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int b = blockIdx.x / C;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int NT = blockDim.x;
    const int g = crank * DPC_WPC + w;
    const int nwarps = C * DPC_WPC;
    const int H = ws.H, W0 = ws.W0, RJ = ws.rj, NB = ws.nbands;

    pdl_launch_dependents();
    pdl_wait();   // the previous update's carved energy and state
    const BufState st0 = ws.st[b];
    int W, slot, removed;
    committed(st0, W, slot, removed);
    if (W <= st0.target) {
        if (crank == 0 && tid == 0) {
            BufState st = st0;
            st.W = W; st.slot = slot; st.removed = removed; st.k_eff = 0;
            ws.st[b] = st;
        }
        return;
    }

    const int32_t *E = ws.E + ((long)b * 2 + slot) * ws.plane;
    const long pitch = ws.pitch;
    const int cbase = g * DPC_OWW - DPC_R + lane * DPC_V;   // lane's first column
    const bool owner = lane >= DPC_HL && lane < 32 - DPC_HL;
    const int dstride = ws.dstride;
    uint32_t *dirs = ws.dirs + (long)b * ws.dbuf;
    uint16_t *J = ws.J + (long)b * NB * ws.jstride;

    // ---- per-warp energy ring: stage s holds rows 1+16s .. 16+16s of the
    //      warp's 128-column window ---------------------------------------------
    uint32_t *wring = reinterpret_cast<uint32_t *>(smraw) + (size_t)w * DPC_NST * DPC_S * DPC_WW;
    // forward terms: the P boxes, in a second ring after the energy ring
    uint32_t *pring = reinterpret_cast<uint32_t *>(smraw + dpc_ring(WPC, V, FWD)) +
                      (size_t)w * DPC_NST * DPC_S * DPC_WW;
    const uint32_t wfw = FWD ? (uint32_t)ws.wf : 0u;
    const int wx = g * DPC_OWW - DPC_R;   // first column of the warp's window
    const int zplane = b * 2 + slot;
    const int nstages = (H - 1 + DPC_S - 1) / DPC_S;
    auto issue = [&](int s) {   // lane 0 of the warp
        if (s >= nstages) return;
        uint64_t *mb = &mring[w][s % DPC_NST];
        mbar_expect_tx(mb, (unsigned)DPC_WSLOT * (FWD ? 2u : 1u));
        tma_load_3d(wring + (size_t)(s % DPC_NST) * DPC_S * DPC_WW, &tmE, wx, 1 + s * DPC_S,
                    zplane, mb);
        if constexpr (FWD)
            tma_load_3d(pring + (size_t)(s % DPC_NST) * DPC_S * DPC_WW, &tmP, wx, 1 + s * DPC_S,
                        zplane, mb);
    };
    // halo bytes a warp receives per refresh: 32 costs and 32 labels per neighbour
    const unsigned in_bytes =
        (g > 0 ? 2u * DPC_R * 4u : 0u) + (g + 1 < nwarps ? 2u * DPC_R * 4u : 0u);
    if (lane == 0) {
        for (int i = 0; i < DPC_NST; ++i) mbar_init(&mring[w][i], 1);
        mbar_init(&minbox[w][0], 1);
        mbar_init(&minbox[w][1], 1);
        if (w == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); }
        fence_mbar_init();
        mbar_expect_tx(&minbox[w][0], in_bytes);   // refreshes 0 and 1
        mbar_expect_tx(&minbox[w][1], in_bytes);
        for (int s2 = 0; s2 < DPC_NST; ++s2) issue(s2);
    }
    __syncwarp();

    // ---- row 0 ----------------------------------------------------------------
    uint32_t cost[DPC_V], lab[DPC_V];
#pragma unroll
    for (int v = 0; v < DPC_V; ++v) {
        const int c = cbase + v;
        cost[v] = (c >= 0 && c < W) ? (uint32_t)__ldcg(E + c) : BIG;
        const uint32_t cc = (uint32_t)c & 0xFFFFu;
        lab[v] = (cc << 16) | cc;
    }
    if (H == 1 && owner) {
#pragma unroll
        for (int v = 0; v < DPC_V; ++v) {
            const int c = cbase + v;
            if (c >= 0 && c < W0) J[c] = (uint16_t)(lab[v] & 0xFFFFu);
        }
    }
    uint32_t dw = 0;
    bool valid[DPC_V];
#pragma unroll
    for (int v = 0; v < DPC_V; ++v) valid[v] = cbase + v >= 0 && cbase + v < W;
    cluster.sync();   // every CTA has read the buffer state and initialised its barriers

    // ---- rows 1 .. H-1, one 16-row TMA stage at a time ------------------------
    // Stage s holds rows 16s+1 .. 16s+16; its last row is where the halos are
    // refreshed.  Band boundaries are multiples of 16, so a band's first row is
    // always a stage's last row (ro = 15) and its last row is ro = 14.
    // Directions are kept per 16-row group G (rows 16G .. 16G+15) as one uint4
    // per 4 columns: component b holds rows 16G+4b .. 16G+4b+3, 2 bits each.
    // With V = 2 a lane pair holds the 4 columns: the odd lane's bits sit 4
    // higher, and the pair ORs its words together before the even lane stores.
    uint32_t wq0 = 0, wq1 = 0, wq2 = 0, wq3 = 0;   // the current group's block words
    const int vsh = V == 2 ? 4 * (lane & 1) : 0;   // bit offset of the lane's columns
    const bool quad_lane = V == 4 || (lane & 1) == 0;
    auto store_group = [&](int G) {
        if constexpr (V == 2) {
            wq0 |= __shfl_xor_sync(0xffffffffu, wq0, 1);
            wq1 |= __shfl_xor_sync(0xffffffffu, wq1, 1);
            wq2 |= __shfl_xor_sync(0xffffffffu, wq2, 1);
            wq3 |= __shfl_xor_sync(0xffffffffu, wq3, 1);
        }
        if (owner && quad_lane && cbase >= 0 && cbase < W0) {
            reinterpret_cast<uint4 *>(dirs)[(long)G * dstride + (cbase >> 2)] =
                make_uint4(wq0, wq1, wq2, wq3);
        }
        wq0 = wq1 = wq2 = wq3 = 0;
    };
    // band edges by countdown (rj is a multiple of 16): the stage whose last
    // row starts a band, and the index of the band that ends one row above
    const int spb = RJ / DPC_S;
    int bleft = spb, bq = 0;
    bool band_edge = false;
    auto stage_rows = [&](int s, auto guarded) {
        constexpr bool GUARD = decltype(guarded)::value;
        const uint32_t *rs = wring + (size_t)(s % DPC_NST) * DPC_S * DPC_WW + lane * DPC_V;
        const uint32_t *ps = pring + (size_t)(s % DPC_NST) * DPC_S * DPC_WW + lane * DPC_V;
        const int ibase = 1 + DPC_S * s;
        // with plain energy the stage's 16 rows are read into registers
        // first, off the rows' dependency chain (with the forward terms the
        // extra registers made the DP slower)
        constexpr bool PRE = V == 2 && !FWD;
        constexpr bool PRE4 = V == 4 && !FWD;
        [[maybe_unused]] uint2 epre[PRE ? DPC_S : 1];
        [[maybe_unused]] uint2 ppre[PRE && FWD ? DPC_S : 1];
        [[maybe_unused]] uint4 epre4[PRE4 ? DPC_S : 1];
        if constexpr (PRE4) {
#pragma unroll
            for (int ro = 0; ro < DPC_S; ++ro) {
                const uint4 ev = *reinterpret_cast<const uint4 *>(rs + ro * DPC_WW);
                epre4[ro] = make_uint4(valid[0] ? ev.x : BIG, valid[1] ? ev.y : BIG,
                                       valid[2] ? ev.z : BIG, valid[3] ? ev.w : BIG);
            }
        }
        if constexpr (PRE) {
#pragma unroll
            for (int ro = 0; ro < DPC_S; ++ro) {
                const uint2 ev = *reinterpret_cast<const uint2 *>(rs + ro * DPC_WW);
                epre[ro] = make_uint2(valid[0] ? ev.x : BIG, valid[1] ? ev.y : BIG);
                if constexpr (FWD) {
                    const uint2 pv = *reinterpret_cast<const uint2 *>(ps + ro * DPC_WW);
                    ppre[ro] = make_uint2(valid[0] ? pv.x : 0u, valid[1] ? pv.y : 0u);
                }
            }
        }
#pragma unroll
        for (int ro = 0; ro < DPC_S; ++ro) {
            const int i = ibase + ro;
            if (!GUARD || i < H) {
                uint32_t e[DPC_V];
                if constexpr (PRE) {
                    e[0] = epre[ro].x;
                    e[DPC_V - 1] = epre[ro].y;
                } else if constexpr (PRE4) {
                    e[0] = epre4[ro].x;
                    e[1 % DPC_V] = epre4[ro].y;
                    e[2 % DPC_V] = epre4[ro].z;
                    e[3 % DPC_V] = epre4[ro].w;
                } else if constexpr (V == 4) {
                    const uint4 ev = *reinterpret_cast<const uint4 *>(rs + ro * DPC_WW);
                    e[0] = valid[0] ? ev.x : BIG;
                    e[1] = valid[1] ? ev.y : BIG;
                    e[2] = valid[2] ? ev.z : BIG;
                    e[3] = valid[3] ? ev.w : BIG;
                } else {
                    const uint2 ev = *reinterpret_cast<const uint2 *>(rs + ro * DPC_WW);
                    e[0] = valid[0] ? ev.x : BIG;
                    e[1] = valid[1] ? ev.y : BIG;
                }
                [[maybe_unused]] uint32_t pw[DPC_V];   // forward terms of the row's pixels (0 outside [0, W))
                if constexpr (FWD && PRE) {
                    pw[0] = ppre[ro].x;
                    pw[DPC_V - 1] = ppre[ro].y;
                } else if constexpr (FWD) {
                    if constexpr (V == 4) {
                        const uint4 pv = *reinterpret_cast<const uint4 *>(ps + ro * DPC_WW);
                        pw[0] = valid[0] ? pv.x : 0u;
                        pw[1] = valid[1] ? pv.y : 0u;
                        pw[2] = valid[2] ? pv.z : 0u;
                        pw[3] = valid[3] ? pv.w : 0u;
                    } else {
                        const uint2 pv = *reinterpret_cast<const uint2 *>(ps + ro * DPC_WW);
                        pw[0] = valid[0] ? pv.x : 0u;
                        pw[1] = valid[1] ? pv.y : 0u;
                    }
                }
                const uint32_t lc = __shfl_up_sync(0xffffffffu, cost[DPC_V - 1], 1);
                const uint32_t ll = __shfl_up_sync(0xffffffffu, lab[DPC_V - 1], 1);
                const uint32_t rc = __shfl_down_sync(0xffffffffu, cost[0], 1);
                const uint32_t rl = __shfl_down_sync(0xffffffffu, lab[0], 1);
                uint32_t nc[DPC_V], nl[DPC_V], dbyte = 0;
#pragma unroll
                for (int v = 0; v < DPC_V; ++v) {
                    uint32_t c0 = v == 0 ? lc : cost[v - 1];
                    const uint32_t l0 = v == 0 ? ll : lab[v - 1];
                    uint32_t c2 = v == DPC_V - 1 ? rc : cost[v + 1];
                    const uint32_t l2 = v == DPC_V - 1 ? rl : lab[v + 1];
                    if constexpr (FWD) {
                        // real cumulative costs with a move's term stay below
                        // 2^31 (checked on the host); 2^31 and up stays put
                        if (c0 < BIG) c0 += wfw * (pw[v] & 0xFFFFu);
                        if (c2 < BIG) c2 += wfw * (pw[v] >> 16);
                    }
                    // the cost chain is two integer mins; the first index that
                    // attains the minimum (lowest column) is chosen off the chain
                    const uint32_t m = __vimin3_u32(c0, cost[v], c2);
                    const bool p0 = c0 == m, p1 = cost[v] == m;
                    nc[v] = m + e[v];
                    nl[v] = p0 ? l0 : (p1 ? lab[v] : l2);
                    dbyte |= (p0 ? 0u : (p1 ? 1u : 2u)) << (2 * v);
                }
#pragma unroll
                for (int v = 0; v < DPC_V; ++v) { cost[v] = nc[v]; lab[v] = nl[v]; }
                if (ro == DPC_S - 1 && band_edge) {
                    // a band's first row: the anchor becomes the parent's
                    // column in the row above (the direction just chosen)
#pragma unroll
                    for (int v = 0; v < DPC_V; ++v)
                        lab[v] = (lab[v] & 0xFFFF0000u) |
                                 ((uint32_t)(cbase + v + (int)((dbyte >> (2 * v)) & 3u) - 1) &
                                  0xFFFFu);
                }
                dw |= dbyte << (8 * ((1 + ro) & 3) + vsh);
                if (((1 + ro) & 3) == 3) {   // row i closes a 4-row block
                    if (ro == 2) wq0 = dw;
                    if (ro == 6) wq1 = dw;
                    if (ro == 10) wq2 = dw;
                    if (ro == 14) { wq3 = dw; }
                    dw = 0;
                    if (ro == 14) store_group(s);   // rows 16s .. 16s+15 are complete
                }
                if (ro == DPC_S - 2 && band_edge && owner) {   // a band's last row
                    uint16_t *Jrow = J + (long)bq * ws.jstride;
#pragma unroll
                    for (int v = 0; v < DPC_V; ++v) {
                        const int c = cbase + v;
                        if (c >= 0 && c < W0) Jrow[c] = (uint16_t)(lab[v] & 0xFFFFu);
                    }
                }
            }
        }
    };
    // After a stage's rows: the edge strips go out to the neighbours first
    // (they wait for them), then lane 0 refills the ring slot and arms the
    // inbox that the previous refresh emptied, then the warp waits for its
    // own inbox.  Each of the three is one divergent region of the warp.
    int arm = -1;   // inbox parity to re-arm at the next stage (-1: none)
    for (int s = 0; s < nstages; ++s) {
        mbar_wait(&mring[w][s % DPC_NST], (unsigned)(s / DPC_NST) & 1u, ws.err, WAIT_NS);
        const int ibase = 1 + DPC_S * s;
        band_edge = --bleft == 0;   // row 16s+16 starts a band
        if (ibase + DPC_S - 1 < H) stage_rows(s, std::false_type{});
        else stage_rows(s, std::true_type{});
        if (band_edge) { bleft = spb; ++bq; }
        const int ilast = ibase + DPC_S - 1;   // the stage's last row
        const bool refresh = (s + 1) % DPC_SPR == 0 && ilast < H - 1;
        const int e = (s + 1) / DPC_SPR - 1, par = e & 1;
        if (refresh) {
            // refresh e: lanes [32-2HL, 32-HL) send to the right neighbour's
            // left inbox, lanes [HL, 2HL) to the left neighbour's right inbox
            const bool toR = lane >= 32 - 2 * DPC_HL && lane < 32 - DPC_HL;
            const bool toL = lane >= DPC_HL && lane < 2 * DPC_HL;
            if ((toR && g + 1 < nwarps) || (toL && g > 0)) {
                const int tg = toR ? g + 1 : g - 1, tr = tg / DPC_WPC, tw = tg % DPC_WPC;
                const int o = (toR ? lane - (32 - 2 * DPC_HL) : lane - DPC_HL) * DPC_V;
                uint32_t *cb = toR ? &inLc[par][tw][o] : &inRc[par][tw][o];
                uint32_t *lb = toR ? &inLl[par][tw][o] : &inRl[par][tw][o];
                const uint32_t mb = mapa_u32(smem_u32(&minbox[tw][par]), tr);
                st_async_v(mapa_u32(smem_u32(cb), tr), cost, mb);
                st_async_v(mapa_u32(smem_u32(lb), tr), lab, mb);
            }
        }
        __syncwarp();   // every lane has read the slot's rows
        if (lane == 0) {
            issue(s + DPC_NST);
            // the inbox of parity `arm` (its refresh already waited for)
            // serves the refresh two later, which a neighbour sends only
            // after it has this warp's refresh e strips (sent above).  Bytes
            // that land before this arrive only take the barrier's
            // transaction count below zero for a while; the phase cannot
            // complete before the arrive, which adds the expected bytes.
            if (arm >= 0) mbar_expect_tx(&minbox[w][arm], in_bytes);
        }
        arm = -1;
        if (refresh) {
            mbar_wait_cluster(&minbox[w][par], (unsigned)(e >> 1) & 1u, ws.err, WAIT_NS);
            if (lane < DPC_HL || lane >= 32 - DPC_HL) {
                const bool left = lane < DPC_HL;
                const int o = (left ? lane : lane - (32 - DPC_HL)) * DPC_V;
                const uint32_t *cs = left ? &inLc[par][w][o] : &inRc[par][w][o];
                const uint32_t *ls = left ? &inLl[par][w][o] : &inRl[par][w][o];
                const bool edge = left ? g == 0 : g == nwarps - 1;
#pragma unroll
                for (int v = 0; v < DPC_V; ++v) {
                    cost[v] = edge ? INF32 : cs[v];
                    lab[v] = ls[v];
                }
            }
            arm = par;
        }
    }
    // the last row: a partial 4-row block, group and band are stored here
    if (H > 1) {
        const int il = H - 1;
        if ((il & 15) != 15) {
            if ((il & 3) != 3) {
                const int bq = (il >> 2) & 3;
                if (bq == 0) wq0 = dw;
                if (bq == 1) wq1 = dw;
                if (bq == 2) wq2 = dw;
                if (bq == 3) wq3 = dw;
            }
            store_group(il >> 4);
        }
        if ((il % RJ) != RJ - 1 && owner) {
            uint16_t *Jrow = J + (long)(il / RJ) * ws.jstride;
#pragma unroll
            for (int v = 0; v < DPC_V; ++v) {
                const int c = cbase + v;
                if (c >= 0 && c < W0) Jrow[c] = (uint16_t)(lab[v] & 0xFFFFu);
            }
        }
    }
    // directions, anchors and band rows are read back through the async proxy
    fence_proxy_async();
    const PostLayout PL(W0, C, ws.kcap, NB, ws.jstride, DPC_LMAX);
    uint64_t *segmin = reinterpret_cast<uint64_t *>(smraw + PL.segmin);
    cluster.sync();   // every CTA is done with its energy ring

    // the walk's bands (every CTA but CTA 0 when there are several) and the
    // staging of their direction words, issued now for the first round
    const int nwalk = C > 1 ? C - 1 : 1, wr = C > 1 ? crank - 1 : crank;
    const int q0 = wr >= 0 ? (wr * NB) / nwalk : 0, q1 = wr >= 0 ? ((wr + 1) * NB) / nwalk : 0;
    const int nbq = q1 - q0;
    const WalkLayout WL(W0, ws.kcap, (NB + nwalk - 1) / nwalk);
    uint32_t *stage = reinterpret_cast<uint32_t *>(smraw + WL.stage);
    const int gpb = RJ / 16;   // 16-row direction groups of a full band
    int cb = nbq > 0 ? (int)(DPC_STAGE_BUDGET / ((size_t)nbq * dstride * 16)) : 1;
    cb = max(1, min(cb, gpb));
    const int rounds = (gpb + cb - 1) / cb;
    auto issue_walk = [&](int j) {   // thread 0: round j's direction words
        unsigned total = 0;
        for (int qq = 0; qq < nbq; ++qq) {
            const int q = q0 + qq;
            const int glo = q * gpb, ghi = (min((q + 1) * RJ, H) + 15) >> 4;
            const int shi = ghi - j * cb, slo = max(glo, shi - cb);
            if (shi > slo) total += (unsigned)(shi - slo) * dstride * 16u;
        }
        mbar_expect_tx(&mbar[1], total);
        for (int qq = 0; qq < nbq; ++qq) {
            const int q = q0 + qq;
            const int glo = q * gpb, ghi = (min((q + 1) * RJ, H) + 15) >> 4;
            const int shi = ghi - j * cb, slo = max(glo, shi - cb);
            if (shi > slo)
                bulk_g2s(stage + (size_t)qq * cb * dstride * 4, dirs + (long)slo * dstride * 4,
                         (unsigned)(shi - slo) * dstride * 16u, &mbar[1]);
        }
    };
    const bool early = C > 1 && nbq > 0;
    if (early && tid == 0) issue_walk(0);

    // ---- Eq. 6: per-parent minima -------------------------------------------------
    // CTA 0 fetches every band's anchors for the band trace now, so the
    // copy overlaps the parents' minima
    if (crank == 0 && tid == 0) {
        const unsigned jbytes = (unsigned)NB * ws.jstride * 2u;
        mbar_expect_tx(&mbar[0], jbytes);
        bulk_g2s(smraw + PL.js, J, jbytes, &mbar[0]);
    }
    uint64_t *lkeys = reinterpret_cast<uint64_t *>(smraw + PL.lkeys);
    uint32_t *llabs = reinterpret_cast<uint32_t *>(smraw + PL.llabs);
    int *lcnt = reinterpret_cast<int *>(smraw + PL.lcnt);
    for (int j = tid; j < W; j += NT) segmin[j] = ~0ull;
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    if (owner) {
        uint64_t run = ~0ull;
#pragma unroll
        for (int v = 0; v < DPC_V; ++v) {
            const int c = cbase + v;
            if (c >= 0 && c < W) {
                const uint64_t key = ((uint64_t)cost[v] << 32) | (uint32_t)c;
                run = key < run ? key : run;
                const bool last = v == DPC_V - 1 || c + 1 >= W ||
                                  (lab[v + (v < DPC_V - 1)] >> 16) != (lab[v] >> 16);
                if (last) {
                    atomicMin(reinterpret_cast<unsigned long long *>(&segmin[lab[v] >> 16]),
                              (unsigned long long)run);
                    run = ~0ull;
                }
            }
        }
    }
    __syncthreads();
    if (crank != 0) {
        // this CTA's minimum of each parent into its list in CTA 0, once per
        // label: at every warp's first owned column and wherever the label
        // changes along the row (labels do not decrease along the row); a
        // label that two warps share appears twice, which the merge absorbs
        uint64_t *rk = cluster.map_shared_rank(lkeys, 0) + (size_t)crank * DPC_LMAX;
        uint32_t *rl = cluster.map_shared_rank(llabs, 0) + (size_t)crank * DPC_LMAX;
        const uint32_t lprev = __shfl_up_sync(0xffffffffu, lab[DPC_V - 1], 1) >> 16;
        if (owner) {
#pragma unroll
            for (int v = 0; v < DPC_V; ++v) {
                const int c = cbase + v;
                const uint32_t l = lab[v] >> 16;
                const uint32_t pl = v == 0 ? lprev : (lab[v > 0 ? v - 1 : 0] >> 16);
                if (c < W && ((v == 0 && lane == DPC_HL) || l != pl)) {
                    const int idx = atomicAdd(&s_cnt, 1);   // < owned columns
                    rk[idx] = segmin[l];
                    rl[idx] = l;
                }
            }
        }
        __syncthreads();
        if (tid == 0) *cluster.map_shared_rank(lcnt + crank, 0) = s_cnt;
    }
    cluster.sync();

    int *dpx = ws.dpx + (long)b * (1 + ws.kcap);
    uint16_t *colbot = ws.colbot + (long)b * NB * ws.kcap;
    if (crank == 0) {
        uint64_t *cand = reinterpret_cast<uint64_t *>(smraw + PL.cand);
        int *sel = reinterpret_cast<int *>(smraw + PL.sel);
        int *pos = reinterpret_cast<int *>(smraw + PL.pos);
        uint16_t *Js = reinterpret_cast<uint16_t *>(smraw + PL.js);
        // the other CTAs' lists, merged in parallel (entry e of the lists
        // laid end to end)
        int total = 0;
        for (int r = 1; r < C; ++r) total += lcnt[r];
        for (int e = tid; e < total; e += NT) {
            int r = 1, x = e;
            while (x >= lcnt[r]) x -= lcnt[r++];
            atomicMin(reinterpret_cast<unsigned long long *>(
                          &segmin[llabs[(size_t)r * DPC_LMAX + x]]),
                      (unsigned long long)lkeys[(size_t)r * DPC_LMAX + x]);
        }
        __syncthreads();
        for (int a = tid; a < W; a += NT) {
            const uint64_t v = segmin[a];
            if (v != ~0ull) cand[atomicAdd(&s_cnt, 1)] = v;
        }
        __syncthreads();
        const int n = s_cnt;
        int keff = min(st0.k > 0 ? st0.k : k, W - st0.target);
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
            dpx[1 + r] = q;
        }
        if (tid == 0) {
            dpx[0] = keff;
            s_keff = keff;
        }
        mbar_wait(&mbar[0], 0u, ws.err, WAIT_NS);
        // each seam's column at every band's last row, band by band upwards
        // (columns are checked against [0, W): a table entry outside it can
        // only come from a fault, which is reported instead of followed)
        for (int s = tid; s < keff; s += NT) {
            int col = sel[s];
            colbot[(long)(NB - 1) * ws.kcap + s] = (uint16_t)col;
            for (int q = NB - 1; q > 0; --q) {
                col = Js[(long)q * ws.jstride + col];   // the band above's last row
                if (col >= W) { atomicExch(ws.err, DEV_EINTERNAL); col = W - 1; }
                colbot[(long)(q - 1) * ws.kcap + s] = (uint16_t)col;
            }
        }
    }
    cluster.sync();

    // ---- trace back: every CTA walks all seams through its bands at once -------
    const int keff = __ldcg(dpx);
    int *cur = reinterpret_cast<int *>(smraw + WL.cur);
    int *pos_s = reinterpret_cast<int *>(smraw + WL.pos);
    const uint16_t *Ocur = ws.O + ((long)b * 2 + slot) * ws.plane;
    uint16_t *rem = ws.rem + (long)b * H * ws.kcap;
    if (nbq > 0) {
        for (int s = tid; s < keff; s += NT) pos_s[s] = __ldcg(dpx + 1 + s);
        for (int x = tid; x < nbq * keff; x += NT) {
            const int qq = x / keff, s = x - qq * keff;
            cur[x] = __ldcg(colbot + (long)(q0 + qq) * ws.kcap + s);
        }
        for (int j = 0; j < rounds; ++j) {
            __syncthreads();   // the previous round's staging is consumed
            if (tid == 0 && !(early && j == 0)) issue_walk(j);
            mbar_wait(&mbar[1], (unsigned)j & 1u, ws.err, WAIT_NS);
            for (int x = tid; x < nbq * keff; x += NT) {
                const int qq = x / keff, s = x - qq * keff;
                const int q = q0 + qq;
                const int rtop = q * RJ, rend = min((q + 1) * RJ, H);
                const int glo = q * gpb, ghi = (rend + 15) >> 4;
                const int shi = ghi - j * cb, slo = max(glo, shi - cb);
                if (shi <= slo) continue;
                const int i_hi = min(shi * 16, rend) - 1, i_lo = max(slo * 16, rtop);
                const uint32_t *sq = stage + (size_t)qq * cb * dstride * 4;
                int col = cur[x];
                if (col >= W) { atomicExch(ws.err, DEV_EINTERNAL); col = W - 1; }
                const int mypos = pos_s[s];
                for (int i = i_hi; i >= i_lo; --i) {
                    rem[(long)i * ws.kcap + mypos] = (uint16_t)col;
                    if (seams)
                        seams[(long)b * seam_stride + (long)(removed + s) * H + i] =
                            (int16_t)Ocur[(long)i * pitch + col];
                    if (i > rtop) {
                        const uint32_t word =
                            sq[((size_t)((i >> 4) - slo) * dstride + (col >> 2)) * 4 + ((i >> 2) & 3)];
                        col += (int)((word >> (8 * (i & 3) + 2 * (col & 3))) & 3u) - 1;
                        if (col < 0 || col >= W) { atomicExch(ws.err, DEV_EINTERNAL); col = min(max(col, 0), W - 1); }
                    }
                }
                cur[x] = col;
            }
        }
    }

    if (crank == 0 && tid == 0) {
        BufState st = st0;
        st.W = W; st.slot = slot; st.removed = removed;
        st.k_eff = s_keff;
        const int it = st0.iters;
        if (it < ws.klog_stride) ws.klog[(long)b * ws.klog_stride + it] = s_keff;
        st.iters = it + 1;
        ws.st[b] = st;
    }
}

size_t dpc_smem(int W0, int H, int rj, int kcap, int C, int R, int WPC, int V, bool fwd) {
    const int nb = (H + rj - 1) / rj;
    const int jstride = (W0 + 7) & ~7;
    const PostLayout PL(W0, C, kcap, nb, jstride, dpc_lmax(R, WPC, V));
    const int nwalk = C > 1 ? C - 1 : 1;
    const WalkLayout WL(W0, kcap, (nb + nwalk - 1) / nwalk);
    size_t m = dpc_ring(WPC, V, fwd) * (fwd ? 2 : 1);
    m = PL.end > m ? PL.end : m;
    m = WL.end > m ? WL.end : m;
    return m;
}

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D view of E, or of P ([nb*2 planes][H][pitch], 32-bit) with 16-row x
// 32V-column boxes.
bool make_energy_map(const CarveWs &ws, const void *plane0, int nb, int V, CUtensorMap *m) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)ws.pitch, (cuuint64_t)ws.H, (cuuint64_t)nb * 2};
    const cuuint64_t strides[2] = {(cuuint64_t)ws.pitch * 4, (cuuint64_t)ws.plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)dpc_ww(V), DPC_S, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, const_cast<void *>(plane0), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool dpc_plan(int W0, int H, int R, int WPC, int V, int *ctas, int *rj, size_t *smem, bool fwd) {
    if ((R != 16 && R != 32) || (WPC != 4 && WPC != 8) || (V != 4 && V != 2)) return false;
    if (V == 2 && R != 16) return false;
    // forward terms: the layouts built with them (R16 x 4 x 2, R32 x 4 x 4)
    if (fwd && !(WPC == 4 && ((R == 16 && V == 2) || (R == 32 && V == 4)))) return false;
    const int nwarps = (W0 + dpc_oww(R, V) - 1) / dpc_oww(R, V);
    const int C = (nwarps + WPC - 1) / WPC;
    if (C > 16) return false;
    // about four bands per CTA: the walk then takes ~rj rows per CTA
    int r = (H + 4 * C - 1) / (4 * C);
    r = ((r + 15) / 16) * 16;
    if (r < 16) r = 16;
    size_t bytes = dpc_smem(W0, H, r, W0, C, R, WPC, V, fwd);
    while (bytes > 220 * 1024 && r < H) {
        r += 16;
        bytes = dpc_smem(W0, H, r, W0, C, R, WPC, V, fwd);
    }
    if (bytes > 220 * 1024) return false;
    // the walk stages at least one 16-row group of every band a CTA owns
    const int nbands = (H + r - 1) / r;
    const size_t dstride = (size_t)((((W0 + 3) / 4) + 3) & ~3);
    const int nwalk = C > 1 ? C - 1 : 1;
    if ((size_t)((nbands + nwalk - 1) / nwalk) * dstride * 16 > DPC_STAGE_BUDGET) return false;
    *ctas = C;
    *rj = r;
    *smem = bytes;
    return true;
}

namespace {

template <int R, int WPC, int V, bool FWD>
bool dpc_available_t(int W0, int H) {
    int C = 0, rj = 0;
    size_t smem = 0;
    if (!dpc_plan(W0, H, R, WPC, V, &C, &rj, &smem, FWD)) return false;
    if (raise_dyn_smem((const void *)k_dpc<R, WPC, V, FWD>, smem) != cudaSuccess) return false;
    if (C > 8 && cudaFuncSetAttribute(k_dpc<R, WPC, V, FWD>,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed,
                                      1) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(WPC * 32);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_dpc<R, WPC, V, FWD>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters > 0;
}

template <int R, int WPC, int V, bool FWD>
cudaError_t launch_dpc_t(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                         cudaStream_t s) {
    int C = 0, rj = 0;
    size_t smem = 0;
    if (!dpc_plan(ws.W0, ws.H, R, WPC, V, &C, &rj, &smem, FWD) || rj != ws.rj)
        return cudaErrorInvalidValue;
    smem = dpc_smem(ws.W0, ws.H, ws.rj, ws.kcap, C, R, WPC, V, FWD);
    cudaError_t e = raise_dyn_smem((const void *)k_dpc<R, WPC, V, FWD>, smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(k_dpc<R, WPC, V, FWD>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb * C);
    cfg.blockDim = dim3(WPC * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    CUtensorMap tm, tp;
    if (!make_energy_map(ws, ws.E, nb, V, &tm)) return cudaErrorInvalidValue;
    if (FWD && (!ws.P || !make_energy_map(ws, ws.P, nb, V, &tp))) return cudaErrorInvalidValue;
    e = cudaLaunchKernelEx(&cfg, k_dpc<R, WPC, V, FWD>, tm, FWD ? tp : tm, ws, k, seams,
                           seam_stride);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool dpc_available_uncached(int W0, int H, int R, int WPC, int V, bool fwd) {
    if (!encode_tiled()) return false;
    if (fwd) {   // the layouts built with the forward terms
        if (WPC == 4 && R == 16 && V == 2) return dpc_available_t<16, 4, 2, true>(W0, H);
        if (WPC == 4 && R == 32 && V == 4) return dpc_available_t<32, 4, 4, true>(W0, H);
        return false;
    }
    if (V == 2) {
        if (R != 16) return false;
        return WPC == 8 ? dpc_available_t<16, 8, 2, false>(W0, H)
                        : WPC == 4 && dpc_available_t<16, 4, 2, false>(W0, H);
    }
    if (V != 4) return false;
    if (WPC == 4)
        return R == 16 ? dpc_available_t<16, 4, 4, false>(W0, H)
                       : R == 32 && dpc_available_t<32, 4, 4, false>(W0, H);
    if (WPC == 8)
        return R == 16 ? dpc_available_t<16, 8, 4, false>(W0, H)
                       : R == 32 && dpc_available_t<32, 8, 4, false>(W0, H);
    return false;
}

// Availability depends only on the size, the layout and the device: cached.
bool dpc_available(int W0, int H, int R, int WPC, int V, bool fwd) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, bool>, bool> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const auto key = std::make_tuple(dev, W0, H, R, WPC, V, fwd);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const bool ok = dpc_available_uncached(W0, H, R, WPC, V, fwd);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = ok;
    return ok;
}

// The layout for a size: the requested one if this GPU can run it, else the
// first that it can run of R16 x 4 warps x 2 columns a lane (the fastest
// where its cluster fits: half the instructions a row of the 4-column
// layouts), R32 x 4 x 4 and R16 x 4 x 4.  With the forward terms (ws.wf > 0)
// the first of R16 x 4 x 2 and R32 x 4 x 4 that runs, whatever was requested
// (the tuner times the plain kernels).  False: use the single-CTA DP.
bool dpc_select(int W0, int H, CarveWs &ws, bool requested) {
    if (ws.wf > 0) {
        static const int fwd_order[2][3] = {{16, 4, 2}, {32, 4, 4}};
        for (const auto &o : fwd_order)
            if (dpc_available(W0, H, o[0], o[1], o[2], true)) {
                ws.dpc_r = o[0];
                ws.dpc_wpc = o[1];
                ws.dpc_v = o[2];
                return true;
            }
        return false;
    }
    if (requested && dpc_available(W0, H, ws.dpc_r, ws.dpc_wpc, ws.dpc_v)) return true;
    static const int order[3][3] = {{16, 4, 2}, {32, 4, 4}, {16, 4, 4}};
    for (const auto &o : order)
        if (dpc_available(W0, H, o[0], o[1], o[2])) {
            ws.dpc_r = o[0];
            ws.dpc_wpc = o[1];
            ws.dpc_v = o[2];
            return true;
        }
    return false;
}

cudaError_t launch_dpc(const CarveWs &ws, int nb, int k, int16_t *seams, long seam_stride,
                       cudaStream_t s) {
    const int wpc = ws.dpc_wpc == 8 ? 8 : 4;
    const int v = ws.dpc_v == 2 ? 2 : 4;
    if (ws.wf > 0) {
        if (ws.dpc_r == 16 && wpc == 4 && v == 2)
            return launch_dpc_t<16, 4, 2, true>(ws, nb, k, seams, seam_stride, s);
        if (ws.dpc_r == 32 && wpc == 4 && v == 4)
            return launch_dpc_t<32, 4, 4, true>(ws, nb, k, seams, seam_stride, s);
        return cudaErrorInvalidValue;
    }
    if (v == 2) {
        if (ws.dpc_r == 16 && wpc == 8)
            return launch_dpc_t<16, 8, 2, false>(ws, nb, k, seams, seam_stride, s);
        if (ws.dpc_r == 16 && wpc == 4)
            return launch_dpc_t<16, 4, 2, false>(ws, nb, k, seams, seam_stride, s);
        return cudaErrorInvalidValue;
    }
    if (ws.dpc_r == 16 && wpc == 4) return launch_dpc_t<16, 4, 4, false>(ws, nb, k, seams, seam_stride, s);
    if (ws.dpc_r == 32 && wpc == 4) return launch_dpc_t<32, 4, 4, false>(ws, nb, k, seams, seam_stride, s);
    if (ws.dpc_r == 16 && wpc == 8) return launch_dpc_t<16, 8, 4, false>(ws, nb, k, seams, seam_stride, s);
    if (ws.dpc_r == 32 && wpc == 8) return launch_dpc_t<32, 8, 4, false>(ws, nb, k, seams, seam_stride, s);
    return cudaErrorInvalidValue;
}

}  // namespace scpl
