// fused_kernels.cuh -- one persistent launch per step for every environment
// of a domain (arXiv 2206.01683, Sec. III-B: the coupled IB-LBM step).
//
// The step's work is cut into items, taken in queue order from one ticket
// counter by persistent blocks (all resident: a cooperative launch):
//   MARK     stamp the 32-slot tiles of the markers' 4x4x4 stencils
//   NODE     post-stream rho and u~ of every cell of the stamped tiles
//   FORCE    interpolate at the markers, F = 2 R (U - U~), spread F dV delta
//   INTERP   (multi-direct forcing, pass p) interpolate the corrected
//            velocity, add the increment to the marker force
//   SPREAD   (pass p) spread the increments
//   CONVERT  (deterministic spread) fixed-point sums of the stamped tiles to
//            the FP32 force field
//   REDUCE   force/torque chunk sums of 256 markers, every segment row
//   SC       one block of the plain stream-collide kernel (pull, moments,
//            frame force, collision with the IB force, open faces)
// Items depend only on items of the same environment that come earlier in
// the queue: a phase waits until every item of the phase before it is done
// (a per-environment completion counter), and an SC block waits for the IB
// only if one of its tiles is stamped.  So the SC blocks of cells no marker
// reaches run while the IB phases are still in progress, and in a batch the
// IB phases of the next environment run beside the SC blocks of the last.
// Since every dependency points to an earlier ticket and every block is
// resident, the queue always progresses; every wait is bounded anyway (a
// block that gives up sets ST_TIMEOUT and an abort word that makes the others
// stop).  The mass partials (one per SC block) and the force/torque chunk
// sums are laid out as the plain kernel and k_reduce lay them out, so
// k_reduce with markers_pre = 1 completes the step.
//
// Data written by one block and read by another in the same launch (tile
// stamps, node values, marker forces, the force field) is read through L2
// (ld.global.cg).
#pragma once

#include "ib_kernels.cuh"
#include "reduce_kernels.cuh"

namespace fl {

constexpr int FUSED_THREADS = 256;        // = IB_THREADS = K1_THREADS = RED_THREADS
constexpr int MAX_IB_PASSES = 8;
constexpr int MARKERS_PER_ITEM = 16;      // one per half-warp
constexpr int TILES_PER_ITEM = 1024;      // stamp checks per NODE / CONVERT item (4 per thread)

// Item kinds and the completion-counter slots of one environment.
enum { W_MARK = 0, W_NODE, W_FORCE, W_INTERP, W_SPREAD, W_CONVERT, W_REDUCE, W_SC };
enum {
    SLOT_MARK = 0,
    SLOT_NODE = 1,
    SLOT_FORCE = 2,                                       // pass 0
    SLOT_PASS0 = 3,                                       // INTERP(p) = 3 + 2 (p - 1), SPREAD(p) = 4 + 2 (p - 1)
    SLOT_CONVERT = SLOT_PASS0 + 2 * (MAX_IB_PASSES - 1),  // 17
    SLOT_REDUCE = SLOT_CONVERT + 1,
    SLOT_SC = SLOT_REDUCE + 1,
    N_SLOTS = SLOT_SC + 1
};

// Words of the work queue: the ticket counter, the ticket the current
// launch started from, blocks that have left, the abort flag, the number of
// items and of segments of the current table.
enum { WQ_TICKET = 0, WQ_BASE, WQ_EXITS, WQ_ABORT, WQ_ITEMS, WQ_SEGS, WQ_WORDS = 8 };

// A run of items of one kind and environment, in queue order.
struct WorkSeg {
    int begin;       // queue position of the first item
    int count;       // items
    int kind;        // W_*
    int env;
    int slot;        // completion counter the items add to
    int dep_slot;    // counter every item waits for (-1: none) ...
    int dep_count;   // ... until it reaches this count
    int cond_slot;   // SC: counter a block with a stamped tile also waits for
    int cond_count;
    int pass;        // INTERP / SPREAD: direct-forcing pass
    int per_item;    // markers (multiple of 16) or tiles per item
    int pad;
};

constexpr uint32_t FUSED_WAIT_LIMIT = 1u << 22;   // polls before a wait gives up

// Segment holding queue position `item` (the last one with begin <= item).
__device__ __forceinline__ int find_seg(const WorkSeg* __restrict__ segs, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&segs[mid].begin) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Wait (thread 0) until *counter >= target; false if the wait gave up (it
// then records ST_TIMEOUT and sets the abort word, so that the other blocks
// stop too) or the launch was aborted.
__device__ __forceinline__ bool wait_count(const int* counter, int target, int* work, int* status,
                                           uint32_t limit = FUSED_WAIT_LIMIT) {
    if (target <= 0) return true;
    for (uint32_t i = 0;; ++i) {
        if ((int)ld_acquire_gpu(reinterpret_cast<const unsigned*>(counter)) >= target) return true;
        if ((i & 63u) == 63u && __ldcg(work + WQ_ABORT) != 0) return false;
        if (i == limit) {
            atomicOr(status, ST_TIMEOUT);
            atomicExch(work + WQ_ABORT, 1);
            return false;
        }
        __nanosleep(32);
    }
}

// Pointers of a step the IB items use.
struct IbArgs {
    const EnvDev* envs;
    const FrameDev* frames;
    const float* X;
    const float* U;
    const float* dV;
    float* Fm;
    float4* fib;
    uint32_t* stamps;
    float4* nodes;
    float* dF;
    unsigned long long* fibq;
    const float* Nrm;
    int* status;
};

// A MARK, FORCE, INTERP or SPREAD item: markers [k per, (k + 1) per) of
// environment e, one per half-warp at a time.
__device__ __forceinline__ void fused_marker_item(const IbArgs& a, int kind, int e, int k, int per, int pass,
                                               uint32_t stamp) {
    const EnvDev& E = a.envs[e];
    const int h = threadIdx.x & 15;
    const int l_end = min((k + 1) * per, E.n_markers);
    for (int l0 = k * per; l0 < l_end; l0 += MARKERS_PER_ITEM) {   // block-uniform
        const int l = l0 + (threadIdx.x >> 4);
        const bool here = l < l_end;
        const int slot = E.marker_off + l;
        if (kind == W_MARK) {
            if (here) {
                const Stencil Sm = marker_stencil(E, a.X, slot);
                if (Sm.ok) ib_mark(E, Sm, h, stamp, a.stamps);   // invalid markers: reported by FORCE
            }
            continue;
        }
        MarkerRef r;
        r.e = e;
        r.slot = slot;
        r.S.ok = false;
        if (here) r = load_marker_slot<false>(E, e, slot, a.X, a.U, a.dV);
        const bool active = here && r.S.ok;
        ColumnNodes cn;
        if (active) cn = column_nodes(E, r, h);
        if (kind == W_SPREAD) {
            if (active) {
                const float* d = a.dF + 3 * slot;
                const float3 F = make_float3(__ldcg(d), __ldcg(d + 1), __ldcg(d + 2));
                if (a.fibq) spread_force_fixed(E, r, cn, F, a.fibq, a.status);
                else spread_force(E, r, cn, F, a.fib);
            }
            continue;
        }
        if (kind == W_FORCE && here && !r.S.ok && h == 0) {
            a.Fm[3 * slot] = 0.f; a.Fm[3 * slot + 1] = 0.f; a.Fm[3 * slot + 2] = 0.f;
            atomicOr(a.status, ST_BAD_MARKER);
        }
        // every lane takes part in the half-warp shuffles
        const float3 F = interp_force(E, r, cn, active, kind == W_FORCE ? 0 : pass, a.fib, a.fibq, a.nodes, a.Nrm);
        if (!active) continue;
        if (kind == W_FORCE) {
            if (a.fibq) spread_force_fixed(E, r, cn, F, a.fibq, a.status);
            else spread_force(E, r, cn, F, a.fib);
            if (h == 0) { a.Fm[3 * slot] = F.x; a.Fm[3 * slot + 1] = F.y; a.Fm[3 * slot + 2] = F.z; }
        } else if (h == 0) {   // INTERP: accumulate, keep the increment for SPREAD
            float* Fl = a.Fm + 3 * slot;
            Fl[0] = __ldcg(Fl) + F.x; Fl[1] = __ldcg(Fl + 1) + F.y; Fl[2] = __ldcg(Fl + 2) + F.z;
            float* d = a.dF + 3 * slot;
            d[0] = F.x; d[1] = F.y; d[2] = F.z;
        }
    }
}

// A NODE or CONVERT item: the stamped tiles among t = k + K j (j < per) of
// environment e, K the segment's item count; a warp per stamped tile.
template <class S>
__device__ __forceinline__ void fused_tile_item(const IbArgs& a, const typename S::raw* __restrict__ gin, int kind, int e,
                                             int k, int K, int per, uint32_t stamp) {
    const EnvDev& E = a.envs[e];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long ntiles = (E.nslot + 31u) >> 5;
    for (int j0 = 0; j0 < per; j0 += FUSED_THREADS) {   // block-uniform
        const long long t = (long long)k + (long long)K * (j0 + threadIdx.x);
        const bool hit = t < ntiles && __ldcg(a.stamps + E.stamp_off + t) == stamp;
        unsigned hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
            const int src = __ffs(hits) - 1;
            hits &= hits - 1u;
            const int tt = (int)((long long)k + (long long)K * (j0 + warp * 32 + src));
            if (kind == W_NODE) {
                ib_nodes_of<S>(gin, E, a.frames[e], tt, lane, a.nodes);
            } else {
                const uint32_t c = (uint32_t)tt * 32u + (uint32_t)lane;
                if (c < E.nslot) {
                    unsigned long long* q = a.fibq + 3ull * (E.slot_off + c);
                    const unsigned long long qx = __ldcg(q), qy = __ldcg(q + 1), qz = __ldcg(q + 2);
                    a.fib[E.slot_off + c] = make_float4(fixed_to_float(qx), fixed_to_float(qy), fixed_to_float(qz), 0.f);
                    q[0] = 0ull; q[1] = 0ull; q[2] = 0ull;
                }
            }
        }
    }
}

// A REDUCE item: chunk k (256 markers) of every force/torque row of
// environment e, computed as block (e, y, k) of k_reduce computes it.
__device__ __forceinline__ void fused_reduce_item(const IbArgs& a, int e, int k, const int* __restrict__ seg,
                                               const float* __restrict__ seg_ref, Pair32* red_partials, int red_zmax,
                                               Pair32 (*sh)[6]) {
    const EnvDev& E = a.envs[e];
    for (int y = 0; y <= E.nseg; ++y) {
        Pair32 acc[6];
        marker_row_terms(E, e, y, k * FUSED_THREADS + threadIdx.x, a.X, a.Fm, a.dV, seg, seg_ref, acc);
        block_pair_sums(acc, 6, sh, red_partials + ((size_t)(e * RED_ROWS + y) * red_zmax + k) * 6);
    }
}

// Resident blocks per SM the fused kernel is compiled for.  With two cells
// per thread the cell update alone needs the 64 registers that four blocks
// allow, and the IB items inlined beside it would spill at four; three give
// 85 registers.
#ifndef FG_FUSED_MINB_PAIR
#define FG_FUSED_MINB_PAIR 3
#endif
template <bool PAIR>
constexpr int fused_minb() { return PAIR ? FG_FUSED_MINB_PAIR : 4; }

template <class S, bool EQ3, bool PAIR>
__global__ void __launch_bounds__(FUSED_THREADS, fused_minb<PAIR>())
k_step_fused(const typename S::raw* __restrict__ gin, typename S::raw* __restrict__ gout, const IbArgs a,
             const StepState* __restrict__ st, const int* __restrict__ seg, const float* __restrict__ seg_ref,
             Pair32* red_partials, int red_zmax, Pair32* mass_part, const WorkSeg* __restrict__ segs, int* work,
             int* done, int n_envs) {
    // queue state in shared memory (thread 0 writes it between barriers), so
    // that the cell update keeps its registers
    __shared__ int s_item, s_seg, s_go, s_last;
    __shared__ int s_seg_lo, s_seg_hi;   // item range of segment s_seg
    __shared__ int s_dep_seg;            // segment whose dependency is known to be met
    __shared__ int s_ib_env;             // environment whose IB phases are known to be complete
    __shared__ int s_cenv;               // environment whose constants C holds
    __shared__ int s_items, s_segs;
    __shared__ unsigned s_base;
    __shared__ uint32_t s_stamp;
    __shared__ CellConsts C;
    __shared__ float wsum[FUSED_THREADS / 32];
    __shared__ Pair32 sh[FUSED_THREADS / 32][6];
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_base = (unsigned)__ldcg(work + WQ_BASE);
        s_items = __ldcg(work + WQ_ITEMS);
        s_segs = __ldcg(work + WQ_SEGS);
        s_stamp = st->stamp;
        s_item = (int)((unsigned)atomicAdd(work + WQ_TICKET, 1) - s_base);
        s_seg = 0;
        s_seg_lo = s_seg_hi = 0;
        s_dep_seg = s_ib_env = s_cenv = -1;
    }
    __syncthreads();
    while (s_item < s_items) {
        const int item = s_item;
        int nxt = 0;   // thread 0: the next ticket, used at the end of the item
        if (tid == 0) {
            nxt = (int)((unsigned)atomicAdd(work + WQ_TICKET, 1) - s_base);
            if (item < s_seg_lo || item >= s_seg_hi) {
                // tickets only grow: search forward from the last segment
                int si = item < s_seg_lo ? 0 : s_seg;
                while (si + 1 < s_segs && __ldg(&segs[si + 1].begin) <= item) ++si;
                s_seg = si;
                s_seg_lo = __ldg(&segs[si].begin);
                s_seg_hi = s_seg_lo + __ldg(&segs[si].count);
            }
            int go = 1;
            if (s_dep_seg != s_seg) {
                const int ds = __ldg(&segs[s_seg].dep_slot);
                if (ds >= 0)
                    go = wait_count(done + (size_t)__ldg(&segs[s_seg].env) * N_SLOTS + ds,
                                    __ldg(&segs[s_seg].dep_count), work, a.status) ? 1 : 0;
                if (go) s_dep_seg = s_seg;
            }
            s_go = go;
        }
        __syncthreads();
        const WorkSeg& g = segs[s_seg];
        const int kind = __ldg(&g.kind), e = __ldg(&g.env), k = item - s_seg_lo;
        bool ok = s_go != 0;
        if (ok && kind == W_SC) {
            const EnvDev& E = a.envs[e];
            const uint32_t stamp = s_stamp;
            if (s_ib_env != e) {   // block-uniform
                // Until this environment's IB phases are known to be complete,
                // a block with a stamped tile waits for them.
                constexpr int TPB = (PAIR ? 2 : 1) * FUSED_THREADS / 32;
                const int ntiles = (int)((E.nslot + 31u) >> 5);
                const int t = k * TPB + tid;
                const int hit = tid < TPB && t < ntiles && __ldcg(a.stamps + E.stamp_off + t) == stamp;
                const int cs = __ldg(&g.cond_slot), cc = __ldg(&g.cond_count);
                if (__syncthreads_or(hit)) {
                    if (tid == 0) {
                        s_go = wait_count(done + (size_t)e * N_SLOTS + cs, cc, work, a.status);
                        if (s_go) s_ib_env = e;
                    }
                    __syncthreads();
                    ok = s_go != 0;
                } else if (tid == 0 && (cc <= 0 || (int)ld_acquire_gpu(reinterpret_cast<const unsigned*>(
                                                        done + (size_t)e * N_SLOTS + cs)) >= cc)) {
                    s_ib_env = e;   // complete already: later blocks skip the check
                }
            }
            if (ok) {
                if (s_cenv != e) {   // block-uniform
                    __syncthreads();
                    if (tid == 0) {
                        C = load_consts(E, a.frames[e]);
                        s_cenv = e;
                    }
                    __syncthreads();
                }
                const float dr = plain_block_cells<S, EQ3, PAIR, true>(gin, gout, E, C, k, a.fib, a.stamps, stamp);
                const float tsum = block_sum_f32(dr, wsum);
                if (tid == 0) {
                    Pair32 p;
                    p.hi = tsum;
                    mass_part[E.block0 + k] = p;
                }
            }
        } else if (ok && (kind == W_NODE || kind == W_CONVERT)) {
            fused_tile_item<S>(a, gin, kind, e, k, __ldg(&g.count), __ldg(&g.per_item), s_stamp);
        } else if (ok && kind == W_REDUCE) {
            fused_reduce_item(a, e, k, seg, seg_ref, red_partials, red_zmax, sh);
        } else if (ok) {
            fused_marker_item(a, kind, e, k, __ldg(&g.per_item), __ldg(&g.pass), s_stamp);
        }
        // The completion counters order an item's writes before the items
        // that wait for it; nothing waits for the cell blocks, which skip it.
        if (kind != W_SC) __syncthreads();   // block-uniform
        if (tid == 0) {
            // a block that gave up counts its item as not done and takes no
            // further item (the segment is read again: nothing of it stays in
            // registers across the item's work)
            if (ok && kind != W_SC)
                red_add_release_gpu(
                    reinterpret_cast<unsigned*>(done + (size_t)e * N_SLOTS + __ldg(&segs[s_seg].slot)), 1u);
            s_item = ok ? nxt : s_items;
        }
        __syncthreads();
    }
    // the last block to leave resets the counters and the queue for the next
    // launch (every other block has left: none reads them any more)
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(work + WQ_EXITS, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = tid; i < n_envs * N_SLOTS; i += FUSED_THREADS) done[i] = 0;
    if (tid == 0) {
        work[WQ_BASE] = __ldcg(work + WQ_TICKET);
        work[WQ_EXITS] = 0;
        work[WQ_ABORT] = 0;
    }
}

// Failure-detection self test of the work queue's bounded wait: a
// dependency counter that never reaches its target.  out[0] = 1 if the wait
// gave up, out[1] = 1 if it set the abort word.
static __global__ void k_selftest_queue_wait(const int* counter, int* work, uint32_t limit, int* out,
                                             int* status) {
    if (threadIdx.x != 0) return;
    out[0] = wait_count(counter, 1, work, status, limit) ? 0 : 1;
    out[1] = __ldcg(work + WQ_ABORT) != 0 ? 1 : 0;
}

}  // namespace fl
