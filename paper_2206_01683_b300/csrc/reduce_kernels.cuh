// reduce_kernels.cuh -- the reductions that end a step (arXiv 2206.01683:
// the body force and torque, tau_ext of Eq. 1, per segment and in total; the
// mass; a NaN watchdog), in compensated FP32 pairs evaluated in FP64.
#pragma once

#include "step_kernels.cuh"
#include "marker_src.cuh"

namespace fl {

// Sum a pair over the block: pair trees inside each warp, then warp 0
// combines the warp totals the same way; the final pair is evaluated in FP64.
// Fixed order, so the result is deterministic; valid in thread 0.
__device__ __forceinline__ double block_sum(Pair32 v, Pair32* sh) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        Pair32 o;
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, k);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, k);
        v.add(o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        Pair32 u;
        if (lane < nw) u = sh[lane];
#pragma unroll
        for (int k = 16; k >= 1; k >>= 1) {
            Pair32 o;
            o.hi = __shfl_xor_sync(0xffffffffu, u.hi, k);
            o.lo = __shfl_xor_sync(0xffffffffu, u.lo, k);
            u.add(o);
        }
        t = (double)u.hi + (double)u.lo;
    }
    return t;
}

constexpr int MASS_PER_THREAD = 8;
constexpr int RED_ROWS = MAX_SEG + 2;   // force/torque rows 0..MAX_SEG, then the mass

// Terms of marker l (counted from environment e's first marker) in
// force/torque row y (y < nseg: segment y, its torque about seg_ref[e][y];
// y == nseg: every marker, torque about the environment's ref): force on the
// body -F_l dV_l and torque (X_l - p) x (-F_l dV_l), added to acc.  Reads
// through L2 (the marker forces may come from another block of the same
// launch).
__device__ __forceinline__ void marker_row_terms(const EnvDev& E, int e, int y, int l, const float* __restrict__ X,
                                                 const float* __restrict__ Fm, const float* __restrict__ dV,
                                                 const int* __restrict__ seg, const float* __restrict__ seg_ref,
                                                 Pair32 (&acc)[6]) {
    const int ns = E.nseg;
    if (l >= E.n_markers) return;
    const int q = E.marker_off + l;
    if (y != ns && __ldcg(seg + q) != y) return;
    const float v = -__ldcg(dV + q);
    const float Fx = __ldcg(Fm + 3 * q) * v, Fy = __ldcg(Fm + 3 * q + 1) * v, Fz = __ldcg(Fm + 3 * q + 2) * v;
    // segment rows about the segment's point, the total row about ref
    const float* rp = seg_ref + ((size_t)e * MAX_SEG + (y < ns ? y : 0)) * 3;
    const float px = y < ns ? __ldcg(rp) : (float)E.ref[0], py = y < ns ? __ldcg(rp + 1) : (float)E.ref[1],
                pz = y < ns ? __ldcg(rp + 2) : (float)E.ref[2];
    const float rx = __ldcg(X + 3 * q) - px, ry = __ldcg(X + 3 * q + 1) - py, rz = __ldcg(X + 3 * q + 2) - pz;
    acc[0].add(Fx); acc[1].add(Fy); acc[2].add(Fz);
    acc[3].add(ry * Fz - rz * Fy);
    acc[4].add(rz * Fx - rx * Fz);
    acc[5].add(rx * Fy - ry * Fx);
}

// Sum components c < ncomp of acc over a block of RED_THREADS threads (a
// shuffle tree per component inside each warp, then the warp totals in warp
// order: a fixed order, so the result is deterministic) and store them to
// out[c] (threads c < ncomp, followed by a fence).  Called by every thread.
__device__ __forceinline__ void block_pair_sums(Pair32 (&acc)[6], int ncomp, Pair32 (*sh)[6], Pair32* out) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    constexpr int NW = RED_THREADS / 32;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        if (c < ncomp) {
#pragma unroll
            for (int k = 16; k >= 1; k >>= 1) {
                Pair32 o;
                o.hi = __shfl_xor_sync(0xffffffffu, acc[c].hi, k);
                o.lo = __shfl_xor_sync(0xffffffffu, acc[c].lo, k);
                acc[c].add(o);
            }
            if (lane == 0) sh[w][c] = acc[c];
        }
    }
    __syncthreads();
    if (tid < ncomp) {
        Pair32 t;
        for (int i = 0; i < NW; ++i) t.add(sh[i][tid]);
        out[tid] = t;
        __threadfence();
    }
    __syncthreads();
}

// Grid (n_envs, rows, chunks), rows and chunks those the environments use
// (reduce_grid).  Block (e, y, z) sums chunk z of row y of environment e:
// y <= nseg is force/torque row y (segment y, its torque about
// seg_ref[e][y]; y == nseg is the total over all markers, its torque about
// the environment's ref), one marker per thread; the grid's last row is the
// mass (row RED_ROWS - 1 of the partials), MASS_PER_THREAD partials per
// thread.  Force on the body
// F = -sum F_l dV_l, torque T = -sum (X_l - ref) x F_l dV_l, mass = ncell +
// sum (rho - 1).  Chunk sums are compensated FP32 pairs (all components of a
// block reduced together: one shuffle tree per component, then the warp
// totals in warp order).  One counter per environment counts its blocks; the
// last one adds, for every row and component, the chunk pairs in chunk order
// (a warp per component), so the result does not depend on which block
// finished last.  Results stay compensated FP32 pairs on the device (ft, the
// mass without the cell count, the history row); the host evaluates hi + lo
// in FP64 when it reads them (FP64 arithmetic is slow on this part).  The
// force/torque rows are also written to host_ft and, by the last environment
// to finish (which advances the step state), the status word to host_status:
// pinned host memory mapped into the device's address space, so a coupled
// step reads them back with no copy (either may be NULL).  markers_pre = 1:
// the force/torque chunk sums are already in `partials` (the fused step
// kernel wrote them, with the same chunks and order); the grid is then
// (n_envs, 1, chunks) and only the mass is summed before the combine.  The
// last block also clears the step's posted marker source (msrc, may be NULL).
static __global__ void __launch_bounds__(RED_THREADS)
k_reduce(const EnvDev* __restrict__ envs, const float* __restrict__ X, const float* __restrict__ Fm,
         const float* __restrict__ dV, const int* __restrict__ seg, const float* __restrict__ seg_ref,
         const Pair32* __restrict__ mass_part,
         Pair32* __restrict__ partials, int* __restrict__ counters, int n_envs, int zmax,
         Pair32* __restrict__ ft, Pair32* __restrict__ mass, Pair32* __restrict__ hist, int hist_cap,
         StepState* __restrict__ st, int* __restrict__ status, Pair32* __restrict__ host_ft,
         int* __restrict__ host_status, long long* __restrict__ host_seq, int markers_pre,
         MarkerSrc* __restrict__ msrc) {
    constexpr int NW = RED_THREADS / 32;
    __shared__ Pair32 sh[NW][6];
    __shared__ int is_last;
    // the grid's last row is the mass (row RED_ROWS - 1 of the partials);
    // the rows before it are force/torque rows 0, 1, ... (markers_pre: the
    // grid has the mass row only)
    const int yg = (int)blockIdx.y;
    const int e = blockIdx.x, y = yg == (int)gridDim.y - 1 ? RED_ROWS - 1 : yg, z = blockIdx.z, tid = threadIdx.x;
    const int w = tid >> 5, lane = tid & 31;
    const EnvDev& E = envs[e];
    const int ns = E.nseg;
    const int nch_f = max(1, (E.n_markers + RED_THREADS - 1) / RED_THREADS);
    const int nch_m = max(1, (E.nparts + RED_THREADS * MASS_PER_THREAD - 1) / (RED_THREADS * MASS_PER_THREAD));
    const bool is_mass = y == RED_ROWS - 1;
    if (is_mass ? z >= nch_m : (y > ns || z >= nch_f)) return;
    Pair32 acc[6];
    // The marker forces come from the IB kernel, which completed before the
    // stream-collide kernel started, so these sums may run while the
    // stream-collide kernel's last blocks finish (reads through L2).
    if (!is_mass) marker_row_terms(E, e, y, z * RED_THREADS + tid, X, Fm, dV, seg, seg_ref, acc);
    // Everything below reads the stream-collide kernel's mass sums or writes
    // what the step's kernels read (the step state), so it waits for that
    // kernel when launched as its programmatic dependent.
    wait_prerequisites();
    if (is_mass) {
        const int per_block = RED_THREADS * MASS_PER_THREAD;
        Pair32 v[MASS_PER_THREAD];
#pragma unroll
        for (int k = 0; k < MASS_PER_THREAD; ++k) {
            const int i = z * per_block + k * RED_THREADS + tid;
            if (i < E.nparts) {
                v[k].hi = __ldcg(&mass_part[E.part0 + i].hi);
                v[k].lo = __ldcg(&mass_part[E.part0 + i].lo);
            }
        }
#pragma unroll
        for (int k = 0; k < MASS_PER_THREAD; ++k) acc[0].add(v[k]);
    }
    const int ncomp = is_mass ? 1 : 6;
    Pair32* slot = partials + ((size_t)(e * RED_ROWS + y) * zmax) * 6;
    if (FG_IN_RANGE(DBG_REDUCE, z, zmax)) block_pair_sums(acc, ncomp, sh, slot + (size_t)z * 6);
    if (tid == 0) {
        is_last = atomicAdd(counters + e, 1) == (markers_pre ? 0 : (ns + 1) * nch_f) + nch_m - 1;
        if (is_last) __threadfence();
    }
    __syncthreads();
    if (!is_last) return;   // the partials are read through L2 (ld.global.cg) below
    // last block of environment e: item k < 6 (ns + 1) is force/torque
    // component k % 6 of row k / 6, item 6 (ns + 1) the mass.  A warp per
    // item; each warp takes ILP items at a time so that their loads are in
    // flight together.
    constexpr int ILP = 8;
    const int items = 6 * (ns + 1) + 1;
    // chunks of the force/torque rows to add: the fused step kernel writes
    // none for an environment without markers (its rows are zero; what the
    // scratch holds there is from another step or environment)
    const int nch_rows = markers_pre && E.n_markers == 0 ? 0 : nch_f;
    for (int k0 = w; k0 < items; k0 += ILP * NW) {
        Pair32 t[ILP];
        const Pair32* src[ILP];
        int nch[ILP], cc[ILP];
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
            const int k = k0 + j * NW;
            const bool m_item = k == items - 1;
            const int yy = m_item ? RED_ROWS - 1 : k / 6;
            cc[j] = m_item ? 0 : k % 6;
            nch[j] = k >= items ? 0 : (m_item ? nch_m : nch_rows);
            src[j] = partials + ((size_t)(e * RED_ROWS + yy) * zmax) * 6;
        }
        const int nmax = max(nch_f, nch_m);
        for (int zz = lane; zz < nmax; zz += 32) {
            Pair32 p[ILP];
#pragma unroll
            for (int j = 0; j < ILP; ++j) {
                if (zz < nch[j]) {
                    p[j].hi = __ldcg(&src[j][(size_t)zz * 6 + cc[j]].hi);
                    p[j].lo = __ldcg(&src[j][(size_t)zz * 6 + cc[j]].lo);
                }
            }
#pragma unroll
            for (int j = 0; j < ILP; ++j) t[j].add(p[j]);
        }
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                Pair32 o;
                o.hi = __shfl_xor_sync(0xffffffffu, t[j].hi, s);
                o.lo = __shfl_xor_sync(0xffffffffu, t[j].lo, s);
                t[j].add(o);
            }
            const int k = k0 + j * NW;
            if (lane == 0 && k < items) {
                if (k == items - 1) {
                    mass[e] = t[j];
                    // mass-drift watchdog (the reference and tolerance are
                    // set by fg_watch_mass)
                    if (E.mass_tol > 0.0f && !(fabsf((t[j].hi - E.mass_ref) + t[j].lo) <= E.mass_tol))
                        atomicOr(status, ST_MASS_DRIFT);
                } else {
                    ft[(size_t)e * FT_ROW + k] = t[j];
                    if (host_ft) host_ft[(size_t)e * FT_ROW + k] = t[j];   // host-mapped copy
                }
                if (!(isfinite(t[j].hi) && isfinite(t[j].lo))) atomicOr(status, ST_NUMERIC);
            }
        }
    }
    __syncthreads();
    if (hist_cap > 0) {
        Pair32* h = hist + ((size_t)e * hist_cap + (size_t)(st->step % hist_cap)) * HIST_ROW;
        for (int k = tid; k < items; k += RED_THREADS)
            h[k == items - 1 ? FT_ROW : k] = k == items - 1 ? mass[e] : ft[(size_t)e * FT_ROW + k];
    }
    if (tid != 0) return;
    counters[e] = 0;   // ready for the next step
    if (n_envs > 1) {
        // the host-mapped rows of this environment are ordered before the
        // sequence word the last environment writes
        if (host_ft) __threadfence_system();
        else __threadfence();
        if (atomicAdd(&st->envs_done, 1) != n_envs - 1) return;
        st->envs_done = 0;
    }
    st->step += 1;
    st->stamp = st->stamp == 0xffffffffu ? 1u : st->stamp + 1u;
    // a marker source posted for this step has been read (by the IB kernel,
    // which completed before the stream-collide kernel began)
    if (msrc) msrc->valid = 0;
    // the step's status word (every kernel of the step, and every
    // environment's combine, has set its bits by now) to the host-mapped copy
    if (host_status) *host_status = atomicOr(status, 0);
    // then the step number: a host waiting for this step's rows may poll it
    if (host_seq) {
        __threadfence_system();
        *reinterpret_cast<volatile long long*>(host_seq) = st->step;
    }
}

// Momentum and angular momentum of the fluid inside a sphere (centre c,
// radius R) in the stored state g of environment E: P = sum alpha j,
// L = sum alpha (x - c) x j, j = sum_i c_i g_i (the rest populations w_i
// carry no momentum), alpha = clamp(R + 1/2 - |x - c|, 0, 1), x - c the
// minimal image on periodic axes (population i where post_loc keeps it under
// layout aa).  The free-body coupling needs it every step
// (the inner fluid's momentum change, Kempe & Froehlich 2012).  Block `blk`
// of `nblk` walks its share of the cells of the sphere's bounding box
// [lo, lo + ext) and writes seven compensated pairs (P, L, sum alpha) to
// out[0..6]; the blocks' pairs are added in block order.  Called by every
// thread of a block of RED_THREADS.
template <class S>
__device__ __forceinline__ void region_block_sums(const typename S::raw* __restrict__ g, const EnvDev& E,
                                                  const float (&c)[3], float R, const int (&lo)[3],
                                                  const int (&ext)[3], int blk, int nblk, Pair32 (*sh)[7],
                                                  Pair32* __restrict__ out, int aa) {
    const typename S::raw* G = g + E.pop_off;
    Pair32 acc[7];
    const long long n_box = (long long)ext[0] * ext[1] * ext[2];
    for (long long k = blk * (long long)blockDim.x + threadIdx.x; k < n_box; k += (long long)nblk * blockDim.x) {
        int p[3] = {lo[0] + (int)(k % ext[0]), lo[1] + (int)((k / ext[0]) % ext[1]),
                    lo[2] + (int)(k / ((long long)ext[0] * ext[1]))};
        float r[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int n = E.n[a];
            r[a] = (float)p[a] - c[a];
            if (E.per[a]) {
                p[a] = ((p[a] % n) + n) % n;
                r[a] -= (float)n * floorf(r[a] / (float)n + 0.5f);
            } else if (p[a] < 0 || p[a] >= n) {
                inside = false;
            }
        }
        if (!inside) continue;
        const float al = fminf(R + 0.5f - sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), 1.0f);
        if (al <= 0.0f) continue;
        const uint32_t slot = (uint32_t)p[0] + (uint32_t)E.P * ((uint32_t)p[1] + (uint32_t)E.n[1] * (uint32_t)p[2]);
        if (!FG_IN_RANGE(DBG_REGION, slot, E.nslot)) continue;
        float j[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int dir;
            const uint32_t loc = post_loc(E, aa, i, p[0], p[1], p[2], slot, &dir);
            if (!FG_IN_RANGE(DBG_REGION, loc, E.nslot)) continue;
            const float v = S::decode(G[(size_t)dir * E.nslot + loc], i);
            j[0] += cx(i) * v;
            j[1] += cy(i) * v;
            j[2] += cz(i) * v;
        }
        acc[0].add(al * j[0]); acc[1].add(al * j[1]); acc[2].add(al * j[2]);
        acc[3].add(al * (r[1] * j[2] - r[2] * j[1]));
        acc[4].add(al * (r[2] * j[0] - r[0] * j[2]));
        acc[5].add(al * (r[0] * j[1] - r[1] * j[0]));
        acc[6].add(al);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            Pair32 o;
            o.hi = __shfl_xor_sync(0xffffffffu, acc[q].hi, s);
            o.lo = __shfl_xor_sync(0xffffffffu, acc[q].lo, s);
            acc[q].add(o);
        }
        if (lane == 0) sh[w][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        Pair32 t;
        for (int i = 0; i < RED_THREADS / 32; ++i) t.add(sh[i][threadIdx.x]);
        out[threadIdx.x] = t;
    }
}

// The sphere's bounding box in the cells of E: [lo, lo + ext) per axis,
// clamped to the domain along an open axis, each cell once along a periodic
// one (the box fg_region_momentum and the device-resident sphere use).
__host__ __device__ inline void sphere_box(const EnvDev& E, const double (&c)[3], double R, int (&lo)[3],
                                           int (&ext)[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int)floor(c[a] - R - 1.0);
        ext[a] = (int)ceil(c[a] + R + 1.0) - lo[a] + 1;
        if (!E.per[a]) {
            const int hi = min(lo[a] + ext[a], E.n[a]);
            lo[a] = max(lo[a], 0);
            ext[a] = max(hi - lo[a], 0);
        } else if (ext[a] > E.n[a]) {
            lo[a] = 0;
            ext[a] = E.n[a];
        }
    }
}

// fg_region_momentum: block b's pairs to part[b][0..6], the host adds them.
template <class S>
__global__ void __launch_bounds__(RED_THREADS)
k_region_momentum(const typename S::raw* __restrict__ g, const EnvDev* __restrict__ envs, int e, float cx_,
                  float cy_, float cz_, float R, int lo_x, int lo_y, int lo_z, int ext_x, int ext_y, int ext_z,
                  Pair32* __restrict__ part, int aa) {
    __shared__ Pair32 sh[RED_THREADS / 32][7];
    const float c[3] = {cx_, cy_, cz_};
    const int lo[3] = {lo_x, lo_y, lo_z}, ext[3] = {ext_x, ext_y, ext_z};
    region_block_sums<S>(g, envs[e], c, R, lo, ext, blockIdx.x, gridDim.x, sh, part + (size_t)blockIdx.x * 7, aa);
}

}  // namespace fl
