// aa_kernels.cuh -- stream-collide in place: one population array instead of
// two (the "AA" access pattern, Bailey, Myre, Walsh, Lilja and Saar,
// "Accelerating lattice Boltzmann fluid flow simulations using graphics
// processors", ICPP 2009).  The step computes what k_stream_collide computes
// (arXiv 2206.01683, Sec. III-B and Eq. 3: the same moments, collision,
// forcing and open-face rule, in the same FP32 order, so the populations
// are bit-identical); only where each population is kept changes.
//
// Layout (one array, locations (direction, slot)), in two phases that
// alternate step by step:
//   phase 0 (after an odd step, and initially): (i, y) holds the population
//     that streamed into y, f*_i(y - c_i); where y - c_i lies beyond an open
//     face, (i, y) holds f*_{26-i}(y) instead, the population of y that left
//     the domain (no step reads it; it keeps the state complete).
//   phase 1 (after an even step): (26 - i, x) holds f*_i(x), the
//     post-collision population of x that has not streamed yet.
// An even step (phase 0 -> 1) reads cell p's 27 populations at (i, p) and
// writes f*_i(p) to (26 - i, p): no neighbour access at all.  An odd step
// (phase 1 -> 0) reads f*_i(p - c_i) from (26 - i, p - c_i) and writes f*_i(p)
// to (i, p + c_i).  In both, each location is read and then overwritten by
// the one thread that owns it and by no other, so the update is race-free
// in place.
//
// Cells on the outer layer of an open face take their update from the
// moments of their inward neighbour x_f = x + n alone (the extrapolation
// rule of cell_coeffs).  x_f's moments are read from locations x_f's thread
// overwrites, so the thread of x_f ("the server") also updates the boundary
// cells it serves -- up to 7 at a corner -- from the moments it already has,
// and writes their outputs: (26 - i, x) in an even step; (i, x + c_i) in an
// odd step, or (26 - i, x) where x + c_i lies beyond an open face (that
// location belongs to nobody in an odd step).  The boundary cells' own
// threads do nothing.  Markers keep their stencils off the outer layer, so
// boundary cells carry no IB force.
#pragma once

#include "step_kernels.cuh"

namespace fl {

// Faces of a cell's position: bit 0 (1) when x is the first (last) cell of
// an open x axis, bits 2, 3 for y, bits 4, 5 for z.
__device__ __forceinline__ unsigned open_bits(const EnvDev& E, int x, int y, int z) {
    const int p[3] = {x, y, z};
    unsigned b = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (!E.per[a]) {
            if (p[a] == 0) b |= 1u << (2 * a);
            if (p[a] == E.n[a] - 1) b |= 2u << (2 * a);
        }
    return b;
}

// Boundary neighbours a cell serves: bit 0 (1) when x - 1 (x + 1) is the
// outer layer of an open x axis, bits 2, 3 for y, bits 4, 5 for z.
__device__ __forceinline__ unsigned serve_bits(const EnvDev& E, int x, int y, int z) {
    const int p[3] = {x, y, z};
    unsigned b = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (!E.per[a]) {
            if (p[a] == 1) b |= 1u << (2 * a);
            if (p[a] == E.n[a] - 2) b |= 2u << (2 * a);
        }
    return b;
}

// The faces (open_bits) that velocity i crosses when it leaves a cell on them.
__host__ __device__ constexpr unsigned leave_mask(int i) {
    return (cx(i) == -1 ? 1u : 0u) | (cx(i) == 1 ? 2u : 0u) | (cy(i) == -1 ? 4u : 0u) | (cy(i) == 1 ? 8u : 0u) |
           (cz(i) == -1 ? 16u : 0u) | (cz(i) == 1 ? 32u : 0u);
}

// A step reads and writes the same 27 locations of a cell, so the compiler
// would keep the 27 addresses of the loads live until the stores (54
// registers).  The stores take their address inputs through opaque()
// instead, which makes them recompute the addresses (one or two integer
// operations each).
template <class T>
__device__ __forceinline__ T* opaque(T* p) {
    asm volatile("" : "+l"(p));
    return p;
}
__device__ __forceinline__ uint32_t opaque(uint32_t v) {
    asm volatile("" : "+r"(v));
    return v;
}
__device__ __forceinline__ PullOffsets opaque(PullOffsets o) {
    asm volatile("" : "+r"(o.xm), "+r"(o.xp), "+r"(o.ym), "+r"(o.yp), "+r"(o.zm), "+r"(o.zp));
    return o;
}

// Store the 27 outputs of one cell (slot s, coefficients h) where a step of
// phase K puts them: K = 0: (26 - i, s); K = 1: (i, s + c_i) with the cell's
// pull offsets o (s + c_i = s - c_{26-i}), or (26 - i, s) where the cell lies
// on an open face that i crosses (bits `open`; OPEN = false: none).
template <class S, bool EQ3, int K, bool OPEN>
__device__ __forceinline__ void aa_emit_cell(const Herm& h, typename S::raw* G, uint32_t nslot, uint32_t s,
                                             const PullOffsets& o, unsigned open) {
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        float v[3];
        line_values<EQ3>(h, l, v[1], v[2], v[0]);   // v[k]: cx = k - 1, i = 3 l + k
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int i = 3 * l + k;
            int dir = Q - 1 - i, idx = (int)s;
            if (K == 1 && !(OPEN && (open & leave_mask(i)))) {
                dir = i;
                idx = (int)s + pull_off(o, Q - 1 - i);
            }
            if (FG_IN_RANGE(DBG_STORE, idx, nslot)) S::emit(G + (size_t)dir * nslot + (uint32_t)idx, v[k], i);
        }
    }
}

// The outputs of two neighbouring cells a (slot s, even) and b (s + 1) of
// one row, as aa_emit_cell places them; pairs of slots that stay adjacent
// and aligned (every output of an even step; velocities with cx = 0 in an
// odd step, whose y/z faces are the same for both cells) are stored with
// one access.
template <class S, bool EQ3, int K, bool OPEN>
__device__ __forceinline__ void aa_emit_pair(const Herm& ha, const Herm& hb, typename S::raw* G, uint32_t nslot,
                                             uint32_t s, const PullOffsets& oa, const PullOffsets& ob,
                                             unsigned open_a, unsigned open_b) {
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        float va[3], vb[3];
        line_values<EQ3>(ha, l, va[1], va[2], va[0]);
        line_values<EQ3>(hb, l, vb[1], vb[2], vb[0]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int i = 3 * l + k;
            if (K == 0 || cx(i) == 0) {
                int dir = Q - 1 - i, idx = (int)s;
                if (K == 1 && !(OPEN && (open_a & leave_mask(i)))) {
                    dir = i;
                    idx = (int)s + pull_off(oa, Q - 1 - i);
                }
                if (FG_IN_RANGE(DBG_STORE, idx + 1, nslot))
                    S::emit2(G + (size_t)dir * nslot + (uint32_t)idx, va[k], vb[k], i);
            } else {
                int dir = Q - 1 - i, idx = (int)s;
                if (!(OPEN && (open_a & leave_mask(i)))) {
                    dir = i;
                    idx = (int)s + pull_off(oa, Q - 1 - i);
                }
                if (FG_IN_RANGE(DBG_STORE, idx, nslot)) S::emit(G + (size_t)dir * nslot + (uint32_t)idx, va[k], i);
                dir = Q - 1 - i;
                idx = (int)s + 1;
                if (!(OPEN && (open_b & leave_mask(i)))) {
                    dir = i;
                    idx = (int)s + 1 + pull_off(ob, Q - 1 - i);
                }
                if (FG_IN_RANGE(DBG_STORE, idx, nslot)) S::emit(G + (size_t)dir * nslot + (uint32_t)idx, vb[k], i);
            }
        }
    }
}

// ------------------------------------------------------ one cell per thread

// The boundary cells cell (x, y, z) at slot c (moments m) serves (bits sv of
// serve_bits): the neighbour at offset d = (dx, dy, dz) with every nonzero
// component a served face has inward normal -d.  Returns their rho_out - 1.
template <class S, bool EQ3, int K>
__device__ __noinline__ float aa_serve_cells(const CellConsts& C, const Moments& m, typename S::raw* G,
                                                const EnvDev& E, int x, int y, int z, uint32_t c, unsigned sv) {
    float drout = 0.0f;
#pragma unroll 1
    for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        if (k == 13) continue;
        if ((dx == -1 && !(sv & 1u)) || (dx == 1 && !(sv & 2u))) continue;
        if ((dy == -1 && !(sv & 4u)) || (dy == 1 && !(sv & 8u))) continue;
        if ((dz == -1 && !(sv & 16u)) || (dz == 1 && !(sv & 32u))) continue;
        const int bx = x + dx, by = y + dy, bz = z + dz;
        const uint32_t bs = (uint32_t)((int)c + dx + (dy + dz * E.n[1]) * E.P);
        const Herm h = cell_coeffs<S, EQ3>(C, m, bx, by, bz, -dx, -dy, -dz, 0.0f, 0.0f, 0.0f);
        aa_emit_cell<S, EQ3, K, true>(h, G, E.nslot, bs, pull_offsets(E, bx, by, bz), open_bits(E, bx, by, bz));
        drout += h.drout;
    }
    return drout;
}

// Cell b * K1_THREADS + threadIdx.x of environment E (G: its populations)
// and the boundary cells it serves; returns the sum of rho_out - 1.
template <class S, bool EQ3, int K>
__device__ __forceinline__ float aa_block_cell(typename S::raw* G, const EnvDev& E, const CellConsts& C, int b,
                                               float4* __restrict__ fib, const uint32_t* __restrict__ stamps,
                                               uint32_t stamp) {
    const uint32_t c = (uint32_t)b * K1_THREADS + threadIdx.x;
    if (c >= E.nslot) return 0.0f;
    const uint32_t row = fdiv(c, E.div_P);
    const int x = (int)(c - row * (uint32_t)E.P);
    if (x >= E.n[0]) return 0.0f;
    const uint32_t zz = fdiv(row, E.div_ny);
    const int y = (int)(row - zz * (uint32_t)E.n[1]);
    const int z = (int)zz;
    if (open_bits(E, x, y, z)) return 0.0f;   // updated by the cell it takes its moments from
    float fx, fy, fz;
    take_ib_force(E, fib, stamps, stamp, c, fx, fy, fz);
    const PullOffsets o = pull_offsets(E, x, y, z);
    const Moments m = layout_moments<S, true, K == 0 ? LAYOUT_AA0 : LAYOUT_AA1, false>(G, E.nslot, c, o);
    const Herm h = cell_coeffs<S, EQ3>(C, m, x, y, z, 0, 0, 0, fx, fy, fz);
    aa_emit_cell<S, EQ3, K, false>(h, opaque(G), opaque(E.nslot), opaque(c), opaque(o), 0u);
    float drout = h.drout;
    const unsigned sv = serve_bits(E, x, y, z);
    if (sv) drout += aa_serve_cells<S, EQ3, K>(C, m, G, E, x, y, z, c, sv);
    return drout;
}

// ------------------------------------------------------ two cells per thread

// The boundary rows that the row of pair (x, x + 1) at (y, z) serves (bits
// sv & 0x3C of serve_bits): the pair at (y + dy, z + dz) takes the moments
// sa, sb the pair's own cells took (its cells' inward neighbours lie in this
// row).  a_open / b_open: x or x + 1 on an open x face.
template <class S, bool EQ3, int K>
__device__ __noinline__ float aa_serve_rows(const CellConsts& C, const Moments& sa, const Moments& sb,
                                               typename S::raw* G, const EnvDev& E, int x, int y, int z, uint32_t c,
                                               bool a_open, bool b_open, unsigned sv) {
    float drout = 0.0f;
#pragma unroll 1
    for (int k = 0; k < 9; ++k) {
        const int dy = k % 3 - 1, dz = k / 3 - 1;
        if (k == 4) continue;
        if ((dy == -1 && !(sv & 4u)) || (dy == 1 && !(sv & 8u))) continue;
        if ((dz == -1 && !(sv & 16u)) || (dz == 1 && !(sv & 32u))) continue;
        const int by = y + dy, bz = z + dz;
        const uint32_t bs = (uint32_t)((int)c + (dy + dz * E.n[1]) * E.P);
        const Herm ha = cell_coeffs<S, EQ3>(C, sa, x, by, bz, a_open ? 1 : 0, -dy, -dz, 0.0f, 0.0f, 0.0f);
        const Herm hb = cell_coeffs<S, EQ3>(C, sb, x + 1, by, bz, b_open ? -1 : 0, -dy, -dz, 0.0f, 0.0f, 0.0f);
        aa_emit_pair<S, EQ3, K, true>(ha, hb, G, E.nslot, bs, pull_offsets(E, x, by, bz),
                                      pull_offsets(E, x + 1, by, bz), open_bits(E, x, by, bz),
                                      open_bits(E, x + 1, by, bz));
        drout += ha.drout + hb.drout;
    }
    return drout;
}

// Cells x (even) and x + 1 of one row (every row length even, so both are
// real cells) and the boundary cells they serve.  An open x face puts a
// boundary cell in the first or last pair of a row, served by its partner.
template <class S, bool EQ3, int K>
__device__ __forceinline__ float aa_block_pair(typename S::raw* G, const EnvDev& E, const CellConsts& C, int b,
                                               float4* __restrict__ fib, const uint32_t* __restrict__ stamps,
                                               uint32_t stamp) {
    const uint32_t c = ((uint32_t)b * K1_THREADS + threadIdx.x) * 2u;
    if (c >= E.nslot) return 0.0f;
    const uint32_t row = fdiv(c, E.div_P);
    const int x = (int)(c - row * (uint32_t)E.P);
    if (x >= E.n[0]) return 0.0f;
    const uint32_t zz = fdiv(row, E.div_ny);
    const int y = (int)(row - zz * (uint32_t)E.n[1]);
    const int z = (int)zz;
    if (open_bits(E, x, y, z) & 0x3Cu) return 0.0f;   // a boundary row: updated by the row inward
    const bool a_open = !E.per[0] && x == 0;
    const bool b_open = !E.per[0] && x + 1 == E.n[0] - 1;
    float fa[3] = {0.0f, 0.0f, 0.0f}, fb[3] = {0.0f, 0.0f, 0.0f};
    if (!a_open) take_ib_force(E, fib, stamps, stamp, c, fa[0], fa[1], fa[2]);
    if (!b_open) take_ib_force(E, fib, stamps, stamp, c + 1, fb[0], fb[1], fb[2]);
    const PullOffsets oa = pull_offsets(E, x, y, z), ob = pull_offsets(E, x + 1, y, z);
    Moments ma = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Moments mb = ma;
    if constexpr (K == 0) {
        // the pair's own slots: one aligned access per velocity
        float ga[Q], gb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float2 v = S::load2_rw(G + (size_t)i * E.nslot + c, i);
            ga[i] = v.x;
            gb[i] = v.y;
        }
        accumulate<true>(ma, ga);
        accumulate<true>(mb, gb);
    } else {
        if (!a_open) ma = layout_moments<S, true, LAYOUT_AA1, false>(G, E.nslot, c, oa);
        if (!b_open) mb = layout_moments<S, true, LAYOUT_AA1, false>(G, E.nslot, c + 1, ob);
    }
    const Moments& sa = a_open ? mb : ma;   // the moments each cell's update takes
    const Moments& sb = b_open ? ma : mb;
    const Herm ha = cell_coeffs<S, EQ3>(C, sa, x, y, z, a_open ? 1 : 0, 0, 0, fa[0], fa[1], fa[2]);
    const Herm hb = cell_coeffs<S, EQ3>(C, sb, x + 1, y, z, b_open ? -1 : 0, 0, 0, fb[0], fb[1], fb[2]);
    if (a_open || b_open)
        aa_emit_pair<S, EQ3, K, true>(ha, hb, opaque(G), opaque(E.nslot), opaque(c), opaque(oa), opaque(ob),
                                      a_open ? 1u : 0u, b_open ? 2u : 0u);
    else
        aa_emit_pair<S, EQ3, K, false>(ha, hb, opaque(G), opaque(E.nslot), opaque(c), opaque(oa), opaque(ob), 0u,
                                       0u);
    float drout = ha.drout + hb.drout;
    const unsigned sv = serve_bits(E, x, y, z) & 0x3Cu;
    if (sv) drout += aa_serve_rows<S, EQ3, K>(C, sa, sb, G, E, x, y, z, c, a_open, b_open, sv);
    return drout;
}

// ------------------------------------------------------------- the kernel


// One step in place over every environment: phase K = 0 (even step) or 1
// (odd step), the blocks and mass partials of the plain kernel.
template <class S, bool EQ3, bool PAIR, int K>
__global__ void __launch_bounds__(K1_THREADS)
k_stream_collide_aa(typename S::raw* g, const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames,
                    int n_envs, float4* __restrict__ fib, const uint32_t* __restrict__ stamps,
                    const StepState* __restrict__ st, Pair32* __restrict__ mass_part) {
    __shared__ float wsum[K1_THREADS / 32];
    __shared__ CellConsts C;
    const uint32_t stamp = st->stamp;
    const int b = blockIdx.x;
    const int e = n_envs > 1 ? env_of<&EnvDev::block0>(envs, n_envs, b) : 0;
    const EnvDev& E = envs[e];
    if (threadIdx.x == 0) C = load_consts(E, frames[e]);
    __syncthreads();
    allow_dependents();
    typename S::raw* G = g + E.pop_off;
    const float drout = PAIR ? aa_block_pair<S, EQ3, K>(G, E, C, b - E.block0, fib, stamps, stamp)
                             : aa_block_cell<S, EQ3, K>(G, E, C, b - E.block0, fib, stamps, stamp);
    const float t = block_sum_f32(drout, wsum);
    if (threadIdx.x == 0) {
        Pair32 p;
        p.hi = t;
        mass_part[b] = p;
    }
}

// ------------------------------------------------ state outside the step

// Raw copy of one environment's state between the layout `aa` of G and the
// two-buffer layout of buf ([27][nslot], the state-buffer format); padding
// slots of buf are zeroed on the way out and ignored on the way in.
template <class S>
__global__ void k_aa_state(typename S::raw* __restrict__ G, const EnvDev* __restrict__ envs, int e, int aa,
                           typename S::raw* __restrict__ buf, int to_buf) {
    const EnvDev& E = envs[e];
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E.nslot) return;
    const uint32_t row = s / (uint32_t)E.P;
    const int x = (int)(s - row * (uint32_t)E.P);
    const int y = (int)(row % (uint32_t)E.n[1]), z = (int)(row / (uint32_t)E.n[1]);
    typename S::raw* Ge = G + E.pop_off;
    for (int i = 0; i < Q; ++i) {
        if (x >= E.n[0]) {
            if (to_buf) buf[(size_t)i * E.nslot + s] = S::encode(0.0f, i);
            continue;
        }
        int dir;
        const uint32_t loc = post_loc(E, aa, i, x, y, z, s, &dir);
        if (!FG_IN_RANGE(DBG_STORE, loc, E.nslot)) continue;
        if (to_buf) buf[(size_t)i * E.nslot + s] = Ge[(size_t)dir * E.nslot + loc];
        else Ge[(size_t)dir * E.nslot + loc] = buf[(size_t)i * E.nslot + s];
    }
}

}  // namespace fl
