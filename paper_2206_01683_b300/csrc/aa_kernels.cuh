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
// rule of cell_coeffs), and x_f's thread overwrites the locations those
// moments are read from.  So a small kernel, k_aa_boundary, updates the
// boundary cells first (one per thread, reading x_f's arriving populations
// before anything overwrites them) and writes their outputs: (26 - i, x) in
// an even step; (i, x + c_i) in an odd step, or (26 - i, x) where x + c_i
// lies beyond an open face (that location belongs to nobody in an odd
// step).  Then the stream-collide kernel updates every other cell.  None of
// the locations the boundary kernel writes is read or written by the
// stream-collide kernel of the step.  (With two cells per thread, a pair
// holding a cell on an open x face updates it from its partner's moments
// instead.)  Markers keep their stencils off the outer layer, so boundary
// cells carry no IB force.
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

// ------------------------------------------------------ boundary cells

// Boundary cell k of environment E, of those the boundary kernel updates:
// first every cell of the rows on open y/z faces (x fastest, rows with z on
// a face, then rows with only y on one), then, with xcells, the cells on
// open x faces of the other rows.  False past the last one.
__device__ __forceinline__ bool aa_boundary_cell(const EnvDev& E, long long k, bool xcells, int& x, int& y,
                                                 int& z) {
    const int nx = E.n[0], ny = E.n[1], nz = E.n[2];
    const int Lx = E.per[0] ? 0 : 2, Ly = E.per[1] ? 0 : 2, Lz = E.per[2] ? 0 : 2;
    const long long rows_z = (long long)Lz * ny;
    const long long rows_y = (long long)Ly * (nz - Lz);
    const long long nrow_cells = (rows_z + rows_y) * nx;
    if (k < nrow_cells) {
        const long long r = k / nx;
        x = (int)(k - r * nx);
        if (r < rows_z) {
            const int zi = (int)(r / ny);
            z = zi == 0 ? 0 : nz - 1;
            y = (int)(r - (long long)zi * ny);
        } else {
            const long long r2 = r - rows_z;
            y = (r2 & 1) == 0 ? 0 : ny - 1;
            z = (int)(r2 >> 1) + (Lz ? 1 : 0);
        }
        return true;
    }
    k -= nrow_cells;
    if (!xcells || Lx == 0) return false;
    const long long ay = ny - Ly;
    if (k >= ay * (nz - Lz) * 2) return false;
    const long long r = k >> 1;
    x = (k & 1) == 0 ? 0 : nx - 1;
    y = (int)(r % ay) + (Ly ? 1 : 0);
    z = (int)(r / ay) + (Lz ? 1 : 0);
    return true;
}

// The number of cells aa_boundary_cell enumerates for E.
__host__ __device__ inline long long aa_boundary_count(const EnvDev& E, bool xcells) {
    const int Lx = E.per[0] ? 0 : 2, Ly = E.per[1] ? 0 : 2, Lz = E.per[2] ? 0 : 2;
    const long long rows = (long long)Lz * E.n[1] + (long long)Ly * (E.n[2] - Lz);
    return rows * E.n[0] + (xcells ? (long long)Lx * (E.n[1] - Ly) * (E.n[2] - Lz) : 0);
}

// The boundary cells of a step of phase K (one per thread), before the
// stream-collide kernel of the step: each takes the moments of its inward
// neighbour x_f from where x_f's populations arrive (read before the
// stream-collide kernel overwrites them) and writes its outputs to its own
// locations, which nothing else reads or writes in the step.  Block b of
// environment E writes its mass partial after E's stream-collide partials.
// xcells: the cells on open x faces of the other rows too (one cell per
// thread in the stream-collide kernel; with two, the pair holding such a
// cell updates it).
template <class S, bool EQ3, int K>
__global__ void __launch_bounds__(K1_THREADS)
k_aa_boundary(typename S::raw* g, const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames,
              int n_envs, Pair32* __restrict__ mass_part, int xcells) {
    __shared__ float wsum[K1_THREADS / 32];
    __shared__ CellConsts C;
    const int b = blockIdx.x;
    const int e = n_envs > 1 ? env_of<&EnvDev::bblock0>(envs, n_envs, b) : 0;
    const EnvDev& E = envs[e];
    if (threadIdx.x == 0) C = load_consts(E, frames[e]);
    __syncthreads();
    float drout = 0.0f;
    const long long k = (long long)(b - E.bblock0) * K1_THREADS + threadIdx.x;
    int x, y, z;
    if (k < E.nbnd && aa_boundary_cell(E, k, xcells != 0, x, y, z)) {
        const int sx = inward(E, 0, x), sy = inward(E, 1, y), sz = inward(E, 2, z);
        const int px = x + sx, py = y + sy, pz = z + sz;
        const uint32_t s = (uint32_t)x + (uint32_t)E.P * ((uint32_t)y + (uint32_t)E.n[1] * (uint32_t)z);
        const uint32_t p = (uint32_t)px + (uint32_t)E.P * ((uint32_t)py + (uint32_t)E.n[1] * (uint32_t)pz);
        typename S::raw* G = g + E.pop_off;
        const Moments m =
            layout_moments<S, true, K == 0 ? LAYOUT_AA0 : LAYOUT_AA1>(G, E.nslot, p, pull_offsets(E, px, py, pz));
        const Herm h = cell_coeffs<S, EQ3>(C, m, x, y, z, sx, sy, sz, 0.0f, 0.0f, 0.0f);
        aa_emit_cell<S, EQ3, K, true>(h, G, E.nslot, s, pull_offsets(E, x, y, z), open_bits(E, x, y, z));
        drout = h.drout;
    }
    const float t = block_sum_f32(drout, wsum);
    if (threadIdx.x == 0) {
        Pair32 q;
        q.hi = t;
        mass_part[E.part0 + E.nblocks + (b - E.bblock0)] = q;
    }
}

// ---------------------------------------------------- the other cells

// Cell b * K1_THREADS + threadIdx.x of environment E (G: its populations),
// unless it is a boundary cell (k_aa_boundary's); returns rho_out - 1.
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
    if (open_bits(E, x, y, z)) return 0.0f;
    float fx, fy, fz;
    take_ib_force(E, fib, stamps, stamp, c, fx, fy, fz);
    const PullOffsets o = pull_offsets(E, x, y, z);
    const Moments m = layout_moments<S, true, K == 0 ? LAYOUT_AA0 : LAYOUT_AA1, false>(G, E.nslot, c, o);
    const Herm h = cell_coeffs<S, EQ3>(C, m, x, y, z, 0, 0, 0, fx, fy, fz);
    aa_emit_cell<S, EQ3, K, false>(h, opaque(G), opaque(E.nslot), opaque(c), opaque(o), 0u);
    return h.drout;
}

__device__ __forceinline__ Moments select_moments(bool first, const Moments& a, const Moments& b) {
    Moments m;
    m.dr = first ? a.dr : b.dr;
    m.jx = first ? a.jx : b.jx;
    m.jy = first ? a.jy : b.jy;
    m.jz = first ? a.jz : b.jz;
    m.sxx = first ? a.sxx : b.sxx;
    m.syy = first ? a.syy : b.syy;
    m.szz = first ? a.szz : b.szz;
    m.sxy = first ? a.sxy : b.sxy;
    m.sxz = first ? a.sxz : b.sxz;
    m.syz = first ? a.syz : b.syz;
    return m;
}

// Cells x (even) and x + 1 of one row (every row length even, so both are
// real cells), unless the row lies on an open y/z face (k_aa_boundary's).
// An open x face puts a boundary cell in the first or last pair of a row;
// the pair updates it from its partner's moments.
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
    if (open_bits(E, x, y, z) & 0x3Cu) return 0.0f;
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
    // the moments each cell's update takes (an open-face cell its partner's)
    const Moments sa = select_moments(!a_open, ma, mb);
    const Moments sb = select_moments(b_open, ma, mb);
    const Herm ha = cell_coeffs<S, EQ3>(C, sa, x, y, z, a_open ? 1 : 0, 0, 0, fa[0], fa[1], fa[2]);
    const Herm hb = cell_coeffs<S, EQ3>(C, sb, x + 1, y, z, b_open ? -1 : 0, 0, 0, fb[0], fb[1], fb[2]);
    if (a_open || b_open)
        aa_emit_pair<S, EQ3, K, true>(ha, hb, opaque(G), opaque(E.nslot), opaque(c), opaque(oa), opaque(ob),
                                      a_open ? 1u : 0u, b_open ? 2u : 0u);
    else
        aa_emit_pair<S, EQ3, K, false>(ha, hb, opaque(G), opaque(E.nslot), opaque(c), opaque(oa), opaque(ob), 0u,
                                       0u);
    return ha.drout + hb.drout;
}

// ------------------------------------------------------------- the kernel

// One step in place over every environment: phase K = 0 (even step) or 1
// (odd step), after k_aa_boundary of the same phase; the blocks of the
// plain kernel, mass partials from E.part0.  Resident blocks per SM it is
// compiled for (aa_minb): three for FP32 storage (80 registers), four for
// the 16-bit formats (64).  On the 256x128x128 swimmer channel, two cells
// per thread, mean of the even and odd phases: FP32 0.1677 ms at three
// against 0.1805 at four (where it spilled 40 bytes); FP16 0.1416 at three
// against 0.1346 at four.  (An earlier form of the kernel measured 0.172 /
// 0.213 ms for even / odd FP32 steps at four blocks against 0.186 / 0.205
// uncapped, and 0.213 / 0.209 against 0.225 / 0.252 with one cell per
// thread, 255 cells per row.)
template <class S>
constexpr int aa_minb() { return sizeof(typename S::raw) == 4 ? 3 : 4; }

template <class S, bool EQ3, bool PAIR, int K>
__global__ void __launch_bounds__(K1_THREADS, aa_minb<S>())
k_stream_collide_aa(typename S::raw* g, const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames,
                    int n_envs, float4* __restrict__ fib, const uint32_t* __restrict__ stamps,
                    const StepState* __restrict__ st, Pair32* __restrict__ mass_part) {
    __shared__ float wsum[K1_THREADS / 32];
    __shared__ CellConsts C;
    const uint32_t stamp = st->stamp;
    // odd steps take the blocks from the end of the domain first, where the
    // even step ended (its outputs are still in L2)
    const int b = K == 1 ? (int)(gridDim.x - 1u - blockIdx.x) : (int)blockIdx.x;
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
        mass_part[E.part0 + (b - E.block0)] = p;
    }
}

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
