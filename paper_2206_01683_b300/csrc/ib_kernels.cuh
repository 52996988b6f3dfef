// ib_kernels.cuh -- the immersed-boundary part of a step (arXiv 2206.01683,
// Sec. III-B: direct-forcing IB with the 4-point Peskin delta) as one
// persistent cooperative kernel in phases separated by grid barriers.
// Neighbouring markers share most of their stencil nodes, so the post-stream
// moments are computed once per node instead of once per (marker, node):
//   mark    one half-warp per marker stamps the 32-slot tiles of its 4x4x4
//           stencil with the step's stamp (plain stores)
//   nodes   warps read the tile stamps, strided over the grid so that the
//           stamped tiles spread evenly; for each stamped tile the warp
//           computes rho and u~ = j/rho + a0/2 of its 32 cells (coalesced
//           pulls), one float4 per cell
//   force   one half-warp per marker: R, U~ from the 64 node float4s,
//           F = 2 R (U - U~), spread F dV delta onto the nodes (vector
//           reductions into the float4 force field); with multi-direct
//           forcing (ib_iters > 1) further passes interpolate the velocity
//           corrected by the force spread so far, then (after a grid
//           barrier) spread their increments
//
// The forces and the grid force density equal those of the single-pass k_ib
// below (same per-node arithmetic, same delta weights), which the adjoint's
// recomputation uses.
// Data written in one phase and read in a later one (tile stamps, node
// values) is read with ld.global.cg, never through the non-coherent path.
#pragma once

#include "step_kernels.cuh"
#include "marker_src.cuh"

namespace fl {

// ------------------------------------------------- single pass (adjoint)

// One warp per marker: lane (kx, ky, kz) with kx = lane & 3, ky = (lane>>2)&3,
// kz = lane >> 4 owns stencil nodes (kx, ky, kz) and (kx, ky, kz + 2).
template <class S>
__global__ void __launch_bounds__(IB_THREADS, 4)
k_ib(const typename S::raw* __restrict__ gin, const EnvDev* __restrict__ envs,
     const FrameDev* __restrict__ frames, int n_envs, int total_markers,
     const float* __restrict__ X, const float* __restrict__ U, const float* __restrict__ dV,
     float* __restrict__ Fm, float4* __restrict__ fib, uint32_t* __restrict__ stamps,
     const StepState* __restrict__ st, int* __restrict__ status) {
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= total_markers) return;  // whole warp
    const uint32_t stamp = st->stamp;
    const int e = n_envs > 1 ? env_of<&EnvDev::mk_begin>(envs, n_envs, warp) : 0;
    const EnvDev& E = envs[e];
    const FrameDev F = frames[e];
    const int slot = E.marker_off + (warp - E.mk_begin);

    float xw[3];
    int base[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = X[3 * slot + a];
        const float N = (float)E.n[a];
        float w = x;
        if (!(fabsf(x) <= 1.0e6f)) ok = false;  // also rejects NaN
        if (E.per[a]) {
            w = x - floorf(x / N) * N;
            if (w >= N) w -= N;
            if (w < 0.0f) w += N;
        } else if (!(x >= 2.0f && x < N - 3.0f)) {
            ok = false;
        }
        xw[a] = w;
        base[a] = ok ? (int)floorf(w) - 1 : 0;
    }
    if (!ok) {
        if (lane == 0) {
            Fm[3 * slot] = 0.f; Fm[3 * slot + 1] = 0.f; Fm[3 * slot + 2] = 0.f;
            atomicOr(status, ST_BAD_MARKER);
        }
        return;
    }
    const int kx = lane & 3, ky = (lane >> 2) & 3, kz = lane >> 4;
    const int mx = base[0] + kx, my = base[1] + ky;
    const float wxy = peskin4(xw[0] - (float)mx) * peskin4(xw[1] - (float)my);
    const int nx = E.n[0], ny = E.n[1], nz = E.n[2];
    // node indices lie in [-1, n+2]; a true modulo also covers periodic axes
    // shorter than the stencil (n < 4)
    const int mxw = ((mx % nx) + nx) % nx;
    const int myw = ((my % ny) + ny) % ny;
    const typename S::raw* G = gin + E.pop_off;

    float R = 0.f, Ux = 0.f, Uy = 0.f, Uz = 0.f;
    float dlt[2];
    uint32_t cell[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int mz = base[2] + kz + 2 * h;
        const int mzw = ((mz % nz) + nz) % nz;
        const float d = wxy * peskin4(xw[2] - (float)mz);
        const uint32_t c = (uint32_t)mxw + (uint32_t)E.P * ((uint32_t)myw + (uint32_t)ny * (uint32_t)mzw);
        const PullOffsets o = pull_offsets(E, mxw, myw, mzw);
        const Moments m = pull_moments<S, false>(G, E.nslot, c, o);
        const float rho = 1.0f + m.dr;
        const float inv = 1.0f / rho;
        float a0[3];
        frame_accel(F, (float)mxw, (float)myw, (float)mzw, a0);
        R += d * rho;
        Ux += d * (m.jx * inv + 0.5f * a0[0]);
        Uy += d * (m.jy * inv + 0.5f * a0[1]);
        Uz += d * (m.jz * inv + 0.5f * a0[2]);
        dlt[h] = d;
        cell[h] = c;
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        R += __shfl_xor_sync(0xffffffffu, R, s);
        Ux += __shfl_xor_sync(0xffffffffu, Ux, s);
        Uy += __shfl_xor_sync(0xffffffffu, Uy, s);
        Uz += __shfl_xor_sync(0xffffffffu, Uz, s);
    }
    // direct forcing: F_l = 2 R_l (U_l - U~_l); the grid receives F_l dV_l delta
    const float Fx = 2.0f * R * (U[3 * slot] - Ux);
    const float Fy = 2.0f * R * (U[3 * slot + 1] - Uy);
    const float Fz = 2.0f * R * (U[3 * slot + 2] - Uz);
    const float v = dV[slot];
    float4* fb = fib + E.slot_off;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float s = v * dlt[h];
        atomicAdd(fb + cell[h], make_float4(Fx * s, Fy * s, Fz * s, 0.f));
        stamps[E.stamp_off + (cell[h] >> 5)] = stamp;
    }
    if (lane == 0) {
        Fm[3 * slot] = Fx; Fm[3 * slot + 1] = Fy; Fm[3 * slot + 2] = Fz;
    }
}

// ------------------------------------------------- k_ib_step (the step)

// Stencil of one marker along each axis (periodic wrap, validity as in k_ib).
struct Stencil {
    float xw[3];
    int base[3];
    bool ok;
};

__device__ __forceinline__ Stencil stencil_at(const EnvDev& E, const float (&xm)[3]) {
    Stencil st;
    st.ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = xm[a];
        const float N = (float)E.n[a];
        float w = x;
        if (!(fabsf(x) <= 1.0e6f)) st.ok = false;  // also rejects NaN
        if (E.per[a]) {
            w = x - floorf(x / N) * N;
            if (w >= N) w -= N;
            if (w < 0.0f) w += N;
        } else if (!(x >= 2.0f && x < N - 3.0f)) {
            st.ok = false;
        }
        st.xw[a] = w;
        st.base[a] = st.ok ? (int)floorf(w) - 1 : 0;
    }
    return st;
}

__device__ __forceinline__ Stencil marker_stencil(const EnvDev& E, const float* __restrict__ X, int slot) {
    const float x[3] = {X[3 * slot], X[3 * slot + 1], X[3 * slot + 2]};
    return stencil_at(E, x);
}

constexpr uint32_t GRID_WAIT_LIMIT = 1u << 22;  // barrier polls before giving up

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of a cooperative launch (all blocks resident at once) on an
// arrival counter bar[0] that only grows; bar[1] holds its value at the
// start of the launch (the base).  Barrier k waits until the counter reaches
// base + k * gridDim.x.  Each block adds 1 with release semantics (its writes
// are ordered before thread 0's arrival by __syncthreads) and polls with
// acquire loads.  Polls are bounded: a block that gives up records
// ST_TIMEOUT and returns false; the host then poisons the domain and zeroes
// both words.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned base, unsigned k, int* status,
                                             uint32_t limit = GRID_WAIT_LIMIT) {
    __shared__ int pass;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = base + k * gridDim.x;
        int ok = 1;
        red_add_release_gpu(bar, 1u);
        uint32_t i = 0;
        while ((int)(ld_acquire_gpu(bar) - target) < 0) {
            if (++i == limit) {
                ok = 0;
                atomicOr(status, ST_TIMEOUT);
                break;
            }
        }
        pass = ok;
    }
    __syncthreads();
    return pass != 0;
}

// Half-warp stencil walk: half-lane h (0..15) owns the stencil column
// (kx, ky) = (h & 3, h >> 2) and its four nodes kz = 0..3.
struct Column {
    int mxw, myw;      // wrapped node x, y
    float wxy;         // phi(X - mx) phi(Y - my)
};

__device__ __forceinline__ Column stencil_column(const EnvDev& E, const Stencil& S, int h) {
    Column col;
    const int mx = S.base[0] + (h & 3), my = S.base[1] + (h >> 2);
    col.wxy = peskin4(S.xw[0] - (float)mx) * peskin4(S.xw[1] - (float)my);
    col.mxw = ((mx % E.n[0]) + E.n[0]) % E.n[0];
    col.myw = ((my % E.n[1]) + E.n[1]) % E.n[1];
    return col;
}

__device__ __forceinline__ uint32_t column_slot(const EnvDev& E, const Column& col, int mz) {
    const int mzw = ((mz % E.n[2]) + E.n[2]) % E.n[2];
    return (uint32_t)col.mxw + (uint32_t)E.P * ((uint32_t)col.myw + (uint32_t)E.n[1] * (uint32_t)mzw);
}

// mark: stamp the tiles of one marker's stencil (plain idempotent stores;
// the tiles of one column are distinct, they differ in z).
__device__ __forceinline__ void ib_mark(const EnvDev& E, const Stencil& S, int h, uint32_t stamp,
                                        uint32_t* stamps) {
    const Column col = stencil_column(E, S, h);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
        const uint32_t c = column_slot(E, col, S.base[2] + kz);
        if (FG_IN_RANGE(DBG_NODE, c, E.nslot)) stamps[E.stamp_off + (c >> 5)] = stamp;
    }
}

// nodes: post-stream rho and u~ of the 32 cells of tile t_local (counted
// from the environment's first tile) of environment E (one warp), the
// populations found where `layout` (LAYOUT_*) keeps them.
template <class S>
__device__ __forceinline__ void ib_nodes_of(const typename S::raw* __restrict__ gin, const EnvDev& E,
                                            const FrameDev& F, int t_local, int lane, float4* nodes,
                                            int layout = LAYOUT_PULL) {
    const uint32_t c = (uint32_t)t_local * 32u + (uint32_t)lane;
    if (c >= E.nslot) return;
    const uint32_t row = fdiv(c, E.div_P);
    const int x = (int)(c - row * (uint32_t)E.P);
    if (x >= E.n[0]) return;
    const uint32_t zz = fdiv(row, E.div_ny);
    const int y = (int)(row - zz * (uint32_t)E.n[1]);
    const int z = (int)zz;
    // the stencil nodes of valid markers lie off the outer layer of an open
    // axis; other cells of the tile may not, and pull_offsets then wraps
    // (in-bounds reads of values that no marker uses)
    const PullOffsets o = pull_offsets(E, x, y, z);
    const typename S::raw* G = gin + E.pop_off;
    const Moments m = layout == LAYOUT_AA0   ? layout_moments<S, false, LAYOUT_AA0>(G, E.nslot, c, o)
                      : layout == LAYOUT_AA1 ? layout_moments<S, false, LAYOUT_AA1>(G, E.nslot, c, o)
                                             : pull_moments<S, false>(G, E.nslot, c, o);
    const float rho = 1.0f + m.dr, inv = 1.0f / rho;
    float a0[3];
    frame_accel(F, (float)x, (float)y, (float)z, a0);
    nodes[E.slot_off + c] = make_float4(rho, m.jx * inv + 0.5f * a0[0], m.jy * inv + 0.5f * a0[1],
                                        m.jz * inv + 0.5f * a0[2]);
}

// nodes of the domain-wide tile t (the environment found from its tile offset)
template <class S>
__device__ __forceinline__ void ib_nodes(const typename S::raw* __restrict__ gin, const EnvDev* __restrict__ envs,
                                         const FrameDev* __restrict__ frames, int n_envs, int t, int lane,
                                         float4* nodes, int layout = LAYOUT_PULL) {
    const int e = n_envs > 1 ? env_of<&EnvDev::stamp_off>(envs, n_envs, t) : 0;
    ib_nodes_of<S>(gin, envs[e], frames[e], t - envs[e].stamp_off, lane, nodes, layout);
}

// One marker of a half-warp: its environment, slot, stencil, U and dV.
struct MarkerRef {
    int e, slot;
    Stencil S;
    float U[3], dV;
};

__device__ __forceinline__ MarkerRef marker_ref(const EnvDev& E, int e, int slot, const float (&x)[3],
                                                const float (&u)[3], const float* __restrict__ dV) {
    MarkerRef r;
    r.e = e;
    r.slot = slot;
    r.S = stencil_at(E, x);
    r.U[0] = u[0]; r.U[1] = u[1]; r.U[2] = u[2];
    r.dV = dV[slot];
    return r;
}

// COHERENT reads X and U through L2 (ld.global.cg): in the step whose IB
// kernel copies the markers into those arrays (a posted MarkerSrc), blocks
// read there what other blocks wrote before a grid barrier.
template <bool COHERENT = false>
__device__ __forceinline__ MarkerRef load_marker_slot(const EnvDev& E, int e, int slot, const float* __restrict__ X,
                                                      const float* __restrict__ U, const float* __restrict__ dV) {
    float x[3], u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = COHERENT ? __ldcg(X + 3 * slot + a) : X[3 * slot + a];
        u[a] = COHERENT ? __ldcg(U + 3 * slot + a) : U[3 * slot + a];
    }
    return marker_ref(E, e, slot, x, u, dV);
}

__device__ __forceinline__ int marker_env(const EnvDev* __restrict__ envs, int n_envs, int m) {
    return n_envs > 1 ? env_of<&EnvDev::mk_begin>(envs, n_envs, m) : 0;
}

template <bool COHERENT = false>
__device__ __forceinline__ MarkerRef load_marker(const EnvDev* __restrict__ envs, int n_envs, int m,
                                                 const float* __restrict__ X, const float* __restrict__ U,
                                                 const float* __restrict__ dV) {
    const int e = marker_env(envs, n_envs, m);
    const EnvDev& E = envs[e];
    return load_marker_slot<COHERENT>(E, e, E.marker_off + (m - E.mk_begin), X, U, dV);
}

// Marker m of a posted MarkerSrc (compact numbering), for a half-warp: lanes
// h = 0..5 each read one value (X then U) and the half-warp shares them, so
// a source in pinned host memory is read once, in a few requests.  Called by
// all 32 lanes of the warp (`here` false for a half without a marker: its
// values are 0).  The lane's own value is returned, for the copy into the
// domain's arrays (marker_store).
__device__ __forceinline__ float marker_fetch(const MarkerSrc& ms, int m, bool here, int lane, float (&x)[3],
                                              float (&u)[3]) {
    const int h = lane & 15;
    float v = 0.0f;
    if (here && h < 6) v = h < 3 ? ms.X[3 * m + h] : ms.U[3 * m + h - 3];
    const int b = lane & 16;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = __shfl_sync(0xffffffffu, v, b + a);
        u[a] = __shfl_sync(0xffffffffu, v, b + 3 + a);
    }
    return v;
}

__device__ __forceinline__ void marker_store(float* X, float* U, int slot, int h, float v) {
    if (h < 3) X[3 * slot + h] = v;
    else if (h < 6) U[3 * slot + h - 3] = v;
}

// Stencil nodes of half-lane h for one marker: the slots of its column's
// four nodes and their delta weights.
struct ColumnNodes {
    float dlt[4];
    uint32_t cell[4];
};

__device__ __forceinline__ ColumnNodes column_nodes(const EnvDev& E, const MarkerRef& r, int h) {
    ColumnNodes cn;
    const Column col = stencil_column(E, r.S, h);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
        const int mz = r.S.base[2] + kz;
        cn.cell[kz] = column_slot(E, col, mz);
        cn.dlt[kz] = col.wxy * peskin4(r.S.xw[2] - (float)mz);
        if (!FG_IN_RANGE(DBG_NODE, cn.cell[kz], E.nslot)) {   // skip the node
            cn.cell[kz] = 0;
            cn.dlt[kz] = 0.0f;
        }
    }
    return cn;
}

// Deterministic spread: every contribution is rounded to a multiple of 2^-48
// and summed as a 64-bit integer.  Integer addition is exact and associative,
// so the sum does not depend on the order in which the reductions land; it
// is converted back to FP32 once.  |contributions| and |sums| must stay below
// 2^15 (force densities here are far smaller); larger contributions are
// flagged as a numeric fault.
constexpr float FIX_SCALE = 281474976710656.0f;        // 2^48
constexpr float FIX_INV = 3.5527136788005009294e-15f;  // 2^-48

__device__ __forceinline__ void spread_force_fixed(const EnvDev& E, const MarkerRef& r, const ColumnNodes& cn,
                                                   float3 F, unsigned long long* fibq, int* status) {
    unsigned long long* q = fibq + 3ull * E.slot_off;
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
        const float s = r.dV * cn.dlt[kz];
        const float v[3] = {F.x * s, F.y * s, F.z * s};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!(fabsf(v[a]) < 16384.0f)) atomicOr(status, ST_NUMERIC);
            atomicAdd(q + 3ull * cn.cell[kz] + a, (unsigned long long)__float2ll_rn(v[a] * FIX_SCALE));
        }
    }
}

__device__ __forceinline__ float fixed_to_float(unsigned long long q) {
    return __ll2float_rn((long long)q) * FIX_INV;
}

// Direct-forcing increment of pass `pass`: R and U~ interpolated from the
// node values, U~ of the velocity corrected by the force density spread in
// the earlier passes (u~ + fib / (2 rho)); dF = 2 R (U - U~), or with slip
// forcing (Nrm != nullptr) its normal component (dF.n) n.  `active` is
// false for a half-warp without a (valid) marker, which still takes part in
// the shuffles; the result is valid in every lane of an active half.
__device__ __forceinline__ float3 interp_force(const EnvDev& E, const MarkerRef& r, const ColumnNodes& cn,
                                               bool active, int pass, const float4* fib,
                                               const unsigned long long* fibq, const float4* nodes,
                                               const float* __restrict__ Nrm) {
    float R = 0.f, Ux = 0.f, Uy = 0.f, Uz = 0.f;
    if (active) {
#pragma unroll
        for (int kz = 0; kz < 4; ++kz) {
            float4 nd = __ldcg(nodes + E.slot_off + cn.cell[kz]);
            if (pass > 0) {   // the force field is zero when the step starts
                float4 f;
                if (fibq) {   // deterministic spread: the fixed-point sums
                    const unsigned long long* q = fibq + 3ull * (E.slot_off + cn.cell[kz]);
                    f = make_float4(fixed_to_float(__ldcg(q)), fixed_to_float(__ldcg(q + 1)),
                                    fixed_to_float(__ldcg(q + 2)), 0.f);
                } else {
                    f = __ldcg(fib + E.slot_off + cn.cell[kz]);
                }
                const float s = 0.5f / nd.x;
                nd.y += f.x * s;
                nd.z += f.y * s;
                nd.w += f.z * s;
            }
            R += cn.dlt[kz] * nd.x;
            Ux += cn.dlt[kz] * nd.y;
            Uy += cn.dlt[kz] * nd.z;
            Uz += cn.dlt[kz] * nd.w;
        }
    }
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
        R += __shfl_xor_sync(0xffffffffu, R, s);
        Ux += __shfl_xor_sync(0xffffffffu, Ux, s);
        Uy += __shfl_xor_sync(0xffffffffu, Uy, s);
        Uz += __shfl_xor_sync(0xffffffffu, Uz, s);
    }
    float3 F = make_float3(2.0f * R * (r.U[0] - Ux), 2.0f * R * (r.U[1] - Uy), 2.0f * R * (r.U[2] - Uz));
    if (Nrm && active) {   // slip forcing: keep the normal component, (F.n) n
        const float nx = __ldg(Nrm + 3 * r.slot), ny = __ldg(Nrm + 3 * r.slot + 1), nz = __ldg(Nrm + 3 * r.slot + 2);
        const float dn = F.x * nx + F.y * ny + F.z * nz;
        F = make_float3(dn * nx, dn * ny, dn * nz);
    }
    return F;
}

// Spread dF dV delta onto the column's nodes (one vector reduction per node).
__device__ __forceinline__ void spread_force(const EnvDev& E, const MarkerRef& r, const ColumnNodes& cn, float3 F,
                                             float4* fib) {
    float4* fb = fib + E.slot_off;
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
        const float s = r.dV * cn.dlt[kz];
        atomicAdd(fb + cn.cell[kz], make_float4(F.x * s, F.y * s, F.z * s, 0.f));
    }
}

// Environments whose tables k_ib_step keeps in dynamic shared memory, and
// the bytes a launch provides for them.
constexpr int IB_SMEM_ENVS = 128;   // 128 x 316 B = 40 KB, within the default 48 KB
static_assert(sizeof(EnvDev) % 8 == 0 && sizeof(FrameDev) % 4 == 0,
              "the tables are copied as 32-bit words and the frames follow the 8-byte aligned EnvDev array");
__host__ __device__ constexpr size_t ib_smem_bytes(int n_envs) {
    return n_envs > 1 && n_envs <= IB_SMEM_ENVS ? (sizeof(EnvDev) + sizeof(FrameDev)) * (size_t)n_envs : 0;
}

// The IB part of one step.  Launched cooperatively with at most as many
// blocks as fit on the device at once; half-warps stride over markers (the
// first marker of each half-warp stays in registers from the mark phase to
// the force phase), warps over tile stamps.  fibq != nullptr selects the
// deterministic spread (fixed-point sums, converted to fib in a last phase).
// layout (LAYOUT_*) says where the node moments find the populations.
// Compiled for three resident blocks per SM (80 registers): at four (64
// registers, 32 bytes of spills) the swimmer's IB took 24.3-24.4 against
// 23.8-24.0 us and the 64-environment batch's 0.246 against 0.238 ms.
template <class S>
__global__ void __launch_bounds__(IB_THREADS, 3)
k_ib_step(const typename S::raw* __restrict__ gin, const EnvDev* __restrict__ envs_g,
          const FrameDev* __restrict__ frames_g, int n_envs, int total_markers, int n_stamps,
          float* X, float* U, const float* __restrict__ dV,
          float* __restrict__ Fm, float4* fib, uint32_t* stamps, const StepState* __restrict__ st,
          float4* nodes, unsigned* bar, int ib_iters, float* dF, unsigned long long* fibq,
          const float* __restrict__ Nrm, int* status, int layout, const MarkerSrc* __restrict__ msrc) {
    // the environments' tables and frames in shared memory, read by every
    // marker and node of the launch (the environment of a marker or tile is
    // found by a binary search over them): one environment in static shared
    // memory, up to IB_SMEM_ENVS in the dynamic shared memory the launch
    // provides (ib_smem_bytes), more read from global memory; the posted
    // marker source, if any
    __shared__ EnvDev sE;
    __shared__ FrameDev sF;
    __shared__ MarkerSrc sM;
    extern __shared__ __align__(16) unsigned char ib_tables[];
    const bool staged_tables = n_envs > 1 && n_envs <= IB_SMEM_ENVS;
    EnvDev* tE = reinterpret_cast<EnvDev*>(ib_tables);
    FrameDev* tF = reinterpret_cast<FrameDev*>(ib_tables + sizeof(EnvDev) * (size_t)n_envs);
    if (staged_tables) {
        const int we = n_envs * (int)(sizeof(EnvDev) / 4), wf = n_envs * (int)(sizeof(FrameDev) / 4);
        for (int k = threadIdx.x; k < we; k += blockDim.x)
            reinterpret_cast<uint32_t*>(tE)[k] = reinterpret_cast<const uint32_t*>(envs_g)[k];
        for (int k = threadIdx.x; k < wf; k += blockDim.x)
            reinterpret_cast<uint32_t*>(tF)[k] = reinterpret_cast<const uint32_t*>(frames_g)[k];
    }
    if (threadIdx.x == 0) {
        if (n_envs == 1) {
            sE = envs_g[0];
            sF = frames_g[0];
        }
        sM = *msrc;
    }
    __syncthreads();
    // posted: the step's markers come from the caller's arrays; the mark
    // phase copies them into X and U, which later phases read through L2
    const MarkerSrc ms = sM;
    const bool posted = ms.valid != 0;
    const EnvDev* envs = n_envs == 1 ? &sE : (staged_tables ? tE : envs_g);
    const FrameDev* frames = n_envs == 1 ? &sF : (staged_tables ? tF : frames_g);
    const int lane = threadIdx.x & 31, h = lane & 15;
    const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const uint32_t stamp = st->stamp;
    const unsigned base = __ldcg(bar + 1);
    // barriers of this launch: mark, nodes, two per extra pass, the conversion
    const unsigned n_bar = 2u * (unsigned)ib_iters + (fibq ? 1u : 0u);
    unsigned nb = 0;
    auto barrier = [&]() -> bool {
        if (!grid_barrier(bar, base, ++nb, status)) return false;
        if (nb == n_bar && blockIdx.x == 0 && threadIdx.x == 0) bar[1] = base + n_bar * gridDim.x;
        return true;
    };
    auto spread = [&](const EnvDev& E, const MarkerRef& r, const ColumnNodes& cn, float3 F) {
        if (fibq) spread_force_fixed(E, r, cn, F, fibq, status);
        else spread_force(E, r, cn, F, fib);
    };
    // marker m of a later phase (after the mark phase's barrier)
    auto reload = [&](int m) -> MarkerRef {
        return posted ? load_marker<true>(envs, n_envs, m, X, U, dV) : load_marker<false>(envs, n_envs, m, X, U, dV);
    };
    const int m0 = 2 * gw + (lane >> 4);
    // mark (half-warps walk markers 2 gw + 2 nw k + (lane >> 4); both halves
    // of a warp iterate alike, for the posted source's shuffles)
    MarkerRef first;
    first.S.ok = false;
    for (int mb = 2 * gw; mb < total_markers; mb += 2 * nw) {
        const int m = mb + (lane >> 4);
        const bool here = m < total_markers;
        MarkerRef r;
        r.S.ok = false;
        if (posted) {
            float x[3], u[3];
            const float v = marker_fetch(ms, m, here, lane, x, u);
            if (here) {
                const int e = marker_env(envs, n_envs, m);
                const EnvDev& E = envs[e];
                const int slot = E.marker_off + (m - E.mk_begin);
                marker_store(X, U, slot, h, v);
                r = marker_ref(E, e, slot, x, u, dV);
            }
        } else if (here) {
            r = load_marker<false>(envs, n_envs, m, X, U, dV);
        }
        if (here && r.S.ok) ib_mark(envs[r.e], r.S, h, stamp, stamps);   // invalid markers: the force phase reports them
        if (mb == 2 * gw) first = r;
    }
    if (!barrier()) return;
    // nodes: lane k of warp gw reads the stamp of tile gw + nw (k + 32 j)
    for (int t0 = gw; t0 < n_stamps; t0 += 32 * nw) {
        const long long t = (long long)t0 + (long long)lane * nw;
        const bool hit = t < n_stamps && __ldcg(stamps + t) == stamp;
        unsigned hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
            const int k = __ffs(hits) - 1;
            hits &= hits - 1u;
            ib_nodes<S>(gin, envs, frames, n_envs, t0 + k * nw, lane, nodes, layout);
        }
    }
    if (!barrier()) return;
    // force, pass 0: interpolate, form F and spread it (nothing reads the
    // force field in this pass)
    for (int mb = 2 * gw; mb < total_markers; mb += 2 * nw) {   // both halves iterate alike
        const int m = mb + (lane >> 4);
        const bool here = m < total_markers;
        MarkerRef r;
        r.e = 0;
        r.slot = 0;
        r.S.ok = false;
        if (here) r = mb == 2 * gw ? first : reload(m);
        if (here && !r.S.ok && h == 0) {
            Fm[3 * r.slot] = 0.f; Fm[3 * r.slot + 1] = 0.f; Fm[3 * r.slot + 2] = 0.f;
            atomicOr(status, ST_BAD_MARKER);
        }
        const bool active = here && r.S.ok;
        const EnvDev& E = envs[r.e];
        ColumnNodes cn;
        if (active) cn = column_nodes(E, r, h);
        const float3 F = interp_force(E, r, cn, active, 0, fib, fibq, nodes, Nrm);
        if (active) {
            spread(E, r, cn, F);
            if (h == 0) { Fm[3 * r.slot] = F.x; Fm[3 * r.slot + 1] = F.y; Fm[3 * r.slot + 2] = F.z; }
        }
    }
    // multi-direct forcing, passes 1 .. ib_iters-1: every marker interpolates
    // the corrected velocity before any spreads this pass's increment (two
    // grid barriers per pass); the increments wait in dF.
    for (int pass = 1; pass < ib_iters; ++pass) {
        if (!barrier()) return;
        for (int mb = 2 * gw; mb < total_markers; mb += 2 * nw) {
            const int m = mb + (lane >> 4);
            const bool here = m < total_markers;
            MarkerRef r;
            r.e = 0;
            r.slot = 0;
            r.S.ok = false;
            if (here) r = mb == 2 * gw ? first : reload(m);
            const bool active = here && r.S.ok;
            const EnvDev& E = envs[r.e];
            ColumnNodes cn;
            if (active) cn = column_nodes(E, r, h);
            const float3 F = interp_force(E, r, cn, active, pass, fib, fibq, nodes, Nrm);
            if (active && h == 0) {
                float* Fl = Fm + 3 * r.slot;
                Fl[0] += F.x; Fl[1] += F.y; Fl[2] += F.z;
                float* d = dF + 3 * r.slot;
                d[0] = F.x; d[1] = F.y; d[2] = F.z;
            }
        }
        if (!barrier()) return;
        for (int m = m0; m < total_markers; m += 2 * nw) {
            const MarkerRef r = m == m0 ? first : reload(m);
            if (!r.S.ok) continue;
            const EnvDev& E = envs[r.e];
            const float* d = dF + 3 * r.slot;
            spread(E, r, column_nodes(E, r, h), make_float3(__ldcg(d), __ldcg(d + 1), __ldcg(d + 2)));
        }
    }
    if (!fibq) return;
    // deterministic spread: convert the fixed-point sums of every stamped tile
    // to the FP32 force field and clear them
    if (!barrier()) return;
    for (int t0 = gw; t0 < n_stamps; t0 += 32 * nw) {
        const long long t = (long long)t0 + (long long)lane * nw;
        const bool hit = t < n_stamps && __ldcg(stamps + t) == stamp;
        unsigned hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
            const int k = __ffs(hits) - 1;
            hits &= hits - 1u;
            const int tt = t0 + k * nw;
            const int e = n_envs > 1 ? env_of<&EnvDev::stamp_off>(envs, n_envs, tt) : 0;
            const EnvDev& E = envs[e];
            const uint32_t c = (uint32_t)(tt - E.stamp_off) * 32u + (uint32_t)lane;
            if (c < E.nslot) {
                unsigned long long* q = fibq + 3ull * (E.slot_off + c);
                const unsigned long long qx = __ldcg(q), qy = __ldcg(q + 1), qz = __ldcg(q + 2);
                fib[E.slot_off + c] = make_float4(fixed_to_float(qx), fixed_to_float(qy), fixed_to_float(qz), 0.f);
                q[0] = 0ull; q[1] = 0ull; q[2] = 0ull;
            }
        }
    }
}

// The mark phase as a kernel of its own, for the step that runs the IB
// beside the stream-collide kernel: half a warp per marker stamps the tiles
// of its stencil and flags the plain stream-collide block of every stencil
// node (blocks of 2^block_shift slots), so that the stream-collide launches
// can split the cells into the blocks the IB force reaches and the rest.
__global__ void __launch_bounds__(IB_THREADS)
k_mark_tiles(const EnvDev* __restrict__ envs, int n_envs, int total_markers, const float* __restrict__ X,
             const StepState* __restrict__ st, uint32_t* __restrict__ stamps, uint32_t* __restrict__ blk_flag,
             int block_shift) {
    const int m = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 4);
    if (m >= total_markers) return;   // whole half-warps
    const int h = threadIdx.x & 15;
    const uint32_t stamp = st->stamp;
    const int e = n_envs > 1 ? env_of<&EnvDev::mk_begin>(envs, n_envs, m) : 0;
    const EnvDev& E = envs[e];
    const Stencil S = marker_stencil(E, X, E.marker_off + (m - E.mk_begin));
    if (!S.ok) return;   // the IB kernel reports it
    const Column col = stencil_column(E, S, h);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
        const uint32_t c = column_slot(E, col, S.base[2] + kz);
        if (FG_IN_RANGE(DBG_NODE, c, E.nslot)) {
            stamps[E.stamp_off + (c >> 5)] = stamp;
            blk_flag[E.block0 + (c >> block_shift)] = stamp;
        }
    }
}

// The IB phases after the mark as separate, non-cooperative kernels, for
// the step that runs the IB beside the stream-collide kernel: no grid
// barrier holds a block between phases, so each block occupies its SM slot
// only while it works (the phase order is the launch order on the stream).
// The arithmetic is k_ib_step's.
//
// Node moments of the stamped tiles: warp w of the launch reads the stamps
// of tiles w + nw (lane + 32 j), so that the stamped tiles, which come in
// runs, spread over the warps; a hit tile is computed by the warp.
// CONVERT != 0: instead, the deterministic spread's fixed-point sums of the
// stamped tiles become the FP32 force field and are cleared.
template <class S, bool CONVERT>
__global__ void __launch_bounds__(IB_THREADS)
k_ib_tiles(const typename S::raw* __restrict__ gin, const EnvDev* __restrict__ envs,
           const FrameDev* __restrict__ frames, int n_envs, int n_stamps, const uint32_t* __restrict__ stamps,
           const StepState* __restrict__ st, float4* __restrict__ nodes, float4* __restrict__ fib,
           unsigned long long* __restrict__ fibq) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const uint32_t stamp = st->stamp;
    for (int t0 = gw; t0 < n_stamps; t0 += 32 * nw) {
        const long long t = (long long)t0 + (long long)lane * nw;
        const bool hit = t < n_stamps && __ldg(stamps + t) == stamp;
        unsigned hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
            const int k = __ffs(hits) - 1;
            hits &= hits - 1u;
            const int tt = t0 + k * nw;
            if (!CONVERT) {
                ib_nodes<S>(gin, envs, frames, n_envs, tt, lane, nodes);
            } else {
                const int e = n_envs > 1 ? env_of<&EnvDev::stamp_off>(envs, n_envs, tt) : 0;
                const EnvDev& E = envs[e];
                const uint32_t c = (uint32_t)(tt - E.stamp_off) * 32u + (uint32_t)lane;
                if (c < E.nslot) {
                    unsigned long long* q = fibq + 3ull * (E.slot_off + c);
                    fib[E.slot_off + c] = make_float4(fixed_to_float(q[0]), fixed_to_float(q[1]),
                                                      fixed_to_float(q[2]), 0.f);
                    q[0] = 0ull; q[1] = 0ull; q[2] = 0ull;
                }
            }
        }
    }
}

// Direct-forcing pass `pass` at half a warp per marker: pass 0 interpolates,
// forms F and spreads it (a marker outside its allowed range gets F = 0 and
// raises ST_BAD_MARKER); a later pass (SPREAD = false) interpolates the
// corrected velocity, adds the increment to F and keeps it in dF; SPREAD =
// true spreads the kept increments.
template <class S, bool SPREAD>
__global__ void __launch_bounds__(IB_THREADS)
k_ib_markers(const EnvDev* __restrict__ envs, int n_envs, int total_markers, const float* __restrict__ X,
             const float* __restrict__ U, const float* __restrict__ dV, float* __restrict__ Fm,
             float4* __restrict__ fib, const float4* __restrict__ nodes, float* __restrict__ dF,
             unsigned long long* __restrict__ fibq, const float* __restrict__ Nrm, int pass, int* status) {
    const int m = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 4);
    const int h = threadIdx.x & 15;
    const bool here = m < total_markers;
    MarkerRef r;
    r.e = 0;
    r.slot = 0;
    r.S.ok = false;
    if (here) r = load_marker(envs, n_envs, m, X, U, dV);
    const bool active = here && r.S.ok;
    const EnvDev& E = envs[r.e];
    ColumnNodes cn;
    if (active) cn = column_nodes(E, r, h);
    if (SPREAD) {
        if (active) {
            const float* d = dF + 3 * r.slot;
            const float3 F = make_float3(d[0], d[1], d[2]);
            if (fibq) spread_force_fixed(E, r, cn, F, fibq, status);
            else spread_force(E, r, cn, F, fib);
        }
        return;
    }
    if (pass == 0 && here && !r.S.ok && h == 0) {
        Fm[3 * r.slot] = 0.f; Fm[3 * r.slot + 1] = 0.f; Fm[3 * r.slot + 2] = 0.f;
        atomicOr(status, ST_BAD_MARKER);
    }
    // every lane takes part in the half-warp shuffles
    const float3 F = interp_force(E, r, cn, active, pass, fib, fibq, nodes, Nrm);
    if (!active) return;
    if (pass == 0) {
        if (fibq) spread_force_fixed(E, r, cn, F, fibq, status);
        else spread_force(E, r, cn, F, fib);
        if (h == 0) { Fm[3 * r.slot] = F.x; Fm[3 * r.slot + 1] = F.y; Fm[3 * r.slot + 2] = F.z; }
    } else if (h == 0) {
        float* Fl = Fm + 3 * r.slot;
        Fl[0] += F.x; Fl[1] += F.y; Fl[2] += F.z;
        float* d = dF + 3 * r.slot;
        d[0] = F.x; d[1] = F.y; d[2] = F.z;
    }
}

// Failure-detection self test of the bounded waits above, on conditions
// that never come: (1) an mbarrier that expects one arrival nobody makes,
// (2) the grid barrier with a target the counter never reaches.  Each wait
// gives up after `limit` polls; out[0], out[1] = 1 when wait (1), (2) gave up.
// One block; no copy is in flight and nothing is left waiting.
static __global__ void k_selftest_waits(unsigned* bar, uint32_t limit, int* out, int* status) {
    __shared__ __align__(8) uint64_t mb;
    if (threadIdx.x == 0) {
        mbar_init(&mb, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) out[0] = mbar_wait_bounded(&mb, 0, limit) ? 0 : 1;
    __syncthreads();
    const unsigned unreachable = __ldcg(bar) + (1u << 30);   // base far beyond any arrival
    const bool passed = grid_barrier(bar, unreachable, 1, status, limit);
    if (threadIdx.x == 0) out[1] = passed ? 0 : 1;
}

}  // namespace fl
