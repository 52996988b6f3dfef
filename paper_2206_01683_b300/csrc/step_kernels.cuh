// step_kernels.cuh -- the stream-collide kernels of one time step (arXiv
// 2206.01683, Sec. III-B) and the device types and per-cell helpers that the
// other kernels of the step share.
//
//   k_stream_collide_staged  pull-stream + moments + frame force (Eq. 3) +
//                            regularized BGK/Guo collision + non-equilibrium
//                            extrapolation, fused; persistent blocks stage the
//                            27 source rows of each row group in shared memory
//                            with bulk copies (TMA), double buffered
//   k_stream_collide         the same update, one thread per cell with direct
//                            global loads (any row length)
//
// The IB kernels are in ib_kernels.cuh, the force/torque/mass reduction in
// reduce_kernels.cuh and the state-access kernels in state_kernels.cuh.
//
// Layout per environment: populations g[27][nslot] with g_i = f_i - w_i (the
// deviation from the fluid at rest) in storage type S; slot = x + P (y + ny z)
// with the row pitch P = nx rounded up to a multiple of 8, so every row starts
// on a 32-byte (FP32) / 16-byte (FP16) boundary.  Slots x >= nx are padding
// and never read.  Arithmetic is FP32; the force/torque and mass sums are
// compensated FP32 pairs, evaluated in FP64 on the host.
#pragma once

#include "async_copy.cuh"
#include "lattice.cuh"

namespace fl {

constexpr int K1_THREADS = 256;  // threads of either stream-collide kernel
constexpr int IB_THREADS = 256;  // 8 markers per block
constexpr int RED_THREADS = 256;
constexpr int MAX_SEG = 16;
constexpr int FT_ROW = (MAX_SEG + 1) * 6;  // force/torque doubles per environment
constexpr int HIST_ROW = FT_ROW + 1;       // + mass
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // mbarrier polls before giving up

enum { BC_PERIODIC = 0, BC_VELOCITY = 1, BC_OUTFLOW = 2, BC_FREESLIP = 3 };
enum { ST_NUMERIC = 1, ST_BAD_MARKER = 2, ST_TIMEOUT = 4, ST_MASS_DRIFT = 8 };

// Static description of one environment on the device.
struct EnvDev {
    int n[3];                 // nx, ny, nz
    int P;                    // row pitch (slots), multiple of 8
    uint32_t nslot;           // P ny nz: stride between population planes
    uint32_t rows;            // ny nz
    FastDiv div_P, div_ny;
    int bc[6];                // face kinds -x,+x,-y,+y,-z,+z
    int per[3];               // axis periodic
    float keep;               // 1 - 1/tau
    float guo;                // 1 - 1/(2 tau)
    float u_in[3];
    float drho_out;           // outflow density - 1
    unsigned long long pop_off;   // first element of this environment's g[27][nslot]
    unsigned long long slot_off;  // first slot in per-slot arrays (IB force density)
    int block0, nblocks;      // blocks of the plain stream-collide kernel
    int group0, ngroups;      // row groups of the staged kernel
    int rpg;                  // rows per group
    int part0, nparts;        // mass partials written by the kernel in use
    int bblock0, nbblocks;    // in-place layout: blocks of the boundary-cell kernel
    int nbnd;                 // in-place layout: cells the boundary-cell kernel updates
    int stamp_off;            // first 32-slot tile stamp
    int mk_begin;             // first marker in the compact marker numbering
    int n_markers;
    int marker_off;           // first marker slot in the marker arrays
    int nseg;
    double ref[3];            // torque reference point
    float mass_ref;           // mass watchdog: reference sum (rho - 1) and the
    float mass_tol;           // largest allowed |change| (<= 0: off)
};

// Frame motion of one environment (Eq. 3), refreshed by fg_step.  Besides
// the raw quantities it carries the affine form of the velocity-independent
// fictitious acceleration, a0(p) = c0 - M p with M = [domega]x +
// [omega]x [omega]x and c0 = -acc + M origin ([v]x r = v x r), computed on the
// host, so a cell evaluates it with 9 multiply-adds.
struct FrameDev {
    float acc[3], om[3], dom[3], org[3];
    float inv_1pom2;          // 1 / (1 + |omega|^2)
    float M[9];               // row-major
    float c0[3];
};

// Per-step values kept on the device, so that a captured step can be
// replayed unchanged: the tile stamp of the current step (never 0), the step
// number (history row), and a count of environments whose reduction is done.
// The last block of k_reduce to finish advances stamp and step.
struct StepState {
    uint32_t stamp;
    int envs_done;
    long long step;
};

// Environment owning index v: the last e with key(e) <= v.
template <int (EnvDev::*KEY)>
__device__ __forceinline__ int env_of(const EnvDev* __restrict__ envs, int n_envs, int v) {
    int lo = 0, hi = n_envs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (envs[mid].*KEY <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Fictitious acceleration of Eq. 3 without the Coriolis term:
// a0 = -acc - domega x r - omega x (omega x r), r = x - origin.
__device__ __forceinline__ void frame_accel(const FrameDev& F, float x, float y, float z, float a[3]) {
    const float rx = x - F.org[0], ry = y - F.org[1], rz = z - F.org[2];
    const float t1x = F.dom[1] * rz - F.dom[2] * ry;
    const float t1y = F.dom[2] * rx - F.dom[0] * rz;
    const float t1z = F.dom[0] * ry - F.dom[1] * rx;
    const float wx = F.om[1] * rz - F.om[2] * ry;
    const float wy = F.om[2] * rx - F.om[0] * rz;
    const float wz = F.om[0] * ry - F.om[1] * rx;
    const float t3x = F.om[1] * wz - F.om[2] * wy;
    const float t3y = F.om[2] * wx - F.om[0] * wz;
    const float t3z = F.om[0] * wy - F.om[1] * wx;
    a[0] = -F.acc[0] - t1x - t3x;
    a[1] = -F.acc[1] - t1y - t3y;
    a[2] = -F.acc[2] - t1z - t3z;
}

// Slot offsets that move a pull source p by -c along each axis, with
// periodic wrap: *m for c = +1 (source p - 1), *p for c = -1 (source p + 1).
// Along a non-periodic axis p is never on the outer layer, so no wrap occurs.
struct PullOffsets {
    int xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ PullOffsets pull_offsets(const EnvDev& E, int px, int py, int pz) {
    PullOffsets o;
    const int nx = E.n[0], ny = E.n[1], nz = E.n[2], P = E.P, plane = E.P * E.n[1];
    o.xm = (px == 0) ? nx - 1 : -1;
    o.xp = (px == nx - 1) ? -(nx - 1) : 1;
    o.ym = (py == 0) ? (ny - 1) * P : -P;
    o.yp = (py == ny - 1) ? -(ny - 1) * P : P;
    o.zm = (pz == 0) ? (nz - 1) * plane : -plane;
    o.zp = (pz == nz - 1) ? -(nz - 1) * plane : plane;
    return o;
}

__device__ __forceinline__ int pull_off(const PullOffsets& o, int i) {
    const int a = cx(i) == 1 ? o.xm : (cx(i) == -1 ? o.xp : 0);
    const int b = cy(i) == 1 ? o.ym : (cy(i) == -1 ? o.yp : 0);
    const int c = cz(i) == 1 ? o.zm : (cz(i) == -1 ? o.zp : 0);
    return a + b + c;
}

// Post-stream moments of the deviation g: dr = sum g, j = sum c g,
// s_ab = sum c_a c_b g.  (rho = 1 + dr, Pi = s + cs2 I.)
struct Moments {
    float dr, jx, jy, jz, sxx, syy, szz, sxy, sxz, syz;
};

template <bool SECOND>
__device__ __forceinline__ void accumulate(Moments& m, const float (&g)[Q]) {
    // Sums by x-lines first: for each (cy, cz) the line sum s, the odd part
    // d = g(+x) - g(-x) and the even part e = g(+x) + g(-x); then by y- and
    // z-lines.  About 80 additions instead of 171 term by term.
    float sl[9], dl[9], el[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {           // l = (cy+1) + 3 (cz+1); i = 3 l + (cx+1)
        el[l] = g[3 * l + 2] + g[3 * l];
        dl[l] = g[3 * l + 2] - g[3 * l];
        sl[l] = el[l] + g[3 * l + 1];
    }
    float dr = 0.f, jx = 0.f, sxx = 0.f;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        dr += sl[l];
        jx += dl[l];
        if (SECOND) sxx += el[l];
    }
    // y-lines (per cz) and z-lines (per cy)
    float jy = 0.f, syy = 0.f, jz = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float yp = sl[2 + 3 * k], ym = sl[0 + 3 * k];     // cy = +1 / -1 at cz = k - 1
        const float zp = sl[k + 6], zm = sl[k];                 // cz = +1 / -1 at cy = k - 1
        jy += yp - ym;
        jz += zp - zm;
        if (SECOND) {
            syy += yp + ym;
            szz += zp + zm;
            sxy += dl[2 + 3 * k] - dl[0 + 3 * k];
            sxz += dl[k + 6] - dl[k];
        }
    }
    m.dr += dr; m.jx += jx; m.jy += jy; m.jz += jz;
    if (SECOND) {
        // sum cy cz s = (s(+,+) - s(+,-)) - (s(-,+) - s(-,-))
        const float syz = (sl[8] - sl[2]) - (sl[6] - sl[0]);
        m.sxx += sxx; m.syy += syy; m.szz += szz; m.sxy += sxy; m.sxz += sxz; m.syz += syz;
    }
}

// The moments from the 27 values as stored and widened to float (S::widen):
// FP32 stores g_i itself; the reduced formats store h_i = s_i g_i with
// s_i = 4^(1 + |c_i|^2).  Along x-line l (cy, cz fixed, q = |cy| + |cz|) the
// cx = +-1 values share the scale sig = 4^(2 + q) and the cx = 0 value has
// sig / 4, so e' = h+ + h-, d' = h+ - h- and s' = 4 h0 + e' (one fused
// multiply-add) are sig times the line sums of accumulate, exactly (powers
// of two commute with rounding).  Each of accumulate's later additions of a
// line quantity becomes a fused multiply-add with the exact product
// (line quantity) x 1/sig, so every sum rounds as in accumulate and the
// moments are bit-identical to accumulate of the decoded values.  The
// instruction count is that of accumulate after the compiler contracts its
// exact decode multiplies into the sums (ncu: 588 instructions per cell
// either way); the kernel measured 1% faster (98.6 against 99.9 us, FP16).
template <class S, bool SECOND>
__device__ __forceinline__ void accumulate_stored(Moments& m, const float (&h)[Q]) {
    if constexpr (!S::SCALED) {
        accumulate<SECOND>(m, h);
    } else {
        // 1/sig of line l = (cy+1) + 3 (cz+1)
        auto inv_sig = [](int l) -> float {
            const int q = (l % 3 != 1 ? 1 : 0) + (l / 3 != 1 ? 1 : 0);
            return q == 0 ? 1.0f / 16.0f : (q == 1 ? 1.0f / 64.0f : 1.0f / 256.0f);
        };
        float sl[9], dl[9], el[9];
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            el[l] = h[3 * l + 2] + h[3 * l];
            dl[l] = h[3 * l + 2] - h[3 * l];
            sl[l] = __fmaf_rn(h[3 * l + 1], 4.0f, el[l]);
        }
        float dr = 0.f, jx = 0.f, sxx = 0.f;
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            dr = __fmaf_rn(sl[l], inv_sig(l), dr);
            jx = __fmaf_rn(dl[l], inv_sig(l), jx);
            if (SECOND) sxx = __fmaf_rn(el[l], inv_sig(l), sxx);
        }
        float jy = 0.f, syy = 0.f, jz = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float wy = inv_sig(3 * k), wz = inv_sig(k);   // lines 3k, 2 + 3k and k, k + 6 pair up
            const float yp = sl[2 + 3 * k], ym = sl[0 + 3 * k];
            const float zp = sl[k + 6], zm = sl[k];
            jy = __fmaf_rn(yp - ym, wy, jy);
            jz = __fmaf_rn(zp - zm, wz, jz);
            if (SECOND) {
                syy = __fmaf_rn(yp + ym, wy, syy);
                szz = __fmaf_rn(zp + zm, wz, szz);
                sxy = __fmaf_rn(dl[2 + 3 * k] - dl[0 + 3 * k], wy, sxy);
                sxz = __fmaf_rn(dl[k + 6] - dl[k], wz, sxz);
            }
        }
        m.dr += dr; m.jx += jx; m.jy += jy; m.jz += jz;
        if (SECOND) {
            const float syz = ((sl[8] - sl[2]) - (sl[6] - sl[0])) * (1.0f / 256.0f);
            m.sxx += sxx; m.syy += syy; m.szz += szz; m.sxy += sxy; m.sxz += sxz; m.syz += syz;
        }
    }
}

// Moments at source slot p by direct (L2-cached) global loads.
template <class S, bool SECOND>
__device__ __forceinline__ Moments pull_moments(const typename S::raw* __restrict__ G, uint32_t nslot,
                                                uint32_t p, const PullOffsets& o) {
    Moments m = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int idx = (int)p + pull_off(o, i);
        g[i] = FG_IN_RANGE(DBG_PULL, idx, nslot) ? S::widen(__ldg(G + (size_t)i * nslot + (uint32_t)idx)) : 0.0f;
    }
    accumulate_stored<S, SECOND>(m, g);
    return m;
}

// ------------------------------------------------ population layouts
// Where the populations arriving at a cell p in the coming step are stored.
//   LAYOUT_PULL  two buffers: population i arrives from (i, p - c_i) of the
//                input buffer (the post-collision state of the last step).
//   LAYOUT_AA0   one buffer in place (AA pattern), even phase: (i, p) holds it.
//   LAYOUT_AA1   one buffer in place, odd phase: (26 - i, p - c_i) holds it.
// (direction, slot) pairs; aa_kernels.cuh describes the in-place layout.
enum { LAYOUT_PULL = 0, LAYOUT_AA0 = 1, LAYOUT_AA1 = 2 };

// Moments of the populations arriving at slot p under a layout.  NC reads
// through the non-coherent path (the array is not written by the launch);
// the in-place step kernels read with ordinary loads.
template <class S, bool SECOND, int LAYOUT, bool NC = true>
__device__ __forceinline__ Moments layout_moments(const typename S::raw* G, uint32_t nslot, uint32_t p,
                                                  const PullOffsets& o) {
    Moments m = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int idx = LAYOUT == LAYOUT_AA0 ? (int)p : (int)p + pull_off(o, i);
        const int dir = LAYOUT == LAYOUT_AA1 ? Q - 1 - i : i;
        const typename S::raw* q = G + (size_t)dir * nslot + (uint32_t)idx;
        g[i] = FG_IN_RANGE(DBG_PULL, idx, nslot) ? S::widen(NC ? __ldg(q) : *q) : 0.0f;
    }
    accumulate_stored<S, SECOND>(m, g);
    return m;
}

// Location of the post-collision population i of cell (x, y, z) (slot s):
// the slot returned, the direction in *dir.  aa < 0: the two-buffer layout,
// (i, s); aa = 1: (26 - i, s); aa = 0: (i, s + c_i) with periodic wrap, or
// (26 - i, s) where s + c_i lies beyond an open face.
__device__ __forceinline__ uint32_t post_loc(const EnvDev& E, int aa, int i, int x, int y, int z, uint32_t s,
                                             int* dir) {
    if (aa < 0) {
        *dir = i;
        return s;
    }
    *dir = Q - 1 - i;
    if (aa == 1) return s;
    int p[3] = {x + cx(i), y + cy(i), z + cz(i)};
    for (int a = 0; a < 3; ++a) {
        const int n = E.n[a];
        if (p[a] < 0 || p[a] >= n) {
            if (!E.per[a]) return s;
            p[a] = p[a] < 0 ? p[a] + n : p[a] - n;
        }
    }
    *dir = i;
    return (uint32_t)p[0] + (uint32_t)E.P * ((uint32_t)p[1] + (uint32_t)E.n[1] * (uint32_t)p[2]);
}

// A sum kept as an unevaluated pair hi + lo of FP32 numbers (compensated
// summation, close to FP64 accuracy for these sums).  B300 runs FP64 --
// conversions included -- at a small fraction of its FP32 rate and with long
// latency, so the reduction trees stay in FP32 pairs and each result is
// evaluated in FP64 once, at the end.
struct Pair32 {
    float hi = 0.f, lo = 0.f;
    // add one term (Kahan/Neumaier step)
    __device__ __forceinline__ void add(float v) {
        const float t = hi + v;
        lo += fabsf(hi) >= fabsf(v) ? (hi - t) + v : (v - t) + hi;
        hi = t;
    }
    // add another pair (TwoSum of the high parts, low parts carried)
    __device__ __forceinline__ void add(const Pair32& o) {
        const float s = hi + o.hi;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (o.hi - bp);
        hi = s;
        lo += o.lo + err;
    }
};

// Constants of the cell update for one environment and step, gathered so a
// kernel can hold them in registers instead of re-reading them per cell.
struct CellConsts {
    float keep, guo, drho_out;
    float u_in[3];
    int bc;                   // 2 bits per face, faces -x,+x,-y,+y,-z,+z
    float om[3], inv_1pom2;
    float c0[3], M[9];
    uint32_t nslot;
};

__device__ __forceinline__ CellConsts load_consts(const EnvDev& E, const FrameDev& F) {
    CellConsts C;
    C.keep = E.keep; C.guo = E.guo; C.drho_out = E.drho_out;
    int bc = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) bc |= (E.bc[k] & 3) << (2 * k);
    C.bc = bc;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C.u_in[a] = E.u_in[a];
        C.om[a] = F.om[a];
        C.c0[a] = F.c0[a];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) C.M[k] = F.M[k];
    C.inv_1pom2 = F.inv_1pom2;
    C.nslot = E.nslot;
    return C;
}

__device__ __forceinline__ int face_kind(int bc, int face) { return (bc >> (2 * face)) & 3; }

// ------------------------------------------------ the per-cell update

// Hermite coefficients of one cell's post-collision deviation, pre-multiplied
// by S::POLY (see line_values), and rho_out - 1.
struct Herm {
    float A, dxx, dyy, dzz, oxy, oxz, oyz, tx, ty, tz;
    float k3, u3x, u3y, u3z, uu3;   // third-order terms (EQ3 only)
    float drout;
};

// Collision (interior) or open-face rule (boundary) from the pulled moments
// m, as the coefficients of the Hermite-2 rebuild of all 27 outputs.
// (sx, sy, sz) is the inward normal of the non-periodic faces the cell lies
// on (0 for interior cells).  EQ3 adds the third-order equilibrium terms the
// lattice carries,
// w_i rho [(c.u)^3 - (c.u)|u|^2] / (2 cs2^3) = 4.5 w_i rho (c.u)((c.u)^2 - |u|^2)
// (the Hermite sum over the index triples that are not all equal: H_aaa
// vanishes on D3Q27), with the collision's (rho, u) inside and (rho_b, u_b)
// on the open faces.
template <class S, bool EQ3 = false>
__device__ __forceinline__ Herm cell_coeffs(const CellConsts& F, const Moments& m, int x, int y, int z, int sx,
                                            int sy, int sz, float fx, float fy, float fz) {
    const float cs2 = 1.0f / 3.0f;
    const float rho = 1.0f + m.dr;
    const float inv = 1.0f / rho;
    float drout, Jx, Jy, Jz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz;
    float r3 = 0.f, u3x = 0.f, u3y = 0.f, u3z = 0.f;   // (rho, u) of the third-order terms
    if ((sx | sy | sz) == 0) {
        // a0 = c0 - M p (the affine form of Eq. 3 without Coriolis)
        const float px = (float)x, py = (float)y, pz = (float)z;
        float a0[3];
        a0[0] = F.c0[0] - (F.M[0] * px + F.M[1] * py + F.M[2] * pz);
        a0[1] = F.c0[1] - (F.M[3] * px + F.M[4] * py + F.M[5] * pz);
        a0[2] = F.c0[2] - (F.M[6] * px + F.M[7] * py + F.M[8] * pz);
        // v = j/rho + a0/2 + fib/(2 rho);  u = (v - w x v + (w.v) w)/(1 + |w|^2)
        const float vx = (m.jx + 0.5f * fx) * inv + 0.5f * a0[0];
        const float vy = (m.jy + 0.5f * fy) * inv + 0.5f * a0[1];
        const float vz = (m.jz + 0.5f * fz) * inv + 0.5f * a0[2];
        const float wv = F.om[0] * vx + F.om[1] * vy + F.om[2] * vz;
        const float ux = (vx - (F.om[1] * vz - F.om[2] * vy) + wv * F.om[0]) * F.inv_1pom2;
        const float uy = (vy - (F.om[2] * vx - F.om[0] * vz) + wv * F.om[1]) * F.inv_1pom2;
        const float uz = (vz - (F.om[0] * vy - F.om[1] * vx) + wv * F.om[2]) * F.inv_1pom2;
        // G = rho a0 + fib - 2 rho w x u  (Eq. 3 with the IB force)
        const float Gx = rho * a0[0] + fx - 2.0f * rho * (F.om[1] * uz - F.om[2] * uy);
        const float Gy = rho * a0[1] + fy - 2.0f * rho * (F.om[2] * ux - F.om[0] * uz);
        const float Gz = rho * a0[2] + fz - 2.0f * rho * (F.om[0] * uy - F.om[1] * ux);
        Jx = m.jx + Gx; Jy = m.jy + Gy; Jz = m.jz + Gz;
        // Q = Pi* - rho cs2 I = rho u u + (1 - 1/tau)(Pi - Pi_eq) + (1 - 1/(2tau))(u G + G u),
        // with Pi - Pi_eq = s - dr cs2 I - rho u u
        const float k = F.keep, gq = F.guo;
        const float ruxx = rho * ux * ux, ruyy = rho * uy * uy, ruzz = rho * uz * uz;
        const float ruxy = rho * ux * uy, ruxz = rho * ux * uz, ruyz = rho * uy * uz;
        Qxx = ruxx + k * (m.sxx - m.dr * cs2 - ruxx) + gq * 2.0f * ux * Gx;
        Qyy = ruyy + k * (m.syy - m.dr * cs2 - ruyy) + gq * 2.0f * uy * Gy;
        Qzz = ruzz + k * (m.szz - m.dr * cs2 - ruzz) + gq * 2.0f * uz * Gz;
        Qxy = ruxy + k * (m.sxy - ruxy) + gq * (ux * Gy + Gx * uy);
        Qxz = ruxz + k * (m.sxz - ruxz) + gq * (ux * Gz + Gx * uz);
        Qyz = ruyz + k * (m.syz - ruyz) + gq * (uy * Gz + Gy * uz);
        drout = m.dr;
        if constexpr (EQ3) {
            r3 = rho; u3x = ux; u3y = uy; u3z = uz;
        }
    } else {
        // non-equilibrium extrapolation (m are the moments of x_f = x + n):
        // f* = f_eq(rho_b, u_b) + (1 - 1/tau) f_neq(x_f); x-faces govern on edges
        const float ufx = m.jx * inv, ufy = m.jy * inv, ufz = m.jz * inv;
        const int gov = sx != 0 ? 0 : (sy != 0 ? 1 : 2);
        const int gs = gov == 0 ? sx : (gov == 1 ? sy : sz);
        const int kind = face_kind(F.bc, 2 * gov + (gs < 0 ? 1 : 0));
        float ubx = ufx, uby = ufy, ubz = ufz;
        drout = m.dr;
        if (kind == BC_VELOCITY) {
            ubx = F.u_in[0]; uby = F.u_in[1]; ubz = F.u_in[2];
        } else if (kind == BC_OUTFLOW) {
            drout = F.drho_out;
        } else {
            if (sx != 0 && face_kind(F.bc, sx < 0 ? 1 : 0) == BC_FREESLIP) ubx = 0.f;
            if (sy != 0 && face_kind(F.bc, sy < 0 ? 3 : 2) == BC_FREESLIP) uby = 0.f;
            if (sz != 0 && face_kind(F.bc, sz < 0 ? 5 : 4) == BC_FREESLIP) ubz = 0.f;
        }
        const float rb = 1.0f + drout;
        const float k = F.keep;
        Jx = rb * ubx; Jy = rb * uby; Jz = rb * ubz;
        Qxx = rb * ubx * ubx + k * (m.sxx - m.dr * cs2 - rho * ufx * ufx);
        Qyy = rb * uby * uby + k * (m.syy - m.dr * cs2 - rho * ufy * ufy);
        Qzz = rb * ubz * ubz + k * (m.szz - m.dr * cs2 - rho * ufz * ufz);
        Qxy = rb * ubx * uby + k * (m.sxy - rho * ufx * ufy);
        Qxz = rb * ubx * ubz + k * (m.sxz - rho * ufx * ufz);
        Qyz = rb * uby * ubz + k * (m.syz - rho * ufy * ufz);
        if constexpr (EQ3) {
            r3 = rb; u3x = ubx; u3y = uby; u3z = ubz;
        }
    }
    Herm h;
    h.k3 = S::POLY * 4.5f * r3;
    h.u3x = u3x; h.u3y = u3y; h.u3z = u3z;
    h.uu3 = u3x * u3x + u3y * u3y + u3z * u3z;
    // Hermite-2 rebuild of the deviation: g*_i = w_i [dr + 3 c.J + 4.5 c c : Q - 1.5 tr Q]
    const float sc = S::POLY;
    h.A = sc * (drout - 1.5f * (Qxx + Qyy + Qzz));
    h.dxx = sc * 4.5f * Qxx; h.dyy = sc * 4.5f * Qyy; h.dzz = sc * 4.5f * Qzz;
    h.oxy = sc * 9.0f * Qxy; h.oxz = sc * 9.0f * Qxz; h.oyz = sc * 9.0f * Qyz;
    h.tx = sc * 3.0f * Jx; h.ty = sc * 3.0f * Jy; h.tz = sc * 3.0f * Jz;
    h.drout = drout;
    return h;
}

// The three outputs of x-line l (cy = l % 3 - 1, cz = l / 3 - 1), organised
// as v(cx) = E + cx^2 dxx + O + cx B with
//   E = A + cy^2 dyy + cz^2 dzz + cy cz oyz,  O = cy ty + cz tz,  B = tx + cy oxy + cz oxz;
// v0, vp, vm for cx = 0, +1, -1 (population 3 l + 1, 3 l + 2, 3 l).
template <bool EQ3>
__device__ __forceinline__ void line_values(const Herm& h, int l, float& v0, float& vp, float& vm) {
    const int ly = l % 3 - 1, lz = l / 3 - 1;      // this line's cy, cz
    float E = h.A, O = 0.0f, B = h.tx;
    if (ly != 0) E += h.dyy;
    if (lz != 0) E += h.dzz;
    if (ly * lz == 1) E += h.oyz; else if (ly * lz == -1) E -= h.oyz;
    if (ly == 1) O += h.ty; else if (ly == -1) O -= h.ty;
    if (lz == 1) O += h.tz; else if (lz == -1) O -= h.tz;
    if (ly == 1) B += h.oxy; else if (ly == -1) B -= h.oxy;
    if (lz == 1) B += h.oxz; else if (lz == -1) B -= h.oxz;
    v0 = E + O;
    const float v1 = v0 + h.dxx;
    vp = v1 + B;
    vm = v1 - B;
    if constexpr (EQ3) {   // c.u = cx u_x + b on this line
        float b = 0.0f;
        if (ly == 1) b += h.u3y; else if (ly == -1) b -= h.u3y;
        if (lz == 1) b += h.u3z; else if (lz == -1) b -= h.u3z;
        const float cp = b + h.u3x, cm = b - h.u3x;
        v0 += h.k3 * b * (b * b - h.uu3);
        vp += h.k3 * cp * (cp * cp - h.uu3);
        vm += h.k3 * cm * (cm * cm - h.uu3);
    }
}

// Collision and rebuild of one cell, all 27 outputs stored at slot.
// Returns rho_out - 1 for the mass sum.
template <class S, bool EQ3 = false>
__device__ __forceinline__ float update_cell(const CellConsts& F, const Moments& m, int x, int y, int z, int sx,
                                             int sy, int sz, float fx, float fy, float fz,
                                             typename S::raw* __restrict__ Go, uint32_t slot) {
    const Herm h = cell_coeffs<S, EQ3>(F, m, x, y, z, sx, sy, sz, fx, fy, fz);
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        float v0, vp, vm;
        line_values<EQ3>(h, l, v0, vp, vm);
        if (FG_IN_RANGE(DBG_STORE, slot, F.nslot)) {
            S::emit(Go + (size_t)(3 * l + 1) * F.nslot + slot, v0, 3 * l + 1);   // cx = 0
            S::emit(Go + (size_t)(3 * l + 2) * F.nslot + slot, vp, 3 * l + 2);   // cx = +1
            S::emit(Go + (size_t)(3 * l) * F.nslot + slot, vm, 3 * l);           // cx = -1
        }
    }
    return h.drout;
}

// The outputs of two neighbouring cells a (at an even slot) and b (slot + 1),
// stored as pairs.
template <class S, bool EQ3>
__device__ __forceinline__ void emit_pair(const Herm& a, const Herm& b, typename S::raw* __restrict__ Go,
                                          uint32_t nslot, uint32_t slot) {
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        float a0, ap, am, b0, bp, bm;
        line_values<EQ3>(a, l, a0, ap, am);
        line_values<EQ3>(b, l, b0, bp, bm);
        if (FG_IN_RANGE(DBG_STORE, slot + 1, nslot)) {
            S::emit2(Go + (size_t)(3 * l + 1) * nslot + slot, a0, b0, 3 * l + 1);
            S::emit2(Go + (size_t)(3 * l + 2) * nslot + slot, ap, bp, 3 * l + 2);
            S::emit2(Go + (size_t)(3 * l) * nslot + slot, am, bm, 3 * l);
        }
    }
}

// Inward normal along one axis for coordinate v (0 on periodic axes).
__device__ __forceinline__ int inward(const EnvDev& E, int axis, int v) {
    if (E.per[axis]) return 0;
    return v == 0 ? 1 : (v == E.n[axis] - 1 ? -1 : 0);
}

// IB force density at a slot if its 32-slot tile was stamped this step; the
// stored value is cleared so the field is zero again for the next step.
// COHERENT reads the stamp and the force through L2 (ld.global.cg), for a
// kernel in which other blocks wrote them earlier in the same launch.
template <bool COHERENT = false>
__device__ __forceinline__ void take_ib_force(const EnvDev& E, float4* __restrict__ fib,
                                              const uint32_t* __restrict__ stamps, uint32_t stamp,
                                              uint32_t slot, float& fx, float& fy, float& fz) {
    fx = fy = fz = 0.f;
    const uint32_t* sp = stamps + E.stamp_off + (slot >> 5);
    if ((COHERENT ? __ldcg(sp) : __ldg(sp)) == stamp) {
        float4* fb = fib + E.slot_off + slot;
        const float4 f = COHERENT ? __ldcg(fb) : *fb;
        fx = f.x; fy = f.y; fz = f.z;
        *fb = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ------------------------------------------------- K1: stream + collide

// Programmatic dependent launch (PTX griddepcontrol).  A kernel launched with
// programmatic stream serialization may start once every block of the kernel
// before it has called allow_dependents (or exited), and must call
// wait_prerequisites before it reads that kernel's results: the wait returns
// when the earlier kernel has completed and its writes are visible.  Both
// are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_prerequisites() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float block_sum_f32(float v, float* wsum) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < K1_THREADS / 32; ++w) t += wsum[w];
    return t;  // valid in thread 0
}

// The cells of plain-kernel block b of environment E (b counted from the
// environment's first block): one cell per thread, or with PAIR two
// neighbouring cells (x even and x + 1) per thread.  Returns the thread's
// sum of rho_out - 1.  C holds the environment's constants.
template <class S, bool EQ3, bool PAIR, bool COHERENT = false>
__device__ __forceinline__ float plain_block_cells(const typename S::raw* __restrict__ gin,
                                                   typename S::raw* __restrict__ gout, const EnvDev& E,
                                                   const CellConsts& C, int b, float4* __restrict__ fib,
                                                   const uint32_t* __restrict__ stamps, uint32_t stamp) {
    float drout = 0.0f;
    if constexpr (PAIR) {
        // cells x (even) and x + 1 of one row; every row length is even, so
        // both are real cells and share a 32-slot tile
        const uint32_t c = ((uint32_t)b * K1_THREADS + threadIdx.x) * 2u;
        if (c < E.nslot) {
            const uint32_t row = fdiv(c, E.div_P);
            const int x = (int)(c - row * (uint32_t)E.P);
            if (x < E.n[0]) {
                const uint32_t zz = fdiv(row, E.div_ny);
                const int y = (int)(row - zz * (uint32_t)E.n[1]);
                const int z = (int)zz;
                float fa[3], fb[3];
                take_ib_force<COHERENT>(E, fib, stamps, stamp, c, fa[0], fa[1], fa[2]);
                take_ib_force<COHERENT>(E, fib, stamps, stamp, c + 1, fb[0], fb[1], fb[2]);
                const int sxa = inward(E, 0, x), sxb = inward(E, 0, x + 1);
                const int sy = inward(E, 1, y), sz = inward(E, 2, z);
                const int ry = (sy + sz * E.n[1]) * E.P;
                const Moments ma = pull_moments<S, true>(gin + E.pop_off, E.nslot, (uint32_t)((int)c + sxa + ry),
                                                         pull_offsets(E, x + sxa, y + sy, z + sz));
                const Moments mb = pull_moments<S, true>(gin + E.pop_off, E.nslot,
                                                         (uint32_t)((int)c + 1 + sxb + ry),
                                                         pull_offsets(E, x + 1 + sxb, y + sy, z + sz));
                const Herm ha = cell_coeffs<S, EQ3>(C, ma, x, y, z, sxa, sy, sz, fa[0], fa[1], fa[2]);
                const Herm hb = cell_coeffs<S, EQ3>(C, mb, x + 1, y, z, sxb, sy, sz, fb[0], fb[1], fb[2]);
                drout = ha.drout + hb.drout;
                emit_pair<S, EQ3>(ha, hb, gout + E.pop_off, E.nslot, c);
            }
        }
    } else {
        const uint32_t c = (uint32_t)b * K1_THREADS + threadIdx.x;
        if (c < E.nslot) {
            const uint32_t row = fdiv(c, E.div_P);
            const int x = (int)(c - row * (uint32_t)E.P);
            if (x < E.n[0]) {
                const uint32_t zz = fdiv(row, E.div_ny);
                const int y = (int)(row - zz * (uint32_t)E.n[1]);
                const int z = (int)zz;
                float fx, fy, fz;
                take_ib_force<COHERENT>(E, fib, stamps, stamp, c, fx, fy, fz);
                const int sx = inward(E, 0, x), sy = inward(E, 1, y), sz = inward(E, 2, z);
                // a boundary cell takes its moments from the inward neighbour x_f
                const int px = x + sx, py = y + sy, pz = z + sz;
                const uint32_t p = (uint32_t)((int)c + sx + (sy + sz * E.n[1]) * E.P);
                const PullOffsets o = pull_offsets(E, px, py, pz);
                const Moments m = pull_moments<S, true>(gin + E.pop_off, E.nslot, p, o);
                drout = update_cell<S, EQ3>(C, m, x, y, z, sx, sy, sz, fx, fy, fz, gout + E.pop_off, c);
            }
        }
    }
    return drout;
}

// Which blocks of the plain kernel a launch updates: all of them, or, when
// the IB runs beside the stream-collide kernel, only the blocks that no
// stencil node of this step falls in (their flag is not this step's stamp)
// or only those that one does.
enum { K1_ALL_BLOCKS = 0, K1_UNFLAGGED_BLOCKS = 1, K1_FLAGGED_BLOCKS = 2 };

// Plain variant: one thread per slot (two with PAIR), direct loads.
template <class S, bool EQ3 = false, bool PAIR = false>
__global__ void __launch_bounds__(K1_THREADS)
k_stream_collide(const typename S::raw* __restrict__ gin, typename S::raw* __restrict__ gout,
                 const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames, int n_envs,
                 float4* __restrict__ fib, const uint32_t* __restrict__ stamps, const StepState* __restrict__ st,
                 Pair32* __restrict__ mass_part, const uint32_t* __restrict__ blk_flag = nullptr,
                 int which = K1_ALL_BLOCKS, int reverse = 0) {
    __shared__ float wsum[K1_THREADS / 32];
    __shared__ CellConsts C;   // the block's environment constants, read by every cell
    const uint32_t stamp = st->stamp;
    // reverse: blocks taken from the end of the domain first (alternate
    // steps sweep in opposite directions, so a step starts where the last
    // one ended, on outputs still in L2)
    const int b = reverse ? (int)(gridDim.x - 1u - blockIdx.x) : (int)blockIdx.x;
    if (which != K1_ALL_BLOCKS && (__ldg(blk_flag + b) == stamp) != (which == K1_FLAGGED_BLOCKS)) return;
    const int e = n_envs > 1 ? env_of<&EnvDev::block0>(envs, n_envs, b) : 0;
    const EnvDev& E = envs[e];
    if (threadIdx.x == 0) C = load_consts(E, frames[e]);
    __syncthreads();
    // the step's reduction may start its marker sums once the last wave of
    // blocks is in (it waits for this kernel before it reads the mass sums)
    allow_dependents();
    const float drout = plain_block_cells<S, EQ3, PAIR>(gin, gout, E, C, b - E.block0, fib, stamps, stamp);
    const float t = block_sum_f32(drout, wsum);
    if (threadIdx.x == 0) {
        Pair32 p;
        p.hi = t;
        mass_part[b] = p;
    }
}

// Staged variant: persistent blocks walk row groups g = blockIdx.x,
// blockIdx.x + gridDim.x, ...  For each group, warp 0 issues one bulk copy per
// (population, row) of the source row it pulls from -- row (y + sy - cy,
// z + sz - cz), whole rows of P slots -- into shared memory, completing on an
// mbarrier.  The next group's copies are in flight while the current group
// is computed from shared memory (two buffers).  Shared memory holds each
// population at a fixed stride of GC slots, so the 27 loads of a cell differ
// only by immediate offsets.  Outputs go straight to global memory.
template <class S, int GC>
__device__ __forceinline__ void issue_group(const EnvDev& E, int g_local, const typename S::raw* __restrict__ gin,
                                            typename S::raw* buf, uint64_t* bar) {
    // Called by every thread of the block: thread 0 arrives on the barrier
    // with the byte count of the whole group, the copies are spread over the
    // threads (one per (population, row)), so no warp carries the issue alone.
    // A copy that lands before the arrival only drives the barrier's pending
    // byte count negative; the phase cannot complete before the arrival.
    typedef typename S::raw raw;
    const int r0 = g_local * E.rpg;
    const int R = min(E.rpg, (int)E.rows - r0);
    const uint32_t row_bytes = (uint32_t)E.P * (uint32_t)sizeof(raw);
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)(Q * R) * row_bytes);
    const int ny = E.n[1], nz = E.n[2];
    const raw* G = gin + E.pop_off;
    for (int k = threadIdx.x; k < Q * R; k += blockDim.x) {
        const int i = k % Q, r = k / Q;
        const int row = r0 + r;
        const int z = (int)fdiv((uint32_t)row, E.div_ny), y = row - z * ny;
        int ys = y + inward(E, 1, y) - cy(i);
        int zs = z + inward(E, 2, z) - cz(i);
        ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);   // only periodic axes wrap
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        const raw* src = G + (size_t)i * E.nslot + (size_t)(ys + ny * zs) * E.P;
        raw* dst = buf + (size_t)i * GC + (size_t)r * E.P;
        // (a skipped copy leaves the group's barrier short: its wait gives up)
        if (FG_IN_RANGE(DBG_COPY, ys, ny) && FG_IN_RANGE(DBG_COPY, zs, nz) &&
            FG_IN_RANGE(DBG_COPY, (r + 1) * E.P - 1, GC))
            bulk_g2s(dst, src, row_bytes, bar);
    }
}

// Moments of the cell at x of staged row r (rb: that row's first slot in
// population 0 of the group buffer), sx its inward x normal.
template <class S, int GC>
__device__ __forceinline__ Moments staged_moments(const typename S::raw* rb, int r, int P, int nx, int x, int sx) {
    const int xs = x + sx;
    const int xm = xs == 0 ? nx - 1 : xs - 1;      // source of c_x = +1
    const int xp = xs == nx - 1 ? 0 : xs + 1;      // source of c_x = -1
    float gv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int xi = cx(i) == 1 ? xm : (cx(i) == -1 ? xp : xs);
        gv[i] = FG_IN_RANGE(DBG_SMEM, r * P + xi, GC) ? S::widen(rb[i * GC + xi]) : 0.0f;
    }
    Moments m = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    accumulate_stored<S, true>(m, gv);
    return m;
}

// Environment scalars a cell update needs, held in registers while a block
// works through groups of one environment.
struct EnvRegs {
    int nx, ny, P, per_x, per_y, per_z, nz;
    uint32_t nslot;
    unsigned long long pop_off;
    int stamp_off;
    unsigned long long slot_off;
    FastDiv div_P, div_ny;
    int group0, rpg, rows;
};

template <class S, int GC, int MINB, bool EQ3 = false, bool PAIR = false>
__global__ void __launch_bounds__(K1_THREADS, MINB)
k_stream_collide_staged(const typename S::raw* __restrict__ gin, typename S::raw* __restrict__ gout,
                        const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames, int n_envs,
                        int total_groups, float4* __restrict__ fib, const uint32_t* __restrict__ stamps,
                        const StepState* __restrict__ st, Pair32* __restrict__ mass_part,
                        int* __restrict__ status, int reverse) {
    typedef typename S::raw raw;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    raw* bufs = reinterpret_cast<raw*>(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float wsum[2][K1_THREADS / 32];
    constexpr uint32_t BUF = (uint32_t)Q * GC;
    const uint32_t stamp = st->stamp;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    allow_dependents();   // as in k_stream_collide

    // the block walks groups blockIdx.x, blockIdx.x + gridDim.x, ... of the
    // sweep; with reverse the sweep takes group total - 1 - j as its j-th
    // (alternate steps run in opposite directions, as in k_stream_collide)
    auto group_of = [&](int j) { return reverse ? total_groups - 1 - j : j; };
    int gs = blockIdx.x;
    if (gs < total_groups) {
        const int g0 = group_of(gs);
        const int e = n_envs > 1 ? env_of<&EnvDev::group0>(envs, n_envs, g0) : 0;
        issue_group<S, GC>(envs[e], g0 - envs[e].group0, gin, bufs, &bar[0]);
    }
    int cur_e = -1;
    EnvRegs R;
    __shared__ CellConsts C;   // constants of the environment in hand, read by every cell
    __shared__ int abort_wait; // a wait gave up in this group
    if (threadIdx.x == 0) abort_wait = 0;
    for (int k = 0; gs < total_groups; gs += gridDim.x, ++k) {
        const int b = k & 1;
        const int g = group_of(gs);
        const int gn = gs + gridDim.x;
        if (gn < total_groups) {
            const int gl = group_of(gn);
            const int en = n_envs > 1 ? env_of<&EnvDev::group0>(envs, n_envs, gl) : 0;
            issue_group<S, GC>(envs[en], gl - envs[en].group0, gin, bufs + (size_t)(b ^ 1) * BUF, &bar[b ^ 1]);
        }
        const int e = n_envs > 1 ? env_of<&EnvDev::group0>(envs, n_envs, g) : 0;
        if (e != cur_e) {   // block-uniform
            const EnvDev& E = envs[e];
            R.nx = E.n[0]; R.ny = E.n[1]; R.nz = E.n[2]; R.P = E.P;
            R.per_x = E.per[0]; R.per_y = E.per[1]; R.per_z = E.per[2];
            R.nslot = E.nslot; R.pop_off = E.pop_off; R.stamp_off = E.stamp_off; R.slot_off = E.slot_off;
            R.div_P = E.div_P; R.div_ny = E.div_ny; R.group0 = E.group0; R.rpg = E.rpg; R.rows = (int)E.rows;
            __syncthreads();   // previous environment's constants no longer in use
            if (threadIdx.x == 0) C = load_consts(E, frames[e]);
            __syncthreads();
            cur_e = e;
        }
        const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)(k >> 1) & 1u, WAIT_LIMIT);
        if (!ok) abort_wait = 1;   // decided for the whole block after the group's barrier
        // With one row per group the copies come from one warp, and starting
        // the warps together after the data arrives measured faster (146.6 us
        // against 163 us on the swimmer channel); with two or more rows per
        // group letting each warp start at once measured faster (148.7 against
        // 160.2 us in FP32, 115.1 against 118.8 us in FP16).
        if constexpr (GC == 256) __syncthreads();
        const raw* sb = bufs + (size_t)b * BUF;
        const int r0 = (g - R.group0) * R.rpg;
        const int span = ok ? min(R.rpg, R.rows - r0) * R.P : 0;
        float drsum = 0.f;
        if constexpr (PAIR) {
            // two neighbouring cells (x even, x + 1) per thread, outputs stored
            // as pairs; every row length is even, so both cells are real
            // cells, share a 32-slot tile and are never both on an x face
            for (int t = threadIdx.x; 2 * t < span; t += K1_THREADS) {
                const int r = (int)fdiv((uint32_t)(2 * t), R.div_P);
                const int x = 2 * t - r * R.P;
                if (x >= R.nx) continue;
                const int row = r0 + r;
                const int z = (int)fdiv((uint32_t)row, R.div_ny);
                const int y = row - z * R.ny;
                const uint32_t slot = (uint32_t)row * (uint32_t)R.P + (uint32_t)x;
                float4 fa = make_float4(0.f, 0.f, 0.f, 0.f), fb2 = fa;
                if (__ldg(stamps + R.stamp_off + (slot >> 5)) == stamp) {
                    float4* fb = fib + R.slot_off + slot;
                    fa = fb[0];
                    fb2 = fb[1];
                    fb[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                    fb[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const int sxa = R.per_x ? 0 : (x == 0 ? 1 : 0);
                const int sxb = R.per_x ? 0 : (x + 1 == R.nx - 1 ? -1 : 0);
                const int sy = R.per_y ? 0 : (y == 0 ? 1 : (y == R.ny - 1 ? -1 : 0));
                const int sz = R.per_z ? 0 : (z == 0 ? 1 : (z == R.nz - 1 ? -1 : 0));
                const raw* rb = sb + r * R.P;
                const Herm ha = cell_coeffs<S, EQ3>(C, staged_moments<S, GC>(rb, r, R.P, R.nx, x, sxa), x, y, z,
                                                    sxa, sy, sz, fa.x, fa.y, fa.z);
                const Herm hb = cell_coeffs<S, EQ3>(C, staged_moments<S, GC>(rb, r, R.P, R.nx, x + 1, sxb), x + 1,
                                                    y, z, sxb, sy, sz, fb2.x, fb2.y, fb2.z);
                drsum += ha.drout + hb.drout;
                emit_pair<S, EQ3>(ha, hb, gout + R.pop_off, R.nslot, slot);
            }
        } else {
            for (int t = threadIdx.x; t < span; t += K1_THREADS) {
                const int r = (int)fdiv((uint32_t)t, R.div_P);
                const int x = t - r * R.P;
                if (x >= R.nx) continue;
                const int row = r0 + r;
                const int z = (int)fdiv((uint32_t)row, R.div_ny);
                const int y = row - z * R.ny;
                const uint32_t slot = (uint32_t)row * (uint32_t)R.P + (uint32_t)x;
                // IB force density of a stamped tile (cleared after use)
                float fx = 0.f, fy = 0.f, fz = 0.f;
                if (__ldg(stamps + R.stamp_off + (slot >> 5)) == stamp) {
                    float4* fb = fib + R.slot_off + slot;
                    const float4 f = *fb;
                    fx = f.x; fy = f.y; fz = f.z;
                    *fb = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const int sx = R.per_x ? 0 : (x == 0 ? 1 : (x == R.nx - 1 ? -1 : 0));
                const int sy = R.per_y ? 0 : (y == 0 ? 1 : (y == R.ny - 1 ? -1 : 0));
                const int sz = R.per_z ? 0 : (z == 0 ? 1 : (z == R.nz - 1 ? -1 : 0));
                const Moments m = staged_moments<S, GC>(sb + r * R.P, r, R.P, R.nx, x, sx);
                drsum += update_cell<S, EQ3>(C, m, x, y, z, sx, sy, sz, fx, fy, fz, gout + R.pop_off, slot);
            }
        }
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) drsum += __shfl_xor_sync(0xffffffffu, drsum, s);
        if ((threadIdx.x & 31) == 0) wsum[b][warp] = drsum;
        __syncthreads();   // buffer b is free again; wsum[b] is complete
        if (abort_wait) {
            // a copy never completed: report, let the copies in flight land, stop
            if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
            mbar_wait_bounded(&bar[b], (uint32_t)(k >> 1) & 1u, WAIT_LIMIT);
            if (gn < total_groups) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((k + 1) >> 1) & 1u, WAIT_LIMIT);
            return;
        }
        if (threadIdx.x == 0) {
            Pair32 t;
#pragma unroll
            for (int w = 0; w < K1_THREADS / 32; ++w) t.add(wsum[b][w]);
            mass_part[g] = t;
        }
    }
}

}  // namespace fl
