// adjoint_kernels.cuh -- the discrete adjoint of one time step (periodic
// domains, FP32 storage), for gradients of force/torque-based losses with
// respect to the marker positions and velocities (and, through them, the
// joint-wave parameters of the swimmer).
//
// Forward step n:  fs = pull(f*^n);  moments m(fs);  IB: R_l = sum delta rho,
// U~_l = sum delta u~, F_l = 2 R_l (U_l - U~_l), fib = sum F_l dV_l delta;
// collision f*^{n+1} = H(q(m, fib)).  Given lam^{n+1} = dL/df*^{n+1} and the
// loss gradient w.r.t. the step's force/torque rows, the adjoint step forms
//   k_adj_tiles           dL/dfib at cells of stamped tiles
//   k_adj_ib              per marker: dL/dF_l, dL/dX_l, dL/dU_l, and the
//                         scatter of dL/drho, dL/du~ onto the stencil nodes
//   k_adj_stream_collide  dL/dfs at every cell (collision adjoint plus the IB
//                         node terms), pushed back along -c_i (the transpose
//                         of the pull): lam^n
// All arithmetic is FP32 (the forward is recomputed in the same order as the
// forward kernels).
#pragma once

#include "step_kernels.cuh"

namespace fl {

// d phi / dr of Peskin's 4-point function.
__device__ __forceinline__ float peskin4_deriv(float r) {
    const float a = fabsf(r);
    float d;
    if (a <= 1.0f)
        d = (-2.0f + (2.0f - 4.0f * a) * rsqrtf(1.0f + 4.0f * a - 4.0f * a * a)) * 0.125f;
    else if (a <= 2.0f)
        d = (-2.0f - (6.0f - 4.0f * a) * rsqrtf(fmaxf(-7.0f + 12.0f * a - 4.0f * a * a, 1e-30f))) * 0.125f;
    else
        d = 0.0f;
    return r < 0.0f ? -d : d;
}

// Adjoint of the interior collision at one cell.  Inputs: post-stream moments
// m, IB force density fib, frame acceleration a0, constants C, and lam[i] =
// dL/df*_i.  Outputs: lg[i] = dL/dfs_i through the collision (without the
// IB node terms) and lfib = dL/dfib.
__device__ __forceinline__ void adj_collide(const CellConsts& C, const Moments& m, const float fib[3],
                                            const float a0[3], const float (&lam)[Q], float (&lg)[Q],
                                            float lfib[3]) {
    const float cs2 = 1.0f / 3.0f;
    // Hermite adjoint: moments of w_i lam_i
    float wl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) wl[i] = wf(i) * lam[i];
    Moments M = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    accumulate<true>(M, wl);
    const float lro = M.dr;                                     // d/d rho_out
    const float lJ[3] = {3.0f * M.jx, 3.0f * M.jy, 3.0f * M.jz};
    // Lam_ab = 4.5 M2_ab - 1.5 M0 delta_ab (full symmetric matrix)
    float Lm[3][3];
    Lm[0][0] = 4.5f * M.sxx - 1.5f * M.dr;
    Lm[1][1] = 4.5f * M.syy - 1.5f * M.dr;
    Lm[2][2] = 4.5f * M.szz - 1.5f * M.dr;
    Lm[0][1] = Lm[1][0] = 4.5f * M.sxy;
    Lm[0][2] = Lm[2][0] = 4.5f * M.sxz;
    Lm[1][2] = Lm[2][1] = 4.5f * M.syz;

    // forward recompute
    const float rho = 1.0f + m.dr, inv = 1.0f / rho;
    const float j[3] = {m.jx, m.jy, m.jz};
    float v[3], u[3], Wu[3], G[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = (j[a] + 0.5f * fib[a]) * inv + 0.5f * a0[a];
    const float* w = C.om;
    const float wv = w[0] * v[0] + w[1] * v[1] + w[2] * v[2];
    u[0] = (v[0] - (w[1] * v[2] - w[2] * v[1]) + wv * w[0]) * C.inv_1pom2;
    u[1] = (v[1] - (w[2] * v[0] - w[0] * v[2]) + wv * w[1]) * C.inv_1pom2;
    u[2] = (v[2] - (w[0] * v[1] - w[1] * v[0]) + wv * w[2]) * C.inv_1pom2;
    Wu[0] = w[1] * u[2] - w[2] * u[1];
    Wu[1] = w[2] * u[0] - w[0] * u[2];
    Wu[2] = w[0] * u[1] - w[1] * u[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) G[a] = rho * a0[a] + fib[a] - 2.0f * rho * Wu[a];

    const float k = C.keep, gq = C.guo;
    // J = j + G
    float lj[3] = {lJ[0], lJ[1], lJ[2]};
    float lG[3] = {lJ[0], lJ[1], lJ[2]};
    // Q = (1-k) rho u u^T + k S - k (rho-1) cs2 I + gq (u G^T + G u^T)
    float Lu[3], LG[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Lu[a] = Lm[a][0] * u[0] + Lm[a][1] * u[1] + Lm[a][2] * u[2];
        LG[a] = Lm[a][0] * G[0] + Lm[a][1] * G[1] + Lm[a][2] * G[2];
    }
    float lrho = lro + (1.0f - k) * (u[0] * Lu[0] + u[1] * Lu[1] + u[2] * Lu[2]) -
                 k * cs2 * (Lm[0][0] + Lm[1][1] + Lm[2][2]);
    float lu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lu[a] = 2.0f * (1.0f - k) * rho * Lu[a] + 2.0f * gq * LG[a];
        lG[a] += 2.0f * gq * Lu[a];
    }
    // G = rho a0 + fib - 2 rho (w x u)
    lrho += lG[0] * (a0[0] - 2.0f * Wu[0]) + lG[1] * (a0[1] - 2.0f * Wu[1]) + lG[2] * (a0[2] - 2.0f * Wu[2]);
    lfib[0] = lG[0]; lfib[1] = lG[1]; lfib[2] = lG[2];
    lu[0] += 2.0f * rho * (w[1] * lG[2] - w[2] * lG[1]);
    lu[1] += 2.0f * rho * (w[2] * lG[0] - w[0] * lG[2]);
    lu[2] += 2.0f * rho * (w[0] * lG[1] - w[1] * lG[0]);
    // u = K (v - w x v + (w.v) w)  =>  lv = K (lu + w x lu + (w.lu) w)
    const float wl_u = w[0] * lu[0] + w[1] * lu[1] + w[2] * lu[2];
    float lv[3];
    lv[0] = (lu[0] + (w[1] * lu[2] - w[2] * lu[1]) + wl_u * w[0]) * C.inv_1pom2;
    lv[1] = (lu[1] + (w[2] * lu[0] - w[0] * lu[2]) + wl_u * w[1]) * C.inv_1pom2;
    lv[2] = (lu[2] + (w[0] * lu[1] - w[1] * lu[0]) + wl_u * w[2]) * C.inv_1pom2;
    // v = (j + fib/2)/rho + a0/2
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lj[a] += lv[a] * inv;
        lfib[a] += 0.5f * lv[a] * inv;
        lrho -= (v[a] - 0.5f * a0[a]) * lv[a] * inv;
    }
    // moments: rho = 1 + sum g, j = sum c g, S = sum c c g (lS = k Lam)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float c0 = (float)cx(i), c1 = (float)cy(i), c2 = (float)cz(i);
        const float quad = c0 * c0 * Lm[0][0] + c1 * c1 * Lm[1][1] + c2 * c2 * Lm[2][2] +
                           2.0f * (c0 * c1 * Lm[0][1] + c0 * c2 * Lm[0][2] + c1 * c2 * Lm[1][2]);
        lg[i] = lrho + c0 * lj[0] + c1 * lj[1] + c2 * lj[2] + k * quad;
    }
}

// Periodic-domain pull moments and frame acceleration at slot c = (x, y, z).
__device__ __forceinline__ Moments adj_forward_moments(const EnvDev& E, const float* __restrict__ G, uint32_t c,
                                                       int x, int y, int z) {
    const PullOffsets o = pull_offsets(E, x, y, z);
    return pull_moments<StoreF32, true>(G, E.nslot, c, o);
}

__device__ __forceinline__ void slot_xyz(const EnvDev& E, uint32_t c, int& x, int& y, int& z) {
    const uint32_t row = fdiv(c, E.div_P);
    x = (int)(c - row * (uint32_t)E.P);
    const uint32_t zz = fdiv(row, E.div_ny);
    y = (int)(row - zz * (uint32_t)E.n[1]);
    z = (int)zz;
}

__device__ __forceinline__ void affine_a0(const CellConsts& C, int x, int y, int z, float a0[3]) {
    const float px = (float)x, py = (float)y, pz = (float)z;
    a0[0] = C.c0[0] - (C.M[0] * px + C.M[1] * py + C.M[2] * pz);
    a0[1] = C.c0[1] - (C.M[3] * px + C.M[4] * py + C.M[5] * pz);
    a0[2] = C.c0[2] - (C.M[6] * px + C.M[7] * py + C.M[8] * pz);
}

// dL/dfib at the cells of stamped tiles (one thread per slot).
__global__ void __launch_bounds__(K1_THREADS)
k_adj_tiles(const float* __restrict__ f, const float* __restrict__ lam, const EnvDev* __restrict__ envs,
            const FrameDev* __restrict__ frames, const float4* __restrict__ fib, const uint32_t* __restrict__ stamps,
            const StepState* __restrict__ st, float* __restrict__ lfib) {
    const EnvDev& E = envs[0];
    __shared__ CellConsts C;   // loaded once per block, read by every cell
    if (threadIdx.x == 0) C = load_consts(E, frames[0]);
    __syncthreads();
    const uint32_t c = blockIdx.x * K1_THREADS + threadIdx.x;
    if (c >= E.nslot) return;
    if (__ldg(stamps + E.stamp_off + (c >> 5)) != st->stamp) return;
    int x, y, z;
    slot_xyz(E, c, x, y, z);
    if (x >= E.n[0]) return;
    const Moments m = adj_forward_moments(E, f, c, x, y, z);
    const float4 f4 = fib[c];
    const float fb[3] = {f4.x, f4.y, f4.z};
    float a0[3];
    affine_a0(C, x, y, z, a0);
    float lm[Q], lg[Q], lf[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) lm[i] = lam[(size_t)i * E.nslot + c];
    adj_collide(C, m, fb, a0, lm, lg, lf);
    lfib[c] = lf[0];
    lfib[E.nslot + c] = lf[1];
    lfib[2ull * E.nslot + c] = lf[2];
}

// Per marker (one warp, nodes as in k_ib): recompute R, U~, F; form
// dL/dF = dV interp(dL/dfib) + the force/torque loss terms; then
//   dL/dU = 2 R dL/dF,  dL/dU~ = -2 R dL/dF,  dL/dR = 2 (U - U~).dL/dF,
// scatter dL/drho = delta dL/dR and dL/du~ = delta dL/dU~ onto the nodes, and
//   dL/dX = dV sum grad(delta) (F.dL/dfib) + sum grad(delta) (rho dL/dR + u~.dL/dU~)
//           - dV (F x gT)   (the torque's lever arm).
// gF: (nseg+1) x 6 loss gradient w.r.t. the step's force/torque rows.
__global__ void __launch_bounds__(IB_THREADS)
k_adj_ib(const float* __restrict__ f, const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames,
         int n, const float* __restrict__ X, const float* __restrict__ U, const float* __restrict__ dV,
         const int* __restrict__ seg, const float* __restrict__ lfib, const float* __restrict__ gF, int nseg,
         float* __restrict__ lrho, float* __restrict__ lut, float* __restrict__ gX, float* __restrict__ gU) {
    const int l = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (l >= n) return;
    const EnvDev& E = envs[0];
    const FrameDev F = frames[0];
    const int q = E.marker_off + l;
    float xw[3];
    int base[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = X[3 * q + a];
        const float N = (float)E.n[a];
        float w = x - floorf(x / N) * N;
        if (w >= N) w -= N;
        if (w < 0.0f) w += N;
        xw[a] = w;
        base[a] = (int)floorf(w) - 1;
    }
    const int kx = lane & 3, ky = (lane >> 2) & 3, kz = lane >> 4;
    const int mx = base[0] + kx, my = base[1] + ky;
    // r = X - node; delta = phi(r_x) phi(r_y) phi(r_z) (phi is even), so
    // d delta / dX_a = phi'(r_a) times the other two factors
    const float rxn = xw[0] - (float)mx, ryn = xw[1] - (float)my;
    const float px = peskin4(rxn), py = peskin4(ryn);
    const float dpx = peskin4_deriv(rxn), dpy = peskin4_deriv(ryn);
    const int nx = E.n[0], ny = E.n[1], nz = E.n[2];
    const int mxw = ((mx % nx) + nx) % nx;
    const int myw = ((my % ny) + ny) % ny;
    // per-lane partial sums
    float R = 0.f, Ut[3] = {0.f, 0.f, 0.f}, Lf[3] = {0.f, 0.f, 0.f};
    float Dr[3] = {0.f, 0.f, 0.f}, Du[3][3] = {{0.f}}, Dl[3][3] = {{0.f}};
    float dlt[2];
    uint32_t cell[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int mz = base[2] + kz + 2 * h;
        const int mzw = ((mz % nz) + nz) % nz;
        const float rzn = xw[2] - (float)mz;
        const float pz = peskin4(rzn), dpz = peskin4_deriv(rzn);
        const float d = px * py * pz;
        const float gd[3] = {dpx * py * pz, px * dpy * pz, px * py * dpz};
        const uint32_t c = (uint32_t)mxw + (uint32_t)E.P * ((uint32_t)myw + (uint32_t)ny * (uint32_t)mzw);
        const PullOffsets o = pull_offsets(E, mxw, myw, mzw);
        const Moments m = pull_moments<StoreF32, false>(f, E.nslot, c, o);
        const float rho = 1.0f + m.dr, inv = 1.0f / rho;
        float a0[3];
        frame_accel(F, (float)mxw, (float)myw, (float)mzw, a0);
        const float ut[3] = {m.jx * inv + 0.5f * a0[0], m.jy * inv + 0.5f * a0[1], m.jz * inv + 0.5f * a0[2]};
        const float lf[3] = {lfib[c], lfib[E.nslot + c], lfib[2ull * E.nslot + c]};
        R += d * rho;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Ut[a] += d * ut[a];
            Lf[a] += d * lf[a];
            Dr[a] += gd[a] * rho;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Du[b][a] += gd[a] * ut[b];   // sum grad_a(delta) u~_b
                Dl[b][a] += gd[a] * lf[b];   // sum grad_a(delta) lfib_b
            }
        }
        dlt[h] = d;
        cell[h] = c;
    }
    // warp sums (all lanes end with the totals)
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        R += __shfl_xor_sync(0xffffffffu, R, s);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Ut[a] += __shfl_xor_sync(0xffffffffu, Ut[a], s);
            Lf[a] += __shfl_xor_sync(0xffffffffu, Lf[a], s);
            Dr[a] += __shfl_xor_sync(0xffffffffu, Dr[a], s);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Du[b][a] += __shfl_xor_sync(0xffffffffu, Du[b][a], s);
                Dl[b][a] += __shfl_xor_sync(0xffffffffu, Dl[b][a], s);
            }
        }
    }
    const float v = dV[q];
    const float Um[3] = {U[3 * q], U[3 * q + 1], U[3 * q + 2]};
    float Fm[3], lF[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Fm[a] = 2.0f * R * (Um[a] - Ut[a]);
    // loss terms: F_body = -sum F dV, T_body = -sum r x F dV (segment row + total row)
    const int s = seg ? seg[q] : 0;
    float gFs[3], gTs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gFs[a] = gF[6 * nseg + a] + (s >= 0 && s < nseg ? gF[6 * s + a] : 0.0f);
        gTs[a] = gF[6 * nseg + 3 + a] + (s >= 0 && s < nseg ? gF[6 * s + 3 + a] : 0.0f);
    }
    const float r[3] = {X[3 * q] - (float)E.ref[0], X[3 * q + 1] - (float)E.ref[1], X[3 * q + 2] - (float)E.ref[2]};
    const float gxr[3] = {gTs[1] * r[2] - gTs[2] * r[1], gTs[2] * r[0] - gTs[0] * r[2], gTs[0] * r[1] - gTs[1] * r[0]};
#pragma unroll
    for (int a = 0; a < 3; ++a) lF[a] = v * Lf[a] - v * gFs[a] - v * gxr[a];
    float lUt[3], lR = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lUt[a] = -2.0f * R * lF[a];
        lR += 2.0f * (Um[a] - Ut[a]) * lF[a];
    }
    // scatter dL/drho and dL/du~ onto the nodes
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        atomicAdd(lrho + cell[h], dlt[h] * lR);
        atomicAdd(lut + cell[h], dlt[h] * lUt[0]);
        atomicAdd(lut + E.nslot + cell[h], dlt[h] * lUt[1]);
        atomicAdd(lut + 2ull * E.nslot + cell[h], dlt[h] * lUt[2]);
    }
    if (lane == 0) {
        const float Fxg[3] = {Fm[1] * gTs[2] - Fm[2] * gTs[1], Fm[2] * gTs[0] - Fm[0] * gTs[2],
                              Fm[0] * gTs[1] - Fm[1] * gTs[0]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float spread = Fm[0] * Dl[0][a] + Fm[1] * Dl[1][a] + Fm[2] * Dl[2][a];
            const float interp = Dr[a] * lR + Du[0][a] * lUt[0] + Du[1][a] * lUt[1] + Du[2][a] * lUt[2];
            gX[3 * l + a] = v * spread + interp - v * Fxg[a];
            gU[3 * l + a] = 2.0f * R * lF[a];
        }
    }
}

// dL/dfs at every cell (collision adjoint + IB node terms), pushed along -c:
// lam_out_i(x - c_i) = dL/dfs_i(x).  Clears the IB fields of stamped tiles.
__global__ void __launch_bounds__(K1_THREADS)
k_adj_stream_collide(const float* __restrict__ f, const float* __restrict__ lam_in, float* __restrict__ lam_out,
                     const EnvDev* __restrict__ envs, const FrameDev* __restrict__ frames, float4* __restrict__ fib,
                     const uint32_t* __restrict__ stamps, const StepState* __restrict__ st,
                     float* __restrict__ lfib, float* __restrict__ lrho, float* __restrict__ lut) {
    const EnvDev& E = envs[0];
    __shared__ CellConsts C;   // loaded once per block, read by every cell
    if (threadIdx.x == 0) C = load_consts(E, frames[0]);
    __syncthreads();
    const uint32_t c = blockIdx.x * K1_THREADS + threadIdx.x;
    if (c >= E.nslot) return;
    int x, y, z;
    slot_xyz(E, c, x, y, z);
    if (x >= E.n[0]) return;
    const bool stamped = __ldg(stamps + E.stamp_off + (c >> 5)) == st->stamp;
    float fb[3] = {0.f, 0.f, 0.f}, lr = 0.f, lu[3] = {0.f, 0.f, 0.f};
    if (stamped) {
        const float4 f4 = fib[c];
        fb[0] = f4.x; fb[1] = f4.y; fb[2] = f4.z;
        lr = lrho[c];
        lu[0] = lut[c]; lu[1] = lut[E.nslot + c]; lu[2] = lut[2ull * E.nslot + c];
        fib[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        lfib[c] = 0.f; lfib[E.nslot + c] = 0.f; lfib[2ull * E.nslot + c] = 0.f;
        lrho[c] = 0.f;
        lut[c] = 0.f; lut[E.nslot + c] = 0.f; lut[2ull * E.nslot + c] = 0.f;
    }
    const Moments m = adj_forward_moments(E, f, c, x, y, z);
    float a0[3];
    affine_a0(C, x, y, z, a0);
    float lm[Q], lg[Q], lf[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) lm[i] = lam_in[(size_t)i * E.nslot + c];
    adj_collide(C, m, fb, a0, lm, lg, lf);
    // IB node terms: rho = 1 + sum g, u~ = j/rho + a0/2
    const float inv = 1.0f / (1.0f + m.dr);
    const float ujl = (m.jx * lu[0] + m.jy * lu[1] + m.jz * lu[2]) * inv;
    const PullOffsets o = pull_offsets(E, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cl = (float)cx(i) * lu[0] + (float)cy(i) * lu[1] + (float)cz(i) * lu[2];
        const float val = lg[i] + lr + (cl - ujl) * inv;
        // the pull read f*_i(x - c_i); its transpose writes there
        lam_out[(size_t)i * E.nslot + (uint32_t)((int)c + pull_off(o, i))] = val;
    }
}

__global__ void k_advance_stamp(StepState* st) {
    st->stamp = st->stamp == 0xffffffffu ? 1u : st->stamp + 1u;
}

}  // namespace fl
