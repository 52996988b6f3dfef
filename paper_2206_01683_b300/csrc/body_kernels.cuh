// body_kernels.cuh -- a free rigid sphere advanced on the device: the body
// update of Eq. 1 (arXiv 2206.01683, Sec. III-A) for a sphere whose only
// generalised forces are the fluid's tau_ext, gravity and buoyancy, two-way
// coupled every step without a host round trip.  Around the fluid step of
// its environment:
//   k_sphere_place   the markers on the shell from the body state,
//                    X = c + R d, U = V + W x (X - c), torque point c
//   (IB, stream-collide, reduction: F and T about c)
//   k_sphere_fluid   momentum P and angular momentum L of the fluid inside
//                    the shell in the new state (region_block_sums)
//   k_sphere_update  the explicit Newton-Euler step with the inner fluid's
//                    momentum change (Kempe & Froehlich, J. Comput. Phys. 231,
//                    2012):  m_p dV = F + dP_in + (m_p - m_f) g,
//                    I_p dW = T + dL_in,  c += (V_old + V_new) / 2.
// The body state is FP64 and every operation on it is an explicitly rounded
// FP64 intrinsic (no contraction into fused multiply-adds), so the sequence
// is exactly that of the plain FP64 formulas.
#pragma once

#include "reduce_kernels.cuh"

namespace fl {

struct SphereDev {
    double c[3], V[3], W[3];   // centre, velocity, spin
    double P_in[3], L_in[3];   // inner-fluid momentum of the last step
    double g[3];               // gravity
    double R, mp, mf, Ip;      // radius, body mass, displaced fluid mass, moment of inertia
    int env, n, mk_off, dir_off;
    int nblk;                  // blocks of the last inner-fluid sum
    int pad;
};

// Markers of sphere blockIdx.y: X = c + R d, U = V + W x (X - c) in FP64,
// stored as float; block 0 also moves the torque points of the environment's
// rows (total and segment 0) to c.
__global__ void k_sphere_place(const SphereDev* __restrict__ sph, const double* __restrict__ dirs,
                               float* __restrict__ X, float* __restrict__ U, EnvDev* __restrict__ envs,
                               float* __restrict__ seg_ref) {
    const SphereDev& s = sph[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < s.n) {
        const double* d = dirs + 3 * (size_t)(s.dir_off + j);
        double x[3], r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = __dadd_rn(s.c[a], __dmul_rn(s.R, d[a]));
            r[a] = __dsub_rn(x[a], s.c[a]);
        }
        const double w[3] = {__dsub_rn(__dmul_rn(s.W[1], r[2]), __dmul_rn(s.W[2], r[1])),
                             __dsub_rn(__dmul_rn(s.W[2], r[0]), __dmul_rn(s.W[0], r[2])),
                             __dsub_rn(__dmul_rn(s.W[0], r[1]), __dmul_rn(s.W[1], r[0]))};
        float* Xm = X + 3 * (size_t)(s.mk_off + j);
        float* Um = U + 3 * (size_t)(s.mk_off + j);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Xm[a] = __double2float_rn(x[a]);
            Um[a] = __double2float_rn(__dadd_rn(s.V[a], w[a]));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 3) {
        const int a = threadIdx.x;
        envs[s.env].ref[a] = s.c[a];
        seg_ref[(size_t)s.env * MAX_SEG * 3 + a] = __double2float_rn(s.c[a]);
    }
}

// Blocks of the inner-fluid sum of a sphere (centre c, radius R) in E: one
// per RED_THREADS cells of its box, at most `grid` (the rule of
// fg_region_momentum, so both give the same partial sums).
__device__ __forceinline__ int sphere_blocks(const EnvDev& E, const double (&c)[3], double R, int grid,
                                             int (&lo)[3], int (&ext)[3]) {
    sphere_box(E, c, R, lo, ext);
    const long long n_box = (long long)ext[0] * ext[1] * ext[2];
    const long long want = (n_box + RED_THREADS - 1) / RED_THREADS;
    return (int)max(1ll, min(want, (long long)grid));
}

// Inner-fluid sums of sphere blockIdx.y in the state g (layout aa, as
// post_loc): block b < nblk writes its seven pairs to part[y][b].
template <class S>
__global__ void __launch_bounds__(RED_THREADS)
k_sphere_fluid(const typename S::raw* __restrict__ g, const EnvDev* __restrict__ envs, SphereDev* sph, int aa,
               Pair32* __restrict__ part) {
    __shared__ Pair32 sh[RED_THREADS / 32][7];
    SphereDev& s = sph[blockIdx.y];
    const EnvDev& E = envs[s.env];
    const double c[3] = {s.c[0], s.c[1], s.c[2]};
    int lo[3], ext[3];
    const int nblk = sphere_blocks(E, c, s.R, gridDim.x, lo, ext);
    if (blockIdx.x == 0 && threadIdx.x == 0) s.nblk = nblk;
    if ((int)blockIdx.x >= nblk) return;
    const float cf[3] = {__double2float_rn(c[0]), __double2float_rn(c[1]), __double2float_rn(c[2])};
    region_block_sums<S>(g, E, cf, __double2float_rn(s.R), lo, ext, blockIdx.x, nblk, sh,
                         part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 7, aa);
}

// The body update of sphere blockIdx.x (one thread): P, L = the block pairs
// of k_sphere_fluid summed in FP64 in block order; F, T = the total
// force/torque row of its environment.  init != 0 only records P and L (at
// attachment).
__global__ void k_sphere_update(SphereDev* sph, const Pair32* __restrict__ part, int grid,
                                const Pair32* __restrict__ ft, int init) {
    if (threadIdx.x != 0) return;
    SphereDev& s = sph[blockIdx.x];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const Pair32* p = part + (size_t)blockIdx.x * grid * 7;
    for (int b = 0; b < s.nblk; ++b)
        for (int q = 0; q < 6; ++q)
            acc[q] = __dadd_rn(acc[q], __dadd_rn((double)p[b * 7 + q].hi, (double)p[b * 7 + q].lo));
    if (!init) {
        // the environment's total row (it follows its single segment row)
        const Pair32* row = ft + (size_t)s.env * FT_ROW + 6;
        double F[6];
        for (int k = 0; k < 6; ++k) F[k] = __dadd_rn((double)row[k].hi, (double)row[k].lo);
        const double excess = __dsub_rn(s.mp, s.mf);
        for (int a = 0; a < 3; ++a) {
            const double dv = __ddiv_rn(__dadd_rn(__dadd_rn(F[a], __dsub_rn(acc[a], s.P_in[a])), __dmul_rn(excess, s.g[a])),
                                        s.mp);
            const double dw = __ddiv_rn(__dadd_rn(F[3 + a], __dsub_rn(acc[3 + a], s.L_in[a])), s.Ip);
            const double v_new = __dadd_rn(s.V[a], dv);
            s.c[a] = __dadd_rn(s.c[a], __dmul_rn(0.5, __dadd_rn(s.V[a], v_new)));
            s.V[a] = v_new;
            s.W[a] = __dadd_rn(s.W[a], dw);
        }
    }
    for (int a = 0; a < 3; ++a) {
        s.P_in[a] = acc[a];
        s.L_in[a] = acc[3 + a];
    }
}

}  // namespace fl
