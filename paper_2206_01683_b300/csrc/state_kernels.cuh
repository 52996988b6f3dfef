// state_kernels.cuh -- initialisation and host access to the populations and
// the macroscopic fields (outside the time step).
#pragma once

#include "aa_kernels.cuh"

namespace fl {

// ----------------------------------------------------- state access
// These run over cells c = x + nx (y + ny z) (the ABI's cell order) and take
// the post-collision population i of a cell where the layout keeps it
// (post_loc; aa < 0: two buffers, else the in-place phase).

__device__ __forceinline__ uint32_t cell_to_slot(const EnvDev& E, uint32_t c) {
    const uint32_t nx = (uint32_t)E.n[0];
    const uint32_t row = c / nx;
    return row * (uint32_t)E.P + (c - row * nx);
}

// Flat index (direction, slot) of the post-collision population i of cell c.
__device__ __forceinline__ size_t cell_pop_index(const EnvDev& E, int aa, uint32_t c, int i) {
    const uint32_t nx = (uint32_t)E.n[0];
    const uint32_t row = c / nx;
    const int x = (int)(c - row * nx), y = (int)(row % (uint32_t)E.n[1]), z = (int)(row / (uint32_t)E.n[1]);
    int dir;
    const uint32_t loc = post_loc(E, aa, i, x, y, z, row * (uint32_t)E.P + (uint32_t)x, &dir);
    return (size_t)dir * E.nslot + loc;
}

// f_eq(rho, u) - w on the Hermite-2 basis (plus, with eq3, the third-order
// terms 4.5 w rho (c.u)((c.u)^2 - |u|^2)), computed in FP64.
template <class S>
__global__ void k_init_eq(typename S::raw* __restrict__ g, const EnvDev* __restrict__ envs, int e,
                          const double* __restrict__ rho, const double* __restrict__ u,
                          double rho0, double u0x, double u0y, double u0z, int eq3, int aa) {
    const EnvDev& E = envs[e];
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t ncell = (uint32_t)E.n[0] * E.n[1] * E.n[2];
    if (c >= ncell) return;
    const double r = rho ? rho[c] : rho0;
    const double ux = u ? u[3 * (size_t)c] : u0x, uy = u ? u[3 * (size_t)c + 1] : u0y,
                 uz = u ? u[3 * (size_t)c + 2] : u0z;
    const double uu = ux * ux + uy * uy + uz * uz;
    typename S::raw* G = g + E.pop_off;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        double f = wd(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        if (eq3) f += wd(i) * r * 4.5 * cu * (cu * cu - uu);
        G[cell_pop_index(E, aa, c, i)] = S::encode((float)(f - wd(i)), i);
    }
}

// out[c][27] = w_i + g_i (FP64), library velocity order.
template <class S>
__global__ void k_get_pop(const typename S::raw* __restrict__ g, const EnvDev* __restrict__ envs, int e,
                          double* __restrict__ out, int aa) {
    const EnvDev& E = envs[e];
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (uint32_t)E.n[0] * E.n[1] * E.n[2]) return;
    const typename S::raw* G = g + E.pop_off;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        out[(size_t)c * Q + i] = wd(i) + (double)S::decode(G[cell_pop_index(E, aa, c, i)], i);
}

template <class S>
__global__ void k_set_pop(typename S::raw* __restrict__ g, const EnvDev* __restrict__ envs, int e,
                          const double* __restrict__ in, int aa) {
    const EnvDev& E = envs[e];
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (uint32_t)E.n[0] * E.n[1] * E.n[2]) return;
    typename S::raw* G = g + E.pop_off;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        G[cell_pop_index(E, aa, c, i)] = S::encode((float)(in[(size_t)c * Q + i] - wd(i)), i);
}

// rho = 1 + sum g, u = sum c g / rho, in FP64 from the stored values.
template <class S>
__global__ void k_get_fields(const typename S::raw* __restrict__ g, const EnvDev* __restrict__ envs, int e,
                             double* __restrict__ rho, double* __restrict__ u, int aa) {
    const EnvDev& E = envs[e];
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (uint32_t)E.n[0] * E.n[1] * E.n[2]) return;
    const typename S::raw* G = g + E.pop_off;
    double dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double v = (double)S::decode(G[cell_pop_index(E, aa, c, i)], i);
        dr += v;
        jx += cx(i) * v; jy += cy(i) * v; jz += cz(i) * v;
    }
    const double r = 1.0 + dr;
    rho[c] = r;
    u[3 * (size_t)c] = jx / r; u[3 * (size_t)c + 1] = jy / r; u[3 * (size_t)c + 2] = jz / r;
}

}  // namespace fl
