// noalloc.cu -- fg_body_force_noalloc: the immersed-boundary force on a
// body from a fluid state the caller owns, computed without allocating any
// memory.
//
// Some callers cannot allocate device memory at the time they need this
// force: a host program whose device memory is entirely owned by another
// framework's memory pool, or a control loop that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  For them this entry point
// keeps its only scratch -- the per-marker force density and an error flag --
// in a file-scope static __device__ array of fixed size, which every GPU that
// loads this library holds until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host that name
// is a stand-in, not a device address.  The device address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call made on a
// device (so that first call should come before any stream capture), and
// looked up again on every later call made outside a stream capture, so that
// a context created anew (after cudaDeviceReset, say) is served at its own
// address; a call under capture uses the address found last.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/fishlbm.h"
#include "reduce_kernels.cuh"

using namespace fl;

void fl_set_last_error(const char* msg);  // fishlbm.cu

namespace {

constexpr int MAX_DEVICES = 64;
constexpr int FLAG_WORDS = 64;   // word 0: invalid-marker flag; rest keeps the forces 256-byte aligned

// The scratch: FLAG_WORDS words, then FG_NOALLOC_MAX_MARKERS x 3 floats.
static __device__ __align__(256) float g_noalloc_scratch[FLAG_WORDS + 3 * FG_NOALLOC_MAX_MARKERS];

float* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mutex;
fg_status nf_fail(fg_status s, const std::string& m) {
    fl_set_last_error(m.c_str());   // reported by fg_last_error()
    return s;
}

// Per-device set-up: the device address of the scratch array, looked up
// outside stream capture (the lookup may load the module), else the address
// found by the last lookup on this device.
fg_status scratch_for_current_device(cudaStream_t s, float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nf_fail(FG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return nf_fail(FG_ERR_INVALID, "device ordinal beyond 63");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return nf_fail(FG_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return nf_fail(FG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<float*>(p);
    } else if (!g_scratch_addr[dev]) {
        return nf_fail(FG_ERR_STATE, "fg_body_force_noalloc: the first call on a device must precede stream capture");
    }
    *out = g_scratch_addr[dev];
    return FG_OK;
}

// Interpolation and direct forcing of k_ib without the spreading: one warp
// per marker writes F_l into the scratch; a marker outside its allowed range
// gets F_l = 0 and raises the flag word.
__global__ void __launch_bounds__(IB_THREADS, 4)
k_ib_force_noalloc(const float* __restrict__ g, EnvDev E, FrameDev F, int n, const float* __restrict__ X,
                   const float* __restrict__ U, float* __restrict__ scratch) {
    const int l = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (l >= n) return;
    float* Fm = scratch + FLAG_WORDS;
    float xw[3];
    int base[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = X[3 * l + a];
        const float N = (float)E.n[a];
        float w = x;
        if (!(fabsf(x) <= 1.0e6f)) ok = false;
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
            Fm[3 * l] = 0.f; Fm[3 * l + 1] = 0.f; Fm[3 * l + 2] = 0.f;
            atomicOr(reinterpret_cast<int*>(scratch), 1);
        }
        return;
    }
    const int kx = lane & 3, ky = (lane >> 2) & 3, kz = lane >> 4;
    const int mx = base[0] + kx, my = base[1] + ky;
    const float wxy = peskin4(xw[0] - (float)mx) * peskin4(xw[1] - (float)my);
    const int nx = E.n[0], ny = E.n[1], nz = E.n[2];
    const int mxw = ((mx % nx) + nx) % nx;
    const int myw = ((my % ny) + ny) % ny;
    float R = 0.f, Ux = 0.f, Uy = 0.f, Uz = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int mz = base[2] + kz + 2 * h;
        const int mzw = ((mz % nz) + nz) % nz;
        const float d = wxy * peskin4(xw[2] - (float)mz);
        const uint32_t c = (uint32_t)mxw + (uint32_t)E.P * ((uint32_t)myw + (uint32_t)ny * (uint32_t)mzw);
        const PullOffsets o = pull_offsets(E, mxw, myw, mzw);
        const Moments m = pull_moments<StoreF32, false>(g, E.nslot, c, o);
        const float rho = 1.0f + m.dr;
        const float inv = 1.0f / rho;
        float a0[3];
        frame_accel(F, (float)mxw, (float)myw, (float)mzw, a0);
        R += d * rho;
        Ux += d * (m.jx * inv + 0.5f * a0[0]);
        Uy += d * (m.jy * inv + 0.5f * a0[1]);
        Uz += d * (m.jz * inv + 0.5f * a0[2]);
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        R += __shfl_xor_sync(0xffffffffu, R, s);
        Ux += __shfl_xor_sync(0xffffffffu, Ux, s);
        Uy += __shfl_xor_sync(0xffffffffu, Uy, s);
        Uz += __shfl_xor_sync(0xffffffffu, Uz, s);
    }
    if (lane == 0) {
        Fm[3 * l] = 2.0f * R * (U[3 * l] - Ux);
        Fm[3 * l + 1] = 2.0f * R * (U[3 * l + 1] - Uy);
        Fm[3 * l + 2] = 2.0f * R * (U[3 * l + 2] - Uz);
    }
}

// The force/torque rows of k_reduce, reading the marker forces from the
// scratch: block y < n_seg sums segment y, block n_seg all markers.  Rows
// become NaN if a marker was rejected.
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_noalloc(const float* __restrict__ scratch, const float* __restrict__ X, const float* __restrict__ dV,
                 const int* __restrict__ seg, int n, int n_seg, double rx0, double ry0, double rz0,
                 double* __restrict__ out) {
    __shared__ Pair32 sh[RED_THREADS / 32];
    const int y = blockIdx.x;
    const float* Fm = scratch + FLAG_WORDS;
    const bool rejected = *reinterpret_cast<const int*>(scratch) != 0;
    const float rfx = (float)rx0, rfy = (float)ry0, rfz = (float)rz0;
    Pair32 acc[6];
#pragma unroll 2
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        const int sg = seg ? seg[l] : 0;
        const float dv = dV[l];
        const float f0 = Fm[3 * l], f1 = Fm[3 * l + 1], f2 = Fm[3 * l + 2];
        const float rx = X[3 * l] - rfx, ry = X[3 * l + 1] - rfy, rz = X[3 * l + 2] - rfz;
        const float v = (y == n_seg || sg == y) ? -dv : 0.0f;
        const float Fx = f0 * v, Fy = f1 * v, Fz = f2 * v;
        acc[0].add(Fx); acc[1].add(Fy); acc[2].add(Fz);
        acc[3].add(ry * Fz - rz * Fy);
        acc[4].add(rz * Fx - rx * Fz);
        acc[5].add(rx * Fy - ry * Fx);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double t = block_sum(acc[k], sh);
        if (threadIdx.x == 0) out[6 * y + k] = rejected ? (double)NAN : t;
    }
}

}  // namespace

extern "C" fg_status fg_body_force_noalloc(const fg_env_desc* env, const float* g, const float* X, const float* U,
                                           const float* dV, const int* seg, int n, int n_seg, const double ref[3],
                                           const fg_frame* frame, double* out, void* cuda_stream) {
    if (!env || !g || !out || n < 0 || (n > 0 && (!X || !U || !dV)))
        return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: missing argument");
    if (n > FG_NOALLOC_MAX_MARKERS)
        return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: more than FG_NOALLOC_MAX_MARKERS (65536) markers "
                                       "do not fit the static scratch");
    if (n_seg < 1 || n_seg > MAX_SEG) return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: n_seg must be in [1, 16]");
    const int dims[3] = {env->nx, env->ny, env->nz};
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > 65536) return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: grid size");
        const int lo = env->face[2 * a], hi = env->face[2 * a + 1];
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3 || (lo == FG_PERIODIC) != (hi == FG_PERIODIC))
            return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: faces");
        if (lo != FG_PERIODIC && dims[a] < 3) return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: open axis < 3");
    }
    const unsigned long long P = (unsigned long long)(env->nx + 7) / 8 * 8;
    if (P * env->ny * env->nz >= (1ull << 31)) return nf_fail(FG_ERR_INVALID, "fg_body_force_noalloc: grid too large");
    float* scratch = nullptr;
    fg_status st = scratch_for_current_device((cudaStream_t)cuda_stream, &scratch);
    if (st != FG_OK) return st;

    EnvDev E;
    memset(&E, 0, sizeof(E));
    E.n[0] = env->nx; E.n[1] = env->ny; E.n[2] = env->nz;
    E.P = (int)P;
    E.nslot = (uint32_t)(P * env->ny * env->nz);
    for (int a = 0; a < 3; ++a) E.per[a] = env->face[2 * a] == FG_PERIODIC;
    FrameDev F;
    memset(&F, 0, sizeof(F));
    double oo = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double org = frame ? frame->origin[a] : (dims[a] - 1) * 0.5;
        F.acc[a] = frame ? (float)frame->acc[a] : 0.f;
        F.om[a] = frame ? (float)frame->omega[a] : 0.f;
        F.dom[a] = frame ? (float)frame->domega[a] : 0.f;
        F.org[a] = (float)org;
        if (frame) oo += frame->omega[a] * frame->omega[a];
    }
    F.inv_1pom2 = (float)(1.0 / (1.0 + oo));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the flag word must start at zero on every call (the scratch keeps the
    // last call's contents); the forces are overwritten
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int), s);
    if (e == cudaSuccess && n > 0) {
        const int blocks = (n + IB_THREADS / 32 - 1) / (IB_THREADS / 32);
        k_ib_force_noalloc<<<blocks, IB_THREADS, 0, s>>>(g, E, F, n, X, U, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const double r0 = ref ? ref[0] : 0.0, r1 = ref ? ref[1] : 0.0, r2 = ref ? ref[2] : 0.0;
        k_reduce_noalloc<<<n_seg + 1, RED_THREADS, 0, s>>>(scratch, X, dV, seg, n, n_seg, r0, r1, r2, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nf_fail(FG_ERR_CUDA, std::string("fg_body_force_noalloc: ") + cudaGetErrorString(e));
    return FG_OK;
}
