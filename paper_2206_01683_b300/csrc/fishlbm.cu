// fishlbm.cu -- host runtime and C ABI of the library (declared in
// include/fishlbm.h).  Owns the device state of a domain: two population
// buffers (pull scheme), the sparse IB force density with its 32-cell tile
// stamps, marker arrays, the reduction outputs (compensated FP32 pairs), and
// the per-step launch sequence on one CUDA stream: k_ib_step (cooperative)
// -> k_stream_collide -> k_reduce (a programmatic dependent of
// k_stream_collide), or with the fused variant k_step_fused (one persistent
// cooperative launch for the IB phases and the stream-collide blocks) ->
// k_reduce.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fishlbm.h"
#include "step_kernels.cuh"
#include "adjoint_kernels.cuh"
#include "ib_kernels.cuh"
#include "reduce_kernels.cuh"
#include "fused_kernels.cuh"
#include "state_kernels.cuh"
#include "body_kernels.cuh"

using namespace fl;

// Marker positions and velocities of every environment from caller-owned
// device arrays in the compact marker order (environment after environment),
// scattered to each environment's marker region in one launch.
__global__ void k_scatter_markers(const fl::EnvDev* __restrict__ envs, int n_envs, int total,
                                  const float* __restrict__ Xs, const float* __restrict__ Us,
                                  float* __restrict__ X, float* __restrict__ U) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int e = n_envs > 1 ? fl::env_of<&fl::EnvDev::mk_begin>(envs, n_envs, k) : 0;
        const int slot = envs[e].marker_off + (k - envs[e].mk_begin);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            X[3 * slot + a] = Xs[3 * k + a];
            U[3 * slot + a] = Us[3 * k + a];
        }
    }
}

// Marker positions and velocities of one environment from caller-owned
// device arrays (count values each), in one launch.
__global__ void k_copy_markers(float* __restrict__ X, float* __restrict__ U, const float* __restrict__ Xs,
                                      const float* __restrict__ Us, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * count; i += gridDim.x * blockDim.x) {
        if (i < count) X[i] = Xs[i];
        else U[i - count] = Us[i - count];
    }
}

namespace {

// NVTX range over a C-ABI call (named in profiler timelines; free when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

namespace {

thread_local std::string g_err;

fg_status fail(fg_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

// Largest single device allocation the library makes (0: no limit), set by
// fg_set_alloc_cap so that the out-of-memory paths can be exercised without
// filling the device.
std::atomic<unsigned long long> g_alloc_cap{0};

fg_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FG_ERR_OOM : FG_ERR_CUDA;
}

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

constexpr int PROFILE_CAP = 1 << 14;
constexpr int MAX_STAGED_P = 512;   // longest row pitch the staged kernel takes

// Stream-collide variants the domain can run (and the autotuner times):
// the plain kernel, the staged kernel with 256 or 512 slots per population
// in shared memory, the fused step kernel (the plain kernel's cell update
// and the IB phases in one persistent launch), and the plain kernel with the
// IB beside it (the IB kernel on a second stream next to the plain kernel's
// blocks that no stencil node falls in).
enum { K1_PLAIN = 0, K1_STAGED256 = 1, K1_STAGED512 = 2, K1_FUSED = 3, K1_OVERLAP = 4, K1_NVARIANTS = 5 };
static_assert((int)K1_FUSED == (int)FG_K1_FUSED && (int)K1_OVERLAP == (int)FG_K1_OVERLAP &&
                  (int)K1_NVARIANTS == (int)FG_K1_NVARIANTS,
              "variant ids of the header");
static_assert(MAX_IB_PASSES == FG_MAX_IB_ITERS, "direct-forcing passes of the fused kernel");

// Blocks per SM the staged kernel is compiled for.  The 512-slot row buffers
// take 2 x 27 x 512 x sizeof(raw) bytes of shared memory, 110.6 KB in FP32
// (two blocks fit) and 55.3 KB in FP16/BF16 (four fit, as for the 256-slot
// kernel in FP32).  With two cells per thread the 16-bit kernels are compiled
// for three: at four their 64 registers spill, and on the swimmer channel
// the 512-slot kernel measured 100.3 us at three against 110.9 us at four and
// 113.5 us at two.
template <class S, int GC, bool PAIR>
constexpr int staged_minb() {
    return sizeof(typename S::raw) == 2 ? (PAIR ? 3 : 4) : (GC == 256 ? 4 : 2);
}

struct MarkerRegion {
    int n = 0, cap = 0, off = 0, nseg = 1;
    bool has_dv = false;
    bool has_normals = false;            // slip forcing: normals of the current markers
    double ref[3] = {0, 0, 0};
    bool has_seg_ref = false;            // segment rows about their own points
    double seg_ref[MAX_SEG][3] = {};
};

}  // namespace

struct fg_domain {
    int n_envs = 0;
    fg_options opt{};
    cudaStream_t stream = nullptr;
    int esize = 4;                       // bytes per stored population
    std::vector<fg_env_desc> desc;
    std::vector<EnvDev> env;             // host copy of the device table
    std::vector<FrameDev> frame;
    std::vector<MarkerRegion> mk;
    EnvDev* d_env = nullptr;
    FrameDev* d_frame = nullptr;         // n_envs frames, then the marker source (d_msrc)
    MarkerSrc* d_msrc = nullptr;         // in the same allocation as d_frame, so one copy carries both
    MarkerSrc msrc_next = {nullptr, nullptr, 0};   // posted for the next step (valid: not uploaded yet)
    void* pop[2] = {nullptr, nullptr};   // the in-place layout: both the one buffer
    int cur = 0;                         // buffer parity; the in-place layout's phase
    bool aa = false;                     // in-place (AA) layout
    unsigned long long pop_elems = 0, total_cells = 0, total_slots = 0;
    float4* fib = nullptr;               // IB force density per slot (x, y, z, unused)
    uint32_t* stamps = nullptr;
    unsigned long long n_stamps = 0;
    float4* ib_nodes = nullptr;          // per slot: rho, u~ of the stamped tiles' cells
    unsigned long long* fibq = nullptr;  // deterministic spread: fixed-point sums [slot][3]
    unsigned* ib_bar = nullptr;          // grid barrier of k_ib_step: arrival counter, base
    int ib_per_sm = 0;                   // resident blocks of k_ib_step per SM
    uint32_t stamp_host = 1;             // host mirror of StepState::stamp
    int n_sms = 0;
    Pair32* mass_part = nullptr;         // mass partial sums of the stream-collide kernel
    Pair32* red_partials = nullptr;      // chunk sums of k_reduce
    int* red_counters = nullptr;         // per environment: finished blocks of k_reduce
    int red_z = 1;                       // chunks per row of k_reduce
    int total_blocks = 0;                // plain stream-collide grid
    int sweep_reverse = 0;               // the step being enqueued sweeps its blocks from the end
    int total_bblocks = 0;               // in-place layout: boundary-cell kernel grid
    int total_groups = 0;                // staged kernel row groups
    int k1 = K1_PLAIN;                   // stream-collide variant in use (K1_*)
    bool staged = false;                 // a staged variant
    int fused_grid = 0;                  // persistent blocks of k_step_fused
    // the IB beside the stream-collide kernel: a second (high-priority)
    // stream, the fork and join events, the blocks flagged by k_mark_tiles
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    uint32_t* blk_flag = nullptr;        // per plain block: the stamp of the last step a stencil node fell in it
    size_t blk_flag_n = 0;
    int prio_high = 0;                   // greatest stream priority
    // work queue of k_step_fused: the segment table (host copy and device),
    // the queue words and the per-environment completion counters
    std::vector<WorkSeg> work_host;
    WorkSeg* work_segs = nullptr;
    int work_seg_cap = 0;
    int* work = nullptr;                 // WQ_WORDS
    int* work_done = nullptr;            // [n_envs][N_SLOTS]
    bool work_dirty = true;              // the table no longer matches the markers or kernel layout
    bool autotune_pending = false;       // autotune option: run fg_autotune before the first step
    int staged_grid = 0;                 // persistent blocks of the staged kernel
    int staged_gc = 256;                 // staged: slots per population in shared memory
    bool staged_pair = false;            // staged: two neighbouring cells per thread
    bool plain_pair = false;             // plain: two neighbouring cells per thread
    size_t staged_smem = 0;
    size_t mass_part_cap = 0;
    int max_P = 8;
    // adjoint state (allocated on first use): lam ping-pong, dL/dfib, dL/drho,
    // dL/du~ fields, and the loss gradient rows of the current step
    float* adj_lam[2] = {nullptr, nullptr};
    int adj_cur = 0;
    float* adj_lfib = nullptr;
    float* adj_lrho = nullptr;
    float* adj_lut = nullptr;
    float* adj_gF = nullptr;
    float *X = nullptr, *U = nullptr, *dV = nullptr, *Fm = nullptr;
    float* dF = nullptr;                 // per-pass force increments of multi-direct forcing
    float* Nrm = nullptr;                // unit marker normals (slip forcing)
    float* seg_ref = nullptr;            // torque points of the segment rows [n_envs][MAX_SEG][3]
    float* mk_stage = nullptr;           // host marker arrays of fg_set_markers_all, staged
    size_t mk_stage_cap = 0;             // floats
    Pair32* region_part = nullptr;       // block partials of fg_region_momentum
    int region_cap = 0;
    int* seg = nullptr;
    int marker_slots = 0;                // allocated marker slots
    int total_markers = 0;
    Pair32* ft = nullptr;                // force/torque rows (compensated pairs)
    Pair32* mass = nullptr;              // sum of (rho - 1) per environment
    Pair32* hist = nullptr;              // history ring: force/torque rows + mass
    int* status = nullptr;
    // pinned host landing area of the per-step reads (force/torque rows and
    // the status word), so those copies are asynchronous and one
    // synchronisation covers them
    struct Readback {
        Pair32 ft[FT_ROW];
        Pair32 mass;
        int status;
        long long seq;                   // the step number k_reduce wrote last
    }* rb = nullptr;
    Pair32* rb_ft_all = nullptr;         // pinned: the force/torque rows of all environments
    // device addresses of the mapped pinned copies k_reduce writes every step
    Pair32* rb_ft_all_dev = nullptr;
    int* rb_status_dev = nullptr;
    long long* rb_seq_dev = nullptr;
    long long steps = 0;
    StepState* d_state = nullptr;        // stamp / step / completion count on the device
    bool poisoned = false;
    // CUDA graphs of one step, one per population-buffer parity; rebuilt when
    // a launch parameter baked into them changes
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    struct GraphKey {
        const void* X = nullptr;
        const void* red = nullptr;
        const void* sph = nullptr;
        int total_markers = -1, red_z = -1, n_sph = 0, sph_max_n = 0, red_gy = -1, red_gz = -1;
        bool operator==(const GraphKey& o) const {
            return X == o.X && red == o.red && total_markers == o.total_markers && red_z == o.red_z &&
                   sph == o.sph && n_sph == o.n_sph && sph_max_n == o.sph_max_n && red_gy == o.red_gy &&
                   red_gz == o.red_gz;
        }
    } graph_key;
    // free spheres advanced on the device (fg_attach_sphere): the host copy
    // of the table (its body state is current only after sphere_download),
    // the device table, the marker directions and the inner-fluid partials
    std::vector<SphereDev> sph_host;
    std::vector<std::vector<double>> sph_dirs_host;
    SphereDev* sph = nullptr;
    double* sph_dirs = nullptr;
    Pair32* sph_part = nullptr;
    int sph_cap = 0, sph_dirs_cap = 0, sph_max_n = 0;
    // the caller's last frame of each environment, and the frame acceleration
    // an attached sphere's box reaction adds to it
    std::vector<fg_frame> user_frame;
    std::vector<std::array<double, 3>> box_acc;
    bool profiling = false;
    std::vector<cudaEvent_t> ev[FG_K_COUNT];
    int ev_used[FG_K_COUNT] = {0, 0, 0};
    double prof_ms[FG_K_COUNT] = {0, 0, 0};
    long long prof_n[FG_K_COUNT] = {0, 0, 0};
};

namespace {

// Torque points of every environment's segment rows: its own points when
// set, else the environment's reference point (device copy in FP32, like the
// marker positions the reduction subtracts them from).
fg_status upload_seg_refs(fg_domain* d) {
    std::vector<float> h((size_t)d->n_envs * MAX_SEG * 3);
    for (int e = 0; e < d->n_envs; ++e)
        for (int sg = 0; sg < MAX_SEG; ++sg)
            for (int a = 0; a < 3; ++a)
                h[((size_t)e * MAX_SEG + sg) * 3 + a] =
                    (float)(d->mk[e].has_seg_ref ? d->mk[e].seg_ref[sg][a] : d->mk[e].ref[a]);
    CK(cudaMemcpyAsync(d->seg_ref, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));   // h is released on return
    return FG_OK;
}

fg_status upload_env(fg_domain* d) {
    CK(cudaMemcpyAsync(d->d_env, d->env.data(), sizeof(EnvDev) * d->n_envs, cudaMemcpyHostToDevice,
                       d->stream));
    return FG_OK;
}

// Byte offset of the marker source after the frames (aligned for its pointers).
size_t msrc_offset(int n_envs) { return (sizeof(FrameDev) * (size_t)n_envs + 15) & ~(size_t)15; }

// The frames; with a marker source posted for the next step, the source in
// the same copy (pageable: the copy takes the bytes when it is issued).
fg_status upload_frames(fg_domain* d) {
    if (!d->msrc_next.valid) {
        CK(cudaMemcpyAsync(d->d_frame, d->frame.data(), sizeof(FrameDev) * d->n_envs,
                           cudaMemcpyHostToDevice, d->stream));
        return FG_OK;
    }
    const size_t off = msrc_offset(d->n_envs);
    unsigned char buf[sizeof(FrameDev) * 4 + 16 + sizeof(MarkerSrc)];
    std::vector<unsigned char> big;
    unsigned char* b = buf;
    if (off + sizeof(MarkerSrc) > sizeof(buf)) {
        big.resize(off + sizeof(MarkerSrc));
        b = big.data();
    }
    std::memcpy(b, d->frame.data(), sizeof(FrameDev) * d->n_envs);
    std::memcpy(b + off, &d->msrc_next, sizeof(MarkerSrc));
    CK(cudaMemcpyAsync(d->d_frame, b, off + sizeof(MarkerSrc), cudaMemcpyHostToDevice, d->stream));
    d->msrc_next.valid = 0;
    return FG_OK;
}

// A posted marker source alone (a step without a new frame).
fg_status upload_msrc(fg_domain* d) {
    if (!d->msrc_next.valid) return FG_OK;
    const MarkerSrc m = d->msrc_next;
    CK(cudaMemcpyAsync(d->d_msrc, &m, sizeof(MarkerSrc), cudaMemcpyHostToDevice, d->stream));
    d->msrc_next.valid = 0;
    return FG_OK;
}

void set_frame(FrameDev& f, const fg_frame& src) {
    double oo = 0;
    for (int a = 0; a < 3; ++a) {
        f.acc[a] = (float)src.acc[a];
        f.om[a] = (float)src.omega[a];
        f.dom[a] = (float)src.domega[a];
        f.org[a] = (float)src.origin[a];
        oo += src.omega[a] * src.omega[a];
    }
    f.inv_1pom2 = (float)(1.0 / (1.0 + oo));
    // a0(p) = -acc - domega x r - omega x (omega x r), r = p - origin
    //       = c0 - M p,  M = [domega]x + omega omega^T - |omega|^2 I,  c0 = -acc + M origin
    const double* w = src.omega;
    const double* dw = src.domega;
    double M[9] = {0.0, -dw[2], dw[1], dw[2], 0.0, -dw[0], -dw[1], dw[0], 0.0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[3 * a + b] += w[a] * w[b] - (a == b ? oo : 0.0);
    for (int k = 0; k < 9; ++k) f.M[k] = (float)M[k];
    for (int a = 0; a < 3; ++a) {
        double c = -src.acc[a];
        for (int b = 0; b < 3; ++b) c += M[3 * a + b] * src.origin[b];
        f.c0[a] = (float)c;
    }
}

// The caller's frame of environment e plus the box reaction of a sphere
// attached there.
void set_env_frame(fg_domain* d, int e, const fg_frame& f) {
    d->user_frame[e] = f;
    fg_frame g = f;
    for (int a = 0; a < 3; ++a) g.acc[a] += d->box_acc[e][a];
    set_frame(d->frame[e], g);
}

fg_status sphere_download(fg_domain* d);
fg_status sphere_upload(fg_domain* d);

// Whether a sphere is attached to environment env.
bool has_sphere(const fg_domain* d, int env) {
    for (const SphereDev& s : d->sph_host)
        if (s.env == env) return true;
    return false;
}

void free_all(fg_domain* d) {
    if (!d) return;
    for (int p = 0; p < 2; ++p)
        if (d->graph[p]) cudaGraphExecDestroy(d->graph[p]);
    void* adj[] = {d->adj_lam[0], d->adj_lam[1], d->adj_lfib, d->adj_lrho, d->adj_lut, d->adj_gF};
    for (void* p : adj)
        if (p) cudaFree(p);
    void* ptrs[] = {d->d_env, d->d_frame, d->pop[0], d->pop[1] != d->pop[0] ? d->pop[1] : nullptr, d->fib, d->stamps, d->ib_nodes, d->ib_bar,
                    d->fibq, d->mass_part, d->red_partials, d->red_counters, d->d_state,
                    d->X, d->U, d->dV, d->Fm, d->dF, d->Nrm, d->seg, d->seg_ref, d->region_part, d->mk_stage, d->ft, d->mass,
                    d->hist, d->status, d->work_segs, d->work, d->work_done, d->sph, d->sph_dirs, d->sph_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (d->rb) cudaFreeHost(d->rb);
    if (d->rb_ft_all) cudaFreeHost(d->rb_ft_all);
    for (int k = 0; k < FG_K_COUNT; ++k)
        for (cudaEvent_t e : d->ev[k]) cudaEventDestroy(e);
    if (d->blk_flag) cudaFree(d->blk_flag);
    if (d->ev_fork) cudaEventDestroy(d->ev_fork);
    if (d->ev_join) cudaEventDestroy(d->ev_join);
    if (d->stream2) cudaStreamDestroy(d->stream2);
}

template <class T>
fg_status dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    const unsigned long long cap = g_alloc_cap.load(std::memory_order_relaxed);
    if (cap != 0 && sizeof(T) * count > cap) return fail(FG_ERR_OOM, "allocation above the fg_set_alloc_cap limit");
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    return FG_OK;
}

// Chunk-sum scratch of k_reduce, sized for the current marker capacities.
fg_status ensure_reduce_scratch(fg_domain* d) {
    int z = 1;
    for (int e = 0; e < d->n_envs; ++e) {
        z = std::max(z, (d->mk[e].cap + RED_THREADS - 1) / RED_THREADS);
        z = std::max(z, (d->env[e].nparts + RED_THREADS * MASS_PER_THREAD - 1) / (RED_THREADS * MASS_PER_THREAD));
    }
    if (d->red_partials && z <= d->red_z) return FG_OK;
    Pair32* p = nullptr;
    fg_status st = dalloc(&p, (size_t)d->n_envs * RED_ROWS * z * 6);
    if (st != FG_OK) return st;
    CK(cudaStreamSynchronize(d->stream));
    if (d->red_partials) cudaFree(d->red_partials);
    d->red_partials = p;
    d->red_z = z;
    return FG_OK;
}

// Grid rows and chunks of k_reduce for the current markers and kernel
// layout: the force/torque rows of the environment with the most segments
// plus the mass row, and the most chunks any environment's rows need (at
// most red_z, the partials' stride).  Launching only these leaves out the
// blocks of unused rows and chunks (RED_ROWS x red_z for 64 fish of five
// segments was 18 x 16, 60% of it rows no environment has).
void reduce_grid(const fg_domain* d, bool markers_pre, int* rows, int* chunks) {
    int r = 1, z = 1;
    for (int e = 0; e < d->n_envs; ++e) {
        const EnvDev& E = d->env[e];
        r = std::max(r, E.nseg + 2);
        z = std::max(z, (E.n_markers + RED_THREADS - 1) / RED_THREADS);
        z = std::max(z, (E.nparts + RED_THREADS * MASS_PER_THREAD - 1) / (RED_THREADS * MASS_PER_THREAD));
    }
    *rows = markers_pre ? 1 : std::min(r, RED_ROWS);
    *chunks = std::min(z, d->red_z);
}

// Re-layout marker storage so environment env can hold n markers.
fg_status grow_markers(fg_domain* d, int env, int n) {
    std::vector<MarkerRegion> nr = d->mk;
    nr[env].cap = std::max(n, std::max(2 * nr[env].cap, 64));
    int off = 0;
    for (auto& r : nr) {
        r.off = off;
        off += r.cap;
    }
    float *X, *U, *dV, *Fm, *dF, *Nr;
    int* sg;
    fg_status s;
    if ((s = dalloc(&X, 3ull * off)) != FG_OK) return s;
    if ((s = dalloc(&U, 3ull * off)) != FG_OK) { cudaFree(X); return s; }
    if ((s = dalloc(&dV, off)) != FG_OK) { cudaFree(X); cudaFree(U); return s; }
    if ((s = dalloc(&Fm, 3ull * off)) != FG_OK) { cudaFree(X); cudaFree(U); cudaFree(dV); return s; }
    if ((s = dalloc(&sg, off)) != FG_OK) {
        cudaFree(X); cudaFree(U); cudaFree(dV); cudaFree(Fm);
        return s;
    }
    if ((s = dalloc(&dF, 3ull * off)) != FG_OK) {
        cudaFree(X); cudaFree(U); cudaFree(dV); cudaFree(Fm); cudaFree(sg);
        return s;
    }
    if ((s = dalloc(&Nr, 3ull * off)) != FG_OK) {
        cudaFree(X); cudaFree(U); cudaFree(dV); cudaFree(Fm); cudaFree(sg); cudaFree(dF);
        return s;
    }
    for (int e = 0; e < d->n_envs; ++e) {
        const MarkerRegion& o = d->mk[e];
        if (o.n == 0) continue;
        CK(cudaMemcpyAsync(X + 3ull * nr[e].off, d->X + 3ull * o.off, sizeof(float) * 3 * o.n,
                           cudaMemcpyDeviceToDevice, d->stream));
        CK(cudaMemcpyAsync(U + 3ull * nr[e].off, d->U + 3ull * o.off, sizeof(float) * 3 * o.n,
                           cudaMemcpyDeviceToDevice, d->stream));
        CK(cudaMemcpyAsync(dV + nr[e].off, d->dV + o.off, sizeof(float) * o.n,
                           cudaMemcpyDeviceToDevice, d->stream));
        CK(cudaMemcpyAsync(Fm + 3ull * nr[e].off, d->Fm + 3ull * o.off, sizeof(float) * 3 * o.n,
                           cudaMemcpyDeviceToDevice, d->stream));
        CK(cudaMemcpyAsync(sg + nr[e].off, d->seg + o.off, sizeof(int) * o.n,
                           cudaMemcpyDeviceToDevice, d->stream));
        CK(cudaMemcpyAsync(Nr + 3ull * nr[e].off, d->Nrm + 3ull * o.off, sizeof(float) * 3 * o.n,
                           cudaMemcpyDeviceToDevice, d->stream));
    }
    CK(cudaStreamSynchronize(d->stream));
    if (d->X) {
        cudaFree(d->X); cudaFree(d->U); cudaFree(d->dV); cudaFree(d->Fm); cudaFree(d->seg); cudaFree(d->dF);
        cudaFree(d->Nrm);
    }
    d->X = X; d->U = U; d->dV = dV; d->Fm = Fm; d->seg = sg; d->dF = dF; d->Nrm = Nr;
    d->marker_slots = off;
    d->mk = nr;
    return ensure_reduce_scratch(d);
}

void refresh_marker_table(fg_domain* d) {
    int begin = 0;
    for (int e = 0; e < d->n_envs; ++e) {
        EnvDev& E = d->env[e];
        E.mk_begin = begin;
        E.n_markers = d->mk[e].n;
        E.marker_off = d->mk[e].off;
        E.nseg = d->mk[e].nseg;
        for (int a = 0; a < 3; ++a) E.ref[a] = d->mk[e].ref[a];
        begin += d->mk[e].n;
    }
    d->total_markers = begin;
    d->work_dirty = true;
}

// Work queue of the fused step kernel for the current markers and kernel
// layout, in queue order.  One environment's IB phases: MARK, NODE, FORCE,
// (INTERP, SPREAD) per extra direct-forcing pass, CONVERT (deterministic
// spread), REDUCE; then its stream-collide blocks (SC).  With several
// environments the IB phases of environment e + 1 come before the SC blocks
// of environment e, so they run beside them: IB(0) IB(1) SC(0) IB(2) SC(1)
// ... SC(n-1).  Every dependency points to earlier items of the same
// environment.
void build_work_table(fg_domain* d) {
    std::vector<WorkSeg>& w = d->work_host;
    w.clear();
    int pos = 0;
    auto add = [&](int kind, int e, int count, int slot, int dep_slot, int dep_count, int pass, int per) {
        if (count <= 0) return;
        WorkSeg g;
        std::memset(&g, 0, sizeof(g));
        g.begin = pos; g.count = count; g.kind = kind; g.env = e; g.slot = slot;
        g.dep_slot = dep_count > 0 ? dep_slot : -1;
        g.dep_count = dep_count; g.cond_slot = -1; g.cond_count = 0; g.pass = pass; g.per_item = per;
        w.push_back(g);
        pos += count;
    };
    const int M = d->opt.ib_iters;
    std::vector<int> ib_slot(d->n_envs, SLOT_MARK), ib_count(d->n_envs, 0);
    auto ib_phases = [&](int e) {
        const EnvDev& E = d->env[e];
        const int n = d->mk[e].n;
        if (n == 0) return;
        const int nm = (n + MARKERS_PER_ITEM - 1) / MARKERS_PER_ITEM;
        const int ntiles = (int)((E.nslot + 31u) / 32u);
        const int nn = (ntiles + TILES_PER_ITEM - 1) / TILES_PER_ITEM;
        add(W_MARK, e, nm, SLOT_MARK, -1, 0, 0, MARKERS_PER_ITEM);
        add(W_NODE, e, nn, SLOT_NODE, SLOT_MARK, nm, 0, TILES_PER_ITEM);
        add(W_FORCE, e, nm, SLOT_FORCE, SLOT_NODE, nn, 0, MARKERS_PER_ITEM);
        int last = SLOT_FORCE, force_final = SLOT_FORCE;
        for (int p = 1; p < M; ++p) {
            const int si = SLOT_PASS0 + 2 * (p - 1), ss = si + 1;
            add(W_INTERP, e, nm, si, last, nm, p, MARKERS_PER_ITEM);
            add(W_SPREAD, e, nm, ss, si, nm, p, MARKERS_PER_ITEM);
            last = ss;
            force_final = si;
        }
        int final_slot = last, final_count = nm;
        if (d->opt.deterministic) {
            add(W_CONVERT, e, nn, SLOT_CONVERT, last, nm, 0, TILES_PER_ITEM);
            final_slot = SLOT_CONVERT;
            final_count = nn;
        }
        add(W_REDUCE, e, (n + FUSED_THREADS - 1) / FUSED_THREADS, SLOT_REDUCE, force_final, nm, 0, FUSED_THREADS);
        ib_slot[e] = final_slot;
        ib_count[e] = final_count;
    };
    auto sc_blocks = [&](int e) {
        const int n = d->mk[e].n;
        const int nm = n > 0 ? (n + MARKERS_PER_ITEM - 1) / MARKERS_PER_ITEM : 0;
        const size_t at = w.size();
        add(W_SC, e, d->env[e].nblocks, SLOT_SC, SLOT_MARK, nm, 0, 0);
        if (w.size() > at) {
            w.back().cond_slot = ib_count[e] > 0 ? ib_slot[e] : -1;
            w.back().cond_count = ib_count[e];
        }
    };
    ib_phases(0);
    for (int e = 0; e < d->n_envs; ++e) {
        if (e + 1 < d->n_envs) ib_phases(e + 1);
        sc_blocks(e);
    }
}

// Upload the fused kernel's work table if it is out of date (on the stream,
// before the step's launches; never inside a capture).
fg_status sync_work_table(fg_domain* d) {
    if (d->k1 != K1_FUSED || !d->work_dirty) return FG_OK;
    build_work_table(d);
    const int n = (int)d->work_host.size();
    if (n > d->work_seg_cap) {
        WorkSeg* p = nullptr;
        fg_status st = dalloc(&p, (size_t)std::max(n, 2 * d->work_seg_cap));
        if (st != FG_OK) return st;
        CK(cudaStreamSynchronize(d->stream));
        if (d->work_segs) cudaFree(d->work_segs);
        d->work_segs = p;
        d->work_seg_cap = std::max(n, 2 * d->work_seg_cap);
    }
    const int items = n > 0 ? d->work_host.back().begin + d->work_host.back().count : 0;
    const int hdr[2] = {items, n};
    if (n > 0)
        CK(cudaMemcpyAsync(d->work_segs, d->work_host.data(), sizeof(WorkSeg) * n, cudaMemcpyHostToDevice,
                           d->stream));
    CK(cudaMemcpyAsync(d->work + WQ_ITEMS, hdr, sizeof(hdr), cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));   // the host table may change on the next call
    d->work_dirty = false;
    return FG_OK;
}

// The stream-collide launch of the variant in use (gin -> gout), with the
// equilibrium order of the domain.
template <class S, int GC, bool EQ3>
void enqueue_staged(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s) {
    if (d->staged_pair)
        k_stream_collide_staged<S, GC, staged_minb<S, GC, true>(), EQ3, true>
            <<<d->staged_grid, K1_THREADS, d->staged_smem, s>>>(gin, gout, d->d_env, d->d_frame, d->n_envs,
                                                                d->total_groups, d->fib, d->stamps, d->d_state,
                                                                d->mass_part, d->status, d->sweep_reverse);
    else
        k_stream_collide_staged<S, GC, staged_minb<S, GC, false>(), EQ3, false>
            <<<d->staged_grid, K1_THREADS, d->staged_smem, s>>>(gin, gout, d->d_env, d->d_frame, d->n_envs,
                                                                d->total_groups, d->fib, d->stamps, d->d_state,
                                                                d->mass_part, d->status, d->sweep_reverse);
}

template <class S, bool EQ3>
void enqueue_k1_order(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s) {
    if (d->k1 == K1_STAGED256) {
        enqueue_staged<S, 256, EQ3>(d, gin, gout, s);
    } else if (d->k1 == K1_STAGED512) {
        enqueue_staged<S, 512, EQ3>(d, gin, gout, s);
    } else {
        if (d->plain_pair)
            k_stream_collide<S, EQ3, true><<<d->total_blocks, K1_THREADS, 0, s>>>(
                gin, gout, d->d_env, d->d_frame, d->n_envs, d->fib, d->stamps, d->d_state, d->mass_part, nullptr,
                K1_ALL_BLOCKS, d->sweep_reverse);
        else
        k_stream_collide<S, EQ3><<<d->total_blocks, K1_THREADS, 0, s>>>(
            gin, gout, d->d_env, d->d_frame, d->n_envs, d->fib, d->stamps, d->d_state, d->mass_part, nullptr,
            K1_ALL_BLOCKS, d->sweep_reverse);
    }
}

template <class S>
void enqueue_k1(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s) {
    if (d->opt.eq_order == 3) enqueue_k1_order<S, true>(d, gin, gout, s);
    else enqueue_k1_order<S, false>(d, gin, gout, s);
}

// The cooperative IB kernel of a step reading gin (all resident blocks: the
// scan phase covers every tile stamp).
template <class S>
fg_status enqueue_ib(fg_domain* d, const typename S::raw* gin, cudaStream_t s, int layout = LAYOUT_PULL) {
    const int blocks = d->ib_per_sm * d->n_sms;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(IB_THREADS);
    cfg.dynamicSmemBytes = ib_smem_bytes(d->n_envs);   // the environments' tables
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_ib_step<S>, gin, (const EnvDev*)d->d_env, (const FrameDev*)d->d_frame,
                          d->n_envs, d->total_markers, (int)d->n_stamps, d->X, d->U,
                          (const float*)d->dV, d->Fm, d->fib, d->stamps, (const StepState*)d->d_state,
                          d->ib_nodes, d->ib_bar, d->opt.ib_iters, d->dF, d->fibq,
                          (const float*)(d->opt.ib_slip ? d->Nrm : nullptr), d->status, layout,
                          (const MarkerSrc*)d->d_msrc));
    return FG_OK;
}

// The in-place stream-collide kernel of phase `phase` (0: even step).
// (the boundary-cell kernel first: it reads populations the stream-collide
// kernel overwrites).
template <class S, bool EQ3, bool PAIR>
void enqueue_aa_of(fg_domain* d, typename S::raw* g, int phase, cudaStream_t s) {
    const int xcells = PAIR ? 0 : 1;
    if (phase == 0) {
        if (d->total_bblocks > 0)
            k_aa_boundary<S, EQ3, 0><<<d->total_bblocks, K1_THREADS, 0, s>>>(g, d->d_env, d->d_frame, d->n_envs,
                                                                            d->mass_part, xcells);
        k_stream_collide_aa<S, EQ3, PAIR, 0><<<d->total_blocks, K1_THREADS, 0, s>>>(
            g, d->d_env, d->d_frame, d->n_envs, d->fib, d->stamps, d->d_state, d->mass_part);
    } else {
        if (d->total_bblocks > 0)
            k_aa_boundary<S, EQ3, 1><<<d->total_bblocks, K1_THREADS, 0, s>>>(g, d->d_env, d->d_frame, d->n_envs,
                                                                            d->mass_part, xcells);
        k_stream_collide_aa<S, EQ3, PAIR, 1><<<d->total_blocks, K1_THREADS, 0, s>>>(
            g, d->d_env, d->d_frame, d->n_envs, d->fib, d->stamps, d->d_state, d->mass_part);
    }
}

template <class S>
void enqueue_aa(fg_domain* d, typename S::raw* g, int phase, cudaStream_t s) {
    const bool eq3 = d->opt.eq_order == 3;
    if (d->plain_pair) {
        if (eq3) enqueue_aa_of<S, true, true>(d, g, phase, s);
        else enqueue_aa_of<S, false, true>(d, g, phase, s);
    } else {
        if (eq3) enqueue_aa_of<S, true, false>(d, g, phase, s);
        else enqueue_aa_of<S, false, false>(d, g, phase, s);
    }
}

// The plain stream-collide kernel over the blocks `which` selects, on
// stream s, at the given launch priority (0: the stream's own).
template <class S, bool EQ3, bool PAIR>
fg_status enqueue_plain_of(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s,
                           int which, int priority) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d->total_blocks);
    cfg.blockDim = dim3(K1_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = priority;
    cfg.attrs = attr;
    cfg.numAttrs = priority != 0 ? 1 : 0;
    CK(cudaLaunchKernelEx(&cfg, k_stream_collide<S, EQ3, PAIR>, gin, gout, (const EnvDev*)d->d_env,
                          (const FrameDev*)d->d_frame, d->n_envs, d->fib, (const uint32_t*)d->stamps,
                          (const StepState*)d->d_state, d->mass_part, (const uint32_t*)d->blk_flag, which,
                          d->sweep_reverse));
    return FG_OK;
}

template <class S>
fg_status enqueue_plain(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s, int which,
                        int priority) {
    const bool eq3 = d->opt.eq_order == 3;
    if (d->plain_pair)
        return eq3 ? enqueue_plain_of<S, true, true>(d, gin, gout, s, which, priority)
                   : enqueue_plain_of<S, false, true>(d, gin, gout, s, which, priority);
    return eq3 ? enqueue_plain_of<S, true, false>(d, gin, gout, s, which, priority)
               : enqueue_plain_of<S, false, false>(d, gin, gout, s, which, priority);
}

// The IB beside the stream-collide kernel (markers present): k_mark_tiles
// stamps the stencil tiles and flags their blocks on stream s; a second,
// high-priority stream then runs the IB phases as separate kernels
// (k_ib_tiles, k_ib_markers) and the flagged blocks, while s runs the
// unflagged blocks; s joins the second stream at the end.  With ev, the IB
// phases are timed on the second stream and the stream-collide section
// (from the unflagged launch to the join) on s.
template <class S>
fg_status enqueue_overlap(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s,
                          cudaEvent_t* const* ev) {
    const int mblocks = (int)(((long long)d->total_markers * 16 + IB_THREADS - 1) / IB_THREADS);
    k_mark_tiles<<<mblocks, IB_THREADS, 0, s>>>((const EnvDev*)d->d_env, d->n_envs, d->total_markers,
                                                (const float*)d->X, (const StepState*)d->d_state, d->stamps,
                                                d->blk_flag, d->plain_pair ? 9 : 8);
    CK(cudaGetLastError());
    CK(cudaEventRecord(d->ev_fork, s));
    CK(cudaStreamWaitEvent(d->stream2, d->ev_fork, 0));
    if (ev) CK(cudaEventRecord(ev[FG_K_IB][0], d->stream2));
    {
        // the IB phases as separate launches at the high priority
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributePriority;
        attr[0].val.priority = d->prio_high;
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(IB_THREADS);
        cfg.stream = d->stream2;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const int tile_blocks = std::max(1, std::min(4 * d->n_sms, (int)((d->n_stamps + 4095) / 4096)));
        const int mk_blocks = (int)(((long long)d->total_markers * 16 + IB_THREADS - 1) / IB_THREADS);
        const float* nrm = d->opt.ib_slip ? d->Nrm : nullptr;
        cfg.gridDim = dim3((unsigned)tile_blocks);
        CK(cudaLaunchKernelEx(&cfg, k_ib_tiles<S, false>, gin, (const EnvDev*)d->d_env, (const FrameDev*)d->d_frame,
                              d->n_envs, (int)d->n_stamps, (const uint32_t*)d->stamps, (const StepState*)d->d_state,
                              d->ib_nodes, d->fib, d->fibq));
        cfg.gridDim = dim3((unsigned)mk_blocks);
        CK(cudaLaunchKernelEx(&cfg, k_ib_markers<S, false>, (const EnvDev*)d->d_env, d->n_envs, d->total_markers,
                              (const float*)d->X, (const float*)d->U, (const float*)d->dV, d->Fm, d->fib,
                              (const float4*)d->ib_nodes, d->dF, d->fibq, nrm, 0, d->status));
        for (int pass = 1; pass < d->opt.ib_iters; ++pass) {
            CK(cudaLaunchKernelEx(&cfg, k_ib_markers<S, false>, (const EnvDev*)d->d_env, d->n_envs,
                                  d->total_markers, (const float*)d->X, (const float*)d->U, (const float*)d->dV,
                                  d->Fm, d->fib, (const float4*)d->ib_nodes, d->dF, d->fibq, nrm, pass, d->status));
            CK(cudaLaunchKernelEx(&cfg, k_ib_markers<S, true>, (const EnvDev*)d->d_env, d->n_envs,
                                  d->total_markers, (const float*)d->X, (const float*)d->U, (const float*)d->dV,
                                  d->Fm, d->fib, (const float4*)d->ib_nodes, d->dF, d->fibq, nrm, pass, d->status));
        }
        if (d->fibq) {
            cfg.gridDim = dim3((unsigned)tile_blocks);
            CK(cudaLaunchKernelEx(&cfg, k_ib_tiles<S, true>, gin, (const EnvDev*)d->d_env,
                                  (const FrameDev*)d->d_frame, d->n_envs, (int)d->n_stamps,
                                  (const uint32_t*)d->stamps, (const StepState*)d->d_state, d->ib_nodes, d->fib,
                                  d->fibq));
        }
    }
    if (ev) CK(cudaEventRecord(ev[FG_K_IB][1], d->stream2));
    fg_status st = enqueue_plain<S>(d, gin, gout, d->stream2, K1_FLAGGED_BLOCKS, d->prio_high);
    if (st != FG_OK) return st;
    CK(cudaEventRecord(d->ev_join, d->stream2));
    if (ev) CK(cudaEventRecord(ev[FG_K_STREAM_COLLIDE][0], s));
    if ((st = enqueue_plain<S>(d, gin, gout, s, K1_UNFLAGGED_BLOCKS, 0)) != FG_OK) return st;
    CK(cudaStreamWaitEvent(s, d->ev_join, 0));
    if (ev) CK(cudaEventRecord(ev[FG_K_STREAM_COLLIDE][1], s));
    return FG_OK;
}

// The fused step kernel (IB phases and stream-collide blocks of every
// environment from one work queue; all blocks resident) reading gin and
// writing gout.
template <class S, bool EQ3, bool PAIR>
fg_status enqueue_fused_of(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d->fused_grid);
    cfg.blockDim = dim3(FUSED_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    IbArgs a;
    a.envs = d->d_env;
    a.frames = d->d_frame;
    a.X = d->X;
    a.U = d->U;
    a.dV = d->dV;
    a.Fm = d->Fm;
    a.fib = d->fib;
    a.stamps = d->stamps;
    a.nodes = d->ib_nodes;
    a.dF = d->dF;
    a.fibq = d->fibq;
    a.Nrm = d->opt.ib_slip ? d->Nrm : nullptr;
    a.status = d->status;
    CK(cudaLaunchKernelEx(&cfg, k_step_fused<S, EQ3, PAIR>, gin, gout, a, (const StepState*)d->d_state,
                          (const int*)d->seg, (const float*)d->seg_ref, d->red_partials, d->red_z, d->mass_part,
                          (const WorkSeg*)d->work_segs, d->work, d->work_done, d->n_envs));
    return FG_OK;
}

template <class S>
fg_status enqueue_fused(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s) {
    const bool eq3 = d->opt.eq_order == 3;
    if (d->plain_pair)
        return eq3 ? enqueue_fused_of<S, true, true>(d, gin, gout, s) : enqueue_fused_of<S, false, true>(d, gin, gout, s);
    return eq3 ? enqueue_fused_of<S, true, false>(d, gin, gout, s) : enqueue_fused_of<S, false, false>(d, gin, gout, s);
}

// Launch the kernels of one step reading gin and writing gout on stream s;
// with ev != nullptr an event pair is recorded around each kernel (the fused
// kernel counts as the stream-collide kernel; it has no separate IB launch).
// aa_phase >= 0: the in-place layout at that phase (gin == gout, the one
// buffer).
template <class S>
fg_status enqueue_step_io(fg_domain* d, const typename S::raw* gin, typename S::raw* gout, cudaStream_t s,
                          cudaEvent_t* const* ev, int aa_phase = -1) {
    const bool fused = d->k1 == K1_FUSED;
    const bool overlap = d->k1 == K1_OVERLAP && d->total_markers > 0;
    const int n_sph = (int)d->sph_host.size();
    if (n_sph > 0)   // attached spheres: their markers from the body state
        k_sphere_place<<<dim3((unsigned)((d->sph_max_n + 255) / 256), (unsigned)n_sph), 256, 0, s>>>(
            d->sph, d->sph_dirs, d->X, d->U, d->d_env, d->seg_ref);
    if (aa_phase >= 0) {
        if (d->total_markers > 0) {
            if (ev) CK(cudaEventRecord(ev[FG_K_IB][0], s));
            fg_status st = enqueue_ib<S>(d, gin, s, aa_phase == 0 ? LAYOUT_AA0 : LAYOUT_AA1);
            if (st != FG_OK) return st;
            if (ev) CK(cudaEventRecord(ev[FG_K_IB][1], s));
        }
        if (ev) CK(cudaEventRecord(ev[FG_K_STREAM_COLLIDE][0], s));
        enqueue_aa<S>(d, gout, aa_phase, s);
        if (ev) CK(cudaEventRecord(ev[FG_K_STREAM_COLLIDE][1], s));
    } else if (overlap) {
        fg_status st = enqueue_overlap<S>(d, gin, gout, s, ev);
        if (st != FG_OK) return st;
    } else {
        if (!fused && d->total_markers > 0) {
            if (ev) CK(cudaEventRecord(ev[FG_K_IB][0], s));
            fg_status st = enqueue_ib<S>(d, gin, s);
            if (st != FG_OK) return st;
            if (ev) CK(cudaEventRecord(ev[FG_K_IB][1], s));
        }
        if (ev) CK(cudaEventRecord(ev[FG_K_STREAM_COLLIDE][0], s));
        if (fused) {
            fg_status st = enqueue_fused<S>(d, gin, gout, s);
            if (st != FG_OK) return st;
        } else {
            enqueue_k1<S>(d, gin, gout, s);
        }
        if (ev) CK(cudaEventRecord(ev[FG_K_STREAM_COLLIDE][1], s));
    }
    if (ev) CK(cudaEventRecord(ev[FG_K_REDUCE][0], s));
    {
        // a programmatic dependent of the stream-collide kernel: its marker
        // sums overlap that kernel's last blocks, the rest waits for it (after
        // the fused kernel, which wrote the marker chunk sums, only the mass
        // is summed)
        cudaLaunchConfig_t cfg = {};
        int gy = 1, gz = 1;
        reduce_grid(d, fused, &gy, &gz);
        cfg.gridDim = dim3((unsigned)d->n_envs, (unsigned)gy, (unsigned)gz);
        cfg.blockDim = dim3(RED_THREADS);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, k_reduce, (const EnvDev*)d->d_env, (const float*)d->X, (const float*)d->Fm,
                              (const float*)d->dV, (const int*)d->seg, (const float*)d->seg_ref,
                              (const Pair32*)d->mass_part, d->red_partials, d->red_counters, d->n_envs, d->red_z,
                              d->ft, d->mass, d->hist, d->opt.record_history, d->d_state, d->status,
                              d->rb_ft_all_dev, d->rb_status_dev, d->rb_seq_dev, fused ? 1 : 0, d->d_msrc));
    }
    if (ev) CK(cudaEventRecord(ev[FG_K_REDUCE][1], s));
    if (n_sph > 0) {
        // the inner fluid's momentum in the new state, then the body update
        const int grid = 4 * d->n_sms;
        k_sphere_fluid<S><<<dim3((unsigned)grid, (unsigned)n_sph), RED_THREADS, 0, s>>>(
            gout, d->d_env, d->sph, aa_phase < 0 ? -1 : (aa_phase ^ 1), d->sph_part);
        k_sphere_update<<<n_sph, 32, 0, s>>>(d->sph, d->sph_part, grid, d->ft, 0);
    }
    CK(cudaGetLastError());
    return FG_OK;
}

template <class S>
fg_status enqueue_step(fg_domain* d, int parity, cudaStream_t s, cudaEvent_t* const* ev) {
    typedef typename S::raw raw;
    d->sweep_reverse = parity;
    const fg_status st = enqueue_step_io<S>(d, (const raw*)d->pop[parity], (raw*)d->pop[parity ^ 1], s, ev,
                                            d->aa ? parity : -1);
    d->sweep_reverse = 0;
    return st;
}

// One step with direct launches (and per-kernel events when profiling).
template <class S>
fg_status launch_step(fg_domain* d) {
    cudaEvent_t* evp[FG_K_COUNT] = {nullptr, nullptr, nullptr};
    bool use_ev = false;
    if (d->profiling) {
        for (int k = 0; k < FG_K_COUNT; ++k) {
            if (d->ev_used[k] + 2 > (int)d->ev[k].size()) {
                // drain: accumulate what is recorded so far
                CK(cudaStreamSynchronize(d->stream));
                for (int i = 0; i + 1 < d->ev_used[k]; i += 2) {
                    float ms = 0;
                    CK(cudaEventElapsedTime(&ms, d->ev[k][i], d->ev[k][i + 1]));
                    d->prof_ms[k] += ms;
                    d->prof_n[k] += 1;
                }
                d->ev_used[k] = 0;
            }
            evp[k] = &d->ev[k][d->ev_used[k]];
            if (k != FG_K_IB || (d->total_markers > 0 && d->k1 != K1_FUSED)) d->ev_used[k] += 2;
        }
        use_ev = true;
    }
    fg_status st = enqueue_step<S>(d, d->cur, d->stream, use_ev ? evp : nullptr);
    if (st != FG_OK) return st;
    d->cur ^= 1;
    d->steps += 1;
    return FG_OK;
}

// One step replayed from a captured graph (captured on first use, and again
// whenever a launch parameter baked into it changes).
template <class S>
fg_status graph_step(fg_domain* d) {
    fg_domain::GraphKey key;
    key.X = d->X;
    key.red = d->red_partials;
    key.total_markers = d->total_markers;
    key.red_z = d->red_z;
    reduce_grid(d, d->k1 == K1_FUSED, &key.red_gy, &key.red_gz);
    key.sph = d->sph;
    key.n_sph = (int)d->sph_host.size();
    key.sph_max_n = d->sph_max_n;
    if (!(key == d->graph_key)) {
        for (int p = 0; p < 2; ++p)
            if (d->graph[p]) {
                cudaGraphExecDestroy(d->graph[p]);
                d->graph[p] = nullptr;
            }
        d->graph_key = key;
    }
    const int p = d->cur;
    if (!d->graph[p]) {
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            fg_status st = enqueue_step<S>(d, p, cs, nullptr);
            e = cudaStreamEndCapture(cs, &g);
            if (st != FG_OK) {
                if (g) cudaGraphDestroy(g);
                cudaStreamDestroy(cs);
                return st;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&d->graph[p], g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(e, "capturing the step graph");
    }
    CK(cudaGraphLaunch(d->graph[p], d->stream));
    d->cur ^= 1;
    d->steps += 1;
    return FG_OK;
}

template <class F>
fg_status dispatch(int storage, F&& f) {
    switch (storage) {
        case FG_F32: return f(StoreF32());
        case FG_F16: return f(StoreF16());
        case FG_BF16: return f(StoreBF16());
    }
    return fail(FG_ERR_INVALID, "unknown storage");
}


// Shared memory, occupancy and persistent grid of the staged kernel.
template <class S, int GC, bool EQ3, bool PAIR>
fg_status staged_occupancy_of(fg_domain* d, int* per_sm) {
    constexpr int MINB = staged_minb<S, GC, PAIR>();
    CK(cudaFuncSetAttribute(k_stream_collide_staged<S, GC, MINB, EQ3, PAIR>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->staged_smem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_stream_collide_staged<S, GC, MINB, EQ3, PAIR>,
                                                     K1_THREADS, d->staged_smem));
    return FG_OK;
}

// The shared-memory limit of the instantiation in use is raised and its
// occupancy returned.
template <class S, int GC>
fg_status staged_occupancy(fg_domain* d, int* per_sm) {
    const bool eq3 = d->opt.eq_order == 3;
    if (d->staged_pair)
        return eq3 ? staged_occupancy_of<S, GC, true, true>(d, per_sm)
                   : staged_occupancy_of<S, GC, false, true>(d, per_sm);
    return eq3 ? staged_occupancy_of<S, GC, true, false>(d, per_sm)
               : staged_occupancy_of<S, GC, false, false>(d, per_sm);
}

bool k1_runnable(const fg_domain* d, int v) {
    if (d->aa) return v == K1_PLAIN;   // the in-place layout has its own plain kernel only
    if (v == K1_PLAIN || v == K1_FUSED || v == K1_OVERLAP) return true;
    if (v == K1_STAGED256) return d->max_P <= 256;
    return v == K1_STAGED512 && d->max_P <= 512;
}

// Select the stream-collide variant: row groups, mass partials, persistent
// grid and shared memory follow from it.  With allocate, grows the buffers
// that depend on it and uploads the environment table (graphs are rebuilt).
fg_status configure_k1(fg_domain* d, int v, bool allocate) {
    if (!k1_runnable(d, v)) return fail(FG_ERR_INVALID, "stream-collide variant cannot run these rows");
    d->k1 = v;
    d->staged = v == K1_STAGED256 || v == K1_STAGED512;
    d->work_dirty = true;
    d->staged_gc = v == K1_STAGED512 ? 512 : 256;
    // 16-bit storage is bound by instruction issue, not by DRAM: two cells
    // per thread share the per-cell index work and store their outputs as
    // 32-bit pairs (needs every row length even).  FP32 is bound by DRAM and
    // measured no faster paired (153.6 against 154.8 us with 512 slots,
    // slower with 256, whose 64 registers then spill).
    d->staged_pair = d->staged && d->esize == 2;
    for (int e = 0; e < d->n_envs; ++e)
        if (d->env[e].n[0] % 2 != 0) d->staged_pair = false;
    // the plain kernel takes two cells per thread when every row length is
    // even: its blocks cover 2 x 256 slots
    d->plain_pair = !d->staged;
    for (int e = 0; e < d->n_envs; ++e)
        if (d->env[e].n[0] % 2 != 0) d->plain_pair = false;
    {
        const unsigned per_block = (d->plain_pair ? 2u : 1u) * K1_THREADS;
        int block0 = 0;
        for (int e = 0; e < d->n_envs; ++e) {
            EnvDev& E = d->env[e];
            E.block0 = block0;
            E.nblocks = (int)((E.nslot + per_block - 1) / per_block);
            block0 += E.nblocks;
        }
        d->total_blocks = block0;
    }
    int group0 = 0, bblock0 = 0, part0 = 0;
    for (int e = 0; e < d->n_envs; ++e) {
        EnvDev& E = d->env[e];
        E.rpg = std::max(1, std::min(d->staged_gc / E.P, (int)E.rows));
        E.group0 = group0;
        E.ngroups = (int)((E.rows + E.rpg - 1) / E.rpg);
        group0 += E.ngroups;
        // one mass partial per row group (staged) or per block (plain)
        E.part0 = d->staged ? E.group0 : E.block0;
        E.nparts = d->staged ? E.ngroups : E.nblocks;
        // in place: the boundary-cell kernel's blocks, and each environment's
        // partials of both kernels side by side
        E.nbnd = d->aa ? (int)aa_boundary_count(E, !d->plain_pair) : 0;
        E.bblock0 = bblock0;
        E.nbblocks = (E.nbnd + K1_THREADS - 1) / K1_THREADS;
        bblock0 += E.nbblocks;
        if (d->aa) {
            E.part0 = part0;
            E.nparts = E.nblocks + E.nbblocks;
            part0 += E.nparts;
        }
    }
    d->total_groups = group0;
    d->total_bblocks = bblock0;
    if (d->staged) {
        d->staged_smem = 2ull * 27 * d->staged_gc * d->esize;
        int dev = 0, sms = 0, per_sm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        fg_status st = dispatch(d->opt.storage, [&](auto tag) -> fg_status {
            typedef decltype(tag) S;
            return v == K1_STAGED256 ? staged_occupancy<S, 256>(d, &per_sm)
                                     : staged_occupancy<S, 512>(d, &per_sm);
        });
        if (st != FG_OK) return st;
        if (per_sm < 1) return fail(FG_ERR_INVALID, "staged kernel does not fit on an SM");
        d->staged_grid = std::min(d->total_groups, sms * per_sm);
    }
    if (v == K1_FUSED) {
        int per_sm = 0;
        fg_status st = dispatch(d->opt.storage, [&](auto tag) -> fg_status {
            typedef decltype(tag) S;
            const bool eq3 = d->opt.eq_order == 3;
            const void* fn = d->plain_pair ? (eq3 ? (const void*)k_step_fused<S, true, true>
                                                  : (const void*)k_step_fused<S, false, true>)
                                           : (eq3 ? (const void*)k_step_fused<S, true, false>
                                                  : (const void*)k_step_fused<S, false, false>);
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FUSED_THREADS, 0));
            return FG_OK;
        });
        if (st != FG_OK) return st;
        if (per_sm < 1) return fail(FG_ERR_CUDA, "fused step kernel cannot be resident");
        d->fused_grid = per_sm * d->n_sms;
    }
    if (!allocate) return FG_OK;
    const size_t need = (size_t)std::max(d->total_blocks + d->total_bblocks, d->total_groups);
    if (need > d->mass_part_cap) {
        Pair32* p = nullptr;
        fg_status st = dalloc(&p, need);
        if (st != FG_OK) return st;
        CK(cudaStreamSynchronize(d->stream));
        if (d->mass_part) cudaFree(d->mass_part);
        d->mass_part = p;
        d->mass_part_cap = need;
    }
    fg_status st = ensure_reduce_scratch(d);
    if (st != FG_OK) return st;
    for (int p = 0; p < 2; ++p)
        if (d->graph[p]) {
            cudaGraphExecDestroy(d->graph[p]);
            d->graph[p] = nullptr;
        }
    d->graph_key = fg_domain::GraphKey();
    return upload_env(d);
}

// The layout argument of the state kernels: -1 for two buffers, else the
// in-place phase.
int aa_of(const fg_domain* d) { return d->aa ? d->cur : -1; }

// FP64 value of a compensated pair produced on the device.
double pair_value(const Pair32& p) { return (double)p.hi + (double)p.lo; }

size_t env_cells(const fg_domain* d, int env) {
    return (size_t)d->env[env].n[0] * d->env[env].n[1] * d->env[env].n[2];
}

fg_status check_env(fg_domain* d, int env) {
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (env < 0 || env >= d->n_envs) return fail(FG_ERR_INVALID, "environment index out of range");
    return FG_OK;
}

}  // namespace

// Lets other translation units of the library report through fg_last_error.
void fl_set_last_error(const char* msg) { g_err = msg; }

extern "C" {

const char* fg_last_error(void) { return g_err.c_str(); }

fg_status fg_lattice(int* c, double* w) {
    if (!c || !w) return fail(FG_ERR_INVALID, "null output");
    for (int i = 0; i < Q; ++i) {
        c[3 * i] = cx(i); c[3 * i + 1] = cy(i); c[3 * i + 2] = cz(i);
        w[i] = wd(i);
    }
    return FG_OK;
}

fg_status fg_create_domain(const fg_env_desc* envs, int n_envs, const fg_options* opt, void* cuda_stream,
                           fg_domain** out) {
    g_err.clear();
    if (!envs || !out || n_envs < 1 || n_envs > 4096) return fail(FG_ERR_INVALID, "bad environment list");
    fg_options o{};
    o.storage = FG_F32; o.layout = 0; o.deterministic = 0; o.ib_iters = 1; o.record_history = 0; o.ib_slip = 0; o.eq_order = 2;
    o.kernel_variant = FG_KERNEL_AUTO;
    o.use_graphs = 1;
    o.autotune = 0;
    if (opt) o = *opt;
    if (o.kernel_variant < FG_KERNEL_AUTO || o.kernel_variant > FG_KERNEL_OVERLAP)
        return fail(FG_ERR_INVALID, "unknown kernel variant");
    if (o.storage < 0 || o.storage > 2) return fail(FG_ERR_INVALID, "unknown storage");
    if (o.layout != FG_LAYOUT_PULL && o.layout != FG_LAYOUT_AA) return fail(FG_ERR_INVALID, "unknown layout");
    if (o.layout == FG_LAYOUT_AA && o.kernel_variant != FG_KERNEL_AUTO && o.kernel_variant != FG_KERNEL_PLAIN)
        return fail(FG_ERR_INVALID, "the in-place layout runs the plain kernel only");
    if (o.ib_iters < 1 || o.ib_iters > FG_MAX_IB_ITERS) return fail(FG_ERR_INVALID, "ib_iters must be in [1, 8]");
    if (o.deterministic != 0 && o.deterministic != 1) return fail(FG_ERR_INVALID, "deterministic must be 0 or 1");
    if (o.ib_slip != 0 && o.ib_slip != 1) return fail(FG_ERR_INVALID, "ib_slip must be 0 or 1");
    if (o.eq_order != 2 && o.eq_order != 3) return fail(FG_ERR_INVALID, "eq_order must be 2 or 3");
    if (o.record_history < 0 || o.record_history > (1 << 20)) return fail(FG_ERR_INVALID, "record_history");
    unsigned long long cells = 0;
    for (int e = 0; e < n_envs; ++e) {
        const fg_env_desc& E = envs[e];
        int n[3] = {E.nx, E.ny, E.nz};
        for (int a = 0; a < 3; ++a) {
            if (n[a] < 1 || n[a] > 65536) return fail(FG_ERR_INVALID, "grid size out of range");
            int lo = E.face[2 * a], hi = E.face[2 * a + 1];
            if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return fail(FG_ERR_INVALID, "unknown face kind");
            if ((lo == FG_PERIODIC) != (hi == FG_PERIODIC))
                return fail(FG_ERR_INVALID, "periodic faces must come in pairs");
            if (lo != FG_PERIODIC && n[a] < 3) return fail(FG_ERR_INVALID, "open axis needs >= 3 cells");
        }
        if (!(E.tau > 0.5) || !std::isfinite(E.tau)) return fail(FG_ERR_INVALID, "tau must exceed 1/2");
        if (!(E.rho0 > 0.0)) return fail(FG_ERR_INVALID, "rho0 must be positive");
        unsigned long long ns = (unsigned long long)((E.nx + 7) / 8 * 8) * E.ny * E.nz;
        if (ns >= (1ull << 31)) return fail(FG_ERR_INVALID, "too many cells in one environment");
        cells += ns;
    }
    fg_domain* d = new (std::nothrow) fg_domain();
    if (!d) return fail(FG_ERR_OOM, "host allocation");
    d->n_envs = n_envs;
    d->opt = o;
    d->stream = (cudaStream_t)cuda_stream;
    d->esize = o.storage == FG_F32 ? 4 : 2;
    d->aa = o.layout == FG_LAYOUT_AA;
    {
        int dev = 0;
        cudaError_t ce = cudaGetDevice(&dev);
        if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&d->n_sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce != cudaSuccess) {
            delete d;
            return cuda_fail(ce, "cudaDeviceGetAttribute");
        }
    }
    d->desc.assign(envs, envs + n_envs);
    d->user_frame.resize(n_envs);
    d->box_acc.assign(n_envs, {0.0, 0.0, 0.0});
    d->env.resize(n_envs);
    d->frame.resize(n_envs);
    d->mk.resize(n_envs);
    unsigned long long slot_off = 0, stamp_off = 0, ncell_all = 0;
    int block0 = 0;
    bool can_stage = true;
    for (int e = 0; e < n_envs; ++e) d->max_P = std::max(d->max_P, (envs[e].nx + 7) / 8 * 8);
    for (int e = 0; e < n_envs; ++e) {
        const fg_env_desc& s = envs[e];
        EnvDev& E = d->env[e];
        std::memset(&E, 0, sizeof(E));
        E.n[0] = s.nx; E.n[1] = s.ny; E.n[2] = s.nz;
        E.P = (s.nx + 7) / 8 * 8;
        E.nslot = (uint32_t)((unsigned long long)E.P * s.ny * s.nz);
        E.rows = (uint32_t)s.ny * (uint32_t)s.nz;
        E.div_P = make_fastdiv((uint32_t)E.P);
        E.div_ny = make_fastdiv((uint32_t)s.ny);
        for (int k = 0; k < 6; ++k) E.bc[k] = s.face[k];
        for (int a = 0; a < 3; ++a) E.per[a] = s.face[2 * a] == FG_PERIODIC;
        E.keep = (float)(1.0 - 1.0 / s.tau);
        E.guo = (float)(1.0 - 0.5 / s.tau);
        for (int a = 0; a < 3; ++a) E.u_in[a] = (float)s.u_in[a];
        E.drho_out = (float)(s.rho0 - 1.0);
        E.pop_off = 27ull * slot_off;
        E.slot_off = slot_off;
        E.block0 = block0;
        E.nblocks = (int)((E.nslot + K1_THREADS - 1) / K1_THREADS);
        E.stamp_off = (int)stamp_off;
        E.nseg = 1;
        if (E.P > MAX_STAGED_P) can_stage = false;
        slot_off += E.nslot;
        ncell_all += (unsigned long long)s.nx * s.ny * s.nz;
        stamp_off += (E.nslot + 31) / 32;
        block0 += E.nblocks;
        fg_frame fr{};
        fr.origin[0] = (s.nx - 1) * 0.5; fr.origin[1] = (s.ny - 1) * 0.5; fr.origin[2] = (s.nz - 1) * 0.5;
        d->user_frame[e] = fr;
        set_frame(d->frame[e], fr);
    }
    if ((o.kernel_variant == FG_KERNEL_STAGED || o.kernel_variant == FG_KERNEL_STAGED512) && !can_stage) {
        delete d;
        return fail(FG_ERR_INVALID, "staged kernel needs rows of at most 512 cells");
    }
    d->total_cells = ncell_all;
    d->total_slots = slot_off;
    d->pop_elems = 27ull * slot_off;
    d->n_stamps = stamp_off;
    d->total_blocks = block0;
    fg_status st = FG_OK;
#define DA(ptr, n)                                   \
    if ((st = dalloc(&(ptr), (n))) != FG_OK) {       \
        free_all(d);                                 \
        delete d;                                    \
        return st;                                   \
    }
    DA(d->d_env, n_envs);
    DA(d->d_frame, n_envs + 1);   // room for the marker source after the frames (msrc_offset)
    d->d_msrc = reinterpret_cast<MarkerSrc*>(reinterpret_cast<unsigned char*>(d->d_frame) + msrc_offset(n_envs));
    {
        char *p0 = nullptr, *p1 = nullptr;
        DA(p0, d->pop_elems * d->esize);
        d->pop[0] = p0;
        if (d->aa) {
            d->pop[1] = p0;   // one buffer, updated in place
        } else {
            DA(p1, d->pop_elems * d->esize);
            d->pop[1] = p1;
        }
    }
    DA(d->fib, slot_off);
    DA(d->stamps, stamp_off);
    DA(d->ib_nodes, slot_off);
    DA(d->ib_bar, 2);
    DA(d->seg_ref, (size_t)n_envs * MAX_SEG * 3);
    if (o.deterministic) DA(d->fibq, 3ull * slot_off);
    DA(d->red_counters, (size_t)n_envs * RED_ROWS);
    DA(d->d_state, 1);
    DA(d->ft, (size_t)n_envs * FT_ROW);   // compensated pairs, evaluated on the host
    DA(d->mass, n_envs);
    if (o.record_history > 0) DA(d->hist, (size_t)n_envs * o.record_history * HIST_ROW);
    DA(d->status, 1);
    DA(d->work, WQ_WORDS);
    DA(d->work_done, (size_t)n_envs * N_SLOTS);
    d->blk_flag_n = (size_t)block0;   // one-cell blocks: the most any layout has
    DA(d->blk_flag, d->blk_flag_n);
#undef DA
    {
        cudaError_t e = cudaHostAlloc((void**)&d->rb, sizeof(*d->rb), cudaHostAllocMapped);
        if (e != cudaSuccess) d->rb = nullptr;
        if (e == cudaSuccess) {
            e = cudaHostAlloc((void**)&d->rb_ft_all, sizeof(Pair32) * n_envs * FT_ROW, cudaHostAllocMapped);
            if (e != cudaSuccess) d->rb_ft_all = nullptr;
        }
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&d->rb_ft_all_dev, d->rb_ft_all, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&d->rb_status_dev, &d->rb->status, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&d->rb_seq_dev, &d->rb->seq, 0);
        if (e == cudaSuccess) d->rb->seq = -1;
        if (e != cudaSuccess) {
            free_all(d);
            delete d;
            return cuda_fail(e, "cudaHostAlloc");
        }
    }
    {
        // the second stream of the IB beside the stream-collide kernel
        int lo = 0, hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&d->stream2, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            free_all(d);
            delete d;
            return cuda_fail(e, "stream or event creation");
        }
        d->prio_high = hi;
    }
    cudaError_t ce;
    StepState initial_state;
    initial_state.stamp = 1;
    initial_state.envs_done = 0;
    initial_state.step = 0;
    if ((ce = cudaMemsetAsync(d->pop[0], 0, d->pop_elems * d->esize, d->stream)) != cudaSuccess ||
        (d->pop[1] != d->pop[0] &&
         (ce = cudaMemsetAsync(d->pop[1], 0, d->pop_elems * d->esize, d->stream)) != cudaSuccess) ||
        (ce = cudaMemsetAsync(d->fib, 0, sizeof(float4) * slot_off, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->stamps, 0, sizeof(uint32_t) * stamp_off, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->ft, 0, sizeof(Pair32) * n_envs * FT_ROW, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->mass, 0, sizeof(Pair32) * n_envs, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->status, 0, sizeof(int), d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->ib_bar, 0, 2 * sizeof(unsigned), d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->d_msrc, 0, sizeof(MarkerSrc), d->stream)) != cudaSuccess ||
        (d->fibq && (ce = cudaMemsetAsync(d->fibq, 0, sizeof(unsigned long long) * 3ull * slot_off,
                                          d->stream)) != cudaSuccess) ||
        (ce = cudaMemsetAsync(d->red_counters, 0, sizeof(int) * n_envs * RED_ROWS, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->work, 0, sizeof(int) * WQ_WORDS, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->blk_flag, 0, sizeof(uint32_t) * d->blk_flag_n, d->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(d->work_done, 0, sizeof(int) * n_envs * N_SLOTS, d->stream)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(d->d_state, &initial_state, sizeof(StepState), cudaMemcpyHostToDevice,
                              d->stream)) != cudaSuccess) {
        st = cuda_fail(ce, "cudaMemsetAsync");
        free_all(d);
        delete d;
        return st;
    }
    refresh_marker_table(d);
    {
        const int first = d->aa                                                  ? K1_PLAIN
                          : o.kernel_variant == FG_KERNEL_OVERLAP                  ? K1_OVERLAP
                          : o.kernel_variant == FG_KERNEL_FUSED                    ? K1_FUSED
                          : o.kernel_variant == FG_KERNEL_PLAIN || !can_stage ? K1_PLAIN
                          : o.kernel_variant == FG_KERNEL_STAGED512              ? K1_STAGED512
                          : (d->max_P <= 256 ? K1_STAGED256 : K1_STAGED512);
        if ((st = configure_k1(d, first, true)) != FG_OK) {
            free_all(d);
            delete d;
            return st;
        }
        // resident blocks per SM of the cooperative IB kernel
        st = dispatch(o.storage, [&](auto tag) -> fg_status {
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d->ib_per_sm, k_ib_step<decltype(tag)>, IB_THREADS,
                                                             ib_smem_bytes(n_envs)));
            return d->ib_per_sm > 0 ? FG_OK : fail(FG_ERR_CUDA, "k_ib_step cannot be resident");
        });
        if (st != FG_OK) {
            free_all(d);
            delete d;
            return st;
        }
    }
    if ((st = upload_env(d)) != FG_OK || (st = upload_frames(d)) != FG_OK || (st = upload_seg_refs(d)) != FG_OK) {
        free_all(d);
        delete d;
        return st;
    }
    for (int e = 0; e < n_envs && st == FG_OK; ++e) st = fg_init_fields(d, e, nullptr, nullptr);
    // the autotuner runs before the first step, when the step's markers are known
    d->autotune_pending = o.autotune && o.kernel_variant == FG_KERNEL_AUTO && !d->aa;
    if (st != FG_OK) {
        free_all(d);
        delete d;
        return st;
    }
    *out = d;
    return FG_OK;
}

void fg_destroy(fg_domain* d) {
    if (!d) return;
    cudaStreamSynchronize(d->stream);
    free_all(d);
    delete d;
}

fg_status fg_init_fields(fg_domain* d, int env, const double* rho, const double* u) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    const size_t ncell = env_cells(d, env);
    double *drho = nullptr, *du = nullptr;
    if (rho) {
        if ((st = dalloc(&drho, ncell)) != FG_OK) return st;
        CK(cudaMemcpyAsync(drho, rho, sizeof(double) * ncell, cudaMemcpyHostToDevice, d->stream));
    }
    if (u) {
        if ((st = dalloc(&du, 3ull * ncell)) != FG_OK) { if (drho) cudaFree(drho); return st; }
        CK(cudaMemcpyAsync(du, u, sizeof(double) * 3 * ncell, cudaMemcpyHostToDevice, d->stream));
    }
    const fg_env_desc& s = d->desc[env];
    const int blocks = (int)((ncell + 255) / 256);
    st = dispatch(d->opt.storage, [&](auto tag) -> fg_status {
        typedef decltype(tag) S;
        k_init_eq<S><<<blocks, 256, 0, d->stream>>>((typename S::raw*)d->pop[d->cur], d->d_env, env, drho, du,
                                                    s.rho0, s.u0[0], s.u0[1], s.u0[2], d->opt.eq_order == 3 ? 1 : 0,
                                                    aa_of(d));
        return FG_OK;
    });
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(d->stream);
    if (drho) cudaFree(drho);
    if (du) cudaFree(du);
    if (e1 != cudaSuccess) return cuda_fail(e1, "k_init_eq");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
    if (st != FG_OK) return st;
    d->poisoned = false;
    d->steps = 0;
    const long long zero_step = 0;
    CK(cudaMemcpyAsync(&d->d_state->step, &zero_step, sizeof(long long), cudaMemcpyHostToDevice, d->stream));
    CK(cudaMemsetAsync(d->status, 0, sizeof(int), d->stream));
    // after a timeout the barrier words and the work queue are inconsistent
    CK(cudaMemsetAsync(d->ib_bar, 0, 2 * sizeof(unsigned), d->stream));
    CK(cudaMemsetAsync(d->work, 0, sizeof(int) * WQ_ITEMS, d->stream));
    CK(cudaMemsetAsync(d->work_done, 0, sizeof(int) * d->n_envs * N_SLOTS, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

// The device address of a host pointer into pinned (page-locked, mapped)
// memory, nullptr for pageable memory.  Kernels read such arrays directly,
// which costs one launch instead of one copy call per array.
static const float* mapped_device_ptr(const float* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // not a CUDA pointer: clear the error
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<const float*>(a.devicePointer) : nullptr;
}

// Host checks of marker positions and velocities: |x| <= 1e6 and finite,
// 2 <= x < n - 3 along non-periodic axes, finite velocities.  The bulk check
// has no early exit so that it vectorises (it runs every step for host
// arrays); the slow pass names the first problem only when one exists.
static bool markers_valid(const EnvDev& E, int n, const float* X, const float* U) {
    // closed bounds per axis: [-1e6, 1e6] on a periodic axis, [2, n - 3) on
    // an open one (the largest float below n - 3 as the closed upper bound)
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = E.per[a] ? -1.0e6f : 2.0f;
        hi[a] = E.per[a] ? 1.0e6f : std::nextafter((float)E.n[a] - 3.0f, -INFINITY);
    }
    // NaN fails every comparison, +-inf fails the bounds; no early exit and
    // no data-dependent branch, so the loops vectorise (37 -> 5 us for 6000
    // markers on a 2.7 GHz Xeon core)
    int bad = 0;
    for (int k = 0; k + 3 <= 3 * n; k += 3) {
        bad |= (int)!(X[k] >= lo[0]) | (int)!(X[k] <= hi[0]);
        bad |= (int)!(X[k + 1] >= lo[1]) | (int)!(X[k + 1] <= hi[1]);
        bad |= (int)!(X[k + 2] >= lo[2]) | (int)!(X[k + 2] <= hi[2]);
    }
    for (int k = 0; k < 3 * n; ++k) bad |= (int)!(U[k] - U[k] == 0.0f);
    return bad == 0;
}

static const char* first_marker_problem(const EnvDev& E, int n, const float* X, const float* U) {
    for (int l = 0; l < n; ++l)
        for (int a = 0; a < 3; ++a) {
            const float x = X[3 * l + a];
            if (!std::isfinite(x) || std::fabs(x) > 1.0e6f) return "marker position not finite";
            if (!E.per[a] && !(x >= 2.0f && x < (float)E.n[a] - 3.0f))
                return "marker within 2 cells of a non-periodic face";
            if (!std::isfinite(U[3 * l + a])) return "marker velocity not finite";
        }
    return "invalid marker";
}

}  // extern "C"

namespace {

fg_status set_markers_impl(fg_domain* d, int env, int n, const float* X, const float* U, const float* dV,
                           const int* seg, int n_seg, const double ref[3], int device_ptrs) {
    fg_status st = FG_OK;
    if (n < 0) return fail(FG_ERR_INVALID, "negative marker count");
    if (n > 0 && (!X || !U)) return fail(FG_ERR_INVALID, "X and U are required");
    if (n_seg < 1 || n_seg > MAX_SEG) return fail(FG_ERR_INVALID, "n_seg must be in [1, 16]");
    MarkerRegion& r = d->mk[env];
    if (n > 0 && !dV && !(r.has_dv && r.n == n))
        return fail(FG_ERR_INVALID, "dV is required when the marker count changes");
    if (!device_ptrs && n > 0) {
        if (!markers_valid(d->env[env], n, X, U))
            return fail(FG_ERR_INVALID, first_marker_problem(d->env[env], n, X, U));
        for (int l = 0; l < n; ++l) {
            if (dV && !std::isfinite(dV[l])) return fail(FG_ERR_INVALID, "marker weight not finite");
            if (seg && (seg[l] < 0 || seg[l] >= n_seg)) return fail(FG_ERR_INVALID, "segment id out of range");
        }
    }
    if (n > r.cap) {
        if ((st = grow_markers(d, env, n)) != FG_OK) return st;
    }
    MarkerRegion& m = d->mk[env];
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n > 0) {
        // pinned host arrays are read by the copy kernel in place
        const float* Xm = device_ptrs ? X : mapped_device_ptr(X);
        const float* Um = device_ptrs ? U : (Xm ? mapped_device_ptr(U) : nullptr);
        if (Xm && Um) {
            // one launch for both arrays (the per-step marker update)
            const int blocks = (int)std::min<long long>((6ll * n + 255) / 256, 4096);
            k_copy_markers<<<blocks, 256, 0, d->stream>>>(d->X + 3ull * m.off, d->U + 3ull * m.off, Xm, Um,
                                                          3 * n);
            CK(cudaGetLastError());
        } else {
            CK(cudaMemcpyAsync(d->X + 3ull * m.off, X, sizeof(float) * 3 * n, kind, d->stream));
            CK(cudaMemcpyAsync(d->U + 3ull * m.off, U, sizeof(float) * 3 * n, kind, d->stream));
        }
        if (dV) CK(cudaMemcpyAsync(d->dV + m.off, dV, sizeof(float) * n, kind, d->stream));
        if (seg) {
            CK(cudaMemcpyAsync(d->seg + m.off, seg, sizeof(int) * n, kind, d->stream));
        } else if (m.n != n || n_seg != m.nseg) {
            CK(cudaMemsetAsync(d->seg + m.off, 0, sizeof(int) * n, d->stream));
        }
    }
    const bool table_changed = m.n != n || m.nseg != n_seg ||
                               (ref && (ref[0] != m.ref[0] || ref[1] != m.ref[1] || ref[2] != m.ref[2])) ||
                               (!ref && (m.ref[0] != 0 || m.ref[1] != 0 || m.ref[2] != 0));
    if (m.n != n) m.has_normals = false;
    if (m.nseg != n_seg) m.has_seg_ref = false;
    m.n = n;
    m.nseg = n_seg;
    if (dV) m.has_dv = true;
    for (int a = 0; a < 3; ++a) m.ref[a] = ref ? ref[a] : 0.0;
    if (table_changed) {
        refresh_marker_table(d);
        if ((st = upload_env(d)) != FG_OK) return st;
        if ((st = upload_seg_refs(d)) != FG_OK) return st;
    }
    return FG_OK;
}

}  // namespace

extern "C" {

fg_status fg_set_markers(fg_domain* d, int env, int n, const float* X, const float* U, const float* dV,
                         const int* seg, int n_seg, const double ref[3], int device_ptrs) {
    NvtxRange nvtx_range("fg_set_markers");
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (has_sphere(d, env)) return fail(FG_ERR_STATE, "the markers follow an attached sphere (fg_detach_sphere)");
    return set_markers_impl(d, env, n, X, U, dV, seg, n_seg, ref, device_ptrs);
}

fg_status fg_region_momentum(fg_domain* d, int env, const double* center, double radius, double* out,
                             double* alpha_sum) {
    NvtxRange nvtx_range("fg_region_momentum");
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!center || !out) return fail(FG_ERR_INVALID, "null argument");
    if (!(radius > 0.0) || !std::isfinite(radius)) return fail(FG_ERR_INVALID, "radius must be positive");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(center[a]) || std::fabs(center[a]) > 1e6) return fail(FG_ERR_INVALID, "centre not finite");
    const EnvDev& E = d->env[env];
    int lo[3], ext[3];
    const double cc[3] = {center[0], center[1], center[2]};
    sphere_box(E, cc, radius, lo, ext);
    const long long n_box = (long long)ext[0] * ext[1] * ext[2];
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n_box + RED_THREADS - 1) / RED_THREADS,
                                                                       4ll * d->n_sms));
    if (d->region_cap < blocks) {
        if (d->region_part) cudaFree(d->region_part);
        d->region_part = nullptr;
        if ((st = dalloc(&d->region_part, (size_t)blocks * 7)) != FG_OK) return st;
        d->region_cap = blocks;
    }
    st = dispatch(d->opt.storage, [&](auto tag) -> fg_status {
        typedef decltype(tag) S;
        k_region_momentum<S><<<blocks, RED_THREADS, 0, d->stream>>>(
            (const typename S::raw*)d->pop[d->cur], d->d_env, env, (float)center[0], (float)center[1],
            (float)center[2], (float)radius, lo[0], lo[1], lo[2], ext[0], ext[1], ext[2], d->region_part,
            aa_of(d));
        CK(cudaGetLastError());
        return FG_OK;
    });
    if (st != FG_OK) return st;
    std::vector<Pair32> h((size_t)blocks * 7);
    CK(cudaMemcpyAsync(h.data(), d->region_part, sizeof(Pair32) * h.size(), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < blocks; ++b)
        for (int q = 0; q < 7; ++q) acc[q] += pair_value(h[(size_t)b * 7 + q]);
    for (int q = 0; q < 6; ++q) out[q] = acc[q];
    if (alpha_sum) *alpha_sum = acc[6];
    return FG_OK;
}

fg_status fg_set_segment_refs(fg_domain* d, int env, int n_seg, const double* refs) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (has_sphere(d, env)) return fail(FG_ERR_STATE, "torques of an attached sphere are about its centre");
    MarkerRegion& m = d->mk[env];
    if (!refs) {
        m.has_seg_ref = false;
        return upload_seg_refs(d);
    }
    if (n_seg != m.nseg) return fail(FG_ERR_INVALID, "one reference point per segment of the last fg_set_markers");
    for (int k = 0; k < 3 * n_seg; ++k)
        if (!std::isfinite(refs[k])) return fail(FG_ERR_INVALID, "reference point not finite");
    for (int sg = 0; sg < n_seg; ++sg)
        for (int a = 0; a < 3; ++a) m.seg_ref[sg][a] = refs[3 * sg + a];
    m.has_seg_ref = true;
    return upload_seg_refs(d);
}

fg_status fg_debug_flags(unsigned int* flags, int reset) {
    if (!flags) return fail(FG_ERR_INVALID, "null flags");
#ifdef FG_DEBUG_BOUNDS
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpyFromSymbol(flags, fl::g_debug_flags, sizeof(unsigned int)));
    if (reset) {
        const unsigned int zero = 0;
        CK(cudaMemcpyToSymbol(fl::g_debug_flags, &zero, sizeof(unsigned int)));
    }
    return FG_OK;
#else
    (void)reset;
    *flags = 0;
    return fail(FG_ERR_STATE, "not a debug build (compile with -DFG_DEBUG_BOUNDS)");
#endif
}

fg_status fg_selftest_waits(unsigned int limit, int* result) {
    if (!result) return fail(FG_ERR_INVALID, "null result");
    if (limit == 0) return fail(FG_ERR_INVALID, "limit must be positive");
    unsigned* bar = nullptr;
    int *out = nullptr, *status = nullptr, *queue = nullptr;
    fg_status st = dalloc(&bar, 1);
    if (st == FG_OK) st = dalloc(&out, 4);
    if (st == FG_OK) st = dalloc(&status, 1);
    if (st == FG_OK) st = dalloc(&queue, 1 + WQ_WORDS);   // a dependency counter and the queue words
    cudaError_t e = cudaSuccess;
    if (st == FG_OK) {
        e = cudaMemset(bar, 0, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(out, 0, 4 * sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(queue, 0, (1 + WQ_WORDS) * sizeof(int));
        if (e == cudaSuccess) {
            k_selftest_waits<<<1, 64>>>(bar, limit, out, status);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_selftest_queue_wait<<<1, 32>>>(queue, queue + 1, limit, out + 2, status);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        int h[5] = {0, 0, 0, 0, 0};
        if (e == cudaSuccess) e = cudaMemcpy(h, out, 4 * sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(h + 4, status, sizeof(int), cudaMemcpyDeviceToHost);
        result[0] = h[0];
        result[1] = h[1];
        result[2] = (h[4] & ST_TIMEOUT) ? 1 : 0;
        result[3] = h[2] && h[3];
        if (e != cudaSuccess) st = cuda_fail(e, "k_selftest_waits");
    }
    if (bar) cudaFree(bar);
    if (out) cudaFree(out);
    if (status) cudaFree(status);
    if (queue) cudaFree(queue);
    return st;
}

fg_status fg_set_markers_all(fg_domain* d, int n, const float* X, const float* U, int device_ptrs) {
    NvtxRange nvtx_range("fg_set_markers_all");
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (n != d->total_markers) return fail(FG_ERR_INVALID, "n must equal the markers of all environments");
    if (!d->sph_host.empty()) return fail(FG_ERR_STATE, "markers follow an attached sphere (fg_detach_sphere)");
    if (n == 0) return FG_OK;
    if (!X || !U) return fail(FG_ERR_INVALID, "null marker array");
    const float* xs = X;
    const float* us = U;
    bool stage = false;   // pageable host arrays: copied to device scratch first
    if (!device_ptrs) {
        size_t k = 0;
        for (int e = 0; e < d->n_envs; ++e) {   // the checks of fg_set_markers, environment by environment
            const int m = d->mk[e].n;
            if (!markers_valid(d->env[e], m, X + 3 * k, U + 3 * k))
                return fail(FG_ERR_INVALID, first_marker_problem(d->env[e], m, X + 3 * k, U + 3 * k));
            k += m;
        }
        const float* Xm = mapped_device_ptr(X);
        const float* Um = Xm ? mapped_device_ptr(U) : nullptr;
        if (Xm && Um) {
            // pinned host arrays: the kernels below read them in place
            xs = Xm;
            us = Um;
        } else if (d->n_envs == 1) {   // already in the compact order: copy in place
            CK(cudaMemcpyAsync(d->X + 3ull * d->mk[0].off, X, sizeof(float) * 3 * n, cudaMemcpyHostToDevice,
                               d->stream));
            CK(cudaMemcpyAsync(d->U + 3ull * d->mk[0].off, U, sizeof(float) * 3 * n, cudaMemcpyHostToDevice,
                               d->stream));
            return FG_OK;
        } else {
            stage = true;
        }
    }
    if (stage) {
        const size_t need = 6ull * n;
        if (d->mk_stage_cap < need) {
            if (d->mk_stage) cudaFree(d->mk_stage);
            d->mk_stage = nullptr;
            d->mk_stage_cap = 0;
            fg_status st = dalloc(&d->mk_stage, need);
            if (st != FG_OK) return st;
            d->mk_stage_cap = need;
        }
        CK(cudaMemcpyAsync(d->mk_stage, X, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, d->stream));
        CK(cudaMemcpyAsync(d->mk_stage + 3ull * n, U, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, d->stream));
        xs = d->mk_stage;
        us = d->mk_stage + 3ull * n;
    }
    const int blocks = std::min((n + 255) / 256, 8 * d->n_sms);
    k_scatter_markers<<<blocks, 256, 0, d->stream>>>(d->d_env, d->n_envs, n, xs, us, d->X, d->U);
    CK(cudaGetLastError());
    return FG_OK;
}

fg_status fg_set_marker_normals(fg_domain* d, int env, int n, const float* N, int device_ptrs) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    MarkerRegion& m = d->mk[env];
    if (n != m.n) return fail(FG_ERR_INVALID, "normals count differs from the marker count");
    if (n > 0 && !N) return fail(FG_ERR_INVALID, "null normals");
    if (!device_ptrs) {
        for (int k = 0; k < 3 * n; ++k)
            if (!std::isfinite(N[k])) return fail(FG_ERR_INVALID, "normal not finite");
    }
    if (n > 0)
        CK(cudaMemcpyAsync(d->Nrm + 3ull * m.off, N, sizeof(float) * 3 * n,
                           device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, d->stream));
    m.has_normals = true;
    return FG_OK;
}

// Called after every launch sequence that advances the device stamp.  When
// the stamp wraps to 1, tiles may still carry 1 from long ago, and k_ib_step
// would take them as stamped this step, so all stamps are cleared then.
static fg_status note_stamp_advance(fg_domain* d) {
    d->stamp_host = d->stamp_host == 0xffffffffu ? 1u : d->stamp_host + 1u;
    if (d->stamp_host == 1u) {
        CK(cudaMemsetAsync(d->stamps, 0, sizeof(uint32_t) * d->n_stamps, d->stream));
        CK(cudaMemsetAsync(d->blk_flag, 0, sizeof(uint32_t) * d->blk_flag_n, d->stream));
    }
    return FG_OK;
}

fg_status fg_step(fg_domain* d, int n_steps, const fg_frame* frames) {
    NvtxRange nvtx_range("fg_step");
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (n_steps < 0) return fail(FG_ERR_INVALID, "negative step count");
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    if (frames) {
        for (int e = 0; e < d->n_envs; ++e) {
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(frames[e].acc[a]) || !std::isfinite(frames[e].omega[a]) ||
                    !std::isfinite(frames[e].domega[a]) || !std::isfinite(frames[e].origin[a]))
                    return fail(FG_ERR_INVALID, "frame not finite");
        }
        for (int e = 0; e < d->n_envs; ++e) set_env_frame(d, e, frames[e]);
        fg_status st = upload_frames(d);   // with a posted marker source, in the same copy
        if (st != FG_OK) return st;
    } else if (fg_status st = upload_msrc(d); st != FG_OK) {
        return st;
    }
    if (d->opt.ib_slip)
        for (int e = 0; e < d->n_envs; ++e)
            if (d->mk[e].n > 0 && !d->mk[e].has_normals)
                return fail(FG_ERR_STATE, "slip forcing needs the markers' normals (fg_set_marker_normals)");
    if (n_steps > 0 && d->autotune_pending) {
        fg_status st = fg_autotune(d, nullptr, nullptr);
        if (st != FG_OK) return st;
    }
    if (fg_status st = sync_work_table(d); st != FG_OK) return st;
    for (const SphereDev& sp : d->sph_host)
        if (sp.mk_off != d->mk[sp.env].off) {   // the marker layout moved: the table follows it
            fg_status st = sphere_download(d);
            if (st == FG_OK) st = sphere_upload(d);
            if (st != FG_OK) return st;
            break;
        }
    const bool graphs = d->opt.use_graphs && !d->profiling;
    for (int s = 0; s < n_steps; ++s) {
        fg_status st = dispatch(d->opt.storage, [&](auto tag) {
            return graphs ? graph_step<decltype(tag)>(d) : launch_step<decltype(tag)>(d);
        });
        if (st != FG_OK) return st;
        if ((st = note_stamp_advance(d)) != FG_OK) return st;
    }
    return FG_OK;
}

fg_status fg_step_state(fg_domain* d, const void* in, void* out, const fg_frame* frames) {
    NvtxRange nvtx_range("fg_step_state");
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (d->n_envs != 1) return fail(FG_ERR_INVALID, "fg_step_state takes a single environment");
    if (!in || !out || in == out) return fail(FG_ERR_INVALID, "in and out must be distinct device buffers");
    if (d->aa) return fail(FG_ERR_INVALID, "fg_step_state steps the two-buffer layout only");
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    if (frames) {
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(frames[0].acc[a]) || !std::isfinite(frames[0].omega[a]) ||
                !std::isfinite(frames[0].domega[a]) || !std::isfinite(frames[0].origin[a]))
                return fail(FG_ERR_INVALID, "frame not finite");
        set_env_frame(d, 0, frames[0]);
        fg_status st = upload_frames(d);
        if (st != FG_OK) return st;
    }
    if (d->opt.ib_slip && d->mk[0].n > 0 && !d->mk[0].has_normals)
        return fail(FG_ERR_STATE, "slip forcing needs the markers' normals (fg_set_marker_normals)");
    if (fg_status st0 = sync_work_table(d); st0 != FG_OK) return st0;
    fg_status st = dispatch(d->opt.storage, [&](auto tag) {
        typedef typename decltype(tag)::raw raw;
        return enqueue_step_io<decltype(tag)>(d, (const raw*)in, (raw*)out, d->stream, nullptr);
    });
    if (st != FG_OK) return st;
    d->steps += 1;
    return note_stamp_advance(d);
}

fg_status fg_get_status(fg_domain* d, int* status) {
    if (!d || !status) return fail(FG_ERR_INVALID, "null argument");
    CK(cudaMemcpyAsync(&d->rb->status, d->status, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    *status = d->rb->status;
    return FG_OK;
}

// Errors from the status word; `s` was read after every launch in question.
static fg_status status_to_error(fg_domain* d, int s) {
    if (s & ST_NUMERIC) {
        d->poisoned = true;
        return fail(FG_ERR_NUMERIC, "NaN or Inf in the force or mass reduction");
    }
    if (s & ST_BAD_MARKER) {
        CK(cudaMemsetAsync(d->status, 0, sizeof(int), d->stream));
        CK(cudaStreamSynchronize(d->stream));
        return fail(FG_ERR_INVALID, "a marker was outside the domain or within 2 cells of a non-periodic face");
    }
    if (s & ST_MASS_DRIFT) {
        d->poisoned = true;
        return fail(FG_ERR_NUMERIC, "mass drift beyond the fg_watch_mass tolerance");
    }
    if (s & ST_TIMEOUT) {
        d->poisoned = true;
        return fail(FG_ERR_TIMEOUT, "a bounded device wait gave up; call fg_init_fields");
    }
    return FG_OK;
}

// The markers of every environment for the next step, in the compact order
// of fg_set_markers_all.  Where that step's IB kernel is k_ib_step (every
// variant but the fused and overlap ones), the arrays are device arrays or
// pinned host arrays read once (each marker the first of its half-warp),
// and no sphere is attached, the arrays are posted to the step (MarkerSrc):
// its IB kernel reads them and fills the domain's marker arrays on the way,
// with no copy launch before the step.  Otherwise fg_set_markers_all copies
// them now.  The caller keeps the arrays unchanged until the step has run.
static fg_status step_markers_in(fg_domain* d, const float* X, const float* U, int device_ptrs) {
    if (d->autotune_pending) {   // the variant is settled before the markers are posted
        fg_status st = fg_autotune(d, nullptr, nullptr);
        if (st != FG_OK) return st;
    }
    const int n = d->total_markers;
    const int ib_warps = d->ib_per_sm * d->n_sms * (IB_THREADS / 32);
    bool post = n > 0 && X && U && d->sph_host.empty() && d->k1 != K1_FUSED && d->k1 != K1_OVERLAP;
    const float* xs = X;
    const float* us = U;
    if (post && !device_ptrs) {
        xs = mapped_device_ptr(X);
        us = xs ? mapped_device_ptr(U) : nullptr;
        post = xs && us && n <= 2 * ib_warps;
        if (post) {   // the checks fg_set_markers_all makes of host arrays
            size_t k = 0;
            for (int e = 0; e < d->n_envs; ++e) {
                const int m = d->mk[e].n;
                if (!markers_valid(d->env[e], m, X + 3 * k, U + 3 * k))
                    return fail(FG_ERR_INVALID, first_marker_problem(d->env[e], m, X + 3 * k, U + 3 * k));
                k += m;
            }
        }
    }
    if (!post) return fg_set_markers_all(d, n, X, U, device_ptrs);
    d->msrc_next.X = xs;
    d->msrc_next.U = us;
    d->msrc_next.valid = 1;
    return FG_OK;
}

// One step after step_markers_in.  A posted source is uploaded by the step
// and cleared on the device by its reduction; if the step fails after the
// upload but before its launches, the device copy is cleared here, so that
// no later step reads the caller's arrays.
static fg_status step_posted(fg_domain* d, const fg_frame* frames) {
    const bool posted = d->msrc_next.valid != 0;
    const long long steps_before = d->steps;
    const fg_status st = fg_step(d, 1, frames);
    d->msrc_next.valid = 0;
    if (posted && d->steps == steps_before)   // nothing launched: no reduction clears it
        cudaMemsetAsync(&d->d_msrc->valid, 0, sizeof(int), d->stream);
    return st;
}

fg_status fg_step_markers(fg_domain* d, const float* X, const float* U, int device_ptrs, const fg_frame* frames) {
    NvtxRange nvtx_range("fg_step_markers");
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if ((X == nullptr) != (U == nullptr)) return fail(FG_ERR_INVALID, "X and U must both be given or both NULL");
    // fg_step's own checks first, so that a failing step posts and copies nothing
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    if (frames)
        for (int e = 0; e < d->n_envs; ++e)
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(frames[e].acc[a]) || !std::isfinite(frames[e].omega[a]) ||
                    !std::isfinite(frames[e].domega[a]) || !std::isfinite(frames[e].origin[a]))
                    return fail(FG_ERR_INVALID, "frame not finite");
    if (d->opt.ib_slip)
        for (int e = 0; e < d->n_envs; ++e)
            if (d->mk[e].n > 0 && !d->mk[e].has_normals)
                return fail(FG_ERR_STATE, "slip forcing needs the markers' normals (fg_set_marker_normals)");
    fg_status st = FG_OK;
    if (X && (st = step_markers_in(d, X, U, device_ptrs)) != FG_OK) return st;
    return step_posted(d, frames);
}

fg_status fg_step_io(fg_domain* d, const float* X, const float* U, int device_ptrs, const fg_frame* frames,
                     double* out) {
    NvtxRange nvtx_range("fg_step_io");
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (!out) return fail(FG_ERR_INVALID, "null output");
    if ((X == nullptr) != (U == nullptr)) return fail(FG_ERR_INVALID, "X and U must both be given or both NULL");
    // fg_step's own checks first, so that a failing step launches no marker copy
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    if (frames)
        for (int e = 0; e < d->n_envs; ++e)
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(frames[e].acc[a]) || !std::isfinite(frames[e].omega[a]) ||
                    !std::isfinite(frames[e].domega[a]) || !std::isfinite(frames[e].origin[a]))
                    return fail(FG_ERR_INVALID, "frame not finite");
    if (d->opt.ib_slip)
        for (int e = 0; e < d->n_envs; ++e)
            if (d->mk[e].n > 0 && !d->mk[e].has_normals)
                return fail(FG_ERR_STATE, "slip forcing needs the markers' normals (fg_set_marker_normals)");
    fg_status st = FG_OK;
    if (X && (st = step_markers_in(d, X, U, device_ptrs)) != FG_OK) return st;
    if ((st = step_posted(d, frames)) != FG_OK) return st;
    // The step's k_reduce writes the rows, the status word and then the step
    // number to mapped pinned memory: no copy to issue.  The host polls the
    // step number (waking from a stream synchronisation takes longer than the
    // step on a busy host) for at most 20 ms, then synchronises the stream.
    {
        const long long want = d->steps;
        volatile const long long* seq = &d->rb->seq;
        const auto t0 = std::chrono::steady_clock::now();
        bool seen = false;
        for (unsigned i = 0;; ++i) {
            if (*seq == want) {
                seen = true;
                break;
            }
            if ((i & 1023u) == 1023u && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(20)) break;
        }
        std::atomic_thread_fence(std::memory_order_acquire);
        if (!seen) CK(cudaStreamSynchronize(d->stream));
        // a launch or execution error of the step, if any, surfaces here
        const cudaError_t q = cudaStreamQuery(d->stream);
        if (q != cudaSuccess && q != cudaErrorNotReady) return cuda_fail(q, "fg_step_io");
    }
    if ((st = status_to_error(d, d->rb->status)) != FG_OK) return st;
    size_t o = 0;
    for (int e = 0; e < d->n_envs; ++e) {
        const int vals = 6 * (d->mk[e].nseg + 1);
        for (int k = 0; k < vals; ++k) out[o++] = pair_value(d->rb_ft_all[(size_t)e * FT_ROW + k]);
    }
    return FG_OK;
}

fg_status fg_get_body_force_torque(fg_domain* d, int env, double* out) {
    NvtxRange nvtx_range("fg_get_body_force_torque");
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!out) return fail(FG_ERR_INVALID, "null output");
    const int rows = d->mk[env].nseg + 1;
    // both copies land in pinned memory: asynchronous, one synchronisation
    CK(cudaMemcpyAsync(d->rb->ft, d->ft + (size_t)env * FT_ROW, sizeof(Pair32) * 6 * rows,
                       cudaMemcpyDeviceToHost, d->stream));
    CK(cudaMemcpyAsync(&d->rb->status, d->status, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    if ((st = status_to_error(d, d->rb->status)) != FG_OK) return st;
    for (int k = 0; k < 6 * rows; ++k) out[k] = pair_value(d->rb->ft[k]);
    return FG_OK;
}

fg_status fg_get_mass(fg_domain* d, int env, double* mass) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!mass) return fail(FG_ERR_INVALID, "null output");
    CK(cudaMemcpyAsync(&d->rb->mass, d->mass + env, sizeof(Pair32), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaMemcpyAsync(&d->rb->status, d->status, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    if ((st = status_to_error(d, d->rb->status)) != FG_OK) return st;
    *mass = (double)env_cells(d, env) + pair_value(d->rb->mass);
    return FG_OK;
}

fg_status fg_set_alloc_cap(unsigned long long bytes) {
    g_alloc_cap.store(bytes, std::memory_order_relaxed);
    return FG_OK;
}

fg_status fg_watch_mass(fg_domain* d, int env, double rel_tol) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!std::isfinite(rel_tol)) return fail(FG_ERR_INVALID, "rel_tol not finite");
    EnvDev& E = d->env[env];
    if (rel_tol <= 0.0) {
        E.mass_tol = 0.0f;
        E.mass_ref = 0.0f;
        return upload_env(d);
    }
    double m = 0.0;
    if ((st = fg_get_mass(d, env, &m)) != FG_OK) return st;   // synchronises
    const double cells = (double)env_cells(d, env);
    E.mass_ref = (float)(m - cells);
    E.mass_tol = (float)(rel_tol * m);
    return upload_env(d);
}

fg_status fg_get_marker_force(fg_domain* d, int env, float* F) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    const MarkerRegion& m = d->mk[env];
    if (m.n == 0) return FG_OK;
    if (!F) return fail(FG_ERR_INVALID, "null output");
    CK(cudaMemcpyAsync(F, d->Fm + 3ull * m.off, sizeof(float) * 3 * m.n, cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

fg_status fg_get_history(fg_domain* d, int env, double* out, int max_steps, int* n_rows) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!out || !n_rows || max_steps < 0) return fail(FG_ERR_INVALID, "bad output");
    const int cap = d->opt.record_history;
    *n_rows = 0;
    if (cap == 0) return fail(FG_ERR_STATE, "history was not enabled at creation");
    const long long avail = std::min<long long>(d->steps, cap);
    const long long nr = std::min<long long>(avail, max_steps);
    std::vector<Pair32> all((size_t)cap * HIST_ROW);
    CK(cudaMemcpyAsync(all.data(), d->hist + (size_t)env * cap * HIST_ROW, sizeof(Pair32) * all.size(),
                       cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    const int w = 6 * (d->mk[env].nseg + 1);
    const double ncell = (double)env_cells(d, env);
    for (long long k = 0; k < nr; ++k) {
        const long long step = d->steps - nr + k;  // oldest first
        const Pair32* row = all.data() + (size_t)(step % cap) * HIST_ROW;
        for (int c = 0; c < w; ++c) out[k * (w + 1) + c] = pair_value(row[c]);
        out[k * (w + 1) + w] = ncell + pair_value(row[FT_ROW]);
    }
    *n_rows = (int)nr;
    return FG_OK;
}

fg_status fg_get_fields(fg_domain* d, int env, double* rho, double* u) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    const size_t ncell = env_cells(d, env);
    double *dr = nullptr, *du = nullptr;
    if ((st = dalloc(&dr, ncell)) != FG_OK) return st;
    if ((st = dalloc(&du, 3ull * ncell)) != FG_OK) { cudaFree(dr); return st; }
    const int blocks = (int)((ncell + 255) / 256);
    dispatch(d->opt.storage, [&](auto tag) -> fg_status {
        typedef decltype(tag) S;
        k_get_fields<S><<<blocks, 256, 0, d->stream>>>((const typename S::raw*)d->pop[d->cur], d->d_env, env,
                                                       dr, du, aa_of(d));
        return FG_OK;
    });
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && rho)
        e = cudaMemcpyAsync(rho, dr, sizeof(double) * ncell, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess && u)
        e = cudaMemcpyAsync(u, du, sizeof(double) * 3 * ncell, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    cudaFree(dr);
    cudaFree(du);
    if (e != cudaSuccess) return cuda_fail(e, "fg_get_fields");
    return FG_OK;
}

fg_status fg_get_populations(fg_domain* d, int env, double* f) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!f) return fail(FG_ERR_INVALID, "null output");
    const size_t ncell = env_cells(d, env);
    double* df = nullptr;
    if ((st = dalloc(&df, 27ull * ncell)) != FG_OK) return st;
    const int blocks = (int)((ncell + 255) / 256);
    dispatch(d->opt.storage, [&](auto tag) -> fg_status {
        typedef decltype(tag) S;
        k_get_pop<S><<<blocks, 256, 0, d->stream>>>((const typename S::raw*)d->pop[d->cur], d->d_env, env, df,
                                                    aa_of(d));
        return FG_OK;
    });
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, df, sizeof(double) * 27 * ncell, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    cudaFree(df);
    if (e != cudaSuccess) return cuda_fail(e, "fg_get_populations");
    return FG_OK;
}

fg_status fg_set_populations(fg_domain* d, int env, const double* f) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!f) return fail(FG_ERR_INVALID, "null input");
    const size_t ncell = env_cells(d, env);
    double* df = nullptr;
    if ((st = dalloc(&df, 27ull * ncell)) != FG_OK) return st;
    cudaError_t e = cudaMemcpyAsync(df, f, sizeof(double) * 27 * ncell, cudaMemcpyHostToDevice, d->stream);
    const int blocks = (int)((ncell + 255) / 256);
    if (e == cudaSuccess) {
        dispatch(d->opt.storage, [&](auto tag) -> fg_status {
            typedef decltype(tag) S;
            k_set_pop<S><<<blocks, 256, 0, d->stream>>>((typename S::raw*)d->pop[d->cur], d->d_env, env, df,
                                                        aa_of(d));
            return FG_OK;
        });
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    cudaFree(df);
    if (e != cudaSuccess) return cuda_fail(e, "fg_set_populations");
    return FG_OK;
}

}  // extern "C"

namespace {

// The in-place layout's state in the two-buffer format ([27][nslot] raw
// values, post-collision population i at (i, slot)): converted on the way
// out and in by k_aa_state, so that a saved state loads at either phase.
// buf is a device buffer of fg_state_bytes bytes.
fg_status aa_state_copy(fg_domain* d, int env, void* buf, bool to_buf) {
    const EnvDev& E = d->env[env];
    const int blocks = (int)((E.nslot + 255) / 256);
    return dispatch(d->opt.storage, [&](auto tag) -> fg_status {
        typedef typename decltype(tag)::raw raw;
        k_aa_state<decltype(tag)><<<blocks, 256, 0, d->stream>>>((raw*)d->pop[0], d->d_env, env, d->cur, (raw*)buf,
                                                                 to_buf ? 1 : 0);
        CK(cudaGetLastError());
        return FG_OK;
    });
}

// The same through a device staging buffer, to or from host memory.
fg_status aa_state_host(fg_domain* d, int env, void* host_buf, bool save) {
    const size_t bytes = 27ull * d->env[env].nslot * d->esize;
    char* tmp = nullptr;
    fg_status st = dalloc(&tmp, bytes);
    if (st != FG_OK) return st;
    cudaError_t e = cudaSuccess;
    if (!save) e = cudaMemcpyAsync(tmp, host_buf, bytes, cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) st = aa_state_copy(d, env, tmp, save);
    if (e == cudaSuccess && st == FG_OK && save)
        e = cudaMemcpyAsync(host_buf, tmp, bytes, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    cudaFree(tmp);
    if (st != FG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, save ? "fg_save_state" : "fg_load_state");
    return FG_OK;
}

}  // namespace

extern "C" {

fg_status fg_state_bytes(fg_domain* d, int env, unsigned long long* bytes) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!bytes) return fail(FG_ERR_INVALID, "null output");
    *bytes = 27ull * d->env[env].nslot * d->esize;
    return FG_OK;
}

fg_status fg_save_state(fg_domain* d, int env, void* host_buf) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!host_buf) return fail(FG_ERR_INVALID, "null buffer");
    if (d->aa) return aa_state_host(d, env, host_buf, true);
    const EnvDev& E = d->env[env];
    const char* src = (const char*)d->pop[d->cur] + E.pop_off * d->esize;
    CK(cudaMemcpyAsync(host_buf, src, 27ull * E.nslot * d->esize, cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

fg_status fg_load_state(fg_domain* d, int env, const void* host_buf) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!host_buf) return fail(FG_ERR_INVALID, "null buffer");
    if (d->aa) return aa_state_host(d, env, const_cast<void*>(host_buf), false);
    const EnvDev& E = d->env[env];
    char* dst = (char*)d->pop[d->cur] + E.pop_off * d->esize;
    CK(cudaMemcpyAsync(dst, host_buf, 27ull * E.nslot * d->esize, cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

fg_status fg_step_count(fg_domain* d, long long* steps) {
    if (!d || !steps) return fail(FG_ERR_INVALID, "null argument");
    *steps = d->steps;
    return FG_OK;
}

fg_status fg_profile(fg_domain* d, int enable) {
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    CK(cudaStreamSynchronize(d->stream));
    if (enable && d->ev[0].empty()) {
        for (int k = 0; k < FG_K_COUNT; ++k) {
            d->ev[k].resize(PROFILE_CAP);
            for (int i = 0; i < PROFILE_CAP; ++i) CK(cudaEventCreate(&d->ev[k][i]));
        }
    }
    d->profiling = enable != 0;
    for (int k = 0; k < FG_K_COUNT; ++k) {
        d->ev_used[k] = 0;
        d->prof_ms[k] = 0;
        d->prof_n[k] = 0;
    }
    return FG_OK;
}

fg_status fg_profile_read(fg_domain* d, double* ms, long long* launches) {
    if (!d || !ms || !launches) return fail(FG_ERR_INVALID, "null argument");
    CK(cudaStreamSynchronize(d->stream));
    for (int k = 0; k < FG_K_COUNT; ++k) {
        for (int i = 0; i + 1 < d->ev_used[k]; i += 2) {
            float t = 0;
            CK(cudaEventElapsedTime(&t, d->ev[k][i], d->ev[k][i + 1]));
            d->prof_ms[k] += t;
            d->prof_n[k] += 1;
        }
        d->ev_used[k] = 0;
        ms[k] = d->prof_ms[k];
        launches[k] = d->prof_n[k];
        d->prof_ms[k] = 0;
        d->prof_n[k] = 0;
    }
    return FG_OK;
}

static fg_status adjoint_check(fg_domain* d) {
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (d->n_envs != 1) return fail(FG_ERR_INVALID, "the adjoint takes a single environment");
    if (d->opt.storage != FG_F32) return fail(FG_ERR_INVALID, "the adjoint takes FP32 storage");
    if (d->aa) return fail(FG_ERR_INVALID, "the adjoint takes the two-buffer layout");
    if (d->opt.ib_iters != 1) return fail(FG_ERR_INVALID, "the adjoint takes one direct-forcing pass");
    if (d->opt.ib_slip) return fail(FG_ERR_INVALID, "the adjoint takes no-slip forcing");
    if (d->opt.eq_order != 2) return fail(FG_ERR_INVALID, "the adjoint takes the second-order equilibrium");
    for (int k = 0; k < 6; ++k)
        if (d->desc[0].face[k] != FG_PERIODIC) return fail(FG_ERR_INVALID, "the adjoint takes periodic domains");
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    if (!d->adj_lam[0]) {
        const size_t ns = d->total_slots;
        fg_status st;
        if ((st = dalloc(&d->adj_lam[0], 27 * ns)) != FG_OK) return st;
        if ((st = dalloc(&d->adj_lam[1], 27 * ns)) != FG_OK) return st;
        if ((st = dalloc(&d->adj_lfib, 3 * ns)) != FG_OK) return st;
        if ((st = dalloc(&d->adj_lrho, ns)) != FG_OK) return st;
        if ((st = dalloc(&d->adj_lut, 3 * ns)) != FG_OK) return st;
        if ((st = dalloc(&d->adj_gF, FT_ROW)) != FG_OK) return st;
        CK(cudaMemsetAsync(d->adj_lam[0], 0, sizeof(float) * 27 * ns, d->stream));
        CK(cudaMemsetAsync(d->adj_lam[1], 0, sizeof(float) * 27 * ns, d->stream));
        CK(cudaMemsetAsync(d->adj_lfib, 0, sizeof(float) * 3 * ns, d->stream));
        CK(cudaMemsetAsync(d->adj_lrho, 0, sizeof(float) * ns, d->stream));
        CK(cudaMemsetAsync(d->adj_lut, 0, sizeof(float) * 3 * ns, d->stream));
    }
    return FG_OK;
}

fg_status fg_adjoint_reset(fg_domain* d) {
    fg_status st = adjoint_check(d);
    if (st != FG_OK) return st;
    CK(cudaMemsetAsync(d->adj_lam[d->adj_cur], 0, sizeof(float) * 27 * d->total_slots, d->stream));
    return FG_OK;
}

static fg_status adjoint_step_from(fg_domain* d, const float* f, const fg_frame* frames, const double* gF,
                                   float* gX, float* gU) {
    fg_status st = FG_OK;
    const int n = d->mk[0].n;
    if (n > 0 && (!gX || !gU)) return fail(FG_ERR_INVALID, "gX and gU are required");
    if (frames) {
        set_env_frame(d, 0, frames[0]);
        if ((st = upload_frames(d)) != FG_OK) return st;
    }
    const int rows = d->mk[0].nseg + 1;
    std::vector<float> g(FT_ROW, 0.0f);
    if (gF)
        for (int k = 0; k < 6 * rows; ++k) g[k] = (float)gF[k];
    CK(cudaMemcpyAsync(d->adj_gF, g.data(), sizeof(float) * FT_ROW, cudaMemcpyHostToDevice, d->stream));
    const float* lam_in = d->adj_lam[d->adj_cur];
    float* lam_out = d->adj_lam[d->adj_cur ^ 1];
    const EnvDev& E = d->env[0];
    const int blocks = (int)((E.nslot + K1_THREADS - 1) / K1_THREADS);
    // the step's IB force field (forward interpolation + spreading)
    if (n > 0) {
        const int wb = IB_THREADS / 32;
        k_ib<StoreF32><<<(n + wb - 1) / wb, IB_THREADS, 0, d->stream>>>(
            f, d->d_env, d->d_frame, 1, n, d->X, d->U, d->dV, d->Fm, d->fib, d->stamps, d->d_state, d->status);
        k_adj_tiles<<<blocks, K1_THREADS, 0, d->stream>>>(f, lam_in, d->d_env, d->d_frame, d->fib, d->stamps,
                                                          d->d_state, d->adj_lfib);
        k_adj_ib<<<(n + wb - 1) / wb, IB_THREADS, 0, d->stream>>>(
            f, d->d_env, d->d_frame, n, d->X, d->U, d->dV, d->seg, d->adj_lfib, d->adj_gF, d->mk[0].nseg,
            d->adj_lrho, d->adj_lut, gX, gU);
    }
    k_adj_stream_collide<<<blocks, K1_THREADS, 0, d->stream>>>(f, lam_in, lam_out, d->d_env, d->d_frame, d->fib,
                                                               d->stamps, d->d_state, d->adj_lfib, d->adj_lrho,
                                                               d->adj_lut);
    k_advance_stamp<<<1, 1, 0, d->stream>>>(d->d_state);
    CK(cudaGetLastError());
    d->adj_cur ^= 1;
    return note_stamp_advance(d);
}

fg_status fg_adjoint_step(fg_domain* d, const fg_frame* frames, const double* gF, float* gX, float* gU) {
    NvtxRange nvtx_range("fg_adjoint_step");
    fg_status st = adjoint_check(d);
    if (st != FG_OK) return st;
    return adjoint_step_from(d, (const float*)d->pop[d->cur], frames, gF, gX, gU);
}

fg_status fg_adjoint_step_state(fg_domain* d, const void* state, const fg_frame* frames, const double* gF,
                                float* gX, float* gU) {
    NvtxRange nvtx_range("fg_adjoint_step_state");
    fg_status st = adjoint_check(d);
    if (st != FG_OK) return st;
    if (!state) return fail(FG_ERR_INVALID, "null state buffer");
    return adjoint_step_from(d, (const float*)state, frames, gF, gX, gU);
}

fg_status fg_get_adjoint(fg_domain* d, double* lam) {
    fg_status st = adjoint_check(d);
    if (st != FG_OK) return st;
    if (!lam) return fail(FG_ERR_INVALID, "null output");
    const EnvDev& E = d->env[0];
    std::vector<float> raw((size_t)27 * E.nslot);
    CK(cudaMemcpyAsync(raw.data(), d->adj_lam[d->adj_cur], sizeof(float) * raw.size(), cudaMemcpyDeviceToHost,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
    const size_t ncell = env_cells(d, 0);
    for (size_t c = 0; c < ncell; ++c) {
        const size_t row = c / E.n[0], x = c - row * E.n[0], s = row * E.P + x;
        for (int i = 0; i < 27; ++i) lam[c * 27 + i] = raw[(size_t)i * E.nslot + s];
    }
    return FG_OK;
}

fg_status fg_set_adjoint(fg_domain* d, const double* lam) {
    fg_status st = adjoint_check(d);
    if (st != FG_OK) return st;
    if (!lam) return fail(FG_ERR_INVALID, "null input");
    const EnvDev& E = d->env[0];
    std::vector<float> raw((size_t)27 * E.nslot, 0.0f);
    const size_t ncell = env_cells(d, 0);
    for (size_t c = 0; c < ncell; ++c) {
        const size_t row = c / E.n[0], x = c - row * E.n[0], s = row * E.P + x;
        for (int i = 0; i < 27; ++i) raw[(size_t)i * E.nslot + s] = (float)lam[c * 27 + i];
    }
    CK(cudaMemcpyAsync(d->adj_lam[d->adj_cur], raw.data(), sizeof(float) * raw.size(), cudaMemcpyHostToDevice,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

fg_status fg_copy_state(fg_domain* d, int env, void* buf, int to_buf) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!buf) return fail(FG_ERR_INVALID, "null buffer");
    if (d->aa) return aa_state_copy(d, env, buf, to_buf != 0);
    const EnvDev& E = d->env[env];
    char* state = (char*)d->pop[d->cur] + E.pop_off * d->esize;
    const size_t bytes = 27ull * E.nslot * d->esize;
    if (to_buf)
        CK(cudaMemcpyAsync(buf, state, bytes, cudaMemcpyDeviceToDevice, d->stream));
    else
        CK(cudaMemcpyAsync(state, buf, bytes, cudaMemcpyDeviceToDevice, d->stream));
    return FG_OK;
}

fg_status fg_autotune(fg_domain* d, int* choice, double* ms) {
    NvtxRange nvtx_range("fg_autotune");
    if (!d) return fail(FG_ERR_INVALID, "null domain");
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    d->autotune_pending = false;
    if (d->aa) {
        // in place, a timed pass would advance the state; the layout has one
        // stream-collide kernel
        if (ms)
            for (int v = 0; v < K1_NVARIANTS; ++v) ms[v] = -1.0;
        if (choice) *choice = K1_PLAIN;
        return FG_OK;
    }
    CK(cudaStreamSynchronize(d->stream));
    // The IB pass of a timed candidate rewrites the marker forces; the last
    // step's are kept aside and put back.
    float* fm_keep = nullptr;
    const size_t fm_n = 3ull * (size_t)d->marker_slots;
    if (d->total_markers > 0) {
        fg_status st0 = dalloc(&fm_keep, fm_n);
        if (st0 != FG_OK) return st0;
        CK(cudaMemcpyAsync(fm_keep, d->Fm, sizeof(float) * fm_n, cudaMemcpyDeviceToDevice, d->stream));
    }
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    // Three rounds over the candidates, each variant's time the minimum of
    // its rounds: the rounds interleave the variants, so a clock still
    // ramping up at the start (or another drift) does not favour the ones
    // timed last.
    constexpr int ROUNDS = 3, REPS = 5;
    double best_of[K1_NVARIANTS];
    for (int v = 0; v < K1_NVARIANTS; ++v) best_of[v] = -1.0;
    fg_status st = FG_OK;
    for (int round = 0; round < ROUNDS && st == FG_OK; ++round) {
        for (int v = 0; v < K1_NVARIANTS && st == FG_OK; ++v) {
            if (!k1_runnable(d, v)) continue;
            if ((st = configure_k1(d, v, true)) != FG_OK) break;
            if ((st = sync_work_table(d)) != FG_OK) break;
            // The step without its reduction: the IB kernel and the
            // stream-collide kernel (the fused kernel does both), reading the
            // current state and writing the other buffer, which the next step
            // overwrites.  The stamp does not advance (the reduction advances
            // it), so the next step stamps the same tiles again; every tile
            // that received IB force is stamped, so the stream-collide pass
            // leaves the force field zero.
            st = dispatch(d->opt.storage, [&](auto tag) -> fg_status {
                typedef decltype(tag) S;
                typedef typename S::raw raw;
                const raw* gin = (const raw*)d->pop[d->cur];
                raw* gout = (raw*)d->pop[d->cur ^ 1];
                auto pass = [&]() -> fg_status {
                    if (v == K1_FUSED) return enqueue_fused<S>(d, gin, gout, d->stream);
                    if (v == K1_OVERLAP && d->total_markers > 0) return enqueue_overlap<S>(d, gin, gout, d->stream, nullptr);
                    if (d->total_markers > 0) {
                        fg_status s1 = enqueue_ib<S>(d, gin, d->stream);
                        if (s1 != FG_OK) return s1;
                    }
                    enqueue_k1<S>(d, gin, gout, d->stream);
                    return FG_OK;
                };
                fg_status s2 = FG_OK;
                for (int w = 0; w < 2 && s2 == FG_OK; ++w) s2 = pass();
                CK(cudaEventRecord(a, d->stream));
                for (int r = 0; r < REPS && s2 == FG_OK; ++r) s2 = pass();
                CK(cudaEventRecord(b, d->stream));
                if (s2 != FG_OK) return s2;
                CK(cudaGetLastError());
                CK(cudaEventSynchronize(b));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, a, b));
                const double per = t / REPS;
                if (best_of[v] < 0.0 || per < best_of[v]) best_of[v] = per;
                return FG_OK;
            });
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (fm_keep) {
        cudaMemcpyAsync(d->Fm, fm_keep, sizeof(float) * fm_n, cudaMemcpyDeviceToDevice, d->stream);
        cudaStreamSynchronize(d->stream);
        cudaFree(fm_keep);
    }
    if (st != FG_OK) return st;
    // Timed alone, the stream-collide variants miss what the step adds around
    // them: on the 256x128x128 swimmer channel the plain and staged-256
    // kernels came out within 1% of each other alone, in either order from
    // run to run, while whole steps with the plain kernel were 2% faster
    // (0.1825 against 0.1864 ms, three runs each).  So a staged variant is
    // kept only when it is faster by more than that.
    constexpr double STAGED_MARGIN = 0.98;
    auto score = [&](int v) { return (v == K1_STAGED256 || v == K1_STAGED512) ? best_of[v] / STAGED_MARGIN : best_of[v]; };
    int best = -1;
    for (int v = 0; v < K1_NVARIANTS; ++v) {
        if (ms) ms[v] = best_of[v];
        if (best_of[v] < 0.0) continue;
        if (best < 0 || score(v) < score(best)) best = v;
    }
    if ((st = configure_k1(d, best, true)) != FG_OK) return st;
    if ((st = sync_work_table(d)) != FG_OK) return st;
    if (choice) *choice = best;
    return FG_OK;
}

fg_status fg_stream_collide_variant(fg_domain* d, int* variant) {
    if (!d || !variant) return fail(FG_ERR_INVALID, "null argument");
    *variant = d->k1;
    return FG_OK;
}

fg_status fg_stream_collide_bytes(fg_domain* d, unsigned long long* bytes) {
    if (!d || !bytes) return fail(FG_ERR_INVALID, "null argument");
    *bytes = 2ull * 27ull * d->total_cells * d->esize;
    return FG_OK;
}

}  // extern "C"

namespace {

// The device table's body states -> the host copy.
fg_status sphere_download(fg_domain* d) {
    if (d->sph_host.empty() || !d->sph) return FG_OK;
    CK(cudaMemcpyAsync(d->sph_host.data(), d->sph, sizeof(SphereDev) * d->sph_host.size(), cudaMemcpyDeviceToHost,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

// The host table -> the device, with the marker offsets of the current
// marker layout; grows the device arrays (a captured step that baked the old
// ones is captured again: the graph key holds the table's address).
fg_status sphere_upload(fg_domain* d) {
    const int n = (int)d->sph_host.size();
    size_t ndirs = 0;
    int max_n = 0;
    for (int k = 0; k < n; ++k) {
        SphereDev& s = d->sph_host[k];
        s.mk_off = d->mk[s.env].off;
        s.dir_off = (int)(ndirs / 3);
        ndirs += d->sph_dirs_host[k].size();
        max_n = std::max(max_n, s.n);
    }
    d->sph_max_n = max_n;
    if (n == 0) return FG_OK;
    if (n > d->sph_cap) {
        SphereDev* p = nullptr;
        Pair32* q = nullptr;
        fg_status st = dalloc(&p, (size_t)n);
        if (st == FG_OK) st = dalloc(&q, (size_t)n * 4 * d->n_sms * 7);
        if (st != FG_OK) {
            if (p) cudaFree(p);
            return st;
        }
        CK(cudaStreamSynchronize(d->stream));
        if (d->sph) cudaFree(d->sph);
        if (d->sph_part) cudaFree(d->sph_part);
        d->sph = p;
        d->sph_part = q;
        d->sph_cap = n;
    }
    if (ndirs > (size_t)d->sph_dirs_cap) {
        double* p = nullptr;
        fg_status st = dalloc(&p, ndirs);
        if (st != FG_OK) return st;
        CK(cudaStreamSynchronize(d->stream));
        if (d->sph_dirs) cudaFree(d->sph_dirs);
        d->sph_dirs = p;
        d->sph_dirs_cap = (int)ndirs;
    }
    std::vector<double> all;
    all.reserve(ndirs);
    for (const auto& v : d->sph_dirs_host) all.insert(all.end(), v.begin(), v.end());
    CK(cudaMemcpyAsync(d->sph_dirs, all.data(), sizeof(double) * ndirs, cudaMemcpyHostToDevice, d->stream));
    CK(cudaMemcpyAsync(d->sph, d->sph_host.data(), sizeof(SphereDev) * n, cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

}  // namespace

extern "C" {

fg_status fg_attach_sphere(fg_domain* d, int env, double radius, const double* center, double density_ratio,
                           const double* gravity, int n, const double* dirs, const float* dV, int box_reaction) {
    NvtxRange nvtx_range("fg_attach_sphere");
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (d->poisoned) return fail(FG_ERR_STATE, "domain poisoned by a numeric fault; call fg_init_fields");
    if (!center || !gravity || !dirs || !dV) return fail(FG_ERR_INVALID, "null argument");
    if (!(radius > 0.0) || !std::isfinite(radius)) return fail(FG_ERR_INVALID, "radius must be positive");
    if (!(density_ratio > 0.0) || !std::isfinite(density_ratio))
        return fail(FG_ERR_INVALID, "density ratio must be positive");
    if (n < 1) return fail(FG_ERR_INVALID, "a sphere needs markers");
    if (box_reaction != 0 && box_reaction != 1) return fail(FG_ERR_INVALID, "box_reaction must be 0 or 1");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(center[a]) || !std::isfinite(gravity[a])) return fail(FG_ERR_INVALID, "not finite");
    for (size_t k = 0; k < 3ull * n; ++k)
        if (!std::isfinite(dirs[k])) return fail(FG_ERR_INVALID, "direction not finite");
    if (has_sphere(d, env)) return fail(FG_ERR_STATE, "a sphere is attached to this environment already");
    // the shell at rest: X = c + R d, U = 0 (the checks of fg_set_markers apply)
    std::vector<float> X(3ull * n), U(3ull * n, 0.0f);
    for (int l = 0; l < n; ++l)
        for (int a = 0; a < 3; ++a) X[3ull * l + a] = (float)(center[a] + radius * dirs[3ull * l + a]);
    if ((st = set_markers_impl(d, env, n, X.data(), U.data(), dV, nullptr, 1, center, 0)) != FG_OK) return st;
    if ((st = sphere_download(d)) != FG_OK) return st;
    SphereDev s;
    std::memset(&s, 0, sizeof(s));
    const double volume = 4.0 * M_PI * std::pow(radius, 3) / 3.0;
    s.R = radius;
    s.mp = density_ratio * volume;
    s.mf = volume;
    s.Ip = 0.4 * s.mp * std::pow(radius, 2);
    for (int a = 0; a < 3; ++a) {
        s.c[a] = center[a];
        s.g[a] = gravity[a];
    }
    s.env = env;
    s.n = n;
    // in a periodic box nothing else holds the excess weight: the fluid gets
    // the reaction as a uniform frame acceleration (Eq. 3's acc term)
    const double fluid_mass = (double)env_cells(d, env);
    for (int a = 0; a < 3; ++a) d->box_acc[env][a] = box_reaction ? (s.mp - s.mf) * gravity[a] / fluid_mass : 0.0;
    set_env_frame(d, env, d->user_frame[env]);
    if ((st = upload_frames(d)) != FG_OK) return st;
    d->sph_host.push_back(s);
    d->sph_dirs_host.emplace_back(dirs, dirs + 3ull * n);
    if ((st = sphere_upload(d)) != FG_OK) {
        d->sph_host.pop_back();
        d->sph_dirs_host.pop_back();
        return st;
    }
    // the inner fluid's momentum in the current state: the first step's dP_in
    // and dL_in are measured from it
    const int k = (int)d->sph_host.size() - 1;
    const int grid = 4 * d->n_sms;
    st = dispatch(d->opt.storage, [&](auto tag) -> fg_status {
        typedef decltype(tag) S;
        k_sphere_fluid<S><<<dim3((unsigned)grid, 1u), RED_THREADS, 0, d->stream>>>(
            (const typename S::raw*)d->pop[d->cur], d->d_env, d->sph + k, aa_of(d), d->sph_part + (size_t)k * grid * 7);
        k_sphere_update<<<1, 32, 0, d->stream>>>(d->sph + k, d->sph_part + (size_t)k * grid * 7, grid, d->ft, 1);
        CK(cudaGetLastError());
        return FG_OK;
    });
    if (st != FG_OK) return st;
    CK(cudaStreamSynchronize(d->stream));
    return FG_OK;
}

fg_status fg_sphere_state(fg_domain* d, int env, double* out) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if (!out) return fail(FG_ERR_INVALID, "null output");
    if ((st = sphere_download(d)) != FG_OK) return st;
    for (const SphereDev& s : d->sph_host)
        if (s.env == env) {
            for (int a = 0; a < 3; ++a) {
                out[a] = s.c[a];
                out[3 + a] = s.V[a];
                out[6 + a] = s.W[a];
            }
            return FG_OK;
        }
    return fail(FG_ERR_STATE, "no sphere attached to this environment");
}

fg_status fg_detach_sphere(fg_domain* d, int env) {
    fg_status st = check_env(d, env);
    if (st != FG_OK) return st;
    if ((st = sphere_download(d)) != FG_OK) return st;
    for (size_t k = 0; k < d->sph_host.size(); ++k)
        if (d->sph_host[k].env == env) {
            d->sph_host.erase(d->sph_host.begin() + (long)k);
            d->sph_dirs_host.erase(d->sph_dirs_host.begin() + (long)k);
            d->box_acc[env] = {0.0, 0.0, 0.0};
            set_env_frame(d, env, d->user_frame[env]);
            if ((st = upload_frames(d)) != FG_OK) return st;
            return sphere_upload(d);
        }
    return fail(FG_ERR_STATE, "no sphere attached to this environment");
}

}  // extern "C"
