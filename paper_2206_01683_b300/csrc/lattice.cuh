// lattice.cuh -- D3Q27 velocity set, population storage types and the small
// device helpers the step kernels share.
//
// Velocity order of this library: i = (cx+1) + 3 (cy+1) + 9 (cz+1), so the
// rest velocity is i = 13 and the opposite of i is 26 - i.  Weights depend on
// |c|^2: 8/27, 2/27, 1/54, 1/216 (c_s^2 = 1/3).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fl {

constexpr int Q = 27;

__host__ __device__ constexpr int cx(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
__host__ __device__ constexpr double wd(int i) {
    return csq(i) == 0 ? 8.0 / 27.0 : csq(i) == 1 ? 2.0 / 27.0 : csq(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
}
__host__ __device__ constexpr float wf(int i) { return (float)wd(i); }

// Reduced-precision storage keeps h_i = s_i (f_i - w_i) with s_i = 4^(1+|c|^2)
// (4, 16, 64, 256).  s_i w_i = 32/27 for every i, so all 27 stored values have
// the same magnitude; powers of two make the scaling exact.
__host__ __device__ constexpr float store_scale(int i) { return (float)(4 << (2 * csq(i))); }

// Population storage.  load/store take the velocity index so that reduced
// formats can apply their per-velocity scale; FP32 stores f_i - w_i as is.
// widen(v) is the stored value as a float without that scale (s_i g_i for
// the reduced formats, SCALED), for moment sums that apply the scales
// themselves (accumulate_stored).
// load2_rw reads two neighbouring slots (the first aligned to twice the
// element size) with one ordinary, coherent load, for a kernel that also
// writes the array it reads.
// emit(v, i) stores the population whose Hermite polynomial value is v
// (g_i = w_i v) given coefficients pre-multiplied by POLY: FP32 stores w_i v;
// the reduced formats store s_i g_i = (32/27) v, so with POLY = 32/27 they
// store v itself and need no per-population multiply.  emit2 stores the
// values of two neighbouring slots (the first at p, which is aligned to
// twice the element size) with one access.
struct StoreF32 {
    typedef float raw;
    static constexpr float POLY = 1.0f;
    static constexpr bool SCALED = false;
    static __device__ __forceinline__ float widen(raw v) { return v; }
    static __device__ __forceinline__ void emit(raw* p, float v, int i) { *p = wf(i) * v; }
    static __device__ __forceinline__ void emit2(raw* p, float a, float b, int i) {
        *reinterpret_cast<float2*>(p) = make_float2(wf(i) * a, wf(i) * b);
    }
    static __device__ __forceinline__ float load(const raw* p, int) { return __ldg(p); }
    static __device__ __forceinline__ float2 load2_rw(const raw* p, int) {
        return *reinterpret_cast<const float2*>(p);
    }
    static __device__ __forceinline__ void store(raw* p, float v, int) { *p = v; }
    static __device__ __forceinline__ float decode(raw v, int) { return v; }
    static __device__ __forceinline__ raw encode(float v, int) { return v; }
};

struct StoreF16 {
    typedef __half raw;
    static constexpr float POLY = 32.0f / 27.0f;
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ float widen(raw v) { return __half2float(v); }   // s_i g_i
    static __device__ __forceinline__ void emit(raw* p, float v, int) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void emit2(raw* p, float a, float b, int) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
    static __device__ __forceinline__ float decode(raw v, int i) {
        return __half2float(v) * (1.0f / store_scale(i));
    }
    static __device__ __forceinline__ raw encode(float v, int i) {
        return __float2half_rn(v * store_scale(i));
    }
    static __device__ __forceinline__ float load(const raw* p, int i) { return decode(__ldg(p), i); }
    static __device__ __forceinline__ float2 load2_rw(const raw* p, int i) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
        return make_float2(v.x * (1.0f / store_scale(i)), v.y * (1.0f / store_scale(i)));
    }
    static __device__ __forceinline__ void store(raw* p, float v, int i) { *p = encode(v, i); }
};

struct StoreBF16 {
    typedef __nv_bfloat16 raw;
    static constexpr float POLY = 32.0f / 27.0f;
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ float widen(raw v) { return __bfloat162float(v); }   // s_i g_i
    static __device__ __forceinline__ void emit(raw* p, float v, int) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void emit2(raw* p, float a, float b, int) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
    static __device__ __forceinline__ float decode(raw v, int i) {
        return __bfloat162float(v) * (1.0f / store_scale(i));
    }
    static __device__ __forceinline__ raw encode(float v, int i) {
        return __float2bfloat16_rn(v * store_scale(i));
    }
    static __device__ __forceinline__ float load(const raw* p, int i) { return decode(__ldg(p), i); }
    static __device__ __forceinline__ float2 load2_rw(const raw* p, int i) {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        return make_float2(v.x * (1.0f / store_scale(i)), v.y * (1.0f / store_scale(i)));
    }
    static __device__ __forceinline__ void store(raw* p, float v, int i) { *p = encode(v, i); }
};

// Unsigned division by a run-time constant d >= 1 for n < 2^31, by a
// multiply-high and a shift (Granlund & Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1,  n / d = (mulhi(n, m) + n) >> l.
struct FastDiv {
    uint32_t m, l;
};

inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    FastDiv f;
    f.m = (uint32_t)m;
    f.l = l;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) {
    return (__umulhi(n, f.m) + n) >> f.l;
}

// Debug builds (-DFG_DEBUG_BOUNDS, libfishlbm_debug.so) check the indices
// the kernels compute before using them: a failed check sets its bit in a
// device flag word (read with fg_debug_flags) and the access is skipped, so
// an indexing error is reported instead of faulting.  In release builds the
// checks compile to nothing.
enum {
    DBG_PULL = 1,       // stream-collide: pulled population outside the plane
    DBG_STORE = 2,      // stream-collide: emitted slot outside the plane
    DBG_COPY = 4,       // staged kernel: source row or buffer range of a bulk copy
    DBG_SMEM = 8,       // staged kernel: staged-row read outside the buffer
    DBG_NODE = 16,      // IB: stencil node outside the plane
    DBG_REDUCE = 32,    // reduction: chunk outside the partial buffer
    DBG_REGION = 64     // region momentum: cell outside the plane
};
#ifdef FG_DEBUG_BOUNDS
static __device__ unsigned int g_debug_flags;
__device__ __forceinline__ bool debug_in_range(unsigned bit, long long idx, long long n) {
    const bool ok = idx >= 0 && idx < n;
    if (!ok) atomicOr(&g_debug_flags, bit);
    return ok;
}
#define FG_IN_RANGE(bit, idx, n) ::fl::debug_in_range((bit), (long long)(idx), (long long)(n))
#else
#define FG_IN_RANGE(bit, idx, n) true
#endif

// Peskin's 4-point function (Peskin 2002, Acta Numerica 11, Sec. 6).
__device__ __forceinline__ float peskin4(float r) {
    r = fabsf(r);
    if (r <= 1.0f) return (3.0f - 2.0f * r + sqrtf(1.0f + 4.0f * r - 4.0f * r * r)) * 0.125f;
    if (r <= 2.0f) return (5.0f - 2.0f * r - sqrtf(-7.0f + 12.0f * r - 4.0f * r * r)) * 0.125f;
    return 0.0f;
}

}  // namespace fl
