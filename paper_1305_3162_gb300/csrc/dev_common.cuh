// Device helpers shared by the CUDA kernels: vector types per precision,
// complex arithmetic, packed cell coordinates and the Kaiser-Bessel window.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "slp_internal.h"

namespace slp {

template <typename T> struct VecT;
template <> struct VecT<float> {
    typedef float2 T2;
    typedef float4 T4;
};
template <> struct VecT<double> {
    typedef double2 T2;
    typedef double4 T4;
};

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmk(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { return cmk(-a.y, a.x); }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return cmk(a.x * s, a.y * s); }

// ---------------------------------------------------------------- cells
// A grid coordinate u = c + f is stored as the fractional part f in [0, 1)
// per axis (x, y, z components) and the integer cell c packed in w:
// cx | cy << 10 | cz << 20 (each axis < 1024).
__device__ __forceinline__ int packed_cell(float w) { return __float_as_int(w); }
__device__ __forceinline__ int packed_cell(double w) { return (int)w; }
// an integer carried in a floating-point slot: bit pattern (FP32) or exact value (FP64)
__device__ __forceinline__ float pack_id(float, int v) { return __int_as_float(v); }
__device__ __forceinline__ double pack_id(double, int v) { return (double)v; }
__device__ __forceinline__ void unpack_cell(int c, int &cx, int &cy, int &cz) {
    cx = c & 1023;
    cy = (c >> 10) & 1023;
    cz = (c >> 20) & 1023;
}

// ---------------------------------------------------------------- window
// Kaiser-Bessel window of the paper's Sec. 3.2 in grid units, truncated to
// |d| <= m and normalised to 1 at d = 0:
//   psi(d) = sinh(beta s) / (s sinh beta),  s = sqrt(1 - (d/m)^2),  beta = b m,
// with the limit beta / sinh(beta) at |d| = m.
__device__ __forceinline__ float kb_window(float d, float inv_m, float beta, float inv_sinh_beta) {
    const float t = d * inv_m;
    const float s2 = 1.0f - t * t;
    if (s2 < 0.0f) return 0.0f;
    const float s = sqrtf(s2);
    const float bs = beta * s;
    const float r = (bs > 1e-3f) ? sinhf(bs) / s : beta * (1.0f + bs * bs * (1.0f / 6.0f));
    return r * inv_sinh_beta;
}
__device__ __forceinline__ double kb_window(double d, double inv_m, double beta, double inv_sinh_beta) {
    const double t = d * inv_m;
    const double s2 = 1.0 - t * t;
    if (s2 < 0.0) return 0.0;
    const double s = sqrt(s2);
    const double bs = beta * s;
    const double r = (bs > 1e-6) ? sinh(bs) / s : beta * (1.0 + bs * bs * (1.0 / 6.0));
    return r * inv_sinh_beta;
}

// Block-wide copy of `total` elements with up to 8 independent loads in
// flight per thread: ld(i) reads element i, st(i, v) stores it.
template <typename V, typename LoadF, typename StoreF>
__device__ __forceinline__ void pipelined_copy(int total, LoadF ld, StoreF st) {
    for (int base = threadIdx.x; base < total; base += 8 * blockDim.x) {
        V tmp[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = base + r * blockDim.x;
            if (i < total) tmp[r] = ld(i);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = base + r * blockDim.x;
            if (i < total) st(i, tmp[r]);
        }
    }
}

// warp sum
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch (sm_90 and later).  Every evaluation kernel
// calls pdl_wait() before it reads or writes any global memory other than
// plan constants (the wait returns once the previous kernel of the stream has
// completed and its writes are visible; at once when the kernel was launched
// without the attribute), and pdl_trigger() right after it, so the next
// kernel of the stream may be scheduled and run its prologue while this one
// works.  Triggering only after the wait keeps at most one waiting kernel
// resident: triggering before it would let the whole chain's blocks occupy
// the SMs while they wait, starving concurrent work.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialization allowed (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, unsigned block, size_t smem, cudaStream_t s,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ void set_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// checked evaluation: record a NaN or Inf among the given values
template <typename T> __device__ __forceinline__ void check_finite3(const DevPlan &p, T a, T b, T c) {
    if (p.check_finite && !(isfinite(a) && isfinite(b) && isfinite(c))) set_error(p.err, DEV_ERR_NONFINITE);
}

}  // namespace slp
