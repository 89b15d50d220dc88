// Kernels of the scalar potential (Alg. 1): phi_1 from the free subsystem of
// the P1 Dirichlet problem (Sec. 2.1), the boundary charges
// g = m.n - dphi_1/dn, and phi_1 + phi_2.
//
// The free subsystem S x = b is solved by iterative refinement: Jacobi-
// preconditioned conjugate gradients in FP32 reduce the residual of the
// current correction equation by FEM_INNER, the correction is added to the
// FP64 solution, and the residual b - S x is recomputed in FP64 (the FP64
// pipe of this GPU is a small fraction of its FP32 rate, while each
// correction needs only a few digits).  Per-thread FP64 work is confined to
// the FP64 residual, the correction and the last block's scalars.
//
// The inner iteration is the conjugate-gradient recurrence with a single
// reduction per step (Chronopoulos and Gear): with u = D^-1 r and w = S u,
//   p_k = u_k + beta_k p_{k-1},  s_k = w_k + beta_k s_{k-1}  (s_k = S p_k),
//   x += alpha_k p_k,  r_{k+1} = r_k - alpha_k s_k,  u_{k+1} = D^-1 r_{k+1},
//   w_{k+1} = S u_{k+1},
//   gamma_{k+1} = r_{k+1} . u_{k+1},  delta_{k+1} = w_{k+1} . u_{k+1},
//   beta_{k+1} = gamma_{k+1} / gamma_k,
//   alpha_{k+1} = gamma_{k+1} / (delta_{k+1} - beta_{k+1} gamma_{k+1} / alpha_k),
// which needs both dot products at one point of the step.  One launch does
// a step: every vector update is per row, and u_{k+1} at the columns the
// product gathers is formed there from r_k, w_k and s_{k-1} (the step reads
// the buffers of one parity and writes those of the other).  The launch's
// block partial sums are combined by its last block (the one whose arrival
// completes the grid; no block waits), in one fixed order, so the solve
// repeats bitwise.  The inner steps give each row one thread over the
// matrix in slices of 32 rows (every lane busy with its own row's update,
// coalesced reads of the entries); the load uses groups of 8 lanes per row
// over CSR.  Steps launched after the inner stop return at once, so a host
// that queues steps ahead of the stopping test wastes only empty launches.
#include <algorithm>
#include <cmath>

#include "slp_fem.h"

namespace slp {
namespace {

constexpr int NT = FEM_THREADS;
constexpr int GROUP = 8;          // lanes per matrix row
constexpr int ROWS = NT / GROUP;  // rows per block and step

// Sum over the block in a fixed order (warp shuffles, then thread 0 adds
// the warps' sums); valid in thread 0 only.  The inner steps sum in FP32:
// this GPU's FP64 pipe is slow enough that a chain of FP64 operations in the
// last block's tail would cost more than the step's product.
template <typename V> __device__ V block_sum(V v, V *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // sh may still be read by a previous call
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    V t = V(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += sh[w];
    return t;
}

// Sum over the GROUP lanes of a row group; the sum lands in the group's first lane.
template <typename V> __device__ V group_sum(V v) {
    for (int o = GROUP / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, GROUP);
    return v;
}

// True when the flag is set (read once per block, so that every thread of
// the block takes the same branch).
__device__ bool block_flag(const int *flag) {
    __shared__ int s_flag;
    if (threadIdx.x == 0) s_flag = *(volatile const int *)flag;
    __syncthreads();
    return s_flag != 0;
}

__device__ __forceinline__ double *partials(const FemDev &d, double) { return d.part; }
__device__ __forceinline__ float *partials(const FemDev &d, float) { return d.part32; }

// Store this block's K partial sums (held by thread 0); returns true in the
// block that arrives last, after which that block may read every block's
// partials (and the arrival counter is reset for the next launch).
template <int K, typename V>
__device__ bool arrive(const FemDev &d, const V (&v)[K], unsigned *counter) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        V *part = partials(d, V(0));
        for (int k = 0; k < K; ++k) part[k * d.nblk_max + blockIdx.x] = v[k];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// Sums of the first n partials of rows 0..K-1 in the last block: every
// thread loads its strided share of all K rows before adding (the loads are
// independent, so they are in flight together: this tail runs while the
// rest of the GPU idles), then a fixed tree; valid in thread 0.
template <int K, typename V>
__device__ void sum_partials(const FemDev &d, int n, V (&out)[K], V *sh) {
    constexpr int PER = 8;  // partials per thread and row loaded at once
    const V *part = partials(d, V(0));
    V v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = V(0);
    for (int i0 = 0; i0 < n; i0 += NT * PER) {
        V buf[K][PER];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int i = i0 + j * NT + threadIdx.x;
                buf[k][j] = i < n ? __ldcg(part + k * d.nblk_max + i) : V(0);
            }
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < PER; ++j) v[k] += buf[k][j];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = block_sum(v[k], sh);
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 t; };
template <> struct Vec4<double> { typedef double4 t; };

// The last block's bookkeeping of a new FP64 residual rho (|rho|^2 = hh):
// the scale of the next inner problem (its right-hand side is rho / scale,
// of unit mean square, so the FP32 inner sums neither underflow nor
// overflow whatever the units of m), and the outer stopping test.
__device__ __forceinline__ void new_residual(const FemDev &d, CgState &s, double hh) {
    s.rr_hi = hh;
    const double scale = sqrt(hh / (double)d.nf);
    s.scale = scale > 0.0 ? scale : 1.0;
    s.inv_scale = 1.0 / s.scale;
    s.bad = s.bad || !isfinite(hh);
    s.outer_done = s.bad || hh <= d.tol2 * s.bb || s.iter >= d.max_iter;
    s.done = s.outer_done;
}

// b(fn) = B m in the plan's precision from the differences m_col - m_row;
// x = 0 and the first residual is b.  The last block sets up the state.
template <typename T>
__global__ void __launch_bounds__(NT) k_fem_load(FemDev d, const T *__restrict__ m) {
    typedef typename Vec4<T>::t T4;
    __shared__ double sh[NT / 32];
    const int gl = threadIdx.x % GROUP;
    const T4 *__restrict__ bv = (const T4 *)d.b_val;
    double bb = 0.0;
    // the loop bound depends on the block only: every lane reaches the shuffles
    for (int64_t i0 = (int64_t)blockIdx.x * ROWS; i0 < d.nf; i0 += (int64_t)gridDim.x * ROWS) {
        const int64_t i = i0 + threadIdx.x / GROUP;
        T b = T(0);
        if (i < d.nf) {
            const int64_t self = d.fnode[i];
            const T mx = m[3 * self], my = m[3 * self + 1], mz = m[3 * self + 2];
            for (int64_t e = d.b_ptr[i] + gl; e < d.b_ptr[i + 1]; e += GROUP) {
                const T4 w = bv[e];
                const int64_t c = d.b_col[e];
                b += w.x * (m[3 * c] - mx) + w.y * (m[3 * c + 1] - my) + w.z * (m[3 * c + 2] - mz);
            }
        }
        b = group_sum(b);
        if (i < d.nf && gl == 0) {
            d.b[i] = (double)b;
            d.rho[i] = (double)b;
            d.x[i] = 0.0;
            bb += (double)b * (double)b;
        }
    }
    const double v[1] = {block_sum(bb, sh)};
    if (!arrive(d, v, &d.st->count[0])) return;
    double t[1];
    sum_partials(d, gridDim.x, t, sh);
    if (threadIdx.x == 0) {
        CgState &s = *d.st;
        s.bb = t[0];
        s.iter = 0;
        s.outer = 0;
        s.bad = 0;
        new_residual(d, s, t[0]);
        if (t[0] == 0.0 || d.max_iter <= 0) s.outer_done = s.done = 1;
    }
}

// The FP64 residual rho = b - S x (one thread per row: no FP64 shuffles);
// the last block decides whether the solve is done.
__global__ void __launch_bounds__(NT) k_fem_residual(FemDev d) {
    __shared__ double sh[NT / 32];
    if (block_flag(&d.st->outer_done)) return;
    double hh = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < d.nf; i += (int64_t)gridDim.x * NT) {
        double sx = 0.0;
        for (int64_t e = d.s_ptr[i]; e < d.s_ptr[i + 1]; ++e) sx += d.s_val[e] * d.x[d.s_col[e]];
        const double rho = d.b[i] - sx;
        d.rho[i] = rho;
        hh += rho * rho;
    }
    const double v[1] = {block_sum(hh, sh)};
    if (!arrive(d, v, &d.st->count[3])) return;
    double t[1];
    sum_partials(d, gridDim.x, t, sh);
    if (threadIdx.x == 0) {
        CgState &s = *d.st;
        s.outer += 1;
        new_residual(d, s, t[0]);
    }
}

// Start of an inner iteration: r_0 = rho / scale in FP32 (parity 0), the
// correction, direction and s zero; gamma_0 = r_0 . D^-1 r_0 and r_0 . r_0.
__global__ void __launch_bounds__(NT) k_cg_scale(FemDev d) {
    __shared__ float sh[NT / 32];
    if (block_flag(&d.st->done)) return;
    const double inv = d.st->inv_scale;
    float rz = 0.f, rr = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < d.nf; i += (int64_t)gridDim.x * NT) {
        const float r = (float)(d.rho[i] * inv);
        d.xc[i] = 0.f;
        d.p[i] = 0.f;
        d.s[0][i] = 0.f;
        d.r[0][i] = r;
        rz += r * (d.dinv[i] * r);
        rr += r * r;
    }
    const float v[2] = {block_sum(rz, sh), block_sum(rr, sh)};
    if (!arrive(d, v, &d.st->count[1])) return;
    float t[2];
    sum_partials(d, gridDim.x, t, sh);
    if (threadIdx.x == 0) {
        CgState &s = *d.st;
        s.gamma = t[0];
        s.rr = s.rr0 = t[1];
    }
}

// Slices of 32 rows handled by the calling warp, one per lane (the loop
// is warp-uniform).
#define FOR_SLICES(t)                                                                            \
    for (int64_t t = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5, nsl_ = (d.nf + 31) >> 5; t < nsl_; \
         t += ((int64_t)gridDim.x * NT) >> 5)

// w_0 = S u_0 (u_0 = D^-1 r_0) and delta_0 = w_0 . u_0; alpha_0 = gamma_0 / delta_0, beta_0 = 0
__global__ void __launch_bounds__(NT) k_cg_init(FemDev d) {
    __shared__ float sh[NT / 32];
    if (block_flag(&d.st->done)) return;
    const int lane = threadIdx.x & 31;
    const float *__restrict__ r0 = d.r[0];
    float dl = 0.f;
    FOR_SLICES(t) {
        const int64_t i = 32 * t + lane;
        const int64_t base = d.sl_ptr[t] + lane;
        const int width = d.sl_w[t];
        float w = 0.f;
#pragma unroll 4
        for (int k = 0; k < width; ++k) {
            const int c = d.sl_col[base + 32 * k];
            w += d.sl_val[base + 32 * k] * (d.dinv[c] * r0[c]);
        }
        if (i < d.nf) {
            d.w[0][i] = w;
            dl += w * (d.dinv[i] * r0[i]);
        }
    }
    const float v[1] = {block_sum(dl, sh)};
    if (!arrive(d, v, &d.st->count[2])) return;
    float t[1];
    sum_partials(d, gridDim.x, t, sh);
    if (threadIdx.x == 0) {
        CgState &s = *d.st;
        s.alpha = s.gamma / t[0];
        s.beta = 0.f;
        const bool bad = !isfinite(s.alpha);
        s.bad = s.bad || bad;
        if (bad) s.done = 1;
    }
}

// One step of the single-reduction recurrence: buffers of parity par are
// read, those of parity par ^ 1 written.
__global__ void __launch_bounds__(NT) k_cg_step(FemDev d, int par) {
    __shared__ float sh[NT / 32];
    if (block_flag(&d.st->done)) return;
    const float alpha = d.st->alpha, beta = d.st->beta;
    const float *__restrict__ r0 = d.r[par];
    const float *__restrict__ w0 = d.w[par];
    const float *__restrict__ s0 = d.s[par];
    float *__restrict__ r1 = d.r[par ^ 1];
    float *__restrict__ w1 = d.w[par ^ 1];
    float *__restrict__ s1 = d.s[par ^ 1];
    const int lane = threadIdx.x & 31;
    float gm = 0.f, dl = 0.f, rr = 0.f;
    FOR_SLICES(t) {
        const int64_t i = 32 * t + lane;
        const int64_t base = d.sl_ptr[t] + lane;
        const int width = d.sl_w[t];
        float w = 0.f;
#pragma unroll 4
        for (int k = 0; k < width; ++k) {
            const int c = d.sl_col[base + 32 * k];
            // u_{k+1} at column c from r_k, w_k and s_{k-1}
            const float rc = r0[c] - alpha * (w0[c] + beta * s0[c]);
            w += d.sl_val[base + 32 * k] * (d.dinv[c] * rc);
        }
        if (i < d.nf) {
            const float di = d.dinv[i];
            const float p = di * r0[i] + beta * d.p[i];
            const float sn = w0[i] + beta * s0[i];
            d.p[i] = p;
            d.xc[i] += alpha * p;
            const float rn = r0[i] - alpha * sn;
            s1[i] = sn;
            r1[i] = rn;
            w1[i] = w;
            const float un = di * rn;
            gm += rn * un;
            dl += w * un;
            rr += rn * rn;
        }
    }
    const float v[3] = {block_sum(gm, sh), block_sum(dl, sh), block_sum(rr, sh)};
    if (!arrive(d, v, &d.st->count[4])) return;
    float t[3];
    sum_partials(d, gridDim.x, t, sh);
    if (threadIdx.x == 0) {
        CgState &s = *d.st;
        const float beta_n = t[0] / s.gamma;
        const float alpha_n = t[0] / (t[1] - beta_n * t[0] / s.alpha);
        s.gamma = t[0];
        s.beta = beta_n;
        s.alpha = alpha_n;
        s.rr = t[2];
        s.iter += 1;
        // a residual that reached the stopping test (exactly zero included,
        // where the next step's coefficients are 0/0) ends the inner iteration
        const bool conv = t[2] <= d.inner2 * s.rr0;
        const bool bad = !isfinite(t[2]) || (!conv && !(isfinite(alpha_n) && isfinite(beta_n)));
        s.bad = s.bad || bad;
        s.done = bad || conv || s.iter >= d.max_iter;
    }
}

// The correction: x += scale xc (FP64), in its own launch so that the
// residual gathers a complete x.
__global__ void __launch_bounds__(NT) k_fem_correct(FemDev d) {
    if (block_flag(&d.st->outer_done)) return;
    const double scale = d.st->scale;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < d.nf; i += (int64_t)gridDim.x * NT)
        d.x[i] += scale * (double)d.xc[i];
}

// g_j = (mean of the nodal m over the triangle) . n_j + phi_1(opposite node) / h_j
// (dphi_1/dn = -phi_1(o)/h_j: the other three nodes are boundary nodes, phi_1 = 0)
template <typename T>
__global__ void __launch_bounds__(NT) k_fem_charges(FemDev d, const T *__restrict__ m, T *__restrict__ g) {
    const int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (j >= d.nfaces) return;
    const int4 f = d.face[j];
    const double4 n = d.face_n[j];
    double mx = 0.0, my = 0.0, mz = 0.0;
    const int v[3] = {f.x, f.y, f.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        mx += (double)m[3 * (int64_t)v[k]];
        my += (double)m[3 * (int64_t)v[k] + 1];
        mz += (double)m[3 * (int64_t)v[k] + 2];
    }
    double val = (mx * n.x + my * n.y + mz * n.z) / 3.0;
    if (f.w >= 0) val += d.x[f.w] * n.w;
    g[j] = (T)val;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_fem_combine(FemDev d, const T *__restrict__ phi2_b,
                                                    const T *__restrict__ phi2_f, T *__restrict__ phi,
                                                    T *__restrict__ phi1) {
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= d.nnodes) return;
    const int s = d.slot[i];
    double a = 0.0, b;
    if (s >= 0) {
        a = d.x[s];
        b = (double)phi2_f[s];
    } else {
        b = (double)phi2_b[-1 - s];
    }
    phi[i] = (T)(a + b);
    if (phi1) phi1[i] = (T)a;
}

unsigned blocks_of(int64_t n) { return (unsigned)((n + NT - 1) / NT); }

// blocks of the row-group kernels and of the element-wise kernels (at most nblk_max)
unsigned row_blocks(const FemDev &d) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((d.nf + ROWS - 1) / ROWS, d.nblk_max));
}
unsigned elem_blocks(const FemDev &d) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((d.nf + NT - 1) / NT, d.nblk_max));
}

}  // namespace

cudaError_t launch_fem_load(const FemDev &d, int prec, const void *m, cudaStream_t s) {
    if (prec == 64)
        k_fem_load<double><<<row_blocks(d), NT, 0, s>>>(d, (const double *)m);
    else
        k_fem_load<float><<<row_blocks(d), NT, 0, s>>>(d, (const float *)m);
    k_cg_scale<<<elem_blocks(d), NT, 0, s>>>(d);
    k_cg_init<<<elem_blocks(d), NT, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const FemDev &d, int parity, cudaStream_t s) {
    k_cg_step<<<elem_blocks(d), NT, 0, s>>>(d, parity);
    return cudaGetLastError();
}

cudaError_t launch_fem_correct(const FemDev &d, cudaStream_t s) {
    k_fem_correct<<<elem_blocks(d), NT, 0, s>>>(d);
    k_fem_residual<<<elem_blocks(d), NT, 0, s>>>(d);
    k_cg_scale<<<elem_blocks(d), NT, 0, s>>>(d);
    k_cg_init<<<elem_blocks(d), NT, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_fem_charges(const FemDev &d, int prec, const void *m, void *g, cudaStream_t s) {
    if (d.nfaces == 0) return cudaSuccess;
    if (prec == 64)
        k_fem_charges<double><<<blocks_of(d.nfaces), NT, 0, s>>>(d, (const double *)m, (double *)g);
    else
        k_fem_charges<float><<<blocks_of(d.nfaces), NT, 0, s>>>(d, (const float *)m, (float *)g);
    return cudaGetLastError();
}

cudaError_t launch_fem_combine(const FemDev &d, int prec, const void *phi2_b, const void *phi2_f, void *phi,
                               void *phi1, cudaStream_t s) {
    if (d.nnodes == 0) return cudaSuccess;
    if (prec == 64)
        k_fem_combine<double><<<blocks_of(d.nnodes), NT, 0, s>>>(d, (const double *)phi2_b, (const double *)phi2_f,
                                                                 (double *)phi, (double *)phi1);
    else
        k_fem_combine<float><<<blocks_of(d.nnodes), NT, 0, s>>>(d, (const float *)phi2_b, (const float *)phi2_f,
                                                                (float *)phi, (float *)phi1);
    return cudaGetLastError();
}

}  // namespace slp
