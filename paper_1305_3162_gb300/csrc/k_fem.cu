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
// the load, the FP64 residual and the correction; the load and the residual
// form their scalars in their last block.
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
// product gathers is formed there from r_k, w_k and s_{k-1}, which a row
// keeps together with its 1 / diagonal in one 16-byte record (the step
// reads the records of one parity and writes those of the other).  A launch
// leaves its blocks' partial sums of gamma_{k+1}, delta_{k+1} and r.r; every
// block of the next launch adds them itself, in one fixed order, and derives
// alpha_{k+1} and beta_{k+1}, so all blocks hold the same scalars, no launch
// ends in a one-block tail, and the solve repeats bitwise.  An inner
// iteration starts with a set-up launch (the same kernel with alpha = beta =
// 0), which forms w_0 = S u_0 and the first partial sums.  The launches are
// chained by programmatic dependent launch: before its dependency wait a
// thread loads its row's first column indices and entries (plan data).  The
// inner steps give each row one thread over the matrix in slices of 32 rows
// (every lane busy with its own row's update, coalesced reads of the
// entries); the load uses groups of 8 lanes per row over CSR.  Launches
// after the inner stop return at once, so the rest of a pass of the solve
// graph's inner loop costs only empty launches.
#include <algorithm>
#include <cmath>

#include "dev_common.cuh"
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
    if (!arrive(d, v, &d.st->count[1])) return;
    double t[1];
    sum_partials(d, gridDim.x, t, sh);
    if (threadIdx.x == 0) {
        CgState &s = *d.st;
        s.outer += 1;
        new_residual(d, s, t[0]);
    }
}

// Start of an inner iteration (per row): the parity-0 records
// {r_0 = rho / scale, w = 0, s = 0, 1 / diagonal}, correction and direction
// zero; the inner record 0 set for the set-up launch.
__global__ void __launch_bounds__(NT) k_cg_scale(FemDev d) {
    if (block_flag(&d.st->done)) return;
    const double inv = d.st->inv_scale;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < d.nf; i += (int64_t)gridDim.x * NT) {
        d.xc[i] = 0.f;
        d.p[i] = 0.f;
        d.v[0][i] = make_float4((float)(d.rho[i] * inv), 0.f, 0.f, d.dinv[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        CgInner &o = d.st->in[0];
        o.gamma = o.alpha = o.rr0 = 0.f;
        o.mode = 0;
        o.iter = d.st->iter;
    }
}

// Sums over the block of K values, the same in every thread (a fixed order:
// shuffles down to lane 0, then the warps' sums in warp order).
template <int K> __device__ void block_sum_all(float (&v)[K], float (*sh)[NT / 32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k][warp] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += sh[k][w];
        v[k] = t;
    }
}

constexpr int CH = 8;  // matrix entries of a row loaded, and columns gathered, at once

// w += (S u)(row) over the row's entries [k0, width) of its slice (base: the
// lane's first entry), u at each column from its record, CH entries at a
// time; entries past the row's width read the row's own record with weight 0.
__device__ __forceinline__ void row_product(const FemDev &d, const float4 *__restrict__ v0, int64_t base, int width,
                                            int k0, int self, float alpha, float beta, float &w) {
    for (; k0 < width; k0 += CH) {
        int c[CH];
        float a[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const bool ok = k0 + j < width;
            c[j] = ok ? d.sl_col[base + 32 * (k0 + j)] : self;
            a[j] = ok ? d.sl_val[base + 32 * (k0 + j)] : 0.f;
        }
        float4 g[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) g[j] = v0[c[j]];
#pragma unroll
        for (int j = 0; j < CH; ++j) w += a[j] * (g[j].w * (g[j].x - alpha * (g[j].y + beta * g[j].z)));
    }
}

// One inner launch of parity q (records and partial sums of parity q read,
// those of parity q ^ 1 written): the set-up launch (mode 0) or a step.
// Before the dependency wait a thread takes its row's first 2 CH entries
// (plan data): CH into registers, CH into shared memory.  After it, the
// loads that do not depend on the step's scalars go out together: the stop
// flag, the inner record, the previous launch's partial sums, the first CH
// gathered columns (their addresses are plan data) and the row's own record;
// alpha and beta are formed while they are in flight.
__global__ void __launch_bounds__(NT, 4) k_cg_step(FemDev d, int q) {
    __shared__ float sh_in[3][NT / 32], sh_out[3][NT / 32];
    __shared__ int s_col[CH][NT];
    __shared__ float s_val[CH][NT];
    __shared__ int s_done;
    const int lane = threadIdx.x & 31;
    const int64_t nsl = (d.nf + 31) >> 5, tstep = ((int64_t)gridDim.x * NT) >> 5;
    int64_t t = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    int64_t base = 0;
    int width = 0;
    int self = 0;
    if (t < nsl) {
        base = d.sl_ptr[t] + lane;
        width = d.sl_w[t];
        self = (int)min(32 * t + lane, d.nf - 1);
    }
    int c[CH];
    float a[CH];
#pragma unroll
    for (int j = 0; j < 2 * CH; ++j) {
        const bool ok = j < width;
        const int cj = ok ? d.sl_col[base + 32 * j] : self;
        const float aj = ok ? d.sl_val[base + 32 * j] : 0.f;
        if (j < CH) {
            c[j] = cj;
            a[j] = aj;
        } else {
            s_col[j - CH][threadIdx.x] = cj;
            s_val[j - CH][threadIdx.x] = aj;
        }
    }
    pdl_wait();
    pdl_trigger();
    int flag = 0;
    if (threadIdx.x == 0) flag = *(volatile const int *)&d.st->done;
    const CgInner in = d.st->in[q];
    const float4 *__restrict__ v0 = d.v[q];
    float4 g[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) g[j] = v0[c[j]];
    // the previous launch's partial sums: gamma, delta and r.r of its result
    // (read whatever the mode; used only after a step)
    float v[3] = {0.f, 0.f, 0.f};
    {
        const float *part = d.part32 + (size_t)q * 3 * d.nblk_max;
        const int n = (int)gridDim.x;
        for (int i0 = 0; i0 < n; i0 += 2 * NT) {
            float b[3][2];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int ii = i0 + j * NT + threadIdx.x;
                    b[k][j] = ii < n ? __ldcg(part + k * d.nblk_max + ii) : 0.f;
                }
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 2; ++j) v[k] += b[k][j];
        }
    }
    if (threadIdx.x == 0) s_done = flag;
    block_sum_all(v, sh_in);  // its barrier also publishes s_done
    if (s_done) return;       // the same in every thread of the block
    float alpha = 0.f, beta = 0.f;
    if (in.mode > 0) {
        const float gm = v[0], dl = v[1], rr = v[2];
        float rr0 = in.rr0;
        if (in.mode == 1) {
            beta = 0.f;
            alpha = gm / dl;
            rr0 = rr;
        } else {
            beta = gm / in.gamma;
            alpha = gm / (dl - beta * gm / in.alpha);
        }
        // a residual that reached the stopping test (exactly zero included,
        // where the coefficients are 0/0) ends the inner iteration
        const bool conv = rr <= d.inner2 * rr0;
        const bool bad = !isfinite(rr) || (!conv && !(isfinite(alpha) && isfinite(beta)));
        const bool stop = bad || conv || in.iter >= d.max_iter;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            CgState &s = *d.st;
            s.gamma = gm;
            s.rr = rr;
            s.iter = stop ? in.iter : in.iter + 1;
            if (stop) {
                s.bad = s.bad || bad;
                s.done = 1;
            } else {
                CgInner &on = s.in[q ^ 1];
                on.gamma = gm;
                on.alpha = alpha;
                on.rr0 = rr0;
                on.mode = 2;
                on.iter = in.iter + 1;
            }
        }
        if (stop) return;  // the same decision in every block
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        CgInner &on = d.st->in[q ^ 1];
        on.gamma = on.alpha = on.rr0 = 0.f;
        on.mode = 1;
        on.iter = in.iter;
    }
    float4 *__restrict__ v1 = d.v[q ^ 1];
    float gm = 0.f, dl = 0.f, rr = 0.f;
    // the row update from its own record and the product w of its row
    auto update = [&](int64_t r, float w, float4 rec, float p_old, float x_old) {
        const float p = rec.w * rec.x + beta * p_old;
        const float sn = rec.y + beta * rec.z;
        d.p[r] = p;
        d.xc[r] = x_old + alpha * p;
        const float rn = rec.x - alpha * sn;
        v1[r] = make_float4(rn, w, sn, rec.w);
        const float un = rec.w * rn;
        gm += rn * un;
        dl += w * un;
        rr += rn * rn;
    };
    int64_t i = 32 * t + lane;
    if (t < nsl) {
        // the row's own record and the second chunk's columns, in flight
        // while the first chunk is added
        const bool row = i < d.nf;
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        float pold = 0.f, xold = 0.f;
        if (row) {
            o = v0[i];
            pold = d.p[i];
            xold = d.xc[i];
        }
        float4 h[CH];
        if (width > CH) {
#pragma unroll
            for (int j = 0; j < CH; ++j) h[j] = v0[s_col[j][threadIdx.x]];
        }
        // u_{k+1} at column c from r_k, w_k and s_{k-1}
        float w = 0.f;
#pragma unroll
        for (int j = 0; j < CH; ++j) w += a[j] * (g[j].w * (g[j].x - alpha * (g[j].y + beta * g[j].z)));
        if (width > CH) {
#pragma unroll
            for (int j = 0; j < CH; ++j)
                w += s_val[j][threadIdx.x] * (h[j].w * (h[j].x - alpha * (h[j].y + beta * h[j].z)));
        }
        if (width > 2 * CH) row_product(d, v0, base, width, 2 * CH, self, alpha, beta, w);
        if (row) update(i, w, o, pold, xold);
    }
    // further slices of the warp (meshes with more rows than one thread each)
    for (t += tstep; t < nsl; t += tstep) {
        base = d.sl_ptr[t] + lane;
        width = d.sl_w[t];
        i = 32 * t + lane;
        self = (int)min(i, d.nf - 1);
        float w = 0.f;
        row_product(d, v0, base, width, 0, self, alpha, beta, w);
        if (i < d.nf) update(i, w, v0[i], d.p[i], d.xc[i]);
    }
    float vo[3] = {gm, dl, rr};
    block_sum_all(vo, sh_out);
    if (threadIdx.x == 0) {
        float *out = d.part32 + (size_t)(q ^ 1) * 3 * d.nblk_max;
        out[blockIdx.x] = vo[0];
        out[d.nblk_max + blockIdx.x] = vo[1];
        out[2 * d.nblk_max + blockIdx.x] = vo[2];
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

// Loop control of the solve graph: WHILE (corrections) { WHILE (inner) {
// FEM_CHUNK inner launches }, correction, residual, next inner start }.  One
// thread sets the handle (the only caller while the kernel runs).  Each loop
// also counts its passes on the device and ends at its bound whatever the
// state says, so both loops end: the corrections at FEM_MAX_OUTER, the inner
// passes (which end by themselves once max_iter steps are done) at a bound
// above that, where the solve is marked bad.
__global__ void k_loop_outer_start(FemDev d, cudaGraphConditionalHandle h) {
    d.st->loops_outer = 0;
    cudaGraphSetConditional(h, d.st->outer_done ? 0u : 1u);
}

__global__ void k_loop_outer_next(FemDev d, cudaGraphConditionalHandle h, int bound) {
    CgState &s = *d.st;
    const int n = ++s.loops_outer;
    cudaGraphSetConditional(h, (!s.outer_done && n < bound) ? 1u : 0u);
}

__global__ void k_loop_inner_start(FemDev d, cudaGraphConditionalHandle h) {
    d.st->loops_inner = 0;
    cudaGraphSetConditional(h, d.st->done ? 0u : 1u);
}

__global__ void k_loop_inner_next(FemDev d, cudaGraphConditionalHandle h, int bound) {
    CgState &s = *d.st;
    const int n = ++s.loops_inner;
    if (!s.done && n >= bound) {
        s.bad = 1;
        s.done = 1;
    }
    cudaGraphSetConditional(h, s.done ? 0u : 1u);
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
    return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const FemDev &d, int parity, cudaStream_t s) {
    return launch_k(k_cg_step, dim3(elem_blocks(d)), NT, 0, s, d, parity);
}

cudaError_t launch_fem_correct(const FemDev &d, cudaStream_t s) {
    k_fem_correct<<<elem_blocks(d), NT, 0, s>>>(d);
    k_fem_residual<<<elem_blocks(d), NT, 0, s>>>(d);
    k_cg_scale<<<elem_blocks(d), NT, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_fem_loop(FemLoop which, const FemDev &d, cudaGraphConditionalHandle h, int bound, cudaStream_t s) {
    switch (which) {
        case LOOP_OUTER_START: k_loop_outer_start<<<1, 1, 0, s>>>(d, h); break;
        case LOOP_OUTER_NEXT: k_loop_outer_next<<<1, 1, 0, s>>>(d, h, bound); break;
        case LOOP_INNER_START: k_loop_inner_start<<<1, 1, 0, s>>>(d, h); break;
        case LOOP_INNER_NEXT: k_loop_inner_next<<<1, 1, 0, s>>>(d, h, bound); break;
    }
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
