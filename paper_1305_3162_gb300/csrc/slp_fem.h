// Device data and launchers of the scalar potential phi = phi_1 + phi_2 on a
// tetrahedral mesh (Alg. 1, Sec. 2.1): the P1 load operator, the conjugate
// gradients for the Dirichlet problem of phi_1 (FP32 iterations refined by
// FP64 residuals), the boundary charges g = m.n - dphi_1/dn and the final sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace slp {

// Scalars an inner step carries to the next one.  A step of parity q reads
// record q and block 0 writes record q ^ 1, so no block reads what another
// block of the same launch writes.
struct CgInner {
    float gamma;     // gamma_k = r_k . D^-1 r_k of the step that wrote the record
    float alpha;     // alpha_k of that step
    float rr0;       // r . r at the start of the inner iteration
    int mode;        // 0: set-up launch (alpha = beta = 0), 1: first step, 2: later steps
    long long iter;  // inner steps so far, all corrections together
};

// Scalars of the solve.  The FP64 fields are written by the last block of the
// load and residual launches; the inner steps write `in` (above) and, from
// block 0, the fields the host reads (gamma, rr, iter, done, bad); the solve
// graph's loop-control kernels keep the loop counters.
struct CgState {
    CgInner in[2];
    float gamma;        // r . D^-1 r of the inner residual
    float rr;           // r . r of the inner residual at the last stopping test
    double bb;          // b . b
    double rr_hi;       // |b - S x|^2 (FP64 residual) after the last correction
    double scale;       // the inner problem's right-hand side is rho / scale
    double inv_scale;
    long long iter;     // inner steps, all corrections together
    long long outer;    // corrections (FP64 residuals) done
    int done;           // the inner iteration has stopped: later inner launches return at once
    int outer_done;     // |b - S x| <= tol |b|, out of iterations, or non-finite
    int bad;            // a non-finite scalar was seen
    unsigned count[2];  // arrival counters of the load and residual launches
    int loops_outer;    // passes of the solve graph's correction loop
    int loops_inner;    // passes of its inner loop in the current correction
};

struct FemDev {
    int64_t nf = 0;    // free nodes: the unknowns of the free subsystem
    int nblk_max = 1;  // most blocks of a launch, hence the row length of the partial sums
    // S(fn, fn): CSR over free rows and columns with FP64 values (the
    // residual), and the same matrix in FP32 in slices of 32 rows for the
    // inner steps (one thread per row: entry k of the slice's lane l at
    // sl_ptr[slice] + 32 k + l, sl_w[slice] entries per row, short rows
    // padded with zero entries at their own column); 1 / diagonal in FP32
    const int64_t *s_ptr = nullptr;
    const int *s_col = nullptr;
    const double *s_val = nullptr;
    const int64_t *sl_ptr = nullptr;
    const int *sl_w = nullptr;
    const int *sl_col = nullptr;
    const float *sl_val = nullptr;
    const float *dinv = nullptr;
    // load operator b(fn) = B m, CSR over free rows, columns are the other
    // nodes of the row's tetrahedra, entries |T|/4 grad eta_row summed over
    // them, applied to the differences m_col - m_row (every free row of B sums
    // to zero, so the row's own column drops out); float4 in FP32 plans,
    // double4 in FP64 plans
    const int *fnode = nullptr;  // node of each free row
    const int64_t *b_ptr = nullptr;
    const int *b_col = nullptr;
    const void *b_val = nullptr;
    double *b = nullptr, *x = nullptr, *rho = nullptr;  // FP64 load, solution and residual
    // the inner iteration (FP32): correction and direction, and per row
    // {r, w = S D^-1 r, s = S p, 1 / diagonal} in buffers of even and odd
    // steps (one 16-byte load gives a column everything the product needs)
    float *xc = nullptr, *p = nullptr;
    float4 *v[2] = {nullptr, nullptr};
    double *part = nullptr;   // [nblk_max] block partial sums, FP64 (load, residual)
    float *part32 = nullptr;  // [2][3][nblk_max] block partial sums of the inner steps, by parity
    CgState *st = nullptr;
    double tol2 = 0.0;    // outer stop: |b - S x|^2 <= tol2 |b|^2
    float inner2 = 0.f;   // inner stop: r.r <= inner2 r0.r0
    long long max_iter = 0;
    // boundary triangles: nodes (a, b, c) wound outward and the free index of the
    // owning tetrahedron's fourth node (-1 when it lies on the boundary); unit
    // normal and 1/h, h the tetrahedron's height over the triangle
    int64_t nfaces = 0;
    const int4 *face = nullptr;
    const double4 *face_n = nullptr;
    // per node: free index (>= 0) or -1 - boundary index
    int64_t nnodes = 0;
    const int *slot = nullptr;
};

constexpr int FEM_THREADS = 256;
constexpr int FEM_CHUNK = 16;       // inner launches per pass of the inner loop (even: parities repeat)
constexpr double FEM_INNER = 1e-4;  // each correction's inner steps cut its residual by this factor
constexpr int FEM_MAX_OUTER = 64;   // corrections at most

// Loop control of the solve graph (one thread each): the value of a WHILE
// node's handle, from the state.
enum FemLoop { LOOP_OUTER_START, LOOP_OUTER_NEXT, LOOP_INNER_START, LOOP_INNER_NEXT };

// b = B m and x = 0; the first inner iteration set up from r = b / scale
cudaError_t launch_fem_load(const FemDev &d, int prec, const void *m, cudaStream_t s);
// one inner launch (parity: the launch's index mod 2; each inner iteration
// starts at parity 0 with a set-up launch, then one step per launch)
cudaError_t launch_cg_iteration(const FemDev &d, int parity, cudaStream_t s);
// x += scale * correction, the FP64 residual, the next inner iteration set up from it
cudaError_t launch_fem_correct(const FemDev &d, cudaStream_t s);
// bound: LOOP_OUTER_NEXT the most corrections, LOOP_INNER_NEXT the most inner passes per correction
cudaError_t launch_fem_loop(FemLoop which, const FemDev &d, cudaGraphConditionalHandle h, int bound, cudaStream_t s);
cudaError_t launch_fem_charges(const FemDev &d, int prec, const void *m, void *g, cudaStream_t s);
cudaError_t launch_fem_combine(const FemDev &d, int prec, const void *phi2_b, const void *phi2_f, void *phi,
                               void *phi1, cudaStream_t s);

}  // namespace slp
