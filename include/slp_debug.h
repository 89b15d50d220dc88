/*
 * slp_debug.h — inspection entry points of the GB300 single-layer-potential
 * library, for tests and profiling.  They expose intermediate buffers and
 * plan-time host arrays; production callers need only slp.h.
 *
 * Same conventions as slp.h: every call returns an slp_status, host/device
 * pointers as documented, the plan's precision for floating-point data.
 */
#ifndef SLP_DEBUG_H
#define SLP_DEBUG_H

#include <stdint.h>

#include "slp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Pipeline stages of one evaluation, in launch order. */
enum {
    SLP_STAGE_CHARGES = 0, /* qbuf = w sigma, sorted sources */
    SLP_STAGE_SPREAD = 1,  /* grid A: gridding tensor (Sec. 3.1, quadrature form) */
    SLP_STAGE_FFT_X = 2,   /* S1: R2C along x, kx < n_x/2 (grid A is zeroed) */
    SLP_STAGE_FFT_Y = 3,   /* S2: along y, pruned to I_n */
    SLP_STAGE_FFT_Z = 4,   /* S2: along z, times D, inverse along z */
    SLP_STAGE_IFFT_Y = 5,  /* S1: inverse along y, zero-padded */
    SLP_STAGE_IFFT_X = 6,  /* grid B: C2R along x */
    SLP_STAGE_GATHER = 7,  /* phi = smooth part (window interpolation) */
    SLP_STAGE_NEAR = 8     /* phi += near-field correction: the full result */
};

/* Device buffers that slp_debug_copy can read back. */
enum {
    SLP_BUF_QBUF = 0,     /* [Q] */
    SLP_BUF_GRID_A = 1,   /* [Lz][Ly][Lx] */
    SLP_BUF_GRID_B = 2,   /* [Lz][Ly][Lx] */
    SLP_BUF_S1 = 3,       /* complex [Lz][Ly][n_x/2] */
    SLP_BUF_S2 = 4,       /* complex [Lz][n_y][n_x/2] */
    SLP_BUF_DTAB = 5      /* [n_z/2][n_y/2][n_x/2] */
};

/* Plan-time host arrays that slp_debug_host_array can copy out. */
enum {
    SLP_HOST_SRC_PERM = 0,     /* int32 [Q]: sorted position -> source index k */
    SLP_HOST_TGT_PERM = 1,     /* int32 [N]: sorted position -> vertex index */
    SLP_HOST_SRC_GRID = 2,     /* double [Q][4]: frac x, y, z, packed cell (sorted) */
    SLP_HOST_TGT_GRID = 3,     /* double [N][4] */
    SLP_HOST_SPREAD_ITEMS = 4, /* int32 [n][8]: c0x, c0y, c0z, begin, end, 0, 0, 0 */
    SLP_HOST_GATHER_ITEMS = 5, /* int32 [n][8] */
    SLP_HOST_NEAR_ITEMS = 6,   /* int32 [n][4]: tbegin, tcount, rbegin, rend */
    SLP_HOST_NEAR_RANGES = 7,  /* int32 [n][2]: begin, end (sorted sources) */
    SLP_HOST_DTAB = 8,         /* double [n_z/2][n_y/2][n_x/2] */
    SLP_HOST_SRC_POINTS = 9,   /* double [Q][3]: quadrature points, sorted order */
    SLP_HOST_TGT_POINTS = 10,  /* double [N][3]: targets, sorted order */
    SLP_HOST_PLANE_ROWS = 11,  /* int32 [Lz][2]: first active row y0 and active row count of each
                                  plane (rows y0 .. y0 + count - 1 modulo Ly; pair aligned) */
    SLP_HOST_ACTIVE_Z = 12,    /* int32 [2]: first active plane z0 and active plane count (mod Lz) */
    SLP_HOST_SPREAD_GROUPS = 13,    /* int32 [n]: spread cell groups, first source within the item
                                       | source count << 16 */
    SLP_HOST_SPREAD_GROUP_OFF = 14, /* int32 [spread items][9]: bounds of the 8 group lists of each item */
    SLP_HOST_EXPSUM = 15            /* double [S'][2]: weight w_k and exponent g_k of the kept exp-sum terms,
                                       w_k exp(-g_k u^2) summing to about 1/u for u = r / P in [eps / P, 1/2]
                                       (EXPSUM plans; empty otherwise) */
};

/* Run the pipeline of slp_eval up to and including stage last_stage, starting
 * from a zeroed spread grid (a partial run leaves its grid behind). */
slp_status slp_debug_run(slp_plan_t plan, int input_kind, const void *d_in, void *d_phi, void *stream,
                         int last_stage);

/* Copy a device buffer (SLP_BUF_*) to host memory (synchronises the device).
 * bytes must equal the buffer size reported by slp_debug_buffer_bytes. */
slp_status slp_debug_copy(slp_plan_t plan, int buffer, void *host, int64_t bytes);
slp_status slp_debug_buffer_bytes(slp_plan_t plan, int buffer, int64_t *bytes);

/* Element count of a host array (SLP_HOST_*) and a copy of it. */
slp_status slp_debug_host_count(slp_plan_t plan, int which, int64_t *count);
slp_status slp_debug_host_array(slp_plan_t plan, int which, void *out, int64_t count);

/* Run one full evaluation as slp_eval does (near-field branch concurrent on
 * the plan's auxiliary stream) with events recorded at its milestones; ms[0..3]
 * receive the times from the start to: the end of the spread, the end of the
 * FFT passes, the end of the near-field branch and the end of the gather.
 * Synchronises the stream. */
slp_status slp_debug_timeline(slp_plan_t plan, int input_kind, const void *d_in, void *d_phi, void *stream,
                              float *ms);

/* Run one full evaluation in launch order on `stream` and time each kernel
 * with a pair of CUDA events recorded around its launch; ms[i] receives the
 * duration of kernel slot i, or -1 when that slot's kernel did not launch
 * for this plan and input (n >= 15 entries; slots are named by
 * slp_debug_stage_name: charges, spread, fft_x, fft_y, fft_z_mul, ifft_y,
 * ifft_x, nodal_prep, near_zero, near, near_reduce, gather, fft_xy, ifft_yx,
 * fft_yzy).  Synchronises the stream. */
slp_status slp_debug_profile(slp_plan_t plan, int input_kind, const void *d_in, void *d_phi, void *stream,
                             float *ms, int n);
const char *slp_debug_stage_name(int i);

/* The normalised Kaiser-Bessel window psi(d) in grid units (Sec. 3.2,
 * Eq. (KBfct) scaled to psi(0) = 1) and its continuous Fourier transform at
 * frequency index l of an L-point grid, both in FP64 on the host. */
double slp_debug_window(int m, double d);
double slp_debug_window_hat(int m, int L, double l);

/* The host set-up of the scalar potential (slp_potential_create without a
 * device; Sec. 2.1 and Alg. 1): the node classes, the boundary triangles,
 * the free-node stiffness matrix and the load operator, in FP64.
 * nodes, tets: as for slp_potential_create.  counts[5] receives n_free,
 * n_boundary, n_faces, the stiffness entries s_nnz and the load entries
 * b_nnz.  Each array that is not NULL receives (a first call with NULL arrays
 * gives the sizes):
 *   node_slot [n_nodes] int32: free index (>= 0) or -1 - boundary index;
 *   faces [n_faces][4] int32: nodes a, b, c wound so that (b - a) x (c - a)
 *     points out of the volume, and the free index of the owning
 *     tetrahedron's fourth node (-1 when it is a boundary node);
 *   face_geom [n_faces][4] double: the unit outward normal and 1/h, h the
 *     owning tetrahedron's height over the triangle;
 *   s_ptr [n_free + 1] int64, s_col [s_nnz] int32, s_val [s_nnz] double:
 *     S(free, free) in CSR over free indices, columns ascending,
 *     S_ab = sum over tetrahedra T of |T| grad eta_a . grad eta_b;
 *   b_ptr [n_free + 1] int64, b_col [b_nnz] int32, b_val [b_nnz][3] double:
 *     the load operator in CSR over free rows, columns node indices
 *     ascending (the row's own node left out): b_a = sum over the row's
 *     entries of b_val . (m_col - m_a), = sum over T of |T| grad eta_a .
 *     mean_T(m) for nodal m.
 * Errors: INVALID_ARG, MESH (as slp_potential_create). */
slp_status slp_debug_fem_assemble(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                                  int64_t counts[5], int32_t *node_slot, int32_t *faces, double *face_geom,
                                  int64_t *s_ptr, int32_t *s_col, double *s_val, int64_t *b_ptr, int32_t *b_col,
                                  double *b_val);

#ifdef __cplusplus
}
#endif

#endif /* SLP_DEBUG_H */
