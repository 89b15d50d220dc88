// Internal declarations shared by the host plan code and the CUDA kernels.
// Not part of the public ABI (see include/slp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace slp {

// Work item of the tiled spread (type-1 gridding) and gather (type-2
// interpolation) kernels: a tile of TS^3 grid cells with base cell c0, and a
// contiguous range [begin, end) of sources (spread) or targets (gather)
// whose cells lie inside the tile, in the plan's sorted order.
struct TileItem {
    int c0x, c0y, c0z;
    int begin, end;
    int pad0, pad1, pad2;
};

// Cell groups of the spread: at most SPREAD_GMAX consecutive sources of one
// cell; each item's groups are dealt to SPREAD_WARPS lists.
constexpr int SPREAD_GMAX = 16;
constexpr int SPREAD_WARPS = 8;

// Magnetisation states whose near-field products share one pass over the
// precomputed operator (scratch for sorted m and near-field parts holds this
// many states).
constexpr int NEAR_STATES = 8;
struct StatePtrs {
    const void *in[NEAR_STATES];
};

// Targets per gather item, at most (the plan splits target tiles into items of
// at most GATHER_CHUNK, or of half that when the full size leaves fewer than
// four items per SM; the gather kernel stages one item per block).
constexpr int GATHER_CHUNK = 64;

// Work item of the near-field kernel: up to 32 sorted targets
// [tbegin, tbegin + tcount) and a slice [rbegin, rend) of the range list,
// each range a contiguous run of sorted sources.
struct NearItem {
    int tbegin, tcount;
    int rbegin, rend;
};

// Error codes written to the plan's sticky status word (the first one stays).
enum { DEV_ERR_NONE = 0, DEV_ERR_BAD_ITEM = 1, DEV_ERR_BAD_INDEX = 2, DEV_ERR_NONFINITE = 3 };

// Device-side view of a plan.  Plain data, passed by value to launchers.
struct DevPlan {
    int prec;           // 32 or 64
    int q;              // points per triangle
    int64_t N, Q, M, NV;
    int L[3];           // oversampled grid (x, y, z)
    int n[3];           // modes per axis, L = 2 n
    int Kx;             // stored x frequencies: n_x / 2
    int m;              // window half-width
    int TS, TE;         // source tile cells per axis; tile extent with halo TS + 2m - 1
    int TSg;            // target (gather) tile cells per axis
    double h[3];        // physical grid spacing P_q / L_q
    double beta;        // Kaiser-Bessel shape b * m, b = pi (2 - 1/alpha)
    const void *wcoef;  // FP32 window polynomials: [2m][wdeg + 1], coefficient k of f^k for point i
    int wdeg;
    double inv_sinh_beta;
    double eps2;        // squared near radius (physical)
    double inv_s_sqrt2; // 1 / (sigma_g sqrt 2)
    int kernel_mode;    // SLP_KERNEL_RADIAL or SLP_KERNEL_SEPARABLE
    int deterministic;

    // sources, sorted (k_sorted); grid coordinates: frac (x,y,z) and packed cell
    const void *src_grid;   // T4 [Q]
    const int *src_perm;    // [Q] sorted -> user index k = j*q + s
    const void *src_wn;     // T4 [Q] sorted: w_k n_j (outward unit normal times the weight w_s |S_j|), w_k
    const int4 *src_tri;    // [Q] sorted: user vertex ids of triangle j, user index k
    const void *lam;        // T [q*3] barycentric points of the rule
    // targets, sorted
    const void *tgt_grid;   // T4 [N]
    const int *tgt_perm;    // [N] sorted -> user vertex index

    // scratch (written during evaluation)
    void *qbuf;    // T [Q] weighted charges, sorted order
    void *m4;      // T4 [NEAR_STATES][N] nodal magnetisation in sorted target order (NODAL_MAG input)
    void *gridA;   // T [Lz][Ly][Lx] spread grid (kept zero between evaluations)
    void *gridB;   // T [Lz][Ly][Lx] interpolation grid
    void *S1;      // T2 [Lz][Ly][Kx]
    void *S2;      // T2 [Lz][n_y][Kx]
    void *phi_near; // T [32 * n_near] near-field partials per work item (deterministic mode)
    void *phi_part; // T [NEAR_STATES][N] near-field correction per sorted target, added by the gather
    const void *Dtab;   // T [n_z/2][n_y/2][Kx] kernel multiplier by |l_z|, |l_y|, l_x
    const void *tw[3];  // T2 [L_q] forward twiddles exp(-2 pi i t / L_q)

    // active rows (spread support of the sources and gather support of the
    // targets): planes z0 .. z0 + nz_act - 1 (mod Lz); in plane z the rows
    // plane_iv[z].x .. plane_iv[z].x + plane_iv[z].y - 1 (mod Ly), pair aligned
    int z0, nz_act;
    const int2 *plane_iv;
    const int *row_pairs;  // [n_row_pairs] z * (Ly / 2) + y / 2
    int n_row_pairs;
    int fuse_pb;           // > 0: fused plane passes with this many row pairs per plane (a power of two)
    int yzy_g;             // > 0: fused column passes (FY, FZ * D * IZ, IY in one cluster launch),
                           // G groups of the column engine per CTA
    int yzy_zc, yzy_zp;    // active planes per CTA of a fused-column cluster, and P's row stride

    const TileItem *spread_items; int n_spread;
    int spread_chunk;             // most sources in one spread item
    int spread_dense;             // 1: at least 8 sources per cell group on average (FP32 M <= 4
                                  // spread at 4 blocks per SM with 64 registers, else 5 with 48)
    int gather_chunk;             // most targets in one gather item (<= GATHER_CHUNK)
    const int *sgroups;           // cell groups: first source (within the item) | count << 16
    const int *sgroup_cell;       // local cell of each group in its item's tile: lx | ly << 8 | lz << 16
    // FP64 plans: window values of every sorted source and target, [count][3][2m]
    // (axis-major per point), computed once at plan time by the same device
    // function the kernels would call (NULL: the kernels evaluate the window)
    const double *wtab64_src, *wtab64_tgt;
    const void *wtab;             // FP32 table spread: [Q][3][WP] window values per sorted source (NULL: the
                                  // spread evaluates the window)
    const int *sgroup_off;        // [n_spread][SPREAD_WARPS + 1] group list bounds of each item
    const TileItem *gather_items; int n_gather;
    const NearItem *near_items;   int n_near;
    const int2 *near_ranges;
    int near_chunk;               // deterministic mode: item slot per target block

    // separable kernel: K_n(d) = A prod_q f_q(d_q / L_q), f_q(t) = sum_l hq[l] cos(2 pi l t)
    const void *sep_h[3]; int sep_nh[3];  // hq[0..nh-1], term l uses weight (l==0 ? 1 : 2) * hq[l]
    double sep_A;

    // exp-sum kernel (EXPSUM): N_s(r) = sum_k es_w[k] exp(-es_g[k] r^2) / (4 pi), physical units
    const void *es_w, *es_g;  // T [es_n]
    int es_n;

    // precomputed near-field operator (NODAL_MAG): CSR over sorted targets
    const int64_t *nm_rowptr;  // [N + 1]
    const int *nm_col;         // [nnz] vertex ids
    const void *nm_val;        // T4 [nnz] (wx, wy, wz, unused)
    int64_t nm_nnz;

    // state batch of one launch (grid.y): ks states, scratch of state y at
    // gridA/gridB + y st_grid, S1 + y st_s1, S2 + y st_s2, phi_part + y N;
    // with ks > 1 the spread reads in_st[y] and the gather writes out_st[y]
    int ks;
    int64_t st_grid, st_s1, st_s2;
    const void *in_st[NEAR_STATES];
    void *out_st[NEAR_STATES];

    int *err;  // device status word (sticky)
    int check_finite;  // 1: inputs and results are checked for NaN/Inf (DEV_ERR_NONFINITE)

    // triangle-integrated discretisation (integration = 1)
    int integration;
    const int4 *tri_v;      // [M] user vertex ids of each triangle
    const void *tri_n3;     // T4 [M] outward unit normal / 3
    void *gbuf;             // T [M] element charges of the current input (scratch)
    // gridding matrix A, CSR over the grid points the triangles' boxes reach
    // (deterministic point plans: the point gridding matrix, columns = sorted sources)
    int det_spread;         // 1: the point spread is the sparse product with am_* applied to qbuf
    int64_t am_rows;
    const int64_t *am_rowptr, *am_row;  // [am_rows + 1], [am_rows] grid linear index
    const int *am_col;                  // triangle of each entry
    const void *am_val;                 // T
    // near-field matrix over triangles, CSR over sorted targets
    const int64_t *nt_rowptr;
    const int *nt_col;
    const void *nt_val;
};

// Duffy-Gauss rule of the triangle-integrated plans (8 x 8 points) and the
// largest box of grid points per axis a triangle's window may reach.
constexpr int TRI_RULE = 64;
constexpr int TRI_BOX = 24;

// Plan-time inputs of the gridding-matrix assembly (FP64).
struct TriBuildA {
    const double3 *ugrid;   // [NV] vertex grid coordinates (cells, 0..L)
    const double3 *xphys;   // [NV] vertex physical coordinates (relative to the torus centre)
    const int4 *tri;        // [M] vertex ids
    int64_t M, NV;
    int m, L[3];
    double beta, isb;
    const double *ra, *rb, *rw;  // rule on the reference triangle {0 <= b <= a <= 1}, weights summing to 1/2
    int np;
    int *err;
};
// Plan-time inputs of the near-field matrix over triangles (FP64).
struct TriBuildN {
    const double3 *tgt;      // [N] sorted targets, physical, relative to the centre
    const int *tgt_perm;     // [N] sorted -> user vertex
    const int *tgt_block;    // [N] target block of each sorted target
    const int *blk_r0;       // [nblk + 1]
    const int2 *ranges;      // candidate vertex ranges (sorted target order)
    const int *vt_ptr, *vt_ent;  // vertex -> adjacent (triangle * 4 + corner)
    const int *tri_min_sorted;   // [M] smallest sorted index among the triangle's vertices
    const double3 *xphys;    // [NV] vertex physical coordinates (relative to the centre)
    const int4 *tri;         // [M]
    int64_t N;
    double eps;
    int kernel_mode;
    double inv_s_sqrt2;
    const double *es_w, *es_g;
    int es_n;
    const double *sep_h[3];
    int sep_nh[3];
    double sep_A4pi;
    double P[3];
    const double *ra, *rb, *rw;
    int np;
    int *err;
};
// Plan-time inputs of the point gridding matrix of deterministic plans (FP64).
struct PointBuild {
    const double4 *src;  // [Q] sorted sources: fractional grid coordinate (x, y, z) and packed cell (w)
    int64_t Q;
    int m, L[3];
    double beta, isb;
    int *err;
};
cudaError_t launch_pmat_count(const PointBuild &b, int *cnt, cudaStream_t s);
cudaError_t launch_pmat_fill(const PointBuild &b, int prec, const int *slot_of, const int64_t *rowptr, int *cursor,
                             int *col, void *val, cudaStream_t s);
cudaError_t launch_amat_count(const TriBuildA &b, int *cnt, cudaStream_t s);
cudaError_t launch_amat_fill(const TriBuildA &b, int prec, const int *slot_of, const int64_t *rowptr, int *cursor,
                             int *col, void *val, cudaStream_t s);
cudaError_t launch_csr_sort(int64_t nrows, int prec, const int64_t *rowptr, int *col, void *val, cudaStream_t s);
cudaError_t launch_nmt_build(const TriBuildN &b, int pass, int prec, int64_t *counts, const int64_t *rowptr,
                             int *col, void *val, cudaStream_t s);
// element charges of NODAL_MAG input into gbuf
cudaError_t launch_p0_charges(const DevPlan &p, const void *d_in, cudaStream_t s);
// y[row_idx ? row_idx[i] : i] = sum over CSR row i of val * x[col]
cudaError_t launch_csr_apply(int prec, int lanes_per_row, int64_t nrows, const int64_t *rowptr, const int64_t *row_idx,
                             const int *col, const void *val, const void *x, void *y, cudaStream_t s);

// Kernel launchers (return the launch error, if any).
cudaError_t launch_nodal_prep(const DevPlan &p, const void *d_in, cudaStream_t s);
cudaError_t launch_charges(const DevPlan &p, int kind, const void *d_in, cudaStream_t s);
// fused_kind >= 0: compute the charges of that input kind inside the spread (no qbuf)
cudaError_t launch_spread(const DevPlan &p, int fused_kind, const void *d_in, cudaStream_t s);
cudaError_t launch_fft_forward_x(const DevPlan &p, cudaStream_t s);
cudaError_t launch_fft_forward_y(const DevPlan &p, cudaStream_t s);
cudaError_t launch_fft_z_multiply(const DevPlan &p, cudaStream_t s);
cudaError_t launch_fft_inverse_y(const DevPlan &p, cudaStream_t s);
cudaError_t launch_fft_inverse_x(const DevPlan &p, cudaStream_t s);
// fused column passes (FY, FZ * D * IZ, IY of one stored x frequency per
// cluster of YZY_CL CTAs; yzy_g > 0)
constexpr int YZY_CL = 4;
cudaError_t launch_fft_yzy(const DevPlan &p, cudaStream_t s);
size_t fused_column_smem(const DevPlan &p, int G, int ZP);
// fused plane passes (FX + FY, IY + IX; one block per active plane, fuse_pb > 0)
cudaError_t launch_fft_forward_xy(const DevPlan &p, cudaStream_t s);
cudaError_t launch_fft_inverse_yx(const DevPlan &p, cudaStream_t s);
// shared memory of the fused plane passes with PB row pairs per plane
size_t fused_plane_smem(const DevPlan &p, int PB);
// phi[perm[t]] = far field at t + phi_part[t]
cudaError_t launch_gather(const DevPlan &p, void *d_phi, cudaStream_t s);
// FP32 table spread: floats per source row of the window table (3 x 2m padded
// to a multiple of 4) and its plan-time build into `out` ([Q] rows)
int spread_table_row(int m);
cudaError_t launch_wtab_build(const DevPlan &p, float *out, cudaStream_t s);
// FP64 window values of n sorted points (sources or targets, grid coordinates
// in pts) into out ([n][3][2m])
cudaError_t launch_wtab64_build(const DevPlan &p, const void *pts, int64_t n, double *out, cudaStream_t s);
// near field into phi_part (atomics: phi_part must be zero; deterministic: per-item partials, then the reduction
// overwrites phi_part)
cudaError_t launch_near(const DevPlan &p, cudaStream_t s);
cudaError_t launch_near_reduce(const DevPlan &p, const int *blk_first, int nblk, cudaStream_t s);
cudaError_t launch_zero(void *ptr, size_t bytes, cudaStream_t s);

// Precomputed near-field operator (k_near.cu): inputs of the plan-time
// assembly of W (FP64, temporary device arrays).
struct NMBuild {
    const double4 *tgt;      // [N] sorted targets, physical coordinates relative to the torus centre
    const int *tgt_perm;     // [N] sorted -> user vertex
    const int *tgt_block;    // [N] target block of each sorted target
    const int *blk_r0;       // [nblk + 1] range list of each block
    const int2 *ranges;      // candidate vertex ranges (sorted target order)
    const int *vt_ptr;       // [NV + 1] vertex -> adjacency entries
    const int *vt_ent;       // triangle * 4 + local vertex index
    const double4 *src;      // [Q] user-order quadrature points (x, y, z relative to the centre, w_k)
    const double4 *nrm;      // [M] outward unit normals
    const double *lam;       // [q * 3]
    int q;
    int64_t N;
    double eps2;
    double inv_s_sqrt2;
    int kernel_mode;
    const double *sep_h[3];
    int sep_nh[3];
    double sep_A4pi;         // 4 pi A
    double P[3];
    const double *es_w, *es_g;  // EXPSUM terms, physical units
    int es_n;
};
cudaError_t launch_nm_build(const NMBuild &b, int pass, int prec, int64_t *counts, int64_t *pairs,
                            const int64_t *rowptr, void *val, cudaStream_t s);
// phi_part = W m (overwrites)
cudaError_t launch_near_matrix(const DevPlan &p, const void *d_m, cudaStream_t s);
// K <= NEAR_STATES states at once: m4[k][.] from in[k] (sorted), then
// phi_part[k][.] = W m_k with one pass over W
cudaError_t launch_nodal_prep_states(const DevPlan &p, const StatePtrs &in, int K, cudaStream_t s);
cudaError_t launch_near_matrix_states(const DevPlan &p, int K, cudaStream_t s);

// Set the thread-local text returned by slp_last_error().
void set_last_error(const char *msg);

}  // namespace slp
