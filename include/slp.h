/*
 * slp.h — C ABI of the GB300 single-layer-potential library.
 *
 * The library evaluates the single layer potential of a surface charge at
 * the boundary nodes of a closed triangle mesh,
 *
 *     phi_i = sum_j sum_s w_s |S_j| sigma_{j,s} / (4 pi |x_i - y_{j,s}|),
 *
 * (Exl & Schrefl, "Non-uniform FFT for the finite element computation of the
 * micromagnetic scalar potential": the discretised single layer potential of
 * Sec. 2.2 with the triangle quadrature of the quadrature form in Sec. 3),
 * by splitting the kernel into a smooth part applied through a non-uniform
 * FFT (spread -> FFT -> multiply -> inverse FFT -> gather, the generalised
 * convolution theorem of Sec. 2.2 and Sec. 5) and a short-range near-field
 * correction (Sec. 3.4).
 *
 * Conventions shared by every entry point:
 *   - every call returns an slp_status; nothing throws across the ABI;
 *   - slp_last_error() returns a thread-local text for the last failure;
 *   - "device" pointers live on the plan's CUDA device; "host" pointers are
 *     ordinary (ideally page-locked) CPU memory;
 *   - the arithmetic type of inputs and outputs is the plan's precision:
 *     float for precision 32, double for precision 64;
 *   - quadrature sources are numbered k = j * q + s (triangle j, rule point s,
 *     the point order of slp_quadrature below); targets are the mesh vertices
 *     in the caller's order.
 */
#ifndef SLP_H
#define SLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slp_plan_s *slp_plan_t;

typedef enum {
    SLP_OK = 0,
    SLP_ERR_INVALID_ARG = 1,          /* null pointer, bad size, unknown enum value */
    SLP_ERR_MESH = 2,                 /* index out of range, degenerate triangle, open or
                                         inconsistently oriented surface, inward normals */
    SLP_ERR_TOLERANCE_INFEASIBLE = 3, /* the forced grid cannot meet the tolerance */
    SLP_ERR_OOM = 4,                  /* device allocation failed */
    SLP_ERR_CUDA = 5,                 /* a CUDA runtime call failed */
    SLP_ERR_TIMEOUT = 6,              /* a bounded device-side wait gave up */
    SLP_ERR_NONFINITE = 7,            /* checked evaluation saw NaN/Inf */
    SLP_ERR_NO_DEVICE = 8,            /* plan built host-only, or no CUDA device */
    SLP_ERR_UNSUPPORTED = 9           /* option combination not implemented */
} slp_status;

/* Triangle rules (barycentric points, weights summing to 1):
 *   SLP_QUAD_1: centroid;
 *   SLP_QUAD_3: (2/3,1/6,1/6) and cyclic shifts, weights 1/3 (degree 2, interior);
 *   SLP_QUAD_7: Radon's degree-5 rule: centroid 9/40; (a,a,1-2a),(a,1-2a,a),(1-2a,a,a)
 *               for a = (6-sqrt15)/21 [weight (155-sqrt15)/1200], then the same three
 *               for a = (6+sqrt15)/21 [weight (155+sqrt15)/1200]. */
enum { SLP_QUAD_1 = 1, SLP_QUAD_3 = 3, SLP_QUAD_7 = 7 };

/* Input kinds of slp_eval:
 *   SIGMA:     sigma at the quadrature points, [Q] (Q = q * n_triangles);
 *   MAG:       m at the quadrature points, [Q][3]; sigma = m . n_j;
 *   NODAL_MAG: m at the mesh vertices, [N][3]; interpolated linearly on each
 *              triangle (P1, Sec. 2.1) to the points; sigma = m(y) . n_j;
 *              in plans with opts.integration = 1 it is projected onto
 *              element-wise constants instead: g_j = (1/|S_j|) int_{S_j} m . n_j
 *              (the L2 projection of Sec. 2.2);
 *   ELEMENT:   element-wise constant charge g_j per triangle, [n_triangles]
 *              (plans with opts.integration = 1 only; SIGMA and MAG need the
 *              quadrature points and are refused there with
 *              SLP_ERR_UNSUPPORTED). */
enum { SLP_INPUT_SIGMA = 0, SLP_INPUT_MAG = 1, SLP_INPUT_NODAL_MAG = 2, SLP_INPUT_ELEMENT = 3 };

/* Smooth-kernel choice (the splitting N = (N - N_s) + N_s of Sec. 2.2):
 *   RADIAL:    N_s = (N truncated at radius R) convolved with an isotropic
 *              Gaussian; near-field kernel erfc(r/(s sqrt2))/(4 pi r) inside eps;
 *   SEPARABLE: N_s = a separable band-limited periodic kernel; every pair is
 *              near and the near kernel is N - N_s evaluated exactly
 *              (for grids too small to resolve RADIAL at the tolerance);
 *   EXPSUM:    the paper's kernel (Sec. 3.3): the body scaled into
 *              (-0.2, 0.2)^3 of a cubic torus of period P (the scaling of the
 *              paper's experiments), 1/r approximated on [eps, P/2] by a sum of
 *              Gaussians sum_k w_k exp(-g_k r^2) truncated to the S' widest
 *              terms that the grid resolves, Fourier coefficients of each
 *              Gaussian integrated over one period per axis (separable,
 *              S' (n_x + n_y + n_z)/2 numbers), near-field kernel
 *              (1/r - sum_k w_k exp(-g_k r^2)) / (4 pi) inside eps.  Its
 *              accuracy is the paper's: the truncated periodic extension of
 *              the widest Gaussians limits it to about 1e-3 relative, so it
 *              is chosen only explicitly;
 *   AUTO:      RADIAL when feasible on the grid, else SEPARABLE for small
 *              meshes at precision 64, else a raised grid (when allowed). */
enum { SLP_KERNEL_AUTO = 0, SLP_KERNEL_RADIAL = 1, SLP_KERNEL_SEPARABLE = 2, SLP_KERNEL_EXPSUM = 3 };

/* Near-field evaluation:
 *   ON_THE_FLY:  kernel values computed per pair in every evaluation;
 *   PRECOMPUTED: for NODAL_MAG input, the near-field operator is assembled
 *                once at plan time as a sparse target-by-vertex matrix
 *                (the precomputed near-field integrals of Sec. 3.4) and
 *                applied as a sparse product; other inputs fall back to
 *                ON_THE_FLY;
 *   AUTO:        PRECOMPUTED when the operator needs at most 24 GiB and at
 *                most half of the free device memory. */
enum { SLP_NEAR_AUTO = 0, SLP_NEAR_ON_THE_FLY = 1, SLP_NEAR_PRECOMPUTED = 2 };

typedef struct {
    const double *vertices;   /* host, [n_vertices][3], read during slp_plan only */
    int64_t n_vertices;
    const int32_t *triangles; /* host, [n_triangles][3], outward (counter-clockwise) winding */
    int64_t n_triangles;
} slp_mesh;

typedef struct {
    int precision;        /* 32 (FP32 spread/FFT/gather/near field) or 64 */
    int grid[3];          /* oversampled FFT grid per axis (power of two, 8..1024); 0 = auto */
    int m;                /* Kaiser-Bessel half-width in grid cells; 0 = from the tolerance */
    int kernel_mode;      /* SLP_KERNEL_* */
    int near_mode;        /* SLP_NEAR_* */
    int deterministic;    /* 1: every sum in a fixed order, so an evaluation repeats bitwise whatever
                             runs beside it: the near field per work item in item order, and the spread
                             as a product with a precomputed point gridding matrix (entry (r, k) the
                             window product of source k at grid point r, 8 bytes per entry, (2m)^3
                             entries per source, rows in ascending source order) in place of the
                             tiled spread's atomics; the matrix is built when it needs at most 24 GiB
                             and half of the free memory (slp_info.deterministic_spread), else the
                             spread keeps its atomics and results repeat to rounding level.  Plans
                             with opts.integration are deterministic in either setting */
    int device;           /* CUDA device ordinal; -1 builds a host-only plan (slp_query works,
                             slp_eval returns SLP_ERR_NO_DEVICE) */
    int allow_grid_raise; /* 1: raise a grid that cannot meet the tolerance (else error) */
    int check_mesh;       /* 1: require a closed, consistently and outward oriented surface */
    int fuse_plane_passes; /* x and y FFT passes fused per z plane (a cluster of four CTAs per
                              plane, the plane spectrum in distributed shared memory): 0 off, 1 on
                              where the plane fits, -1 automatic (on when there are at least two
                              active planes per SM) */
    int fuse_column_passes; /* the y pass, the z pass with the kernel multiply and the inverse y pass
                               fused, one cluster of four CTAs per stored x frequency holding that
                               slab of the spectrum in distributed shared memory (needs equal y and
                               z grids of 32..256 and unfused plane passes): 0 off, 1 on where it
                               applies, -1 automatic (off: the separate passes, chained by
                               programmatic dependent launch, measured faster) */
    int check_finite;     /* 1: every evaluation checks its input and its result for NaN/Inf on the
                             device, in kernels that read them anyway; a non-finite value sets the
                             plan's status word, which slp_check then reports as SLP_ERR_NONFINITE
                             (the evaluation still completes; nothing traps) */
    int integration;      /* 0: point quadrature (the quadrature form of Sec. 3: sources at the rule's
                             points, the oracle's definition); 1: triangle integrals (Sec. 2.2,
                             Eq. (slayer3) with element-wise constant charges g_j): the gridding
                             matrix A_rj = int_{S_j} Psi(r - y) dA of Sec. 3.1 assembled once per plan
                             (8 x 8 Duffy-Gauss rule per triangle) and applied as a sparse product,
                             and the near-field integrals of Sec. 3.4 computed exactly (closed form of
                             the 1/r part, which covers the weakly singular case) and applied as a
                             second sparse product.  Grids of at most 2^27 points and triangles up to
                             24 - 2m grid cells across; otherwise SLP_ERR_UNSUPPORTED */
    int spread_table;     /* FP32 spread with m <= 4: 1 reads each source's window values from a
                             plan-time table (3 x 2m floats per source, 96 bytes at m = 4) instead
                             of evaluating the window per group; 0 or -1 (automatic) evaluates them.
                             Alone the table spread is 7-13 % faster, but its streamed table loads
                             wait behind a concurrent near-field product that saturates HBM (the
                             2000 x 500 x 20 plate: 1.28 against 0.91 ms per evaluation), so only
                             the autotuner, which times both, turns it on */
    int gather_item_targets;  /* most targets per gather work item: 32 or 64; 0 automatic (64, or 32 when
                                 items of 64 would give fewer than four per SM) */
    int spread_blocks;        /* FP32 spread with m <= 4: register budget for 4 or 5 blocks per SM; 0
                                 automatic (4 where cell groups hold >= 8 sources on average, else 5) */
} slp_plan_opts;

typedef struct {
    int64_t n_targets;       /* N, mesh vertices */
    int64_t n_sources;       /* Q = q * n_triangles */
    int64_t n_triangles;
    int quadrature;
    int precision;
    int grid[3];             /* oversampled grid used (alpha n, alpha = 2) */
    int modes[3];            /* n per axis */
    int m;                   /* window half-width */
    int kernel_mode;         /* resolved SLP_KERNEL_* */
    int near_mode;           /* resolved SLP_NEAR_* for NODAL_MAG input */
    int grid_raised;         /* 1 if the requested grid was raised */
    double center[3];        /* torus centre */
    double period[3];        /* torus period per axis (physical units) */
    double sigma_g;          /* Gaussian smoothing width (RADIAL) */
    double trunc_radius;     /* truncation radius R (RADIAL) */
    double eps_near;         /* near-field radius (infinite for SEPARABLE) */
    double tolerance;
    int64_t near_pairs;          /* (target, source) pairs visited per on-the-fly evaluation */
    int64_t near_pairs_within;   /* of those, pairs closer than eps_near */
    int64_t near_matrix_nnz;     /* (target, vertex) entries of the precomputed operator */
    int64_t bytes_device;        /* device memory held by the plan */
    int64_t n_spread_items;
    int64_t n_gather_items;
    int64_t n_near_items;
    int launches_per_eval;       /* kernels launched by one slp_eval */
    int64_t active_rows;         /* grid rows (z, y) the FFT passes transform along x: those within
                                    the window of some source or target, widened to row pairs */
    int active_planes;           /* z planes the FFT passes along y work on */
    int fused_plane_passes;      /* 1: the x and y passes run fused, one four-CTA cluster per active
                                    plane */
    int fused_column_passes;     /* 1: FY, FZ * D * IZ and IY run as one cluster launch */
    int gather_item_targets;     /* most targets in one gather work item (64, or 32 when items of 64
                                    would give fewer than four per SM) */
    int spread_blocks_per_sm;    /* FP32 spread with m <= 4: the register budget's blocks per SM, 4
                                    where cell groups hold >= 8 sources on average, else 5; 0 for
                                    the other spread kernels */
    int spread_table;            /* 1: the spread reads plan-time window tables (opts.spread_table) */
    int expsum_terms;            /* EXPSUM: Gaussians kept in the smooth kernel (S'); 0 otherwise */
    int integration;             /* opts.integration of the plan */
    int64_t grid_matrix_nnz;     /* integration = 1: entries of the gridding matrix A */
    int64_t grid_matrix_rows;    /* integration = 1: grid points A reaches (its rows) */
    int64_t near_tri_nnz;        /* integration = 1: (target, triangle) entries of the near-field matrix */
    int deterministic_spread;    /* 1: deterministic point plan whose spread is the precomputed point gridding
                                    matrix (then grid_matrix_nnz/rows describe that matrix) */
} slp_info;

/* Fill opts with defaults: precision 32, automatic grid/m/kernel/near mode,
 * device 0, grid raise allowed, mesh checks on. */
slp_status slp_default_opts(slp_plan_opts *opts);

/* Build a plan (the setup phase of Alg. 1: geometry-only precomputation).
 * mesh:       host arrays, only read during the call;
 * quadrature: SLP_QUAD_1/3/7;
 * tolerance:  target relative L2 error of phi against the exact quadrature sum
 *             (drives m, the smoothing width and the near radius);
 * opts:       may be NULL (defaults);
 * out:        receives the plan; release with slp_destroy.
 * Allocates all device memory the plan will use; evaluation allocates nothing.
 * Errors: INVALID_ARG, MESH, TOLERANCE_INFEASIBLE, OOM, CUDA, NO_DEVICE. */
slp_status slp_plan(const slp_mesh *mesh, int quadrature, double tolerance,
                    const slp_plan_opts *opts, slp_plan_t *out);

/* Evaluate phi at the mesh vertices (the computation phase of Alg. 1:
 * spread, FFT, kernel multiply, inverse FFT, gather, near-field correction).
 * d_in:   device, layout per input_kind (SLP_INPUT_*), plan precision;
 * d_phi:  device, [n_targets], plan precision, overwritten;
 * stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 * Stream-ordered: returns after enqueueing.  Calls on one plan must not
 * overlap in time on different streams (they share the plan's scratch).
 * Errors: INVALID_ARG, NO_DEVICE, CUDA. */
slp_status slp_eval(slp_plan_t plan, int input_kind, const void *d_in, void *d_phi, void *stream);

/* Evaluate n_states inputs of one plan in one call: d_in holds the states
 * back to back (each in the layout of input_kind), d_phi receives
 * [n_states][n_targets].  For nodal input with the precomputed near field,
 * up to 8 states share one pass over the near-field operator (the operator is
 * read once per 8 states instead of once per state); each result equals that
 * of slp_eval on the same state.  Stream-ordered; same rules as slp_eval.
 * Errors: INVALID_ARG, NO_DEVICE, CUDA. */
slp_status slp_eval_states(slp_plan_t plan, int input_kind, int n_states, const void *d_in, void *d_phi,
                           void *stream);

/* Same as slp_eval with host buffers: copies h_in to the plan's staging
 * buffer, evaluates, copies phi back to h_phi and synchronises the stream.
 * Page-locked host memory gives asynchronous copies. */
slp_status slp_eval_host(slp_plan_t plan, int input_kind, const void *h_in, void *h_phi, void *stream);

/* ---- Evaluation at other points (probes) ----
 * The paper evaluates phi_2 at every finite-element node, the interior ones
 * included (Sec. 2.1, Alg. 1).  A probe set attaches such points to a plan:
 * they are sorted into the plan's grid cells and get their own gather work
 * list and rows of the near-field operator (the vertex operator of a plan
 * with the precomputed near field, or the triangle operator of a plan with
 * opts.integration = 1).  points: host [n][3], read during the call.  Each
 * point must lie in the mesh's bounding box (the period isolates that box
 * from its images) and in the ball about the box centre through the
 * farthest vertex (within it every source is nearer than the smooth
 * kernel's truncation radius), else SLP_ERR_INVALID_ARG; and its window
 * must fall on grid rows the pruned transforms compute (rows that some
 * vertex or source window reaches; the interior of a closed mesh always
 * does), else SLP_ERR_UNSUPPORTED.
 * slp_eval_probe runs slp_eval on the mesh vertices (d_phi, [n_targets])
 * and then, on the same stream, the probes' near-field product and window
 * interpolation from the same interpolation grid (d_phi_points, [n]).  It
 * takes NODAL_MAG input, or ELEMENT in plans with triangle integrals.
 * Errors: INVALID_ARG, NO_DEVICE, UNSUPPORTED (a point plan without the
 * precomputed near field, or a point off the computed rows), OOM, CUDA. */
typedef struct slp_probe_s *slp_probe_t;
slp_status slp_probe_create(slp_plan_t plan, const double *points, int64_t n_points, slp_probe_t *out);
slp_status slp_eval_probe(slp_plan_t plan, slp_probe_t probe, int input_kind, const void *d_in, void *d_phi,
                          void *d_phi_points, void *stream);
/* Points and near-field operator entries of the probe set. */
slp_status slp_probe_query(slp_probe_t probe, int64_t *n_points, int64_t *near_nnz);
/* Release a probe set (before its plan).  NULL is accepted. */
slp_status slp_probe_destroy(slp_probe_t probe);

/* ---- The scalar potential phi = phi_1 + phi_2 on a tetrahedral mesh (Alg. 1) ----
 * The split of Sec. 2.1: phi_1 solves the Dirichlet problem of Sec. 2.1
 * (P1 elements, zero on the boundary, only the free (non-boundary) nodes are
 * unknowns) and phi_2 is the single layer potential of
 * g = m.n - d phi_1/dn on the boundary, at every node.
 * Setup (slp_potential_create): the boundary (faces of one tetrahedron only,
 * wound away from its fourth node), the free-node stiffness matrix and the
 * load operator b = B m of Sec. 2.1 (host FP64), the boundary's
 * triangle-integrated plan (opts.integration is set; Sec. 3) and a probe set
 * of the free nodes.
 * Computation (slp_potential_eval): b = B m (in the plan's precision);
 * phi_1 by iterative refinement on the device: Jacobi-preconditioned
 * conjugate gradients in FP32 cut the residual of the current correction
 * equation by 1e-4, the correction joins the FP64 solution and the residual
 * b - S x is recomputed in FP64, until |b - S x| <= cg_tolerance |b|;
 * g_j = (mean of m over boundary triangle j) . n_j + phi_1(o) / h_j, o the
 * owning tetrahedron's fourth node and h_j its height over the triangle
 * (d phi_1/dn = -phi_1(o)/h_j, phi_1 being zero on the triangle); phi_2 at
 * the boundary nodes (the plan's targets) and the free nodes (its probes);
 * phi = phi_1 + phi_2.
 * nodes: host [n_nodes][3]; tets: host [n_tets][4], either orientation, read
 * during the call; every node in some tetrahedron, every face in at most two,
 * the boundary closed as slp_plan requires (it may have several components,
 * as a shell's two spheres).  tolerance, opts: as for slp_plan
 * (opts->device must be a device), except that an automatic grid (all three
 * entries 0) is sized for the boundary and free nodes together: per axis the
 * power of two nearest 3.0 ((n_boundary + n_free) F)^(1/5) times the axis'
 * share of the period, F the boundary triangles (for L cells per axis the
 * grid work grows as L^3 and the exact near field as
 * (n_boundary + n_free) F / L^2), halved while a triangle spans more cells
 * than the plan's triangle integrals allow.  cg_tolerance: 0 picks
 * tolerance / 100 (at least 1e-14); cg_max_iterations (FP32 steps in all):
 * 0 picks 10000.
 * Errors: INVALID_ARG, MESH, TOLERANCE_INFEASIBLE, OOM, CUDA, NO_DEVICE. */
typedef struct slp_potential_s *slp_potential_t;
typedef struct {
    int64_t n_nodes, n_tets;
    int64_t n_free;            /* unknowns of phi_1 */
    int64_t n_boundary;        /* boundary nodes: the plan's targets */
    int64_t n_faces;           /* boundary triangles */
    int64_t stiffness_nnz;     /* entries of S(free, free) */
    int64_t load_nnz;          /* entries of the load operator */
    int64_t cg_iterations;     /* FP32 steps of the last evaluation (-1 before the first) */
    int64_t cg_corrections;    /* its FP64 residual corrections */
    int64_t cg_max_iterations;
    double cg_residual;        /* |b - S x| / |b| after the last evaluation */
    double cg_tolerance;
    double ms_phi1;            /* device time of the last evaluation's load and solve (-1: not finished) */
    double ms_phi2;            /* ... of its charges, single layer potential and sum */
    slp_plan_t surface_plan;   /* the boundary's plan, owned by the potential (query only) */
} slp_potential_info;
slp_status slp_potential_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                                double tolerance, const slp_plan_opts *opts, double cg_tolerance,
                                int cg_max_iterations, slp_potential_t *out);
/* d_m: device [n_nodes][3] (plan precision), the nodal magnetisation;
 * d_phi: device [n_nodes], overwritten with phi; d_phi_1: NULL or device
 * [n_nodes], overwritten with phi_1.  Enqueued on `stream`: the load, the
 * solve (one graph whose loops over corrections and inner steps run on the
 * device until the solve stops), phi_2 and the sum.  The call then waits
 * for the solve, not for phi_2, to return its status, so it cannot be
 * captured into a CUDA graph.  Errors: INVALID_ARG, CUDA, NONFINITE (the iteration met
 * NaN/Inf), TOLERANCE_INFEASIBLE (cg_max_iterations reached: phi is still
 * written, from the last iterate). */
slp_status slp_potential_eval(slp_potential_t pot, const void *d_m, void *d_phi, void *d_phi_1, void *stream);
slp_status slp_potential_query(slp_potential_t pot, slp_potential_info *info);
/* Release the potential with its plan and probe set.  NULL is accepted. */
slp_status slp_potential_destroy(slp_potential_t pot);

/* Pipelined host-buffer evaluation: enqueues, without waiting, the copy of
 * h_in into one of the plan's two staging slots (on an internal copy-in
 * stream), the evaluation (on `stream`) and the copy of phi into h_phi (on
 * an internal copy-out stream), alternating slots, so that the copy-in of the
 * next call and the copy-out of the previous one overlap this evaluation.
 * h_in must stay unchanged and h_phi unread until slp_eval_host_wait returns;
 * page-locked memory keeps the copies asynchronous.  Calls on one plan come
 * from one host thread; the staging slots are allocated with the plan.
 * Errors: INVALID_ARG, NO_DEVICE, UNSUPPORTED, CUDA. */
slp_status slp_eval_host_async(slp_plan_t plan, int input_kind, const void *h_in, void *h_phi, void *stream);

/* Blocks until the results of every earlier slp_eval_host_async call on the
 * plan are in host memory. */
slp_status slp_eval_host_wait(slp_plan_t plan);

/* Allocation-free evaluation for callers that cannot call cudaMalloc where
 * they need phi: host code running inside another framework's memory pool,
 * which forbids raw device allocations, and solver loops that must not touch
 * the allocator after start-up.  Such callers cannot build a plan (slp_plan
 * allocates).  The paper has no counterpart: this evaluates the same
 * quantity as slp_eval, phi at the mesh vertices, by direct summation over
 * all (vertex, quadrature point) pairs, without a plan.
 * d_vertices:  device, [n_vertices][3] double;  d_triangles: device, [n_triangles][3]
 *              int32, outward winding (indices are bounds-checked: a triangle with
 *              an index out of range carries no charge);
 * quadrature:  SLP_QUAD_1/3/7;  precision: 32 or 64 (type of d_in and d_phi);
 * input_kind:  SLP_INPUT_* with the layouts of slp_eval;
 * d_phi:       device, [n_vertices], overwritten;  stream: cudaStream_t or NULL.
 * Scratch: one 32 MiB static device array inside the library (held by every
 * GPU that loads it, until exit): at most 2,097,152 sources (q * n_triangles)
 * at precision 32, 1,048,576 at precision 64; larger meshes return
 * SLP_ERR_INVALID_ARG with the sizes in slp_last_error().  Nothing in the
 * array needs to start at zero.  All calls share the array, so calls that
 * overlap on the GPU (other streams, other host threads) race: order them.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Sums are compensated (Neumaier), so the FP32
 * result stays within about 1e-6 relative of the exact quadrature sum up to
 * the source limit.  A CUDA error pending from the caller's earlier work is
 * reported (SLP_ERR_CUDA) and left in place, and nothing is launched.
 * Costs O(N Q): meant for small meshes. */
slp_status slp_eval_direct_static(const double *d_vertices, int64_t n_vertices, const int32_t *d_triangles,
                                  int64_t n_triangles, int quadrature, int precision, int input_kind,
                                  const void *d_in, void *d_phi, void *stream);

/* ---- Batched evaluation (many states, many meshes, one CUDA graph) ----
 * An item evaluates plans[plan_of[i]] on d_in[i] -> d_phi[i] (device buffers
 * with the layouts of slp_eval; they must stay valid and fixed for the life of
 * the batch: the caller refills d_in and reads d_phi between runs).
 * lanes_per_plan (1..64) scratch sets per plan run that plan's items
 * concurrently on separate streams (lane 0 is the plan's own scratch, the
 * others are allocated here); items are dealt round-robin to the lanes.  A
 * lane evaluates its items as slp_eval_states does (shared near-field passes,
 * state-batched far field), so one lane per plan is usually the fastest and
 * needs no extra scratch.
 * slp_batch_create captures every item into one CUDA graph (fork/join over
 * the lanes); slp_batch_run launches it on `stream`.  All plans must share a
 * device.  A plan must not be evaluated elsewhere while a batch that uses it
 * runs (lane 0 shares the plan's scratch). */
typedef struct slp_batch_s *slp_batch_t;
slp_status slp_batch_create(int n_plans, const slp_plan_t *plans, int n_items, const int *plan_of, int input_kind,
                            const void *const *d_in, void *const *d_phi, int lanes_per_plan, slp_batch_t *out);
slp_status slp_batch_run(slp_batch_t batch, void *stream);
slp_status slp_batch_query(slp_batch_t batch, int64_t *n_items, int64_t *n_lanes, int64_t *kernel_launches,
                           int64_t *extra_scratch_bytes);
slp_status slp_batch_destroy(slp_batch_t batch);

/* One-call batched evaluation (the batched form as a single entry point):
 * plans[i] evaluates n_states_each[i] states, held back to back in d_in[i]
 * (device, each state in the slp_eval layout of input_kind), into d_phi[i]
 * (device, [n_states_each[i]][n_targets of plans[i]]).  A plan may appear in
 * several entries.  Every state of every entry runs in one CUDA graph
 * launched on `stream` (the states of one plan share the near-field passes
 * and the state-batched far field, as in slp_eval_states; different plans
 * overlap on the device).  The first call with a given argument set (plans,
 * buffers, counts, input kind) captures that graph; later calls with the
 * same set replay it, so buffers that are refilled in place between calls
 * cost no capture.  The library keeps up to 8 such graphs (least recently
 * used dropped first); slp_destroy releases those that use the plan.  The
 * plans must not be evaluated on other streams while a call runs (the graph
 * uses each plan's own scratch).  Stream-ordered.
 * Errors: INVALID_ARG, NO_DEVICE, OOM, CUDA. */
slp_status slp_eval_batched(int n, const slp_plan_t *plans, int input_kind, const void *const *d_in,
                            void *const *d_phi, const int *n_states_each, void *stream);

/* ---- Autotuner ----
 * Grid: considers equal-spacing grids whose largest axis spans 32, 64, ...,
 * 512 cells (powers of two per axis), drops grids that cannot meet the
 * tolerance (allow_grid_raise is forced off), ranks the rest by a cost model
 * from host-only plans (grid points, near-field pairs, sources), builds the
 * two cheapest on the opts' device and times `reps` evaluations of each with
 * nodal input.  Then, from the faster one, one knob at a time (coordinate
 * descent): the spread's window source (table or evaluated) and register
 * budget (4 or 5 blocks per SM), the gather item size (32 or 64 targets) and
 * the FFT pass arrangement (separate, fused plane passes, fused column
 * passes), each alternative built and timed, and kept when faster than the
 * incumbent by more than 1 %.  Knobs the plan does not use (FP64, wide
 * windows) are skipped.  Returns the fastest plan in *out; info (may be NULL)
 * receives every timed candidate's settings and mean milliseconds and the
 * index chosen.  Options other than the tuned ones apply to every
 * candidate. */
#define SLP_TUNE_MAX 16
typedef struct {
    int n_candidates;
    int chosen;
    int grid[SLP_TUNE_MAX][3];
    double ms[SLP_TUNE_MAX];
    int kernel_mode[SLP_TUNE_MAX];
    int spread_table[SLP_TUNE_MAX];         /* 1: window tables */
    int spread_blocks[SLP_TUNE_MAX];        /* 4 or 5; 0 when the spread has no such build */
    int gather_item_targets[SLP_TUNE_MAX];
    int fft_passes[SLP_TUNE_MAX];           /* 0 separate, 1 fused plane passes, 2 fused column passes */
} slp_tune_info;
slp_status slp_plan_autotune(const slp_mesh *mesh, int quadrature, double tolerance, const slp_plan_opts *opts,
                             int reps, slp_plan_t *out, slp_tune_info *info);

/* ---- Serving: continuous batching of requests on resident plans ----
 * A server keeps the given plans resident, gives each plan slots_per_plan
 * execution slots (a CUDA stream and a scratch set each; slot 0 uses the
 * plan's own scratch) and allocates one device arena for request buffers:
 * hbm_budget_bytes minus the extra slot scratch.  slp_server_submit queues a
 * request of n_states inputs for one plan (host buffers: n_states
 * consecutive inputs with the slp_eval layout of input_kind, and n_states
 * consecutive outputs of n_targets values; page-locked memory keeps the
 * copies asynchronous; both must stay valid until the request finishes).  A
 * scheduler thread admits queued requests in arrival order as soon as a slot
 * of their plan is free and their device buffers fit the arena, letting
 * later requests pass one that cannot start yet, and runs each admitted
 * request on its slot's stream (copy in, one evaluation per state, copy
 * out), so the work of several requests overlaps on the device.  A request
 * that can never fit the arena is REJECTED at once (SLP_ERR_OOM).  Requests
 * remain queryable until the server is destroyed; destroying it cancels the
 * queued requests and waits for the running ones.  The plans must not be
 * evaluated elsewhere while the server exists. */
typedef struct slp_server_s *slp_server_t;
enum { SLP_REQ_QUEUED = 1, SLP_REQ_RUNNING = 2, SLP_REQ_DONE = 3, SLP_REQ_REJECTED = 4, SLP_REQ_CANCELLED = 5,
       SLP_REQ_FAILED = 6 };
typedef struct {
    int slots_per_plan;         /* 1..16, default 2 */
    int64_t hbm_budget_bytes;   /* default 8 GiB */
    int reserved[6];
} slp_server_opts;
typedef struct {
    int64_t completed, rejected, cancelled, queued;
    int64_t targets_done;                    /* sum over completed requests of n_states * n_targets */
    double latency_p50_ms, latency_p99_ms, latency_max_ms;  /* submit -> completion observed */
    double queue_wait_p50_ms, queue_wait_p99_ms;            /* submit -> admission */
    double makespan_s;                       /* first submission -> last completion */
    int64_t arena_bytes, arena_peak_bytes, slot_scratch_bytes, n_slots, max_inflight;
} slp_server_statistics;
slp_status slp_server_default_opts(slp_server_opts *opts);
slp_status slp_server_create(int n_plans, const slp_plan_t *plans, int input_kind, const slp_server_opts *opts,
                             slp_server_t *out);
slp_status slp_server_submit(slp_server_t server, int plan_index, int n_states, const void *h_in, void *h_out,
                             int64_t *request_id);
/* state: SLP_REQ_*; result: the request's status once finished */
slp_status slp_server_status(slp_server_t server, int64_t request_id, int *state, slp_status *result);
/* Blocks until the request leaves QUEUED/RUNNING or timeout_s passes
 * (SLP_ERR_TIMEOUT); returns the request's own status. */
slp_status slp_server_wait(slp_server_t server, int64_t request_id, double timeout_s, int *state);
/* Cancels a request that is still queued. */
slp_status slp_server_cancel(slp_server_t server, int64_t request_id);
slp_status slp_server_stats(slp_server_t server, slp_server_statistics *stats);
slp_status slp_server_destroy(slp_server_t server);

/* Plan parameters and sizes. */
slp_status slp_query(slp_plan_t plan, slp_info *info);

/* Quadrature point coordinates in the source order k = j*q + s: host [Q][3]. */
slp_status slp_query_points(slp_plan_t plan, double *points);

/* Synchronise the plan's device and report (and clear) the sticky device
 * status word written by the kernels: SLP_ERR_NONFINITE when a checked
 * evaluation (opts.check_finite) saw NaN/Inf in its input or result,
 * SLP_ERR_CUDA for an inconsistent work item. */
slp_status slp_check(slp_plan_t plan);

/* Release the plan and all its device memory.  NULL is accepted. */
slp_status slp_destroy(slp_plan_t plan);

/* Static description of a status code; never NULL. */
const char *slp_status_string(slp_status status);

/* Thread-local detail of the last failing call on this thread ("" if none). */
const char *slp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SLP_H */
