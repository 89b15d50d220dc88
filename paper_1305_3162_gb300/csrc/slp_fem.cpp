// The scalar potential phi = phi_1 + phi_2 on a tetrahedral mesh (Alg. 1).
//
// Setup (slp_potential_create), host FP64:
//   * the boundary: faces that belong to one tetrahedron only, wound so that
//     their normal points away from the tetrahedron's fourth node;
//   * P1 elements (Sec. 2.1): on each tetrahedron the hat-function gradients
//     (rows of the inverse edge matrix), the stiffness entries
//     |T| grad eta_a . grad eta_b restricted to free rows and columns (phi_1
//     is zero on the boundary, so the free subsystem is all that is solved),
//     and the load operator b_a = sum_T |T| grad eta_a . mean_T(m), mean_T(m)
//     the mean of the four nodal values (m is P1);
//   * the boundary's triangle-integrated plan (opts.integration = 1) and a
//     probe set of the free nodes, so that phi_2 reaches every node;
//   * the solve as one CUDA graph: WHILE nodes over the corrections and,
//     inside each, over passes of FEM_CHUNK inner conjugate-gradient
//     launches, their handles set on the device from the solver's state.
// Evaluation (slp_potential_eval): b = B m; the solve graph (FP32 inner
// steps, FP64 corrections, no host round trip); the charges g; phi_2 through
// the plan and its probes; phi = phi_1 + phi_2.  The host waits for the
// solve's state only, to return its status.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/slp_debug.h"
#include "slp_fem.h"
#include "slp_plan_internal.h"

#define FTRY(x)                        \
    do {                               \
        const slp_status st_ = (x);    \
        if (st_ != SLP_OK) return st_; \
    } while (0)

struct slp_potential_s {
    int device = 0, prec = 32;
    int64_t n_nodes = 0, n_tets = 0, nf = 0, nb = 0, nfaces = 0, s_nnz = 0, b_nnz = 0;
    slp_plan_t plan = nullptr;
    slp_probe_t probe = nullptr;
    slp::FemDev d;
    void *g = nullptr, *phi2_b = nullptr, *phi2_f = nullptr;  // plan precision
    slp::CgState *h_st = nullptr;                               // page-locked
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};  // start, phi_1 done, phi done (timing)
    bool timed = false;
    double cg_tol = 0.0;
    int64_t last_iter = -1, last_outer = 0;
    double last_res = 0.0;
    std::vector<void *> allocs;
};

namespace {

slp_status cu(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SLP_OK;
    cudaGetLastError();
    return slp_fail(e == cudaErrorMemoryAllocation ? SLP_ERR_OOM : SLP_ERR_CUDA, "%s: %s", what,
                    cudaGetErrorString(e));
}

template <typename X> slp_status upload(slp_potential_s &p, X **dst, const X *src, size_t n) {
    void *ptr = nullptr;
    FTRY(cu(cudaMalloc(&ptr, std::max<size_t>(n * sizeof(X), 16)), "potential allocation"));
    p.allocs.push_back(ptr);
    if (src && n) FTRY(cu(cudaMemcpy(ptr, src, n * sizeof(X), cudaMemcpyHostToDevice), "potential upload"));
    *dst = (X *)ptr;
    return SLP_OK;
}

// Captures the launches of `launch` into graph g after the nodes dep[0..ndep);
// *last is the node the captured work ends in.
template <typename F>
cudaError_t capture_into(cudaGraph_t g, cudaStream_t s, const cudaGraphNode_t *dep, size_t ndep, F launch,
                         cudaGraphNode_t *last) {
    cudaError_t e = cudaStreamBeginCaptureToGraph(s, g, dep, nullptr, ndep, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = launch();
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *tail = nullptr;
    size_t ntail = 0;
    cudaError_t ie = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &tail, nullptr, &ntail);
    if (ie == cudaSuccess && ntail == 1)
        *last = tail[0];
    else if (ie == cudaSuccess)
        ie = cudaErrorInvalidValue;  // the captured work must end in one node
    cudaGraph_t out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &out);
    return le != cudaSuccess ? le : ie != cudaSuccess ? ie : ce;
}

// A WHILE node on `handle` after node dep; *body is the graph it repeats.
cudaError_t add_while(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle handle, cudaGraphNode_t *node,
                      cudaGraph_t *body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    const cudaError_t e = cudaGraphAddNode(node, g, &dep, nullptr, 1, &cp);
    if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
    return e;
}

// The solve: [outer start] -> WHILE (corrections) { [inner start] -> WHILE
// (inner) { FEM_CHUNK inner launches -> [inner next] } -> correction,
// residual, next inner start -> [outer next] }.  The handles start at 0 and
// only the loop-control kernels set them.
cudaError_t build_solve_graph(slp_potential_s &P) {
    const slp::FemDev &d = P.d;
    cudaStream_t s = P.cap;
    const int inner_bound = (int)std::min<long long>((d.max_iter + slp::FEM_CHUNK - 1) / slp::FEM_CHUNK + 3, 1 << 30);
    cudaError_t e = cudaGraphCreate(&P.graph, 0);
    cudaGraphConditionalHandle ho = 0, hi = 0;
    cudaGraphNode_t start = nullptr, outer = nullptr, istart = nullptr, inner = nullptr, last = nullptr;
    cudaGraph_t obody = nullptr, ibody = nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ho, P.graph, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = capture_into(P.graph, s, nullptr, 0, [&] { return slp::launch_fem_loop(slp::LOOP_OUTER_START, d, ho, 0, s); },
                         &start);
    if (e == cudaSuccess) e = add_while(P.graph, start, ho, &outer, &obody);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, obody, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = capture_into(obody, s, nullptr, 0, [&] { return slp::launch_fem_loop(slp::LOOP_INNER_START, d, hi, 0, s); },
                         &istart);
    if (e == cudaSuccess) e = add_while(obody, istart, hi, &inner, &ibody);
    if (e == cudaSuccess)
        e = capture_into(ibody, s, nullptr, 0,
                         [&] {
                             cudaError_t le = cudaSuccess;
                             for (int k = 0; k < slp::FEM_CHUNK && le == cudaSuccess; ++k)
                                 le = slp::launch_cg_iteration(d, k & 1, s);
                             if (le != cudaSuccess) return le;
                             return slp::launch_fem_loop(slp::LOOP_INNER_NEXT, d, hi, inner_bound, s);
                         },
                         &last);
    if (e == cudaSuccess)
        e = capture_into(obody, s, &inner, 1,
                         [&] {
                             const cudaError_t le = slp::launch_fem_correct(d, s);
                             if (le != cudaSuccess) return le;
                             return slp::launch_fem_loop(slp::LOOP_OUTER_NEXT, d, ho, slp::FEM_MAX_OUTER, s);
                         },
                         &last);
    return e;
}

void release(slp_potential_s *p) {
    if (!p) return;
    SlpDeviceGuard g(p->device);
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : p->tev)
        if (e) cudaEventDestroy(e);
    if (p->h_st) cudaFreeHost(p->h_st);
    for (void *a : p->allocs) cudaFree(a);
    if (p->probe) slp_probe_destroy(p->probe);
    if (p->plan) slp_destroy(p->plan);
    delete p;
}

struct Vec3 {
    double x, y, z;
};
inline Vec3 sub3(const double *a, const double *b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
inline Vec3 cross3(const Vec3 &a, const Vec3 &b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double dot3(const Vec3 &a, const Vec3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Hat-function gradients and volume of one tetrahedron: with the edge matrix
// J = [x1 - x0, x2 - x0, x3 - x0] (columns), grad eta_{1,2,3} are the rows of
// J^-1 (the cofactors over det J) and grad eta_0 = -(their sum).
bool tet_gradients(const double *X, const int32_t *t, double grad[4][3], double &vol) {
    const Vec3 e1 = sub3(X + 3 * (int64_t)t[1], X + 3 * (int64_t)t[0]);
    const Vec3 e2 = sub3(X + 3 * (int64_t)t[2], X + 3 * (int64_t)t[0]);
    const Vec3 e3 = sub3(X + 3 * (int64_t)t[3], X + 3 * (int64_t)t[0]);
    const Vec3 c23 = cross3(e2, e3), c31 = cross3(e3, e1), c12 = cross3(e1, e2);
    const double det = dot3(e1, c23);
    const double scale = std::max({dot3(e1, e1), dot3(e2, e2), dot3(e3, e3)});
    if (!(std::fabs(det) > 1e-12 * scale * std::sqrt(scale))) return false;
    const Vec3 g[3] = {c23, c31, c12};  // rows of J^-1 times det
    for (int a = 0; a < 3; ++a) {
        grad[a + 1][0] = g[a].x / det;
        grad[a + 1][1] = g[a].y / det;
        grad[a + 1][2] = g[a].z / det;
    }
    for (int k = 0; k < 3; ++k) grad[0][k] = -(grad[1][k] + grad[2][k] + grad[3][k]);
    vol = std::fabs(det) / 6.0;
    return true;
}

struct Face {
    int32_t k[3];  // sorted node ids
    int64_t tet;
    int local;  // the tetrahedron's node opposite the face
};

// Automatic grid of the potential's plan.  The evaluation's grid work grows
// as L^3 per axis length L, and its exact near field (boundary nodes and free
// nodes within the truncation radius of a triangle, a radius that shrinks as
// 1/L) as n_points F / L^2, so the cheapest grid grows as (n_points F)^(1/5).
// The factor 3.0 lies inside the range that picks the grid measured best on
// tetrahedral balls of 17k, 134k and 449k nodes (128, 256 and 256 cells per
// axis; any factor from 2.6 to 3.46 does); each axis gets its share of the
// period as in the plan's own automatic grid, rounded to the nearest power of
// two.
void potential_grid(const std::vector<double> &V, int64_t n_points, int64_t F, int grid[3]) {
    const int64_t n = (int64_t)V.size() / 3;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], V[3 * i + d]);
            hi[d] = std::max(hi[d], V[3 * i + d]);
        }
    double r2 = 0.0, D[3], dmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        D[d] = hi[d] - lo[d];
        dmax = std::max(dmax, D[d]);
    }
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) s += (V[3 * i + d] - 0.5 * (lo[d] + hi[d])) * (V[3 * i + d] - 0.5 * (lo[d] + hi[d]));
        r2 = std::max(r2, s);
    }
    const double diam = 2.0 * std::sqrt(r2);
    const double cells = 3.0 * std::pow((double)std::max<int64_t>(n_points, 1) * (double)std::max<int64_t>(F, 1), 0.2);
    for (int d = 0; d < 3; ++d) {
        const double want = cells * (D[d] + diam) / (dmax + diam);
        int v = 16;
        while (v < 1024 && want >= v * 1.4142135623730951) v <<= 1;
        grid[d] = v;
    }
}

// The set-up on the host (FP64): node classes and numbering, the boundary
// triangles wound outward with their normals and 1/h, S(free, free) in CSR
// and the load operator in CSR over free rows.
struct FemHost {
    int64_t nf = 0, nb = 0, F = 0;
    std::vector<int> slot;  // per node: free index (>= 0) or -1 - boundary index
    std::vector<int64_t> free_nodes, bnd_nodes;
    std::vector<int32_t> Ts;       // [F][3] boundary triangles in boundary-node indices, wound outward
    std::vector<int4> face;        // nodes a, b, c (outward) and the free index of the fourth node, or -1
    std::vector<double4> face_n;   // unit outward normal and 1/h
    std::vector<int64_t> s_ptr, b_ptr;
    std::vector<int> s_col, b_col;  // free indices (S), node indices (B)
    std::vector<double> s_val, dinv;
    std::vector<float> s_val32;
    std::vector<double4> b_val;    // (x, y, z, 0)
};

slp_status assemble(const double *X, int64_t N, const int32_t *tets, int64_t K, FemHost &H) {
    // hat-function gradients of every tetrahedron
    std::vector<double> grads((size_t)K * 12), vols(K);
    for (int64_t t = 0; t < K; ++t) {
        for (int a = 0; a < 4; ++a)
            if (tets[4 * t + a] < 0 || tets[4 * t + a] >= N)
                return slp_fail(SLP_ERR_MESH, "tetrahedron %lld has a node index out of range", (long long)t);
        double g[4][3];
        if (!tet_gradients(X, tets + 4 * t, g, vols[t]))
            return slp_fail(SLP_ERR_MESH, "tetrahedron %lld is degenerate", (long long)t);
        memcpy(&grads[12 * t], g, sizeof g);
    }
    // faces: boundary = faces of one tetrahedron only
    std::vector<Face> faces((size_t)K * 4);
    for (int64_t t = 0; t < K; ++t)
        for (int o = 0; o < 4; ++o) {
            Face &f = faces[4 * t + o];
            int c = 0;
            for (int a = 0; a < 4; ++a)
                if (a != o) f.k[c++] = tets[4 * t + a];
            std::sort(f.k, f.k + 3);
            f.tet = t;
            f.local = o;
        }
    std::sort(faces.begin(), faces.end(), [](const Face &a, const Face &b) {
        return std::lexicographical_compare(a.k, a.k + 3, b.k, b.k + 3);
    });
    std::vector<Face> bfaces;
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && std::equal(faces[i].k, faces[i].k + 3, faces[j].k)) ++j;
        if (j - i > 2) return slp_fail(SLP_ERR_MESH, "a face is shared by more than two tetrahedra");
        if (j - i == 1) bfaces.push_back(faces[i]);
        i = j;
    }
    if (bfaces.empty()) return slp_fail(SLP_ERR_MESH, "the mesh has no boundary");
    // node classes and numbering (ascending node order within each class)
    std::vector<char> used(N, 0), bnd(N, 0);
    for (int64_t i = 0; i < 4 * K; ++i) used[tets[i]] = 1;
    for (int64_t i = 0; i < N; ++i)
        if (!used[i]) return slp_fail(SLP_ERR_MESH, "node %lld belongs to no tetrahedron", (long long)i);
    for (const Face &f : bfaces)
        for (int a = 0; a < 3; ++a) bnd[f.k[a]] = 1;
    std::vector<int> &slot = H.slot;
    std::vector<int64_t> &free_nodes = H.free_nodes, &bnd_nodes = H.bnd_nodes;
    slot.assign(N, 0);
    for (int64_t i = 0; i < N; ++i) {
        if (bnd[i]) {
            slot[i] = -1 - (int)bnd_nodes.size();
            bnd_nodes.push_back(i);
        } else {
            slot[i] = (int)free_nodes.size();
            free_nodes.push_back(i);
        }
    }
    const int64_t nf = (int64_t)free_nodes.size(), nb = (int64_t)bnd_nodes.size(), F = (int64_t)bfaces.size();
    H.nf = nf;
    H.nb = nb;
    H.F = F;
    // boundary triangles wound outward, their normals and 1/h
    std::vector<int32_t> &Ts = H.Ts;
    std::vector<int4> &face = H.face;
    std::vector<double4> &face_n = H.face_n;
    Ts.assign((size_t)F * 3, 0);
    face.assign(F, int4{});
    face_n.assign(F, double4{});
    for (int64_t j = 0; j < F; ++j) {
        const Face &f = bfaces[j];
        const int32_t o = tets[4 * f.tet + f.local];
        int32_t a = f.k[0], b = f.k[1], c = f.k[2];
        Vec3 n = cross3(sub3(X + 3 * (int64_t)b, X + 3 * (int64_t)a), sub3(X + 3 * (int64_t)c, X + 3 * (int64_t)a));
        if (dot3(n, sub3(X + 3 * (int64_t)o, X + 3 * (int64_t)a)) > 0) {
            std::swap(b, c);
            n = {-n.x, -n.y, -n.z};
        }
        const double area2 = std::sqrt(dot3(n, n));
        face[j] = make_int4(a, b, c, bnd[o] ? -1 : slot[o]);
        // h = 3 |T| / |S| = 6 |T| / (2 |S|)
        face_n[j] = make_double4(n.x / area2, n.y / area2, n.z / area2, area2 / (6.0 * vols[f.tet]));
        Ts[3 * j] = -1 - slot[a];
        Ts[3 * j + 1] = -1 - slot[b];
        Ts[3 * j + 2] = -1 - slot[c];
    }
    // stiffness on free rows and columns, and the load operator, as sorted triples
    struct E {
        int64_t key;
        double v[3];
    };
    std::vector<E> se, be;
    se.reserve((size_t)K * 16);
    be.reserve((size_t)K * 12);
    for (int64_t t = 0; t < K; ++t) {
        const double(*g)[3] = (const double(*)[3]) & grads[12 * t];
        const double v = vols[t];
        for (int a = 0; a < 4; ++a) {
            const int ra = slot[tets[4 * t + a]];
            if (ra < 0) continue;
            for (int b = 0; b < 4; ++b) {
                const int nbk = tets[4 * t + b];
                const int cb = slot[nbk];
                if (cb >= 0)
                    se.push_back({(int64_t)ra * nf + cb,
                                  {v * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]), 0.0, 0.0}});
                if (b != a)  // the row's own column multiplies m_row - m_row = 0
                    be.push_back({(int64_t)ra * N + nbk, {0.25 * v * g[a][0], 0.25 * v * g[a][1], 0.25 * v * g[a][2]}});
            }
        }
    }
    auto merge = [](std::vector<E> &e) {
        std::stable_sort(e.begin(), e.end(), [](const E &a, const E &b) { return a.key < b.key; });
        size_t w = 0;
        for (size_t i = 0; i < e.size();) {
            E s = e[i];
            size_t j = i + 1;
            for (; j < e.size() && e[j].key == s.key; ++j)
                for (int k = 0; k < 3; ++k) s.v[k] += e[j].v[k];
            e[w++] = s;
            i = j;
        }
        e.resize(w);
    };
    merge(se);
    merge(be);
    std::vector<int64_t> &s_ptr = H.s_ptr, &b_ptr = H.b_ptr;
    std::vector<int> &s_col = H.s_col, &b_col = H.b_col;
    std::vector<double> &s_val = H.s_val, &dinv = H.dinv;
    std::vector<float> &s_val32 = H.s_val32;
    std::vector<double4> &b_val = H.b_val;
    s_ptr.assign(nf + 1, 0);
    b_ptr.assign(nf + 1, 0);
    s_col.assign(se.size(), 0);
    b_col.assign(be.size(), 0);
    s_val.assign(se.size(), 0.0);
    dinv.assign(nf, 0.0);
    s_val32.assign(se.size(), 0.f);
    b_val.assign(be.size(), double4{});
    for (size_t i = 0; i < se.size(); ++i) {
        const int64_t r = se[i].key / nf, c = se[i].key % nf;
        ++s_ptr[r + 1];
        s_col[i] = (int)c;
        s_val[i] = se[i].v[0];
        s_val32[i] = (float)se[i].v[0];
        if (r == c) dinv[r] = 1.0 / se[i].v[0];
    }
    for (size_t i = 0; i < be.size(); ++i) {
        const int64_t r = be[i].key / N;
        ++b_ptr[r + 1];
        b_col[i] = (int)(be[i].key % N);
        b_val[i] = make_double4(be[i].v[0], be[i].v[1], be[i].v[2], 0.0);
    }
    for (int64_t i = 0; i < nf; ++i) {
        s_ptr[i + 1] += s_ptr[i];
        b_ptr[i + 1] += b_ptr[i];
        if (!(dinv[i] > 0) || !std::isfinite(dinv[i]))
            return slp_fail(SLP_ERR_MESH, "free node %lld has no positive stiffness diagonal", (long long)free_nodes[i]);
    }
    se.clear();
    se.shrink_to_fit();
    be.clear();
    be.shrink_to_fit();

    return SLP_OK;
}

slp_status build(slp_potential_s &P, const double *X, int64_t N, const int32_t *tets, int64_t K, double tolerance,
                 const slp_plan_opts *opts) {
    FemHost H;
    FTRY(assemble(X, N, tets, K, H));
    const int64_t nf = H.nf, nb = H.nb, F = H.F;
    P.nf = nf;
    P.nb = nb;
    P.nfaces = F;
    P.s_nnz = (int64_t)H.s_col.size();
    P.b_nnz = (int64_t)H.b_col.size();
    const std::vector<int> &slot = H.slot;
    const std::vector<int64_t> &free_nodes = H.free_nodes, &bnd_nodes = H.bnd_nodes;
    const std::vector<int32_t> &Ts = H.Ts;
    const std::vector<int4> &face = H.face;
    const std::vector<double4> &face_n = H.face_n;
    const std::vector<int64_t> &s_ptr = H.s_ptr, &b_ptr = H.b_ptr;
    const std::vector<int> &s_col = H.s_col, &b_col = H.b_col;
    const std::vector<double> &s_val = H.s_val, &dinv = H.dinv;
    const std::vector<float> &s_val32 = H.s_val32;
    const std::vector<double4> &b_val = H.b_val;

    // the boundary's plan and the free nodes as its probes
    std::vector<double> Vs((size_t)nb * 3), Xf((size_t)nf * 3);
    for (int64_t i = 0; i < nb; ++i)
        for (int k = 0; k < 3; ++k) Vs[3 * i + k] = X[3 * bnd_nodes[i] + k];
    for (int64_t i = 0; i < nf; ++i)
        for (int k = 0; k < 3; ++k) Xf[3 * i + k] = X[3 * free_nodes[i] + k];
    slp_plan_opts o;
    slp_default_opts(&o);
    if (opts) o = *opts;
    o.integration = 1;
    slp_mesh mesh{Vs.data(), nb, Ts.data(), F};
    const bool auto_grid = o.grid[0] == 0 && o.grid[1] == 0 && o.grid[2] == 0;
    if (auto_grid) potential_grid(Vs, nb + nf, F, o.grid);
    slp_status pst = slp_plan(&mesh, 3, tolerance, &o, &P.plan);
    // a triangle wider than the plan's triangle integrals allow on this grid: coarsen it
    while (auto_grid && pst == SLP_ERR_UNSUPPORTED && std::max(o.grid[0], std::max(o.grid[1], o.grid[2])) > 16) {
        for (int d = 0; d < 3; ++d) o.grid[d] = std::max(8, o.grid[d] / 2);
        pst = slp_plan(&mesh, 3, tolerance, &o, &P.plan);
    }
    FTRY(pst);
    slp_info info;
    FTRY(slp_query(P.plan, &info));
    P.prec = info.precision;
    P.device = o.device;
    if (P.device < 0) return slp_fail(SLP_ERR_NO_DEVICE, "the scalar potential needs a device");
    SlpDeviceGuard guard(P.device);
    if (nf > 0) FTRY(slp_probe_create(P.plan, Xf.data(), nf, &P.probe));

    // device data
    slp::FemDev &d = P.d;
    d.nf = nf;
    d.nblk_max = 8 * 152;
    FTRY(upload(P, (int64_t **)&d.s_ptr, s_ptr.data(), s_ptr.size()));
    FTRY(upload(P, (int **)&d.s_col, s_col.data(), s_col.size()));
    FTRY(upload(P, (double **)&d.s_val, s_val.data(), s_val.size()));
    {
        // FP32 copy in slices of 32 rows (column-major within a slice)
        const int64_t nsl = (nf + 31) / 32;
        std::vector<int64_t> sl_ptr(nsl + 1, 0);
        std::vector<int> sl_w(nsl, 0);
        for (int64_t t = 0; t < nsl; ++t) {
            int w = 0;
            for (int64_t i = 32 * t; i < std::min(nf, 32 * t + 32); ++i) w = std::max<int>(w, (int)(s_ptr[i + 1] - s_ptr[i]));
            sl_w[t] = w;
            sl_ptr[t + 1] = sl_ptr[t] + 32 * (int64_t)w;
        }
        std::vector<int> sl_col(std::max<int64_t>(sl_ptr[nsl], 1), 0);
        std::vector<float> sl_val(sl_col.size(), 0.f);
        for (int64_t t = 0; t < nsl; ++t)
            for (int l = 0; l < 32; ++l) {
                const int64_t i = 32 * t + l;
                for (int k = 0; k < sl_w[t]; ++k) {
                    const int64_t at = sl_ptr[t] + 32 * (int64_t)k + l;
                    if (i < nf && s_ptr[i] + k < s_ptr[i + 1]) {
                        sl_col[at] = s_col[s_ptr[i] + k];
                        sl_val[at] = s_val32[s_ptr[i] + k];
                    } else {
                        sl_col[at] = (int)std::min<int64_t>(i, nf - 1);  // padding: own column, zero value
                    }
                }
            }
        FTRY(upload(P, (int64_t **)&d.sl_ptr, sl_ptr.data(), sl_ptr.size()));
        FTRY(upload(P, (int **)&d.sl_w, sl_w.data(), sl_w.size()));
        FTRY(upload(P, (int **)&d.sl_col, sl_col.data(), sl_col.size()));
        FTRY(upload(P, (float **)&d.sl_val, sl_val.data(), sl_val.size()));
    }
    {
        std::vector<float> d32(dinv.begin(), dinv.end());
        FTRY(upload(P, (float **)&d.dinv, d32.data(), d32.size()));
        std::vector<int> fn(free_nodes.begin(), free_nodes.end());
        FTRY(upload(P, (int **)&d.fnode, fn.data(), fn.size()));
    }
    FTRY(upload(P, (int64_t **)&d.b_ptr, b_ptr.data(), b_ptr.size()));
    FTRY(upload(P, (int **)&d.b_col, b_col.data(), b_col.size()));
    if (P.prec == 64) {
        FTRY(upload(P, (double4 **)&d.b_val, b_val.data(), b_val.size()));
    } else {
        std::vector<float4> b32(b_val.size());
        for (size_t i = 0; i < b_val.size(); ++i)
            b32[i] = make_float4((float)b_val[i].x, (float)b_val[i].y, (float)b_val[i].z, 0.f);
        FTRY(upload(P, (float4 **)&d.b_val, b32.data(), b32.size()));
    }
    const int64_t stride = std::max<int64_t>(nf, 1);
    double *vec = nullptr;
    FTRY(upload(P, &vec, (const double *)nullptr, (size_t)stride * 3 + 3 * d.nblk_max));
    d.b = vec;
    d.x = vec + stride;
    d.rho = vec + 2 * stride;
    d.part = vec + 3 * stride;
    float *v32 = nullptr;
    FTRY(upload(P, &v32, (const float *)nullptr, (size_t)stride * 2 + 6 * d.nblk_max));
    d.xc = v32;
    d.p = v32 + stride;
    d.part32 = v32 + 2 * stride;
    float4 *v4 = nullptr;
    FTRY(upload(P, &v4, (const float4 *)nullptr, (size_t)stride * 2));
    d.v[0] = v4;
    d.v[1] = v4 + stride;
    FTRY(upload(P, &d.st, (const slp::CgState *)nullptr, 1));
    FTRY(cu(cudaMemset(d.st, 0, sizeof(slp::CgState)), "state"));
    FTRY(cu(cudaMemset(d.x, 0, sizeof(double) * stride), "phi_1"));
    d.tol2 = P.cg_tol * P.cg_tol;
    d.inner2 = (float)(slp::FEM_INNER * slp::FEM_INNER);
    d.nfaces = F;
    FTRY(upload(P, (int4 **)&d.face, face.data(), face.size()));
    FTRY(upload(P, (double4 **)&d.face_n, face_n.data(), face_n.size()));
    d.nnodes = N;
    FTRY(upload(P, (int **)&d.slot, slot.data(), slot.size()));
    const size_t es = P.prec == 64 ? 8 : 4;
    unsigned char *tb = nullptr;
    FTRY(upload(P, &tb, (const unsigned char *)nullptr, es * (size_t)(F + nb + std::max<int64_t>(nf, 1)) + 64));
    P.g = tb;
    P.phi2_b = tb + es * ((F + 7) / 8 * 8);
    P.phi2_f = (unsigned char *)P.phi2_b + es * ((nb + 7) / 8 * 8);
    FTRY(cu(cudaHostAlloc((void **)&P.h_st, sizeof(slp::CgState), cudaHostAllocDefault), "host state"));
    for (auto &e : P.ev) FTRY(cu(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event"));
    for (auto &e : P.tev) FTRY(cu(cudaEventCreate(&e), "event"));

    // the solve graph
    if (nf > 0) {
        FTRY(cu(cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking), "stream"));
        FTRY(cu(build_solve_graph(P), "solve graph"));
        FTRY(cu(cudaGraphInstantiate(&P.exec, P.graph, 0), "solve graph"));
    }
    return cu(cudaDeviceSynchronize(), "potential setup");
}

}  // namespace

extern "C" {

slp_status slp_potential_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                                double tolerance, const slp_plan_opts *opts, double cg_tolerance,
                                int cg_max_iterations, slp_potential_t *out) {
    if (!out) return slp_fail(SLP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!nodes || !tets || n_nodes < 4 || n_tets < 1)
        return slp_fail(SLP_ERR_INVALID_ARG, "nodes or tetrahedra missing");
    if (n_nodes >= (1LL << 31) || n_tets >= (1LL << 31)) return slp_fail(SLP_ERR_INVALID_ARG, "mesh too large");
    if (!(cg_tolerance >= 0.0) || cg_max_iterations < 0 || !(tolerance > 0.0))
        return slp_fail(SLP_ERR_INVALID_ARG, "tolerances must be positive and the iteration limit non-negative");
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
        if (!std::isfinite(nodes[i])) return slp_fail(SLP_ERR_INVALID_ARG, "node coordinates must be finite");
    if (opts && opts->device < 0) return slp_fail(SLP_ERR_NO_DEVICE, "the scalar potential needs a device");
    slp_potential_s *P = new slp_potential_s();
    P->n_nodes = n_nodes;
    P->n_tets = n_tets;
    P->cg_tol = cg_tolerance > 0.0 ? cg_tolerance : std::max(1e-2 * tolerance, 1e-14);
    P->d.max_iter = cg_max_iterations > 0 ? cg_max_iterations : 10000;
    const slp_status st = build(*P, nodes, n_nodes, tets, n_tets, tolerance, opts);
    if (st != SLP_OK) {
        release(P);
        return st;
    }
    *out = P;
    return SLP_OK;
}

slp_status slp_potential_eval(slp_potential_t P, const void *d_m, void *d_phi, void *d_phi_1, void *stream) {
    if (!P || !d_m || !d_phi) return slp_fail(SLP_ERR_INVALID_ARG, "potential, m or phi missing");
    SlpDeviceGuard guard(P->device);
    cudaStream_t s = (cudaStream_t)stream;
    const slp::FemDev &d = P->d;
    int64_t iters = 0, outer = 0;
    double res = 0.0;
    bool bad = false, converged = true;
    FTRY(cu(cudaEventRecord(P->tev[0], s), "event"));
    if (P->nf > 0) {
        // the load, then the solve graph (its loops end on the device: the
        // inner steps at max_iter in all, the corrections at FEM_MAX_OUTER);
        // the state is copied behind it for the status
        FTRY(cu(slp::launch_fem_load(d, P->prec, d_m, s), "load"));
        FTRY(cu(cudaGraphLaunch(P->exec, s), "solve graph"));
        FTRY(cu(cudaMemcpyAsync(P->h_st, d.st, sizeof(slp::CgState), cudaMemcpyDeviceToHost, s), "state copy"));
        FTRY(cu(cudaEventRecord(P->ev[0], s), "event"));
    }
    FTRY(cu(cudaEventRecord(P->tev[1], s), "event"));
    FTRY(cu(slp::launch_fem_charges(d, P->prec, d_m, P->g, s), "charges"));
    if (P->probe)
        FTRY(slp_eval_probe(P->plan, P->probe, SLP_INPUT_ELEMENT, P->g, P->phi2_b, P->phi2_f, s));
    else
        FTRY(slp_eval(P->plan, SLP_INPUT_ELEMENT, P->g, P->phi2_b, s));
    FTRY(cu(slp::launch_fem_combine(d, P->prec, P->phi2_b, P->phi2_f, d_phi, d_phi_1, s), "sum"));
    FTRY(cu(cudaEventRecord(P->tev[2], s), "event"));
    if (P->nf > 0) {
        FTRY(cu(cudaEventSynchronize(P->ev[0]), "solve wait"));
        const slp::CgState &h = *P->h_st;
        iters = h.iter;
        outer = h.outer;
        res = h.bb > 0 ? std::sqrt(std::max(h.rr_hi, 0.0) / h.bb) : 0.0;
        bad = h.bad != 0;
        converged = h.outer_done && !bad && (h.bb == 0.0 || h.rr_hi <= d.tol2 * h.bb);
    }
    P->timed = true;
    P->last_iter = iters;
    P->last_outer = outer;
    P->last_res = res;
    if (bad) return slp_fail(SLP_ERR_NONFINITE, "the iteration met a non-finite value");
    if (!converged)
        return slp_fail(SLP_ERR_TOLERANCE_INFEASIBLE,
                        "the solve stopped at relative residual %.3e after %lld steps", res, (long long)iters);
    return SLP_OK;
}

slp_status slp_potential_query(slp_potential_t P, slp_potential_info *info) {
    if (!P || !info) return slp_fail(SLP_ERR_INVALID_ARG, "potential or info missing");
    memset(info, 0, sizeof *info);
    info->n_nodes = P->n_nodes;
    info->n_tets = P->n_tets;
    info->n_free = P->nf;
    info->n_boundary = P->nb;
    info->n_faces = P->nfaces;
    info->stiffness_nnz = P->s_nnz;
    info->load_nnz = P->b_nnz;
    info->cg_iterations = P->last_iter;
    info->cg_corrections = P->last_outer;
    info->cg_max_iterations = P->d.max_iter;
    info->cg_residual = P->last_res;
    info->cg_tolerance = P->cg_tol;
    info->ms_phi1 = info->ms_phi2 = -1.0;
    if (P->timed) {
        SlpDeviceGuard guard(P->device);
        if (cudaEventQuery(P->tev[2]) == cudaSuccess) {
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, P->tev[0], P->tev[1]) == cudaSuccess &&
                cudaEventElapsedTime(&b, P->tev[1], P->tev[2]) == cudaSuccess) {
                info->ms_phi1 = a;
                info->ms_phi2 = b;
            }
        }
        cudaGetLastError();
    }
    info->surface_plan = P->plan;
    return SLP_OK;
}

slp_status slp_potential_destroy(slp_potential_t P) {
    release(P);
    return SLP_OK;
}

slp_status slp_debug_fem_assemble(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                                  int64_t counts[5], int32_t *node_slot, int32_t *faces, double *face_geom,
                                  int64_t *s_ptr, int32_t *s_col, double *s_val, int64_t *b_ptr, int32_t *b_col,
                                  double *b_val) {
    if (!counts) return slp_fail(SLP_ERR_INVALID_ARG, "counts is NULL");
    if (!nodes || !tets || n_nodes < 4 || n_tets < 1)
        return slp_fail(SLP_ERR_INVALID_ARG, "nodes or tetrahedra missing");
    if (n_nodes >= (1LL << 31) || n_tets >= (1LL << 31)) return slp_fail(SLP_ERR_INVALID_ARG, "mesh too large");
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
        if (!std::isfinite(nodes[i])) return slp_fail(SLP_ERR_INVALID_ARG, "node coordinates must be finite");
    FemHost H;
    FTRY(assemble(nodes, n_nodes, tets, n_tets, H));
    counts[0] = H.nf;
    counts[1] = H.nb;
    counts[2] = H.F;
    counts[3] = (int64_t)H.s_col.size();
    counts[4] = (int64_t)H.b_col.size();
    if (node_slot)
        for (int64_t i = 0; i < n_nodes; ++i) node_slot[i] = H.slot[i];
    for (int64_t j = 0; j < H.F; ++j) {
        if (faces) {
            faces[4 * j] = H.face[j].x;
            faces[4 * j + 1] = H.face[j].y;
            faces[4 * j + 2] = H.face[j].z;
            faces[4 * j + 3] = H.face[j].w;
        }
        if (face_geom) {
            face_geom[4 * j] = H.face_n[j].x;
            face_geom[4 * j + 1] = H.face_n[j].y;
            face_geom[4 * j + 2] = H.face_n[j].z;
            face_geom[4 * j + 3] = H.face_n[j].w;
        }
    }
    if (s_ptr) std::copy(H.s_ptr.begin(), H.s_ptr.end(), s_ptr);
    if (s_col) std::copy(H.s_col.begin(), H.s_col.end(), s_col);
    if (s_val) std::copy(H.s_val.begin(), H.s_val.end(), s_val);
    if (b_ptr) std::copy(H.b_ptr.begin(), H.b_ptr.end(), b_ptr);
    if (b_col) std::copy(H.b_col.begin(), H.b_col.end(), b_col);
    if (b_val)
        for (size_t e = 0; e < H.b_val.size(); ++e) {
            b_val[3 * e] = H.b_val[e].x;
            b_val[3 * e + 1] = H.b_val[e].y;
            b_val[3 * e + 2] = H.b_val[e].z;
        }
    return SLP_OK;
}

}  // extern "C"
