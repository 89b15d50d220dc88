/*
 * FP64 oracle for the triangle-quadrature single layer potential.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct CPU
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library under paper_1305_3162_gb300/ never includes, links or calls it.
 *
 * What it computes (paper Sec. 2.2, the discretised single layer potential,
 * with the surface integrals replaced by a triangle quadrature as in the
 * quadrature form of Sec. 3):
 *
 *     phi_i = (1 / 4 pi) * sum_j sum_s  w_s |S_j| sigma_{j,s} / |x_i - y_{j,s}|
 *
 *   x_i      the mesh vertices (the boundary nodes),
 *   S_j      the flat surface triangles, |S_j| their areas, n_j the outward
 *            unit normal from the vertex winding (v1 - v0) x (v2 - v0),
 *   y_{j,s}  = sum_a lambda_{s,a} v_{j,a}, the quadrature points,
 *   w_s      the rule weights (summing to one),
 *   sigma    the surface charge m . n (Sec. 2, g = m.n when phi_1 = 0).
 *
 * The sum is taken directly over every (target, source) pair, O(N Q), with
 * Neumaier-compensated accumulation per target and OpenMP over targets.
 * No blocking, no splitting of the kernel, no approximation.
 *
 * A second definition, for the triangle-integrated discretisation (paper
 * Sec. 2.2, Eq. (slayer3) itself, no quadrature): element-wise constant
 * charges g_j (the L2 projection of m . n onto constants per triangle,
 * i.e. its integral mean) and exact triangle integrals,
 *
 *     phi_i = (1 / 4 pi) * sum_j g_j * int_{S_j} 1 / |x_i - y| dA(y),
 *
 * each integral by the edge-sum closed form for a uniformly charged flat
 * polygon (Wilton et al. 1984; Graglia 1993), again over every pair.
 *
 * Quadrature rules (the point order is part of the library contract: the
 * source index is k = j * q + s):
 *   q = 3: degree-2 rule with interior points, barycentric (2/3, 1/6, 1/6)
 *          and its cyclic shifts, weights 1/3;
 *   q = 7: Radon's degree-5 rule: centroid with weight 9/40, the points
 *          (a, a, 1 - 2a) for a = (6 - sqrt 15)/21 with weight
 *          (155 - sqrt 15)/1200 and for a = (6 + sqrt 15)/21 with weight
 *          (155 + sqrt 15)/1200, each in the order (a,a,1-2a), (a,1-2a,a),
 *          (1-2a,a,a).
 *   q = 1: centroid rule (weight 1).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Barycentric points lam[q][3] and weights w[q] of the q-point rule. */
int slpo_rule(int q, double *lam, double *w)
{
    if (q == 1) {
        lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
        w[0] = 1.0;
        return 0;
    }
    if (q == 3) {
        for (int s = 0; s < 3; ++s) {
            for (int a = 0; a < 3; ++a) lam[3 * s + a] = (a == s) ? 2.0 / 3.0 : 1.0 / 6.0;
            w[s] = 1.0 / 3.0;
        }
        return 0;
    }
    if (q == 7) {
        const double r15 = sqrt(15.0);
        const double a[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
        const double wa[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
        lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
        w[0] = 9.0 / 40.0;
        int s = 1;
        for (int g = 0; g < 2; ++g) {
            const double o = 1.0 - 2.0 * a[g];
            /* (a, a, o), (a, o, a), (o, a, a) */
            for (int p = 0; p < 3; ++p, ++s) {
                for (int c = 0; c < 3; ++c) lam[3 * s + c] = a[g];
                lam[3 * s + (2 - p)] = o;
                w[s] = wa[g];
            }
        }
        return 0;
    }
    return -1;
}

/* Quadrature points y[nt*q][3], weights wk[nt*q] = w_s |S_j| and outward unit
 * normals nrm[nt][3].  Returns -2 for a degenerate triangle, -3 for a bad index. */
int slpo_sources(const double *V, int64_t nv, const int32_t *T, int64_t nt, int q,
                 double *y, double *wk, double *nrm)
{
    double lam[21], w[7];
    if (slpo_rule(q, lam, w) != 0) return -1;
    for (int64_t j = 0; j < nt; ++j) {
        const int32_t i0 = T[3 * j], i1 = T[3 * j + 1], i2 = T[3 * j + 2];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) return -3;
        const double *v0 = V + 3 * i0, *v1 = V + 3 * i1, *v2 = V + 3 * i2;
        const double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
        const double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1],
                             e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double twice_area = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(twice_area > 0.0)) return -2;
        for (int d = 0; d < 3; ++d) nrm[3 * j + d] = c[d] / twice_area;
        for (int s = 0; s < q; ++s) {
            const int64_t k = j * q + s;
            for (int d = 0; d < 3; ++d)
                y[3 * k + d] = lam[3 * s] * v0[d] + lam[3 * s + 1] * v1[d] + lam[3 * s + 2] * v2[d];
            wk[k] = w[s] * 0.5 * twice_area;
        }
    }
    return 0;
}

/* Weighted charges qk = w_s |S_j| sigma_{j,s} for the three input kinds:
 *   kind 0: input = sigma at the quadrature points, [nt*q];
 *   kind 1: input = m at the quadrature points, [nt*q][3], sigma = m . n_j;
 *   kind 2: input = m at the vertices, [nv][3], interpolated linearly (P1)
 *           to the quadrature points, sigma = m(y) . n_j. */
int slpo_charges(int kind, const double *V, int64_t nv, const int32_t *T, int64_t nt, int q,
                 const double *input, double *qk)
{
    double lam[21], w[7];
    if (slpo_rule(q, lam, w) != 0) return -1;
    for (int64_t j = 0; j < nt; ++j) {
        const int32_t iv[3] = {T[3 * j], T[3 * j + 1], T[3 * j + 2]};
        for (int a = 0; a < 3; ++a)
            if (iv[a] < 0 || iv[a] >= nv) return -3;
        const double *v0 = V + 3 * iv[0], *v1 = V + 3 * iv[1], *v2 = V + 3 * iv[2];
        const double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
        const double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1],
                             e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double twice_area = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(twice_area > 0.0)) return -2;
        const double n[3] = {c[0] / twice_area, c[1] / twice_area, c[2] / twice_area};
        for (int s = 0; s < q; ++s) {
            const int64_t k = j * q + s;
            double sigma;
            if (kind == 0) {
                sigma = input[k];
            } else if (kind == 1) {
                sigma = input[3 * k] * n[0] + input[3 * k + 1] * n[1] + input[3 * k + 2] * n[2];
            } else if (kind == 2) {
                double m[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 3; ++d) m[d] += lam[3 * s + a] * input[3 * iv[a] + d];
                sigma = m[0] * n[0] + m[1] * n[1] + m[2] * n[2];
            } else {
                return -1;
            }
            qk[k] = w[s] * 0.5 * twice_area * sigma;
        }
    }
    return 0;
}

/* phi_i = (1/4pi) sum_k qk / |x_i - y_k| over all pairs, Neumaier summation.
 * nthreads <= 0 uses the OpenMP default.  Returns the thread count used. */
int slpo_direct(const double *x, int64_t nx, const double *y, const double *qk, int64_t nq,
                double *phi, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int64_t i = 0; i < nx; ++i) {
        const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
        double sum = 0.0, comp = 0.0;
        for (int64_t k = 0; k < nq; ++k) {
            const double d0 = xi0 - y[3 * k], d1 = xi1 - y[3 * k + 1], d2 = xi2 - y[3 * k + 2];
            const double v = qk[k] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double t = sum + v;
            if (fabs(sum) >= fabs(v))
                comp += (sum - t) + v;
            else
                comp += (v - t) + sum;
            sum = t;
        }
        phi[i] = (sum + comp) / (4.0 * ORACLE_PI);
    }
    return used;
}

/* Direct sum restricted to a subset of targets (indices sel[ns]); used to
 * time a bounded sample and to check large workloads at sampled nodes. */
int slpo_direct_subset(const double *x, const int64_t *sel, int64_t ns, const double *y,
                       const double *qk, int64_t nq, double *phi, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int64_t t = 0; t < ns; ++t) {
        const int64_t i = sel[t];
        const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
        double sum = 0.0, comp = 0.0;
        for (int64_t k = 0; k < nq; ++k) {
            const double d0 = xi0 - y[3 * k], d1 = xi1 - y[3 * k + 1], d2 = xi2 - y[3 * k + 2];
            const double v = qk[k] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double tt = sum + v;
            if (fabs(sum) >= fabs(v))
                comp += (sum - tt) + v;
            else
                comp += (v - tt) + sum;
            sum = tt;
        }
        phi[t] = (sum + comp) / (4.0 * ORACLE_PI);
    }
    return used;
}

/* ---------------------------------------------------------------- triangle integrals
 * int_{S} 1/|x - y| dA(y) over the flat triangle S = (v0, v1, v2).  With n the
 * unit normal of the winding, h = (x - v0) . n the signed height of x over
 * the plane and rho = x - h n its projection, and for each edge e from p- to
 * p+ (counter-clockwise about n): l the unit edge direction, u = l x n the
 * in-plane outward normal, l-/l+ = (p-/+ - rho) . l, P0 = (p- - rho) . u,
 * R-/R+ = |x - p-/+| and R0^2 = P0^2 + h^2:
 *
 *   I = sum_e P0 ln((R+ + l+) / (R- + l-))
 *       - |h| sum_e [atan(P0 l+ / (R0^2 + |h| R+)) - atan(P0 l- / (R0^2 + |h| R-))].
 *
 * An edge whose line passes through rho (P0 = 0) contributes nothing: its log
 * term vanishes with P0, and so do its atan terms. */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

double slpo_triangle_integral(const double *v0, const double *v1, const double *v2, const double *x)
{
    const double *v[3] = {v0, v1, v2};
    double e1[3], e2[3], n[3], d[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    const double nn = sqrt(dot3(n, n));
    if (!(nn > 0.0)) return 0.0;
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    sub3(x, v0, d);
    const double h = dot3(d, n), ah = fabs(h);
    const double rho[3] = {x[0] - h * n[0], x[1] - h * n[1], x[2] - h * n[2]};
    double total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *pm = v[e], *pp = v[(e + 1) % 3];
        double L[3], l[3], u[3], am[3], ap[3], xm[3], xp[3];
        sub3(pp, pm, L);
        const double len = sqrt(dot3(L, L));
        l[0] = L[0] / len; l[1] = L[1] / len; l[2] = L[2] / len;
        cross3(l, n, u);
        sub3(pm, rho, am);
        sub3(pp, rho, ap);
        const double lm = dot3(am, l), lp = dot3(ap, l), P0 = dot3(am, u);
        sub3(x, pm, xm);
        sub3(x, pp, xp);
        const double Rm = sqrt(dot3(xm, xm)), Rp = sqrt(dot3(xp, xp));
        const double R02 = P0 * P0 + h * h;
        if (fabs(P0) > 1e-14 * len) total += P0 * log((Rp + lp) / (Rm + lm));
        if (ah > 0.0) total -= ah * (atan(P0 * lp / (R02 + ah * Rp)) - atan(P0 * lm / (R02 + ah * Rm)));
    }
    return total;
}

/* Element charges: g_j = (1/|S_j|) int_{S_j} m . n_j dA for the nodal m
 * interpolated linearly (P1) on the triangle, which is n_j . (m_a + m_b + m_c) / 3
 * (the integral mean of a linear function is its value at the centroid). */
int slpo_element_charges(const double *V, int64_t nv, const int32_t *T, int64_t nt, const double *m, double *g)
{
    for (int64_t j = 0; j < nt; ++j) {
        const int32_t a = T[3 * j], b = T[3 * j + 1], c = T[3 * j + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) return 1;
        double e1[3], e2[3], n[3];
        sub3(V + 3 * (int64_t)b, V + 3 * (int64_t)a, e1);
        sub3(V + 3 * (int64_t)c, V + 3 * (int64_t)a, e2);
        cross3(e1, e2, n);
        const double nn = sqrt(dot3(n, n));
        if (!(nn > 0.0)) return 2;
        double mc[3];
        for (int k = 0; k < 3; ++k) mc[k] = (m[3 * (int64_t)a + k] + m[3 * (int64_t)b + k] + m[3 * (int64_t)c + k]) / 3.0;
        g[j] = dot3(mc, n) / nn;
    }
    return 0;
}

/* phi_t = (1/4pi) sum_j g_j int_{S_j} 1/|x_{sel[t]} - y| dA(y) over every
 * triangle, Neumaier summation, OpenMP over targets; sel == NULL takes every
 * target (ns = nx).  Returns the thread count used. */
int slpo_direct_p0(const double *x, const int64_t *sel, int64_t ns, const double *V, int64_t nv,
                   const int32_t *T, int64_t nt, const double *g, double *phi, int nthreads)
{
    int used = 1;
    (void)nv;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t t = 0; t < ns; ++t) {
        const int64_t i = sel ? sel[t] : t;
        double sum = 0.0, comp = 0.0;
        for (int64_t j = 0; j < nt; ++j) {
            const double v = g[j] * slpo_triangle_integral(V + 3 * (int64_t)T[3 * j], V + 3 * (int64_t)T[3 * j + 1],
                                                           V + 3 * (int64_t)T[3 * j + 2], x + 3 * i);
            const double tt = sum + v;
            if (fabs(sum) >= fabs(v))
                comp += (sum - tt) + v;
            else
                comp += (v - tt) + sum;
            sum = tt;
        }
        phi[t] = (sum + comp) / (4.0 * ORACLE_PI);
    }
    return used;
}
