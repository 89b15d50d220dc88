// Host side of the library: the C ABI, plan construction (the setup phase of
// the paper's Alg. 1) and the launch sequence of one evaluation (its
// computation phase).
//
// Plan construction, all in FP64 on the host:
//   1. validate the mesh (indices, degenerate triangles, closed and
//      consistently outward oriented surface);
//   2. quadrature sources y_{j,s} = sum_a lambda_{s,a} v_{j,a}, weights
//      w_s |S_j|, outward normals (Sec. 2.2 discretisation, quadrature form of
//      Sec. 3);
//   3. parameters: window half-width m from the NFFT error bound C(2, m)
//      (Sec. 3.2, Eq. (error_bound_nufft)), the torus (centre, period), the
//      smooth kernel and the near-field radius (see choose_radial);
//   4. grid coordinates, tile sort of sources and targets, work lists of the
//      spread, gather and near-field kernels;
//   5. the kernel multiplier table D (Sec. 3, Eq. (deconv) and Sec. 5, Eq.
//      (BEM_NFFT_compact2): kernel Fourier coefficients divided by the squared
//      window coefficients of Eq. (cFB)) and the FFT twiddles;
//   6. device allocation and upload.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "slp_plan_internal.h"

namespace {

thread_local std::string g_last_error;

slp_status fail(slp_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- rules
// Barycentric points and weights (see slp.h for the point order).
bool quad_rule(int q, std::vector<double> &lam, std::vector<double> &w) {
    lam.assign(3 * q, 0.0);
    w.assign(q, 0.0);
    if (q == 1) {
        lam = {1.0 / 3, 1.0 / 3, 1.0 / 3};
        w = {1.0};
        return true;
    }
    if (q == 3) {
        for (int s = 0; s < 3; ++s) {
            for (int a = 0; a < 3; ++a) lam[3 * s + a] = (a == s) ? 2.0 / 3.0 : 1.0 / 6.0;
            w[s] = 1.0 / 3.0;
        }
        return true;
    }
    if (q == 7) {
        const double r = std::sqrt(15.0);
        lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
        w[0] = 9.0 / 40.0;
        const double av[2] = {(6.0 - r) / 21.0, (6.0 + r) / 21.0};
        const double wv[2] = {(155.0 - r) / 1200.0, (155.0 + r) / 1200.0};
        int s = 1;
        for (int g = 0; g < 2; ++g) {
            const double a = av[g], o = 1.0 - 2.0 * a;
            const double pts[3][3] = {{a, a, o}, {a, o, a}, {o, a, a}};
            for (int p = 0; p < 3; ++p, ++s) {
                for (int c = 0; c < 3; ++c) lam[3 * s + c] = pts[p][c];
                w[s] = wv[g];
            }
        }
        return true;
    }
    return false;
}

// ---------------------------------------------------------------- window
const double KB_B = PI * (2.0 - 1.0 / 2.0);  // b = pi (2 - 1/alpha), alpha = 2

double kb_window_host(int m, double d) {
    const double beta = KB_B * m;
    const double t = d / m;
    const double s2 = 1.0 - t * t;
    if (s2 < 0.0) return 0.0;
    const double s = std::sqrt(s2);
    const double r = (beta * s > 1e-8) ? std::sinh(beta * s) / s : beta;
    return r / std::sinh(beta);
}

// Continuous Fourier transform of the normalised window at the frequency of
// index l on an L-point grid: (pi m / sinh beta) I0(m sqrt(b^2 - (2 pi l / L)^2))
// (Eq. (cFB) times L, times the normalisation pi m / sinh beta).
double kb_hat_host(int m, int L, double l) {
    const double beta = KB_B * m;
    const double om = 2.0 * PI * l / L;
    const double a2 = KB_B * KB_B - om * om;
    if (a2 <= 0.0) return 0.0;
    return PI * m / std::sinh(beta) * std::cyl_bessel_i(0.0, m * std::sqrt(a2));
}

// NFFT error bound C(alpha, m) of Eq. (error_bound_nufft), alpha = 2.
double nfft_bound(int m) {
    const double a = 2.0;
    return 4.0 * PI * (std::sqrt((double)m) + m) * std::pow(1.0 - 1.0 / a, 0.25) *
           std::exp(-2.0 * PI * m * std::sqrt(1.0 - 1.0 / a));
}

// inverse of erfc on (0, 1] by bisection (monotone), FP64
double erfc_inv(double y) {
    double lo = 0.0, hi = 30.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (std::erfc(mid) > y)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

// Per-interval polynomial of the window for the FP32 kernels:
// p_i(f) = sum_k c[i][k] f^k interpolates psi(f + m - 1 - i) at deg + 1
// Chebyshev nodes of f in [0, 1] (psi = sinh(beta s)/s is entire in the
// offset, so the interpolant converges geometrically: degree 9 is within
// 1e-10 of psi(0) for m <= 6).
std::vector<double> window_polynomials(int m, int deg) {
    const int n = deg + 1;
    std::vector<double> out((size_t)2 * m * n, 0.0);
    std::vector<double> x(n);
    for (int k = 0; k < n; ++k) x[k] = 0.5 - 0.5 * std::cos(PI * (k + 0.5) / n);
    for (int i = 0; i < 2 * m; ++i) {
        // Vandermonde system A c = y, Gaussian elimination with partial pivoting
        std::vector<double> A((size_t)n * n), y(n);
        for (int r = 0; r < n; ++r) {
            double pw = 1.0;
            for (int c = 0; c < n; ++c) {
                A[(size_t)r * n + c] = pw;
                pw *= x[r];
            }
            y[r] = kb_window_host(m, x[r] + m - 1 - i);
        }
        for (int c = 0; c < n; ++c) {
            int piv = c;
            for (int r = c + 1; r < n; ++r)
                if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
            if (piv != c) {
                for (int cc = 0; cc < n; ++cc) std::swap(A[(size_t)c * n + cc], A[(size_t)piv * n + cc]);
                std::swap(y[c], y[piv]);
            }
            for (int r = c + 1; r < n; ++r) {
                const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
                for (int cc = c; cc < n; ++cc) A[(size_t)r * n + cc] -= f * A[(size_t)c * n + cc];
                y[r] -= f * y[c];
            }
        }
        for (int r = n - 1; r >= 0; --r) {
            double v = y[r];
            for (int cc = r + 1; cc < n; ++cc) v -= A[(size_t)r * n + cc] * out[(size_t)i * n + cc];
            out[(size_t)i * n + r] = v / A[(size_t)r * n + r];
        }
    }
    return out;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Morton code of a cell inside its tile (3 bits per axis level)
uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t c = 0;
    for (int b = 0; b < 10; ++b) {
        c |= ((x >> b) & 1u) << (3 * b);
        c |= ((y >> b) & 1u) << (3 * b + 1);
        c |= ((z >> b) & 1u) << (3 * b + 2);
    }
    return c;
}

// error-budget factors of the RADIAL split (relative to the tolerance):
// band-limit tail of the Gaussian and the erfc tail left outside eps.
const double KFAC = 10.0;
const double NFAC = 2.0;

}  // namespace

namespace {

// many sources per spread cell group (at least 8 on average): the FP32 spread
// for m <= 4 then runs at 4 blocks per SM with 64 registers, else at 5 with 48
bool spread_dense(const slp_plan_s &p) {
    if (p.opts.spread_blocks) return p.opts.spread_blocks == 4;
    return p.sgroups.size() > 0 && (double)p.Q >= 8.0 * (double)p.sgroups.size();
}

// ---------------------------------------------------------------- mesh
slp_status validate_mesh(slp_plan_s &p) {
    const int64_t N = p.N, M = p.M;
    for (int64_t j = 0; j < M; ++j) {
        const int32_t *t = &p.T[3 * j];
        for (int a = 0; a < 3; ++a)
            if (t[a] < 0 || t[a] >= N) return fail(SLP_ERR_MESH, "triangle %lld has vertex index %d out of range", (long long)j, t[a]);
        if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2])
            return fail(SLP_ERR_MESH, "triangle %lld repeats a vertex", (long long)j);
    }
    if (!p.opts.check_mesh) return SLP_OK;
    // closed and consistently oriented: every directed edge once, and its reverse once
    std::vector<uint64_t> e, r;
    e.reserve(3 * M);
    r.reserve(3 * M);
    for (int64_t j = 0; j < M; ++j) {
        for (int a = 0; a < 3; ++a) {
            const uint64_t u = (uint32_t)p.T[3 * j + a], v = (uint32_t)p.T[3 * j + (a + 1) % 3];
            e.push_back((u << 32) | v);
            r.push_back((v << 32) | u);
        }
    }
    std::sort(e.begin(), e.end());
    std::sort(r.begin(), r.end());
    if (std::adjacent_find(e.begin(), e.end()) != e.end())
        return fail(SLP_ERR_MESH, "a directed edge is used twice: the surface is non-manifold or inconsistently oriented");
    if (e != r) return fail(SLP_ERR_MESH, "the surface is not closed (an edge has no opposite half-edge)");
    // outward orientation: signed volume > 0
    double vol = 0.0;
    for (int64_t j = 0; j < M; ++j) {
        const double *a = &p.V[3 * p.T[3 * j]], *b = &p.V[3 * p.T[3 * j + 1]], *c = &p.V[3 * p.T[3 * j + 2]];
        vol += a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    if (!(vol > 0.0)) return fail(SLP_ERR_MESH, "the enclosed signed volume is not positive: normals point inward");
    return SLP_OK;
}

slp_status build_sources(slp_plan_s &p) {
    if (!quad_rule(p.q, p.lam, p.wq)) return fail(SLP_ERR_INVALID_ARG, "unsupported quadrature %d (use 1, 3 or 7)", p.q);
    p.Q = p.M * p.q;
    p.y.assign(3 * p.Q, 0.0);
    p.wk.assign(p.Q, 0.0);
    p.nrm.assign(3 * p.M, 0.0);
    for (int64_t j = 0; j < p.M; ++j) {
        const double *v0 = &p.V[3 * p.T[3 * j]], *v1 = &p.V[3 * p.T[3 * j + 1]], *v2 = &p.V[3 * p.T[3 * j + 2]];
        const double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
        const double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double a2 = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        double scale = 0;
        for (int d = 0; d < 3; ++d) scale = std::max(scale, std::fabs(e1[d]) + std::fabs(e2[d]));
        if (!(a2 > 1e-14 * scale * scale)) return fail(SLP_ERR_MESH, "triangle %lld is degenerate (zero area)", (long long)j);
        for (int d = 0; d < 3; ++d) p.nrm[3 * j + d] = c[d] / a2;
        for (int s = 0; s < p.q; ++s) {
            const int64_t k = j * p.q + s;
            for (int d = 0; d < 3; ++d)
                p.y[3 * k + d] = p.lam[3 * s] * v0[d] + p.lam[3 * s + 1] * v1[d] + p.lam[3 * s + 2] * v2[d];
            p.wk[k] = p.wq[s] * 0.5 * a2;
        }
    }
    return SLP_OK;
}

// ---------------------------------------------------------------- parameters
// RADIAL smooth kernel (the reading of Sec. 3.3 this library uses):
//   N_s = (N 1_{|x| <= R}) * g_s, g_s an isotropic Gaussian of width s.
// Its Fourier transform is closed form, Khat(k) = 2 sin^2(k R / 2) / k^2 exp(-s^2 k^2 / 2),
// and for |x| <= R - c s, N_s(x) = erf(|x| / (s sqrt 2)) / (4 pi |x|), so the near-field
// kernel N - N_s = erfc(r / (s sqrt 2)) / (4 pi r) decays like a Gaussian.
// Conditions (c = sqrt(2 ln(1/tau_k))):
//   band limit  s >= c P_q / (pi n_q)           (Gaussian below tau_k at |l_q| = n_q/2)
//   isolation   P_q >= D_q + R + c s,  R = diam + c s  (no periodic image overlaps)
//   near radius erfc(eps / (s sqrt 2)) = tau_nf
// which give s = max_q c (D_q + diam) / (pi n_q - 2 c^2), feasible iff pi n_q > 2 c^2.
bool radial_feasible(const slp_plan_s &p, const int n[3], double c) {
    for (int d = 0; d < 3; ++d)
        if (!(PI * n[d] > 2.0 * c * c * 1.05)) return false;
    return true;
}

void radial_params(slp_plan_s &p, double c) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s = std::max(s, c * (p.D[d] + p.diam) / (PI * p.n[d] - 2.0 * c * c));
    p.sigma_g = s;
    for (int d = 0; d < 3; ++d) p.P[d] = p.D[d] + p.diam + 2.0 * c * s;
    p.R = p.diam + c * s;
    const double tnf = std::min(0.5, p.tol * NFAC);
    p.eps = s * std::sqrt(2.0) * erfc_inv(tnf);
}

// ---------------------------------------------------------------- exp-sum kernel (Sec. 3.3)
// Sum of Gaussians for 1/r on [rmin, beta] (torus units) by the trapezoidal
// rule applied to 1/r = (2/sqrt(pi)) int exp(t - r^2 e^{2t}) dt over the real
// line: node t_k gives g_k = e^{2 t_k} and w_k = (2h/sqrt(pi)) e^{t_k}.  The
// range of t is cut where the integrand's tails fall below delta (left:
// (2/sqrt(pi)) e^{t} r <= delta at r = beta; right: r^2 e^{2t} past
// log(1/delta) at r = rmin), and the step h is halved from 1 until the sum
// meets 1/r to relative delta/2 on a log-spaced check grid of [rmin, beta].
// Terms come out ordered from the widest Gaussian to the narrowest.
void expsum_terms(double rmin, double beta, double delta, std::vector<double> &w, std::vector<double> &g) {
    const double t_lo = std::log(delta * std::sqrt(PI) / (2.0 * beta)) - 1.0;
    const double t_hi = std::log(std::sqrt(std::log(4.0 / delta) + 4.0) / rmin) + 0.5;
    for (double h = 1.0; h > 1e-3; h *= 0.8) {
        w.clear();
        g.clear();
        for (double t = t_lo; t <= t_hi + 1e-12; t += h) {
            w.push_back(2.0 * h / std::sqrt(PI) * std::exp(t));
            g.push_back(std::exp(2.0 * t));
        }
        double worst = 0.0;
        for (int i = 0; i <= 400; ++i) {
            const double r = rmin * std::pow(beta / rmin, i / 400.0);
            double s = 0.0;
            for (size_t k = 0; k < w.size(); ++k) s += w[k] * std::exp(-g[k] * r * r);
            worst = std::max(worst, std::fabs(s * r - 1.0));
        }
        if (worst <= 0.5 * delta) return;
    }
}

// I(g, l) = int_{-1/2}^{1/2} exp(-g u^2) cos(2 pi l u) du, the Fourier
// coefficient over one period of the torus (the definition of c_l(N_s) in
// Sec. 2.2): the whole-line transform when the Gaussian has decayed at the
// cell face, else composite 10-point Gauss-Legendre on [0, 1/2] with two
// panels per period of the cosine.
double gauss_period_coeff(double g, int l) {
    if (g * 0.25 > 45.0) return std::sqrt(PI / g) * std::exp(-PI * PI * (double)l * l / g);
    static const double X[5] = {0.1488743389816312, 0.4333953941292472, 0.6794095682990244, 0.8650633666889845,
                                0.9739065285171717};
    static const double Wt[5] = {0.2955242247147529, 0.2692667193099963, 0.2190863625159820, 0.1494513491505806,
                                 0.0666713443086881};
    const int np = 2 * std::abs(l) + 8;
    const double hw = 0.25 / np;  // half panel width on [0, 1/2]
    double s = 0.0;
    for (int k = 0; k < np; ++k) {
        const double c = (2 * k + 1) * hw;
        for (int j = 0; j < 5; ++j)
            for (int sg = -1; sg <= 1; sg += 2) {
                const double u = c + sg * X[j] * hw;
                s += Wt[j] * std::exp(-g * u * u) * std::cos(2.0 * PI * l * u);
            }
    }
    return 2.0 * s * hw;
}

// Parameters of the EXPSUM kernel: cubic torus of period P = D_max / 0.4,
// the sum for 1/r on [r0, 1/2] (torus units; r0 far below any near radius),
// the widest terms the grid resolves (Fourier factor below tau_k at
// |l| = n/2 for the smallest n), and the near radius eps: the smallest r from
// which the kept terms still meet 1/r to relative tol.
slp_status expsum_params(slp_plan_s &p) {
    const double dmax = std::max(p.D[0], std::max(p.D[1], p.D[2]));
    const double P = dmax / 0.4;
    for (int d = 0; d < 3; ++d) p.P[d] = P;
    const double delta = std::min(0.1, p.tol);
    const double tk = std::min(0.1, p.tol);
    std::vector<double> w, g;
    expsum_terms(1e-4, 0.5, delta, w, g);
    const int nmin = std::min(p.n[0], std::min(p.n[1], p.n[2]));
    const double gmax = PI * PI * (0.5 * nmin) * (0.5 * nmin) / std::log(1.0 / tk);
    p.es_w.clear();
    p.es_g.clear();
    for (size_t k = 0; k < w.size(); ++k)
        if (g[k] <= gmax) {
            p.es_w.push_back(w[k]);
            p.es_g.push_back(g[k]);
        }
    if (p.es_w.empty())
        return fail(SLP_ERR_TOLERANCE_INFEASIBLE, "grid too small for any exp-sum term (n = %d)", nmin);
    // near radius (torus units): scan down from 1/2 while the kept sum meets 1/r
    double eps_u = 0.5;
    for (int i = 0; i <= 2000; ++i) {
        const double r = 0.5 * std::pow(1e-4 / 0.5, i / 2000.0);
        double s = 0.0;
        for (size_t k = 0; k < p.es_w.size(); ++k) s += p.es_w[k] * std::exp(-p.es_g[k] * r * r);
        if (std::fabs(s * r - 1.0) > delta) break;
        eps_u = r;
    }
    p.eps = eps_u * P;
    p.sigma_g = 0;
    p.R = 0;
    return SLP_OK;
}

slp_status choose_parameters(slp_plan_s &p) {
    // bounding box and enclosing-ball diameter of targets (sources are convex
    // combinations of targets, so they lie inside both)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < p.N; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], p.V[3 * i + d]);
            hi[d] = std::max(hi[d], p.V[3 * i + d]);
        }
    double rad2 = 0;
    for (int d = 0; d < 3; ++d) {
        p.ctr[d] = 0.5 * (lo[d] + hi[d]);
        p.D[d] = hi[d] - lo[d];
    }
    for (int64_t i = 0; i < p.N; ++i) {
        double r2 = 0;
        for (int d = 0; d < 3; ++d) r2 += (p.V[3 * i + d] - p.ctr[d]) * (p.V[3 * i + d] - p.ctr[d]);
        rad2 = std::max(rad2, r2);
    }
    p.diam = 2.0 * std::sqrt(rad2) * (1.0 + 1e-12);
    if (!(p.diam > 0)) return fail(SLP_ERR_MESH, "mesh has zero extent");

    // window half-width from the NFFT bound
    int m = p.opts.m;
    if (m == 0) {
        m = 2;
        while (nfft_bound(m) > p.tol / 4.0 && m < 8) ++m;
        if (p.prec == 32) m = std::min(m, 6);
    }
    if (m < 2 || m > 8) return fail(SLP_ERR_INVALID_ARG, "window half-width m = %d outside [2, 8]", m);
    p.m = m;

    // requested grid
    int L[3];
    for (int d = 0; d < 3; ++d) {
        L[d] = p.opts.grid[d];
        if (L[d] == 0) L[d] = -1;
        if (L[d] > 0 && (!is_pow2(L[d]) || L[d] < 8 || L[d] > 1024))
            return fail(SLP_ERR_INVALID_ARG, "grid[%d] = %d must be a power of two in [8, 1024]", d, L[d]);
    }
    const double tk = std::min(0.1, p.tol * KFAC);
    const double c = std::sqrt(2.0 * std::log(1.0 / tk));
    p.c_band = c;
    if (L[0] < 0 || L[1] < 0 || L[2] < 0) {
        // automatic: equal spacing at about (Q + N)^(1/2) cells across the body
        const double target_cells = std::max(16.0, 2.0 * std::sqrt((double)(p.Q + p.N)));
        const double dmax = std::max(p.D[0], std::max(p.D[1], p.D[2]));
        for (int d = 0; d < 3; ++d) {
            if (L[d] > 0) continue;
            // cells of the oversampled grid across the period ~ 2.3x the body
            double want = target_cells * (p.D[d] + p.diam) / (dmax + p.diam) * 1.0;
            int v = 16;
            while (v < want && v < 1024) v <<= 1;
            L[d] = v;
        }
    }
    int nreq[3] = {L[0] / 2, L[1] / 2, L[2] / 2};

    int mode = p.opts.kernel_mode;
    if (mode == SLP_KERNEL_AUTO) {
        if (radial_feasible(p, nreq, c))
            mode = SLP_KERNEL_RADIAL;
        else if (p.prec == 64 && (double)p.Q * (double)p.N <= (double)(1 << 24))
            mode = SLP_KERNEL_SEPARABLE;  // FP64 only: in FP32 the all-pairs difference loses digits
        else if (p.opts.allow_grid_raise)
            mode = -SLP_KERNEL_RADIAL;  // radial after raising the grid
        else
            return fail(SLP_ERR_TOLERANCE_INFEASIBLE,
                        "grid %dx%dx%d cannot resolve the smooth kernel at tolerance %g (needs pi n > %.1f per axis)",
                        L[0], L[1], L[2], p.tol, 2 * c * c * 1.05);
    }
    if (mode == SLP_KERNEL_RADIAL && !radial_feasible(p, nreq, c)) {
        if (!p.opts.allow_grid_raise)
            return fail(SLP_ERR_TOLERANCE_INFEASIBLE,
                        "grid %dx%dx%d cannot resolve the smooth kernel at tolerance %g (needs pi n > %.1f per axis)",
                        L[0], L[1], L[2], p.tol, 2 * c * c * 1.05);
        mode = -SLP_KERNEL_RADIAL;
    }
    if (mode == -SLP_KERNEL_RADIAL) {
        // raise: take the best-resolved feasible axis' smoothing width, and give
        // every axis the grid that resolves it (nearest power of two, never below
        // the request and at least the feasibility limit)
        double sbest = 1e300;
        for (int d = 0; d < 3; ++d)
            if (PI * nreq[d] > 2.0 * c * c * 1.05) sbest = std::min(sbest, c * (p.D[d] + p.diam) / (PI * nreq[d] - 2.0 * c * c));
        int nmin = 8;
        while (!(PI * nmin > 2.0 * c * c * 1.05)) nmin <<= 1;
        for (int d = 0; d < 3; ++d) {
            int nn = nreq[d];
            if (sbest < 1e299) {
                const double need = c * (p.D[d] + p.diam + 2 * c * sbest) / (PI * sbest);
                int v = 4;
                while (v < need) v <<= 1;
                if (v / 2 >= 4 && need / (v / 2) < (double)v / need) v /= 2;  // nearest in log scale
                nn = std::max(nn, v);
            }
            nn = std::max(nn, nmin);
            if (nn > 512) return fail(SLP_ERR_TOLERANCE_INFEASIBLE, "raised grid exceeds 1024 cells per axis");
            if (nn != nreq[d]) p.grid_raised = 1;
            nreq[d] = nn;
        }
        mode = SLP_KERNEL_RADIAL;
    }
    for (int d = 0; d < 3; ++d) {
        p.n[d] = nreq[d];
        p.L[d] = 2 * nreq[d];
    }
    p.kernel_mode = mode;

    if (mode == SLP_KERNEL_RADIAL) {
        if (!radial_feasible(p, p.n, c))
            return fail(SLP_ERR_TOLERANCE_INFEASIBLE, "grid %dx%dx%d cannot resolve the smooth kernel at tolerance %g",
                        p.L[0], p.L[1], p.L[2], p.tol);
        radial_params(p, c);
    } else if (mode == SLP_KERNEL_EXPSUM) {
        const slp_status st = expsum_params(p);
        if (st != SLP_OK) return st;
    } else if (mode == SLP_KERNEL_SEPARABLE) {
        // every pair is near; the far kernel is any band-limited periodic
        // function that the near kernel can subtract exactly
        const double dmax = std::max(p.D[0], std::max(p.D[1], p.D[2]));
        for (int d = 0; d < 3; ++d) {
            p.P[d] = 1.5 * std::max(p.D[d], 0.25 * dmax) + 1e-9 * dmax;
            const int nh = p.n[d] / 2;  // modes 0 .. n/2 - 1 (Nyquist dropped)
            p.sep_h[d].assign(nh, 0.0);
            for (int l = 0; l < nh; ++l) {
                const double t = (double)l / (0.5 * p.n[d]);
                p.sep_h[d][l] = std::exp(-2.0 * t * t);
            }
        }
        // scale: K_n(0) = 0.1 / (4 pi diam), a small smooth part next to 1/(4 pi r)
        double k0 = 1.0;
        for (int d = 0; d < 3; ++d) {
            double f = p.sep_h[d][0];
            for (size_t l = 1; l < p.sep_h[d].size(); ++l) f += 2.0 * p.sep_h[d][l];
            k0 *= f;
        }
        p.sep_A = 0.1 / (4.0 * PI * p.diam) / k0;
        p.eps = INFINITY;
        p.sigma_g = 0;
        p.R = 0;
    } else {
        return fail(SLP_ERR_INVALID_ARG, "unknown kernel_mode %d", p.opts.kernel_mode);
    }
    // grid spacing must put the whole body strictly inside the period
    for (int d = 0; d < 3; ++d)
        if (!(p.P[d] > p.D[d])) return fail(SLP_ERR_INVALID_ARG, "period does not contain the mesh");

    // tile size: 8^3 cells, halved while a halo tile (padded layout of the
    // spread/gather kernels) exceeds 40 KB, so several warps get a private copy
    // (FP32 m <= 5 keeps 8: on sparse meshes the larger tiles flush less halo
    // per source; FP64 ends at 4 or 2).  Windows wider than 10 points are
    // spread into one tile per block (no private copies): halved while that
    // tile exceeds 96 KB.
    const size_t esz = p.prec == 64 ? 8 : 4;
    p.TS = 8;
    if (p.m > 5) {
        auto tile_bytes = [&](int ts) {  // TileGeom's padded layout
            const int te = ts + 2 * p.m - 1, xo = (4 - ((p.m - 1) % 4)) % 4, xe = (xo + te + 3) / 4 * 4;
            const int rs = xe % 8 == 4 ? xe : xe + 4, ps = (te * rs + 31) / 32 * 32 + 1;
            return (size_t)te * ps * esz;
        };
        while (p.TS > 2 && tile_bytes(p.TS) > 96 * 1024) p.TS /= 2;
    } else {
        while (p.TS > 2 && std::pow((double)(p.TS + 2 * p.m + 3), 3) * esz > 40 * 1024) p.TS /= 2;
    }
    // targets: larger tiles (fewer gather items, each tile load shared by more targets)
    p.TSg = 8;
    while (p.TSg > 2 && std::pow((double)(p.TSg + 2 * p.m + 3), 3) * esz > 40 * 1024) p.TSg /= 2;
    p.TE = p.TS + 2 * p.m - 1;
    return SLP_OK;
}

// ---------------------------------------------------------------- sorting / items
void grid_coords(const slp_plan_s &p, const double *x, double *g, int &cx, int &cy, int &cz) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
        const double u = (x[d] - p.ctr[d]) / p.P[d] * p.L[d] + 0.5 * p.L[d];
        double f = std::floor(u);
        int ci = (int)f;
        double fr = u - f;
        if (fr >= 1.0) {  // rounding guard
            fr = 0.0;
            ci += 1;
        }
        ci = ((ci % p.L[d]) + p.L[d]) % p.L[d];
        c[d] = ci;
        g[d] = fr;
    }
    cx = c[0];
    cy = c[1];
    cz = c[2];
    const uint32_t packed = (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20);
    g[3] = (double)packed;
}

// sort points by (tile, Morton order inside the tile); fills perm and grid[.][4]
void sort_points(const slp_plan_s &p, const double *pts, int64_t n, int ts, std::vector<int32_t> &perm,
                 std::vector<double> &grid, std::vector<uint64_t> &keys_sorted) {
    std::vector<double> g(4 * n);
    std::vector<uint64_t> key(n);
    const int ntx = (p.L[0] + ts - 1) / ts, nty = (p.L[1] + ts - 1) / ts;
    for (int64_t i = 0; i < n; ++i) {
        int cx, cy, cz;
        grid_coords(p, pts + 3 * i, &g[4 * i], cx, cy, cz);
        const uint64_t tile = ((uint64_t)(cz / ts) * nty + (cy / ts)) * ntx + (cx / ts);
        const uint32_t mort = morton3(cx % ts, cy % ts, cz % ts);
        key[i] = (tile << 32) | mort;
    }
    perm.resize(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    grid.resize(4 * n);
    keys_sorted.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 4; ++d) grid[4 * i + d] = g[4 * perm[i] + d];
        keys_sorted[i] = key[perm[i]];
    }
}

void tile_items(const std::vector<double> &grid, const std::vector<uint64_t> &keys, int64_t n, int ts, int chunk,
                std::vector<slp::TileItem> &items) {
    items.clear();
    int64_t i = 0;
    while (i < n) {
        int64_t j = i;
        const uint64_t tile = keys[i] >> 32;
        while (j < n && (keys[j] >> 32) == tile) ++j;
        const uint32_t packed = (uint32_t)grid[4 * i + 3];
        const int cx = packed & 1023, cy = (packed >> 10) & 1023, cz = (packed >> 20) & 1023;
        for (int64_t b = i; b < j; b += chunk) {
            slp::TileItem it;
            it.c0x = cx / ts * ts;
            it.c0y = cy / ts * ts;
            it.c0z = cz / ts * ts;
            it.begin = (int)b;
            it.end = (int)std::min<int64_t>(j, b + chunk);
            it.pad0 = it.pad1 = it.pad2 = 0;
            items.push_back(it);
        }
        i = j;
    }
}

// Cell groups of each spread item (runs of one cell, at most SPREAD_GMAX
// sources; the sort makes a cell's sources contiguous), dealt largest first to
// SPREAD_WARPS lists, each group to the list with the least work so far (work
// of a group ~ a fixed part for its tile update plus one part per source).
void spread_groups(slp_plan_s &p) {
    p.sgroups.clear();
    p.sgroup_cell.clear();
    p.sgroup_off.assign(p.spread_items.size() * (slp::SPREAD_WARPS + 1), 0);
    std::vector<std::pair<int, int>> g;  // (count, first)
    std::vector<std::vector<int>> lists(slp::SPREAD_WARPS);
    for (size_t k = 0; k < p.spread_items.size(); ++k) {
        const slp::TileItem &it = p.spread_items[k];
        g.clear();
        for (int i = it.begin; i < it.end;) {
            const uint32_t cell = (uint32_t)p.src_grid[4 * (int64_t)i + 3];
            int j = i + 1;
            while (j < it.end && j - i < slp::SPREAD_GMAX && (uint32_t)p.src_grid[4 * (int64_t)j + 3] == cell) ++j;
            g.push_back({j - i, i - it.begin});
            i = j;
        }
        std::stable_sort(g.begin(), g.end(), [](const std::pair<int, int> &a, const std::pair<int, int> &b) {
            return a.first > b.first;
        });
        std::vector<int> load(slp::SPREAD_WARPS, 0);
        for (auto &l : lists) l.clear();
        for (const auto &gr : g) {
            const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            load[w] += 4 + gr.first;
            lists[w].push_back(gr.second | (gr.first << 16));
        }
        int32_t *off = &p.sgroup_off[k * (slp::SPREAD_WARPS + 1)];
        for (int w = 0; w < slp::SPREAD_WARPS; ++w) {
            off[w] = (int32_t)p.sgroups.size();
            p.sgroups.insert(p.sgroups.end(), lists[w].begin(), lists[w].end());
            // the group's cell relative to the tile's base cell
            for (int gd : lists[w]) {
                const uint32_t cell = (uint32_t)p.src_grid[4 * (int64_t)(it.begin + (gd & 0xffff)) + 3];
                const int lx = (int)(cell & 1023) - it.c0x, ly = (int)((cell >> 10) & 1023) - it.c0y,
                          lz = (int)((cell >> 20) & 1023) - it.c0z;
                p.sgroup_cell.push_back(lx | (ly << 8) | (lz << 16));
            }
        }
        off[slp::SPREAD_WARPS] = (int32_t)p.sgroups.size();
    }
}

// physical position (relative to the torus centre) of a sorted grid entry
inline void phys(const slp_plan_s &p, const double *g, double *x) {
    const uint32_t packed = (uint32_t)g[3];
    const int c[3] = {(int)(packed & 1023), (int)((packed >> 10) & 1023), (int)((packed >> 20) & 1023)};
    for (int d = 0; d < 3; ++d) x[d] = ((c[d] + g[d]) - 0.5 * p.L[d]) * (p.P[d] / p.L[d]);
}

// near-field work list: target blocks of <= 32 sorted targets in one tile,
// candidate source bins (aligned 2x2x2 cell blocks, contiguous in the sort)
// whose bounding box lies within eps of the block's bounding box.
void near_items(slp_plan_s &p, const std::vector<uint64_t> &skeys, const std::vector<uint64_t> &tkeys) {
    p.near_items.clear();
    p.near_ranges.clear();
    p.near_blk_first.clear();
    p.near_pairs = 0;
    const int64_t NCH = 2048;  // sources per item
    // target blocks
    std::vector<std::pair<int, int>> blocks;
    for (int64_t i = 0; i < p.N;) {
        int64_t j = i;
        const uint64_t tile = tkeys[i] >> 32;
        while (j < p.N && (tkeys[j] >> 32) == tile && j - i < 32) ++j;
        blocks.push_back({(int)i, (int)(j - i)});
        i = j;
    }
    const bool all_pairs = p.kernel_mode == SLP_KERNEL_SEPARABLE || !(p.eps < p.diam);
    // source bins: key = (tile, morton >> 3)
    struct Bin {
        int b, e;
        double lo[3], hi[3];
    };
    std::vector<Bin> bins;
    std::unordered_map<uint64_t, int> bin_of;  // cell-block coordinate -> bin
    if (!all_pairs) {
        for (int64_t i = 0; i < p.Q;) {
            int64_t j = i;
            const uint64_t bk = skeys[i] >> 3;
            while (j < p.Q && (skeys[j] >> 3) == bk) ++j;
            Bin bn;
            bn.b = (int)i;
            bn.e = (int)j;
            for (int d = 0; d < 3; ++d) {
                bn.lo[d] = 1e300;
                bn.hi[d] = -1e300;
            }
            for (int64_t k = i; k < j; ++k) {
                double x[3];
                phys(p, &p.src_grid[4 * k], x);
                for (int d = 0; d < 3; ++d) {
                    bn.lo[d] = std::min(bn.lo[d], x[d]);
                    bn.hi[d] = std::max(bn.hi[d], x[d]);
                }
            }
            const uint32_t packed = (uint32_t)p.src_grid[4 * i + 3];
            const uint64_t bx = (packed & 1023) / 2, by = ((packed >> 10) & 1023) / 2, bz = ((packed >> 20) & 1023) / 2;
            bin_of[(bz << 40) | (by << 20) | bx] = (int)bins.size();
            bins.push_back(bn);
            i = j;
        }
    }
    const double eps = p.eps;
    std::vector<int> found;
    for (const auto &blk : blocks) {
        std::vector<int2> rng;
        if (all_pairs) {
            rng.push_back(make_int2(0, (int)p.Q));
        } else {
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (int t = blk.first; t < blk.first + blk.second; ++t) {
                double x[3];
                phys(p, &p.tgt_grid[4 * t], x);
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::min(lo[d], x[d]);
                    hi[d] = std::max(hi[d], x[d]);
                }
            }
            int b0[3], b1[3];
            for (int d = 0; d < 3; ++d) {
                const double h = p.P[d] / p.L[d];
                const double u0 = (lo[d] - eps) / h + 0.5 * p.L[d], u1 = (hi[d] + eps) / h + 0.5 * p.L[d];
                b0[d] = std::max(0, (int)std::floor(u0) - 1) / 2;
                b1[d] = std::min(p.L[d] - 1, (int)std::floor(u1) + 1) / 2;
            }
            found.clear();
            for (int bz = b0[2]; bz <= b1[2]; ++bz)
                for (int by = b0[1]; by <= b1[1]; ++by)
                    for (int bx = b0[0]; bx <= b1[0]; ++bx) {
                        auto itb = bin_of.find(((uint64_t)bz << 40) | ((uint64_t)by << 20) | (uint64_t)bx);
                        if (itb == bin_of.end()) continue;
                        const Bin &bn = bins[itb->second];
                        double d2 = 0;
                        for (int d = 0; d < 3; ++d) {
                            const double g = std::max(0.0, std::max(bn.lo[d] - hi[d], lo[d] - bn.hi[d]));
                            d2 += g * g;
                        }
                        if (d2 <= eps * eps * (1.0 + 1e-9)) found.push_back(itb->second);
                    }
            std::sort(found.begin(), found.end(), [&](int a, int b) { return bins[a].b < bins[b].b; });
            for (int f : found) {
                if (!rng.empty() && rng.back().y == bins[f].b)
                    rng.back().y = bins[f].e;
                else
                    rng.push_back(make_int2(bins[f].b, bins[f].e));
            }
        }
        // chunk into items of <= NCH sources
        p.near_blk_first.push_back((int)p.near_items.size());
        int64_t acc = 0;
        slp::NearItem it;
        it.tbegin = blk.first;
        it.tcount = blk.second;
        it.rbegin = (int)p.near_ranges.size();
        for (int2 r : rng) {
            int b = r.x;
            while (b < r.y) {
                const int take = (int)std::min<int64_t>(r.y - b, NCH - acc);
                p.near_ranges.push_back(make_int2(b, b + take));
                acc += take;
                b += take;
                p.near_pairs += (int64_t)take * blk.second;
                if (acc == NCH) {
                    it.rend = (int)p.near_ranges.size();
                    p.near_items.push_back(it);
                    it.rbegin = it.rend;
                    acc = 0;
                }
            }
        }
        if (acc > 0) {
            it.rend = (int)p.near_ranges.size();
            p.near_items.push_back(it);
        }
        if ((int)p.near_items.size() == p.near_blk_first.back()) {
            // no candidate sources: keep an empty item so the block is represented
            it.rbegin = it.rend = (int)p.near_ranges.size();
            p.near_items.push_back(it);
        }
    }
    p.near_blk_first.push_back((int)p.near_items.size());
}

// kernel multiplier table D[|kz|][|ky|][kx] (l in I_n, Nyquist dropped)
void build_dtab(slp_plan_s &p) {
    const int Kx = p.n[0] / 2, hy = p.n[1] / 2, hz = p.n[2] / 2;
    if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
        // the S' (n_x + n_y + n_z) / 2 one-period Fourier factors of the Gaussians
        const int hn[3] = {Kx, hy, hz};
        const size_t S = p.es_w.size();
        for (int d = 0; d < 3; ++d) {
            p.es_I[d].assign(S * hn[d], 0.0);
            for (size_t k = 0; k < S; ++k)
                for (int l = 0; l < hn[d]; ++l) p.es_I[d][k * hn[d] + l] = gauss_period_coeff(p.es_g[k], l);
        }
    }
    p.Dtab.assign((size_t)hz * hy * Kx, 0.0);
    std::vector<double> W[3];
    const int hn[3] = {Kx, hy, hz};
    for (int d = 0; d < 3; ++d) {
        W[d].resize(hn[d]);
        for (int l = 0; l < hn[d]; ++l) W[d][l] = kb_hat_host(p.m, p.L[d], (double)l);
    }
    const double V = p.P[0] * p.P[1] * p.P[2];
    for (int kz = 0; kz < hz; ++kz)
        for (int ky = 0; ky < hy; ++ky)
            for (int kx = 0; kx < Kx; ++kx) {
                double cl;
                if (p.kernel_mode == SLP_KERNEL_RADIAL) {
                    const double ax = 2 * PI * kx / p.P[0], ay = 2 * PI * ky / p.P[1], az = 2 * PI * kz / p.P[2];
                    const double k2 = ax * ax + ay * ay + az * az;
                    const double k = std::sqrt(k2);
                    double kh;
                    if (k * p.R < 1e-6)
                        kh = 0.5 * p.R * p.R;
                    else {
                        const double sn = std::sin(0.5 * k * p.R);
                        kh = 2.0 * sn * sn / k2;
                    }
                    kh *= std::exp(-0.5 * p.sigma_g * p.sigma_g * k2);
                    cl = kh / V;
                } else if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
                    // separable factors: c_l = (1 / (4 pi P)) sum_k w_k I_k(l_x) I_k(l_y) I_k(l_z)
                    const size_t S = p.es_w.size();
                    cl = 0.0;
                    for (size_t k = 0; k < S; ++k)
                        cl += p.es_w[k] * p.es_I[0][k * Kx + kx] * p.es_I[1][k * hy + ky] * p.es_I[2][k * hz + kz];
                    cl /= 4.0 * PI * p.P[0];
                } else {
                    cl = p.sep_A * p.sep_h[0][kx] * p.sep_h[1][ky] * p.sep_h[2][kz];
                }
                const double w = W[0][kx] * W[1][ky] * W[2][kz];
                p.Dtab[((size_t)kz * hy + ky) * Kx + kx] = cl / (w * w);
            }
}

// ---------------------------------------------------------------- active rows
// Shortest cyclic interval of Z_L holding every set entry s[i * stride]:
// the complement of the longest cyclic run of unset entries.
void cyclic_cover(const uint8_t *s, int L, size_t stride, int &start, int &len) {
    int best = 0, best_end = -1, run = 0;
    for (int i = 0; i < 2 * L; ++i) {
        if (!s[(size_t)(i % L) * stride]) {
            if (++run > best) {
                best = run;
                best_end = i;
            }
        } else {
            run = 0;
        }
    }
    if (best >= L) {  // nothing set
        start = 0;
        len = 0;
    } else if (best == 0) {
        start = 0;
        len = L;
    } else {
        start = (best_end + 1) % L;
        len = L - best;
    }
}

// Grid A is nonzero only on rows (z, y) within the window of some source,
// and the gather reads grid B only on rows within the window of some target
// (offsets -m+1 .. m of the point's cell on each axis).  The FFT passes work
// on the cyclic z interval covering those rows and, per plane, on the cyclic
// y interval covering them, widened to whole row pairs; every other row of
// grid A, S1 and grid B is zero or never read (Sec. 5: the transforms only
// need the data the spread can produce and the gather consumes).
void active_region(slp_plan_s &p) {
    const int Ly = p.L[1], Lz = p.L[2], m = p.m;
    std::vector<uint8_t> col((size_t)Lz * Ly, 0), dy((size_t)Lz * Ly, 0), dz((size_t)Lz * Ly, 0);
    auto mark = [&](const std::vector<double> &grid, int64_t n) {
        for (int64_t i = 0; i < n; ++i) {
            const uint32_t pk = (uint32_t)grid[4 * i + 3];
            col[(size_t)((pk >> 20) & 1023) * Ly + ((pk >> 10) & 1023)] = 1;
        }
    };
    mark(p.src_grid, p.Q);
    mark(p.tgt_grid, p.N);
    if (p.opts.integration) {
        // triangle integrals reach every cell of each triangle's bounding box
        for (int64_t j = 0; j < p.M; ++j) {
            int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
            for (int a = 0; a < 3; ++a) {
                double g[4];
                int c[3];
                grid_coords(p, &p.V[3 * (int64_t)p.T[3 * j + a]], g, c[0], c[1], c[2]);
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::min(lo[d], c[d]);
                    hi[d] = std::max(hi[d], c[d]);
                }
            }
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y) col[(size_t)(((z % Lz) + Lz) % Lz) * Ly + (((y % Ly) + Ly) % Ly)] = 1;
        }
    }
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            if (col[(size_t)z * Ly + y])
                for (int o = -m + 1; o <= m; ++o) dy[(size_t)z * Ly + (((y + o) % Ly) + Ly) % Ly] = 1;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            if (dy[(size_t)z * Ly + y])
                for (int o = -m + 1; o <= m; ++o) dz[(size_t)((((z + o) % Lz) + Lz) % Lz) * Ly + y] = 1;
    std::vector<uint8_t> zany(Lz, 0);
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y) zany[z] |= dz[(size_t)z * Ly + y];
    cyclic_cover(zany.data(), Lz, 1, p.z0, p.nz_act);
    p.plane_iv.assign(Lz, make_int2(0, 0));
    p.row_pairs.clear();
    for (int i = 0; i < p.nz_act; ++i) {
        const int z = (p.z0 + i) % Lz;
        int y0, ny;
        cyclic_cover(&dz[(size_t)z * Ly], Ly, 1, y0, ny);
        if (ny > 0) {
            int ye = y0 + ny;
            y0 &= ~1;
            ye = (ye + 1) & ~1;
            ny = std::min(ye - y0, Ly);
            if (ny == Ly) y0 = 0;
        }
        p.plane_iv[z] = make_int2(y0, ny);
        for (int j = 0; j < ny / 2; ++j) p.row_pairs.push_back(z * (Ly / 2) + ((y0 + 2 * j) % Ly) / 2);
    }
}

// ---------------------------------------------------------------- device upload
slp_status cuda_status(cudaError_t e, const char *what);

template <typename T> struct V4;
template <> struct V4<float> { typedef float4 t; typedef float2 t2; };
template <> struct V4<double> { typedef double4 t; typedef double2 t2; };

slp_status dalloc(slp_plan_s &p, void **ptr, size_t bytes) {
    bytes = (size_t)round_up((int64_t)std::max<size_t>(bytes, 16), 256);
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SLP_ERR_OOM : SLP_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    p.allocs.push_back(*ptr);
    p.bytes_device += (int64_t)bytes;
    return SLP_OK;
}

template <typename S> slp_status upload(slp_plan_s &p, void **ptr, const S *src, size_t count) {
    slp_status st = dalloc(p, ptr, count * sizeof(S));
    if (st != SLP_OK) return st;
    if (count == 0) return SLP_OK;
    cudaError_t e = cudaMemcpy(*ptr, src, count * sizeof(S), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(SLP_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    return SLP_OK;
}

#define TRY(x)                          \
    do {                                \
        slp_status _s = (x);            \
        if (_s != SLP_OK) return _s;    \
    } while (0)

template <typename T> slp_status upload_all(slp_plan_s &p) {
    typedef typename V4<T>::t T4;
    typedef typename V4<T>::t2 T2;
    slp::DevPlan &d = p.dp;
    memset(&d, 0, sizeof d);
    d.prec = p.prec;
    d.q = p.q;
    d.N = p.N;
    d.Q = p.Q;
    d.M = p.M;
    d.NV = p.N;
    for (int a = 0; a < 3; ++a) {
        d.L[a] = p.L[a];
        d.n[a] = p.n[a];
        d.h[a] = p.P[a] / p.L[a];
    }
    d.Kx = p.n[0] / 2;
    d.m = p.m;
    d.TS = p.TS;
    d.TSg = p.TSg;
    d.TE = p.TE;
    d.beta = KB_B * p.m;
    {
        const int deg = 9;
        const std::vector<double> wc = window_polynomials(p.m, deg);
        std::vector<float> wcf(wc.begin(), wc.end());
        void *wp;
        TRY(upload(p, &wp, wcf.data(), wcf.size()));
        d.wcoef = wp;
        d.wdeg = deg;
    }
    d.inv_sinh_beta = 1.0 / std::sinh(d.beta);
    d.eps2 = std::isfinite(p.eps) ? p.eps * p.eps : 1e300;
    d.inv_s_sqrt2 = p.sigma_g > 0 ? 1.0 / (p.sigma_g * std::sqrt(2.0)) : 0.0;
    d.kernel_mode = p.kernel_mode;
    d.deterministic = p.opts.deterministic;
    d.check_finite = p.opts.check_finite ? 1 : 0;

    // sources / targets in sorted order
    std::vector<T4> sg(p.Q), tg(p.N);
    for (int64_t i = 0; i < p.Q; ++i) {
        const double *g = &p.src_grid[4 * i];
        T w;
        if (sizeof(T) == 4) {
            const uint32_t pk = (uint32_t)g[3];
            float f;
            memcpy(&f, &pk, 4);
            w = (T)f;
        } else {
            w = (T)g[3];
        }
        sg[i].x = (T)g[0];
        sg[i].y = (T)g[1];
        sg[i].z = (T)g[2];
        sg[i].w = w;
        // guard: a fraction that rounds up to 1 in FP32 stays below 1
        if (sg[i].x >= T(1)) sg[i].x = std::nextafter(T(1), T(0));
        if (sg[i].y >= T(1)) sg[i].y = std::nextafter(T(1), T(0));
        if (sg[i].z >= T(1)) sg[i].z = std::nextafter(T(1), T(0));
    }
    for (int64_t i = 0; i < p.N; ++i) {
        const double *g = &p.tgt_grid[4 * i];
        T w;
        if (sizeof(T) == 4) {
            const uint32_t pk = (uint32_t)g[3];
            float f;
            memcpy(&f, &pk, 4);
            w = (T)f;
        } else {
            w = (T)g[3];
        }
        tg[i].x = (T)g[0];
        tg[i].y = (T)g[1];
        tg[i].z = (T)g[2];
        tg[i].w = w;
        if (tg[i].x >= T(1)) tg[i].x = std::nextafter(T(1), T(0));
        if (tg[i].y >= T(1)) tg[i].y = std::nextafter(T(1), T(0));
        if (tg[i].z >= T(1)) tg[i].z = std::nextafter(T(1), T(0));
    }
    // per sorted source: w_k n_j (and w_k), and the triangle's vertices with the user index k
    std::vector<T4> swn(p.Q);
    std::vector<int4> stri(p.Q);
    for (int64_t i = 0; i < p.Q; ++i) {
        const int64_t k = p.src_perm[i], j = k / p.q;
        const double w = p.wk[k];
        swn[i].x = (T)(w * p.nrm[3 * j]);
        swn[i].y = (T)(w * p.nrm[3 * j + 1]);
        swn[i].z = (T)(w * p.nrm[3 * j + 2]);
        swn[i].w = (T)w;
        stri[i] = make_int4(p.T[3 * j], p.T[3 * j + 1], p.T[3 * j + 2], (int)k);
    }
    std::vector<T> lamT(p.lam.begin(), p.lam.end());
    void *ptr;
    TRY(upload(p, &ptr, sg.data(), sg.size()));
    d.src_grid = ptr;
    TRY(upload(p, &ptr, p.src_perm.data(), p.src_perm.size()));
    d.src_perm = (const int *)ptr;
    TRY(upload(p, &ptr, swn.data(), swn.size()));
    d.src_wn = ptr;
    TRY(upload(p, &ptr, stri.data(), stri.size()));
    d.src_tri = (const int4 *)ptr;
    TRY(upload(p, &ptr, lamT.data(), lamT.size()));
    d.lam = ptr;
    TRY(upload(p, &ptr, tg.data(), tg.size()));
    d.tgt_grid = ptr;
    TRY(upload(p, &ptr, p.tgt_perm.data(), p.tgt_perm.size()));
    d.tgt_perm = (const int *)ptr;

    // scratch
    const int64_t G = (int64_t)p.L[0] * p.L[1] * p.L[2];
    const int Kx = p.n[0] / 2;
    TRY(dalloc(p, &d.qbuf, sizeof(T) * p.Q));
    TRY(dalloc(p, &d.m4, 4 * sizeof(T) * p.N * slp::NEAR_STATES));
    TRY(dalloc(p, &d.phi_part, sizeof(T) * p.N * slp::NEAR_STATES));
    // far-field scratch for a batch of kf states (slp_far_batch)
    p.kf = slp_far_batch(p);
    d.ks = 1;
    d.st_grid = G;
    d.st_s1 = (int64_t)p.L[2] * p.L[1] * Kx;
    d.st_s2 = (int64_t)p.L[2] * p.n[1] * Kx;
    TRY(dalloc(p, &d.gridA, sizeof(T) * G * p.kf));
    TRY(dalloc(p, &d.gridB, sizeof(T) * G * p.kf));
    TRY(dalloc(p, &d.S1, sizeof(T2) * d.st_s1 * p.kf));
    TRY(dalloc(p, &d.S2, sizeof(T2) * d.st_s2 * p.kf));
    // grid A starts zero; rows outside the active region of S1, S2 and grid B
    // are never written, so they are cleared once here
    if (cudaMemset(d.gridA, 0, sizeof(T) * G * p.kf) != cudaSuccess ||
        cudaMemset(d.gridB, 0, sizeof(T) * G * p.kf) != cudaSuccess ||
        cudaMemset(d.S1, 0, sizeof(T2) * d.st_s1 * p.kf) != cudaSuccess ||
        cudaMemset(d.S2, 0, sizeof(T2) * d.st_s2 * p.kf) != cudaSuccess)
        return fail(SLP_ERR_CUDA, "cudaMemset failed");

    std::vector<T> Dt(p.Dtab.begin(), p.Dtab.end());
    TRY(upload(p, &ptr, Dt.data(), Dt.size()));
    d.Dtab = ptr;
    for (int a = 0; a < 3; ++a) {
        std::vector<T2> tw(p.L[a]);
        for (int t = 0; t < p.L[a]; ++t) {
            const double ang = 2.0 * PI * t / p.L[a];
            tw[t].x = (T)std::cos(ang);
            tw[t].y = (T)(-std::sin(ang));
        }
        TRY(upload(p, &ptr, tw.data(), tw.size()));
        d.tw[a] = ptr;
    }
    d.z0 = p.z0;
    d.nz_act = p.nz_act;
    TRY(upload(p, &ptr, p.plane_iv.data(), p.plane_iv.size()));
    d.plane_iv = (const int2 *)ptr;
    TRY(upload(p, &ptr, p.row_pairs.data(), p.row_pairs.size()));
    d.row_pairs = (const int *)ptr;
    d.n_row_pairs = (int)p.row_pairs.size();
    {
        // fused plane passes when both fit in shared memory
        int maxp = 0;
        for (const int2 &v : p.plane_iv) maxp = std::max(maxp, v.y / 2);
        int PB = 4;  // at least one pair per CTA of the four-CTA cluster
        while (PB < maxp) PB <<= 1;
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.device);
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p.device);
        const size_t sm = slp::fused_plane_smem(d, PB);
        const bool fits = maxp > 0 && sm <= std::min<size_t>((size_t)optin, 200 * 1024);
        const int want = p.opts.fuse_plane_passes;
        d.fuse_pb = (fits && (want == 1 || (want < 0 && p.nz_act >= 2 * nsm))) ? PB : 0;
        // fused column passes: equal y and z lengths the column engine
        // compiles (32..256), at most 512 threads a CTA, within shared memory
        d.yzy_g = d.yzy_zc = d.yzy_zp = 0;
        const int Ly = p.L[1];
        if (d.fuse_pb == 0 && Ly == p.L[2] && Ly >= 32 && Ly <= 256 && p.nz_act > 0 && d.Kx >= 1) {
            const int ZC = (p.nz_act + slp::YZY_CL - 1) / slp::YZY_CL;
            const int KC = p.n[1] / slp::YZY_CL;
            const int G = (std::max(ZC, KC) + 7) / 8;
            const int ZP = ZC + 1;
            const size_t ysm = slp::fused_column_smem(d, G, ZP);
            const bool yfits = G * Ly <= 512 && ysm <= std::min<size_t>((size_t)optin, 200 * 1024);
            const int ywant = p.opts.fuse_column_passes;
            // opt-in only: on the 128^3 sphere the three PDL-chained passes
            // measured 14.4 us for FY..IX against 15.4 us fused
            if (yfits && ywant == 1) {
                d.yzy_g = G;
                d.yzy_zc = ZC;
                d.yzy_zp = ZP;
            }
        }
    }
    TRY(upload(p, &ptr, p.spread_items.data(), p.spread_items.size()));
    d.spread_items = (const slp::TileItem *)ptr;
    d.n_spread = (int)p.spread_items.size();
    d.spread_chunk = 1;
    for (const auto &it : p.spread_items) d.spread_chunk = std::max(d.spread_chunk, it.end - it.begin);
    TRY(upload(p, &ptr, p.sgroups.data(), p.sgroups.size()));
    d.sgroups = (const int *)ptr;
    TRY(upload(p, &ptr, p.sgroup_off.data(), p.sgroup_off.size()));
    d.sgroup_off = (const int *)ptr;
    TRY(upload(p, &ptr, p.sgroup_cell.data(), p.sgroup_cell.size()));
    d.sgroup_cell = (const int *)ptr;
    d.wtab = nullptr;
    if (sizeof(T) == 4 && p.m <= 4 && p.Q > 0 && p.opts.spread_table > 0) {
        // FP32 table spread: window values of every sorted source, built once here
        void *wt = nullptr;
        TRY(dalloc(p, &wt, sizeof(float) * (size_t)p.Q * slp::spread_table_row(p.m)));
        TRY(cuda_status(slp::launch_wtab_build(d, (float *)wt, 0), "window table"));
        TRY(cuda_status(cudaDeviceSynchronize(), "window table"));
        d.wtab = wt;
    }
    d.wtab64_src = d.wtab64_tgt = nullptr;
    if (sizeof(T) == 8) {
        // FP64: the window values of every sorted source and target, built once
        // here (this GPU's FP64 rate makes the window's sqrt and sinh the
        // largest cost of the FP64 spread and gather); at most 2 GB
        const size_t per = sizeof(double) * 3 * 2 * (size_t)p.m;
        const size_t nsrc = p.opts.integration ? 0 : (size_t)p.Q;
        if (per * (nsrc + (size_t)p.N) <= ((size_t)2 << 30)) {
            void *ws = nullptr, *wt = nullptr;
            if (nsrc > 0) {
                TRY(dalloc(p, &ws, per * nsrc));
                TRY(cuda_status(slp::launch_wtab64_build(d, d.src_grid, (int64_t)nsrc, (double *)ws, 0), "window table"));
            }
            TRY(dalloc(p, &wt, std::max<size_t>(per * (size_t)p.N, 16)));
            TRY(cuda_status(slp::launch_wtab64_build(d, d.tgt_grid, p.N, (double *)wt, 0), "window table"));
            TRY(cuda_status(cudaDeviceSynchronize(), "window table"));
            d.wtab64_src = (const double *)ws;
            d.wtab64_tgt = (const double *)wt;
        }
    }
    TRY(upload(p, &ptr, p.gather_items.data(), p.gather_items.size()));
    d.gather_items = (const slp::TileItem *)ptr;
    d.n_gather = (int)p.gather_items.size();
    d.gather_chunk = p.gather_chunk;
    d.spread_dense = spread_dense(p) ? 1 : 0;
    TRY(upload(p, &ptr, p.near_items.data(), p.near_items.size()));
    d.near_items = (const slp::NearItem *)ptr;
    d.n_near = (int)p.near_items.size();
    TRY(upload(p, &ptr, p.near_ranges.data(), p.near_ranges.size()));
    d.near_ranges = (const int2 *)ptr;
    TRY(upload(p, &ptr, p.near_blk_first.data(), p.near_blk_first.size()));
    p.d_blk_first = (int *)ptr;
    if (p.opts.deterministic) TRY(dalloc(p, &d.phi_near, sizeof(T) * 32 * std::max<size_t>(1, p.near_items.size())));
    d.integration = p.opts.integration ? 1 : 0;
    if (d.integration) {
        // triangles: vertex ids and n_j / 3 for the element charges of nodal input
        std::vector<int4> tv(p.M);
        std::vector<T4> n3(p.M);
        for (int64_t j = 0; j < p.M; ++j) {
            tv[j] = make_int4(p.T[3 * j], p.T[3 * j + 1], p.T[3 * j + 2], 0);
            n3[j].x = (T)(p.nrm[3 * j] / 3.0);
            n3[j].y = (T)(p.nrm[3 * j + 1] / 3.0);
            n3[j].z = (T)(p.nrm[3 * j + 2] / 3.0);
            n3[j].w = T(0);
        }
        TRY(upload(p, &ptr, tv.data(), tv.size()));
        d.tri_v = (const int4 *)ptr;
        TRY(upload(p, &ptr, n3.data(), n3.size()));
        d.tri_n3 = ptr;
        TRY(dalloc(p, &d.gbuf, sizeof(T) * (size_t)std::max<int64_t>(p.M, 1)));
    }
    if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
        std::vector<T> w(p.es_w.size()), g(p.es_g.size());
        for (size_t k = 0; k < w.size(); ++k) {
            w[k] = (T)(p.es_w[k] / p.P[0]);
            g[k] = (T)(p.es_g[k] / (p.P[0] * p.P[0]));
        }
        TRY(upload(p, &ptr, w.data(), w.size()));
        d.es_w = ptr;
        TRY(upload(p, &ptr, g.data(), g.size()));
        d.es_g = ptr;
        d.es_n = (int)w.size();
    }
    if (p.kernel_mode == SLP_KERNEL_SEPARABLE) {
        for (int a = 0; a < 3; ++a) {
            std::vector<T> h(p.sep_h[a].begin(), p.sep_h[a].end());
            TRY(upload(p, &ptr, h.data(), h.size()));
            d.sep_h[a] = ptr;
            d.sep_nh[a] = (int)h.size();
        }
        d.sep_A = 4.0 * PI * p.sep_A;
    }
    void *errp;
    TRY(dalloc(p, &errp, sizeof(int)));
    if (cudaMemset(errp, 0, sizeof(int)) != cudaSuccess) return fail(SLP_ERR_CUDA, "cudaMemset failed");
    d.err = (int *)errp;
    // staging buffers for slp_eval_host
    TRY(dalloc(p, &p.d_stage_in, sizeof(T) * 3 * std::max(p.Q, p.N)));
    TRY(dalloc(p, &p.d_stage_phi, sizeof(T) * p.N));
    for (int k = 0; k < 2; ++k) {
        TRY(dalloc(p, &p.d_astage_in[k], sizeof(T) * 3 * std::max(p.Q, p.N)));
        TRY(dalloc(p, &p.d_astage_phi[k], sizeof(T) * p.N));
    }
    // on-the-fly near field: charges, spread, 5 FFT passes (3 when the plane
    // passes are fused), gather, and either zeroing + atomic near field or
    // near field + ordered reduction
    p.launches_per_eval = d.fuse_pb > 0 ? 8 : (d.yzy_g > 0 ? 8 : 10);
    return SLP_OK;
}

void free_device(slp_plan_s &p) {
    if (p.device < 0) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p.device);
    slp_exec_destroy(p.exec);
    for (int k = 0; k < 2; ++k) {
        if (p.ev_in[k]) cudaEventDestroy(p.ev_in[k]);
        if (p.ev_eval[k]) cudaEventDestroy(p.ev_eval[k]);
        if (p.ev_out[k]) cudaEventDestroy(p.ev_out[k]);
    }
    if (p.cs_in) cudaStreamDestroy(p.cs_in);
    if (p.cs_out) cudaStreamDestroy(p.cs_out);
    for (void *a : p.allocs) cudaFree(a);
    p.allocs.clear();
    cudaSetDevice(prev);
}

slp_status cuda_status(cudaError_t e, const char *what);

// Temporary device buffer released at scope exit (plan-time only).
struct TmpBuf {
    void *p = nullptr;
    ~TmpBuf() {
        if (p) cudaFree(p);
    }
};

template <typename S> slp_status tmp_upload(TmpBuf &b, const S *src, size_t n) {
    const size_t bytes = std::max<size_t>(16, n * sizeof(S));
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SLP_ERR_OOM : SLP_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    if (n && cudaMemcpy(b.p, src, n * sizeof(S), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(SLP_ERR_CUDA, "cudaMemcpy failed");
    return SLP_OK;
}

// Assemble the vertex-based near-field operator W (see k_near.cu) on the
// device.  Candidate vertices of each target block: aligned 2x2x2-cell bins
// of the sorted targets whose bounding box lies within eps + r_adj of the
// block, r_adj being the largest distance from a vertex to a quadrature point
// of an adjacent triangle.  Returns SLP_OK without building when the matrix
// would exceed the memory budget (near_mode stays ON_THE_FLY).
// Candidates of the near-field operators: for every target block of the
// near-field work list, the ranges of sorted vertices (2x2x2-cell bins,
// contiguous in the sort) whose bounding boxes lie within rad of the block's
// bounding box (all vertices when all_pairs), plus the vertex -> (triangle,
// corner) adjacency and the sorted targets' positions relative to the centre.
struct NearCandidates {
    std::vector<int> vt_ptr, vt_ent;
    std::vector<double4> tgt;
    std::vector<int> tgt_block, blk_r0;
    std::vector<int2> ranges;
};

// Bins of the sorted targets (vertices): runs of one aligned 2x2x2-cell block,
// contiguous in the sort, with their bounding boxes.
struct TargetBins {
    struct Bin {
        int b, e;
        double lo[3], hi[3];
    };
    std::vector<Bin> bins;
    std::unordered_map<uint64_t, int> bin_of;
};

void target_bins(const slp_plan_s &p, const std::vector<uint64_t> &tkeys, const std::vector<double4> &tgt,
                 TargetBins &tb) {
    const int64_t N = p.N;
    tb.bins.clear();
    tb.bin_of.clear();
    for (int64_t i = 0; i < N;) {
        int64_t j = i;
        const uint64_t bk = tkeys[i] >> 3;
        while (j < N && (tkeys[j] >> 3) == bk) ++j;
        TargetBins::Bin bn;
        bn.b = (int)i;
        bn.e = (int)j;
        for (int d = 0; d < 3; ++d) {
            bn.lo[d] = 1e300;
            bn.hi[d] = -1e300;
        }
        for (int64_t k = i; k < j; ++k) {
            const double x[3] = {tgt[k].x, tgt[k].y, tgt[k].z};
            for (int d = 0; d < 3; ++d) {
                bn.lo[d] = std::min(bn.lo[d], x[d]);
                bn.hi[d] = std::max(bn.hi[d], x[d]);
            }
        }
        const uint32_t packed = (uint32_t)p.tgt_grid[4 * i + 3];
        const uint64_t bx = (packed & 1023) / 2, by = ((packed >> 10) & 1023) / 2, bz = ((packed >> 20) & 1023) / 2;
        tb.bin_of[(bz << 40) | (by << 20) | bx] = (int)tb.bins.size();
        tb.bins.push_back(bn);
        i = j;
    }
}

// Append to `ranges` the runs of sorted vertices in bins within rad of the box [lo, hi].
void bins_within(const slp_plan_s &p, const TargetBins &tb, const double *lo, const double *hi, double rad,
                 std::vector<int2> &ranges) {
    const size_t first = ranges.size();
    int b0[3], b1[3];
    for (int d = 0; d < 3; ++d) {
        const double h = p.P[d] / p.L[d];
        const double u0 = (lo[d] - rad) / h + 0.5 * p.L[d], u1 = (hi[d] + rad) / h + 0.5 * p.L[d];
        b0[d] = std::max(0, (int)std::floor(u0) - 1) / 2;
        b1[d] = std::min(p.L[d] - 1, (int)std::floor(u1) + 1) / 2;
    }
    std::vector<int> found;
    for (int bz = b0[2]; bz <= b1[2]; ++bz)
        for (int by = b0[1]; by <= b1[1]; ++by)
            for (int bx = b0[0]; bx <= b1[0]; ++bx) {
                auto itb = tb.bin_of.find(((uint64_t)bz << 40) | ((uint64_t)by << 20) | (uint64_t)bx);
                if (itb == tb.bin_of.end()) continue;
                const TargetBins::Bin &bn = tb.bins[itb->second];
                double d2 = 0;
                for (int d = 0; d < 3; ++d) {
                    const double g = std::max(0.0, std::max(bn.lo[d] - hi[d], lo[d] - bn.hi[d]));
                    d2 += g * g;
                }
                if (d2 <= rad * rad) found.push_back(itb->second);
            }
    std::sort(found.begin(), found.end(), [&](int a2, int b2) { return tb.bins[a2].b < tb.bins[b2].b; });
    for (int f : found) {
        if (ranges.size() > first && ranges.back().y == tb.bins[f].b)
            ranges.back().y = tb.bins[f].e;
        else
            ranges.push_back(make_int2(tb.bins[f].b, tb.bins[f].e));
    }
}

void near_candidates(const slp_plan_s &p, const std::vector<uint64_t> &tkeys, double rad, bool all_pairs,
                     NearCandidates &c) {
    const int64_t N = p.N, M = p.M;
    // vertex -> adjacent (triangle, local vertex)
    std::vector<int> &vt_ptr = c.vt_ptr, &vt_ent = c.vt_ent;
    vt_ptr.assign(N + 1, 0);
    vt_ent.assign(3 * M, 0);
    for (int64_t j = 0; j < M; ++j)
        for (int a = 0; a < 3; ++a) vt_ptr[p.T[3 * j + a] + 1]++;
    for (int64_t i = 0; i < N; ++i) vt_ptr[i + 1] += vt_ptr[i];
    {
        std::vector<int> fillc(vt_ptr.begin(), vt_ptr.end() - 1);
        for (int64_t j = 0; j < M; ++j)
            for (int a = 0; a < 3; ++a) vt_ent[fillc[p.T[3 * j + a]]++] = (int)(j * 4 + a);
    }
    // target physical positions (sorted, relative to the centre)
    std::vector<double4> &tgt = c.tgt;
    tgt.resize(N);
    for (int64_t i = 0; i < N; ++i) {
        const double *v = &p.V[3 * (int64_t)p.tgt_perm[i]];
        tgt[i] = make_double4(v[0] - p.ctr[0], v[1] - p.ctr[1], v[2] - p.ctr[2], 0.0);
    }
    // target blocks (as in the near-field work list)
    const int nblk = (int)p.near_blk_first.size() - 1;
    std::vector<int> &tgt_block = c.tgt_block, &blk_r0 = c.blk_r0;
    tgt_block.assign(N, 0);
    blk_r0.assign(nblk + 1, 0);
    std::vector<int2> &ranges = c.ranges;
    ranges.clear();
    TargetBins tb;
    if (!all_pairs) target_bins(p, tkeys, tgt, tb);
    for (int b = 0; b < nblk; ++b) {
        const slp::NearItem &it = p.near_items[p.near_blk_first[b]];
        for (int t = it.tbegin; t < it.tbegin + it.tcount; ++t) tgt_block[t] = b;
        blk_r0[b] = (int)ranges.size();
        if (all_pairs) {
            ranges.push_back(make_int2(0, (int)N));
            continue;
        }
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int t = it.tbegin; t < it.tbegin + it.tcount; ++t) {
            const double x[3] = {tgt[t].x, tgt[t].y, tgt[t].z};
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], x[d]);
                hi[d] = std::max(hi[d], x[d]);
            }
        }
        bins_within(p, tb, lo, hi, rad, ranges);
    }
    blk_r0[nblk] = (int)ranges.size();
}

slp_status build_near_matrix(slp_plan_s &p, const std::vector<uint64_t> &tkeys) {
    const int64_t N = p.N, M = p.M, q = p.q;
    double r_adj = 0.0;
    for (int64_t j = 0; j < M; ++j)
        for (int a = 0; a < 3; ++a) {
            const double *v = &p.V[3 * p.T[3 * j + a]];
            for (int s2 = 0; s2 < q; ++s2) {
                const double *y = &p.y[3 * (j * q + s2)];
                const double d = std::sqrt((v[0] - y[0]) * (v[0] - y[0]) + (v[1] - y[1]) * (v[1] - y[1]) +
                                           (v[2] - y[2]) * (v[2] - y[2]));
                r_adj = std::max(r_adj, d);
            }
        }
    const bool all_pairs = p.kernel_mode == SLP_KERNEL_SEPARABLE || !(p.eps < p.diam);
    const double rad = all_pairs ? INFINITY : p.eps + r_adj * (1.0 + 1e-9) + 1e-12 * p.diam;
    NearCandidates cand;
    near_candidates(p, tkeys, rad, all_pairs, cand);
    std::vector<int> &vt_ptr = cand.vt_ptr, &vt_ent = cand.vt_ent, &tgt_block = cand.tgt_block, &blk_r0 = cand.blk_r0;
    std::vector<double4> &tgt = cand.tgt;
    std::vector<int2> &ranges = cand.ranges;

    // device inputs
    std::vector<double4> src(p.Q), nrm(M);
    for (int64_t k = 0; k < p.Q; ++k)
        src[k] = make_double4(p.y[3 * k] - p.ctr[0], p.y[3 * k + 1] - p.ctr[1], p.y[3 * k + 2] - p.ctr[2], p.wk[k]);
    for (int64_t j = 0; j < M; ++j) nrm[j] = make_double4(p.nrm[3 * j], p.nrm[3 * j + 1], p.nrm[3 * j + 2], 0.0);
    TmpBuf b_tgt, b_blk, b_r0, b_rng, b_vtp, b_vte, b_src, b_nrm, b_lam, b_h[3], b_cnt, b_pairs;
    TRY(tmp_upload(b_tgt, tgt.data(), tgt.size()));
    TRY(tmp_upload(b_blk, tgt_block.data(), tgt_block.size()));
    TRY(tmp_upload(b_r0, blk_r0.data(), blk_r0.size()));
    TRY(tmp_upload(b_rng, ranges.data(), ranges.size()));
    TRY(tmp_upload(b_vtp, vt_ptr.data(), vt_ptr.size()));
    TRY(tmp_upload(b_vte, vt_ent.data(), vt_ent.size()));
    TRY(tmp_upload(b_src, src.data(), src.size()));
    TRY(tmp_upload(b_nrm, nrm.data(), nrm.size()));
    TRY(tmp_upload(b_lam, p.lam.data(), p.lam.size()));
    std::vector<int64_t> zeros(N + 1, 0);
    TRY(tmp_upload(b_cnt, zeros.data(), zeros.size()));
    TRY(tmp_upload(b_pairs, zeros.data(), zeros.size()));
    slp::NMBuild nb;
    memset(&nb, 0, sizeof nb);
    nb.tgt = (const double4 *)b_tgt.p;
    nb.tgt_perm = p.dp.tgt_perm;
    nb.tgt_block = (const int *)b_blk.p;
    nb.blk_r0 = (const int *)b_r0.p;
    nb.ranges = (const int2 *)b_rng.p;
    nb.vt_ptr = (const int *)b_vtp.p;
    nb.vt_ent = (const int *)b_vte.p;
    nb.src = (const double4 *)b_src.p;
    nb.nrm = (const double4 *)b_nrm.p;
    nb.lam = (const double *)b_lam.p;
    nb.q = p.q;
    nb.N = N;
    nb.eps2 = std::isfinite(p.eps) ? p.eps * p.eps : 1e300;
    nb.inv_s_sqrt2 = p.sigma_g > 0 ? 1.0 / (p.sigma_g * std::sqrt(2.0)) : 0.0;
    nb.kernel_mode = p.kernel_mode;
    if (p.kernel_mode == SLP_KERNEL_SEPARABLE) {
        for (int a = 0; a < 3; ++a) {
            TRY(tmp_upload(b_h[a], p.sep_h[a].data(), p.sep_h[a].size()));
            nb.sep_h[a] = (const double *)b_h[a].p;
            nb.sep_nh[a] = (int)p.sep_h[a].size();
        }
        nb.sep_A4pi = 4.0 * PI * p.sep_A;
    }
    for (int a = 0; a < 3; ++a) nb.P[a] = p.P[a];
    TmpBuf b_esw, b_esg;
    if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
        std::vector<double> w(p.es_w.size()), g(p.es_g.size());
        for (size_t k = 0; k < w.size(); ++k) {
            w[k] = p.es_w[k] / p.P[0];
            g[k] = p.es_g[k] / (p.P[0] * p.P[0]);
        }
        TRY(tmp_upload(b_esw, w.data(), w.size()));
        TRY(tmp_upload(b_esg, g.data(), g.size()));
        nb.es_w = (const double *)b_esw.p;
        nb.es_g = (const double *)b_esg.p;
        nb.es_n = (int)w.size();
    }
    TRY(cuda_status(slp::launch_nm_build(nb, 0, p.prec, (int64_t *)b_cnt.p, (int64_t *)b_pairs.p, nullptr, nullptr, 0),
                    "near matrix count"));
    std::vector<int64_t> cnt(N), prs(N);
    TRY(cuda_status(cudaMemcpy(cnt.data(), b_cnt.p, sizeof(int64_t) * N, cudaMemcpyDeviceToHost), "count copy"));
    TRY(cuda_status(cudaMemcpy(prs.data(), b_pairs.p, sizeof(int64_t) * N, cudaMemcpyDeviceToHost), "pairs copy"));
    std::vector<int64_t> rowptr(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) rowptr[i + 1] = rowptr[i] + cnt[i];
    const int64_t nnz = rowptr[N];
    p.near_pairs_within = 0;
    for (int64_t i = 0; i < N; ++i) p.near_pairs_within += prs[i];
    const size_t vbytes = (size_t)nnz * (p.prec == 64 ? 32 : 16);
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    if (vbytes > ((size_t)24 << 30) || vbytes > freeb / 2) return SLP_OK;  // budget: keep the on-the-fly near field
    void *ptr = nullptr;
    TRY(upload(p, &ptr, rowptr.data(), rowptr.size()));
    p.dp.nm_rowptr = (const int64_t *)ptr;
    TRY(dalloc(p, &ptr, vbytes));
    p.dp.nm_val = ptr;
    TRY(cuda_status(slp::launch_nm_build(nb, 1, p.prec, nullptr, nullptr, p.dp.nm_rowptr, ptr, 0), "near matrix fill"));
    TRY(cuda_status(cudaDeviceSynchronize(), "near matrix build"));
    p.dp.nm_nnz = nnz;
    p.nm_nnz = nnz;
    p.near_mode = SLP_NEAR_PRECOMPUTED;
    // prep, spread (charges fused), 5 (fused: 3) FFT passes, gather, near-field product
    p.launches_per_eval = p.dp.fuse_pb > 0 ? 7 : (p.dp.yzy_g > 0 ? 7 : 9);
    return SLP_OK;
}

// Duffy-Gauss rule of the triangle-integrated plans on the reference triangle
// {0 <= b <= a <= 1} (area 1/2): a = s, b = s t for Gauss-Legendre nodes s, t
// on [0, 1] and weight w_s w_t s (the Jacobian of (s, t) -> (s, s t)).  The
// Gauss-Legendre nodes are roots of P_n found by Newton's method from
// cos(pi (i + 3/4) / (n + 1/2)), with weights 2 / ((1 - x^2) P_n'(x)^2).
void tri_rule(int n, std::vector<double> &ra, std::vector<double> &rb, std::vector<double> &rw) {
    std::vector<double> x(n), w(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);  // [0, 1]
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // half of the [-1, 1] weight
    }
    ra.clear();
    rb.clear();
    rw.clear();
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            ra.push_back(x[i]);
            rb.push_back(x[i] * x[k]);
            rw.push_back(w[i] * w[k] * x[i]);
        }
}

// Deterministic point plans: the gridding matrix of the sorted point sources,
// CSR over grid points, the entries of a row in ascending source order (the
// spread then writes every grid point once, with a fixed summation order).
// Kept when it needs at most 24 GiB and half of the free device memory;
// otherwise the plan keeps the tiled spread (results repeat to rounding level).
template <typename T> slp_status build_point_matrix(slp_plan_s &p) {
    const int64_t G = (int64_t)p.L[0] * p.L[1] * p.L[2];
    const int64_t W = 2 * p.m;
    const size_t need = (size_t)p.Q * W * W * W * (sizeof(T) + sizeof(int));
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    if (G > ((int64_t)1 << 28) || need > ((size_t)24 << 30) || need > freeb / 2) return SLP_OK;
    std::vector<double4> src(p.Q);
    for (int64_t k = 0; k < p.Q; ++k)
        src[k] = make_double4(p.src_grid[4 * k], p.src_grid[4 * k + 1], p.src_grid[4 * k + 2], p.src_grid[4 * k + 3]);
    TmpBuf b_src, b_cnt;
    TRY(tmp_upload(b_src, src.data(), src.size()));
    {
        std::vector<int> zeros(G, 0);
        TRY(tmp_upload(b_cnt, zeros.data(), zeros.size()));
    }
    slp::PointBuild pb;
    memset(&pb, 0, sizeof pb);
    pb.src = (const double4 *)b_src.p;
    pb.Q = p.Q;
    pb.m = p.m;
    for (int d = 0; d < 3; ++d) pb.L[d] = p.L[d];
    pb.beta = KB_B * p.m;
    pb.isb = 1.0 / std::sinh(pb.beta);
    pb.err = p.dp.err;
    TRY(cuda_status(slp::launch_pmat_count(pb, (int *)b_cnt.p, 0), "point gridding matrix count"));
    TRY(cuda_status(cudaDeviceSynchronize(), "point gridding matrix count"));
    std::vector<int> cnt(G), slot_of(G, -1);
    TRY(cuda_status(cudaMemcpy(cnt.data(), b_cnt.p, sizeof(int) * G, cudaMemcpyDeviceToHost), "count copy"));
    std::vector<int64_t> rowptr(1, 0), rowidx;
    for (int64_t g = 0; g < G; ++g)
        if (cnt[g] > 0) {
            slot_of[g] = (int)rowidx.size();
            rowidx.push_back(g);
            rowptr.push_back(rowptr.back() + cnt[g]);
        }
    const int64_t nrows = (int64_t)rowidx.size(), nnz = rowptr.back();
    void *ptr = nullptr;
    TRY(upload(p, &ptr, rowptr.data(), rowptr.size()));
    p.dp.am_rowptr = (const int64_t *)ptr;
    TRY(upload(p, &ptr, rowidx.data(), rowidx.size()));
    p.dp.am_row = (const int64_t *)ptr;
    TRY(dalloc(p, &ptr, sizeof(int) * (size_t)std::max<int64_t>(nnz, 1)));
    p.dp.am_col = (const int *)ptr;
    TRY(dalloc(p, &ptr, sizeof(T) * (size_t)std::max<int64_t>(nnz, 1)));
    p.dp.am_val = ptr;
    p.dp.am_rows = nrows;
    TmpBuf b_slot, b_cur;
    TRY(tmp_upload(b_slot, slot_of.data(), slot_of.size()));
    {
        std::vector<int> z(std::max<int64_t>(nrows, 1), 0);
        TRY(tmp_upload(b_cur, z.data(), z.size()));
    }
    TRY(cuda_status(slp::launch_pmat_fill(pb, p.prec, (const int *)b_slot.p, p.dp.am_rowptr, (int *)b_cur.p,
                                          (int *)p.dp.am_col, (void *)p.dp.am_val, 0), "point gridding matrix fill"));
    TRY(cuda_status(slp::launch_csr_sort(nrows, p.prec, p.dp.am_rowptr, (int *)p.dp.am_col, (void *)p.dp.am_val, 0),
                    "point gridding matrix order"));
    TRY(cuda_status(cudaDeviceSynchronize(), "point gridding matrix fill"));
    int code = 0;
    TRY(cuda_status(cudaMemcpy(&code, p.dp.err, sizeof(int), cudaMemcpyDeviceToHost), "status"));
    if (code != 0) return fail(SLP_ERR_CUDA, "point gridding matrix: device status word %d", code);
    p.am_nnz = nnz;
    p.dp.det_spread = 1;
    return SLP_OK;
}

// Triangle-integrated plans: the gridding matrix A (CSR over grid points) and
// the near-field matrix over triangles (CSR over sorted targets), both
// assembled on the device in FP64 and stored at the plan precision.
template <typename T> slp_status build_tri_matrices(slp_plan_s &p, const std::vector<uint64_t> &tkeys) {
    const int64_t N = p.N, M = p.M;
    const int64_t G = (int64_t)p.L[0] * p.L[1] * p.L[2];
    if (G > ((int64_t)1 << 27)) return fail(SLP_ERR_UNSUPPORTED, "triangle integrals need a grid of at most 2^27 points");
    std::vector<double3> ug(N), xp(N);
    for (int64_t i = 0; i < N; ++i) {
        const double *v = &p.V[3 * i];
        xp[i] = make_double3(v[0] - p.ctr[0], v[1] - p.ctr[1], v[2] - p.ctr[2]);
        ug[i] = make_double3((v[0] - p.ctr[0]) / p.P[0] * p.L[0] + 0.5 * p.L[0],
                             (v[1] - p.ctr[1]) / p.P[1] * p.L[1] + 0.5 * p.L[1],
                             (v[2] - p.ctr[2]) / p.P[2] * p.L[2] + 0.5 * p.L[2]);
    }
    std::vector<int4> tri(M);
    for (int64_t j = 0; j < M; ++j) tri[j] = make_int4(p.T[3 * j], p.T[3 * j + 1], p.T[3 * j + 2], 0);
    std::vector<double> ra, rb, rw;
    tri_rule(8, ra, rb, rw);
    TmpBuf b_ug, b_xp, b_tri, b_ra, b_rb, b_rw, b_cnt;
    TRY(tmp_upload(b_ug, ug.data(), ug.size()));
    TRY(tmp_upload(b_xp, xp.data(), xp.size()));
    TRY(tmp_upload(b_tri, tri.data(), tri.size()));
    TRY(tmp_upload(b_ra, ra.data(), ra.size()));
    TRY(tmp_upload(b_rb, rb.data(), rb.size()));
    TRY(tmp_upload(b_rw, rw.data(), rw.size()));
    slp::TriBuildA ba;
    memset(&ba, 0, sizeof ba);
    ba.ugrid = (const double3 *)b_ug.p;
    ba.xphys = (const double3 *)b_xp.p;
    ba.tri = (const int4 *)b_tri.p;
    ba.M = M;
    ba.NV = N;
    ba.m = p.m;
    for (int d = 0; d < 3; ++d) ba.L[d] = p.L[d];
    ba.beta = KB_B * p.m;
    ba.isb = 1.0 / std::sinh(ba.beta);
    ba.ra = (const double *)b_ra.p;
    ba.rb = (const double *)b_rb.p;
    ba.rw = (const double *)b_rw.p;
    ba.np = (int)ra.size();
    ba.err = p.dp.err;
    // the status word of the plan is clear here; the assembly kernels report into it
    auto status = [&](const char *what) -> slp_status {
        int code = 0;
        TRY(cuda_status(cudaDeviceSynchronize(), what));
        TRY(cuda_status(cudaMemcpy(&code, p.dp.err, sizeof(int), cudaMemcpyDeviceToHost), what));
        if (code == slp::DEV_ERR_BAD_ITEM)
            return fail(SLP_ERR_UNSUPPORTED, "%s: a triangle spans more than %d grid cells", what, slp::TRI_BOX - 2 * p.m);
        if (code != 0) return fail(SLP_ERR_CUDA, "%s: device status word %d", what, code);
        return SLP_OK;
    };
    {
        std::vector<int> zeros(G, 0);
        TRY(tmp_upload(b_cnt, zeros.data(), zeros.size()));
    }
    TRY(cuda_status(slp::launch_amat_count(ba, (int *)b_cnt.p, 0), "gridding matrix count"));
    TRY(status("gridding matrix count"));
    std::vector<int> cnt(G), slot_of(G, -1);
    TRY(cuda_status(cudaMemcpy(cnt.data(), b_cnt.p, sizeof(int) * G, cudaMemcpyDeviceToHost), "count copy"));
    std::vector<int64_t> rowptr(1, 0), rowidx;
    for (int64_t g = 0; g < G; ++g)
        if (cnt[g] > 0) {
            slot_of[g] = (int)rowidx.size();
            rowidx.push_back(g);
            rowptr.push_back(rowptr.back() + cnt[g]);
        }
    const int64_t nrows = (int64_t)rowidx.size(), annz = rowptr.back();
    void *ptr = nullptr;
    TRY(upload(p, &ptr, rowptr.data(), rowptr.size()));
    p.dp.am_rowptr = (const int64_t *)ptr;
    TRY(upload(p, &ptr, rowidx.data(), rowidx.size()));
    p.dp.am_row = (const int64_t *)ptr;
    TRY(dalloc(p, &ptr, sizeof(int) * (size_t)std::max<int64_t>(annz, 1)));
    p.dp.am_col = (const int *)ptr;
    TRY(dalloc(p, &ptr, sizeof(T) * (size_t)std::max<int64_t>(annz, 1)));
    p.dp.am_val = ptr;
    p.dp.am_rows = nrows;
    {
        TmpBuf b_slot, b_cur;
        TRY(tmp_upload(b_slot, slot_of.data(), slot_of.size()));
        std::vector<int> z(std::max<int64_t>(nrows, 1), 0);
        TRY(tmp_upload(b_cur, z.data(), z.size()));
        TRY(cuda_status(slp::launch_amat_fill(ba, p.prec, (const int *)b_slot.p, p.dp.am_rowptr, (int *)b_cur.p,
                                              (int *)p.dp.am_col, (void *)p.dp.am_val, 0), "gridding matrix fill"));
        TRY(cuda_status(slp::launch_csr_sort(nrows, p.prec, p.dp.am_rowptr, (int *)p.dp.am_col, (void *)p.dp.am_val, 0),
                        "gridding matrix order"));
        TRY(status("gridding matrix fill"));
    }
    p.am_nnz = annz;

    // near-field matrix: every triangle within eps of the target (point-triangle distance)
    double emax = 0.0;
    for (int64_t j = 0; j < M; ++j)
        for (int a = 0; a < 3; ++a) {
            const double *u = &p.V[3 * (int64_t)p.T[3 * j + a]], *v = &p.V[3 * (int64_t)p.T[3 * j + (a + 1) % 3]];
            emax = std::max(emax, std::sqrt((u[0] - v[0]) * (u[0] - v[0]) + (u[1] - v[1]) * (u[1] - v[1]) +
                                            (u[2] - v[2]) * (u[2] - v[2])));
        }
    const bool all_pairs = p.kernel_mode == SLP_KERNEL_SEPARABLE || !(p.eps < p.diam);
    const double rad = all_pairs ? INFINITY : p.eps + emax * (1.0 + 1e-9) + 1e-12 * p.diam;
    NearCandidates cand;
    near_candidates(p, tkeys, rad, all_pairs, cand);
    std::vector<int> inv(N), tmin(M);
    for (int64_t i = 0; i < N; ++i) inv[p.tgt_perm[i]] = (int)i;
    for (int64_t j = 0; j < M; ++j)
        tmin[j] = std::min(inv[p.T[3 * j]], std::min(inv[p.T[3 * j + 1]], inv[p.T[3 * j + 2]]));
    std::vector<double3> tg(N);
    for (int64_t i = 0; i < N; ++i) tg[i] = make_double3(cand.tgt[i].x, cand.tgt[i].y, cand.tgt[i].z);
    TmpBuf b_tg, b_blk, b_r0, b_rng, b_vtp, b_vte, b_tmin, b_h[3], b_esw, b_esg, b_ncnt;
    TRY(tmp_upload(b_tg, tg.data(), tg.size()));
    TRY(tmp_upload(b_blk, cand.tgt_block.data(), cand.tgt_block.size()));
    TRY(tmp_upload(b_r0, cand.blk_r0.data(), cand.blk_r0.size()));
    TRY(tmp_upload(b_rng, cand.ranges.data(), std::max<size_t>(cand.ranges.size(), 1)));
    TRY(tmp_upload(b_vtp, cand.vt_ptr.data(), cand.vt_ptr.size()));
    TRY(tmp_upload(b_vte, cand.vt_ent.data(), cand.vt_ent.size()));
    TRY(tmp_upload(b_tmin, tmin.data(), tmin.size()));
    slp::TriBuildN bn;
    memset(&bn, 0, sizeof bn);
    bn.tgt = (const double3 *)b_tg.p;
    bn.tgt_perm = p.dp.tgt_perm;
    bn.tgt_block = (const int *)b_blk.p;
    bn.blk_r0 = (const int *)b_r0.p;
    bn.ranges = (const int2 *)b_rng.p;
    bn.vt_ptr = (const int *)b_vtp.p;
    bn.vt_ent = (const int *)b_vte.p;
    bn.tri_min_sorted = (const int *)b_tmin.p;
    bn.xphys = (const double3 *)b_xp.p;
    bn.tri = (const int4 *)b_tri.p;
    bn.N = N;
    bn.eps = std::isfinite(p.eps) ? p.eps : 1e300;
    bn.kernel_mode = p.kernel_mode;
    bn.inv_s_sqrt2 = p.sigma_g > 0 ? 1.0 / (p.sigma_g * std::sqrt(2.0)) : 0.0;
    if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
        std::vector<double> w(p.es_w.size()), g(p.es_g.size());
        for (size_t k = 0; k < w.size(); ++k) {
            w[k] = p.es_w[k] / p.P[0];
            g[k] = p.es_g[k] / (p.P[0] * p.P[0]);
        }
        TRY(tmp_upload(b_esw, w.data(), w.size()));
        TRY(tmp_upload(b_esg, g.data(), g.size()));
        bn.es_w = (const double *)b_esw.p;
        bn.es_g = (const double *)b_esg.p;
        bn.es_n = (int)w.size();
    }
    if (p.kernel_mode == SLP_KERNEL_SEPARABLE) {
        for (int a = 0; a < 3; ++a) {
            TRY(tmp_upload(b_h[a], p.sep_h[a].data(), p.sep_h[a].size()));
            bn.sep_h[a] = (const double *)b_h[a].p;
            bn.sep_nh[a] = (int)p.sep_h[a].size();
        }
        bn.sep_A4pi = 4.0 * PI * p.sep_A;
    }
    for (int a = 0; a < 3; ++a) bn.P[a] = p.P[a];
    bn.ra = (const double *)b_ra.p;
    bn.rb = (const double *)b_rb.p;
    bn.rw = (const double *)b_rw.p;
    bn.np = (int)ra.size();
    bn.err = p.dp.err;
    {
        std::vector<int64_t> z(N + 1, 0);
        TRY(tmp_upload(b_ncnt, z.data(), z.size()));
    }
    TRY(cuda_status(slp::launch_nmt_build(bn, 0, p.prec, (int64_t *)b_ncnt.p, nullptr, nullptr, nullptr, 0),
                    "near-field matrix count"));
    TRY(status("near-field matrix count"));
    std::vector<int64_t> ncnt(N), nrp(N + 1, 0);
    TRY(cuda_status(cudaMemcpy(ncnt.data(), b_ncnt.p, sizeof(int64_t) * N, cudaMemcpyDeviceToHost), "count copy"));
    for (int64_t i = 0; i < N; ++i) nrp[i + 1] = nrp[i] + ncnt[i];
    const int64_t nnnz = nrp[N];
    TRY(upload(p, &ptr, nrp.data(), nrp.size()));
    p.dp.nt_rowptr = (const int64_t *)ptr;
    TRY(dalloc(p, &ptr, sizeof(int) * (size_t)std::max<int64_t>(nnnz, 1)));
    p.dp.nt_col = (const int *)ptr;
    TRY(dalloc(p, &ptr, sizeof(T) * (size_t)std::max<int64_t>(nnnz, 1)));
    p.dp.nt_val = ptr;
    TRY(cuda_status(slp::launch_nmt_build(bn, 1, p.prec, nullptr, p.dp.nt_rowptr, (int *)p.dp.nt_col,
                                          (void *)p.dp.nt_val, 0), "near-field matrix fill"));
    TRY(status("near-field matrix fill"));
    p.nt_nnz = nnnz;
    p.near_mode = SLP_NEAR_PRECOMPUTED;
    // element charges (nodal input), gridding product, 5 FFT passes, near-field product, gather
    p.launches_per_eval = 9;
    return SLP_OK;
}

}  // namespace

// A probe set: extra evaluation points of a plan (see slp_probe_create).
struct slp_probe_s {
    slp_plan_s *plan = nullptr;
    int device = 0;
    int64_t n = 0;
    int64_t near_nnz = 0;
    slp::DevPlan view;            // the plan's view with the probes as targets
    std::vector<void *> allocs;
};

namespace {

template <typename T> slp_status probe_build(slp_plan_s &p, const double *pts, int64_t n, slp_probe_s &pr) {
    typedef typename V4<T>::t T4;
    const bool tri = p.opts.integration != 0;
    // sorted probes in the plan's cells, their gather items
    std::vector<int32_t> perm;
    std::vector<double> grid;
    std::vector<uint64_t> keys;
    sort_points(p, pts, n, p.TSg, perm, grid, keys);
    // every probe's window rows must lie in the region the transforms compute
    {
        const int Ly = p.L[1], Lz = p.L[2], m = p.m;
        auto in_iv = [](int v, int start, int len, int L) { return ((v - start) % L + L) % L < len; };
        for (int64_t i = 0; i < n; ++i) {
            const uint32_t pk = (uint32_t)grid[4 * i + 3];
            const int cy = (pk >> 10) & 1023, cz = (pk >> 20) & 1023;
            for (int oz = -m + 1; oz <= m; ++oz) {
                const int z = ((cz + oz) % Lz + Lz) % Lz;
                bool ok = in_iv(z, p.z0, p.nz_act, Lz);
                for (int oy = -m + 1; ok && oy <= m; ++oy)
                    ok = in_iv(((cy + oy) % Ly + Ly) % Ly, p.plane_iv[z].x, p.plane_iv[z].y, Ly);
                if (!ok)
                    return fail(SLP_ERR_UNSUPPORTED, "point %lld lies outside the grid rows this plan transforms",
                                (long long)perm[i]);
            }
        }
    }
    std::vector<slp::TileItem> items;
    tile_items(grid, keys, n, p.TSg, p.gather_chunk, items);
    std::stable_sort(items.begin(), items.end(),
                     [](const slp::TileItem &a, const slp::TileItem &b) { return a.end - a.begin > b.end - b.begin; });
    auto alloc_up = [&](void **dst, const void *src, size_t bytes) -> slp_status {
        const cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? SLP_ERR_OOM : SLP_ERR_CUDA, "probe allocation: %s",
                        cudaGetErrorString(e));
        }
        pr.allocs.push_back(*dst);
        if (src && bytes) TRY(cuda_status(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "probe upload"));
        return SLP_OK;
    };
    slp::DevPlan v = p.dp;
    v.N = n;
    v.ks = 1;
    v.wtab64_tgt = nullptr;  // the plan's target window table does not cover the probes
    std::vector<T4> tg(n);
    for (int64_t i = 0; i < n; ++i) {
        const double *g = &grid[4 * i];
        tg[i].x = (T)g[0];
        tg[i].y = (T)g[1];
        tg[i].z = (T)g[2];
        uint32_t pk = (uint32_t)g[3];
        if (sizeof(T) == 4) {
            float f;
            memcpy(&f, &pk, 4);
            tg[i].w = (T)f;
        } else {
            tg[i].w = (T)pk;
        }
        if (tg[i].x >= T(1)) tg[i].x = std::nextafter(T(1), T(0));
        if (tg[i].y >= T(1)) tg[i].y = std::nextafter(T(1), T(0));
        if (tg[i].z >= T(1)) tg[i].z = std::nextafter(T(1), T(0));
    }
    void *ptr = nullptr;
    TRY(alloc_up(&ptr, tg.data(), sizeof(T4) * n));
    v.tgt_grid = ptr;
    TRY(alloc_up(&ptr, perm.data(), sizeof(int32_t) * n));
    v.tgt_perm = (const int *)ptr;
    TRY(alloc_up(&ptr, items.data(), sizeof(slp::TileItem) * items.size()));
    v.gather_items = (const slp::TileItem *)ptr;
    v.n_gather = (int)items.size();
    TRY(alloc_up(&ptr, nullptr, sizeof(T) * ((n + 3) / 4 * 4)));
    v.phi_part = ptr;

    // near-field candidates: blocks of 32 consecutive sorted probes, the plan's
    // vertex bins within eps plus the largest triangle (or quadrature point) reach
    std::vector<double4> ptg(n);
    for (int64_t i = 0; i < n; ++i) {
        const double *x = &pts[3 * (int64_t)perm[i]];
        ptg[i] = make_double4(x[0] - p.ctr[0], x[1] - p.ctr[1], x[2] - p.ctr[2], 0.0);
    }
    double reach = 0.0;
    for (int64_t j = 0; j < p.M; ++j)
        for (int a = 0; a < 3; ++a) {
            const double *u = &p.V[3 * (int64_t)p.T[3 * j + a]], *w = &p.V[3 * (int64_t)p.T[3 * j + (a + 1) % 3]];
            reach = std::max(reach, std::sqrt((u[0] - w[0]) * (u[0] - w[0]) + (u[1] - w[1]) * (u[1] - w[1]) +
                                              (u[2] - w[2]) * (u[2] - w[2])));
        }
    const bool all_pairs = p.kernel_mode == SLP_KERNEL_SEPARABLE || !(p.eps < p.diam);
    const double rad = all_pairs ? INFINITY : p.eps + reach * (1.0 + 1e-9) + 1e-12 * p.diam;
    NearCandidates cand;
    {
        std::vector<uint64_t> tkeys;
        std::vector<int32_t> tperm;
        std::vector<double> tgrid;
        sort_points(p, p.V.data(), p.N, p.TSg, tperm, tgrid, tkeys);
        near_candidates(p, tkeys, rad, all_pairs, cand);  // vertex adjacency and bins of the plan's targets
        TargetBins tb;
        if (!all_pairs) target_bins(p, tkeys, cand.tgt, tb);
        const int64_t nblk = (n + 31) / 32;
        cand.tgt_block.assign(n, 0);
        cand.blk_r0.assign(nblk + 1, 0);
        cand.ranges.clear();
        for (int64_t b = 0; b < nblk; ++b) {
            cand.blk_r0[b] = (int)cand.ranges.size();
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (int64_t t = 32 * b; t < std::min(n, 32 * b + 32); ++t) {
                cand.tgt_block[t] = (int)b;
                const double x[3] = {ptg[t].x, ptg[t].y, ptg[t].z};
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::min(lo[d], x[d]);
                    hi[d] = std::max(hi[d], x[d]);
                }
            }
            if (all_pairs)
                cand.ranges.push_back(make_int2(0, (int)p.N));
            else
                bins_within(p, tb, lo, hi, rad, cand.ranges);
        }
        cand.blk_r0[nblk] = (int)cand.ranges.size();
    }
    TmpBuf b_blk, b_r0, b_rng, b_vtp, b_vte, b_cnt, b_pairs;
    TRY(tmp_upload(b_blk, cand.tgt_block.data(), cand.tgt_block.size()));
    TRY(tmp_upload(b_r0, cand.blk_r0.data(), cand.blk_r0.size()));
    TRY(tmp_upload(b_rng, cand.ranges.data(), std::max<size_t>(cand.ranges.size(), 1)));
    TRY(tmp_upload(b_vtp, cand.vt_ptr.data(), cand.vt_ptr.size()));
    TRY(tmp_upload(b_vte, cand.vt_ent.data(), cand.vt_ent.size()));
    {
        std::vector<int64_t> z(n + 1, 0);
        TRY(tmp_upload(b_cnt, z.data(), z.size()));
        TRY(tmp_upload(b_pairs, z.data(), z.size()));
    }
    std::vector<int64_t> cnt(n), rowptr(n + 1, 0);
    if (tri) {
        // rows of the triangle operator (the plan's assembly, probes as targets)
        std::vector<double3> tg3(n), xp(p.N);
        for (int64_t i = 0; i < n; ++i) tg3[i] = make_double3(ptg[i].x, ptg[i].y, ptg[i].z);
        for (int64_t i = 0; i < p.N; ++i)
            xp[i] = make_double3(p.V[3 * i] - p.ctr[0], p.V[3 * i + 1] - p.ctr[1], p.V[3 * i + 2] - p.ctr[2]);
        std::vector<int4> trv(p.M);
        std::vector<int> inv(p.N), tmin(p.M);
        for (int64_t j = 0; j < p.M; ++j) trv[j] = make_int4(p.T[3 * j], p.T[3 * j + 1], p.T[3 * j + 2], 0);
        for (int64_t i = 0; i < p.N; ++i) inv[p.tgt_perm[i]] = (int)i;
        for (int64_t j = 0; j < p.M; ++j)
            tmin[j] = std::min(inv[p.T[3 * j]], std::min(inv[p.T[3 * j + 1]], inv[p.T[3 * j + 2]]));
        std::vector<double> ra, rb, rw;
        tri_rule(8, ra, rb, rw);
        TmpBuf b_tg, b_xp, b_tri, b_tmin, b_ra, b_rb, b_rw, b_esw, b_esg, b_h[3];
        TRY(tmp_upload(b_tg, tg3.data(), tg3.size()));
        TRY(tmp_upload(b_xp, xp.data(), xp.size()));
        TRY(tmp_upload(b_tri, trv.data(), trv.size()));
        TRY(tmp_upload(b_tmin, tmin.data(), tmin.size()));
        TRY(tmp_upload(b_ra, ra.data(), ra.size()));
        TRY(tmp_upload(b_rb, rb.data(), rb.size()));
        TRY(tmp_upload(b_rw, rw.data(), rw.size()));
        slp::TriBuildN bn;
        memset(&bn, 0, sizeof bn);
        bn.tgt = (const double3 *)b_tg.p;
        bn.tgt_perm = p.dp.tgt_perm;
        bn.tgt_block = (const int *)b_blk.p;
        bn.blk_r0 = (const int *)b_r0.p;
        bn.ranges = (const int2 *)b_rng.p;
        bn.vt_ptr = (const int *)b_vtp.p;
        bn.vt_ent = (const int *)b_vte.p;
        bn.tri_min_sorted = (const int *)b_tmin.p;
        bn.xphys = (const double3 *)b_xp.p;
        bn.tri = (const int4 *)b_tri.p;
        bn.N = n;
        bn.eps = std::isfinite(p.eps) ? p.eps : 1e300;
        bn.kernel_mode = p.kernel_mode;
        bn.inv_s_sqrt2 = p.sigma_g > 0 ? 1.0 / (p.sigma_g * std::sqrt(2.0)) : 0.0;
        if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
            std::vector<double> w(p.es_w.size()), g(p.es_g.size());
            for (size_t k = 0; k < w.size(); ++k) {
                w[k] = p.es_w[k] / p.P[0];
                g[k] = p.es_g[k] / (p.P[0] * p.P[0]);
            }
            TRY(tmp_upload(b_esw, w.data(), w.size()));
            TRY(tmp_upload(b_esg, g.data(), g.size()));
            bn.es_w = (const double *)b_esw.p;
            bn.es_g = (const double *)b_esg.p;
            bn.es_n = (int)w.size();
        }
        if (p.kernel_mode == SLP_KERNEL_SEPARABLE) {
            for (int a = 0; a < 3; ++a) {
                TRY(tmp_upload(b_h[a], p.sep_h[a].data(), p.sep_h[a].size()));
                bn.sep_h[a] = (const double *)b_h[a].p;
                bn.sep_nh[a] = (int)p.sep_h[a].size();
            }
            bn.sep_A4pi = 4.0 * PI * p.sep_A;
        }
        for (int a = 0; a < 3; ++a) bn.P[a] = p.P[a];
        bn.ra = (const double *)b_ra.p;
        bn.rb = (const double *)b_rb.p;
        bn.rw = (const double *)b_rw.p;
        bn.np = (int)ra.size();
        bn.err = p.dp.err;
        TRY(cuda_status(slp::launch_nmt_build(bn, 0, p.prec, (int64_t *)b_cnt.p, nullptr, nullptr, nullptr, 0),
                        "probe near count"));
        TRY(cuda_status(cudaMemcpy(cnt.data(), b_cnt.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost), "count copy"));
        for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + cnt[i];
        TRY(alloc_up(&ptr, rowptr.data(), sizeof(int64_t) * (n + 1)));
        v.nt_rowptr = (const int64_t *)ptr;
        TRY(alloc_up(&ptr, nullptr, sizeof(int) * (size_t)std::max<int64_t>(rowptr[n], 1)));
        v.nt_col = (const int *)ptr;
        TRY(alloc_up(&ptr, nullptr, sizeof(T) * (size_t)std::max<int64_t>(rowptr[n], 1)));
        v.nt_val = ptr;
        TRY(cuda_status(slp::launch_nmt_build(bn, 1, p.prec, nullptr, v.nt_rowptr, (int *)v.nt_col, (void *)v.nt_val, 0),
                        "probe near fill"));
    } else {
        // rows of the vertex operator (the plan's assembly, probes as targets)
        std::vector<double4> src(p.Q), nrm(p.M);
        for (int64_t k = 0; k < p.Q; ++k)
            src[k] = make_double4(p.y[3 * k] - p.ctr[0], p.y[3 * k + 1] - p.ctr[1], p.y[3 * k + 2] - p.ctr[2], p.wk[k]);
        for (int64_t j = 0; j < p.M; ++j) nrm[j] = make_double4(p.nrm[3 * j], p.nrm[3 * j + 1], p.nrm[3 * j + 2], 0.0);
        TmpBuf b_tg, b_src, b_nrm, b_lam, b_h[3];
        TRY(tmp_upload(b_tg, ptg.data(), ptg.size()));
        TRY(tmp_upload(b_src, src.data(), src.size()));
        TRY(tmp_upload(b_nrm, nrm.data(), nrm.size()));
        TRY(tmp_upload(b_lam, p.lam.data(), p.lam.size()));
        slp::NMBuild nb;
        memset(&nb, 0, sizeof nb);
        nb.tgt = (const double4 *)b_tg.p;
        nb.tgt_perm = p.dp.tgt_perm;
        nb.tgt_block = (const int *)b_blk.p;
        nb.blk_r0 = (const int *)b_r0.p;
        nb.ranges = (const int2 *)b_rng.p;
        nb.vt_ptr = (const int *)b_vtp.p;
        nb.vt_ent = (const int *)b_vte.p;
        nb.src = (const double4 *)b_src.p;
        nb.nrm = (const double4 *)b_nrm.p;
        nb.lam = (const double *)b_lam.p;
        nb.q = p.q;
        nb.N = n;
        nb.eps2 = std::isfinite(p.eps) ? p.eps * p.eps : 1e300;
        nb.inv_s_sqrt2 = p.sigma_g > 0 ? 1.0 / (p.sigma_g * std::sqrt(2.0)) : 0.0;
        nb.kernel_mode = p.kernel_mode;
        TmpBuf b_esw, b_esg;
        if (p.kernel_mode == SLP_KERNEL_SEPARABLE) {
            for (int a = 0; a < 3; ++a) {
                TRY(tmp_upload(b_h[a], p.sep_h[a].data(), p.sep_h[a].size()));
                nb.sep_h[a] = (const double *)b_h[a].p;
                nb.sep_nh[a] = (int)p.sep_h[a].size();
            }
            nb.sep_A4pi = 4.0 * PI * p.sep_A;
        }
        if (p.kernel_mode == SLP_KERNEL_EXPSUM) {
            std::vector<double> w(p.es_w.size()), g(p.es_g.size());
            for (size_t k = 0; k < w.size(); ++k) {
                w[k] = p.es_w[k] / p.P[0];
                g[k] = p.es_g[k] / (p.P[0] * p.P[0]);
            }
            TRY(tmp_upload(b_esw, w.data(), w.size()));
            TRY(tmp_upload(b_esg, g.data(), g.size()));
            nb.es_w = (const double *)b_esw.p;
            nb.es_g = (const double *)b_esg.p;
            nb.es_n = (int)w.size();
        }
        for (int a = 0; a < 3; ++a) nb.P[a] = p.P[a];
        TRY(cuda_status(slp::launch_nm_build(nb, 0, p.prec, (int64_t *)b_cnt.p, (int64_t *)b_pairs.p, nullptr, nullptr, 0),
                        "probe near count"));
        TRY(cuda_status(cudaMemcpy(cnt.data(), b_cnt.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost), "count copy"));
        for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + cnt[i];
        TRY(alloc_up(&ptr, rowptr.data(), sizeof(int64_t) * (n + 1)));
        v.nm_rowptr = (const int64_t *)ptr;
        TRY(alloc_up(&ptr, nullptr, sizeof(T4) * (size_t)std::max<int64_t>(rowptr[n], 1)));
        v.nm_val = ptr;
        TRY(cuda_status(slp::launch_nm_build(nb, 1, p.prec, nullptr, nullptr, v.nm_rowptr, ptr, 0), "probe near fill"));
    }
    TRY(cuda_status(cudaDeviceSynchronize(), "probe near build"));
    int code = 0;
    TRY(cuda_status(cudaMemcpy(&code, p.dp.err, sizeof(int), cudaMemcpyDeviceToHost), "status"));
    if (code != 0) return fail(SLP_ERR_CUDA, "probe near build: device status word %d", code);
    pr.near_nnz = rowptr[n];
    pr.view = v;
    return SLP_OK;
}

slp_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SLP_OK;
    return fail(SLP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Kernel slots of the profiler entry point (slp_debug_profile).  A serial
// profiled evaluation brackets each kernel it launches with a pair of events
// on the launch stream; slots whose kernel did not launch report -1.
const char *const STAGE_NAMES[SLP_PROFILE_SLOTS] = {
    "charges", "spread", "fft_x", "fft_y", "fft_z_mul", "ifft_y", "ifft_x", "nodal_prep",
    "near_zero", "near", "near_reduce", "gather", "fft_xy", "ifft_yx", "fft_yzy"};
enum {
    SLOT_CHARGES, SLOT_SPREAD, SLOT_FFT_X, SLOT_FFT_Y, SLOT_FFT_Z, SLOT_IFFT_Y, SLOT_IFFT_X, SLOT_NODAL_PREP,
    SLOT_NEAR_ZERO, SLOT_NEAR, SLOT_NEAR_REDUCE, SLOT_GATHER, SLOT_FFT_XY, SLOT_IFFT_YX, SLOT_FFT_YZY
};

// Enqueue the evaluation up to stage `last`.
//   serial (prof != NULL, or ex == NULL): charges, spread, 5 FFT passes, near
//     field into phi_part, gather (far field + phi_part) on s; with prof,
//     every launched kernel is bracketed by its slot's two events;
//   concurrent (ex != NULL, no prof): the near field runs on ex->aux (lowest
//     priority) while the spread, FFT passes and gather run on ex->main
//     (highest priority, so the latency-bound FFT blocks are dispatched ahead
//     of pending near-field blocks); both fork from s, the gather waits for
//     the near field, and s waits for the gather.
slp_status run_pipeline(slp_plan_s &p, const slp::DevPlan &d, int kind, const void *d_in, void *d_phi,
                        cudaStream_t s, int last, SlpProfile *prof, SlpExec *ex) {
    // launch `fn` on stream t, bracketed by the slot's events when profiling
    auto timed = [&](int slot, cudaStream_t t, auto fn, const char *what) -> slp_status {
        if (prof) cudaEventRecord(prof->ev[2 * slot], t);
        TRY(cuda_status(fn(), what));
        if (prof) {
            cudaEventRecord(prof->ev[2 * slot + 1], t);
            prof->launched[slot] = true;
        }
        return SLP_OK;
    };
    // triangle integrals: element charges, then two sparse products (gridding
    // matrix into grid A, near-field matrix into phi_part)
    const bool tri = p.opts.integration != 0;
    const void *gch = kind == SLP_INPUT_ELEMENT ? d_in : d.gbuf;
    // nodal input with the precomputed near field: the charges are only needed
    // by the spread, which computes them itself
    const bool use_matrix = !tri && kind == SLP_INPUT_NODAL_MAG && p.near_mode == SLP_NEAR_PRECOMPUTED;
    // deterministic point plans: the spread is the sparse product with the
    // point gridding matrix, which reads the charges from qbuf
    const bool det = !tri && d.det_spread;
    const bool fuse = use_matrix && !det && last > SLP_STAGE_CHARGES;
    const bool concurrent = ex != nullptr && prof == nullptr && last >= SLP_STAGE_NEAR;
    const size_t es = p.prec == 64 ? 8 : 4;
    const size_t part_bytes = (es * (size_t)p.N + 15) / 16 * 16;
    // near-field branch on stream t
    auto near_branch = [&](cudaStream_t t) -> slp_status {
        if (tri) {
            TRY(timed(SLOT_NEAR, t, [&] {
                return slp::launch_csr_apply(p.prec, 32, p.N, d.nt_rowptr, nullptr, d.nt_col, d.nt_val, gch,
                                             d.phi_part, t);
            }, "near-field matrix"));
            return SLP_OK;
        }
        if (use_matrix) {
            TRY(timed(SLOT_NODAL_PREP, t, [&] { return slp::launch_nodal_prep(d, d_in, t); }, "nodal prep"));
            TRY(timed(SLOT_NEAR, t, [&] { return slp::launch_near_matrix(d, d_in, t); }, "near-field matrix"));
            return SLP_OK;
        }
        if (!p.opts.deterministic)
            TRY(timed(SLOT_NEAR_ZERO, t, [&] { return slp::launch_zero(d.phi_part, part_bytes, t); },
                      "zero near field"));
        TRY(timed(SLOT_NEAR, t, [&] { return slp::launch_near(d, t); }, "near field"));
        if (p.opts.deterministic)
            TRY(timed(SLOT_NEAR_REDUCE, t, [&] {
                return slp::launch_near_reduce(d, p.d_blk_first, (int)p.near_blk_first.size() - 1, t);
            }, "near reduce"));
        return SLP_OK;
    };
    cudaEvent_t *tl = concurrent ? ex->timeline : nullptr;
    if (tl) TRY(cuda_status(cudaEventRecord(tl[0], s), "timeline"));
    if (tri) {
        if (kind == SLP_INPUT_NODAL_MAG)
            TRY(timed(SLOT_CHARGES, s, [&] { return slp::launch_p0_charges(d, d_in, s); }, "element charges"));
    } else if (!fuse) {
        TRY(timed(SLOT_CHARGES, s, [&] { return slp::launch_charges(d, kind, d_in, s); }, "charges"));
    }
    if (last <= SLP_STAGE_CHARGES) return SLP_OK;
    cudaStream_t caller = s;
    if (concurrent) {
        TRY(cuda_status(cudaEventRecord(ex->fork, s), "fork"));
        TRY(cuda_status(cudaStreamWaitEvent(ex->aux, ex->fork, 0), "fork wait"));
        TRY(cuda_status(cudaStreamWaitEvent(ex->main, ex->fork, 0), "fork wait"));
        s = ex->main;
        TRY(near_branch(ex->aux));
        if (tl) TRY(cuda_status(cudaEventRecord(tl[3], ex->aux), "timeline"));
        TRY(cuda_status(cudaEventRecord(ex->join, ex->aux), "join"));
    }
    if (tri || det)
        TRY(timed(SLOT_SPREAD, s, [&] {
            return slp::launch_csr_apply(p.prec, 8, d.am_rows, d.am_rowptr, d.am_row, d.am_col, d.am_val,
                                         tri ? gch : d.qbuf, d.gridA, s);
        }, "gridding matrix"));
    else
        TRY(timed(SLOT_SPREAD, s, [&] { return slp::launch_spread(d, fuse ? kind : -1, d_in, s); }, "spread"));
    if (tl) TRY(cuda_status(cudaEventRecord(tl[1], s), "timeline"));
    if (last <= SLP_STAGE_SPREAD) return SLP_OK;
    // fused plane passes (FX + FY, IY + IX) unless the run stops between them
    const bool fused = d.fuse_pb > 0;
    // fused column passes (FY, FZ, IY) unless the run stops between them
    const bool yzy = !fused && d.yzy_g > 0 && last >= SLP_STAGE_IFFT_Y;
    if (fused && last >= SLP_STAGE_FFT_Y) {
        TRY(timed(SLOT_FFT_XY, s, [&] { return slp::launch_fft_forward_xy(d, s); }, "fft xy"));
    } else {
        TRY(timed(SLOT_FFT_X, s, [&] { return slp::launch_fft_forward_x(d, s); }, "fft x"));
        if (last <= SLP_STAGE_FFT_X) return SLP_OK;
        if (yzy)
            TRY(timed(SLOT_FFT_YZY, s, [&] { return slp::launch_fft_yzy(d, s); }, "fft yzy"));
        else
            TRY(timed(SLOT_FFT_Y, s, [&] { return slp::launch_fft_forward_y(d, s); }, "fft y"));
    }
    if (last <= SLP_STAGE_FFT_Y) return SLP_OK;
    if (!yzy) TRY(timed(SLOT_FFT_Z, s, [&] { return slp::launch_fft_z_multiply(d, s); }, "fft z"));
    if (last <= SLP_STAGE_FFT_Z) return SLP_OK;
    if (fused && last >= SLP_STAGE_IFFT_X) {
        TRY(timed(SLOT_IFFT_YX, s, [&] { return slp::launch_fft_inverse_yx(d, s); }, "ifft yx"));
    } else {
        if (!yzy) TRY(timed(SLOT_IFFT_Y, s, [&] { return slp::launch_fft_inverse_y(d, s); }, "ifft y"));
        if (last <= SLP_STAGE_IFFT_Y) return SLP_OK;
        TRY(timed(SLOT_IFFT_X, s, [&] { return slp::launch_fft_inverse_x(d, s); }, "ifft x"));
    }
    if (last <= SLP_STAGE_IFFT_X) return SLP_OK;
    if (tl) TRY(cuda_status(cudaEventRecord(tl[2], s), "timeline"));
    if (concurrent) {
        TRY(cuda_status(cudaStreamWaitEvent(s, ex->join, 0), "join wait"));
    } else if (last >= SLP_STAGE_NEAR) {
        TRY(near_branch(s));
    } else {
        // far field only
        TRY(timed(SLOT_NEAR_ZERO, s, [&] { return slp::launch_zero(d.phi_part, part_bytes, s); }, "zero near field"));
    }
    TRY(timed(SLOT_GATHER, s, [&] { return slp::launch_gather(d, d_phi, s); }, "gather"));
    if (tl) TRY(cuda_status(cudaEventRecord(tl[4], s), "timeline"));
    if (concurrent) {
        TRY(cuda_status(cudaEventRecord(ex->done, s), "done"));
        TRY(cuda_status(cudaStreamWaitEvent(caller, ex->done, 0), "done wait"));
    }
    return SLP_OK;
}

slp_status run_pipeline(slp_plan_s &p, int kind, const void *d_in, void *d_phi, cudaStream_t s, int last,
                        SlpProfile *prof = nullptr) {
    return run_pipeline(p, p.dp, kind, d_in, d_phi, s, last, prof, prof ? nullptr : &p.exec);
}

// S states of nodal input with the precomputed near field, in chunks of up
// to NEAR_STATES: per chunk, one sorting prep and one pass over the near-field
// operator for all of the chunk's states run on ex->aux, while ex->main runs
// the spread, FFT passes and gather for batches of kf states at a time (one
// launch per kernel per batch; the gather of state k reads near-field part k).
// Each chunk's branch starts after the previous chunk's gathers (they read the
// same scratch).  Other inputs or near modes run the single-state pipeline per
// state.
slp_status run_states(slp_plan_s &p, const slp::DevPlan &d, int kind, const void *const *ins, void *const *outs,
                      int S, cudaStream_t s, SlpExec *ex, int *launches) {
    // the state-batched far field uses the tiled spread; deterministic point
    // plans evaluate their states one by one
    const bool use_matrix = !p.opts.integration && !d.det_spread && kind == SLP_INPUT_NODAL_MAG &&
                            p.near_mode == SLP_NEAR_PRECOMPUTED;
    if (!use_matrix || !ex) {
        for (int k = 0; k < S; ++k) {
            TRY(run_pipeline(p, d, kind, ins[k], outs[k], s, SLP_STAGE_NEAR, nullptr, ex));
            if (launches) *launches += p.launches_per_eval;
        }
        return SLP_OK;
    }
    const size_t es = p.prec == 64 ? 8 : 4;
    cudaStream_t m = ex->main;
    TRY(cuda_status(cudaEventRecord(ex->fork, s), "fork"));
    TRY(cuda_status(cudaStreamWaitEvent(m, ex->fork, 0), "fork wait"));
    for (int c0 = 0; c0 < S; c0 += slp::NEAR_STATES) {
        const int K = std::min(slp::NEAR_STATES, S - c0);
        slp::StatePtrs sp = {};
        for (int k = 0; k < K; ++k) sp.in[k] = ins[c0 + k];
        TRY(cuda_status(cudaEventRecord(ex->fork, m), "fork"));
        TRY(cuda_status(cudaStreamWaitEvent(ex->aux, ex->fork, 0), "fork wait"));
        TRY(cuda_status(slp::launch_nodal_prep_states(d, sp, K, ex->aux), "nodal prep"));
        TRY(cuda_status(slp::launch_near_matrix_states(d, K, ex->aux), "near-field matrix"));
        TRY(cuda_status(cudaEventRecord(ex->join, ex->aux), "join"));
        // the far field in batches of kf states: one launch per kernel per batch
        // (grid.y = state), state f at scratch copy f and near-field part f0 + f
        int nbatch = 0;
        for (int f0 = 0; f0 < K; f0 += p.kf, ++nbatch) {
            const int kb = std::min(p.kf, K - f0);
            slp::DevPlan dk = d;
            dk.ks = kb;
            for (int f = 0; f < kb; ++f) {
                dk.in_st[f] = ins[c0 + f0 + f];
                dk.out_st[f] = outs[c0 + f0 + f];
            }
            dk.phi_part = (char *)d.phi_part + es * (size_t)p.N * f0;
            TRY(cuda_status(slp::launch_spread(dk, kind, ins[c0 + f0], m), "spread"));
            if (d.fuse_pb > 0) {
                TRY(cuda_status(slp::launch_fft_forward_xy(dk, m), "fft xy"));
                TRY(cuda_status(slp::launch_fft_z_multiply(dk, m), "fft z"));
                TRY(cuda_status(slp::launch_fft_inverse_yx(dk, m), "ifft yx"));
            } else if (d.yzy_g > 0) {
                TRY(cuda_status(slp::launch_fft_forward_x(dk, m), "fft x"));
                TRY(cuda_status(slp::launch_fft_yzy(dk, m), "fft yzy"));
                TRY(cuda_status(slp::launch_fft_inverse_x(dk, m), "ifft x"));
            } else {
                TRY(cuda_status(slp::launch_fft_forward_x(dk, m), "fft x"));
                TRY(cuda_status(slp::launch_fft_forward_y(dk, m), "fft y"));
                TRY(cuda_status(slp::launch_fft_z_multiply(dk, m), "fft z"));
                TRY(cuda_status(slp::launch_fft_inverse_y(dk, m), "ifft y"));
                TRY(cuda_status(slp::launch_fft_inverse_x(dk, m), "ifft x"));
            }
            if (f0 == 0) TRY(cuda_status(cudaStreamWaitEvent(m, ex->join, 0), "join wait"));
            TRY(cuda_status(slp::launch_gather(dk, outs[c0 + f0], m), "gather"));
        }
        if (launches) *launches += 2 + nbatch * (p.launches_per_eval - 2);
    }
    TRY(cuda_status(cudaEventRecord(ex->done, m), "done"));
    TRY(cuda_status(cudaStreamWaitEvent(s, ex->done, 0), "done wait"));
    return SLP_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

void slp::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

slp_status slp_check_kind(const slp_plan_s &p, int kind) {
    if (kind < SLP_INPUT_SIGMA || kind > SLP_INPUT_ELEMENT) return slp_fail(SLP_ERR_INVALID_ARG, "unknown input kind %d", kind);
    if (p.opts.integration && (kind == SLP_INPUT_SIGMA || kind == SLP_INPUT_MAG))
        return slp_fail(SLP_ERR_UNSUPPORTED, "plans with triangle integrals take element charges or nodal m");
    if (!p.opts.integration && kind == SLP_INPUT_ELEMENT)
        return slp_fail(SLP_ERR_UNSUPPORTED, "element charges need a plan with opts.integration = 1");
    return SLP_OK;
}

slp_status slp_fail(slp_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

slp_status slp_run_pipeline(slp_plan_s &p, const slp::DevPlan &d, int kind, const void *d_in, void *d_phi,
                            cudaStream_t s, int last, SlpProfile *prof, SlpExec *ex) {
    return run_pipeline(p, d, kind, d_in, d_phi, s, last, prof, ex);
}

slp_status slp_run_states(slp_plan_s &p, const slp::DevPlan &d, int kind, const void *const *ins, void *const *outs,
                          int n, cudaStream_t s, SlpExec *ex, int *launches) {
    return run_states(p, d, kind, ins, outs, n, s, ex, launches);
}

cudaError_t slp_exec_create(SlpExec &e) {
    int least = 0, greatest = 0;
    cudaError_t r = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (r == cudaSuccess) r = cudaStreamCreateWithPriority(&e.aux, cudaStreamNonBlocking, least);
    if (r == cudaSuccess) r = cudaStreamCreateWithPriority(&e.main, cudaStreamNonBlocking, greatest);
    if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming);
    if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e.join, cudaEventDisableTiming);
    if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming);
    return r;
}

void slp_exec_destroy(SlpExec &e) {
    if (e.done) cudaEventDestroy(e.done);
    if (e.join) cudaEventDestroy(e.join);
    if (e.fork) cudaEventDestroy(e.fork);
    if (e.main) cudaStreamDestroy(e.main);
    if (e.aux) cudaStreamDestroy(e.aux);
    e = SlpExec();
}

int slp_far_batch(const slp_plan_s &p) {
    const int64_t es = p.prec == 64 ? 8 : 4;
    const int64_t G = (int64_t)p.L[0] * p.L[1] * p.L[2];
    const int64_t Kx = p.n[0] / 2;
    const int64_t per = es * (2 * G + 2 * (int64_t)p.L[2] * p.L[1] * Kx + 2 * (int64_t)p.L[2] * p.n[1] * Kx);
    const int64_t budget = (int64_t)2 << 30;
    int64_t k = per > 0 ? budget / per : 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>(slp::NEAR_STATES, k));
}

int64_t slp_scratch_bytes(const slp_plan_s &p) {
    const int64_t es = p.prec == 64 ? 8 : 4;
    const int64_t G = (int64_t)p.L[0] * p.L[1] * p.L[2];
    const int64_t Kx = p.n[0] / 2;
    const int64_t kf = slp_far_batch(p);
    int64_t b = es * p.Q + 5 * es * p.N * slp::NEAR_STATES +
                kf * (2 * es * G + 2 * es * p.L[2] * p.L[1] * Kx + 2 * es * p.L[2] * p.n[1] * Kx);
    if (p.opts.deterministic) b += es * 32 * (int64_t)std::max<size_t>(1, p.near_items.size());
    return b;
}

slp_status slp_alloc_scratch(slp_plan_s &p, slp::DevPlan &out, std::vector<void *> &allocs, int64_t *bytes) {
    out = p.dp;
    const int64_t es = p.prec == 64 ? 8 : 4;
    const int64_t G = (int64_t)p.L[0] * p.L[1] * p.L[2];
    const int64_t Kx = p.n[0] / 2;
    struct Req {
        void **dst;
        int64_t n;
    } reqs[] = {{&out.qbuf, es * p.Q},
                {&out.m4, 4 * es * p.N * slp::NEAR_STATES},
                {&out.phi_part, es * p.N * slp::NEAR_STATES},
                {&out.gridA, es * G * p.kf},
                {&out.gridB, es * G * p.kf},
                {&out.S1, 2 * es * p.L[2] * p.L[1] * Kx * p.kf},
                {&out.S2, 2 * es * p.L[2] * p.n[1] * Kx * p.kf},
                {&out.phi_near, p.opts.deterministic ? es * 32 * (int64_t)std::max<size_t>(1, p.near_items.size()) : 0},
                {&out.gbuf, p.opts.integration ? es * p.M : 0}};
    int64_t total = 0;
    for (auto &r : reqs) {
        if (r.n == 0) continue;
        const size_t nb = (size_t)((r.n + 255) / 256 * 256);
        void *ptr = nullptr;
        const cudaError_t e = cudaMalloc(&ptr, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return slp_fail(e == cudaErrorMemoryAllocation ? SLP_ERR_OOM : SLP_ERR_CUDA, "scratch allocation of %zu bytes: %s",
                            nb, cudaGetErrorString(e));
        }
        allocs.push_back(ptr);
        *r.dst = ptr;
        total += (int64_t)nb;
    }
    if (cudaMemset(out.gridA, 0, es * G * p.kf) != cudaSuccess || cudaMemset(out.gridB, 0, es * G * p.kf) != cudaSuccess ||
        cudaMemset(out.S1, 0, 2 * es * p.L[2] * p.L[1] * Kx * p.kf) != cudaSuccess ||
        cudaMemset(out.S2, 0, 2 * es * p.L[2] * p.n[1] * Kx * p.kf) != cudaSuccess)
        return slp_fail(SLP_ERR_CUDA, "cudaMemset failed");
    if (bytes) *bytes = total;
    return SLP_OK;
}

// ======================================================================= C ABI
extern "C" {

slp_status slp_default_opts(slp_plan_opts *o) {
    if (!o) return fail(SLP_ERR_INVALID_ARG, "opts is NULL");
    memset(o, 0, sizeof *o);
    o->precision = 32;
    o->kernel_mode = SLP_KERNEL_AUTO;
    o->near_mode = SLP_NEAR_AUTO;
    o->device = 0;
    o->allow_grid_raise = 1;
    o->check_mesh = 1;
    o->fuse_plane_passes = -1;
    o->fuse_column_passes = -1;
    o->spread_table = -1;
    return SLP_OK;
}

slp_status slp_plan(const slp_mesh *mesh, int quadrature, double tolerance, const slp_plan_opts *opts,
                    slp_plan_t *out) {
    g_last_error.clear();
    if (!out) return fail(SLP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!mesh || !mesh->vertices || !mesh->triangles) return fail(SLP_ERR_INVALID_ARG, "mesh or its arrays are NULL");
    if (mesh->n_vertices < 3 || mesh->n_triangles < 1) return fail(SLP_ERR_INVALID_ARG, "mesh is empty");
    if (mesh->n_vertices > (1LL << 30) || mesh->n_triangles * 7 > (1LL << 30))
        return fail(SLP_ERR_INVALID_ARG, "mesh too large for 32-bit indices");
    if (!(tolerance > 0.0 && tolerance < 1.0)) return fail(SLP_ERR_INVALID_ARG, "tolerance must be in (0, 1)");
    slp_plan_opts o;
    if (opts)
        o = *opts;
    else
        slp_default_opts(&o);
    if (o.precision != 32 && o.precision != 64) return fail(SLP_ERR_INVALID_ARG, "precision must be 32 or 64");

    slp_plan_s *p = new slp_plan_s();
    p->opts = o;
    p->q = quadrature;
    p->prec = o.precision;
    p->tol = tolerance;
    p->N = mesh->n_vertices;
    p->M = mesh->n_triangles;
    p->device = o.device;
    p->V.assign(mesh->vertices, mesh->vertices + 3 * p->N);
    p->T.assign(mesh->triangles, mesh->triangles + 3 * p->M);
    for (double v : p->V)
        if (!std::isfinite(v)) {
            delete p;
            return fail(SLP_ERR_MESH, "vertex coordinates must be finite");
        }
    slp_status st = validate_mesh(*p);
    if (st == SLP_OK) st = build_sources(*p);
    if (st == SLP_OK) st = choose_parameters(*p);
    if (st != SLP_OK) {
        delete p;
        return st;
    }
    std::vector<uint64_t> skeys, tkeys;
    sort_points(*p, p->y.data(), p->Q, p->TS, p->src_perm, p->src_grid, skeys);
    sort_points(*p, p->V.data(), p->N, p->TSg, p->tgt_perm, p->tgt_grid, tkeys);
    {
        // spread chunk: about four items per SM, 128..1024 sources, a multiple of 32
        int64_t ch = (p->Q + 152 * 4 - 1) / (152 * 4);
        ch = std::max<int64_t>(128, std::min<int64_t>(1024, (ch + 31) / 32 * 32));
        tile_items(p->src_grid, skeys, p->Q, p->TS, (int)ch, p->spread_items);
    }
    // gather items of GATHER_CHUNK targets, or of half that when the full
    // size leaves fewer than four items per SM (small, latency-bound gathers)
    if (o.gather_item_targets != 0 && o.gather_item_targets != 32 && o.gather_item_targets != 64) {
        delete p;
        return fail(SLP_ERR_INVALID_ARG, "gather_item_targets must be 0, 32 or 64");
    }
    if (o.spread_blocks != 0 && o.spread_blocks != 4 && o.spread_blocks != 5) {
        delete p;
        return fail(SLP_ERR_INVALID_ARG, "spread_blocks must be 0, 4 or 5");
    }
    p->gather_chunk = o.gather_item_targets ? o.gather_item_targets : slp::GATHER_CHUNK;
    tile_items(p->tgt_grid, tkeys, p->N, p->TSg, p->gather_chunk, p->gather_items);
    if (o.gather_item_targets == 0 && p->gather_items.size() < 4 * 152) {
        p->gather_chunk = slp::GATHER_CHUNK / 2;
        tile_items(p->tgt_grid, tkeys, p->N, p->TSg, p->gather_chunk, p->gather_items);
    }
    // largest items first: blocks are dispatched in index order, so this
    // schedules the long items early and the short ones fill the tail
    auto by_size = [](const slp::TileItem &a, const slp::TileItem &b) { return a.end - a.begin > b.end - b.begin; };
    std::stable_sort(p->spread_items.begin(), p->spread_items.end(), by_size);
    std::stable_sort(p->gather_items.begin(), p->gather_items.end(), by_size);
    spread_groups(*p);
    near_items(*p, skeys, tkeys);
    build_dtab(*p);
    active_region(*p);
    p->near_mode = SLP_NEAR_ON_THE_FLY;

    if (p->device >= 0) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= p->device) {
            cudaGetLastError();
            delete p;
            return fail(SLP_ERR_NO_DEVICE, "CUDA device %d is not available", o.device);
        }
        DeviceGuard g(p->device);
        st = p->prec == 64 ? upload_all<double>(*p) : upload_all<float>(*p);
        if (st == SLP_OK && o.integration)
            st = p->prec == 64 ? build_tri_matrices<double>(*p, tkeys) : build_tri_matrices<float>(*p, tkeys);
        else if (st == SLP_OK && o.near_mode != SLP_NEAR_ON_THE_FLY)
            st = build_near_matrix(*p, tkeys);
        if (st == SLP_OK && o.deterministic && !o.integration)
            st = p->prec == 64 ? build_point_matrix<double>(*p) : build_point_matrix<float>(*p);
        if (st == SLP_OK && slp_exec_create(p->exec) != cudaSuccess) st = fail(SLP_ERR_CUDA, "stream creation failed");
        if (st == SLP_OK) {
            bool ok = cudaStreamCreateWithFlags(&p->cs_in, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&p->cs_out, cudaStreamNonBlocking) == cudaSuccess;
            for (int k = 0; k < 2 && ok; ++k)
                ok = cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&p->ev_eval[k], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&p->ev_out[k], cudaEventDisableTiming) == cudaSuccess;
            if (!ok) st = fail(SLP_ERR_CUDA, "copy stream creation failed");
        }
        if (st != SLP_OK) {
            free_device(*p);
            delete p;
            return st;
        }
    }
    *out = p;
    return SLP_OK;
}

slp_status slp_eval(slp_plan_t p, int kind, const void *d_in, void *d_phi, void *stream) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan cannot evaluate");
    TRY(slp_check_kind(*p, kind));
    if (!d_in || !d_phi) return fail(SLP_ERR_INVALID_ARG, "input or output pointer is NULL");
    DeviceGuard g(p->device);
    return run_pipeline(*p, kind, d_in, d_phi, (cudaStream_t)stream, SLP_STAGE_NEAR);
}

slp_status slp_eval_states(slp_plan_t p, int kind, int n_states, const void *d_in, void *d_phi, void *stream) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan cannot evaluate");
    TRY(slp_check_kind(*p, kind));
    if (n_states < 1) return fail(SLP_ERR_INVALID_ARG, "n_states must be positive");
    if (!d_in || !d_phi) return fail(SLP_ERR_INVALID_ARG, "input or output pointer is NULL");
    DeviceGuard g(p->device);
    const size_t es = p->prec == 64 ? 8 : 4;
    const size_t in_elems = kind == SLP_INPUT_SIGMA ? (size_t)p->Q : (kind == SLP_INPUT_MAG ? 3 * (size_t)p->Q : 3 * (size_t)p->N);
    std::vector<const void *> ins(n_states);
    std::vector<void *> outs(n_states);
    for (int k = 0; k < n_states; ++k) {
        ins[k] = (const char *)d_in + es * in_elems * k;
        outs[k] = (char *)d_phi + es * (size_t)p->N * k;
    }
    return run_states(*p, p->dp, kind, ins.data(), outs.data(), n_states, (cudaStream_t)stream, &p->exec, nullptr);
}

slp_status slp_eval_host(slp_plan_t p, int kind, const void *h_in, void *h_phi, void *stream) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan cannot evaluate");
    TRY(slp_check_kind(*p, kind));
    if (!h_in || !h_phi) return fail(SLP_ERR_INVALID_ARG, "input or output pointer is NULL");
    DeviceGuard g(p->device);
    const size_t es = p->prec == 64 ? 8 : 4;
    const size_t nin = (size_t)slp_input_count(*p, kind);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(cuda_status(cudaMemcpyAsync(p->d_stage_in, h_in, nin * es, cudaMemcpyHostToDevice, s), "copy in"));
    TRY(run_pipeline(*p, kind, p->d_stage_in, p->d_stage_phi, s, SLP_STAGE_NEAR));
    TRY(cuda_status(cudaMemcpyAsync(h_phi, p->d_stage_phi, (size_t)p->N * es, cudaMemcpyDeviceToHost, s), "copy out"));
    TRY(cuda_status(cudaStreamSynchronize(s), "synchronize"));
    return SLP_OK;
}

slp_status slp_eval_host_async(slp_plan_t p, int kind, const void *h_in, void *h_phi, void *stream) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan cannot evaluate");
    TRY(slp_check_kind(*p, kind));
    if (!h_in || !h_phi) return fail(SLP_ERR_INVALID_ARG, "input or output pointer is NULL");
    DeviceGuard g(p->device);
    const size_t es = p->prec == 64 ? 8 : 4;
    const size_t nin = (size_t)slp_input_count(*p, kind);
    cudaStream_t s = (cudaStream_t)stream;
    const int k = p->aslot;
    p->aslot ^= 1;
    // copy-in: after the evaluation that last read this slot
    TRY(cuda_status(cudaStreamWaitEvent(p->cs_in, p->ev_eval[k], 0), "copy-in wait"));
    TRY(cuda_status(cudaMemcpyAsync(p->d_astage_in[k], h_in, nin * es, cudaMemcpyHostToDevice, p->cs_in), "copy in"));
    TRY(cuda_status(cudaEventRecord(p->ev_in[k], p->cs_in), "copy-in event"));
    // evaluation: after its input arrived and the copy-out that last read this slot's phi
    TRY(cuda_status(cudaStreamWaitEvent(s, p->ev_in[k], 0), "evaluation wait"));
    TRY(cuda_status(cudaStreamWaitEvent(s, p->ev_out[k], 0), "evaluation wait"));
    TRY(run_pipeline(*p, kind, p->d_astage_in[k], p->d_astage_phi[k], s, SLP_STAGE_NEAR));
    TRY(cuda_status(cudaEventRecord(p->ev_eval[k], s), "evaluation event"));
    // copy-out
    TRY(cuda_status(cudaStreamWaitEvent(p->cs_out, p->ev_eval[k], 0), "copy-out wait"));
    TRY(cuda_status(cudaMemcpyAsync(h_phi, p->d_astage_phi[k], (size_t)p->N * es, cudaMemcpyDeviceToHost, p->cs_out),
                    "copy out"));
    TRY(cuda_status(cudaEventRecord(p->ev_out[k], p->cs_out), "copy-out event"));
    return SLP_OK;
}

slp_status slp_probe_create(slp_plan_t p, const double *points, int64_t n, slp_probe_t *out) {
    if (!out) return fail(SLP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !points || n < 1) return fail(SLP_ERR_INVALID_ARG, "plan, points or count missing");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan");
    if (n > (1LL << 30)) return fail(SLP_ERR_INVALID_ARG, "too many points");
    if (!p->opts.integration && p->near_mode != SLP_NEAR_PRECOMPUTED)
        return fail(SLP_ERR_UNSUPPORTED, "probes need the precomputed near field or triangle integrals");
    // the bounding box keeps the pairs clear of periodic images; the ball of
    // diameter diam about its centre keeps every source within the distance
    // where the truncated smooth kernel is still the smoothed 1/r
    for (int64_t i = 0; i < n; ++i) {
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double x = points[3 * i + d];
            if (!std::isfinite(x) || std::fabs(x - p->ctr[d]) > 0.5 * p->D[d] * (1.0 + 1e-9) + 1e-12 * p->diam)
                return fail(SLP_ERR_INVALID_ARG, "point %lld lies outside the mesh's bounding box", (long long)i);
            r2 += (x - p->ctr[d]) * (x - p->ctr[d]);
        }
        if (std::sqrt(r2) > 0.5 * p->diam)
            return fail(SLP_ERR_INVALID_ARG, "point %lld lies outside the mesh's enclosing ball", (long long)i);
    }
    DeviceGuard g(p->device);
    slp_probe_s *pr = new slp_probe_s();
    pr->plan = p;
    pr->device = p->device;
    pr->n = n;
    const slp_status st = p->prec == 64 ? probe_build<double>(*p, points, n, *pr) : probe_build<float>(*p, points, n, *pr);
    if (st != SLP_OK) {
        for (void *a : pr->allocs) cudaFree(a);
        delete pr;
        return st;
    }
    *out = pr;
    return SLP_OK;
}

slp_status slp_eval_probe(slp_plan_t p, slp_probe_t pr, int kind, const void *d_in, void *d_phi, void *d_phi_points,
                          void *stream) {
    if (!p || !pr || pr->plan != p) return fail(SLP_ERR_INVALID_ARG, "plan and probe set do not belong together");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan cannot evaluate");
    TRY(slp_check_kind(*p, kind));
    if (kind != SLP_INPUT_NODAL_MAG && kind != SLP_INPUT_ELEMENT)
        return fail(SLP_ERR_UNSUPPORTED, "probes take nodal or element input");
    if (!d_in || !d_phi || !d_phi_points) return fail(SLP_ERR_INVALID_ARG, "input or output pointer is NULL");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(run_pipeline(*p, kind, d_in, d_phi, s, SLP_STAGE_NEAR));
    // the probes' near-field part, then their interpolation from the same grid B
    const slp::DevPlan &v = pr->view;
    if (p->opts.integration) {
        const void *gch = kind == SLP_INPUT_ELEMENT ? d_in : p->dp.gbuf;
        TRY(cuda_status(slp::launch_csr_apply(p->prec, 32, pr->n, v.nt_rowptr, nullptr, v.nt_col, v.nt_val, gch,
                                              v.phi_part, s), "probe near field"));
    } else {
        TRY(cuda_status(slp::launch_near_matrix(v, nullptr, s), "probe near field"));
    }
    TRY(cuda_status(slp::launch_gather(v, d_phi_points, s), "probe gather"));
    return SLP_OK;
}

slp_status slp_probe_query(slp_probe_t pr, int64_t *n_points, int64_t *near_nnz) {
    if (!pr) return fail(SLP_ERR_INVALID_ARG, "probe is NULL");
    if (n_points) *n_points = pr->n;
    if (near_nnz) *near_nnz = pr->near_nnz;
    return SLP_OK;
}

slp_status slp_probe_destroy(slp_probe_t pr) {
    if (!pr) return SLP_OK;
    {
        DeviceGuard g(pr->device);
        cudaDeviceSynchronize();
        for (void *a : pr->allocs) cudaFree(a);
    }
    delete pr;
    return SLP_OK;
}

slp_status slp_eval_host_wait(slp_plan_t p) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return SLP_OK;
    DeviceGuard g(p->device);
    return cuda_status(cudaStreamSynchronize(p->cs_out), "synchronize copy-out");
}

slp_status slp_query(slp_plan_t p, slp_info *info) {
    if (!p || !info) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof *info);
    info->n_targets = p->N;
    info->n_sources = p->Q;
    info->n_triangles = p->M;
    info->quadrature = p->q;
    info->precision = p->prec;
    for (int d = 0; d < 3; ++d) {
        info->grid[d] = p->L[d];
        info->modes[d] = p->n[d];
        info->center[d] = p->ctr[d];
        info->period[d] = p->P[d];
    }
    info->m = p->m;
    info->kernel_mode = p->kernel_mode;
    info->near_mode = p->near_mode;
    info->grid_raised = p->grid_raised;
    info->sigma_g = p->sigma_g;
    info->trunc_radius = p->R;
    info->eps_near = p->eps;
    info->tolerance = p->tol;
    info->near_pairs = p->near_pairs;
    info->near_pairs_within = p->near_pairs_within;
    info->near_matrix_nnz = p->nm_nnz;
    info->bytes_device = p->bytes_device;
    info->n_spread_items = (int64_t)p->spread_items.size();
    info->n_gather_items = (int64_t)p->gather_items.size();
    info->n_near_items = (int64_t)p->near_items.size();
    info->launches_per_eval = p->launches_per_eval;
    info->active_rows = 2 * (int64_t)p->row_pairs.size();
    info->active_planes = p->nz_act;
    info->fused_plane_passes = p->device >= 0 && p->dp.fuse_pb > 0 ? 1 : 0;
    info->fused_column_passes = p->device >= 0 && p->dp.yzy_g > 0 ? 1 : 0;
    info->gather_item_targets = p->gather_chunk;
    info->spread_blocks_per_sm = (p->prec == 32 && p->m <= 4) ? (spread_dense(*p) ? 4 : 5) : 0;
    info->spread_table = p->dp.wtab != nullptr ? 1 : 0;
    info->expsum_terms = p->kernel_mode == SLP_KERNEL_EXPSUM ? (int)p->es_w.size() : 0;
    info->integration = p->opts.integration ? 1 : 0;
    info->grid_matrix_nnz = p->am_nnz;
    info->grid_matrix_rows = p->dp.am_rows;
    info->deterministic_spread = p->dp.det_spread;
    info->near_tri_nnz = p->nt_nnz;
    return SLP_OK;
}

slp_status slp_query_points(slp_plan_t p, double *points) {
    if (!p || !points) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    memcpy(points, p->y.data(), sizeof(double) * 3 * p->Q);
    return SLP_OK;
}

slp_status slp_check(slp_plan_t p) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return SLP_OK;
    DeviceGuard g(p->device);
    TRY(cuda_status(cudaDeviceSynchronize(), "synchronize"));
    int code = 0;
    TRY(cuda_status(cudaMemcpy(&code, p->dp.err, sizeof(int), cudaMemcpyDeviceToHost), "read status"));
    if (code != 0) {
        cudaMemset(p->dp.err, 0, sizeof(int));
        if (code == slp::DEV_ERR_NONFINITE)
            return fail(SLP_ERR_NONFINITE, "checked evaluation saw a NaN or Inf in its input or result");
        return fail(SLP_ERR_CUDA, "device status word %d (a kernel saw an inconsistent work item)", code);
    }
    return SLP_OK;
}

slp_status slp_destroy(slp_plan_t p) {
    if (!p) return SLP_OK;
    slp_batch_cache_drop(p);
    free_device(*p);
    delete p;
    return SLP_OK;
}

const char *slp_status_string(slp_status s) {
    switch (s) {
        case SLP_OK: return "ok";
        case SLP_ERR_INVALID_ARG: return "invalid argument";
        case SLP_ERR_MESH: return "invalid mesh";
        case SLP_ERR_TOLERANCE_INFEASIBLE: return "tolerance infeasible on this grid";
        case SLP_ERR_OOM: return "out of device memory";
        case SLP_ERR_CUDA: return "CUDA error";
        case SLP_ERR_TIMEOUT: return "device wait timed out";
        case SLP_ERR_NONFINITE: return "non-finite value";
        case SLP_ERR_NO_DEVICE: return "no CUDA device";
        case SLP_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char *slp_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------- debug ABI
slp_status slp_debug_run(slp_plan_t p, int kind, const void *d_in, void *d_phi, void *stream, int last) {
    if (!p) return fail(SLP_ERR_INVALID_ARG, "plan is NULL");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan");
    if (!d_in || !d_phi) return fail(SLP_ERR_INVALID_ARG, "bad input");
    TRY(slp_check_kind(*p, kind));
    DeviceGuard g(p->device);
    // a partial run may have left a spread grid behind: start from zero
    const size_t es = p->prec == 64 ? 8 : 4;
    TRY(cuda_status(slp::launch_zero(p->dp.gridA, es * (size_t)p->L[0] * p->L[1] * p->L[2], (cudaStream_t)stream),
                    "zero grid"));
    return run_pipeline(*p, kind, d_in, d_phi, (cudaStream_t)stream, last);
}

slp_status slp_debug_buffer_bytes(slp_plan_t p, int buf, int64_t *bytes) {
    if (!p || !bytes) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    const int64_t es = p->prec == 64 ? 8 : 4;
    const int64_t G = (int64_t)p->L[0] * p->L[1] * p->L[2];
    const int64_t Kx = p->n[0] / 2;
    switch (buf) {
        case SLP_BUF_QBUF: *bytes = es * p->Q; break;
        case SLP_BUF_GRID_A:
        case SLP_BUF_GRID_B: *bytes = es * G; break;
        case SLP_BUF_S1: *bytes = 2 * es * p->L[2] * p->L[1] * Kx; break;
        case SLP_BUF_S2: *bytes = 2 * es * p->L[2] * p->n[1] * Kx; break;
        case SLP_BUF_DTAB: *bytes = es * (int64_t)p->Dtab.size(); break;
        default: return fail(SLP_ERR_INVALID_ARG, "unknown buffer %d", buf);
    }
    return SLP_OK;
}

slp_status slp_debug_copy(slp_plan_t p, int buf, void *host, int64_t bytes) {
    if (!p || !host) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan");
    int64_t need = 0;
    TRY(slp_debug_buffer_bytes(p, buf, &need));
    if (bytes != need) return fail(SLP_ERR_INVALID_ARG, "buffer %d holds %lld bytes", buf, (long long)need);
    const void *src = nullptr;
    switch (buf) {
        case SLP_BUF_QBUF: src = p->dp.qbuf; break;
        case SLP_BUF_GRID_A: src = p->dp.gridA; break;
        case SLP_BUF_GRID_B: src = p->dp.gridB; break;
        case SLP_BUF_S1: src = p->dp.S1; break;
        case SLP_BUF_S2: src = p->dp.S2; break;
        case SLP_BUF_DTAB: src = p->dp.Dtab; break;
    }
    DeviceGuard g(p->device);
    TRY(cuda_status(cudaDeviceSynchronize(), "synchronize"));
    TRY(cuda_status(cudaMemcpy(host, src, (size_t)bytes, cudaMemcpyDeviceToHost), "copy"));
    return SLP_OK;
}

slp_status slp_debug_host_count(slp_plan_t p, int which, int64_t *count) {
    if (!p || !count) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    switch (which) {
        case SLP_HOST_SRC_PERM: *count = p->Q; break;
        case SLP_HOST_TGT_PERM: *count = p->N; break;
        case SLP_HOST_SRC_GRID: *count = 4 * p->Q; break;
        case SLP_HOST_TGT_GRID: *count = 4 * p->N; break;
        case SLP_HOST_SPREAD_ITEMS: *count = 8 * (int64_t)p->spread_items.size(); break;
        case SLP_HOST_GATHER_ITEMS: *count = 8 * (int64_t)p->gather_items.size(); break;
        case SLP_HOST_NEAR_ITEMS: *count = 4 * (int64_t)p->near_items.size(); break;
        case SLP_HOST_NEAR_RANGES: *count = 2 * (int64_t)p->near_ranges.size(); break;
        case SLP_HOST_DTAB: *count = (int64_t)p->Dtab.size(); break;
        case SLP_HOST_SRC_POINTS: *count = 3 * p->Q; break;
        case SLP_HOST_TGT_POINTS: *count = 3 * p->N; break;
        case SLP_HOST_PLANE_ROWS: *count = 2 * (int64_t)p->plane_iv.size(); break;
        case SLP_HOST_ACTIVE_Z: *count = 2; break;
        case SLP_HOST_SPREAD_GROUPS: *count = (int64_t)p->sgroups.size(); break;
        case SLP_HOST_EXPSUM: *count = (int64_t)(2 * p->es_w.size()); break;
        case SLP_HOST_SPREAD_GROUP_OFF: *count = (int64_t)p->sgroup_off.size(); break;
        default: return fail(SLP_ERR_INVALID_ARG, "unknown host array %d", which);
    }
    return SLP_OK;
}

slp_status slp_debug_host_array(slp_plan_t p, int which, void *out, int64_t count) {
    int64_t need = 0;
    TRY(slp_debug_host_count(p, which, &need));
    if (!out || count != need) return fail(SLP_ERR_INVALID_ARG, "array %d has %lld elements", which, (long long)need);
    switch (which) {
        case SLP_HOST_SRC_PERM: memcpy(out, p->src_perm.data(), 4 * count); break;
        case SLP_HOST_TGT_PERM: memcpy(out, p->tgt_perm.data(), 4 * count); break;
        case SLP_HOST_SRC_GRID: memcpy(out, p->src_grid.data(), 8 * count); break;
        case SLP_HOST_TGT_GRID: memcpy(out, p->tgt_grid.data(), 8 * count); break;
        case SLP_HOST_SPREAD_ITEMS: memcpy(out, p->spread_items.data(), 4 * count); break;
        case SLP_HOST_GATHER_ITEMS: memcpy(out, p->gather_items.data(), 4 * count); break;
        case SLP_HOST_NEAR_ITEMS: memcpy(out, p->near_items.data(), 4 * count); break;
        case SLP_HOST_NEAR_RANGES: memcpy(out, p->near_ranges.data(), 4 * count); break;
        case SLP_HOST_DTAB: memcpy(out, p->Dtab.data(), 8 * count); break;
        case SLP_HOST_SRC_POINTS: {
            double *o = (double *)out;
            for (int64_t i = 0; i < p->Q; ++i)
                for (int d = 0; d < 3; ++d) o[3 * i + d] = p->y[3 * (int64_t)p->src_perm[i] + d];
            break;
        }
        case SLP_HOST_TGT_POINTS: {
            double *o = (double *)out;
            for (int64_t i = 0; i < p->N; ++i)
                for (int d = 0; d < 3; ++d) o[3 * i + d] = p->V[3 * (int64_t)p->tgt_perm[i] + d];
            break;
        }
        case SLP_HOST_PLANE_ROWS: memcpy(out, p->plane_iv.data(), 4 * count); break;
        case SLP_HOST_SPREAD_GROUPS: memcpy(out, p->sgroups.data(), 4 * count); break;
        case SLP_HOST_EXPSUM:
            for (size_t k = 0; k < p->es_w.size(); ++k) {
                ((double *)out)[2 * k] = p->es_w[k];
                ((double *)out)[2 * k + 1] = p->es_g[k];
            }
            break;
        case SLP_HOST_SPREAD_GROUP_OFF: memcpy(out, p->sgroup_off.data(), 4 * count); break;
        case SLP_HOST_ACTIVE_Z: {
            int32_t *o = (int32_t *)out;
            o[0] = p->z0;
            o[1] = p->nz_act;
            break;
        }
    }
    return SLP_OK;
}

slp_status slp_debug_profile(slp_plan_t p, int kind, const void *d_in, void *d_phi, void *stream, float *ms,
                             int n) {
    if (!p || !ms) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan");
    if (n < SLP_PROFILE_SLOTS) return fail(SLP_ERR_INVALID_ARG, "need room for %d timings", SLP_PROFILE_SLOTS);
    if (!d_in || !d_phi) return fail(SLP_ERR_INVALID_ARG, "bad input");
    TRY(slp_check_kind(*p, kind));
    DeviceGuard g(p->device);
    SlpProfile prof;
    for (int i = 0; i < 2 * SLP_PROFILE_SLOTS; ++i)
        if (cudaEventCreate(&prof.ev[i]) != cudaSuccess) return fail(SLP_ERR_CUDA, "cudaEventCreate");
    for (int i = 0; i < SLP_PROFILE_SLOTS; ++i) prof.launched[i] = false;
    slp_status st = run_pipeline(*p, kind, d_in, d_phi, (cudaStream_t)stream, SLP_STAGE_NEAR, &prof);
    if (st == SLP_OK) st = cuda_status(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    for (int i = 0; i < SLP_PROFILE_SLOTS && st == SLP_OK; ++i) {
        float t = -1.f;
        if (prof.launched[i]) st = cuda_status(cudaEventElapsedTime(&t, prof.ev[2 * i], prof.ev[2 * i + 1]), "elapsed");
        ms[i] = t;
    }
    for (int i = 0; i < 2 * SLP_PROFILE_SLOTS; ++i) cudaEventDestroy(prof.ev[i]);
    return st;
}

slp_status slp_debug_timeline(slp_plan_t p, int kind, const void *d_in, void *d_phi, void *stream, float *ms) {
    if (!p || !ms) return fail(SLP_ERR_INVALID_ARG, "NULL argument");
    if (p->device < 0) return fail(SLP_ERR_NO_DEVICE, "host-only plan");
    if (!d_in || !d_phi) return fail(SLP_ERR_INVALID_ARG, "bad input");
    TRY(slp_check_kind(*p, kind));
    DeviceGuard g(p->device);
    cudaEvent_t tl[5];
    for (int i = 0; i < 5; ++i)
        if (cudaEventCreate(&tl[i]) != cudaSuccess) return fail(SLP_ERR_CUDA, "cudaEventCreate");
    p->exec.timeline = tl;
    slp_status st = run_pipeline(*p, kind, d_in, d_phi, (cudaStream_t)stream, SLP_STAGE_NEAR);
    p->exec.timeline = nullptr;
    if (st == SLP_OK) st = cuda_status(cudaEventSynchronize(tl[4]), "event sync");
    for (int i = 1; i < 5 && st == SLP_OK; ++i) st = cuda_status(cudaEventElapsedTime(&ms[i - 1], tl[0], tl[i]), "elapsed");
    for (int i = 0; i < 5; ++i) cudaEventDestroy(tl[i]);
    return st;
}

const char *slp_debug_stage_name(int i) { return (i >= 0 && i < SLP_PROFILE_SLOTS) ? STAGE_NAMES[i] : ""; }

double slp_debug_window(int m, double d) { return kb_window_host(m, d); }
double slp_debug_window_hat(int m, int L, double l) { return kb_hat_host(m, L, l); }

}  // extern "C"
