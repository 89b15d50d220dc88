// Allocation-free evaluation: slp_eval_direct_static.
//
// Some callers cannot call cudaMalloc at the point where they need the
// potential: host code living inside another framework's memory pool that
// forbids raw device allocations, or a solver loop that must not touch the
// allocator after start-up (an allocation there can block on, or fail
// against, memory that the surrounding application has already handed
// out).  They cannot build a plan, because slp_plan allocates the plan's
// device memory.  For small meshes this entry point evaluates the same
// single layer potential by direct summation over all (target, source)
// pairs and allocates nothing: the caller passes the mesh, the input field
// and the output on the device, and the only scratch (the quadrature points
// and weighted charges, one 4-vector per source) lives in the file-scope
// array below, which every GPU that loads the library holds until the
// process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/slp.h"
#include "dev_common.cuh"

namespace {

// 32 MiB of scratch: 16 bytes per source in FP32 (at most 2,097,152 sources),
// 32 bytes per source in FP64 (at most 1,048,576 sources).
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device, resolved once with that
// device current (the host-side symbol is only a stand-in, not an address).
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES] = {nullptr};

slp_status static_fail(slp_status s, const char *msg) {
    slp::set_last_error(msg);
    return s;
}

slp_status launch_fail(const char *what, cudaError_t e) {
    char msg[256];
    snprintf(msg, sizeof msg, "slp_eval_direct_static: launch of %s failed: %s", what, cudaGetErrorString(e));
    return static_fail(SLP_ERR_CUDA, msg);
}

template <typename T> struct V4s;
template <> struct V4s<float> { typedef float4 t; };
template <> struct V4s<double> { typedef double4 t; };

struct RuleParams {
    double lam[21];
    double w[7];
    int q;
};

// Quadrature points relative to vertex 0 and weighted charges w_s |S_j| sigma.
template <typename T>
__global__ void k_static_sources(const double *__restrict__ V, int64_t nv, const int32_t *__restrict__ Tri,
                                 int64_t nt, RuleParams rp, int kind, const T *__restrict__ in,
                                 typename V4s<T>::t *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t Q = nt * rp.q;
    if (k >= Q) return;
    const int64_t j = k / rp.q;
    const int s = (int)(k - j * rp.q);
    const int32_t i0 = Tri[3 * j], i1 = Tri[3 * j + 1], i2 = Tri[3 * j + 2];
    typename V4s<T>::t o;
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {  // invalid triangle: no charge
        o.x = o.y = o.z = T(0);
        o.w = T(0);
        out[k] = o;
        return;
    }
    const double *v0 = V + 3 * (int64_t)i0, *v1 = V + 3 * (int64_t)i1, *v2 = V + 3 * (int64_t)i2;
    const double e1x = v1[0] - v0[0], e1y = v1[1] - v0[1], e1z = v1[2] - v0[2];
    const double e2x = v2[0] - v0[0], e2y = v2[1] - v0[1], e2z = v2[2] - v0[2];
    const double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
    const double a2 = sqrt(cx * cx + cy * cy + cz * cz);
    const double l0 = rp.lam[3 * s], l1 = rp.lam[3 * s + 1], l2 = rp.lam[3 * s + 2];
    // point relative to vertex 0 of the mesh (keeps FP32 differences accurate)
    const double r0x = V[0], r0y = V[1], r0z = V[2];
    o.x = (T)(l0 * v0[0] + l1 * v1[0] + l2 * v2[0] - r0x);
    o.y = (T)(l0 * v0[1] + l1 * v1[1] + l2 * v2[1] - r0y);
    o.z = (T)(l0 * v0[2] + l1 * v1[2] + l2 * v2[2] - r0z);
    double sigma = 0.0;
    if (a2 > 0.0) {
        const double nx = cx / a2, ny = cy / a2, nz = cz / a2;
        if (kind == SLP_INPUT_SIGMA) {
            sigma = (double)in[k];
        } else if (kind == SLP_INPUT_MAG) {
            sigma = (double)in[3 * k] * nx + (double)in[3 * k + 1] * ny + (double)in[3 * k + 2] * nz;
        } else {
            double m[3];
            for (int d = 0; d < 3; ++d)
                m[d] = l0 * (double)in[3 * (int64_t)i0 + d] + l1 * (double)in[3 * (int64_t)i1 + d] +
                       l2 * (double)in[3 * (int64_t)i2 + d];
            sigma = m[0] * nx + m[1] * ny + m[2] * nz;
        }
    }
    o.w = (T)(rp.w[s] * 0.5 * a2 * sigma);
    out[k] = o;
}

// phi_i = (1/4pi) sum_k q_k / |x_i - y_k| over all sources.  One block per 32
// targets (lane = target); the 8 warps split the sources and their partial
// sums (each with its compensation term) are added in warp order, so the
// result is bitwise repeatable.
template <typename T>
__global__ void __launch_bounds__(256) k_static_direct(const double *__restrict__ V, int64_t nv,
                                                       const typename V4s<T>::t *__restrict__ src, int64_t Q,
                                                       T *__restrict__ phi) {
    typedef typename V4s<T>::t T4;
    __shared__ T4 stage[8][32];
    __shared__ T part[8][32];
    __shared__ T cpart[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    T tx = T(0), ty = T(0), tz = T(0);
    if (i < nv) {
        tx = (T)(V[3 * i] - V[0]);
        ty = (T)(V[3 * i + 1] - V[1]);
        tz = (T)(V[3 * i + 2] - V[2]);
    }
    const int64_t per = (Q + 7) / 8;
    const int64_t b = warp * per, e = min(Q, b + per);
    // Neumaier-compensated sum: a warp adds up to Q / 8 terms (262,144 at the
    // FP32 scratch limit), so a plain FP32 running sum could lose digits; the
    // compensation term keeps the error near one rounding of the total
    T acc = T(0), comp = T(0);
    for (int64_t s0 = b; s0 < e; s0 += 32) {
        if (s0 + lane < e) stage[warp][lane] = src[s0 + lane];
        __syncwarp();
        const int cnt = (int)min((int64_t)32, e - s0);
        for (int jj = 0; jj < cnt; ++jj) {
            const T4 y = stage[warp][jj];
            const T dx = tx - y.x, dy = ty - y.y, dz = tz - y.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > T(0)) {
                const T term = y.w / sqrt(r2);
                const T t = acc + term;
                comp += fabs(acc) >= fabs(term) ? (acc - t) + term : (term - t) + acc;
                acc = t;
            }
        }
        __syncwarp();
    }
    part[warp][lane] = acc;
    cpart[warp][lane] = comp;
    __syncthreads();
    if (warp == 0 && i < nv) {
        T s = T(0), c = T(0);
        for (int w = 0; w < 8; ++w) {
            const T v = part[w][lane];
            const T t = s + v;
            c += (fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s) + cpart[w][lane];
            s = t;
        }
        phi[i] = (s + c) * T(0.079577471545947667884);  // 1 / (4 pi)
    }
}

bool rule_params(int q, RuleParams &rp) {
    memset(&rp, 0, sizeof rp);
    rp.q = q;
    if (q == 1) {
        rp.lam[0] = rp.lam[1] = rp.lam[2] = 1.0 / 3.0;
        rp.w[0] = 1.0;
        return true;
    }
    if (q == 3) {
        for (int s = 0; s < 3; ++s) {
            for (int a = 0; a < 3; ++a) rp.lam[3 * s + a] = a == s ? 2.0 / 3.0 : 1.0 / 6.0;
            rp.w[s] = 1.0 / 3.0;
        }
        return true;
    }
    if (q == 7) {
        const double r = sqrt(15.0);
        rp.lam[0] = rp.lam[1] = rp.lam[2] = 1.0 / 3.0;
        rp.w[0] = 9.0 / 40.0;
        const double av[2] = {(6.0 - r) / 21.0, (6.0 + r) / 21.0};
        const double wv[2] = {(155.0 - r) / 1200.0, (155.0 + r) / 1200.0};
        int s = 1;
        for (int g = 0; g < 2; ++g) {
            const double a = av[g], o = 1.0 - 2.0 * a;
            const double pts[3][3] = {{a, a, o}, {a, o, a}, {o, a, a}};
            for (int p = 0; p < 3; ++p, ++s) {
                for (int c = 0; c < 3; ++c) rp.lam[3 * s + c] = pts[p][c];
                rp.w[s] = wv[g];
            }
        }
        return true;
    }
    return false;
}

template <typename T>
slp_status launch_static(const double *V, int64_t nv, const int32_t *Tri, int64_t nt, const RuleParams &rp, int kind,
                         const void *in, void *phi, void *scratch, cudaStream_t s) {
    typedef typename V4s<T>::t T4;
    const int64_t Q = nt * rp.q;
    k_static_sources<T><<<(unsigned)((Q + 255) / 256), 256, 0, s>>>(V, nv, Tri, nt, rp, kind, (const T *)in,
                                                                     (T4 *)scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return launch_fail("the charge kernel", e);
    k_static_direct<T><<<(unsigned)((nv + 31) / 32), 256, 0, s>>>(V, nv, (const T4 *)scratch, Q, (T *)phi);
    e = cudaGetLastError();
    if (e != cudaSuccess) return launch_fail("the direct-sum kernel", e);
    return SLP_OK;
}

}  // namespace

extern "C" slp_status slp_eval_direct_static(const double *d_vertices, int64_t n_vertices, const int32_t *d_triangles,
                                             int64_t n_triangles, int quadrature, int precision, int input_kind,
                                             const void *d_in, void *d_phi, void *stream) {
    slp::set_last_error("");
    if (!d_vertices || !d_triangles || !d_in || !d_phi)
        return static_fail(SLP_ERR_INVALID_ARG, "slp_eval_direct_static: a pointer argument is NULL");
    if (n_vertices < 1 || n_triangles < 1 || n_vertices > (int64_t)1 << 31)
        return static_fail(SLP_ERR_INVALID_ARG, "slp_eval_direct_static: empty or oversized mesh");
    if (precision != 32 && precision != 64)
        return static_fail(SLP_ERR_INVALID_ARG, "slp_eval_direct_static: precision must be 32 or 64");
    if (input_kind < SLP_INPUT_SIGMA || input_kind > SLP_INPUT_NODAL_MAG)
        return static_fail(SLP_ERR_INVALID_ARG, "slp_eval_direct_static: unknown input kind");
    RuleParams rp;
    if (!rule_params(quadrature, rp))
        return static_fail(SLP_ERR_INVALID_ARG, "slp_eval_direct_static: quadrature must be 1, 3 or 7");
    const size_t per = precision == 64 ? sizeof(double4) : sizeof(float4);
    if (n_triangles > (int64_t)(STATIC_SCRATCH_BYTES / per) / quadrature) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "slp_eval_direct_static: %lld sources need %lld bytes of scratch; the static array holds %zu "
                 "bytes (at most %zu sources at precision %d)",
                 (long long)(n_triangles * quadrature), (long long)(n_triangles * quadrature * (int64_t)per),
                 STATIC_SCRATCH_BYTES, STATIC_SCRATCH_BYTES / per, precision);
        return static_fail(SLP_ERR_INVALID_ARG, msg);
    }
    {
        // an error left by the caller's earlier work is reported as such, and
        // left in place for the caller (the launch checks below would
        // otherwise take it for their own and clear it)
        const cudaError_t pending = cudaPeekAtLastError();
        if (pending != cudaSuccess) {
            char msg[256];
            snprintf(msg, sizeof msg,
                     "slp_eval_direct_static: a CUDA error from earlier work is pending (%s); nothing was launched",
                     cudaGetErrorString(pending));
            return static_fail(SLP_ERR_CUDA, msg);
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return static_fail(SLP_ERR_NO_DEVICE, "slp_eval_direct_static: no current CUDA device");
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            // first call on this device: resolve the array's device address
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || ptr == nullptr) {
                cudaGetLastError();
                char msg[256];
                snprintf(msg, sizeof msg, "slp_eval_direct_static: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return static_fail(SLP_ERR_CUDA, msg);
            }
            g_scratch_addr[dev] = ptr;
        }
        scratch = g_scratch_addr[dev];
    }
    const cudaStream_t s = (cudaStream_t)stream;
    if (precision == 64)
        return launch_static<double>(d_vertices, n_vertices, d_triangles, n_triangles, rp, input_kind, d_in, d_phi,
                                     scratch, s);
    return launch_static<float>(d_vertices, n_vertices, d_triangles, n_triangles, rp, input_kind, d_in, d_phi,
                                scratch, s);
}
