// Near-field correction (paper Sec. 3.4, Eq. (nfcorr)):
//
//   phi_i += sum_{k : |x_i - y_k| < eps} qk (N - N_s)(x_i - y_k),
//
// where N_s is the smooth kernel the far path actually applies:
//   RADIAL:    (N - N_s)(r) = erfc(r / (s sqrt 2)) / (4 pi r)  (r < eps);
//   SEPARABLE: (N - N_s)(d) = 1/(4 pi |d|) - A prod_q f_q(d_q / L_q), every pair;
//   EXPSUM:    (N - N_s)(r) = (1/r - sum_k w_k exp(-g_k r^2)) / (4 pi)  (r < eps,
//              the exponential sum of Sec. 3.3).
//
// One warp per work item: lane t owns target tbegin + t; the warp walks the
// item's source ranges 32 sources at a time, staging them in shared memory
// and broadcasting each to all lanes.  Pair distances are formed from the
// integer cell difference plus the fractional offsets, so they keep full
// precision however far the mesh sits from the origin.
#include "dev_common.cuh"

namespace slp {

constexpr int NEAR_WARPS = 8;

template <typename T> __device__ __forceinline__ T near_erfc(T x);
template <> __device__ __forceinline__ float near_erfc<float>(float x) { return erfcf(x); }
template <> __device__ __forceinline__ double near_erfc<double>(double x) { return erfc(x); }
__device__ __forceinline__ float near_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double near_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float near_cospi(float x) { return cospif(x); }
__device__ __forceinline__ double near_cospi(double x) { return cospi(x); }
__device__ __forceinline__ float near_exp(float x) { return expf(x); }
__device__ __forceinline__ double near_exp(double x) { return exp(x); }

// sum_k w_k exp(-g_k r2) of the exp-sum kernel
template <typename T> __device__ __forceinline__ T expsum_value(const T *__restrict__ w, const T *__restrict__ g, int n, T r2) {
    T s = T(0);
    for (int k = 0; k < n; ++k) s += w[k] * near_exp(-g[k] * r2);
    return s;
}

// f(t) = h[0] + 2 sum_{l>=1} h[l] cos(2 pi l t), by Clenshaw's recurrence in x = cos(2 pi t).
template <typename T> __device__ __forceinline__ T sep_factor(const T *__restrict__ h, int nh, T t) {
    const T x = near_cospi(T(2) * t);
    T b1 = T(0), b2 = T(0);
    for (int l = nh - 1; l >= 1; --l) {
        const T b0 = T(2) * h[l] + T(2) * x * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    // sum_{l>=1} c_l T_l(x) = x b1 - b2 with c_l = 2 h[l]; plus c_0 = h[0]
    return h[0] + x * b1 - b2;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NEAR_WARPS * 32) k_near(DevPlan p) {
    pdl_wait();
    pdl_trigger();
    typedef typename VecT<T>::T4 T4;
    __shared__ T4 sg[NEAR_WARPS][32];
    __shared__ T sq[NEAR_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * NEAR_WARPS + warp;
    if (item >= p.n_near) return;
    const NearItem it = p.near_items[item];
    const bool active = lane < it.tcount;
    int ctx = 0, cty = 0, ctz = 0;
    T ftx = T(0), fty = T(0), ftz = T(0);
    if (active) {
        const T4 g = ((const T4 *)p.tgt_grid)[it.tbegin + lane];
        unpack_cell(packed_cell(g.w), ctx, cty, ctz);
        ftx = g.x;
        fty = g.y;
        ftz = g.z;
    }
    const T hx = (T)p.h[0], hy = (T)p.h[1], hz = (T)p.h[2];
    const T eps2 = (T)p.eps2;
    const T a = (T)p.inv_s_sqrt2;
    const T4 *src = (const T4 *)p.src_grid;
    const T *qb = (const T *)p.qbuf;
    T acc = T(0);
    for (int r = it.rbegin; r < it.rend; ++r) {
        const int2 rg = p.near_ranges[r];
        for (int s0 = rg.x; s0 < rg.y; s0 += 32) {
            const int s = s0 + lane;
            if (s < rg.y) {
                sg[warp][lane] = src[s];
                sq[warp][lane] = qb[s];
            }
            __syncwarp();
            const int cnt = min(32, rg.y - s0);
            for (int j = 0; j < cnt; ++j) {
                const T4 g = sg[warp][j];
                int csx, csy, csz;
                unpack_cell(packed_cell(g.w), csx, csy, csz);
                const T dx = (T(ctx - csx) + (ftx - g.x)) * hx;
                const T dy = (T(cty - csy) + (fty - g.y)) * hy;
                const T dz = (T(ctz - csz) + (ftz - g.z)) * hz;
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (MODE == 1) {
                    if (r2 < eps2) {
                        const T ri = near_rsqrt(r2);
                        acc += sq[warp][j] * near_erfc<T>(r2 * ri * a) * ri;
                    }
                } else if (MODE == 3) {
                    if (r2 < eps2)
                        acc += sq[warp][j] *
                               (near_rsqrt(r2) - expsum_value((const T *)p.es_w, (const T *)p.es_g, p.es_n, r2));
                } else {
                    const T ri = near_rsqrt(r2);
                    const T ux = (T(ctx - csx) + (ftx - g.x)) / T(p.L[0]);
                    const T uy = (T(cty - csy) + (fty - g.y)) / T(p.L[1]);
                    const T uz = (T(ctz - csz) + (ftz - g.z)) / T(p.L[2]);
                    const T kn = sep_factor((const T *)p.sep_h[0], p.sep_nh[0], ux) *
                                 sep_factor((const T *)p.sep_h[1], p.sep_nh[1], uy) *
                                 sep_factor((const T *)p.sep_h[2], p.sep_nh[2], uz);
                    acc += sq[warp][j] * (ri - T(p.sep_A) * kn);
                }
            }
            __syncwarp();
        }
    }
    if (active) {
        const T v = acc * T(0.079577471545947667884);  // 1 / (4 pi)
        if (p.deterministic)
            ((T *)p.phi_near)[(int64_t)item * 32 + lane] = v;
        else
            atomicAdd((T *)p.phi_part + it.tbegin + lane, v);
    }
}

// Deterministic mode: items of one target block are consecutive; add their
// partials in item order.  blk_items[b] = first item of block b (CSR).
template <typename T>
__global__ void k_near_reduce(DevPlan p, const int *__restrict__ blk_first, int nblk) {
    pdl_wait();
    pdl_trigger();
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int i0 = blk_first[b], i1 = blk_first[b + 1];
    const NearItem it0 = p.near_items[i0];
    if (lane >= it0.tcount) return;
    T s = T(0);
    for (int i = i0; i < i1; ++i) s += ((const T *)p.phi_near)[(int64_t)i * 32 + lane];
    ((T *)p.phi_part)[it0.tbegin + lane] = s;
}

template <typename T> static cudaError_t near_t(const DevPlan &p, cudaStream_t s) {
    if (p.n_near == 0) return cudaSuccess;
    const int nb = (p.n_near + NEAR_WARPS - 1) / NEAR_WARPS;
    if (p.kernel_mode == 2)
        { const cudaError_t le = launch_k(k_near<T, 2>, nb, NEAR_WARPS * 32, 0, s, p); if (le != cudaSuccess) return le; }
    else if (p.kernel_mode == 3)
        { const cudaError_t le = launch_k(k_near<T, 3>, nb, NEAR_WARPS * 32, 0, s, p); if (le != cudaSuccess) return le; }
    else
        { const cudaError_t le = launch_k(k_near<T, 1>, nb, NEAR_WARPS * 32, 0, s, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

cudaError_t launch_near(const DevPlan &p, cudaStream_t s) {
    return p.prec == 64 ? near_t<double>(p, s) : near_t<float>(p, s);
}

cudaError_t launch_near_reduce(const DevPlan &p, const int *blk_first, int nblk, cudaStream_t s) {
    if (nblk == 0) return cudaSuccess;
    const int nb = (nblk + 7) / 8;
    if (p.prec == 64)
        { const cudaError_t le = launch_k(k_near_reduce<double>, nb, 256, 0, s, p, blk_first, nblk); if (le != cudaSuccess) return le; }
    else
        { const cudaError_t le = launch_k(k_near_reduce<float>, nb, 256, 0, s, p, blk_first, nblk); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

}  // namespace slp

// =====================================================================
// Precomputed near-field operator for nodal magnetisation input.
//
// With sigma_k = m(y_k) . n_j and m interpolated linearly from the vertices
// (P1, Sec. 2.1), the near-field correction is linear in the nodal m:
//   phi_i += sum_v W_iv . m_v,
//   W_iv = sum_{k near x_i, v a vertex of tri(k)} w_k (N - N_s)(x_i - y_k) lambda_{s(k), a(v)} n_{j(k)}.
// The paper precomputes the near-field integrals in the set-up phase and
// applies them as a sparse matrix (Sec. 3.4); here W is assembled once per
// plan on the GPU in FP64 (two passes: count, fill) and stored as one
// 4-vector (W_x, W_y, W_z, vertex id) per non-zero, rows in sorted target
// order.  Each evaluation is then a sparse product streamed from HBM.
namespace slp {

__device__ __forceinline__ double nm_kernel(const NMBuild &b, double dx, double dy, double dz, double r2) {
    const double ri = rsqrt(r2);
    if (b.kernel_mode == 2) {
        const double kn = sep_factor(b.sep_h[0], b.sep_nh[0], dx / b.P[0]) *
                          sep_factor(b.sep_h[1], b.sep_nh[1], dy / b.P[1]) *
                          sep_factor(b.sep_h[2], b.sep_nh[2], dz / b.P[2]);
        return (ri - b.sep_A4pi * kn) * 0.079577471545947667884;
    }
    if (b.kernel_mode == 3) return (ri - expsum_value(b.es_w, b.es_g, b.es_n, r2)) * 0.079577471545947667884;
    return erfc(r2 * ri * b.inv_s_sqrt2) * ri * 0.079577471545947667884;
}

// pass 0: count non-zeros per row (and near pairs); pass 1: fill.
template <typename T4>
__global__ void __launch_bounds__(256) k_nm_build(NMBuild b, int pass, int64_t *__restrict__ counts,
                                                  int64_t *__restrict__ pairs, const int64_t *__restrict__ rowptr,
                                                  T4 *__restrict__ val) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 8 + warp;
    if (t >= b.N) return;
    const double4 xt = b.tgt[t];
    const int blk = b.tgt_block[t];
    int64_t out = pass == 1 ? rowptr[t] : 0;
    int64_t cnt = 0, npairs = 0;
    for (int r = b.blk_r0[blk]; r < b.blk_r0[blk + 1]; ++r) {
        const int2 rg = b.ranges[r];
        for (int u0 = rg.x; u0 < rg.y; u0 += 32) {
            const int u = u0 + lane;
            double wx = 0.0, wy = 0.0, wz = 0.0;
            int v = -1;
            if (u < rg.y) {
                v = b.tgt_perm[u];
                for (int e = b.vt_ptr[v]; e < b.vt_ptr[v + 1]; ++e) {
                    const int ent = b.vt_ent[e];
                    const int j = ent >> 2, a = ent & 3;
                    const double4 n = b.nrm[j];
                    double acc = 0.0;
                    for (int s = 0; s < b.q; ++s) {
                        const double4 y = b.src[(int64_t)j * b.q + s];
                        const double dx = xt.x - y.x, dy = xt.y - y.y, dz = xt.z - y.z;
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < b.eps2 && r2 > 0.0) {
                            acc += y.w * nm_kernel(b, dx, dy, dz, r2) * b.lam[3 * s + a];
                            if (a == 0) ++npairs;
                        }
                    }
                    wx += acc * n.x;
                    wy += acc * n.y;
                    wz += acc * n.z;
                }
            }
            const bool nz = (v >= 0) && (wx != 0.0 || wy != 0.0 || wz != 0.0);
            const unsigned bal = __ballot_sync(0xffffffffu, nz);
            if (pass == 1 && nz) {
                const int pos = __popc(bal & ((1u << lane) - 1u));
                T4 o;
                o.x = wx;
                o.y = wy;
                o.z = wz;
                o.w = pack_id(o.w, u);  // vertex (sorted target position) in the fourth component
                val[out + cnt + pos] = o;
            }
            cnt += __popc(bal);
        }
    }
    npairs = warp_sum((long long)npairs);
    if (pass == 0 && lane == 0) {
        counts[t] = cnt;
        pairs[t] = npairs;
    }
}

cudaError_t launch_nm_build(const NMBuild &b, int pass, int prec, int64_t *counts, int64_t *pairs,
                            const int64_t *rowptr, void *val, cudaStream_t s) {
    const unsigned nb = (unsigned)((b.N + 7) / 8);
    if (prec == 64)
        k_nm_build<double4><<<nb, 256, 0, s>>>(b, pass, counts, pairs, rowptr, (double4 *)val);
    else
        k_nm_build<float4><<<nb, 256, 0, s>>>(b, pass, counts, pairs, rowptr, (float4 *)val);
    return cudaGetLastError();
}

// phi[perm[t]] += sum_e W_e . m[col_e] over row t (sorted target order); one
// warp per row, rows read front to back, lanes combined in a fixed order.
// streaming (evict-first) 16/32-byte load of one matrix entry
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ double4 ld_stream(const double4 *p) {
    const double2 a = __ldcs((const double2 *)p), b = __ldcs((const double2 *)p + 1);
    return make_double4(a.x, a.y, b.x, b.y);
}

// One batch of a near-field row: lane l takes entries j + l + 32 u (u < U),
// 16-byte loads all issued before the gathered m; FULL batches need no
// predicates, the tail batch reads zero weights past the row's end.  The K
// sorted magnetisations are m4[k N + column]; lane l adds its entries in
// order, so a row's sums do not depend on K.
template <typename T, int K, int U, bool FULL>
__device__ __forceinline__ void near_batch(const typename VecT<T>::T4 *__restrict__ row, int j, int n, int lane,
                                           const typename VecT<T>::T4 *__restrict__ m4, int64_t N, T (&acc)[K]) {
    typedef typename VecT<T>::T4 T4;
    T4 w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (FULL || j + lane + 32 * u < n) {
            w[u] = ld_stream(row + j + 32 * u);  // streamed once per evaluation
        } else {
            w[u].x = w[u].y = w[u].z = T(0);
            w[u].w = pack_id(w[u].w, 0);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int col = packed_cell(w[u].w);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T4 mv = m4[k * N + col];
            acc[k] += w[u].x * mv.x + w[u].y * mv.y + w[u].z * mv.z;
        }
    }
}

// Row t of the operator applied to K states: batches of 32 U entries (U
// loads in flight per lane), the full ones without predicates and at 32-bit
// offsets from the row start, then one predicated tail.
template <typename T, int K>
__device__ __forceinline__ void near_row(const DevPlan &p, int64_t t, int lane) {
    typedef typename VecT<T>::T4 T4;
    constexpr int U = 8;
    const T4 *m4 = (const T4 *)p.m4;  // sorted nodal m (k_nodal_prep), K copies
    const int64_t e0 = p.nm_rowptr[t];
    const int n = (int)(p.nm_rowptr[t + 1] - e0);  // a row holds < 2^31 entries
    const T4 *row = (const T4 *)p.nm_val + e0 + lane;
    T acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = T(0);
    int j = 0;
    for (; j + 32 * U <= n; j += 32 * U) near_batch<T, K, U, true>(row, j, n, lane, m4, p.N, acc);
    if (j < n) near_batch<T, K, U, false>(row, j, n, lane, m4, p.N, acc);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T a = warp_sum(acc[k]);
        if (lane == 0) ((T *)p.phi_part)[k * p.N + t] = a;
    }
}

// phi_part[t] = row t of the precomputed operator times the sorted nodal m:
// one warp per row
template <typename T>
__global__ void __launch_bounds__(128) k_near_matrix(DevPlan p) {
    pdl_wait();
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 4 + warp;
    if (t >= p.N) return;
    near_row<T, 1>(p, t, lane);
}

// K states with one pass over the operator: each entry is streamed once and
// applied to the K sorted magnetisations (phi_part[k][t]); the per-state sums
// run in the same order as in k_near_matrix.
template <typename T, int K>
__global__ void __launch_bounds__(128) k_near_matrix_states(DevPlan p) {
    pdl_wait();
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 4 + warp;
    if (t >= p.N) return;
    near_row<T, K>(p, t, lane);
}

template <typename T> static cudaError_t near_states_t(const DevPlan &p, int K, cudaStream_t s) {
    const unsigned nb = (unsigned)((p.N + 3) / 4);
    switch (K) {
        case 1: return launch_k(k_near_matrix_states<T, 1>, nb, 128, 0, s, p);
        case 2: return launch_k(k_near_matrix_states<T, 2>, nb, 128, 0, s, p);
        case 3: return launch_k(k_near_matrix_states<T, 3>, nb, 128, 0, s, p);
        case 4: return launch_k(k_near_matrix_states<T, 4>, nb, 128, 0, s, p);
        case 5: return launch_k(k_near_matrix_states<T, 5>, nb, 128, 0, s, p);
        case 6: return launch_k(k_near_matrix_states<T, 6>, nb, 128, 0, s, p);
        case 7: return launch_k(k_near_matrix_states<T, 7>, nb, 128, 0, s, p);
        case 8: return launch_k(k_near_matrix_states<T, 8>, nb, 128, 0, s, p);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_near_matrix_states(const DevPlan &p, int K, cudaStream_t s) {
    if (p.N == 0 || K <= 0) return cudaSuccess;
    return p.prec == 64 ? near_states_t<double>(p, K, s) : near_states_t<float>(p, K, s);
}

cudaError_t launch_near_matrix(const DevPlan &p, const void *, cudaStream_t s) {
    if (p.N == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((p.N + 3) / 4);
    if (p.prec == 64)
        { const cudaError_t le = launch_k(k_near_matrix<double>, nb, 128, 0, s, p); if (le != cudaSuccess) return le; }
    else
        { const cudaError_t le = launch_k(k_near_matrix<float>, nb, 128, 0, s, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

}  // namespace slp
