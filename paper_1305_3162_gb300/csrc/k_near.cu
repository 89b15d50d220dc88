// Near-field correction (paper Sec. 3.4, Eq. (nfcorr)):
//
//   phi_i += sum_{k : |x_i - y_k| < eps} qk (N - N_s)(x_i - y_k),
//
// where N_s is the smooth kernel the far path actually applies:
//   RADIAL:    (N - N_s)(r) = erfc(r / (s sqrt 2)) / (4 pi r)  (r < eps);
//   SEPARABLE: (N - N_s)(d) = 1/(4 pi |d|) - A prod_q f_q(d_q / L_q), every pair.
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
__global__ void __launch_bounds__(NEAR_WARPS * 32) k_near(DevPlan p, T *__restrict__ phi) {
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
            atomicAdd(phi + p.tgt_perm[it.tbegin + lane], v);
    }
}

// Deterministic mode: items of one target block are consecutive; add their
// partials in item order.  blk_items[b] = first item of block b (CSR).
template <typename T>
__global__ void k_near_reduce(DevPlan p, const int *__restrict__ blk_first, int nblk, T *__restrict__ phi) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int i0 = blk_first[b], i1 = blk_first[b + 1];
    const NearItem it0 = p.near_items[i0];
    if (lane >= it0.tcount) return;
    T s = T(0);
    for (int i = i0; i < i1; ++i) s += ((const T *)p.phi_near)[(int64_t)i * 32 + lane];
    phi[p.tgt_perm[it0.tbegin + lane]] += s;
}

template <typename T> static cudaError_t near_t(const DevPlan &p, void *phi, cudaStream_t s) {
    if (p.n_near == 0) return cudaSuccess;
    const int nb = (p.n_near + NEAR_WARPS - 1) / NEAR_WARPS;
    if (p.kernel_mode == 2)
        k_near<T, 2><<<nb, NEAR_WARPS * 32, 0, s>>>(p, (T *)phi);
    else
        k_near<T, 1><<<nb, NEAR_WARPS * 32, 0, s>>>(p, (T *)phi);
    return cudaGetLastError();
}

cudaError_t launch_near(const DevPlan &p, void *phi, cudaStream_t s) {
    return p.prec == 64 ? near_t<double>(p, phi, s) : near_t<float>(p, phi, s);
}

cudaError_t launch_near_reduce(const DevPlan &p, const int *blk_first, int nblk, void *phi, cudaStream_t s) {
    if (nblk == 0) return cudaSuccess;
    const int nb = (nblk + 7) / 8;
    if (p.prec == 64)
        k_near_reduce<double><<<nb, 256, 0, s>>>(p, blk_first, nblk, (double *)phi);
    else
        k_near_reduce<float><<<nb, 256, 0, s>>>(p, blk_first, nblk, (float *)phi);
    return cudaGetLastError();
}

}  // namespace slp
