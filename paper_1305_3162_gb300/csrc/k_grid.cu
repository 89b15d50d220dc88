// Charge assembly, spreading (type-1 gridding) and interpolation (type-2
// gather) kernels.
//
// Spread: the gridding tensor of Sec. 3 in the quadrature form of Eq.
// (naive_gridding), a_r = sum_k qk prod_q psi(u_{k,q} - r_q), over the 2m
// grid points per axis around each source (u in grid units).  Sources are
// sorted by tile; one CTA accumulates one tile (plus its halo of m cells)
// in shared memory, one warp per source with the lanes spread over the
// (y, z) rows of the window box, then adds the tile to the global grid.
//
// Gather: the window interpolation of the forward NFFT (Sec. 2.2, Eq.
// (smooth_phi) evaluated by NFFT): phi_i = sum_r g_r prod_q psi(u_{i,q} - r_q).
// One CTA loads a tile plus halo of the grid into shared memory; one warp
// per target.
#include "dev_common.cuh"

namespace slp {

// ---------------------------------------------------------------- charges
// qbuf[k] = w_k * sigma_k in sorted source order, for the three input kinds.
template <typename T>
__global__ void __launch_bounds__(256) k_charges(DevPlan p, int kind, const T *__restrict__ in) {
    typedef typename VecT<T>::T4 T4;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.Q) return;
    const int u = p.src_perm[k];
    const T w = ((const T *)p.src_w)[k];
    T sigma;
    if (kind == 0) {
        sigma = in[u];
    } else {
        const int j = u / p.q;
        const int s = u - j * p.q;
        const T4 nrm = ((const T4 *)p.tri_nrm)[j];
        T mx, my, mz;
        if (kind == 1) {
            mx = in[3 * (int64_t)u];
            my = in[3 * (int64_t)u + 1];
            mz = in[3 * (int64_t)u + 2];
        } else {
            const int4 v = p.tri_vtx[j];
            const T *lam = (const T *)p.lam + 3 * s;
            const T l0 = lam[0], l1 = lam[1], l2 = lam[2];
            const int64_t a = 3 * (int64_t)v.x, b = 3 * (int64_t)v.y, c = 3 * (int64_t)v.z;
            mx = l0 * in[a] + l1 * in[b] + l2 * in[c];
            my = l0 * in[a + 1] + l1 * in[b + 1] + l2 * in[c + 1];
            mz = l0 * in[a + 2] + l1 * in[b + 2] + l2 * in[c + 2];
        }
        sigma = mx * nrm.x + my * nrm.y + mz * nrm.z;
    }
    ((T *)p.qbuf)[k] = w * sigma;
}

// ---------------------------------------------------------------- spread
// Each warp accumulates into its own copy of the halo tile, so the updates
// are plain read-modify-writes: within one warp instruction every lane owns a
// different (y, z) row of the source's window box, and consecutive sources of
// a warp are ordered by __syncwarp.  The warp copies are summed in a fixed
// order before the tile is added to the global grid.
template <typename T, int M>
__global__ void __launch_bounds__(256) k_spread(DevPlan p) {
    typedef typename VecT<T>::T4 T4;
    constexpr int W = 2 * M;  // window points per axis
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TE = p.TE;
    const int TE2 = TE * TE;
    const int TE3 = TE2 * TE;
    const int TEP = (TE3 + 31) & ~31;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    T *tiles = (T *)smem_raw;
    T *wv = tiles + (size_t)nwarps * TEP + warp * (3 * W);
    T *my = tiles + (size_t)warp * TEP;

    const TileItem it = p.spread_items[blockIdx.x];
    for (int i = threadIdx.x; i < nwarps * TEP; i += blockDim.x) tiles[i] = T(0);
    __syncthreads();

    const T4 *src = (const T4 *)p.src_grid;
    const T *qb = (const T *)p.qbuf;
    const T inv_m = T(1) / T(M);
    const T beta = (T)p.beta, isb = (T)p.inv_sinh_beta;
    for (int k = it.begin + warp; k < it.end; k += nwarps) {
        const T4 g = src[k];
        const T qk = qb[k];
        int cx, cy, cz;
        unpack_cell(packed_cell(g.w), cx, cy, cz);
        const int lx = cx - it.c0x, ly = cy - it.c0y, lz = cz - it.c0z;
        if ((unsigned)lx >= (unsigned)p.TS || (unsigned)ly >= (unsigned)p.TS || (unsigned)lz >= (unsigned)p.TS) {
            set_error(p.err, DEV_ERR_BAD_ITEM);
            continue;
        }
        // window values: wv[axis * W + i] = psi(f + M - 1 - i)
        for (int j = lane; j < 3 * W; j += 32) {
            const int ax = j / W, i = j - ax * W;
            const T f = ax == 0 ? g.x : (ax == 1 ? g.y : g.z);
            wv[j] = kb_window(f + T(M - 1 - i), inv_m, beta, isb);
        }
        __syncwarp();
        T wx[W];
#pragma unroll
        for (int ix = 0; ix < W; ++ix) wx[ix] = wv[ix];
        for (int pi = lane; pi < W * W; pi += 32) {
            const int iy = pi % W, iz = pi / W;
            const T wyz = qk * wv[2 * W + iz] * wv[W + iy];
            T *row = my + (lz + iz) * TE2 + (ly + iy) * TE + lx;
            T r[W];
#pragma unroll
            for (int ix = 0; ix < W; ++ix) r[ix] = row[ix];
#pragma unroll
            for (int ix = 0; ix < W; ++ix) row[ix] = r[ix] + wyz * wx[ix];
        }
        __syncwarp();
    }
    __syncthreads();

    // sum the warp copies in order, then add the tile (with the periodic
    // wrap-around) to the global grid
    const int Lx = p.L[0], Ly = p.L[1], Lz = p.L[2];
    const int gx0 = it.c0x - M + 1, gy0 = it.c0y - M + 1, gz0 = it.c0z - M + 1;
    T *grid = (T *)p.gridA;
    for (int i = threadIdx.x; i < TE3; i += blockDim.x) {
        T v = T(0);
        for (int w = 0; w < nwarps; ++w) v += tiles[(size_t)w * TEP + i];
        if (v == T(0)) continue;
        const int iz = i / TE2;
        const int r = i - iz * TE2;
        const int iy = r / TE;
        const int ix = r - iy * TE;
        const int gx = (gx0 + ix) & (Lx - 1);
        const int gy = (gy0 + iy) & (Ly - 1);
        const int gz = (gz0 + iz) & (Lz - 1);
        atomicAdd(grid + ((int64_t)gz * Ly + gy) * Lx + gx, v);
    }
}

// ---------------------------------------------------------------- gather
template <typename T, int M>
__global__ void __launch_bounds__(256) k_gather(DevPlan p, T *__restrict__ phi) {
    typedef typename VecT<T>::T4 T4;
    constexpr int W = 2 * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TE = p.TE;
    const int TE2 = TE * TE;
    const int TE3 = TE2 * TE;
    T *tile = (T *)smem_raw;
    T *wall = tile + ((TE3 + 3) & ~3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    T *wv = wall + warp * (3 * W);

    const TileItem it = p.gather_items[blockIdx.x];
    const int Lx = p.L[0], Ly = p.L[1], Lz = p.L[2];
    const int gx0 = it.c0x - M + 1, gy0 = it.c0y - M + 1, gz0 = it.c0z - M + 1;
    const T *grid = (const T *)p.gridB;
    for (int i = threadIdx.x; i < TE3; i += blockDim.x) {
        const int iz = i / TE2;
        const int r = i - iz * TE2;
        const int iy = r / TE;
        const int ix = r - iy * TE;
        const int gx = (gx0 + ix) & (Lx - 1);
        const int gy = (gy0 + iy) & (Ly - 1);
        const int gz = (gz0 + iz) & (Lz - 1);
        tile[i] = grid[((int64_t)gz * Ly + gy) * Lx + gx];
    }
    __syncthreads();

    const T4 *tg = (const T4 *)p.tgt_grid;
    const T inv_m = T(1) / T(M);
    const T beta = (T)p.beta, isb = (T)p.inv_sinh_beta;
    for (int t = it.begin + warp; t < it.end; t += nwarps) {
        const T4 g = tg[t];
        int cx, cy, cz;
        unpack_cell(packed_cell(g.w), cx, cy, cz);
        const int lx = cx - it.c0x, ly = cy - it.c0y, lz = cz - it.c0z;
        if ((unsigned)lx >= (unsigned)p.TS || (unsigned)ly >= (unsigned)p.TS || (unsigned)lz >= (unsigned)p.TS) {
            set_error(p.err, DEV_ERR_BAD_ITEM);
            continue;
        }
        for (int j = lane; j < 3 * W; j += 32) {
            const int ax = j / W, i = j - ax * W;
            const T f = ax == 0 ? g.x : (ax == 1 ? g.y : g.z);
            wv[j] = kb_window(f + T(M - 1 - i), inv_m, beta, isb);
        }
        __syncwarp();
        T acc = T(0);
        for (int pi = lane; pi < W * W; pi += 32) {
            const int iy = pi % W, iz = pi / W;
            const T *row = tile + (lz + iz) * TE2 + (ly + iy) * TE + lx;
            T s = T(0);
#pragma unroll
            for (int ix = 0; ix < W; ++ix) s += row[ix] * wv[ix];
            acc += s * wv[2 * W + iz] * wv[W + iy];
        }
        acc = warp_sum(acc);
        if (lane == 0) phi[p.tgt_perm[t]] = acc;
        __syncwarp();
    }
}

// ---------------------------------------------------------------- zero
__global__ void k_zero4(float4 *p, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- launchers
static size_t tile_smem_bytes(const DevPlan &p, size_t elem) {
    const size_t TE3 = (size_t)p.TE * p.TE * p.TE;
    return (((TE3 + 3) & ~(size_t)3) + 8 * 3 * 2 * (size_t)p.m) * elem;
}

// warps per spread block: as many private tiles as fit in ~110 KB (two blocks per SM)
static int spread_warps(const DevPlan &p, size_t elem) {
    const size_t TE3 = (size_t)p.TE * p.TE * p.TE;
    const size_t TEP = (TE3 + 31) & ~(size_t)31;
    int nw = 8;
    while (nw > 1 && nw * (TEP + 3 * 2 * (size_t)p.m) * elem > 110 * 1024) nw >>= 1;
    return nw;
}

template <typename T, int M> static cudaError_t spread_t(const DevPlan &p, cudaStream_t s) {
    const int nw = spread_warps(p, sizeof(T));
    const size_t TE3 = (size_t)p.TE * p.TE * p.TE;
    const size_t sm = (nw * ((TE3 + 31) & ~(size_t)31) + nw * 3 * 2 * (size_t)M) * sizeof(T);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_spread<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (p.n_spread > 0) k_spread<T, M><<<p.n_spread, 32 * nw, sm, s>>>(p);
    return cudaGetLastError();
}

template <typename T, int M> static cudaError_t gather_t(const DevPlan &p, void *phi, cudaStream_t s) {
    const size_t sm = tile_smem_bytes(p, sizeof(T));
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gather<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (p.n_gather > 0) k_gather<T, M><<<p.n_gather, 256, sm, s>>>(p, (T *)phi);
    return cudaGetLastError();
}

#define SLP_DISPATCH_M(FN, T, ...)                                  \
    switch (p.m) {                                                  \
        case 2: return FN<T, 2>(__VA_ARGS__);                       \
        case 3: return FN<T, 3>(__VA_ARGS__);                       \
        case 4: return FN<T, 4>(__VA_ARGS__);                       \
        case 5: return FN<T, 5>(__VA_ARGS__);                       \
        case 6: return FN<T, 6>(__VA_ARGS__);                       \
        case 7: return FN<T, 7>(__VA_ARGS__);                       \
        case 8: return FN<T, 8>(__VA_ARGS__);                       \
        default: return cudaErrorInvalidValue;                      \
    }

cudaError_t launch_spread(const DevPlan &p, cudaStream_t s) {
    if (p.prec == 64) { SLP_DISPATCH_M(spread_t, double, p, s) }
    SLP_DISPATCH_M(spread_t, float, p, s)
}

cudaError_t launch_gather(const DevPlan &p, void *phi, cudaStream_t s) {
    if (p.prec == 64) { SLP_DISPATCH_M(gather_t, double, p, phi, s) }
    SLP_DISPATCH_M(gather_t, float, p, phi, s)
}

cudaError_t launch_charges(const DevPlan &p, int kind, const void *d_in, cudaStream_t s) {
    if (p.Q == 0) return cudaSuccess;
    const int nb = (int)((p.Q + 255) / 256);
    if (p.prec == 64)
        k_charges<double><<<nb, 256, 0, s>>>(p, kind, (const double *)d_in);
    else
        k_charges<float><<<nb, 256, 0, s>>>(p, kind, (const float *)d_in);
    return cudaGetLastError();
}

cudaError_t launch_zero(void *ptr, size_t bytes, cudaStream_t s) {
    // plan buffers are 256-byte aligned and sized in multiples of 16 bytes
    const int64_t n4 = (int64_t)(bytes / 16);
    if (n4 == 0) return cudaSuccess;
    int nb = (int)((n4 + 255) / 256);
    if (nb > 152 * 16) nb = 152 * 16;
    k_zero4<<<nb, 256, 0, s>>>((float4 *)ptr, n4);
    return cudaGetLastError();
}

}  // namespace slp
