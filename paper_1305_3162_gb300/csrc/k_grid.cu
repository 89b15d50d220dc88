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
// Nodal magnetisation in sorted target order, one 4-vector per vertex, so the
// precomputed near-field product reads it coalesced.
template <typename T>
__global__ void __launch_bounds__(256) k_nodal_prep(DevPlan p, const T *__restrict__ in) {
    pdl_wait();
    pdl_trigger();
    typedef typename VecT<T>::T4 T4;
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= p.N) return;
    const int64_t v = p.tgt_perm[u];
    T4 o;
    o.x = in[3 * v];
    o.y = in[3 * v + 1];
    o.z = in[3 * v + 2];
    o.w = T(0);
    check_finite3(p, o.x, o.y, o.z);
    ((T4 *)p.m4)[u] = o;
}

// w_k * sigma_k of sorted source k for the three input kinds (NODAL_MAG
// interpolates the user-order nodal values of the triangle's vertices).
// The plan part of a source's charge (its triangle's vertices and user index,
// and w n), loaded apart from the input so that kernels can fetch it before
// they wait for the previous kernel.
template <typename T> struct ChargeRecipe {
    int4 v;
    typename VecT<T>::T4 wn;
};
template <typename T> __device__ __forceinline__ ChargeRecipe<T> charge_recipe(const DevPlan &p, int64_t k) {
    typedef typename VecT<T>::T4 T4;
    return {p.src_tri[k], ((const T4 *)p.src_wn)[k]};
}
template <typename T>
__device__ __forceinline__ T charge_apply(const DevPlan &p, const ChargeRecipe<T> &r, int kind, const T *__restrict__ in) {
    const int4 v = r.v;
    const auto wn = r.wn;
    const int u = v.w;
    if (kind == 0) return wn.w * in[u];
    T mx, my, mz;
    if (kind == 1) {
        mx = in[3 * (int64_t)u];
        my = in[3 * (int64_t)u + 1];
        mz = in[3 * (int64_t)u + 2];
    } else {
        // rule point of source u = j q + s (q is 1, 3 or 7: divisions by constants)
        const int s = p.q == 7 ? u % 7 : (p.q == 3 ? u % 3 : 0);
        const T *lam = (const T *)p.lam + 3 * s;
        const T l0 = lam[0], l1 = lam[1], l2 = lam[2];
        const T *a = in + 3 * (int64_t)v.x, *b = in + 3 * (int64_t)v.y, *c = in + 3 * (int64_t)v.z;
        mx = l0 * a[0] + l1 * b[0] + l2 * c[0];
        my = l0 * a[1] + l1 * b[1] + l2 * c[1];
        mz = l0 * a[2] + l1 * b[2] + l2 * c[2];
    }
    return mx * wn.x + my * wn.y + mz * wn.z;
}
template <typename T>
__device__ __forceinline__ T source_charge(const DevPlan &p, int64_t k, int kind, const T *__restrict__ in) {
    return charge_apply<T>(p, charge_recipe<T>(p, k), kind, in);
}

// qbuf[k] = w_k * sigma_k in sorted source order.
template <typename T>
__global__ void __launch_bounds__(256) k_charges(DevPlan p, int kind, const T *__restrict__ in) {
    pdl_wait();
    pdl_trigger();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.Q) return;
    const T q = source_charge<T>(p, k, kind, in);
    check_finite3(p, q, q, q);  // a NaN or Inf among the inputs this charge reads
    ((T *)p.qbuf)[k] = q;
}

// ---------------------------------------------------------------- tile geometry
// A tile covers TS^3 cells; with the window's halo it spans TE = TS + 2M - 1
// grid points per axis.  In shared memory a tile is stored with x extent XE
// (TE widened so that the first x point is 16-byte aligned in the global
// grid), row stride RS and plane stride PS chosen so that the 32 lanes of a
// warp, one per (y, z) row of a window box (8 x 4 rows for M = 4), fall on 32
// different banks.
template <int M, int TS> struct TileGeom {
    static constexpr int W = 2 * M;
    static constexpr int TE = TS + W - 1;
    static constexpr int XO = (4 - ((M - 1) % 4)) % 4;  // x offset of the halo start inside the aligned row
    static constexpr int XE = ((XO + TE + 3) / 4) * 4;
    static constexpr int RS = (XE % 8 == 4) ? XE : XE + 4;
    static constexpr int PS = ((TE * RS + 31) / 32) * 32 + 1;
    static constexpr int SIZE = TE * PS;                  // elements of one tile copy
};

// Window values w[axis][i] = psi(f_axis + M - 1 - i) for the 3 x 2M window
// points of a source or target.  FP32: per-interval polynomial in the
// fraction f (coefficients fitted on the host, max error ~1e-10 of psi(0));
// FP64: the closed form (or the plan's FP64 window tables).
constexpr int WDEG = 9;  // degree of the FP32 window polynomials (set by the plan)

// ---------------------------------------------------------------- spread, cell groups
// Variant for 2M <= 10: runs of consecutive sources that share a grid cell
// (the Morton sort makes them contiguous) have the same window box, so a warp
// sums a whole run in registers and updates its private tile once per run.
//   * groups: the plan lists, per item, runs of one cell (at most
//     SPREAD_GMAX sources), dealt largest first to SPREAD_WARPS lists of
//     about equal work, so the warps of a block finish together;
//   * window values: lane (axis, i) evaluates psi(f_axis + M - 1 - i) for
//     every source of the run (FP32: the per-interval polynomial, its
//     coefficients held in registers), the charge folded into the x values;
//     rows of WP (W rounded up to 4) values, so the y row is read as 16-byte
//     vectors;
//   * accumulation: lanes map to (x offset ix, z offset izs); a lane holds
//     the box column (ix, iz = izs + ZL h, all iy) as H x W accumulators.  The
//     plane stride is congruent to W modulo 32, so the 8 x 4 lanes of a row
//     update hit 32 different banks;
//   * the tile: FP32 keeps one tile per block, updated with shared-memory
//     atomic adds (the order of the adds, like that of the global adds below,
//     is not fixed); FP64 keeps one private tile per warp (plain
//     read-modify-writes, warp copies summed in a fixed order).
template <int M, int TS> struct TileGeomG {
    static constexpr int W = 2 * M;
    static constexpr int TE = TS + W - 1;
    static constexpr int XO = (4 - ((M - 1) % 4)) % 4;
    static constexpr int XE = ((XO + TE + 3) / 4) * 4;
    static constexpr int RS = XE;
    static constexpr int PS = ((TE * RS - W + 31) / 32) * 32 + W;  // >= TE RS, == W mod 32
    static constexpr int SIZE = TE * PS;
    static constexpr int ZL = 32 / W;                   // z offsets per lane group
    static constexpr int H = (W + ZL - 1) / ZL;         // z offsets per lane
    static constexpr int WP = (W + 3) & ~3;             // padded row of window values
};

// SPREAD_GMAX (sources per cell group) and SPREAD_WARPS (group lists per
// item) are set with the plan's group lists (slp_internal.h)

// row of WP window values from shared memory, 16 bytes per load
template <int WP> __device__ __forceinline__ void load_row(const float *src, float *dst) {
#pragma unroll
    for (int j = 0; j < WP / 4; ++j) {
        const float4 v = ((const float4 *)src)[j];
        dst[4 * j] = v.x;
        dst[4 * j + 1] = v.y;
        dst[4 * j + 2] = v.z;
        dst[4 * j + 3] = v.w;
    }
}
template <int WP> __device__ __forceinline__ void load_row(const double *src, double *dst) {
#pragma unroll
    for (int j = 0; j < WP / 2; ++j) {
        const double2 v = ((const double2 *)src)[j];
        dst[2 * j] = v.x;
        dst[2 * j + 1] = v.y;
    }
}

template <typename T, int M, int TS> struct SpreadSmem {
    typedef TileGeomG<M, TS> G;
    static constexpr bool SHARED_ATOMIC = sizeof(T) == 4;
    static constexpr int AX = SPREAD_GMAX * G::WP;  // window values of one axis of one warp
    __host__ __device__ static int copies(int nwarps) { return SHARED_ATOMIC ? 1 : nwarps; }
    // offsets in elements of T: tiles, window values (16-byte aligned), sources
    __host__ __device__ static size_t wv(int nwarps) { return ((size_t)copies(nwarps) * G::SIZE + 3) & ~(size_t)3; }
    __host__ __device__ static size_t head(int nwarps) { return (wv(nwarps) + (size_t)nwarps * 3 * AX + 3) & ~(size_t)3; }
    __host__ __device__ static size_t bytes(int nwarps, int chunk) { return head(nwarps) * sizeof(T) + (size_t)chunk * 5 * sizeof(T); }
};

// MINB: blocks per SM the register budget is set for.  Meshes with many
// sources per cell group run best at 4 (64 registers, no spills); sparse
// meshes, where the per-group overheads dominate, at 5 (48 registers).
template <typename T, int M, int TS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_spread_groups(DevPlan p, int fused_kind, const T *__restrict__ in) {
    typedef typename VecT<T>::T4 T4;
    typedef TileGeomG<M, TS> G;
    typedef SpreadSmem<T, M, TS> SM;
    constexpr int W = G::W, TS_ = TS, RS = G::RS, PS = G::PS, XO = G::XO, ZL = G::ZL, H = G::H, WP = G::WP;
    constexpr int AX = SM::AX;
    static_assert(3 * W <= 32, "one lane per window point and axis");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    T *tiles = (T *)smem_raw;
    T *wv = tiles + SM::wv(nwarps) + (size_t)warp * 3 * AX;
    T4 *sg = (T4 *)(tiles + SM::head(nwarps));
    T *sq = (T *)(sg + p.spread_chunk);
    constexpr bool SA = SM::SHARED_ATOMIC;
    const int ncopies = SM::copies(nwarps);
    T *my = tiles + (SA ? 0 : warp * G::SIZE);

    const TileItem it = p.spread_items[blockIdx.x];
    const int nsrc = it.end - it.begin;
    if (p.ks > 1) in = (const T *)p.in_st[blockIdx.y];  // state of a batched launch
    {
        // the tile copies (and the padding up to the window values), 16 bytes per store
        const int n4 = (int)(SM::wv(nwarps) * sizeof(T) / 16);
        for (int i = threadIdx.x; i < n4; i += blockDim.x) ((float4 *)tiles)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    // lane (wax, wi) evaluates window point wi along axis wax
    const int wax = lane / W, wi = lane - wax * W;
    const bool wlane = lane < 3 * W;
    T cf[WDEG + 1];
#pragma unroll
    for (int k = 0; k <= WDEG; ++k) cf[k] = T(0);
    if (sizeof(T) == 4 && wlane) {
#pragma unroll
        for (int k = 0; k <= WDEG; ++k) cf[k] = ((const T *)p.wcoef)[wi * (WDEG + 1) + k];
    }
    const T inv_m = T(1) / T(M);
    const T beta = (T)p.beta, isb = (T)p.inv_sinh_beta;
    // plan data, fetched before the wait: source positions, the charge recipe
    // of the thread's first source, and the first 32 cell groups of the
    // warp's first list (one per lane)
    {
        const T4 *src = (const T4 *)p.src_grid + it.begin;
        for (int i = threadIdx.x; i < nsrc; i += blockDim.x) sg[i] = src[i];
    }
    ChargeRecipe<T> r0;
    if (fused_kind >= 0 && (int)threadIdx.x < nsrc) r0 = charge_recipe<T>(p, it.begin + threadIdx.x);
    // the plan's cell groups of this item, dealt to SPREAD_WARPS lists; a
    // block with fewer warps takes lists w, w + nwarps, ...
    const int *goff = p.sgroup_off + (int64_t)blockIdx.x * (SPREAD_WARPS + 1);
    const int gl0 = goff[warp], gl1 = goff[warp + 1];
    const int gpre = gl0 + lane < gl1 ? p.sgroups[gl0 + lane] : 0;
    // charges and grid A may be the previous kernel's output
    pdl_wait();
    pdl_trigger();
    {
        const T *qb = (const T *)p.qbuf + it.begin;
        for (int i = threadIdx.x; i < nsrc; i += blockDim.x) {
            if (fused_kind >= 0)
                sq[i] = charge_apply<T>(p, i == (int)threadIdx.x ? r0 : charge_recipe<T>(p, it.begin + i), fused_kind, in);
            else
                sq[i] = qb[i];
        }
    }
    __syncthreads();

    const int ix = lane % W, izs = lane / W;
    const bool lane_on = lane < W * ZL;
    for (int wl = warp; wl < SPREAD_WARPS; wl += nwarps)
    for (int gi = goff[wl]; gi < goff[wl + 1]; ++gi) {
        const int gd = (wl == warp && gi - gl0 < 32) ? __shfl_sync(0xffffffffu, gpre, gi - gl0) : p.sgroups[gi];
        const int g0 = gd & 0xffff, ng = gd >> 16;
        if (g0 + ng > nsrc || ng < 1 || ng > SPREAD_GMAX) {
            set_error(p.err, DEV_ERR_BAD_ITEM);
            continue;
        }
        const int cell = packed_cell(sg[g0].w);
        int cx, cy, cz;
        unpack_cell(cell, cx, cy, cz);
        const int lx = cx - it.c0x, ly = cy - it.c0y, lz = cz - it.c0z;
        if ((unsigned)lx >= (unsigned)TS_ || (unsigned)ly >= (unsigned)TS_ || (unsigned)lz >= (unsigned)TS_) {
            set_error(p.err, DEV_ERR_BAD_ITEM);
            continue;
        }
        if (wlane) {
            T *dst = wv + wax * AX + wi;
            if constexpr (sizeof(T) == 4) {
                // two sources per step, paired FP32 multiply-adds
                for (int g = 0; g < ng; g += 2) {
                    const int g1 = g + 1 < ng ? g + 1 : g;
                    const float2 f2 = make_float2(((const float *)(sg + g0 + g))[wax], ((const float *)(sg + g0 + g1))[wax]);
                    float2 v = make_float2(cf[WDEG], cf[WDEG]);
#pragma unroll
                    for (int k = WDEG - 1; k >= 0; --k) v = __ffma2_rn(v, f2, make_float2(cf[k], cf[k]));
                    if (wax == 0) {
                        v.x *= sq[g0 + g];
                        v.y *= sq[g0 + g1];
                    }
                    dst[g * WP] = v.x;
                    if (g + 1 < ng) dst[(g + 1) * WP] = v.y;
                }
            } else {
                const double *tab = p.wtab64_src ? p.wtab64_src + (int64_t)(it.begin + g0) * 3 * W + wax * W + wi : nullptr;
                for (int g = 0; g < ng; ++g) {
                    const T f = ((const T *)(sg + g0 + g))[wax];
                    T v = tab ? (T)tab[g * 3 * W] : kb_window(f + T(M - 1 - wi), inv_m, beta, isb);
                    if (wax == 0) v *= sq[g0 + g];
                    dst[g * WP] = v;
                }
            }
        }
        __syncwarp();
        if (lane_on) {
            // acc[h][iy] of box point (ix, iy, izs + ZL h); FP32 pairs (iy, iy + 1)
            constexpr int W2 = (W + 1) / 2;
            typedef typename VecT<T>::T2 P2;
            P2 acc[H][W2];
#pragma unroll
            for (int h = 0; h < H; ++h)
#pragma unroll
                for (int j = 0; j < W2; ++j) acc[h][j].x = acc[h][j].y = T(0);
            // two sources per iteration where the 64-register budget holds
            // them without spills (the 4-block build)
#pragma unroll(MINB == 4 ? 2 : 1)
            for (int g = 0; g < ng; ++g) {
                const T a = wv[g * WP + ix];
                const T *wz = wv + 2 * AX + g * WP;
                T b[H];
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const int iz = izs + ZL * h;
                    b[h] = iz < W ? a * wz[iz] : T(0);
                }
                T wy[WP];
                load_row<WP>(wv + AX + g * WP, wy);
#pragma unroll
                for (int j = 0; j < W2; ++j)
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        if constexpr (sizeof(T) == 4) {
                            acc[h][j] = __ffma2_rn(make_float2(b[h], b[h]), make_float2(wy[2 * j], wy[2 * j + 1]), acc[h][j]);
                        } else {
                            acc[h][j].x += b[h] * wy[2 * j];
                            acc[h][j].y += b[h] * wy[2 * j + 1];
                        }
                    }
            }
            T *base = my + lz * PS + ly * RS + lx + XO + ix;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int iz = izs + ZL * h;
                if (iz < W) {
#pragma unroll
                    for (int iy = 0; iy < W; ++iy) {
                        T *a = base + iz * PS + iy * RS;
                        const T v = (iy & 1) ? acc[h][iy >> 1].y : acc[h][iy >> 1].x;
                        if constexpr (SA)
                            atomicAdd(a, v);
                        else
                            *a = *a + v;
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();

    constexpr int TE = G::TE, XE = G::XE;
    const int Lx = p.L[0], Ly = p.L[1], Lz = p.L[2];
    const int gxs = it.c0x - M + 1 - XO, gy0 = it.c0y - M + 1, gz0 = it.c0z - M + 1;
    T *grid = (T *)p.gridA + blockIdx.y * p.st_grid;
    const bool xin = gxs >= 0 && gxs + XE <= Lx && (gxs & 3) == 0;
    if (sizeof(T) == 4 && TS % 4 == 0 && xin) {
        constexpr int NV = XE / 4;
        for (int i = threadIdx.x; i < TE * TE * NV; i += blockDim.x) {
            const int v = i % NV, r = i / NV;
            const int iy = r % TE, iz = r / TE;
            float a[4] = {0.f, 0.f, 0.f, 0.f};
            for (int w = 0; w < ncopies; ++w) {
                const float *t = (const float *)tiles + w * G::SIZE + iz * PS + iy * RS + 4 * v;
                if constexpr (PS % 4 == 0 && G::SIZE % 4 == 0) {
                    const float4 f = *(const float4 *)t;
                    a[0] += f.x;
                    a[1] += f.y;
                    a[2] += f.z;
                    a[3] += f.w;
                } else if constexpr (PS % 2 == 0 && G::SIZE % 2 == 0) {
                    const float2 f0 = *(const float2 *)t, f1 = *(const float2 *)(t + 2);
                    a[0] += f0.x;
                    a[1] += f0.y;
                    a[2] += f1.x;
                    a[3] += f1.y;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) a[e] += t[e];
                }
            }
            if (a[0] == 0.f && a[1] == 0.f && a[2] == 0.f && a[3] == 0.f) continue;
            const int gy = (gy0 + iy) & (Ly - 1), gz = (gz0 + iz) & (Lz - 1);
            float4 *dst = (float4 *)((float *)grid + ((int64_t)gz * Ly + gy) * Lx + gxs) + v;
            atomicAdd(dst, make_float4(a[0], a[1], a[2], a[3]));
        }
    } else {
        for (int i = threadIdx.x; i < TE * TE * XE; i += blockDim.x) {
            const int x = i % XE, r = i / XE;
            const int iy = r % TE, iz = r / TE;
            T v = T(0);
            for (int w = 0; w < ncopies; ++w) v += tiles[w * G::SIZE + iz * PS + iy * RS + x];
            if (v == T(0)) continue;
            const int gx = (gxs + x) & (Lx - 1);
            const int gy = (gy0 + iy) & (Ly - 1), gz = (gz0 + iz) & (Lz - 1);
            atomicAdd(grid + ((int64_t)gz * Ly + gy) * Lx + gx, v);
        }
    }
}

// ---------------------------------------------------------------- spread, window tables (FP32)
// Variant for FP32 and 2M <= 8 that reads the window values of every source
// from a plan-time table instead of evaluating the window: per sorted source
// one row of 3 x WP floats (psi along x, y, z at the 2M points of its box,
// each axis padded to WP = 2M rounded up to 4).  A warp walks its list of
// cell groups; each group's table rows (contiguous) are copied into one of
// two per-warp buffers with 16-byte asynchronous copies issued one group
// ahead of use, so no registers are held for them while the current group
// accumulates.  The group's box is accumulated in registers and added to the
// block's shared tile.  Lane (ix, izs) holds the box column (ix, iz = izs +
// ZL h, all iy) as H x W/2 pairs; the group's local cell comes with the group
// list, so the tile address of every update is a per-lane constant plus
// compile-time offsets.
template <int M> struct TabGeom {
    static constexpr int W = 2 * M;
    static constexpr int WP = (W + 3) & ~3;
    static constexpr int ROW = 3 * WP;          // floats per source row
    static constexpr int PARTS = ROW / 4;       // float4 per source row
    static constexpr int GF4 = SPREAD_GMAX * PARTS;  // float4 of one full group
    static constexpr int LD = (GF4 + 31) / 32;  // copies per lane per group
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// shared memory: tile, two table buffers per warp, charges and the item's
// group descriptors and cells (at most one group per source)
template <int M> __host__ __device__ constexpr size_t spread_tab_smem(int nwarps, int chunk, int size) {
    return (((size_t)size + 3) & ~(size_t)3) * 4 + (size_t)nwarps * 2 * SPREAD_GMAX * TabGeom<M>::ROW * 4 +
           (size_t)chunk * 4 * 3 + (SPREAD_WARPS + 1) * 4;
}

template <int M, int TS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_spread_tab(DevPlan p, int fused_kind, const float *__restrict__ in) {
    typedef TileGeomG<M, TS> G;
    typedef TabGeom<M> TG;
    constexpr int W = G::W, RS = G::RS, PS = G::PS, XO = G::XO, ZL = G::ZL, H = G::H;
    constexpr int WP = TG::WP, ROW = TG::ROW, PARTS = TG::PARTS, LD = TG::LD;
    constexpr int BUF = SPREAD_GMAX * ROW;  // floats of one warp buffer
    static_assert(W <= 8, "2M <= 8");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    float *tile = (float *)smem_raw;
    float *wbuf = tile + ((G::SIZE + 3) & ~3) + (size_t)warp * 2 * BUF;
    float *sq = tile + ((G::SIZE + 3) & ~3) + (size_t)nwarps * 2 * BUF;

    const TileItem it = p.spread_items[blockIdx.x];
    const int nsrc = it.end - it.begin;
    // the item's group lists: descriptors and cells staged in shared memory
    int *sgd = (int *)(sq + p.spread_chunk);
    int *sgc = sgd + p.spread_chunk;
    int *soff = sgc + p.spread_chunk;
    if (p.ks > 1) in = (const float *)p.in_st[blockIdx.y];  // state of a batched launch
    {
        const int n4 = ((G::SIZE + 3) & ~3) / 4;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) ((float4 *)tile)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 *wtab = (const float4 *)p.wtab + (int64_t)it.begin * PARTS;
    {
        // group lists of the item (plan data): offsets relative to the item's first group
        const int *goff = p.sgroup_off + (int64_t)blockIdx.x * (SPREAD_WARPS + 1);
        const int gfirst = goff[0], ng_item = min(goff[SPREAD_WARPS] - gfirst, p.spread_chunk);
        if (threadIdx.x <= SPREAD_WARPS) soff[threadIdx.x] = min(max(goff[threadIdx.x] - gfirst, 0), ng_item);
        for (int i = threadIdx.x; i < ng_item; i += blockDim.x) {
            sgd[i] = p.sgroups[gfirst + i];
            sgc[i] = p.sgroup_cell[gfirst + i];
        }
    }
    __syncthreads();
    // the warp's group lists (a block with fewer warps takes lists w, w + nwarps, ...)
    const int *goff = soff;
    int wl = warp, gi = goff[warp], gend = goff[warp + 1];
    // advance (wl, gi) to the warp's next group, if any
    auto next = [&]() -> bool {
        while (gi >= gend) {
            wl += nwarps;
            if (wl >= SPREAD_WARPS) return false;
            gi = goff[wl];
            gend = goff[wl + 1];
        }
        return true;
    };
    // group gi's descriptor, and its table rows copied into buffer b
    auto fetch = [&](int b, int &g0, int &ng, int &cell) {
        const int gd = sgd[gi];
        g0 = gd & 0xffff;
        ng = gd >> 16;
        cell = sgc[gi];
        const int nf = (ng >= 1 && ng <= SPREAD_GMAX && g0 + ng <= nsrc) ? ng * PARTS : 0;
        const float4 *src = wtab + (int64_t)g0 * PARTS;
        float4 *dst = (float4 *)(wbuf + b * BUF);
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int f = lane + 32 * u;
            if (f < nf) cp_async16(dst + f, src + f);
        }
        cp_async_commit();
    };
    // plan data before the wait: the charge recipe of the thread's first
    // source and the table rows of the warp's first group
    ChargeRecipe<float> r0;
    if (fused_kind >= 0 && (int)threadIdx.x < nsrc) r0 = charge_recipe<float>(p, it.begin + threadIdx.x);
    bool have = next();
    int g0 = 0, ng = 0, cell = 0, cur = 0;
    if (have) fetch(0, g0, ng, cell);
    // charges may be the previous kernel's output (or computed here from the input)
    pdl_wait();
    pdl_trigger();
    for (int i = threadIdx.x; i < nsrc; i += blockDim.x) {
        if (fused_kind >= 0)
            sq[i] = charge_apply<float>(p, i == (int)threadIdx.x ? r0 : charge_recipe<float>(p, it.begin + i),
                                        fused_kind, in);
        else
            sq[i] = ((const float *)p.qbuf)[it.begin + i];
    }
    __syncthreads();

    const int ix = lane % W, izs = lane / W;
    const bool lane_on = lane < W * ZL;
    // lane's fixed part of every tile update: column ix, first z offset izs
    float *const lane_tile = tile + XO + ix + izs * PS;
    while (have) {
        const int c_g0 = g0, c_ng = ng, c_cell = cell;
        ++gi;
        have = next();
        if (have) {
            fetch(cur ^ 1, g0, ng, cell);  // the next group's rows copy while this one accumulates
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        if (c_g0 + c_ng > nsrc || c_ng < 1 || c_ng > SPREAD_GMAX) {
            set_error(p.err, DEV_ERR_BAD_ITEM);
        } else if (lane_on) {
            constexpr int W2 = (W + 1) / 2;
            float2 acc[H][W2];
#pragma unroll
            for (int h = 0; h < H; ++h)
#pragma unroll
                for (int j = 0; j < W2; ++j) acc[h][j] = make_float2(0.f, 0.f);
            const float *r = wbuf + cur * BUF;
            const float *qg = sq + c_g0;
#pragma unroll 2
            for (int g = 0; g < c_ng; ++g, r += ROW) {
                const float a = r[ix] * qg[g];
                float b[H];
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const int iz = izs + ZL * h;
                    b[h] = (ZL * H == W || iz < W) ? a * r[2 * WP + iz] : 0.f;
                }
                float wy[WP];
                load_row<WP>(r + WP, wy);
#pragma unroll
                for (int j = 0; j < W2; ++j)
#pragma unroll
                    for (int h = 0; h < H; ++h)
                        acc[h][j] = __ffma2_rn(make_float2(b[h], b[h]), make_float2(wy[2 * j], wy[2 * j + 1]), acc[h][j]);
            }
            float *base = lane_tile + (c_cell >> 16) * PS + ((c_cell >> 8) & 0xff) * RS + (c_cell & 0xff);
#pragma unroll
            for (int h = 0; h < H; ++h) {
                if (ZL * H == W || izs + ZL * h < W) {
#pragma unroll
                    for (int iy = 0; iy < W; ++iy)
                        atomicAdd(base + ZL * h * PS + iy * RS, (iy & 1) ? acc[h][iy >> 1].y : acc[h][iy >> 1].x);
                }
            }
        }
        // every lane is done with buffer `cur` before the next copy into it
        __syncwarp();
        cur ^= 1;
    }
    __syncthreads();

    constexpr int TE = G::TE, XE = G::XE;
    const int Lx = p.L[0], Ly = p.L[1], Lz = p.L[2];
    const int gxs = it.c0x - M + 1 - XO, gy0 = it.c0y - M + 1, gz0 = it.c0z - M + 1;
    float *grid = (float *)p.gridA + blockIdx.y * p.st_grid;
    const bool xin = gxs >= 0 && gxs + XE <= Lx && (gxs & 3) == 0;
    if (TS % 4 == 0 && xin && (256 % (XE / 4)) == 0 && blockDim.x == 256) {
        // thread t adds vector v = t % NV of rows r = t / NV + (256 / NV) j
        constexpr int NV = XE / 4, RSTEP = 256 / NV, NROW = TE * TE;
        const int v = threadIdx.x % NV;
        int r = threadIdx.x / NV;
        int iy = r % TE, iz = r / TE;
        for (; r < NROW; r += RSTEP) {
            const float *t = tile + iz * PS + iy * RS + 4 * v;
            float a[4];
            if constexpr (PS % 4 == 0) {
                const float4 f = *(const float4 *)t;
                a[0] = f.x; a[1] = f.y; a[2] = f.z; a[3] = f.w;
            } else if constexpr (PS % 2 == 0) {
                const float2 f0 = *(const float2 *)t, f1 = *(const float2 *)(t + 2);
                a[0] = f0.x; a[1] = f0.y; a[2] = f1.x; a[3] = f1.y;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) a[e] = t[e];
            }
            if (a[0] != 0.f || a[1] != 0.f || a[2] != 0.f || a[3] != 0.f) {
                const int gy = (gy0 + iy) & (Ly - 1), gz = (gz0 + iz) & (Lz - 1);
                float4 *dst = (float4 *)(grid + ((int64_t)gz * Ly + gy) * Lx + gxs) + v;
                atomicAdd(dst, make_float4(a[0], a[1], a[2], a[3]));
            }
            // advance (iy, iz) by RSTEP rows
            iy += RSTEP % TE;
            iz += RSTEP / TE;
            if (iy >= TE) {
                iy -= TE;
                ++iz;
            }
        }
    } else {
        for (int i = threadIdx.x; i < TE * TE * XE; i += blockDim.x) {
            const int x = i % XE, rr = i / XE;
            const int iy = rr % TE, iz = rr / TE;
            const float v = tile[iz * PS + iy * RS + x];
            if (v == 0.f) continue;
            const int gx = (gxs + x) & (Lx - 1);
            const int gy = (gy0 + iy) & (Ly - 1), gz = (gz0 + iz) & (Lz - 1);
            atomicAdd(grid + ((int64_t)gz * Ly + gy) * Lx + gx, v);
        }
    }
}

// Plan-time window table of the FP32 table spread: row k (sorted source k)
// holds psi(f_q + M - 1 - i) for axis q and point i < 2M, evaluated in FP64
// from the source's fractional grid coordinate, each axis padded with zeros
// to WP values.
template <int M>
__global__ void k_wtab_build(const float4 *__restrict__ src_grid, int64_t Q, double beta, double isb,
                             float *__restrict__ out) {
    typedef TabGeom<M> TG;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Q) return;
    const float4 g = src_grid[k];
    const double f[3] = {(double)g.x, (double)g.y, (double)g.z};
    float *row = out + k * TG::ROW;
    for (int ax = 0; ax < 3; ++ax)
        for (int i = 0; i < TG::WP; ++i)
            row[ax * TG::WP + i] =
                i < TG::W ? (float)kb_window(f[ax] + double(M - 1 - i), 1.0 / M, beta, isb) : 0.f;
}

// ---------------------------------------------------------------- gather
// One block per work item (a tile and up to GATHER_CHUNK of its targets): the
// tile plus halo of grid B is staged in shared memory (same padded layout as
// the spread), together with the item's target coordinates, permutation,
// near-field parts and window values; then one warp per target sums its
// (2M)^3 window box, lanes over the (y, z) rows of the box.

template <typename T, int M, int TS>
__global__ void __launch_bounds__(256) k_gather(DevPlan p, T *__restrict__ phi) {
    typedef typename VecT<T>::T4 T4;
    typedef TileGeom<M, TS> G;
    constexpr int W = G::W, TE = G::TE, RS = G::RS, PS = G::PS, XO = G::XO;
    constexpr int GW = 3 * W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int GC = p.gather_chunk;
    T *tile = (T *)smem_raw;
    T *wv = tile + ((G::SIZE + 3) & ~3);  // [GC][3W]
    T *sf = wv + GC * GW;               // [3][GC] fractions
    T *sphi = sf + 3 * GC;              // [GC] near-field parts
    int *sidx = (int *)(sphi + GC);     // [2][GC] packed cell, output index

    const TileItem it = p.gather_items[blockIdx.x];
    const int nt = it.end - it.begin;
    if (nt > GC || GC > GATHER_CHUNK) {
        if (threadIdx.x == 0) set_error(p.err, DEV_ERR_BAD_ITEM);
        return;
    }
    const int Lx = p.L[0], Ly = p.L[1], Lz = p.L[2];
    const int gx0 = it.c0x - M + 1, gy0 = it.c0y - M + 1, gz0 = it.c0z - M + 1;
    const T *grid = (const T *)p.gridB + blockIdx.y * p.st_grid;
    if (p.ks > 1) phi = (T *)p.out_st[blockIdx.y];  // state of a batched launch
    // plan data first (target positions, permutation, window values): none of
    // it depends on the previous kernel, so it overlaps that kernel's tail
    if (threadIdx.x < nt) {
        const int t = it.begin + threadIdx.x;
        const T4 g = ((const T4 *)p.tgt_grid)[t];
        sf[threadIdx.x] = g.x;
        sf[GC + threadIdx.x] = g.y;
        sf[2 * GC + threadIdx.x] = g.z;
        sidx[threadIdx.x] = packed_cell(g.w);
        sidx[GC + threadIdx.x] = p.tgt_perm[t];
    }
    __syncthreads();

    // window values of the warp's targets, wv[t * 3W + axis * W + i]: lane
    // j = (wax, wi) evaluates point wi along axis wax (FP32: the interval
    // polynomial, coefficients in registers), and point j + 32 where 3W > 32
    {
        const T inv_m = T(1) / T(M);
        const T beta = (T)p.beta, isb = (T)p.inv_sinh_beta;
#pragma unroll
        for (int j0 = 0; j0 < GW; j0 += 32) {
            const int j = j0 + lane;
            if (j < GW) {
                const int wax = j / W, wi = j - wax * W;
                T cf[WDEG + 1];
                if (sizeof(T) == 4) {
#pragma unroll
                    for (int k = 0; k <= WDEG; ++k) cf[k] = ((const T *)p.wcoef)[wi * (WDEG + 1) + k];
                }
                for (int t = warp; t < nt; t += nwarps) {
                    const T f = sf[wax * GC + t];
                    T v;
                    if (sizeof(T) == 4) {
                        v = cf[WDEG];
#pragma unroll
                        for (int k = WDEG - 1; k >= 0; --k) v = v * f + cf[k];
                    } else if (p.wtab64_tgt) {
                        v = (T)p.wtab64_tgt[(int64_t)(it.begin + t) * GW + j];
                    } else {
                        v = kb_window(f + T(M - 1 - wi), inv_m, beta, isb);
                    }
                    wv[t * GW + j] = v;
                }
            }
        }
    }

    // grid B and the near-field parts are the previous kernels' output
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x < nt) sphi[threadIdx.x] = ((const T *)p.phi_part)[blockIdx.y * p.N + it.begin + threadIdx.x];
    constexpr int XE = G::XE;
    const int gxs = gx0 - XO;  // a multiple of 4 when TS is
    if (sizeof(T) == 4 && TS % 4 == 0 && gxs >= 0 && gxs + XE <= Lx) {
        // rows of XE/4 aligned 16-byte vectors (the tile's x extent widened to XE)
        constexpr int NV = XE / 4;
        pipelined_copy<float4>(
            TE * TE * NV,
            [&](int i) {
                const int v = i % NV, r = i / NV;
                const int gy = (gy0 + r % TE) & (Ly - 1);
                const int gz = (gz0 + r / TE) & (Lz - 1);
                return ((const float4 *)((const float *)grid + ((int64_t)gz * Ly + gy) * Lx + gxs))[v];
            },
            [&](int i, float4 v) {
                const int vv = i % NV, r = i / NV;
                float *d = (float *)tile + (r / TE) * PS + (r % TE) * RS + 4 * vv;
                d[0] = v.x;
                d[1] = v.y;
                d[2] = v.z;
                d[3] = v.w;
            });
    } else {
        pipelined_copy<T>(
            TE * TE * TE,
            [&](int i) {
                const int x = i % TE, r = i / TE;
                const int gx = (gx0 + x) & (Lx - 1);
                const int gy = (gy0 + r % TE) & (Ly - 1);
                const int gz = (gz0 + r / TE) & (Lz - 1);
                return grid[((int64_t)gz * Ly + gy) * Lx + gx];
            },
            [&](int i, T v) {
                const int x = i % TE, r = i / TE;
                tile[(r / TE) * PS + (r % TE) * RS + x + XO] = v;
            });
    }
    __syncthreads();

    for (int t = warp; t < nt; t += nwarps) {
        int cx, cy, cz;
        unpack_cell(sidx[t], cx, cy, cz);
        const int lx = cx - it.c0x, ly = cy - it.c0y, lz = cz - it.c0z;
        if ((unsigned)lx >= (unsigned)TS || (unsigned)ly >= (unsigned)TS || (unsigned)lz >= (unsigned)TS) {
            set_error(p.err, DEV_ERR_BAD_ITEM);
            continue;
        }
        const T *w = wv + t * GW;
        const T *base = tile + lz * PS + ly * RS + lx + XO;
        T acc = T(0);
#pragma unroll
        for (int rep = 0; rep < (W * W + 31) / 32; ++rep) {
            const int pi = lane + 32 * rep;
            if (pi < W * W) {
                const int iy = pi % W, iz = pi / W;
                const T *row = base + iz * PS + iy * RS;
                T s = T(0);
#pragma unroll
                for (int ix = 0; ix < W; ++ix) s += row[ix] * w[ix];
                acc += s * w[2 * W + iz] * w[W + iy];
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const T v = acc + sphi[t];
            check_finite3(p, v, v, v);
            phi[sidx[GC + t]] = v;
        }
    }
}

// ---------------------------------------------------------------- zero
__global__ void k_zero4(float4 *p, int64_t n4) {
    pdl_wait();
    pdl_trigger();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- launchers
// Spread of wide windows (2m > 10): one tile per block, no per-warp copies.
// The block stages the window values of SB sources at a time in shared
// memory (from the FP64 window table or evaluated), the x values times the
// charge; then warp w adds, source after source, the box points of the
// tile's z planes z = w, w + nwarps, ... (lanes over the (x, y) points of a
// plane), so every tile element is updated by one warp in source order: no
// atomics, and one tile holds many sources, so the flush of the halo tile
// into the grid (global atomics) is shared by all of them.
template <typename T, int M, int TS> struct PlaneSmem {
    typedef TileGeom<M, TS> G;
    static constexpr int SB = 32;  // sources per staged batch
    __host__ __device__ static size_t coef_off() { return ((size_t)G::SIZE + 3) & ~(size_t)3; }
    __host__ __device__ static size_t wv_off(int wdeg) {
        return coef_off() + (((size_t)2 * M * (wdeg + 1) + 3) & ~(size_t)3);
    }
    __host__ __device__ static size_t bytes(int wdeg) {
        return (wv_off(wdeg) + (size_t)SB * 3 * 2 * M) * sizeof(T) + (size_t)SB * sizeof(int);
    }
};

template <typename T, int M, int TS>
__global__ void __launch_bounds__(256) k_spread_planes(DevPlan p, int fused_kind, const T *__restrict__ in) {
    pdl_wait();
    pdl_trigger();
    typedef typename VecT<T>::T4 T4;
    typedef TileGeom<M, TS> G;
    typedef PlaneSmem<T, M, TS> SM;
    constexpr int W = G::W, TE = G::TE, RS = G::RS, PS = G::PS, XO = G::XO, XE = G::XE, SB = SM::SB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    T *tile = (T *)smem_raw;
    T *coef = tile + SM::coef_off();
    T *wv = tile + SM::wv_off(p.wdeg);  // [SB][3W]
    int *cell = (int *)(wv + SB * 3 * W);
    const int ncoef = W * (p.wdeg + 1);

    const TileItem it = p.spread_items[blockIdx.x];
    const int nsrc = it.end - it.begin;
    if (p.ks > 1) in = (const T *)p.in_st[blockIdx.y];  // state of a batched launch
    for (int i = threadIdx.x; i < G::SIZE; i += blockDim.x) tile[i] = T(0);
    if (sizeof(T) == 4)
        for (int i = threadIdx.x; i < ncoef; i += blockDim.x) coef[i] = ((const T *)p.wcoef)[i];
    const T inv_m = T(1) / T(M);
    const T beta = (T)p.beta, isb = (T)p.inv_sinh_beta;
    const T4 *src = (const T4 *)p.src_grid;
    for (int b0 = 0; b0 < nsrc; b0 += SB) {
        const int nb = min(SB, nsrc - b0);
        __syncthreads();  // the previous batch's values are no longer read; the tile and coef are set
        for (int idx = threadIdx.x; idx < nb * 3 * W; idx += blockDim.x) {
            const int sidx = idx / (3 * W), j = idx - sidx * 3 * W, ax = j / W, i = j - ax * W;
            const int k = it.begin + b0 + sidx;
            T v;
            if (sizeof(T) == 8 && p.wtab64_src) {
                v = (T)p.wtab64_src[(int64_t)k * 3 * W + j];
            } else {
                const T4 g = src[k];
                const T f = ax == 0 ? g.x : (ax == 1 ? g.y : g.z);
                if (sizeof(T) == 4) {
                    const T *c = coef + i * (WDEG + 1);
                    v = c[WDEG];
#pragma unroll
                    for (int e = WDEG - 1; e >= 0; --e) v = v * f + c[e];
                } else {
                    v = kb_window(f + T(M - 1 - i), inv_m, beta, isb);
                }
            }
            if (ax == 0)
                v *= fused_kind >= 0 ? source_charge<T>(p, k, fused_kind, in) : ((const T *)p.qbuf)[k];
            wv[sidx * 3 * W + j] = v;
        }
        for (int sidx = threadIdx.x; sidx < nb; sidx += blockDim.x) {
            int cx, cy, cz;
            unpack_cell(packed_cell(src[it.begin + b0 + sidx].w), cx, cy, cz);
            const int lx = cx - it.c0x, ly = cy - it.c0y, lz = cz - it.c0z;
            if ((unsigned)lx >= (unsigned)TS || (unsigned)ly >= (unsigned)TS || (unsigned)lz >= (unsigned)TS) {
                set_error(p.err, DEV_ERR_BAD_ITEM);
                cell[sidx] = -1;
            } else {
                cell[sidx] = lx | (ly << 8) | (lz << 16);
            }
        }
        __syncthreads();
        for (int sidx = 0; sidx < nb; ++sidx) {
            const int c = cell[sidx];
            if (c < 0) continue;
            const int lx = c & 255, ly = (c >> 8) & 255, lz = c >> 16;
            const T *w = wv + sidx * 3 * W;
            // the first of the warp's planes at or after lz
            int iz = ((warp - lz) % nwarps + nwarps) % nwarps;
            for (; iz < W; iz += nwarps) {
                const T wz = w[2 * W + iz];
                T *plane = tile + (lz + iz) * PS + ly * RS + lx + XO;
                for (int pi = lane; pi < W * W; pi += 32) {
                    const int iy = pi / W, ix = pi - iy * W;
                    plane[iy * RS + ix] += w[ix] * (w[W + iy] * wz);
                }
            }
        }
    }
    __syncthreads();

    const int Lx = p.L[0], Ly = p.L[1], Lz = p.L[2];
    const int gxs = it.c0x - M + 1 - XO, gy0 = it.c0y - M + 1, gz0 = it.c0z - M + 1;
    T *grid = (T *)p.gridA + blockIdx.y * p.st_grid;
    for (int i = threadIdx.x; i < TE * TE * XE; i += blockDim.x) {
        const int x = i % XE, r = i / XE;
        const int iy = r % TE, iz = r / TE;
        const T v = tile[iz * PS + iy * RS + x];
        if (v == T(0)) continue;
        const int gx = (gxs + x) & (Lx - 1);
        const int gy = (gy0 + iy) & (Ly - 1), gz = (gz0 + iz) & (Lz - 1);
        atomicAdd(grid + ((int64_t)gz * Ly + gy) * Lx + gx, v);
    }
}

template <typename T, int M, int TS>
static cudaError_t spread_mt(const DevPlan &p, int fused_kind, const void *in, cudaStream_t s) {
    if constexpr (M <= 5) {
        int nw = 8;
        while (nw > 1 && SpreadSmem<T, M, TS>::bytes(nw, p.spread_chunk) > 100 * 1024) nw >>= 1;
        const size_t sm = SpreadSmem<T, M, TS>::bytes(nw, p.spread_chunk);
        auto go = [&](auto kern) -> cudaError_t {
            if (sm > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e != cudaSuccess) return e;
            }
            if (p.n_spread > 0) {
                const cudaError_t le = launch_k(kern, dim3(p.n_spread, p.ks), 32 * nw, sm, s, p, fused_kind, (const T *)in);
                if (le != cudaSuccess) return le;
            }
            return cudaGetLastError();
        };
        if constexpr (sizeof(T) == 4 && M <= 4) {
            if (p.wtab) {
                typedef TileGeomG<M, TS> G;
                const size_t smt = spread_tab_smem<M>(nw, p.spread_chunk, G::SIZE);
                auto go_t = [&](auto kern) -> cudaError_t {
                    if (smt > 48 * 1024) {
                        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
                        if (e != cudaSuccess) return e;
                    }
                    if (p.n_spread > 0) {
                        const cudaError_t le = launch_k(kern, dim3(p.n_spread, p.ks), 32 * nw, smt, s, p, fused_kind,
                                                        (const float *)in);
                        if (le != cudaSuccess) return le;
                    }
                    return cudaGetLastError();
                };
                if (p.spread_dense) return go_t(k_spread_tab<M, TS, 4>);
                return go_t(k_spread_tab<M, TS, 5>);
            }
        }
        if constexpr (sizeof(T) == 4 && M <= 4) {
            if (p.spread_dense) return go(k_spread_groups<T, M, TS, 4>);
            return go(k_spread_groups<T, M, TS, 5>);
        } else {
            return go(k_spread_groups<T, M, TS, 1>);
        }
    }
    const size_t sm = PlaneSmem<T, M, TS>::bytes(p.wdeg);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_spread_planes<T, M, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (p.n_spread > 0) {
        const cudaError_t le = launch_k(k_spread_planes<T, M, TS>, dim3(p.n_spread, p.ks), 256, sm, s, p, fused_kind,
                                        (const T *)in);
        if (le != cudaSuccess) return le;
    }
    return cudaGetLastError();
}

template <typename T, int M, int TS> static cudaError_t gather_mt(const DevPlan &p, void *phi, cudaStream_t s) {
    typedef TileGeom<M, TS> G;
    const size_t GC = (size_t)p.gather_chunk;
    const size_t sm = ((size_t)((G::SIZE + 3) & ~3) + GC * (3 * 2 * M + 4)) * sizeof(T) + 2 * GC * sizeof(int);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gather<T, M, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (p.n_gather > 0) { const cudaError_t le = launch_k(k_gather<T, M, TS>, dim3(p.n_gather, p.ks), 256, sm, s, p, (T *)phi); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

template <typename T, int M>
static cudaError_t spread_t(const DevPlan &p, int fused_kind, const void *in, cudaStream_t s) {
    switch (p.TS) {
        case 2: return spread_mt<T, M, 2>(p, fused_kind, in, s);
        case 4: return spread_mt<T, M, 4>(p, fused_kind, in, s);
        case 8: return spread_mt<T, M, 8>(p, fused_kind, in, s);
    }
    return cudaErrorInvalidValue;
}
template <typename T, int M> static cudaError_t gather_t(const DevPlan &p, void *phi, cudaStream_t s) {
    switch (p.TSg) {
        case 2: return gather_mt<T, M, 2>(p, phi, s);
        case 4: return gather_mt<T, M, 4>(p, phi, s);
        case 8: return gather_mt<T, M, 8>(p, phi, s);
    }
    return cudaErrorInvalidValue;
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

cudaError_t launch_spread(const DevPlan &p, int fused_kind, const void *in, cudaStream_t s) {
    if (p.prec == 64) { SLP_DISPATCH_M(spread_t, double, p, fused_kind, in, s) }
    SLP_DISPATCH_M(spread_t, float, p, fused_kind, in, s)
}

template <int M> static cudaError_t wtab_m(const DevPlan &p, float *out, cudaStream_t s) {
    if (p.Q == 0) return cudaSuccess;
    k_wtab_build<M><<<(unsigned)((p.Q + 255) / 256), 256, 0, s>>>((const float4 *)p.src_grid, p.Q, p.beta,
                                                                  p.inv_sinh_beta, out);
    return cudaGetLastError();
}

int spread_table_row(int m) { return 3 * ((2 * m + 3) & ~3); }

// FP64 window values, one thread per (point, axis, window point): the same
// expression the spread and gather kernels evaluate (inv_m = 1/M), so a
// table entry is bitwise the value the kernel would compute.
template <int M>
__global__ void __launch_bounds__(256) k_wtab64_build(const double4 *__restrict__ pts, int64_t n, double beta,
                                                      double isb, double *__restrict__ out) {
    constexpr int W = 2 * M;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * 3 * W) return;
    const int64_t pt = idx / (3 * W);
    const int j = (int)(idx - pt * 3 * W), ax = j / W, i = j - ax * W;
    const double4 g = pts[pt];
    const double f = ax == 0 ? g.x : (ax == 1 ? g.y : g.z);
    const double inv_m = 1.0 / double(M);
    out[idx] = kb_window(f + double(M - 1 - i), inv_m, beta, isb);
}

template <int M> static cudaError_t wtab64_m(const void *pts, int64_t n, double beta, double isb, double *out,
                                             cudaStream_t s) {
    const int64_t total = n * 3 * 2 * M;
    if (total == 0) return cudaSuccess;
    k_wtab64_build<M><<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const double4 *)pts, n, beta, isb, out);
    return cudaGetLastError();
}

cudaError_t launch_wtab64_build(const DevPlan &p, const void *pts, int64_t n, double *out, cudaStream_t s) {
    switch (p.m) {
        case 2: return wtab64_m<2>(pts, n, p.beta, p.inv_sinh_beta, out, s);
        case 3: return wtab64_m<3>(pts, n, p.beta, p.inv_sinh_beta, out, s);
        case 4: return wtab64_m<4>(pts, n, p.beta, p.inv_sinh_beta, out, s);
        case 5: return wtab64_m<5>(pts, n, p.beta, p.inv_sinh_beta, out, s);
        case 6: return wtab64_m<6>(pts, n, p.beta, p.inv_sinh_beta, out, s);
        case 7: return wtab64_m<7>(pts, n, p.beta, p.inv_sinh_beta, out, s);
        case 8: return wtab64_m<8>(pts, n, p.beta, p.inv_sinh_beta, out, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_wtab_build(const DevPlan &p, float *out, cudaStream_t s) {
    switch (p.m) {
        case 2: return wtab_m<2>(p, out, s);
        case 3: return wtab_m<3>(p, out, s);
        case 4: return wtab_m<4>(p, out, s);
        case 5: return wtab_m<5>(p, out, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_gather(const DevPlan &p, void *phi, cudaStream_t s) {
    if (p.prec == 64) { SLP_DISPATCH_M(gather_t, double, p, phi, s) }
    SLP_DISPATCH_M(gather_t, float, p, phi, s)
}

cudaError_t launch_nodal_prep(const DevPlan &p, const void *d_in, cudaStream_t s) {
    if (p.N == 0) return cudaSuccess;
    const int nb = (int)((p.N + 255) / 256);
    if (p.prec == 64)
        { const cudaError_t le = launch_k(k_nodal_prep<double>, nb, 256, 0, s, p, (const double *)d_in); if (le != cudaSuccess) return le; }
    else
        { const cudaError_t le = launch_k(k_nodal_prep<float>, nb, 256, 0, s, p, (const float *)d_in); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

// K states: block row y = state
template <typename T>
__global__ void __launch_bounds__(256) k_nodal_prep_states(DevPlan p, StatePtrs sp) {
    typedef typename VecT<T>::T4 T4;
    pdl_wait();
    pdl_trigger();
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= p.N) return;
    const T *in = (const T *)sp.in[blockIdx.y];
    const int64_t v = p.tgt_perm[u];
    T4 o;
    o.x = in[3 * v];
    o.y = in[3 * v + 1];
    o.z = in[3 * v + 2];
    o.w = T(0);
    check_finite3(p, o.x, o.y, o.z);
    ((T4 *)p.m4)[(int64_t)blockIdx.y * p.N + u] = o;
}

cudaError_t launch_nodal_prep_states(const DevPlan &p, const StatePtrs &in, int K, cudaStream_t s) {
    if (p.N == 0 || K <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((p.N + 255) / 256), (unsigned)K);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (p.prec == 64) return cudaLaunchKernelEx(&cfg, k_nodal_prep_states<double>, p, in);
    return cudaLaunchKernelEx(&cfg, k_nodal_prep_states<float>, p, in);
}

cudaError_t launch_charges(const DevPlan &p, int kind, const void *d_in, cudaStream_t s) {
    if (p.Q == 0) return cudaSuccess;
    const int nb = (int)((p.Q + 255) / 256);
    if (p.prec == 64)
        { const cudaError_t le = launch_k(k_charges<double>, nb, 256, 0, s, p, kind, (const double *)d_in); if (le != cudaSuccess) return le; }
    else
        { const cudaError_t le = launch_k(k_charges<float>, nb, 256, 0, s, p, kind, (const float *)d_in); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

cudaError_t launch_zero(void *ptr, size_t bytes, cudaStream_t s) {
    // plan buffers are 256-byte aligned and sized in multiples of 16 bytes
    const int64_t n4 = (int64_t)(bytes / 16);
    if (n4 == 0) return cudaSuccess;
    int nb = (int)((n4 + 255) / 256);
    if (nb > 152 * 16) nb = 152 * 16;
    { const cudaError_t le = launch_k(k_zero4, nb, 256, 0, s, (float4 *)ptr, n4); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

}  // namespace slp
