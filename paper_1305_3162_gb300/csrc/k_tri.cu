// Triangle-integrated discretisation (opts.integration = 1): element-wise
// constant charges g_j and exact integrals over the flat triangles, the
// discretised single layer potential of Sec. 2.2, Eq. (slayer3), without a
// point quadrature.
//
//   * gridding tensor (Sec. 3.1, Eq. (gridding2)):
//       a_r = sum_j g_j A_rj,  A_rj = int_{S_j} Psi(r - u(y)) dA(y),
//     the window Psi in grid units and u(y) the grid coordinate of y.  A is a
//     geometry-only matrix, assembled once per plan (the paper's set-up phase)
//     with an 8 x 8 Duffy-Gauss rule per triangle and stored by grid point
//     (CSR over the grid points the triangles' boxes reach), so one
//     evaluation is a sparse product that writes each grid point once;
//   * near field (Sec. 3.4, Eq. (nfcorr)), for every target x_i and triangle
//     S_j within eps (point-triangle distance, the index sets of Eq.
//     (nf_index)):
//       W_ij = int_{S_j} (N - N_s)(x_i - y) dA(y)
//            = I_j(x_i) / (4 pi) - int_{S_j} N_s(x_i - y) dA(y),
//     I_j the integral of 1/|x - y| over S_j in closed form (Wilton et al.
//     1984; Graglia 1993; this handles the weakly singular x_i in S_j
//     exactly, the case the paper treats by the Duffy substitution), and the
//     smooth N_s part by the same Duffy-Gauss rule; stored as CSR over the
//     sorted targets and applied as a second sparse product.
//
// Input NODAL_MAG is projected to element charges first (the integral mean
// of m . n over each triangle, Sec. 2.2), ELEMENT input gives g directly.
#include "dev_common.cuh"

namespace slp {

// ---------------------------------------------------------------- closed form
// int_{S} 1/|x - y| dA(y) for the flat triangle (v0, v1, v2): with n the unit
// normal of the winding, h the signed height of x and rho its projection on
// the plane, and per edge (p-, p+): l the unit direction, u = l x n, l-/l+ =
// (p-/+ - rho) . l, P0 = (p- - rho) . u, R-/R+ = |x - p-/+|, R0^2 = P0^2 + h^2:
//   I = sum P0 ln((R+ + l+) / (R- + l-)) - |h| sum [atan(P0 l+ / (R0^2 + |h| R+)) - atan(P0 l- / (R0^2 + |h| R-))];
// an edge with P0 = 0 contributes nothing.
__device__ double tri_inv_r_integral(const double3 v0, const double3 v1, const double3 v2, const double3 x) {
    const double3 v[3] = {v0, v1, v2};
    const double e1x = v1.x - v0.x, e1y = v1.y - v0.y, e1z = v1.z - v0.z;
    const double e2x = v2.x - v0.x, e2y = v2.y - v0.y, e2z = v2.z - v0.z;
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const double nn = sqrt(nx * nx + ny * ny + nz * nz);
    if (!(nn > 0.0)) return 0.0;
    nx /= nn;
    ny /= nn;
    nz /= nn;
    const double h = (x.x - v0.x) * nx + (x.y - v0.y) * ny + (x.z - v0.z) * nz, ah = fabs(h);
    const double rx = x.x - h * nx, ry = x.y - h * ny, rz = x.z - h * nz;
    double total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double3 pm = v[e], pp = v[(e + 1) % 3];
        const double Lx = pp.x - pm.x, Ly = pp.y - pm.y, Lz = pp.z - pm.z;
        const double len = sqrt(Lx * Lx + Ly * Ly + Lz * Lz);
        const double lx = Lx / len, ly = Ly / len, lz = Lz / len;
        const double ux = ly * nz - lz * ny, uy = lz * nx - lx * nz, uz = lx * ny - ly * nx;
        const double amx = pm.x - rx, amy = pm.y - ry, amz = pm.z - rz;
        const double apx = pp.x - rx, apy = pp.y - ry, apz = pp.z - rz;
        const double lm = amx * lx + amy * ly + amz * lz, lp = apx * lx + apy * ly + apz * lz;
        const double P0 = amx * ux + amy * uy + amz * uz;
        const double Rm = sqrt((x.x - pm.x) * (x.x - pm.x) + (x.y - pm.y) * (x.y - pm.y) + (x.z - pm.z) * (x.z - pm.z));
        const double Rp = sqrt((x.x - pp.x) * (x.x - pp.x) + (x.y - pp.y) * (x.y - pp.y) + (x.z - pp.z) * (x.z - pp.z));
        const double R02 = P0 * P0 + h * h;
        if (fabs(P0) > 1e-14 * len) total += P0 * log((Rp + lp) / (Rm + lm));
        if (ah > 0.0) total -= ah * (atan(P0 * lp / (R02 + ah * Rp)) - atan(P0 * lm / (R02 + ah * Rm)));
    }
    return total;
}

// distance from x to the flat triangle (v0, v1, v2)
__device__ double point_triangle_distance(const double3 a, const double3 b, const double3 c, const double3 x) {
    // closest point by the region tests of the barycentric parametrisation
    const double abx = b.x - a.x, aby = b.y - a.y, abz = b.z - a.z;
    const double acx = c.x - a.x, acy = c.y - a.y, acz = c.z - a.z;
    const double apx = x.x - a.x, apy = x.y - a.y, apz = x.z - a.z;
    const double d1 = abx * apx + aby * apy + abz * apz, d2 = acx * apx + acy * apy + acz * apz;
    double qx, qy, qz;
    auto at = [&](double s, double t) {
        qx = a.x + s * abx + t * acx;
        qy = a.y + s * aby + t * acy;
        qz = a.z + s * abz + t * acz;
    };
    const double bpx = x.x - b.x, bpy = x.y - b.y, bpz = x.z - b.z;
    const double d3 = abx * bpx + aby * bpy + abz * bpz, d4 = acx * bpx + acy * bpy + acz * bpz;
    const double cpx = x.x - c.x, cpy = x.y - c.y, cpz = x.z - c.z;
    const double d5 = abx * cpx + aby * cpy + abz * cpz, d6 = acx * cpx + acy * cpy + acz * cpz;
    const double vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
    if (d1 <= 0 && d2 <= 0) at(0, 0);
    else if (d3 >= 0 && d4 <= d3) at(1, 0);
    else if (d6 >= 0 && d5 <= d6) at(0, 1);
    else if (vc <= 0 && d1 >= 0 && d3 <= 0) at(d1 / (d1 - d3), 0);
    else if (vb <= 0 && d2 >= 0 && d6 <= 0) at(0, d2 / (d2 - d6));
    else if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
        const double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        at(1 - w, w);
    } else {
        const double den = 1.0 / (va + vb + vc);
        at(vb * den, vc * den);
    }
    return sqrt((x.x - qx) * (x.x - qx) + (x.y - qy) * (x.y - qy) + (x.z - qz) * (x.z - qz));
}

// ---------------------------------------------------------------- gridding matrix (plan time, FP64)
// Box of grid points reached by triangle j: per axis from floor(min u) - m + 1
// to floor(max u) + m (the window's 2m points around every point of the
// triangle), at most TRI_BOX points per axis.
struct TriBox {
    int lo[3], n[3];
};
__device__ __forceinline__ bool tri_box(const TriBuildA &b, int64_t j, double3 &u0, double3 &u1, double3 &u2,
                                        TriBox &bx) {
    const int4 t = b.tri[j];
    if (t.x < 0 || t.y < 0 || t.z < 0 || t.x >= b.NV || t.y >= b.NV || t.z >= b.NV) return false;
    u0 = b.ugrid[t.x];
    u1 = b.ugrid[t.y];
    u2 = b.ugrid[t.z];
    const double lo[3] = {fmin(u0.x, fmin(u1.x, u2.x)), fmin(u0.y, fmin(u1.y, u2.y)), fmin(u0.z, fmin(u1.z, u2.z))};
    const double hi[3] = {fmax(u0.x, fmax(u1.x, u2.x)), fmax(u0.y, fmax(u1.y, u2.y)), fmax(u0.z, fmax(u1.z, u2.z))};
    for (int q = 0; q < 3; ++q) {
        bx.lo[q] = (int)floor(lo[q]) - b.m + 1;
        bx.n[q] = (int)floor(hi[q]) + b.m - bx.lo[q] + 1;
        if (bx.n[q] < 1 || bx.n[q] > TRI_BOX) return false;
    }
    return true;
}

__device__ __forceinline__ int64_t grid_lin(const TriBuildA &b, int x, int y, int z) {
    x = ((x % b.L[0]) + b.L[0]) % b.L[0];
    y = ((y % b.L[1]) + b.L[1]) % b.L[1];
    z = ((z % b.L[2]) + b.L[2]) % b.L[2];
    return ((int64_t)z * b.L[1] + y) * b.L[0] + x;
}

// pass 0: entries per grid point (one per triangle whose box reaches it)
__global__ void k_amat_count(TriBuildA b, int *__restrict__ cnt) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b.M) return;
    double3 u0, u1, u2;
    TriBox bx;
    if (!tri_box(b, j, u0, u1, u2, bx)) {
        set_error(b.err, DEV_ERR_BAD_ITEM);
        return;
    }
    for (int iz = 0; iz < bx.n[2]; ++iz)
        for (int iy = 0; iy < bx.n[1]; ++iy)
            for (int ix = 0; ix < bx.n[0]; ++ix)
                atomicAdd(cnt + grid_lin(b, bx.lo[0] + ix, bx.lo[1] + iy, bx.lo[2] + iz), 1);
}

// pass 1: one warp per triangle.  The 1-D window values of the rule's points
// go to shared memory ([point][axis][TRI_BOX]); the lanes then take the box
// points, sum w_p psi_x psi_y psi_z over the points in FP64 and place
// (j, A_rj) in the row of grid point r (slot order fixed afterwards by
// k_amat_sort).
template <typename T>
__global__ void __launch_bounds__(32) k_amat_fill(TriBuildA b, const int *__restrict__ slot_of,
                                                  const int64_t *__restrict__ rowptr, int *__restrict__ cursor,
                                                  int *__restrict__ col, T *__restrict__ val) {
    __shared__ double sw[TRI_RULE * 3 * TRI_BOX];
    __shared__ double swt[TRI_RULE];
    const int64_t j = blockIdx.x;
    const int lane = threadIdx.x;
    if (j >= b.M) return;
    double3 u0, u1, u2;
    TriBox bx;
    if (!tri_box(b, j, u0, u1, u2, bx)) return;  // counted as an error in pass 0
    const int4 t = b.tri[j];
    const double3 x0 = b.xphys[t.x], x1 = b.xphys[t.y], x2 = b.xphys[t.z];
    const double cx = (x1.y - x0.y) * (x2.z - x0.z) - (x1.z - x0.z) * (x2.y - x0.y);
    const double cy = (x1.z - x0.z) * (x2.x - x0.x) - (x1.x - x0.x) * (x2.z - x0.z);
    const double cz = (x1.x - x0.x) * (x2.y - x0.y) - (x1.y - x0.y) * (x2.x - x0.x);
    const double area2 = sqrt(cx * cx + cy * cy + cz * cz);  // 2 |S_j|, physical
    for (int pt = lane; pt < b.np; pt += 32) {
        const double a = b.ra[pt], c = b.rb[pt];
        const double uy[3] = {u0.x + a * (u1.x - u0.x) + c * (u2.x - u1.x), u0.y + a * (u1.y - u0.y) + c * (u2.y - u1.y),
                              u0.z + a * (u1.z - u0.z) + c * (u2.z - u1.z)};
        swt[pt] = b.rw[pt] * area2;
        for (int q = 0; q < 3; ++q)
            for (int i = 0; i < TRI_BOX; ++i)
                sw[(pt * 3 + q) * TRI_BOX + i] =
                    i < bx.n[q] ? kb_window((double)(bx.lo[q] + i) - uy[q], 1.0 / b.m, b.beta, b.isb) : 0.0;
    }
    __syncwarp();
    const int nbox = bx.n[0] * bx.n[1] * bx.n[2];
    for (int k = lane; k < nbox; k += 32) {
        const int ix = k % bx.n[0], iy = (k / bx.n[0]) % bx.n[1], iz = k / (bx.n[0] * bx.n[1]);
        double s = 0.0;
        for (int pt = 0; pt < b.np; ++pt)
            s += swt[pt] * sw[(pt * 3 + 0) * TRI_BOX + ix] * sw[(pt * 3 + 1) * TRI_BOX + iy] *
                 sw[(pt * 3 + 2) * TRI_BOX + iz];
        const int64_t g = grid_lin(b, bx.lo[0] + ix, bx.lo[1] + iy, bx.lo[2] + iz);
        const int slot = slot_of[g];
        if (slot < 0) {
            set_error(b.err, DEV_ERR_BAD_INDEX);
            continue;
        }
        const int64_t pos = rowptr[slot] + atomicAdd(cursor + slot, 1);
        if (pos >= rowptr[slot + 1]) {
            set_error(b.err, DEV_ERR_BAD_INDEX);
            continue;
        }
        col[pos] = (int)j;
        val[pos] = (T)s;
    }
}

// entries of each row in ascending triangle order (a fixed summation order
// whatever order the fill placed them in): insertion sort per row
template <typename T>
__global__ void k_csr_sort(int64_t nrows, const int64_t *__restrict__ rowptr, int *__restrict__ col,
                           T *__restrict__ val) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int64_t a = rowptr[r], e = rowptr[r + 1];
    for (int64_t i = a + 1; i < e; ++i) {
        const int c = col[i];
        const T v = val[i];
        int64_t k = i - 1;
        while (k >= a && col[k] > c) {
            col[k + 1] = col[k];
            val[k + 1] = val[k];
            --k;
        }
        col[k + 1] = c;
        val[k + 1] = v;
    }
}

// ---------------------------------------------------------------- near-field matrix (plan time, FP64)
// N_s(r) of the plan's kernel, without the 1/(4 pi) (as in the near kernels)
__device__ __forceinline__ double tri_smooth_kernel(const TriBuildN &b, double dx, double dy, double dz) {
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (b.kernel_mode == 1) {
        if (r2 == 0.0) return 2.0 * b.inv_s_sqrt2 / 1.7724538509055160273;  // lim erf(a r) / r = 2a / sqrt(pi)
        const double r = sqrt(r2);
        return erf(r * b.inv_s_sqrt2) / r;
    }
    if (b.kernel_mode == 3) {
        double s = 0.0;
        for (int k = 0; k < b.es_n; ++k) s += b.es_w[k] * exp(-b.es_g[k] * r2);
        return s;
    }
    // separable band-limited kernel: 4 pi A prod_q f_q(d_q / P_q)
    double kn = b.sep_A4pi;
    const double d[3] = {dx, dy, dz};
    for (int q = 0; q < 3; ++q) {
        const double xq = cospi(2.0 * d[q] / b.P[q]);
        double b1 = 0.0, b2 = 0.0;
        for (int l = b.sep_nh[q] - 1; l >= 1; --l) {
            const double b0 = 2.0 * b.sep_h[q][l] + 2.0 * xq * b1 - b2;
            b2 = b1;
            b1 = b0;
        }
        kn *= b.sep_h[q][0] + xq * b1 - b2;
    }
    return kn;
}

// W_ij of target x (physical, relative to the torus centre) and triangle j
__device__ double tri_near_entry(const TriBuildN &b, const double3 x, int64_t j, bool &near) {
    const int4 t = b.tri[j];
    const double3 v0 = b.xphys[t.x], v1 = b.xphys[t.y], v2 = b.xphys[t.z];
    near = point_triangle_distance(v0, v1, v2, x) <= b.eps;
    if (!near) return 0.0;
    const double cx = (v1.y - v0.y) * (v2.z - v0.z) - (v1.z - v0.z) * (v2.y - v0.y);
    const double cy = (v1.z - v0.z) * (v2.x - v0.x) - (v1.x - v0.x) * (v2.z - v0.z);
    const double cz = (v1.x - v0.x) * (v2.y - v0.y) - (v1.y - v0.y) * (v2.x - v0.x);
    const double area2 = sqrt(cx * cx + cy * cy + cz * cz);
    double smooth = 0.0;
    for (int pt = 0; pt < b.np; ++pt) {
        const double a = b.ra[pt], c = b.rb[pt];
        const double yx = v0.x + a * (v1.x - v0.x) + c * (v2.x - v1.x);
        const double yy = v0.y + a * (v1.y - v0.y) + c * (v2.y - v1.y);
        const double yz = v0.z + a * (v1.z - v0.z) + c * (v2.z - v1.z);
        smooth += b.rw[pt] * tri_smooth_kernel(b, x.x - yx, x.y - yy, x.z - yz);
    }
    return (tri_inv_r_integral(v0, v1, v2, x) - area2 * smooth) * 0.079577471545947667884;
}

// pass 0 counts, pass 1 fills, one warp per sorted target: the candidate
// vertex ranges of its target block, each vertex's adjacent triangles, each
// triangle taken from its first vertex (in sorted order) that the ranges
// list, so once; lanes over 32 vertices, triangles emitted in (vertex,
// adjacency) order by ballots, which the two passes share.
template <typename T>
__global__ void __launch_bounds__(256) k_nmt_build(TriBuildN b, int pass, int64_t *__restrict__ counts,
                                                   const int64_t *__restrict__ rowptr, int *__restrict__ col,
                                                   T *__restrict__ val) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 8 + warp;
    if (t >= b.N) return;
    const double3 x = b.tgt[t];
    const int blk = b.tgt_block[t];
    int64_t out = pass == 1 ? rowptr[t] : 0;
    int64_t cnt = 0;
    for (int r = b.blk_r0[blk]; r < b.blk_r0[blk + 1]; ++r) {
        const int2 rg = b.ranges[r];
        for (int u0 = rg.x; u0 < rg.y; u0 += 32) {
            const int u = u0 + lane;
            int e0 = 0, e1 = 0;
            if (u < rg.y) {
                const int v = b.tgt_perm[u];
                e0 = b.vt_ptr[v];
                e1 = b.vt_ptr[v + 1];
            }
            int deg = e1 - e0;
            int maxdeg = deg;
            for (int o = 16; o > 0; o >>= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xffffffffu, maxdeg, o));
            for (int k = 0; k < maxdeg; ++k) {
                bool nz = false;
                double w = 0.0;
                int jj = -1;
                if (k < deg) {
                    const int ent = b.vt_ent[e0 + k];
                    jj = ent >> 2;
                    // the triangle's first listed vertex: its smallest sorted index
                    if (b.tri_min_sorted[jj] == u) {
                        bool near;
                        w = tri_near_entry(b, x, jj, near);
                        nz = near;
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, nz);
                if (pass == 1 && nz) {
                    const int64_t pos = out + cnt + __popc(bal & ((1u << lane) - 1u));
                    if (pos < rowptr[t + 1]) {
                        col[pos] = jj;
                        val[pos] = (T)w;
                    } else {
                        set_error(b.err, DEV_ERR_BAD_INDEX);
                    }
                }
                cnt += __popc(bal);
            }
        }
    }
    if (pass == 0 && lane == 0) counts[t] = cnt;
}

// ---------------------------------------------------------------- point gridding matrix (deterministic mode)
// For plans with opts.deterministic the spread of the point sources is also a
// precomputed sparse product: entry (r, k) = prod_q psi(r_q - u_{k,q}) over
// the 2m^3 box of sorted source k, stored by grid point with the sources of a
// row in ascending order, applied to the charges w_k sigma_k.  Every grid
// point is then written once with a sum in a fixed order, where the tiled
// spread adds tiles with atomics in whatever order the blocks finish.
__device__ __forceinline__ void point_box(const PointBuild &b, int64_t k, int &cx, int &cy, int &cz, double3 &f) {
    const double4 g = b.src[k];
    const int c = (int)g.w;
    cx = c & 1023;
    cy = (c >> 10) & 1023;
    cz = (c >> 20) & 1023;
    f = make_double3(g.x, g.y, g.z);
}

__global__ void k_pmat_count(PointBuild b, int *__restrict__ cnt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= b.Q) return;
    int cx, cy, cz;
    double3 f;
    point_box(b, k, cx, cy, cz, f);
    const int W = 2 * b.m;
    for (int iz = 0; iz < W; ++iz)
        for (int iy = 0; iy < W; ++iy)
            for (int ix = 0; ix < W; ++ix) {
                const int x = (((cx - b.m + 1 + ix) % b.L[0]) + b.L[0]) % b.L[0];
                const int y = (((cy - b.m + 1 + iy) % b.L[1]) + b.L[1]) % b.L[1];
                const int z = (((cz - b.m + 1 + iz) % b.L[2]) + b.L[2]) % b.L[2];
                atomicAdd(cnt + ((int64_t)z * b.L[1] + y) * b.L[0] + x, 1);
            }
}

template <typename T>
__global__ void k_pmat_fill(PointBuild b, const int *__restrict__ slot_of, const int64_t *__restrict__ rowptr,
                            int *__restrict__ cursor, int *__restrict__ col, T *__restrict__ val) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= b.Q) return;
    int cx, cy, cz;
    double3 f;
    point_box(b, k, cx, cy, cz, f);
    const int W = 2 * b.m;
    double w[3][16];
    const double fr[3] = {f.x, f.y, f.z};
    for (int q = 0; q < 3; ++q)
        for (int i = 0; i < W; ++i) w[q][i] = kb_window(fr[q] + double(b.m - 1 - i), 1.0 / b.m, b.beta, b.isb);
    for (int iz = 0; iz < W; ++iz)
        for (int iy = 0; iy < W; ++iy)
            for (int ix = 0; ix < W; ++ix) {
                const int x = (((cx - b.m + 1 + ix) % b.L[0]) + b.L[0]) % b.L[0];
                const int y = (((cy - b.m + 1 + iy) % b.L[1]) + b.L[1]) % b.L[1];
                const int z = (((cz - b.m + 1 + iz) % b.L[2]) + b.L[2]) % b.L[2];
                const int slot = slot_of[((int64_t)z * b.L[1] + y) * b.L[0] + x];
                if (slot < 0) {
                    set_error(b.err, DEV_ERR_BAD_INDEX);
                    continue;
                }
                const int64_t pos = rowptr[slot] + atomicAdd(cursor + slot, 1);
                if (pos >= rowptr[slot + 1]) {
                    set_error(b.err, DEV_ERR_BAD_INDEX);
                    continue;
                }
                col[pos] = (int)k;
                val[pos] = (T)(w[0][ix] * w[1][iy] * w[2][iz]);
            }
}

cudaError_t launch_pmat_count(const PointBuild &b, int *cnt, cudaStream_t s) {
    if (b.Q == 0) return cudaSuccess;
    k_pmat_count<<<(unsigned)((b.Q + 255) / 256), 256, 0, s>>>(b, cnt);
    return cudaGetLastError();
}

cudaError_t launch_pmat_fill(const PointBuild &b, int prec, const int *slot_of, const int64_t *rowptr, int *cursor,
                             int *col, void *val, cudaStream_t s) {
    if (b.Q == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((b.Q + 127) / 128);
    if (prec == 64)
        k_pmat_fill<double><<<nb, 128, 0, s>>>(b, slot_of, rowptr, cursor, col, (double *)val);
    else
        k_pmat_fill<float><<<nb, 128, 0, s>>>(b, slot_of, rowptr, cursor, col, (float *)val);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- evaluation
// g_j = (n_j / 3) . (m_a + m_b + m_c): the integral mean of m . n_j for P1 m
template <typename T>
__global__ void __launch_bounds__(256) k_p0_charges(DevPlan p, const T *__restrict__ in) {
    typedef typename VecT<T>::T4 T4;
    const int4 *tv = p.tri_v;
    const T4 *n3 = (const T4 *)p.tri_n3;
    pdl_wait();
    pdl_trigger();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.M) return;
    const int4 v = tv[j];
    const T4 n = n3[j];
    const T *a = in + 3 * (int64_t)v.x, *b = in + 3 * (int64_t)v.y, *c = in + 3 * (int64_t)v.z;
    const T g = n.x * (a[0] + b[0] + c[0]) + n.y * (a[1] + b[1] + c[1]) + n.z * (a[2] + b[2] + c[2]);
    check_finite3(p, g, g, g);
    ((T *)p.gbuf)[j] = g;
}

// y[out(i)] = sum_e val[e] x[col[e]] over CSR row i: LPR lanes per row (their
// partial sums combined in a fixed order), rows in order; out(i) = row_idx[i]
// when row_idx is given (grid points), else i.
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_csr_apply(int64_t nrows, const int64_t *__restrict__ rowptr,
                                                   const int64_t *__restrict__ row_idx, const int *__restrict__ col,
                                                   const T *__restrict__ val, const T *__restrict__ x,
                                                   T *__restrict__ y) {
    pdl_wait();
    pdl_trigger();
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = gt / LPR;
    const int sub = (int)(gt % LPR);
    const bool live = r < nrows;
    T acc = T(0);
    if (live) {
        const int64_t a = rowptr[r], e = rowptr[r + 1];
        for (int64_t k = a + sub; k < e; k += LPR) acc += __ldcs(val + k) * x[__ldcs(col + k)];
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, LPR);
    if (live && sub == 0) y[row_idx ? row_idx[r] : r] = acc;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_amat_count(const TriBuildA &b, int *cnt, cudaStream_t s) {
    if (b.M == 0) return cudaSuccess;
    k_amat_count<<<(unsigned)((b.M + 255) / 256), 256, 0, s>>>(b, cnt);
    return cudaGetLastError();
}

cudaError_t launch_amat_fill(const TriBuildA &b, int prec, const int *slot_of, const int64_t *rowptr, int *cursor,
                             int *col, void *val, cudaStream_t s) {
    if (b.M == 0) return cudaSuccess;
    if (prec == 64)
        k_amat_fill<double><<<(unsigned)b.M, 32, 0, s>>>(b, slot_of, rowptr, cursor, col, (double *)val);
    else
        k_amat_fill<float><<<(unsigned)b.M, 32, 0, s>>>(b, slot_of, rowptr, cursor, col, (float *)val);
    return cudaGetLastError();
}

cudaError_t launch_csr_sort(int64_t nrows, int prec, const int64_t *rowptr, int *col, void *val, cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nrows + 255) / 256);
    if (prec == 64)
        k_csr_sort<double><<<nb, 256, 0, s>>>(nrows, rowptr, col, (double *)val);
    else
        k_csr_sort<float><<<nb, 256, 0, s>>>(nrows, rowptr, col, (float *)val);
    return cudaGetLastError();
}

cudaError_t launch_nmt_build(const TriBuildN &b, int pass, int prec, int64_t *counts, const int64_t *rowptr,
                             int *col, void *val, cudaStream_t s) {
    if (b.N == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((b.N + 7) / 8);
    if (prec == 64)
        k_nmt_build<double><<<nb, 256, 0, s>>>(b, pass, counts, rowptr, col, (double *)val);
    else
        k_nmt_build<float><<<nb, 256, 0, s>>>(b, pass, counts, rowptr, col, (float *)val);
    return cudaGetLastError();
}

cudaError_t launch_p0_charges(const DevPlan &p, const void *d_in, cudaStream_t s) {
    if (p.M == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((p.M + 255) / 256);
    cudaError_t e;
    if (p.prec == 64)
        e = launch_k(k_p0_charges<double>, nb, 256, 0, s, p, (const double *)d_in);
    else
        e = launch_k(k_p0_charges<float>, nb, 256, 0, s, p, (const float *)d_in);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T, int LPR>
static cudaError_t csr_go(int64_t nrows, const int64_t *rowptr, const int64_t *row_idx, const int *col, const void *val,
                          const void *x, void *y, cudaStream_t s) {
    const int64_t threads = nrows * LPR;
    const unsigned nb = (unsigned)((threads + 255) / 256);
    return launch_k(k_csr_apply<T, LPR>, nb, 256, 0, s, nrows, rowptr, row_idx, col, (const T *)val, (const T *)x,
                    (T *)y);
}

cudaError_t launch_csr_apply(int prec, int lanes_per_row, int64_t nrows, const int64_t *rowptr, const int64_t *row_idx,
                             const int *col, const void *val, const void *x, void *y, cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    cudaError_t e;
    if (prec == 64)
        e = lanes_per_row >= 32 ? csr_go<double, 32>(nrows, rowptr, row_idx, col, val, x, y, s)
                                : csr_go<double, 8>(nrows, rowptr, row_idx, col, val, x, y, s);
    else
        e = lanes_per_row >= 32 ? csr_go<float, 32>(nrows, rowptr, row_idx, col, val, x, y, s)
                                : csr_go<float, 8>(nrows, rowptr, row_idx, col, val, x, y, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace slp
