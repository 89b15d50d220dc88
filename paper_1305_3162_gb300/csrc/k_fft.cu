// Pruned 3-D FFT passes of the smooth part (paper Sec. 2.2 / Sec. 5):
//
//   phi^s = NFFT( c(N_s) (.) FFT(A) / c(Upsilon) ),
//
// with the two window deconvolutions and c_l(N_s) folded into one real,
// even table D.  Only l in I_n (|l_q| < n_q / 2; the Nyquist index is
// dropped, which keeps the result real) survives the multiply, so each
// pass transforms one axis and keeps or restores only the modes it needs:
//
//   FX  grid A[z][y][x] (real)  -> S1[z][y][kx],  kx < n_x/2   (R2C, two rows per complex FFT)
//   FY  S1 -> S2[z][ky'][kx],  ky' over n_y signed modes       (column FFT, pruned output)
//   FZ  S2 in place: FFT along z, multiply by D, inverse FFT    (fused pencil)
//   IY  S2 -> S1, zero-padded inverse along y
//   IX  S1 -> grid B (real), two rows per complex inverse FFT
//
// Each pass stages a batch of 1-D transforms in shared memory and runs a
// mixed-radix (8/4/2) Stockham autosort FFT on them; consecutive threads
// work on consecutive columns, so shared-memory accesses are conflict free
// and global accesses coalesce along the contiguous axis.  FX also writes
// zeros back to grid A so the next spread starts from a clean grid.
//
// All passes are restricted to the plan's active region: the row pairs of
// grid A the spread can reach (FX), and the rows of grid B the gather reads
// (IX); FY / IY run on the active z planes only and read / write only the
// plane's active y interval, FZ reads and writes only active z.  Rows outside
// stay zero in every buffer, which is what the full transforms would compute
// for grid A's zero rows; grid B's inactive rows are never read.
#include <cooperative_groups.h>

#include "dev_common.cuh"

namespace slp {

// 16-byte vector access to real rows: 4 floats or 2 doubles
template <typename T> struct VecW;
template <> struct VecW<float> {
    typedef float4 V;
    static constexpr int W = 4;
    __device__ static void split(const V &v, float *r) { r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w; }
    __device__ static V join(const float *r) { return make_float4(r[0], r[1], r[2], r[3]); }
    __device__ static V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <> struct VecW<double> {
    typedef double2 V;
    static constexpr int W = 2;
    __device__ static void split(const V &v, double *r) { r[0] = v.x; r[1] = v.y; }
    __device__ static V join(const double *r) { return make_double2(r[0], r[1]); }
    __device__ static V zero() { return make_double2(0.0, 0.0); }
};

// ---------------------------------------------------------------- small DFTs
template <typename C> __device__ __forceinline__ void dft2(C &a, C &b) {
    const C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C &a, C &b, C &c, C &d) {
    const C s0 = cadd(a, c), d0 = csub(a, c);
    const C s1 = cadd(b, d), d1 = csub(b, d);
    const C r1 = INV ? cmul_pi(d1) : cmul_mi(d1);
    a = cadd(s0, s1);
    c = csub(s0, s1);
    b = cadd(d0, r1);
    d = csub(d0, r1);
}

template <typename C, bool INV> __device__ __forceinline__ void dft8(C *v) {
    typedef decltype(v[0].x) R;
    const R h = R(0.70710678118654752440);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    // twiddles w8^k, w8 = exp(-+ 2 pi i / 8)
    const C t1 = INV ? cmk(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cmk(h * (o1.x + o1.y), h * (o1.y - o1.x));
    const C t2 = INV ? cmul_pi(o2) : cmul_mi(o2);
    const C t3 = INV ? cmk(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cmk(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3);
    v[7] = csub(e3, t3);
}

template <typename C, int R, bool INV> __device__ __forceinline__ void dftR(C *v) {
    if constexpr (R == 2) dft2(v[0], v[1]);
    if constexpr (R == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
    if constexpr (R == 8) dft8<C, INV>(v);
}

// One radix-R Stockham stage on B columns of length L (all powers of two,
// passed as log2 so the index arithmetic is shifts and masks).
// Column b, element j lives at buf[j * ld + b].  tw[t] = exp(-2 pi i t / L).
template <typename C, int R, bool INV>
__device__ __forceinline__ void stockham_stage(const C *__restrict__ src, C *__restrict__ dst, int lgL, int lgNs,
                                               int ld, int lgB, const C *__restrict__ tw) {
    constexpr int LGR = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int L = 1 << lgL;
    const int nj = L >> LGR;
    const int lgt = lgL - lgNs - LGR;  // log2 of the twiddle stride L / (Ns R)
    const int Bm = (1 << lgB) - 1, Nm = (1 << lgNs) - 1;
    const int total = nj << lgB;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int b = w & Bm;
        const int j = w >> lgB;
        const int k = j & Nm;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nj) * ld + b];
        if (lgNs > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C t = tw[((r * k) << lgt) & (L - 1)];
                if (INV) t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        dftR<C, R, INV>(v);
        const int base = ((j - k) << LGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + (r << lgNs)) * ld + b] = v[r];
    }
}

// Full length-L transform of B columns; returns the buffer holding the result.
// L = 2^p: p/3 radix-8 stages, then one radix-4 (p%3 == 2) or radix-2 (p%3 == 1).
template <typename C, bool INV>
__device__ C *fft_columns(C *b0, C *b1, int L, int ld, int B, const C *__restrict__ tw) {
    const int lg = __ffs(L) - 1;
    const int lgB = __ffs(B) - 1;
    const int n8 = lg / 3, rem = lg - 3 * n8;
    int lgNs = 0;
    C *src = b0, *dst = b1;
    for (int st = 0; st < n8 + (rem ? 1 : 0); ++st) {
        if (st < n8) {
            stockham_stage<C, 8, INV>(src, dst, lg, lgNs, ld, lgB, tw);
            lgNs += 3;
        } else if (rem == 2) {
            stockham_stage<C, 4, INV>(src, dst, lg, lgNs, ld, lgB, tw);
            lgNs += 2;
        } else {
            stockham_stage<C, 2, INV>(src, dst, lg, lgNs, ld, lgB, tw);
            lgNs += 1;
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// ---------------------------------------------------------------- in-place column FFT
// In-place mixed-radix transform of B columns of length L = 2^p (column b,
// element j at buf[j * ld + b]), used by the column passes so that a block
// needs one buffer instead of two and can hold more columns.
//   forward: decimation in frequency, stages s = 0 .. S-1 with radices
//     R_s (8, ..., then 4 or 2); stage s splits each block of length
//     N_s = L / (R_0 ... R_{s-1}) into R_s interleaved sub-sequences: DFT of
//     {x[k0 + j + r N_s / R_s]}_r, then twiddle W_{N_s}^{j r}, written back in
//     place.  Output: frequency k at position pos(k) (digit reversal below).
//   inverse: the same stages in reverse order, each undone (conjugate
//     twiddle first, then the DFT with the opposite sign): input at pos(k),
//     output in natural order, unnormalised.
// Radices: n8 = lgL / 3 stages of 8, then one stage of 2^rem (rem = lgL % 3)
// when rem > 0; stage s has N_s = 2^(lgL - 3 s).
struct RadixPlan {
    int n8, rem, S;
};
__device__ __forceinline__ RadixPlan radix_plan(int lgL) {
    RadixPlan r;
    r.n8 = lgL / 3;
    r.rem = lgL - 3 * r.n8;
    r.S = r.n8 + (r.rem ? 1 : 0);
    return r;
}
// position of frequency k after the forward transform: the stage-s digit of
// k (3 bits, or rem bits for the last stage, least significant first) sits at
// bit lgL - 3 (s + 1) of the position (bit 0 for the last digit)
__device__ __forceinline__ int fft_pos(const RadixPlan &rp, int lgL, int k) {
    int pos = 0;
    for (int s = 0; s < rp.n8; ++s) pos |= ((k >> (3 * s)) & 7) << (lgL - 3 * (s + 1));
    if (rp.rem) pos |= k >> (3 * rp.n8);
    return pos;
}
// frequency held at position p after the forward transform (inverse of fft_pos)
__device__ __forceinline__ int fft_freq(const RadixPlan &rp, int lgL, int p) {
    int k = 0;
    for (int s = 0; s < rp.n8; ++s) k |= ((p >> (lgL - 3 * (s + 1))) & 7) << (3 * s);
    if (rp.rem) k |= (p & ((1 << rp.rem) - 1)) << (3 * rp.n8);
    return k;
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void inplace_stage(C *__restrict__ buf, int lgL, int lgNs, int ld, int lgB,
                                              const C *__restrict__ tw) {
    constexpr int LGR = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int lgQ = lgNs - LGR;  // log2 of N_s / R
    const int Qm = (1 << lgQ) - 1, Bm = (1 << lgB) - 1;
    const int total = 1 << (lgL - LGR + lgB);
    const int lgt = lgL - lgNs;  // twiddle stride L / N_s
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int b = w & Bm;
        const int t = w >> lgB;
        const int j = t & Qm;
        const int k0 = (t >> lgQ) << lgNs;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = buf[(k0 + j + (r << lgQ)) * ld + b];
        if (INV && j != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C t2 = tw[((r * j) << lgt) & ((1 << lgL) - 1)];
                t2.y = -t2.y;
                v[r] = cmul(v[r], t2);
            }
        }
        dftR<C, R, INV>(v);
        if (!INV && j != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[((r * j) << lgt) & ((1 << lgL) - 1)]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(k0 + j + (r << lgQ)) * ld + b] = v[r];
    }
}

// All stages; ends with __syncthreads().
template <typename C, bool INV>
__device__ void fft_columns_inplace(C *buf, int lgL, int ld, int lgB, const C *__restrict__ tw) {
    const RadixPlan rp = radix_plan(lgL);
    for (int i = 0; i < rp.S; ++i) {
        const int s = INV ? rp.S - 1 - i : i;
        const int lgNs = lgL - 3 * s;
        if (s < rp.n8)
            inplace_stage<C, 8, INV>(buf, lgL, lgNs, ld, lgB, tw);
        else if (rp.rem == 2)
            inplace_stage<C, 4, INV>(buf, lgL, lgNs, ld, lgB, tw);
        else
            inplace_stage<C, 2, INV>(buf, lgL, lgNs, ld, lgB, tw);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- FX
// PB row pairs per CTA; pair pr covers rows y0 = 2*(pr % (Ly/2)) and y0+1 of plane z.
template <typename T>
__global__ void __launch_bounds__(256) k_fx(DevPlan p, int PB) {
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lx = p.L[0], Ly = p.L[1], Kx = p.Kx;
    const int ld = PB + 1;
    const int lgLx = __ffs(Lx) - 1, lgKx = __ffs(Kx) - 1, lgHy = __ffs(Ly) - 2;
    C *b0 = (C *)smem_raw;
    C *b1 = b0 + Lx * ld;
    // twiddles of this axis in shared memory (plan constants: loaded before the wait)
    C *stw = b1 + Lx * ld;
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) stw[i] = ((const C *)p.tw[0])[i];
    pdl_wait();
    pdl_trigger();
    const int npairs = p.n_row_pairs;
    const int pr0 = blockIdx.x * PB;
    T *A = (T *)p.gridA + blockIdx.y * p.st_grid;
    // rows y0 and y0+1 of each pair, VW elements per vector load; all loads are
    // issued before the zeroing stores so they overlap
    typedef typename VecW<T>::V V;
    constexpr int VW = VecW<T>::W;
    constexpr int lgVW = VW == 4 ? 2 : 1;
    const int nv = Lx / VW;
    for (int i = threadIdx.x; i < PB * nv; i += blockDim.x) {
        const int b = i >> (lgLx - lgVW), xv = i & (nv - 1);
        T ra[VW], rb[VW];
        if (pr0 + b < npairs) {
            const int pr = p.row_pairs[pr0 + b];
            const int64_t z = pr >> lgHy;
            const int y0 = 2 * (pr & ((Ly >> 1) - 1));
            const int64_t r0 = (z * Ly + y0) * Lx;
            const V va = ((const V *)(A + r0))[xv];
            const V vb = ((const V *)(A + r0 + Lx))[xv];
            VecW<T>::split(va, ra);
            VecW<T>::split(vb, rb);
        } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) ra[e] = rb[e] = T(0);
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) b0[(xv * VW + e) * ld + b] = cmk(ra[e], rb[e]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PB * nv; i += blockDim.x) {
        const int b = i >> (lgLx - lgVW), xv = i & (nv - 1);
        if (pr0 + b >= npairs) continue;
        const int pr = p.row_pairs[pr0 + b];
        const int64_t z = pr >> lgHy;
        const int y0 = 2 * (pr & ((Ly >> 1) - 1));
        const int64_t r0 = (z * Ly + y0) * Lx;
        ((V *)(A + r0))[xv] = VecW<T>::zero();
        ((V *)(A + r0 + Lx))[xv] = VecW<T>::zero();
    }
    const C *res = fft_columns<C, false>(b0, b1, Lx, ld, PB, stw);
    C *S1 = (C *)p.S1 + blockIdx.y * p.st_s1;
    for (int i = threadIdx.x; i < PB * Kx; i += blockDim.x) {
        const int b = i >> lgKx, k = i & (Kx - 1);
        if (pr0 + b >= npairs) continue;
        const int pr = p.row_pairs[pr0 + b];
        const int64_t z = pr >> lgHy;
        const int y0 = 2 * (pr & ((Ly >> 1) - 1));
        const C Z = res[k * ld + b];
        const C Zc = cconj(res[((Lx - k) & (Lx - 1)) * ld + b]);
        const C xa = cscale(cadd(Z, Zc), T(0.5));
        const C xb = cscale(cmul_mi(csub(Z, Zc)), T(0.5));  // (Z - Zc) / (2i)
        const int64_t o = (z * Ly + y0) * Kx + k;
        S1[o] = xa;
        S1[o + Kx] = xb;
    }
}

// ---------------------------------------------------------------- FY
// CTA: plane z, columns kx0 .. kx0 + B; one in-place buffer [Ly][B + 1].
template <typename T>
__global__ void __launch_bounds__(256) k_fy(DevPlan p, int B) {
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ly = p.L[1], Kx = p.Kx, ny = p.n[1];
    const int ld = B + 1;
    const int lgB = __ffs(B) - 1, lgLy = __ffs(Ly) - 1;
    C *buf = (C *)smem_raw;
    // twiddles of this axis in shared memory (plan constants: loaded before the wait)
    C *stw = buf + Ly * ld;
    for (int i = threadIdx.x; i < Ly; i += blockDim.x) stw[i] = ((const C *)p.tw[1])[i];
    pdl_wait();
    pdl_trigger();
    const int ntile = Kx / B;
    const int zi = blockIdx.x / ntile;
    const int z = (p.z0 + zi) & (p.L[2] - 1);
    const int kx0 = (blockIdx.x - zi * ntile) * B;
    const int2 iv = p.plane_iv[z];  // active rows y0 .. y0 + rows - 1 (mod Ly)
    const C *S1 = (const C *)p.S1 + blockIdx.y * p.st_s1 + (int64_t)z * Ly * Kx + kx0;
    pipelined_copy<C>(
        Ly * B,
        [&](int i) {
            const int y = i >> lgB;
            C v = cmk(T(0), T(0));
            if (((y - iv.x) & (Ly - 1)) < iv.y) v = S1[(int64_t)y * Kx + (i & (B - 1))];
            return v;
        },
        [&](int i, C v) { buf[(i >> lgB) * ld + (i & (B - 1))] = v; });
    __syncthreads();
    fft_columns_inplace<C, false>(buf, lgLy, ld, lgB, stw);
    const RadixPlan rp = radix_plan(lgLy);
    C *S2 = (C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)z * ny * Kx + kx0;
    for (int i = threadIdx.x; i < ny * B; i += blockDim.x) {
        const int kp = i >> lgB, b = i & (B - 1);
        C v = cmk(T(0), T(0));
        if (kp != ny / 2) {
            const int k = kp < ny / 2 ? kp : Ly - ny + kp;
            v = buf[fft_pos(rp, lgLy, k) * ld + b];
        }
        S2[(int64_t)kp * Kx + b] = v;
    }
}

// ---------------------------------------------------------------- FZ * D * IZ
// CTA: row ky', columns kx0 .. kx0 + B; the pencil along z stays in shared
// memory: forward transform in place (frequencies at digit-reversed
// positions), multiply by D there, inverse transform in place (natural order).
template <typename T>
__global__ void __launch_bounds__(256) k_fz(DevPlan p, int B) {
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lz = p.L[2], Kx = p.Kx, ny = p.n[1], nz = p.n[2];
    const int ld = B + 1;
    const int lgB = __ffs(B) - 1, lgLz = __ffs(Lz) - 1;
    C *buf = (C *)smem_raw;
    // twiddles of this axis in shared memory (plan constants: loaded before the wait)
    C *stw = buf + Lz * ld;
    for (int i = threadIdx.x; i < Lz; i += blockDim.x) stw[i] = ((const C *)p.tw[2])[i];
    pdl_wait();
    pdl_trigger();
    const int ntile = Kx / B;
    const int kp = blockIdx.x / ntile;
    const int kx0 = (blockIdx.x - kp * ntile) * B;
    C *S2 = (C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)kp * Kx + kx0;
    const int64_t zs = (int64_t)ny * Kx;
    const int z0 = p.z0, nza = p.nz_act;
    if (kp == ny / 2) {  // Nyquist row in y: dropped
        for (int i = threadIdx.x; i < Lz * B; i += blockDim.x) {
            const int z = i >> lgB, b = i & (B - 1);
            if (((z - z0) & (Lz - 1)) < nza) S2[z * zs + b] = cmk(T(0), T(0));
        }
        return;
    }
    pipelined_copy<C>(
        Lz * B,
        [&](int i) {
            const int z = i >> lgB;
            C v = cmk(T(0), T(0));
            if (((z - z0) & (Lz - 1)) < nza) v = S2[z * zs + (i & (B - 1))];
            return v;
        },
        [&](int i, C v) { buf[(i >> lgB) * ld + (i & (B - 1))] = v; });
    __syncthreads();
    fft_columns_inplace<C, false>(buf, lgLz, ld, lgB, stw);
    const RadixPlan rp = radix_plan(lgLz);
    const int aky = kp < ny / 2 ? kp : ny - kp;
    const T *D = (const T *)p.Dtab;
    for (int i = threadIdx.x; i < Lz * B; i += blockDim.x) {
        const int pz = i >> lgB, b = i & (B - 1);
        const int kz = fft_freq(rp, lgLz, pz);
        const int akz = kz < Lz / 2 ? kz : Lz - kz;
        C v = cmk(T(0), T(0));
        if (akz < nz / 2) {
            const T d = D[((int64_t)akz * (ny / 2) + aky) * Kx + kx0 + b];
            v = cscale(buf[pz * ld + b], d);
        }
        buf[pz * ld + b] = v;
    }
    __syncthreads();
    fft_columns_inplace<C, true>(buf, lgLz, ld, lgB, stw);
    for (int i = threadIdx.x; i < nza * B; i += blockDim.x) {
        const int z = (z0 + (i >> lgB)) & (Lz - 1), b = i & (B - 1);
        S2[z * zs + b] = buf[z * ld + b];
    }
}

// ---------------------------------------------------------------- IY
template <typename T>
__global__ void __launch_bounds__(256) k_iy(DevPlan p, int B) {
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ly = p.L[1], Kx = p.Kx, ny = p.n[1];
    const int ld = B + 1;
    const int lgB = __ffs(B) - 1, lgLy = __ffs(Ly) - 1;
    C *buf = (C *)smem_raw;
    // twiddles of this axis in shared memory (plan constants: loaded before the wait)
    C *stw = buf + Ly * ld;
    for (int i = threadIdx.x; i < Ly; i += blockDim.x) stw[i] = ((const C *)p.tw[1])[i];
    pdl_wait();
    pdl_trigger();
    const int ntile = Kx / B;
    const int zi = blockIdx.x / ntile;
    const int z = (p.z0 + zi) & (p.L[2] - 1);
    const int kx0 = (blockIdx.x - zi * ntile) * B;
    const int2 iv = p.plane_iv[z];
    const C *S2 = (const C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)z * ny * Kx + kx0;
    // position q holds frequency k = fft_freq(q): mode k (k < ny/2) or mode
    // k - Ly (k > Ly - ny/2), zero elsewhere
    const RadixPlan rp = radix_plan(lgLy);
    pipelined_copy<C>(
        Ly * B,
        [&](int i) {
            const int k = fft_freq(rp, lgLy, i >> lgB), b = i & (B - 1);
            C v = cmk(T(0), T(0));
            if (k < ny / 2)
                v = S2[(int64_t)k * Kx + b];
            else if (k > Ly - ny / 2)
                v = S2[(int64_t)(k - Ly + ny) * Kx + b];
            return v;
        },
        [&](int i, C v) { buf[(i >> lgB) * ld + (i & (B - 1))] = v; });
    __syncthreads();
    fft_columns_inplace<C, true>(buf, lgLy, ld, lgB, stw);
    C *S1 = (C *)p.S1 + blockIdx.y * p.st_s1 + (int64_t)z * Ly * Kx + kx0;
    for (int i = threadIdx.x; i < iv.y * B; i += blockDim.x) {
        const int y = (iv.x + (i >> lgB)) & (Ly - 1), b = i & (B - 1);
        S1[(int64_t)y * Kx + b] = buf[y * ld + b];
    }
}

// ---------------------------------------------------------------- IX
template <typename T>
__global__ void __launch_bounds__(256) k_ix(DevPlan p, int PB) {
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lx = p.L[0], Ly = p.L[1], Kx = p.Kx;
    const int ld = PB + 1;
    const int lgLx = __ffs(Lx) - 1, lgKx = __ffs(Kx) - 1, lgHy = __ffs(Ly) - 2;
    C *b0 = (C *)smem_raw;
    C *b1 = b0 + Lx * ld;
    // twiddles of this axis in shared memory (plan constants: loaded before the wait)
    C *stw = b1 + Lx * ld;
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) stw[i] = ((const C *)p.tw[0])[i];
    const int npairs = p.n_row_pairs;
    const int pr0 = blockIdx.x * PB;
    for (int i = threadIdx.x; i < PB * Lx; i += blockDim.x) b0[(i & (Lx - 1)) * ld + (i >> lgLx)] = cmk(T(0), T(0));
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    const C *S1 = (const C *)p.S1 + blockIdx.y * p.st_s1;
    typedef typename VecT<T>::T4 T4;  // (xa, xb) of one mode, loaded together
    pipelined_copy<T4>(
        PB * Kx,
        [&](int i) {
            const int b = i >> lgKx, k = i & (Kx - 1);
            T4 v;
            v.x = v.y = v.z = v.w = T(0);
            if (pr0 + b < npairs) {
                const int pr = p.row_pairs[pr0 + b];
                const int64_t z = pr >> lgHy;
                const int y0 = 2 * (pr & ((Ly >> 1) - 1));
                const int64_t o = (z * Ly + y0) * Kx + k;
                const C xa = S1[o], xb = S1[o + Kx];
                v.x = xa.x;
                v.y = xa.y;
                v.z = xb.x;
                v.w = xb.y;
            }
            return v;
        },
        [&](int i, T4 v) {
            const int b = i >> lgKx, k = i & (Kx - 1);
            if (pr0 + b >= npairs) return;
            if (k == 0) {
                b0[b] = cmk(v.x, v.z);
            } else {
                b0[k * ld + b] = cmk(v.x - v.w, v.y + v.z);          // xa + i xb
                b0[(Lx - k) * ld + b] = cmk(v.x + v.w, v.z - v.y);   // conj(xa) + i conj(xb)
            }
        });
    __syncthreads();
    const C *res = fft_columns<C, true>(b0, b1, Lx, ld, PB, stw);
    T *G = (T *)p.gridB + blockIdx.y * p.st_grid;
    typedef typename VecW<T>::V V;
    constexpr int VW = VecW<T>::W;
    constexpr int lgVW = VW == 4 ? 2 : 1;
    const int nv = Lx / VW;
    for (int i = threadIdx.x; i < PB * nv; i += blockDim.x) {
        const int b = i >> (lgLx - lgVW), xv = i & (nv - 1);
        if (pr0 + b >= npairs) continue;
        const int pr = p.row_pairs[pr0 + b];
        const int64_t z = pr >> lgHy;
        const int y0 = 2 * (pr & ((Ly >> 1) - 1));
        const int64_t r0 = (z * Ly + y0) * Lx;
        T ra[VW], rb[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const C v = res[(xv * VW + e) * ld + b];
            ra[e] = v.x;
            rb[e] = v.y;
        }
        ((V *)(G + r0))[xv] = VecW<T>::join(ra);
        ((V *)(G + r0 + Lx))[xv] = VecW<T>::join(rb);
    }
}

// ---------------------------------------------------------------- column engine
// Column passes with the transform length L = 2^LG fixed at compile time (so
// all index arithmetic folds) and the stages kept in registers: a block of
// 8 L/8 threads transforms CB = 8 columns; thread (t, b) (b the column) owns
// eight elements of column b in every stage, the in-place decimation-in-
// frequency stages of fft_columns_inplace (radix 8, then 4 or 2 for the
// remaining bits).  Stage 0 reads its elements from global memory and the
// last stage writes them back; between stages the elements are exchanged
// through one shared buffer [L][CB + 1] with one barrier per exchange.  A
// thread writes back exactly the positions it read, so a stage needs no
// barrier between its read and its write.
constexpr int CB = 8;
// Register budget: blocks of L threads are asked to fit 1024 / L per SM (at
// most 64 registers a thread) for L <= 256, and for the z pass at every L;
// the y passes at L >= 512 use the variants without a minimum (`_long`).
// Chosen by measurement on the 128^3 sphere and the 1024^3 cube.

template <int LG> struct ColShape {
    static constexpr int L = 1 << LG, S8 = LG / 3, REM = LG - 3 * S8, NS = S8 + (REM ? 1 : 0);
};

// position of element r of task t in stage S
template <int LG, int S> __device__ __forceinline__ int col_idx(int t, int r) {
    typedef ColShape<LG> Sh;
    if constexpr (S < Sh::S8) {
        constexpr int lgNs = LG - 3 * S, lgQ = lgNs - 3;
        const int j = t & ((1 << lgQ) - 1), k0 = (t >> lgQ) << lgNs;
        return k0 + j + (r << lgQ);
    } else {
        return (t << 3) + r;  // the last stage, radix 2^REM: 8 / 2^REM butterflies of consecutive elements
    }
}

// frequency at position p after the forward stages
template <int LG> __device__ __forceinline__ int col_freq(int p) {
    typedef ColShape<LG> Sh;
    int k = 0;
#pragma unroll
    for (int s = 0; s < Sh::S8; ++s) k |= ((p >> (LG - 3 * (s + 1))) & 7) << (3 * s);
    if constexpr (Sh::REM > 0) k |= (p & ((1 << Sh::REM) - 1)) << (3 * Sh::S8);
    return k;
}

// stage S on the eight elements of task t (forward: DFT then twiddle;
// inverse: conjugate twiddle then DFT)
template <typename C, int LG, int S, bool INV> __device__ __forceinline__ void col_stage(C (&v)[8], int t, const C *tw) {
    typedef ColShape<LG> Sh;
    if constexpr (S < Sh::S8) {
        constexpr int lgQ = LG - 3 * S - 3;
        const int j = t & ((1 << lgQ) - 1);
        if (INV && j != 0) {
#pragma unroll
            for (int r = 1; r < 8; ++r) {
                C w = tw[((r * j) << (3 * S)) & (Sh::L - 1)];
                w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft8<C, INV>(v);
        if (!INV && j != 0) {
#pragma unroll
            for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], tw[((r * j) << (3 * S)) & (Sh::L - 1)]);
        }
    } else if constexpr (Sh::REM == 2) {
        dft4<C, INV>(v[0], v[1], v[2], v[3]);
        dft4<C, INV>(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) dft2(v[2 * u], v[2 * u + 1]);
    }
}

template <typename C, int LG, int S> __device__ __forceinline__ void col_put(C *buf, const C (&v)[8], int t, int b) {
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[col_idx<LG, S>(t, r) * (CB + 1) + b] = v[r];
}
template <typename C, int LG, int S> __device__ __forceinline__ void col_get(const C *buf, C (&v)[8], int t, int b) {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = buf[col_idx<LG, S>(t, r) * (CB + 1) + b];
}

// forward stages S .. NS-1 (the elements of stage S - 1 are in v and are
// exchanged first); on return v holds the last stage's elements
template <typename C, int LG, int S> __device__ __forceinline__ void col_forward_from(C *buf, C (&v)[8], int t, int b,
                                                                                   const C *tw) {
    if constexpr (S < ColShape<LG>::NS) {
        col_put<C, LG, S - 1>(buf, v, t, b);
        __syncthreads();
        col_get<C, LG, S>(buf, v, t, b);
        col_stage<C, LG, S, false>(v, t, tw);
        col_forward_from<C, LG, S + 1>(buf, v, t, b, tw);
    }
}
// inverse stages S .. 0 (v holds the elements of stage S + 1 after its inverse)
template <typename C, int LG, int S> __device__ __forceinline__ void col_inverse_from(C *buf, C (&v)[8], int t, int b,
                                                                                   const C *tw) {
    if constexpr (S >= 0) {
        col_put<C, LG, S + 1>(buf, v, t, b);
        __syncthreads();
        col_get<C, LG, S>(buf, v, t, b);
        col_stage<C, LG, S, true>(v, t, tw);
        col_inverse_from<C, LG, S - 1>(buf, v, t, b, tw);
    }
}

// FY: plane z, columns kx0 .. kx0 + 8; active rows in, the n_y kept modes out
template <typename T, int LG>
__device__ __forceinline__ void k_fy_c_body(const DevPlan &p) {
    typedef typename VecT<T>::T2 C;
    typedef ColShape<LG> Sh;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = (C *)smem_raw;
    C *tw = buf + Sh::L * (CB + 1);
    for (int i = threadIdx.x; i < Sh::L; i += blockDim.x) tw[i] = ((const C *)p.tw[1])[i];
    const int b = threadIdx.x & (CB - 1), t = threadIdx.x >> 3;
    const int Kx = p.Kx, ny = p.n[1];
    const int ntile = Kx / CB;
    const int zi = blockIdx.x / ntile;
    const int z = (p.z0 + zi) & (p.L[2] - 1);
    const int kx0 = (blockIdx.x - zi * ntile) * CB;
    pdl_wait();
    pdl_trigger();
    const int2 iv = p.plane_iv[z];
    const C *S1 = (const C *)p.S1 + blockIdx.y * p.st_s1 + (int64_t)z * Sh::L * Kx + kx0 + b;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int y = col_idx<LG, 0>(t, r);
        v[r] = ((y - iv.x) & (Sh::L - 1)) < iv.y ? S1[(int64_t)y * Kx] : cmk(T(0), T(0));
    }
    __syncthreads();  // twiddles
    col_stage<C, LG, 0, false>(v, t, tw);
    col_forward_from<C, LG, 1>(buf, v, t, b, tw);
    C *S2 = (C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)z * ny * Kx + kx0 + b;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int k = col_freq<LG>(col_idx<LG, Sh::NS - 1>(t, r));
        if (k < ny / 2)
            S2[(int64_t)k * Kx] = v[r];
        else if (k > Sh::L - ny / 2)
            S2[(int64_t)(k - Sh::L + ny) * Kx] = v[r];
    }
}
// at L <= 256 a block asks for 1024 / L blocks per SM (at most 64 registers);
// longer transforms keep the compiler's own choice
template <typename T, int LG>
__global__ void __launch_bounds__(1 << LG, (1024 >> LG)) k_fy_c(DevPlan p) { k_fy_c_body<T, LG>(p); }
template <typename T, int LG>
__global__ void __launch_bounds__(1 << LG) k_fy_c_long(DevPlan p) { k_fy_c_body<T, LG>(p); }

// FZ * D * IZ: row ky', columns kx0 .. kx0 + 8; the last forward stage, the
// multiply and the first inverse stage share the same registers
template <typename T, int LG>
__global__ void __launch_bounds__(1 << LG, (1024 >> LG) > 0 ? (1024 >> LG) : 1) k_fz_c(DevPlan p) {
    typedef typename VecT<T>::T2 C;
    typedef ColShape<LG> Sh;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = (C *)smem_raw;
    C *tw = buf + Sh::L * (CB + 1);
    for (int i = threadIdx.x; i < Sh::L; i += blockDim.x) tw[i] = ((const C *)p.tw[2])[i];
    const int b = threadIdx.x & (CB - 1), t = threadIdx.x >> 3;
    const int Kx = p.Kx, ny = p.n[1], nz = p.n[2];
    const int ntile = Kx / CB;
    const int kp = blockIdx.x / ntile;
    const int kx0 = (blockIdx.x - kp * ntile) * CB;
    const int z0 = p.z0, nza = p.nz_act;
    const int64_t zs = (int64_t)ny * Kx;
    pdl_wait();
    pdl_trigger();
    C *S2 = (C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)kp * Kx + kx0 + b;
    if (kp == ny / 2) {  // Nyquist row in y: dropped
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int z = col_idx<LG, 0>(t, r);
            if (((z - z0) & (Sh::L - 1)) < nza) S2[z * zs] = cmk(T(0), T(0));
        }
        return;
    }
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int z = col_idx<LG, 0>(t, r);
        v[r] = ((z - z0) & (Sh::L - 1)) < nza ? S2[z * zs] : cmk(T(0), T(0));
    }
    // the multipliers of the elements this thread holds after the forward
    // stages depend on its positions only: load them now, beside the pencil
    const int aky = kp < ny / 2 ? kp : ny - kp;
    const T *D = (const T *)p.Dtab + (int64_t)aky * Kx + kx0 + b;
    const int64_t dz = (int64_t)(ny / 2) * Kx;
    T dv[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int kz = col_freq<LG>(col_idx<LG, Sh::NS - 1>(t, r));
        const int akz = kz < Sh::L / 2 ? kz : Sh::L - kz;
        dv[r] = akz < nz / 2 ? D[akz * dz] : T(0);
    }
    __syncthreads();  // twiddles
    col_stage<C, LG, 0, false>(v, t, tw);
    col_forward_from<C, LG, 1>(buf, v, t, b, tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = cscale(v[r], dv[r]);
    col_stage<C, LG, Sh::NS - 1, true>(v, t, tw);
    col_inverse_from<C, LG, Sh::NS - 2>(buf, v, t, b, tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int z = col_idx<LG, 0>(t, r);
        if (((z - z0) & (Sh::L - 1)) < nza) S2[z * zs] = v[r];
    }
}

// IY: plane z, columns kx0 .. kx0 + 8; the kept modes in (zero padded),
// active rows out
template <typename T, int LG>
__device__ __forceinline__ void k_iy_c_body(const DevPlan &p) {
    typedef typename VecT<T>::T2 C;
    typedef ColShape<LG> Sh;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = (C *)smem_raw;
    C *tw = buf + Sh::L * (CB + 1);
    for (int i = threadIdx.x; i < Sh::L; i += blockDim.x) tw[i] = ((const C *)p.tw[1])[i];
    const int b = threadIdx.x & (CB - 1), t = threadIdx.x >> 3;
    const int Kx = p.Kx, ny = p.n[1];
    const int ntile = Kx / CB;
    const int zi = blockIdx.x / ntile;
    const int z = (p.z0 + zi) & (p.L[2] - 1);
    const int kx0 = (blockIdx.x - zi * ntile) * CB;
    pdl_wait();
    pdl_trigger();
    const int2 iv = p.plane_iv[z];
    const C *S2 = (const C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)z * ny * Kx + kx0 + b;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int k = col_freq<LG>(col_idx<LG, Sh::NS - 1>(t, r));
        C x = cmk(T(0), T(0));
        if (k < ny / 2)
            x = S2[(int64_t)k * Kx];
        else if (k > Sh::L - ny / 2)
            x = S2[(int64_t)(k - Sh::L + ny) * Kx];
        v[r] = x;
    }
    __syncthreads();  // twiddles
    col_stage<C, LG, Sh::NS - 1, true>(v, t, tw);
    col_inverse_from<C, LG, Sh::NS - 2>(buf, v, t, b, tw);
    C *S1 = (C *)p.S1 + blockIdx.y * p.st_s1 + (int64_t)z * Sh::L * Kx + kx0 + b;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int y = col_idx<LG, 0>(t, r);
        if (((y - iv.x) & (Sh::L - 1)) < iv.y) S1[(int64_t)y * Kx] = v[r];
    }
}
// at L <= 256 a block asks for 1024 / L blocks per SM (at most 64 registers);
// longer transforms keep the compiler's own choice
template <typename T, int LG>
__global__ void __launch_bounds__(1 << LG, (1024 >> LG)) k_iy_c(DevPlan p) { k_iy_c_body<T, LG>(p); }
template <typename T, int LG>
__global__ void __launch_bounds__(1 << LG) k_iy_c_long(DevPlan p) { k_iy_c_body<T, LG>(p); }

// ---------------------------------------------------------------- x inverse, compile-time length
// The inverse row pass with Lx = 2^LG fixed at compile time: CB row pairs per block,
// L / 8 threads per pair (t fastest, so a warp touches consecutive x), one
// radix-8 butterfly per thread per stage (radix 8 stages, then 4 or 2).
// Stockham stages take natural-order input (the first stage reads the
// spectrum straight from S1) and leave natural-order output, which is read
// back by consecutive x.  One shared buffer: a stage reads its eight inputs,
// waits, writes its eight outputs, waits.
template <typename C, int LG, int S, bool INV>
__device__ __forceinline__ void stk_compute_store(C *buf, C (&v)[8], int t, int b, const C *tw) {
    typedef ColShape<LG> Sh;
    constexpr int LGR = S < Sh::S8 ? 3 : Sh::REM;
    constexpr int R = 1 << LGR, NB = 8 / R, lgNs = 3 * S;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = t + u * (Sh::L / 8);
        const int k = j & ((1 << lgNs) - 1);
        C *w = v + u * R;
        if constexpr (lgNs > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C tt = tw[((r * k) << (LG - lgNs - LGR)) & (Sh::L - 1)];
                if (INV) tt.y = -tt.y;
                w[r] = cmul(w[r], tt);
            }
        }
        if constexpr (R == 8) dft8<C, INV>(w);
        if constexpr (R == 4) dft4<C, INV>(w[0], w[1], w[2], w[3]);
        if constexpr (R == 2) dft2(w[0], w[1]);
        const int base = ((j - k) << LGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + (r << lgNs)) * (CB + 1) + b] = w[r];
    }
}
// inputs of stage S for thread t: elements j + r L / R, j = t + u L / 8
template <typename C, int LG, int S>
__device__ __forceinline__ void stk_load(const C *buf, C (&v)[8], int t, int b) {
    typedef ColShape<LG> Sh;
    constexpr int LGR = S < Sh::S8 ? 3 : Sh::REM;
    constexpr int R = 1 << LGR, NB = 8 / R;
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) v[u * R + r] = buf[(t + u * (Sh::L / 8) + r * (Sh::L >> LGR)) * (CB + 1) + b];
}
// stages S .. NS-1 (stage S - 1 already stored); ends with a barrier
template <typename C, int LG, int S, bool INV>
__device__ __forceinline__ void stk_from(C *buf, int t, int b, const C *tw) {
    if constexpr (S < ColShape<LG>::NS) {
        C v[8];
        stk_load<C, LG, S>(buf, v, t, b);
        __syncthreads();
        stk_compute_store<C, LG, S, INV>(buf, v, t, b, tw);
        __syncthreads();
        stk_from<C, LG, S + 1, INV>(buf, t, b, tw);
    }
}

template <typename T, int LG>
__global__ void __launch_bounds__(1 << LG) k_ix_s(DevPlan p) {
    typedef typename VecT<T>::T2 C;
    typedef ColShape<LG> Sh;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = (C *)smem_raw;
    C *tw = buf + Sh::L * (CB + 1);
    for (int i = threadIdx.x; i < Sh::L; i += blockDim.x) tw[i] = ((const C *)p.tw[0])[i];
    constexpr int TPB = Sh::L / 8;
    const int b = threadIdx.x / TPB, t = threadIdx.x - b * TPB;
    const int Ly = p.L[1], Kx = p.Kx;
    const int lgHy = __ffs(Ly) - 2;
    const int pr = blockIdx.x * CB + b;
    const bool on = pr < p.n_row_pairs;
    pdl_wait();
    pdl_trigger();
    int64_t r0 = 0;
    if (on) {
        const int rp = p.row_pairs[pr];
        r0 = ((int64_t)(rp >> lgHy) * Ly + 2 * (rp & ((Ly >> 1) - 1))) * Sh::L;
    }
    // stage 0 reads frequencies t + r L / 8 of the pair's complex spectrum
    // Y(k) = xa(k) + i xb(k), Y(L - k) = conj(xa(k)) + i conj(xb(k))
    const C *S1 = (const C *)p.S1 + blockIdx.y * p.st_s1 + r0 / Sh::L * Kx;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int k = t + r * TPB;
        C y = cmk(T(0), T(0));
        if (on) {
            if (k == 0) {
                y = cmk(S1[0].x, S1[Kx].x);
            } else if (k < Kx) {
                const C xa = S1[k], xb = S1[Kx + k];
                y = cmk(xa.x - xb.y, xa.y + xb.x);
            } else if (k > Sh::L - Kx) {
                const C xa = S1[Sh::L - k], xb = S1[Kx + Sh::L - k];
                y = cmk(xa.x + xb.y, xb.x - xa.y);
            }
        }
        v[r] = y;
    }
    __syncthreads();  // twiddles
    stk_compute_store<C, LG, 0, true>(buf, v, t, b, tw);
    __syncthreads();
    stk_from<C, LG, 1, true>(buf, t, b, tw);
    if (!on) return;
    T *G = (T *)p.gridB + blockIdx.y * p.st_grid + r0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int x = t + r * TPB;
        const C y = buf[x * (CB + 1) + b];
        G[x] = y.x;
        G[Sh::L + x] = y.y;
    }
}

// ---------------------------------------------------------------- fused plane passes
// FX + FY and IY + IX of one active z plane run in a thread-block cluster of
// FUSE_CL CTAs that exchange the plane spectrum through distributed shared
// memory, so S1 never goes to global memory and two launches disappear.
// CTA c of a cluster owns row pairs [c PB/CL, (c+1) PB/CL) of the plane for
// the x transforms and spectrum columns [c Kx/CL, (c+1) Kx/CL) for the y
// transforms.  Per CTA: X0, X1 [Lx][PB/CL + 1] (x transforms), P [Ly][Kx/CL + 1]
// (its columns of the plane spectrum), twiddles of x and y.  Every CTA passes
// both cluster barriers (no early exit), so each remote store lands in live
// shared memory before the barrier that orders it.
constexpr int FUSE_CL = 4;

template <typename T>
__global__ void __launch_bounds__(256) k_fxy(DevPlan p, int PB) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lx = p.L[0], Ly = p.L[1], Kx = p.Kx, ny = p.n[1];
    const int c = (int)cluster.block_rank();
    const int PBc = PB / FUSE_CL, KC = Kx / FUSE_CL;
    const int ldx = PBc + 1, ldp = KC + 1;
    const int lgKx = __ffs(Kx) - 1, lgKC = __ffs(KC) - 1, lgLy = __ffs(Ly) - 1;
    C *X0 = (C *)smem_raw;
    C *X1 = X0 + Lx * ldx;
    C *P = X1 + Lx * ldx;
    C *twx = P + Ly * ldp;
    C *twy = twx + Lx;
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) twx[i] = ((const C *)p.tw[0])[i];
    for (int i = threadIdx.x; i < Ly; i += blockDim.x) twy[i] = ((const C *)p.tw[1])[i];
    for (int i = threadIdx.x; i < Ly * ldp; i += blockDim.x) P[i] = cmk(T(0), T(0));
    const int z = (p.z0 + (int)blockIdx.x / FUSE_CL) & (p.L[2] - 1);
    pdl_wait();
    pdl_trigger();
    const int2 iv = p.plane_iv[z];
    const int npr = iv.y >> 1;
    const int j0 = c * PBc;
    const int nj = npr - j0 < 0 ? 0 : (npr - j0 > PBc ? PBc : npr - j0);
    T *A = (T *)p.gridA + blockIdx.y * p.st_grid + (int64_t)z * Ly * Lx;
    typedef typename VecW<T>::V V;
    constexpr int VW = VecW<T>::W;
    const int nv = Lx / VW, lgnv = __ffs(nv) - 1;
    // own pairs: rows ya, ya + 1 -> column j of X0
    for (int i = threadIdx.x; i < (PBc << lgnv); i += blockDim.x) {
        const int j = i >> lgnv, xv = i & (nv - 1);
        T ra[VW], rb[VW];
        if (j < nj) {
            const int ya = (iv.x + 2 * (j0 + j)) & (Ly - 1);
            VecW<T>::split(((const V *)(A + (int64_t)ya * Lx))[xv], ra);
            VecW<T>::split(((const V *)(A + (int64_t)(ya + 1) * Lx))[xv], rb);
        } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) ra[e] = rb[e] = T(0);
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) X0[(xv * VW + e) * ldx + j] = cmk(ra[e], rb[e]);
    }
    // every CTA's P is clear before any remote store; X0 is complete
    cluster.sync();
    for (int i = threadIdx.x; i < (nj << lgnv); i += blockDim.x) {
        const int j = i >> lgnv, xv = i & (nv - 1);
        const int ya = (iv.x + 2 * (j0 + j)) & (Ly - 1);
        ((V *)(A + (int64_t)ya * Lx))[xv] = VecW<T>::zero();
        ((V *)(A + (int64_t)(ya + 1) * Lx))[xv] = VecW<T>::zero();
    }
    const C *res = fft_columns<C, false>(X0, X1, Lx, ldx, PBc, twx);
    // pair j, frequency k -> rows ya, ya + 1, column k & (KC - 1) of CTA k / KC
    for (int i = threadIdx.x; i < (nj << lgKx); i += blockDim.x) {
        const int j = i >> lgKx, k = i & (Kx - 1);
        const int ya = (iv.x + 2 * (j0 + j)) & (Ly - 1);
        const C Z = res[k * ldx + j];
        const C Zc = cconj(res[((Lx - k) & (Lx - 1)) * ldx + j]);
        C *dst = cluster.map_shared_rank(P, k >> lgKC);
        dst[ya * ldp + (k & (KC - 1))] = cscale(cadd(Z, Zc), T(0.5));
        dst[(ya + 1) * ldp + (k & (KC - 1))] = cscale(cmul_mi(csub(Z, Zc)), T(0.5));
    }
    // all rows of this CTA's columns have arrived
    cluster.sync();
    fft_columns_inplace<C, false>(P, lgLy, ldp, lgKC, twy);
    const RadixPlan rp = radix_plan(lgLy);
    C *S2 = (C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)z * ny * Kx + c * KC;
    for (int i = threadIdx.x; i < ny * KC; i += blockDim.x) {
        const int kp = i >> lgKC, b = i & (KC - 1);
        C v = cmk(T(0), T(0));
        if (kp != ny / 2) {
            const int k = kp < ny / 2 ? kp : Ly - ny + kp;
            v = P[fft_pos(rp, lgLy, k) * ldp + b];
        }
        S2[(int64_t)kp * Kx + b] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_iyx(DevPlan p, int PB) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    typedef typename VecT<T>::T2 C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lx = p.L[0], Ly = p.L[1], Kx = p.Kx, ny = p.n[1];
    const int c = (int)cluster.block_rank();
    const int PBc = PB / FUSE_CL, KC = Kx / FUSE_CL;
    const int ldx = PBc + 1, ldp = KC + 1;
    const int lgKC = __ffs(KC) - 1, lgPBc = __ffs(PBc) - 1, lgLy = __ffs(Ly) - 1;
    C *X0 = (C *)smem_raw;
    C *X1 = X0 + Lx * ldx;
    C *P = X1 + Lx * ldx;
    C *twx = P + Ly * ldp;
    C *twy = twx + Lx;
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) twx[i] = ((const C *)p.tw[0])[i];
    for (int i = threadIdx.x; i < Ly; i += blockDim.x) twy[i] = ((const C *)p.tw[1])[i];
    for (int i = threadIdx.x; i < Lx * ldx; i += blockDim.x) X0[i] = cmk(T(0), T(0));
    const int z = (p.z0 + (int)blockIdx.x / FUSE_CL) & (p.L[2] - 1);
    pdl_wait();
    pdl_trigger();
    const int2 iv = p.plane_iv[z];
    const int npr = iv.y >> 1;
    const int j0 = c * PBc;
    const int nj = npr - j0 < 0 ? 0 : (npr - j0 > PBc ? PBc : npr - j0);
    // this CTA's columns of the plane spectrum at the positions of the
    // in-place inverse: position q holds mode k = fft_freq(q) (k < ny/2), or
    // k - Ly (k > Ly - ny/2), zero elsewhere
    const RadixPlan rp = radix_plan(lgLy);
    const C *S2 = (const C *)p.S2 + blockIdx.y * p.st_s2 + (int64_t)z * ny * Kx + c * KC;
    pipelined_copy<C>(
        Ly * KC,
        [&](int i) {
            const int k = fft_freq(rp, lgLy, i >> lgKC), b = i & (KC - 1);
            C v = cmk(T(0), T(0));
            if (k < ny / 2)
                v = S2[(int64_t)k * Kx + b];
            else if (k > Ly - ny / 2)
                v = S2[(int64_t)(k - Ly + ny) * Kx + b];
            return v;
        },
        [&](int i, C v) { P[(i >> lgKC) * ldp + (i & (KC - 1))] = v; });
    // every CTA's X0 is clear before any remote store; P is complete
    cluster.sync();
    fft_columns_inplace<C, true>(P, lgLy, ldp, lgKC, twy);
    // pair jj of the plane, frequency k of this CTA -> column jj % PBc of CTA jj / PBc:
    // one complex inverse transform carries row ya (real part) and ya + 1 (imaginary part)
    for (int i = threadIdx.x; i < (npr << lgKC); i += blockDim.x) {
        const int jj = i >> lgKC, kl = i & (KC - 1);
        const int k = c * KC + kl;
        const int ya = (iv.x + 2 * jj) & (Ly - 1);
        const C xa = P[ya * ldp + kl], xb = P[(ya + 1) * ldp + kl];
        C *dst = cluster.map_shared_rank(X0, jj >> lgPBc);
        const int jl = jj & (PBc - 1);
        if (k == 0) {
            dst[jl] = cmk(xa.x, xb.x);
        } else {
            dst[k * ldx + jl] = cmk(xa.x - xb.y, xa.y + xb.x);          // xa + i xb
            dst[(Lx - k) * ldx + jl] = cmk(xa.x + xb.y, xb.x - xa.y);   // conj(xa) + i conj(xb)
        }
    }
    // all frequencies of this CTA's pairs have arrived
    cluster.sync();
    const C *res = fft_columns<C, true>(X0, X1, Lx, ldx, PBc, twx);
    T *G = (T *)p.gridB + blockIdx.y * p.st_grid + (int64_t)z * Ly * Lx;
    typedef typename VecW<T>::V V;
    constexpr int VW = VecW<T>::W;
    const int nv = Lx / VW, lgnv = __ffs(nv) - 1;
    for (int i = threadIdx.x; i < (nj << lgnv); i += blockDim.x) {
        const int j = i >> lgnv, xv = i & (nv - 1);
        const int ya = (iv.x + 2 * (j0 + j)) & (Ly - 1);
        T ra[VW], rb[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const C v = res[(xv * VW + e) * ldx + j];
            ra[e] = v.x;
            rb[e] = v.y;
        }
        ((V *)(G + (int64_t)ya * Lx))[xv] = VecW<T>::join(ra);
        ((V *)(G + (int64_t)(ya + 1) * Lx))[xv] = VecW<T>::join(rb);
    }
}

// ---------------------------------------------------------------- fused column passes
// FY, FZ * D * IZ and IY of one stored x frequency kx run in a cluster of
// YZY_CL CTAs; the kx slab of the spectrum, P[ky'][z] over the n_y kept
// modes and the active z planes, never leaves distributed shared memory.
// CTA c owns the active planes zi in [c ZC, (c+1) ZC) of the slab:
//   1. FY of its planes (column engine, S1 rows in, kept modes into its P);
//   2. after a cluster barrier, the z pencils of rows ky' in [c KC, (c+1) KC):
//      each element is read from, and written back to, the P of the CTA that
//      owns its plane (every element has one reader and one writer);
//   3. after a second barrier, IY of its planes from its own P into S1.
// A block of G L threads runs G groups of the column engine side by side
// (group g transforms columns 8 g .. 8 g + 7 with its own exchange buffer).
// No CTA touches another's shared memory after the second barrier, so CTAs
// may exit in any order.  Needs L_y = L_z = L.

template <typename T, int LG>
__global__ void __launch_bounds__(512) k_yzy(DevPlan p, int ZC, int ZP) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    typedef typename VecT<T>::T2 C;
    typedef ColShape<LG> Sh;
    constexpr int L = Sh::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kx = p.Kx, ny = p.n[1], nz = p.n[2];
    const int KC = ny / YZY_CL;
    const int c = (int)cluster.block_rank();
    const int kx = (int)blockIdx.x / YZY_CL;
    const int g = threadIdx.x >> LG, lt = threadIdx.x & (L - 1);
    const int b = lt & (CB - 1), t = lt >> 3;
    const int col = g * CB + b;
    C *P = (C *)smem_raw;                 // [ny][ZP]
    C *tw = P + (size_t)ny * ZP;          // [L]
    C *buf = tw + L + (size_t)g * L * (CB + 1);  // this group's exchange buffer
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = ((const C *)p.tw[1])[i];
    const int z0 = p.z0, nza = p.nz_act;

    // step 1 / 3 column: active plane zi of this CTA
    const int zi = c * ZC + col;
    const bool on13 = col < ZC && zi < nza;
    const int z = (z0 + zi) & (L - 1);
    // step 2 column: row ky' (the Nyquist row ny / 2 is dropped)
    const int kp = c * KC + col;
    const bool on2 = col < KC && kp != ny / 2;
    // multipliers of step 2 (plan data, loaded before the wait)
    T dv[8];
    {
        const int aky = kp < ny / 2 ? kp : ny - kp;
        const T *D = (const T *)p.Dtab + (int64_t)aky * Kx + kx;
        const int64_t dz = (int64_t)(ny / 2) * Kx;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int kz = col_freq<LG>(col_idx<LG, Sh::NS - 1>(t, r));
            const int akz = kz < L / 2 ? kz : L - kz;
            dv[r] = (on2 && akz < nz / 2) ? D[akz * dz] : T(0);
        }
    }
    const int2 iv = on13 ? p.plane_iv[z] : make_int2(0, 0);
    pdl_wait();
    pdl_trigger();
    C *S1 = (C *)p.S1 + blockIdx.y * p.st_s1 + (int64_t)z * L * Kx + kx;

    // 1. FY of plane z: active rows in, kept modes to P[ky'][col]
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int y = col_idx<LG, 0>(t, r);
        v[r] = (on13 && ((y - iv.x) & (L - 1)) < iv.y) ? S1[(int64_t)y * Kx] : cmk(T(0), T(0));
    }
    __syncthreads();  // twiddles
    col_stage<C, LG, 0, false>(v, t, tw);
    col_forward_from<C, LG, 1>(buf, v, t, b, tw);
    if (on13) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int k = col_freq<LG>(col_idx<LG, Sh::NS - 1>(t, r));
            if (k < ny / 2)
                P[k * ZP + col] = v[r];
            else if (k > L - ny / 2)
                P[(k - L + ny) * ZP + col] = v[r];
        }
    }
    cluster.sync();

    // 2. z pencil of row kp: element z lives in the P of CTA (z - z0) / ZC
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int zr = col_idx<LG, 0>(t, r);
        const int zir = (zr - z0) & (L - 1);
        C x = cmk(T(0), T(0));
        if (on2 && zir < nza) {
            const int q = zir / ZC;
            x = *cluster.map_shared_rank(P + kp * ZP + (zir - q * ZC), q);
        }
        v[r] = x;
    }
    col_stage<C, LG, 0, false>(v, t, tw);
    col_forward_from<C, LG, 1>(buf, v, t, b, tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = cscale(v[r], dv[r]);
    col_stage<C, LG, Sh::NS - 1, true>(v, t, tw);
    col_inverse_from<C, LG, Sh::NS - 2>(buf, v, t, b, tw);
    if (on2) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int zr = col_idx<LG, 0>(t, r);
            const int zir = (zr - z0) & (L - 1);
            if (zir < nza) {
                const int q = zir / ZC;
                *cluster.map_shared_rank(P + kp * ZP + (zir - q * ZC), q) = v[r];
            }
        }
    }
    cluster.sync();

    // 3. IY of plane z: kept modes from P (zero padded), active rows to S1
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int k = col_freq<LG>(col_idx<LG, Sh::NS - 1>(t, r));
        C x = cmk(T(0), T(0));
        if (on13) {
            if (k < ny / 2)
                x = P[k * ZP + col];
            else if (k > L - ny / 2)
                x = P[(k - L + ny) * ZP + col];
        }
        v[r] = x;
    }
    col_stage<C, LG, Sh::NS - 1, true>(v, t, tw);
    col_inverse_from<C, LG, Sh::NS - 2>(buf, v, t, b, tw);
    if (on13) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int y = col_idx<LG, 0>(t, r);
            if (((y - iv.x) & (L - 1)) < iv.y) S1[(int64_t)y * Kx] = v[r];
        }
    }
}

// ---------------------------------------------------------------- launchers
// Batch sizes: at most 8 transforms per block (more blocks for the small
// grids, where the passes are latency-bound), two buffers of (L x (B+1))
// complex within ~64 KB.
static int row_batch(int L, size_t celem) {
    int pb = L <= 128 ? 4 : 8;  // short rows: more, smaller blocks (measured on the 128^3 sphere)
    while (pb > 1 && (2 * (size_t)L * (pb + 1) + L) * celem > 64 * 1024) pb >>= 1;
    return pb;
}
// Column passes: one in-place buffer (L x (B+1)) plus the twiddles; up to 16
// columns per block (128-byte row segments) within ~100 KB of shared memory,
// but no fewer than two blocks per SM while halving B keeps it at >= 8.
static int col_batch(int L, int Kx, size_t celem, int64_t rows_of_blocks) {
    int b = 16;
    if (b > Kx) b = Kx;
    while (b > 1 && ((size_t)L * (b + 1) + L) * celem > 100 * 1024) b >>= 1;
    while (b > 8 && rows_of_blocks * (Kx / b) < 2 * 152) b >>= 1;
    return b;
}

template <typename K> static cudaError_t prep(K kern, size_t sm) {
    if (sm > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return cudaSuccess;
}

// column engine launch: L = 2^lg threads, 8 columns per block
#define SLP_COL_DISPATCH(KERN, T, LGV, NBLK, SM, S)                                                      \
    switch (LGV) {                                                                                       \
        case 5: { cudaError_t e_ = prep(KERN<T, 5>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 5>, NBLK, 32, SM, S, p); }                                     \
        case 6: { cudaError_t e_ = prep(KERN<T, 6>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 6>, NBLK, 64, SM, S, p); }                                     \
        case 7: { cudaError_t e_ = prep(KERN<T, 7>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 7>, NBLK, 128, SM, S, p); }                                    \
        case 8: { cudaError_t e_ = prep(KERN<T, 8>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 8>, NBLK, 256, SM, S, p); }                                    \
        case 9: { cudaError_t e_ = prep(KERN<T, 9>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 9>, NBLK, 512, SM, S, p); }                                    \
        case 10: { cudaError_t e_ = prep(KERN<T, 10>, SM); if (e_ != cudaSuccess) return e_;             \
                   return launch_k(KERN<T, 10>, NBLK, 1024, SM, S, p); }                                 \
    }
#define SLP_COL_DISPATCH2(KERN, KERNL, T, LGV, NBLK, SM, S)                                                      \
    switch (LGV) {                                                                                       \
        case 5: { cudaError_t e_ = prep(KERN<T, 5>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 5>, NBLK, 32, SM, S, p); }                                     \
        case 6: { cudaError_t e_ = prep(KERN<T, 6>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 6>, NBLK, 64, SM, S, p); }                                     \
        case 7: { cudaError_t e_ = prep(KERN<T, 7>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 7>, NBLK, 128, SM, S, p); }                                    \
        case 8: { cudaError_t e_ = prep(KERN<T, 8>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERN<T, 8>, NBLK, 256, SM, S, p); }                                    \
        case 9: { cudaError_t e_ = prep(KERNL<T, 9>, SM); if (e_ != cudaSuccess) return e_;               \
                  return launch_k(KERNL<T, 9>, NBLK, 512, SM, S, p); }                                    \
        case 10: { cudaError_t e_ = prep(KERNL<T, 10>, SM); if (e_ != cudaSuccess) return e_;             \
                   return launch_k(KERNL<T, 10>, NBLK, 1024, SM, S, p); }                                 \
    }
// the engine applies for 32 <= L <= 1024 and at least 8 stored x frequencies
static bool col_engine_ok(const DevPlan &p, int L) { return L >= 32 && L <= 1024 && p.Kx >= CB; }

template <typename T> static cudaError_t fx_t(const DevPlan &p, cudaStream_t s) {
    const size_t ce = 2 * sizeof(T);
    const int PB = row_batch(p.L[0], ce);
    const size_t sm = (2 * (size_t)p.L[0] * (PB + 1) + p.L[0]) * ce;
    cudaError_t e = prep(k_fx<T>, sm);
    if (e != cudaSuccess) return e;
    if (p.n_row_pairs == 0) return cudaSuccess;
    { const cudaError_t le = launch_k(k_fx<T>, dim3((p.n_row_pairs + PB - 1) / PB, p.ks), 256, sm, s, p, PB); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}
template <typename T> static cudaError_t ix_t(const DevPlan &p, cudaStream_t s) {
    // the compile-time inverse pays off for long rows (measured at 1024);
    // short, latency-bound rows keep the runtime kernel
    if (col_engine_ok(p, p.L[0]) && p.L[0] >= 512) {
        if (p.n_row_pairs == 0) return cudaSuccess;
        const size_t sm = ((size_t)p.L[0] * (CB + 1) + p.L[0]) * 2 * sizeof(T);
        const dim3 nb((unsigned)((p.n_row_pairs + CB - 1) / CB), (unsigned)p.ks);
        SLP_COL_DISPATCH(k_ix_s, T, __builtin_ctz(p.L[0]), nb, sm, s)
    }
    const size_t ce = 2 * sizeof(T);
    const int PB = row_batch(p.L[0], ce);
    const size_t sm = (2 * (size_t)p.L[0] * (PB + 1) + p.L[0]) * ce;
    cudaError_t e = prep(k_ix<T>, sm);
    if (e != cudaSuccess) return e;
    if (p.n_row_pairs == 0) return cudaSuccess;
    { const cudaError_t le = launch_k(k_ix<T>, dim3((p.n_row_pairs + PB - 1) / PB, p.ks), 256, sm, s, p, PB); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}
template <typename T> static cudaError_t fy_t(const DevPlan &p, cudaStream_t s) {
    if (col_engine_ok(p, p.L[1])) {
        if (p.nz_act == 0) return cudaSuccess;
        const size_t sm = ((size_t)p.L[1] * (CB + 1) + p.L[1]) * 2 * sizeof(T);
        const dim3 nb((unsigned)(p.nz_act * (p.Kx / CB)), (unsigned)p.ks);
        SLP_COL_DISPATCH2(k_fy_c, k_fy_c_long, T, __builtin_ctz(p.L[1]), nb, sm, s)
    }
    const size_t ce = 2 * sizeof(T);
    const int B = col_batch(p.L[1], p.Kx, ce, p.nz_act);
    const size_t sm = ((size_t)p.L[1] * (B + 1) + p.L[1]) * ce;
    cudaError_t e = prep(k_fy<T>, sm);
    if (e != cudaSuccess) return e;
    if (p.nz_act == 0) return cudaSuccess;
    { const cudaError_t le = launch_k(k_fy<T>, dim3(p.nz_act * (p.Kx / B), p.ks), 256, sm, s, p, B); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}
template <typename T> static cudaError_t iy_t(const DevPlan &p, cudaStream_t s) {
    if (col_engine_ok(p, p.L[1])) {
        if (p.nz_act == 0) return cudaSuccess;
        const size_t sm = ((size_t)p.L[1] * (CB + 1) + p.L[1]) * 2 * sizeof(T);
        const dim3 nb((unsigned)(p.nz_act * (p.Kx / CB)), (unsigned)p.ks);
        SLP_COL_DISPATCH2(k_iy_c, k_iy_c_long, T, __builtin_ctz(p.L[1]), nb, sm, s)
    }
    const size_t ce = 2 * sizeof(T);
    const int B = col_batch(p.L[1], p.Kx, ce, p.nz_act);
    const size_t sm = ((size_t)p.L[1] * (B + 1) + p.L[1]) * ce;
    cudaError_t e = prep(k_iy<T>, sm);
    if (e != cudaSuccess) return e;
    if (p.nz_act == 0) return cudaSuccess;
    { const cudaError_t le = launch_k(k_iy<T>, dim3(p.nz_act * (p.Kx / B), p.ks), 256, sm, s, p, B); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}
template <typename T> static cudaError_t fz_t(const DevPlan &p, cudaStream_t s) {
    if (col_engine_ok(p, p.L[2])) {
        if (p.nz_act == 0) return cudaSuccess;
        const size_t sm = ((size_t)p.L[2] * (CB + 1) + p.L[2]) * 2 * sizeof(T);
        const dim3 nb((unsigned)(p.n[1] * (p.Kx / CB)), (unsigned)p.ks);
        SLP_COL_DISPATCH(k_fz_c, T, __builtin_ctz(p.L[2]), nb, sm, s)
    }
    const size_t ce = 2 * sizeof(T);
    const int B = col_batch(p.L[2], p.Kx, ce, p.n[1]);
    const size_t sm = ((size_t)p.L[2] * (B + 1) + p.L[2]) * ce;
    cudaError_t e = prep(k_fz<T>, sm);
    if (e != cudaSuccess) return e;
    if (p.nz_act == 0) return cudaSuccess;
    { const cudaError_t le = launch_k(k_fz<T>, dim3(p.n[1] * (p.Kx / B), p.ks), 256, sm, s, p, B); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

// shared memory of one CTA of the fused plane passes
static size_t fused_cta_smem(const DevPlan &p, int PB, size_t ce) {
    const size_t xb = (size_t)p.L[0] * (PB / FUSE_CL + 1), pb = (size_t)p.L[1] * (p.Kx / FUSE_CL + 1);
    return (2 * xb + pb + p.L[0] + p.L[1]) * ce;
}

template <typename K> static cudaError_t launch_cluster(K kern, const DevPlan &p, size_t sm, cudaStream_t s) {
    cudaError_t e = prep(kern, sm);
    if (e != cudaSuccess) return e;
    if (p.nz_act == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.nz_act * FUSE_CL, p.ks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = FUSE_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, p, p.fuse_pb);
}
template <typename T> static cudaError_t fxy_t(const DevPlan &p, cudaStream_t s) {
    return launch_cluster(k_fxy<T>, p, fused_cta_smem(p, p.fuse_pb, 2 * sizeof(T)), s);
}
template <typename T> static cudaError_t iyx_t(const DevPlan &p, cudaStream_t s) {
    return launch_cluster(k_iyx<T>, p, fused_cta_smem(p, p.fuse_pb, 2 * sizeof(T)), s);
}

// shared memory of one CTA of the fused column passes: P [ny][ZP], the
// twiddles, G exchange buffers [L][CB + 1]
static size_t yzy_cta_smem(const DevPlan &p, int G, int ZP, size_t ce) {
    const size_t L = (size_t)p.L[1];
    return ((size_t)p.n[1] * ZP + L + (size_t)G * L * (CB + 1)) * ce;
}
template <typename K> static cudaError_t launch_yzy_cluster(K kern, const DevPlan &p, size_t sm, cudaStream_t s) {
    cudaError_t e = prep(kern, sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.Kx * YZY_CL, p.ks);
    cfg.blockDim = dim3(p.yzy_g * p.L[1]);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = YZY_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, p, p.yzy_zc, p.yzy_zp);
}
template <typename T> static cudaError_t yzy_t(const DevPlan &p, cudaStream_t s) {
    if (p.nz_act == 0) return cudaSuccess;
    if (p.yzy_g < 1 || p.yzy_g * p.L[1] > 512 || p.L[1] != p.L[2]) return cudaErrorInvalidConfiguration;
    const size_t sm = yzy_cta_smem(p, p.yzy_g, p.yzy_zp, 2 * sizeof(T));
    switch (__builtin_ctz(p.L[1])) {
        case 5: return launch_yzy_cluster(k_yzy<T, 5>, p, sm, s);
        case 6: return launch_yzy_cluster(k_yzy<T, 6>, p, sm, s);
        case 7: return launch_yzy_cluster(k_yzy<T, 7>, p, sm, s);
        case 8: return launch_yzy_cluster(k_yzy<T, 8>, p, sm, s);
    }
    return cudaErrorInvalidConfiguration;
}
size_t fused_column_smem(const DevPlan &p, int G, int ZP) {
    return yzy_cta_smem(p, G, ZP, 2 * (p.prec == 64 ? sizeof(double) : sizeof(float)));
}
cudaError_t launch_fft_yzy(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? yzy_t<double>(p, s) : yzy_t<float>(p, s); }

size_t fused_plane_smem(const DevPlan &p, int PB) {
    if (PB < FUSE_CL || p.Kx < FUSE_CL) return (size_t)-1;  // not applicable
    return fused_cta_smem(p, PB, 2 * (p.prec == 64 ? sizeof(double) : sizeof(float)));
}
cudaError_t launch_fft_forward_xy(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? fxy_t<double>(p, s) : fxy_t<float>(p, s); }
cudaError_t launch_fft_inverse_yx(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? iyx_t<double>(p, s) : iyx_t<float>(p, s); }

cudaError_t launch_fft_forward_x(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? fx_t<double>(p, s) : fx_t<float>(p, s); }
cudaError_t launch_fft_forward_y(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? fy_t<double>(p, s) : fy_t<float>(p, s); }
cudaError_t launch_fft_z_multiply(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? fz_t<double>(p, s) : fz_t<float>(p, s); }
cudaError_t launch_fft_inverse_y(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? iy_t<double>(p, s) : iy_t<float>(p, s); }
cudaError_t launch_fft_inverse_x(const DevPlan &p, cudaStream_t s) { return p.prec == 64 ? ix_t<double>(p, s) : ix_t<float>(p, s); }

}  // namespace slp
