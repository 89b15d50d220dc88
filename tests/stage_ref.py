"""Plain numpy references of the individual kernels, for kernel unit tests.

These mirror one stage each (spread, the pruned FFT passes, gather, near
field) on the plan's own sorted data, so a kernel can be checked in
isolation.  They are not the oracle: end-to-end parity is judged against
``oracle`` (the direct sum), which shares nothing with the library.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc

B_KB = np.pi * 1.5  # b = pi (2 - 1/alpha), alpha = 2


def kb_window(d, m):
    """Normalised Kaiser-Bessel window in grid units (psi(0) = 1), |d| <= m."""
    beta = B_KB * m
    s2 = 1.0 - (np.asarray(d, float) / m) ** 2
    s = np.sqrt(np.clip(s2, 0.0, None))
    with np.errstate(invalid="ignore", divide="ignore"):
        v = np.where(s * beta > 1e-8, np.sinh(beta * s) / np.where(s > 0, s, 1.0), beta)
    return np.where(s2 >= 0, v / np.sinh(beta), 0.0)


def unpack(grid4):
    g = grid4.reshape(-1, 4)
    packed = g[:, 3].astype(np.int64)
    c = np.stack([packed & 1023, (packed >> 10) & 1023, (packed >> 20) & 1023], axis=1)
    return g[:, :3], c


def spread(grid4, q, L, m):
    f, c = unpack(grid4)
    Lx, Ly, Lz = L
    A = np.zeros(Lz * Ly * Lx)
    W = 2 * m
    idx = []
    wts = []
    for ax in range(3):
        i = np.arange(W)
        r = (c[:, ax:ax + 1] - m + 1 + i[None, :]) % L[ax]
        w = kb_window(f[:, ax:ax + 1] + (m - 1 - i[None, :]), m)
        idx.append(r)
        wts.append(w)
    for iz in range(W):
        for iy in range(W):
            base = (idx[2][:, iz] * Ly + idx[1][:, iy]) * Lx
            wyz = q * wts[2][:, iz] * wts[1][:, iy]
            for ix in range(W):
                A += np.bincount(base + idx[0][:, ix], wyz * wts[0][:, ix], minlength=A.size)
    return A.reshape(Lz, Ly, Lx)


def gather(grid4, G, L, m):
    f, c = unpack(grid4)
    Lx, Ly, Lz = L
    Gf = G.reshape(-1)
    W = 2 * m
    idx = []
    wts = []
    for ax in range(3):
        i = np.arange(W)
        idx.append((c[:, ax:ax + 1] - m + 1 + i[None, :]) % L[ax])
        wts.append(kb_window(f[:, ax:ax + 1] + (m - 1 - i[None, :]), m))
    out = np.zeros(f.shape[0])
    for iz in range(W):
        for iy in range(W):
            base = (idx[2][:, iz] * Ly + idx[1][:, iy]) * Lx
            wyz = wts[2][:, iz] * wts[1][:, iy]
            for ix in range(W):
                out += Gf[base + idx[0][:, ix]] * wyz * wts[0][:, ix]
    return out


def fft_x(A, Kx):
    return np.fft.rfft(A, axis=2)[:, :, :Kx]


def _ysel(F, ny, Ly, axis):
    out_shape = list(F.shape)
    out_shape[axis] = ny
    out = np.zeros(out_shape, complex)
    for kp in range(ny):
        if kp < ny // 2:
            src = kp
        elif kp > ny // 2:
            src = Ly - ny + kp
        else:
            continue
        sl_o = [slice(None)] * F.ndim
        sl_i = [slice(None)] * F.ndim
        sl_o[axis] = kp
        sl_i[axis] = src
        out[tuple(sl_o)] = F[tuple(sl_i)]
    return out


def fft_y(S1, ny):
    Ly = S1.shape[1]
    return _ysel(np.fft.fft(S1, axis=1), ny, Ly, 1)


def expand_dtab(dtab, n):
    nx, ny, nz = n
    Kx, hy, hz = nx // 2, ny // 2, nz // 2
    D = dtab.reshape(hz, hy, Kx)
    return D


def fft_z_multiply(S2, dtab, n, Lz):
    nx, ny, nz = n
    D = expand_dtab(dtab, n)
    F = np.fft.fft(S2, axis=0)
    kz = np.fft.fftfreq(Lz, 1.0 / Lz).astype(int)
    ky = np.array([kp if kp < ny // 2 else kp - ny for kp in range(ny)])
    out = np.zeros_like(F)
    for iz in range(Lz):
        if abs(kz[iz]) >= nz // 2:
            continue
        for iy in range(ny):
            if iy == ny // 2:
                continue
            out[iz, iy, :] = F[iz, iy, :] * D[abs(kz[iz]), abs(ky[iy]), :]
    return np.fft.ifft(out, axis=0) * Lz


def ifft_y(S2, Ly):
    Lz, ny, Kx = S2.shape
    F = np.zeros((Lz, Ly, Kx), complex)
    for kp in range(ny):
        if kp < ny // 2:
            F[:, kp] = S2[:, kp]
        elif kp > ny // 2:
            F[:, Ly - ny + kp] = S2[:, kp]
    return np.fft.ifft(F, axis=1) * Ly


def ifft_x(S1, Lx):
    Lz, Ly, Kx = S1.shape
    X = np.zeros((Lz, Ly, Lx // 2 + 1), complex)
    X[:, :, :Kx] = S1
    X[:, :, 0] = X[:, :, 0].real
    return np.fft.irfft(X, n=Lx, axis=2) * Lx


def _near(tgt_pts, src_pts, q, eps, kern):
    from scipy.spatial import cKDTree
    tree = cKDTree(src_pts)
    lists = tree.query_ball_point(tgt_pts, eps)
    out = np.zeros(tgt_pts.shape[0])
    for i, lst in enumerate(lists):
        if not lst:
            continue
        lst = np.asarray(lst)
        r = np.linalg.norm(tgt_pts[i] - src_pts[lst], axis=1)
        keep = r < eps
        out[i] = np.sum(q[lst][keep] * kern(r[keep])) / (4 * np.pi)
    return out


def near_radial(tgt_pts, src_pts, q, eps, sigma_g):
    """Near-field part with the radial kernel erfc(r / (s sqrt 2)) / (4 pi r)."""
    return _near(tgt_pts, src_pts, q, eps, lambda r: erfc(r / (sigma_g * np.sqrt(2))) / r)


def near_expsum(tgt_pts, src_pts, q, eps, w, g, P):
    """Near-field part with the exp-sum kernel (1/r - sum_k w_k exp(-g_k (r/P)^2) / P) / (4 pi),
    (w, g) the terms in torus units."""
    def kern(r):
        u = r / P
        return 1.0 / r - (w[None, :] * np.exp(-g[None, :] * u[:, None] ** 2)).sum(axis=1) / P
    return _near(tgt_pts, src_pts, q, eps, kern)
