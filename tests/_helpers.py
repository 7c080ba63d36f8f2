"""Test-side helpers: format conversions and textbook dense constructions.

Nothing here is the method's arithmetic; these turn the stencil storage into
dense matrices so that library routines (numpy matmul / solve) can serve as
independent references.
"""
import numpy as np


def offsets(dim):
    if dim == 3:
        return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return [(dx, dy, 0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def stencil_to_dense(dim, n, A):
    """[nv, nb, 4] stencil blocks -> dense (2nv x 2nv); unknown 2v+alpha."""
    nx, ny, nz = n
    nv = nx * ny * nz
    D = np.zeros((2 * nv, 2 * nv))
    offs = offsets(dim)
    for v in range(nv):
        i, j, k = v % nx, (v // nx) % ny, v // (nx * ny)
        for b, (dx, dy, dz) in enumerate(offs):
            ii, jj, kk = i + dx, j + dy, k + dz
            if not (0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz):
                continue
            w = ii + nx * (jj + ny * kk)
            D[2 * v:2 * v + 2, 2 * w:2 * w + 2] = A[v, b].reshape(2, 2)
    return D


def dense_to_stencil(dim, n, D):
    nx, ny, nz = n
    nv = nx * ny * nz
    offs = offsets(dim)
    A = np.zeros((nv, len(offs), 4))
    for v in range(nv):
        i, j, k = v % nx, (v // nx) % ny, v // (nx * ny)
        for b, (dx, dy, dz) in enumerate(offs):
            ii, jj, kk = i + dx, j + dy, k + dz
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                w = ii + nx * (jj + ny * kk)
                A[v, b] = D[2 * v:2 * v + 2, 2 * w:2 * w + 2].ravel()
    return A


def coarse_dims(dim, n):
    return tuple(((t - 1) // 2 + 1) if ax < dim else 1 for ax, t in enumerate(n))


def dense_prolongation(dim, nf, nc, dmf=None, dmc=None):
    """Textbook (bi/tri)linear interpolation on a vertex-nested grid, per
    component; component 0 rows/columns dropped at Dirichlet vertices."""
    nvf = int(np.prod(nf))
    nvc = int(np.prod(nc))
    P = np.zeros((2 * nvf, 2 * nvc))
    for vf in range(nvf):
        f = (vf % nf[0], (vf // nf[0]) % nf[1], vf // (nf[0] * nf[1]))
        # 1D interpolation weights per axis
        per_axis = []
        for ax in range(3):
            if ax >= dim:
                per_axis.append([(0, 1.0)])
            elif f[ax] % 2 == 0:
                per_axis.append([(f[ax] // 2, 1.0)])
            else:
                per_axis.append([((f[ax] - 1) // 2, 0.5), ((f[ax] + 1) // 2, 0.5)])
        for I, wi in per_axis[0]:
            for J, wj in per_axis[1]:
                for K, wk in per_axis[2]:
                    vc = I + nc[0] * (J + nc[1] * K)
                    w = wi * wj * wk
                    P[2 * vf + 1, 2 * vc + 1] = w
                    masked = (dmf is not None and dmf[vf]) or (dmc is not None and dmc[vc])
                    P[2 * vf, 2 * vc] = 0.0 if masked else w
    return P


def colour(dim, n):
    nx, ny, nz = n
    v = np.arange(nx * ny * nz)
    i, j, k = v % nx, (v // nx) % ny, v // (nx * ny)
    return (i & 1) | ((j & 1) << 1) | ((k & 1) << 2)


def buckley_leverett_sw(x, t, q, phi, mu_w, mu_n, lam=2.0):
    """Textbook Buckley-Leverett solution (no gravity, no capillarity) for water
    injected at total Darcy velocity q into a medium at S_w = 0 (S_wr = S_nr =
    0): fractional flow f = lam_w / (lam_w + lam_n) with the Brooks-Corey
    relative permeabilities k_rw = S^((2+3lam)/lam), k_rn = (1-S)^2 (1 -
    S^((2+lam)/lam)); the front saturation S_f is Welge's tangent point,
    max f(S)/S; behind the front x(S) = q t f'(S) / phi (S_f <= S <= 1)."""
    S = np.linspace(0.0, 1.0, 200001)
    krw = S ** ((2 + 3 * lam) / lam)
    krn = (1 - S) ** 2 * (1 - S ** ((2 + lam) / lam))
    f = (krw / mu_w) / (krw / mu_w + krn / mu_n)
    df = np.gradient(f, S)
    ratio = np.where(S > 0, f / np.where(S > 0, S, 1.0), 0.0)
    k = int(np.argmax(ratio))
    Sf = S[k]
    xs = q * t * df[k:] / phi           # decreasing from the front to 0 at S = 1
    Ss = S[k:]
    x = np.asarray(x, dtype=float)
    out = np.zeros_like(x)
    behind = x <= xs[0]
    # x(S) is monotone decreasing on [S_f, 1]: interpolate S as a function of x
    out[behind] = np.interp(x[behind], xs[::-1], Ss[::-1])
    return out, Sf, xs[0]


def lp_error_1d(xv, sv, exact, p, samples=40):
    """(integral over [x0, x_end] of |s_h - s|^p dx)^(1/p) with s_h the piecewise
    linear interpolant of vertex values sv at xv and s = exact(x), by the
    midpoint rule on `samples` points per element."""
    tot = 0.0
    for a in range(len(xv) - 1):
        h = xv[a + 1] - xv[a]
        xm = xv[a] + (np.arange(samples) + 0.5) / samples * h
        sh = sv[a] + (sv[a + 1] - sv[a]) * (xm - xv[a]) / h
        tot += (np.abs(sh - exact(xm)) ** p).sum() * h / samples
    return tot ** (1.0 / p)
