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


def poly_kr(S, law):
    """The polynomial relative permeabilities of one medium, law = (kind,
    a_w, n_w, a_n, b_n, c_n): k_rw = a_w S^n_w and k_rn = a_n (1 - b_n S)^2
    (1 - c_n S^2) up to the first root of either factor, 0 beyond (S clamped
    to [0, 1])."""
    _, aw, nw, an, bn, cn = law
    S = np.clip(S, 0.0, 1.0)
    r, q = 1.0 - bn * S, 1.0 - cn * S * S
    return aw * S ** nw, np.where((r > 0) & (q > 0), an * r * r * q, 0.0)


def extended_buckley_leverett_sw(x, t, q, phi, mu_w, mu_n, law1, law2, x_if, ns=400001):
    """Water saturation of the extended Buckley-Leverett problem (two media
    meeting at x_if, no gravity, no capillarity, water injected at S_w = 1 and
    total Darcy velocity q into S_w = 0), by characteristics.  Both fractional
    flows f_m = lam_w / (lam_w + lam_n) increase with S, so information moves
    downstream only:
      medium 1: the textbook solution, Welge front S_f1, x = q t f1'(S) / phi;
      at x_if the water flux is continuous, f2(S_2) = f1(S_1) (the saturation
      jumps there), and the front arrives at t_a = x_if phi / (q f1'(S_f1));
      medium 2: from (x_if, t_a) a centred wave, Welge front S_f2 of f2 and a
      fan x = x_if + q (t - t_a) f2'(S) / phi up to S_2(t_a); behind it the
      characteristics of the inflow, leaving x_if at tau with S_2(tau) (the
      interface value of medium 1 at tau), x = x_if + q (t - tau) f2'(S_2) /
      phi.  These neither cross nor leave gaps when f2' decreases above S_f2,
      which is checked."""
    S = np.linspace(0.0, 1.0, ns)

    def frac(law):
        kw, kn = poly_kr(S, law)
        lw, ln = kw / mu_w, kn / mu_n
        return lw / (lw + ln)

    F1, F2 = frac(law1), frac(law2)
    d1, d2 = np.gradient(F1, S), np.gradient(F2, S)
    k1 = int(np.argmax(np.where(S > 0, F1 / np.where(S > 0, S, 1.0), 0.0)))
    k2 = int(np.argmax(np.where(S > 0, F2 / np.where(S > 0, S, 1.0), 0.0)))
    assert np.all(np.diff(d2[k2:]) <= 1e-9 * max(1.0, d2.max())), "f2' must decrease above the front"
    x = np.asarray(x, dtype=float)
    out = np.zeros_like(x)
    # medium 1
    xs1 = q * t * d1[k1:] / phi
    a = x <= x_if
    xa = x[a]
    o = np.zeros_like(xa)
    beh = xa <= xs1[0]
    o[beh] = np.interp(xa[beh], xs1[::-1], S[k1:][::-1])
    out[a] = o
    ta = x_if * phi / (q * d1[k1])
    if t <= ta:
        return out
    # medium 2: inflow characteristics (S_1 at the interface at time tau)
    pos = d1[k1:] > 0
    s1 = S[k1:][pos]
    tau = x_if * phi / (q * d1[k1:][pos])
    keep = tau <= t
    s1, tau = s1[keep], tau[keep]
    s2 = np.interp(np.interp(s1, S, F1), F2, S)
    xb = x_if + q * (t - tau) * np.interp(s2, S, d2) / phi
    s2a = np.interp(F1[k1], F2, S)
    fan = (S >= S[k2]) & (S <= s2a)
    xf = x_if + q * (t - ta) * d2[fan] / phi
    X = np.concatenate((xf, xb))
    SS = np.concatenate((S[fan], s2))
    order = np.argsort(X, kind="stable")
    X, SS = X[order], SS[order]
    b = ~a
    xb_ = x[b]
    o = np.zeros_like(xb_)
    inside = xb_ <= X[-1]
    o[inside] = np.interp(xb_[inside], X, SS)
    out[b] = o
    return out
