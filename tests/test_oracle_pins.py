"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test fixes one part of the oracle by something other than the oracle's
own formula: a value printed in the paper, a closed form, an invariant, a
library routine on a dense matrix, or brute force.  CPU only.
"""
import os

import numpy as np
import pytest

from paper_2506_04763_gb300 import inputs as I
from tests import _helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = v
    return out


def _poisson_problem(dim, nv, K=1e-10):
    """Constant K, uniform p_d, S_n = 0, no gravity: the p-block of J is the
    VCFVM Laplacian with coefficient K rho_w / mu_w."""
    p = I.random_problem(dim, nv, 3, gravity=False)
    p["K"][:] = K
    p["pd"][:] = 755.0
    p["u0"][0::2] = I.P_TOP
    p["u0"][1::2] = 0.0
    return p


# ---------------------------------------------------------------- P9 / grid
def test_dof_counts_match_paper():
    """Sec. 5 scaling tables: DoF = 2 x (elements+1 per axis) vertices."""
    with open(os.path.join(GOLDEN, "dof_counts.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for mesh, dof in rows:
        el = [int(t) for t in mesh.split("x")]
        nv = int(np.prod([e + 1 for e in el]))
        assert 2 * nv == int(dof)


# ---------------------------------------------------------------- laws
def test_brooks_corey_special_values(oracle):
    m = oracle.Model(I.lens_square_2d())
    kr = oracle.brooks_corey(m, 1.0)
    assert kr[0] == 1.0 and kr[2] == 0.0 and kr[4] == 1.0     # krw(1)=1, krn(1)=0, J(1)=1
    kr = oracle.brooks_corey(m, 0.0)
    assert kr[0] == 0.0 and kr[2] == 1.0                        # krw(0)=0, krn(0)=1
    # clamps outside [0,1] for k_r, linear continuation of J
    for s in (-0.3, 1.4):
        kr = oracle.brooks_corey(m, s)
        assert kr[1] == 0.0 and kr[3] == 0.0
    assert oracle.brooks_corey(m, 1.4)[4] == pytest.approx(1.0 - 0.5 * 0.4)


def test_brooks_corey_lambda2_path_equals_general_pow_path(oracle):
    """The sqrt/integer-power special case for lambda=2 agrees with the general
    pow() path evaluated at lambda = 2 + 1e-12."""
    p = I.lens_square_2d()
    m2 = oracle.Model(p)
    p2 = dict(p)
    p2["lam"] = 2.0 + 1e-12
    mg = oracle.Model(p2)
    for s in np.linspace(0.005, 1.2, 41):
        a = oracle.brooks_corey(m2, s)
        b = oracle.brooks_corey(mg, s)
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)


def test_brooks_corey_derivatives_by_finite_differences(oracle):
    m = oracle.Model(I.lens_square_2d())
    for s in np.linspace(0.02, 0.98, 25):
        d = 1e-6
        f0 = oracle.brooks_corey(m, s)
        fp = oracle.brooks_corey(m, s + d)
        fm = oracle.brooks_corey(m, s - d)
        for val, der in ((0, 1), (2, 3), (4, 5)):
            fd = (fp[val] - fm[val]) / (2 * d)
            assert fd == pytest.approx(f0[der], rel=1e-6, abs=1e-9)
    # J is C^1 at the continuation points 0.01 and 1
    for s in (0.01, 1.0):
        lo = oracle.brooks_corey(m, s - 1e-9)
        hi = oracle.brooks_corey(m, s + 1e-9)
        assert abs(lo[4] - hi[4]) <= 1.01 * 2e-9 * abs(hi[5])   # no jump in J
        assert lo[5] == pytest.approx(hi[5], rel=1e-5)           # no jump in J'


def test_case4_threshold_saturation(oracle):
    """Paper, Case 4: S_w* = 0.7778 at the layer-2/layer-3 interface.  The
    oracle's S hat (Eq. hSw) must switch from the capped branch (S_e hat = 1,
    NAPL blocked) to the open branch exactly at that wetting saturation."""
    g = _read_golden("case4_threshold.txt")
    p = I.lens_square_2d()
    p["S_wr"], p["S_nr"], p["lam"] = float(g["S_wr"]), float(g["S_nr"]), float(g["lambda"])
    m = oracle.Model(p)
    pd2 = float(g["pd_coef"]) * float(g["K2"]) ** float(g["pd_exp"])
    pd3 = float(g["pd_coef"]) * float(g["K3"]) ** float(g["pd_exp"])
    den = 1.0 - p["S_wr"] - p["S_nr"]

    def capped(Sw):
        return oracle.shat(m, (Sw - p["S_wr"]) / den, pd3, pd2)[0] >= 1.0

    lo, hi = 0.3, 0.9 - 1e-9   # open at lo, capped at hi
    assert not capped(lo) and capped(hi)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if capped(mid):
            hi = mid
        else:
            lo = mid
    assert round(hi, int(g["digits"])) == float(g["S_w_star"])
    # continuity of S hat at the cap
    s_star = (hi - p["S_wr"]) / den
    assert oracle.shat(m, s_star - 1e-12, pd3, pd2)[0] == pytest.approx(1.0, abs=1e-9)


def test_shat_branches(oracle):
    m = oracle.Model(I.lens_square_2d())
    assert list(oracle.shat(m, 0.4, 755.0, 755.0)) == [0.4, 1.0]      # case 1
    r2 = (1163.0 / 755.0) ** 2
    out = oracle.shat(m, 0.3, 1163.0, 755.0)                           # case 3
    assert out[0] == pytest.approx(r2 * 0.3) and out[1] == pytest.approx(r2)
    assert list(oracle.shat(m, 0.9, 1163.0, 755.0)) == [1.0, 0.0]      # case 2
    # sand/lens threshold of the synthetic workloads: S_e* = (755/1163)^2
    se_star = (755.0 / 1163.0) ** 2
    assert oracle.shat(m, se_star * (1 - 1e-9), 1163.0, 755.0)[0] < 1.0
    assert oracle.shat(m, se_star * (1 + 1e-9), 1163.0, 755.0)[0] == 1.0


# ---------------------------------------------------------------- P1 stencil
@pytest.mark.parametrize("dim,nv,expect", [
    (2, (9, 9), {(0, 0, 0): -3.0, (1, 0, 0): 0.5, (0, 1, 0): 0.5, (1, 1, 0): 0.25}),
    (3, (9, 9, 9), {(0, 0, 0): -27 / 8, (1, 0, 0): 3 / 16, (1, 1, 0): 5 / 32, (1, 1, 1): 3 / 64}),
])
def test_p1_laplacian_stencil_closed_form(oracle, dim, nv, expect):
    """Constant K, S_n = 0, g = 0: the (w, p_w) entries of J are the VCFVM
    Laplacian stencil of bilinear/trilinear elements with midpoint SCVF
    quadrature: 2D centre -3, face 1/2, corner 1/4; 3D (times h) centre
    -27/8, face 3/16, edge 5/32, corner 3/64 (per unit K rho_w/mu_w)."""
    K = 1e-10
    p = _poisson_problem(dim, nv, K)
    p["dir"][:] = 0
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    scale = K * p["rho_w"] / p["mu_w"] * (p["h"][0] if dim == 3 else 1.0)
    offs = H.offsets(dim)
    c = tuple(t // 2 for t in m.n)
    v = c[0] + m.n[0] * (c[1] + m.n[1] * c[2])
    for b, off in enumerate(offs):
        key = tuple(sorted(np.abs(off), reverse=True))
        key = (key[0], key[1], key[2] if dim == 3 else 0) if dim == 3 else (key[0], key[1], 0)
        assert J[v, b, 0] / scale == pytest.approx(expect[key], rel=1e-12, abs=1e-14)
        assert J[v, b, 2] == 0.0          # k_rn(S_e = 1) = 0
    # symmetric, zero row and column sums
    D = H.stencil_to_dense(dim, m.n, J)[0::2, 0::2]
    np.testing.assert_allclose(D, D.T, atol=1e-12 * np.abs(D).max())
    assert np.abs(D.sum(axis=1)).max() <= 1e-13 * np.abs(D).max()
    assert np.abs(F).max() == 0.0


# ---------------------------------------------------------------- P3 exact J
@pytest.mark.parametrize("scheme,laws", [(0, False), (2, False), (0, True)])
@pytest.mark.parametrize("dim,nv,seed", [(2, (7, 6), 11), (3, (5, 4, 5), 12)])
def test_p3_jacobian_equals_finite_differences(oracle, dim, nv, seed, scheme, laws):
    """J = F_u exactly (Sec. 4): central differences of the oracle's own F,
    entry by entry; columns where one-sided differences disagree (a kink or an
    upwind switch inside the step) are skipped.  scheme 2: Darcy-velocity
    upwinding of the water flux; laws: each cell with one of Brooks-Corey and
    the two polynomial laws of Case 2."""
    p = I.random_problem(dim, nv, seed)
    if laws:
        p = I.mixed_kr_laws(p, seed)
    p["scheme"] = scheme
    m = oracle.Model(p)
    u = p["u0"].copy()
    F0, J, md = oracle.assemble(m, u)
    Jd = H.stencil_to_dense(dim, m.n, J)
    checked = skipped = 0
    for col in range(2 * m.nv):
        d = (1e-7 * 1e5) if col % 2 == 0 else 1e-7
        up, um = u.copy(), u.copy()
        up[col] += d
        um[col] -= d
        Fp = oracle.assemble(m, up, jacobian=False)[0]
        Fm = oracle.assemble(m, um, jacobian=False)[0]
        fwd, bwd = (Fp - F0) / d, (F0 - Fm) / d
        cen = (Fp - Fm) / (2 * d)
        scale = np.abs(Jd[:, col]).max() + 1e-300
        if np.abs(fwd - bwd).max() > 1e-3 * scale:
            skipped += 1
            continue
        checked += 1
        assert np.abs(cen - Jd[:, col]).max() <= 1e-6 * scale
    assert checked > 0.9 * (checked + skipped)


# ---------------------------------------------------------------- P4 conservation
@pytest.mark.parametrize("scheme", [0, 2])
@pytest.mark.parametrize("dim,nv", [(2, (9, 7)), (3, (5, 6, 5))])
def test_p4_discrete_conservation(oracle, dim, nv, scheme):
    """Without Dirichlet rows: sum_i F_alpha,i = sum_i q_alpha,i (every face
    flux leaves one control volume and enters its neighbour), and every column
    of J sums to zero."""
    p = I.random_problem(dim, nv, 5, stress=True, dirichlet=False)
    p["scheme"] = scheme
    rng = np.random.default_rng(9)
    p["q_in"] = rng.normal(0, 1e-6, 2 * int(np.prod(p["n"])))
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    p0 = dict(p)
    p0["q_in"] = None
    Fnoq = oracle.assemble(oracle.Model(p0), p["u0"], jacobian=False)[0]
    flux_scale = np.abs(Fnoq).sum()
    for a in (0, 1):
        assert abs(F[a::2].sum() - p["q_in"][a::2].sum()) <= 1e-13 * flux_scale
    D = H.stencil_to_dense(dim, m.n, J)
    assert np.abs(D.sum(axis=0)).max() <= 1e-13 * np.abs(D).max()


# ---------------------------------------------------------------- P5 equilibrium
@pytest.mark.parametrize("scheme", [0, 3])
@pytest.mark.parametrize("dim,nv", [(2, (17, 17)), (3, (9, 9, 9))])
def test_p5_hydrostatic_equilibrium(oracle, dim, nv, scheme):
    """Exact hydrostatic p_w with S_n = 0 in heterogeneous K and p_d: F = 0 up
    to rounding, and a LIMEX step leaves the state unchanged."""
    p = I.random_problem(dim, nv, 21)
    n, h = p["n"], p["h"]
    nvx = int(np.prod(n))
    v = np.arange(nvx)
    vert = ((v // n[0]) % n[1]) * h[1] if dim == 2 else (v // (n[0] * n[1])) * h[2]
    u = np.zeros(2 * nvx)
    u[0::2] = I.P_TOP + p["rho_w"] * I.GRAV * (1.0 - vert)
    u[1::2] = 0.0
    p["u0"] = u
    p["scheme"] = scheme
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, u)
    flux = p["K"].max() * p["rho_w"] ** 2 * I.GRAV / p["mu_w"] * h[0] ** (dim - 1)
    assert np.abs(F).max() <= 1e-11 * flux
    u1, info = oracle.limex_step(m, u, 10.0, kappa=3, nlevels=3, rtol=1e-12)
    assert info["status"] == 0
    np.testing.assert_allclose(u1[0::2], u[0::2], rtol=1e-12)
    assert np.abs(u1[1::2]).max() <= 1e-12


def test_p5_no_gravity_uniform_saturation_is_stationary(oracle):
    p = I.random_problem(2, (9, 9), 4, gravity=False)
    p["pd"][:] = 755.0
    p["u0"][0::2] = I.P_TOP
    p["u0"][1::2] = 0.3
    m = oracle.Model(p)
    F = oracle.assemble(m, p["u0"], jacobian=False)[0]
    assert np.abs(F).max() <= 1e-20


# ---------------------------------------------------------------- algebra
def test_spmv_and_make_A_match_dense(oracle):
    p = I.random_problem(3, (5, 4, 6), 8)
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    A = oracle.make_A(J, md, 0.37)
    Md = np.zeros((2 * m.nv, 2 * m.nv))
    for v in range(m.nv):
        Md[2 * v, 2 * v + 1] = md[v, 0]
        Md[2 * v + 1, 2 * v + 1] = md[v, 1]
    Ad = 0.37 * Md - H.stencil_to_dense(3, m.n, J)
    np.testing.assert_allclose(H.stencil_to_dense(3, m.n, A), Ad, rtol=0, atol=1e-15 * np.abs(Ad).max())
    x = np.random.default_rng(1).standard_normal(2 * m.nv)
    np.testing.assert_allclose(oracle.spmv(3, m.n, A, x), Ad @ x, rtol=1e-12, atol=1e-14 * np.abs(Ad @ x).max())


def test_dense_lu_matches_numpy(oracle):
    rng = np.random.default_rng(2)
    for N in (1, 5, 50):
        M = rng.standard_normal((N, N)) + np.diag(rng.uniform(0, 0.1, N))
        b = rng.standard_normal(N)
        np.testing.assert_allclose(oracle.lu_solve_dense(M, b), np.linalg.solve(M, b), rtol=1e-10)


def test_transfer_operators(oracle):
    """Prolongation = textbook trilinear interpolation (dense reference), it
    reproduces linear functions, and restriction is its exact transpose."""
    dim, nf = 3, (9, 5, 7)
    nc = H.coarse_dims(dim, nf)
    rng = np.random.default_rng(3)
    dmf = (rng.uniform(size=int(np.prod(nf))) < 0.2).astype(np.uint8)
    dmc = np.zeros(int(np.prod(nc)), np.uint8)
    for vc in range(len(dmc)):
        I_, J_, K_ = vc % nc[0], (vc // nc[0]) % nc[1], vc // (nc[0] * nc[1])
        dmc[vc] = dmf[2 * I_ + nf[0] * (2 * J_ + nf[1] * 2 * K_)]
    P = H.dense_prolongation(dim, nf, nc, dmf, dmc)
    xc = rng.standard_normal(P.shape[1])
    xf = rng.standard_normal(P.shape[0])
    np.testing.assert_allclose(oracle.prolong_add(dim, nf, dmf, nc, dmc, xc, xf), xf + P @ xc, rtol=1e-14, atol=1e-14)
    rf = rng.standard_normal(P.shape[0])
    np.testing.assert_allclose(oracle.restrict(dim, nf, dmf, nc, dmc, rf), P.T @ rf, rtol=1e-14, atol=1e-14)
    # linear reproduction (no mask)
    z = np.zeros(int(np.prod(nf)), np.uint8)
    zc = np.zeros(int(np.prod(nc)), np.uint8)
    cv = np.arange(int(np.prod(nc)))
    fc = np.arange(int(np.prod(nf)))
    lin_c = np.zeros(2 * len(cv))
    lin_c[1::2] = 2 * (cv % nc[0]) + 3 * 2 * ((cv // nc[0]) % nc[1]) - 2 * (cv // (nc[0] * nc[1]))
    lin_f = 1 * (fc % nf[0]) + 3 * ((fc // nf[0]) % nf[1]) - 1 * (fc // (nf[0] * nf[1]))
    out = oracle.prolong_add(dim, nf, z, nc, zc, lin_c, np.zeros(2 * len(fc)))
    np.testing.assert_allclose(out[1::2], lin_f, atol=1e-12)


@pytest.mark.parametrize("dim,nf", [(2, (9, 7)), (3, (5, 7, 5))])
def test_galerkin_equals_dense_PtAP(oracle, dim, nf):
    p = I.random_problem(dim, nf if dim == 3 else nf, 6)
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    A = oracle.make_A(J, md, 0.1)
    nc = H.coarse_dims(dim, m.n)
    dmf = p["dir"]
    dmc = np.array([dmf[2 * (v % nc[0]) + m.n[0] * (2 * ((v // nc[0]) % nc[1]) + m.n[1] * 2 * (v // (nc[0] * nc[1])))]
                    for v in range(int(np.prod(nc)))], np.uint8)
    P = H.dense_prolongation(dim, m.n, nc, dmf, dmc)
    Ac_dense = P.T @ H.stencil_to_dense(dim, m.n, A) @ P
    for vc in np.nonzero(dmc)[0]:
        Ac_dense[2 * vc, 2 * vc] = 1.0
    Ac = oracle.galerkin(dim, m.n, dmf, A, nc, dmc)
    np.testing.assert_allclose(H.stencil_to_dense(dim, nc, Ac), Ac_dense, rtol=0, atol=1e-13 * np.abs(Ac_dense).max())
    # Galerkin of the 3^d stencil stays within the 3^d stencil
    assert np.allclose(H.dense_to_stencil(dim, nc, Ac_dense), Ac, atol=1e-13 * np.abs(Ac_dense).max())


def test_smoothers_match_dense_formulas(oracle):
    """Jacobi: x + w D^-1 (b - A x).  Forward multicolour GS: one sweep equals
    solving (D + L) x_new = b - U x_old with L/U the couplings to earlier/later
    colours in colour order (numpy dense solve)."""
    dim = 3
    p = I.random_problem(dim, (5, 5, 4), 7)
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    A = oracle.make_A(J, md, 0.1)
    Ad = H.stencil_to_dense(dim, m.n, A)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(2 * m.nv)
    x = rng.standard_normal(2 * m.nv)
    Dinv = np.zeros_like(Ad)
    for v in range(m.nv):
        Dinv[2 * v:2 * v + 2, 2 * v:2 * v + 2] = np.linalg.inv(Ad[2 * v:2 * v + 2, 2 * v:2 * v + 2])
    ref = x + 0.8 * Dinv @ (b - Ad @ x)
    np.testing.assert_allclose(oracle.jacobi(dim, m.n, A, b, x, 0.8), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    col = np.repeat(H.colour(dim, m.n), 2)
    for forward in (True, False):
        order = col if forward else (7 - col)
        lower = order[:, None] > order[None, :]
        same_v = np.kron(np.eye(m.nv), np.ones((2, 2))).astype(bool)
        DL = np.where(lower | same_v, Ad, 0.0)
        U = np.where(~(lower | same_v), Ad, 0.0)
        ref = np.linalg.solve(DL, b - U @ x)
        got = oracle.gs_sweep(dim, m.n, A, b, x, forward=forward)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


# ---------------------------------------------------------------- P6 / P7 solver
@pytest.mark.parametrize("dim,nv,smoother", [(2, (9, 9), 0), (3, (5, 5, 5), 1), (3, (9, 9, 9), 0)])
def test_p6_bicgstab_gmg_matches_dense_solve(oracle, dim, nv, smoother):
    p = I.random_problem(dim, nv, 13)
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    A = oracle.make_A(J, md, 0.1)
    g = oracle.GMG(dim, m.n, A, p["dir"], 3, smoother=smoother)
    x, info = oracle.bicgstab(dim, m.n, A, g, F, rtol=1e-14, maxit=100)
    Ad = H.stencil_to_dense(dim, m.n, A)
    xr = np.linalg.solve(Ad, F)
    assert info["status"] == 0
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()


@pytest.mark.parametrize("dim,nv,levels", [(2, (33, 33), 4), (3, (17, 17, 17), 4)])
@pytest.mark.parametrize("smoother", [0, 1])
def test_p7_gmg_convergence_factor_poisson(oracle, dim, nv, levels, smoother):
    """V(2,2) on the constant-coefficient VCFVM Laplacian: asymptotic factor
    <= 0.15 (local Fourier analysis gives ~0.05-0.1 for these smoothers)."""
    p = _poisson_problem(dim, nv)
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    A = oracle.make_A(J, md, 0.1)
    g = oracle.GMG(dim, m.n, A, p["dir"], levels, smoother=smoother)
    assert g.nlevels == levels
    rng = np.random.default_rng(0)
    x = rng.standard_normal(2 * m.nv)
    x[0::2][p["dir"].astype(bool)] = 0.0
    rs = []
    for _ in range(20):
        r = -oracle.spmv(dim, m.n, A, x)
        rs.append(np.linalg.norm(r))
        x = x + g.vcycle(r)
    factor = (rs[-1] / rs[-6]) ** (1 / 5)
    assert factor <= 0.15


# ---------------------------------------------------------------- P8 LIMEX
def test_p8_extrapolation_order_on_linear_ode(oracle):
    """y' = lam y: the linearly implicit Euler column with n steps gives
    (1 - lam H/n)^-n exactly; extrapolating kappa columns of the harmonic
    sequence has local error O(H^(kappa+1)) against exp(lam H)."""
    lam = -1.3
    for kappa in (1, 2, 3, 4):
        errs = []
        Hs = np.array([0.02, 0.01, 0.005])
        for Hh in Hs:
            T1 = np.array([[(1 - lam * Hh / j) ** (-j)] for j in range(1, kappa + 1)])
            Tkk, _ = oracle.extrapolate(T1, list(range(1, kappa + 1)))
            errs.append(abs(Tkk[0] - np.exp(lam * Hh)))
        slope = np.polyfit(np.log(Hs), np.log(errs), 1)[0]
        assert abs(slope - (kappa + 1)) < 0.1


def test_p8_w_method_keeps_the_order_with_an_inexact_jacobian(oracle):
    """LIMEX is a W-method (Sec. 4: no algebraic conditions on the matrix): for
    y' = lam y, columns built with W = 1 - h J~, J~ = 1.3 lam != lam, i.e.
    y_{k+1} = y_k + h (1 - h J~)^-1 lam y_k, still extrapolate to local order
    kappa + 1.  (The order reduction to q = 2 that the step control assumes
    comes from stiff DAE structure, not from the inexact matrix.)"""
    lam = -1.3
    Jt = 1.3 * lam
    for kappa in (2, 3, 4):
        errs = []
        Hs = np.array([0.02, 0.01, 0.005])
        for Hh in Hs:
            T1 = np.array([[(1 + (Hh / j) * lam / (1 - (Hh / j) * Jt)) ** j] for j in range(1, kappa + 1)])
            Tkk, _ = oracle.extrapolate(T1, list(range(1, kappa + 1)))
            errs.append(abs(Tkk[0] - np.exp(lam * Hh)))
        slope = np.polyfit(np.log(Hs), np.log(errs), 1)[0]
        assert abs(slope - (kappa + 1)) < 0.1


def test_limex_columns_match_dense_linearly_implicit_euler(oracle):
    """kappa = 2 LIMEX step of the oracle = dense reconstruction: columns of
    linearly implicit Euler with the frozen J(u0), M(u0) (numpy solves), then
    T22 = T21 + (T21 - T11)/(2/1 - 1)."""
    p = I.random_problem(2, (9, 9), 17)
    m = oracle.Model(p)
    u0 = p["u0"]
    Hh = 5.0
    F0, J, md = oracle.assemble(m, u0)
    Jd = H.stencil_to_dense(2, m.n, J)
    Md = np.zeros_like(Jd)
    for v in range(m.nv):
        Md[2 * v, 2 * v + 1] = md[v, 0]
        Md[2 * v + 1, 2 * v + 1] = md[v, 1]
    T11 = u0 + np.linalg.solve(Md / Hh - Jd, F0)
    u = u0 + np.linalg.solve(Md / (Hh / 2) - Jd, F0)
    F1 = oracle.assemble(m, u, jacobian=False)[0]
    T21 = u + np.linalg.solve(Md / (Hh / 2) - Jd, F1)
    T22 = T21 + (T21 - T11) / (2.0 / 1.0 - 1.0)
    u_out, info = oracle.limex_step(m, u0, Hh, kappa=2, tol=1e9, nlevels=3, rtol=1e-14, maxit=300)
    assert info["accepted"] == 1 and info["solves"] == 3
    np.testing.assert_allclose(u_out[0::2], T22[0::2], rtol=1e-11)
    np.testing.assert_allclose(u_out[1::2], T22[1::2], atol=1e-11)


def test_step_control_order_clamps_and_rejection(oracle):
    """Step control of Sec. 4 with the order reduced to q = 2: the estimate eps
    does not depend on TOL, the new step grows with TOL^(1/(q+1)) (eight times
    the tolerance doubles it) and is clamped to [0.2, 4] times H; a step with
    eps > TOL is rejected and leaves the state unchanged."""
    p = I.random_problem(2, (9, 9), 18)
    m = oracle.Model(p)
    Hh, rho = 2.0, 0.75
    kw = dict(kappa=3, rho=rho, nlevels=3, rtol=1e-13, maxit=300)
    _, ref = oracle.limex_step(m, p["u0"], Hh, tol=1e9, **kw)
    eps = ref["eps"]
    assert eps > 0 and ref["H_new"] == 4.0 * Hh and ref["accepted"] == 1
    t1 = 1.5 * eps / rho                 # (rho TOL / eps)^(1/3) = 1.5^(1/3), unclamped
    _, a = oracle.limex_step(m, p["u0"], Hh, tol=t1, **kw)
    _, b = oracle.limex_step(m, p["u0"], Hh, tol=8.0 * t1, **kw)
    assert a["eps"] == eps and b["eps"] == eps
    assert a["accepted"] == 1 and b["accepted"] == 1
    assert b["H_new"] / a["H_new"] == pytest.approx(2.0, rel=1e-12)
    u_r, r = oracle.limex_step(m, p["u0"], Hh, tol=1e-6 * eps, **kw)
    assert r["accepted"] == 0 and r["H_new"] == pytest.approx(0.2 * Hh, rel=1e-15)
    assert np.array_equal(u_r, p["u0"])


def test_error_norm_quadratures(oracle):
    """H1 seminorm of a linear function = |a|^2 |Omega|; of x*y on the unit
    square = 2/3 (bilinear, exact); lumped L2 of 1 = |Omega|."""
    n = (9, 5, 1)
    h = (1 / 8, 1 / 4, 1.0)
    v = np.arange(45)
    x, y = (v % 9) * h[0], (v // 9) * h[1]
    assert oracle.h1_seminorm2(2, n, h, 2 * x - 3 * y) == pytest.approx(13.0, rel=1e-13)
    assert oracle.h1_seminorm2(2, n, h, x * y) == pytest.approx(2 / 3, rel=1e-13)
    assert oracle.lumped_l2norm2(2, n, h, np.ones(45)) == pytest.approx(1.0, rel=1e-14)
    n3 = (5, 3, 9)
    h3 = (0.25, 0.5, 0.125)
    v3 = np.arange(int(np.prod(n3)))
    z = (v3 // 15) * h3[2]
    assert oracle.h1_seminorm2(3, n3, h3, 4 * z) == pytest.approx(16.0, rel=1e-13)


def test_pdmin_and_storage_invariants(oracle):
    p = I.random_problem(3, (6, 5, 4), 2)
    m = oracle.Model(p)
    pdm = oracle.pdmin(m)
    assert set(np.unique(pdm)) <= set(np.unique(p["pd"]))
    assert pdm.min() == p["pd"].min()
    phiv = oracle.phiv(m)
    vol = np.prod(p["h"])
    assert phiv.sum() == pytest.approx((p["phi"] * vol).sum(), rel=1e-13)


# ---------------------------------------------------------------- discretisation variants
def _cell_weights(p):
    """Per vertex: list of (cell, Phi_c |c| / 2^d) of the cells around it."""
    dim, n, h = p["dim"], p["n"], p["h"]
    cx, cy = n[0] - 1, n[1] - 1
    cz = n[2] - 1 if dim == 3 else 1
    vol = h[0] * h[1] * (h[2] if dim == 3 else 1.0)
    out = []
    for v in range(n[0] * n[1] * n[2]):
        i, j, k = v % n[0], (v // n[0]) % n[1], v // (n[0] * n[1])
        cells = []
        for dz in ((0, 1) if dim == 3 else (0,)):
            for dy in (0, 1):
                for dx in (0, 1):
                    ci, cj, ck = i - dx, j - dy, k - dz
                    if 0 <= ci < cx and 0 <= cj < cy and 0 <= ck < cz:
                        c = ci + cx * (cj + cy * ck)
                        cells.append((c, p["phi"][c] * vol / 2 ** dim))
        out.append(cells)
    return out


def test_darcy_upwind_water_flux_needs_a_water_potential_gradient(oracle):
    """Darcy-velocity upwinding moves water only along grad p_w - rho_w g: with
    uniform p_w, no gravity and a varying S_n over two materials the water
    residual is exactly zero, while the split scheme of Sec. 3.2 (capillary
    diffusion not upwinded) gives a nonzero water flux."""
    p = I.random_problem(2, (9, 8), 31, gravity=False, dirichlet=False)
    p["u0"][0::2] = I.P_TOP
    p["scheme"] = 2
    F = oracle.assemble(oracle.Model(p), p["u0"], jacobian=False)[0]
    assert np.all(F[0::2] == 0.0)
    assert np.abs(F[1::2]).max() > 0.0
    p["scheme"] = 0
    F0 = oracle.assemble(oracle.Model(p), p["u0"], jacobian=False)[0]
    assert np.abs(F0[0::2]).max() > 1e-3 * np.abs(F0[1::2]).max()


@pytest.mark.parametrize("dim,nv", [(2, (9, 7)), (3, (5, 5, 4))])
def test_darcy_upwind_equals_split_scheme_without_capillary_gradient(oracle, dim, nv):
    """One material and uniform S_n: p_c is uniform, T_c = 0 and the two
    upwindings coincide (T_pw and T_w differ by rounding only)."""
    p = I.random_problem(dim, nv, 32)
    p["pd"][:] = 755.0
    p["u0"][1::2] = 0.25
    out = []
    for scheme in (0, 2):
        p["scheme"] = scheme
        out.append(oracle.assemble(oracle.Model(p), p["u0"]))
    (F0, J0, m0), (F2, J2, m2) = out
    assert np.abs(F2 - F0).max() <= 1e-12 * np.abs(F0).max()
    assert np.abs(J2 - J0).max() <= 1e-12 * np.abs(J0).max()
    assert np.array_equal(m0, m2)


@pytest.mark.parametrize("dim,nv", [(2, (9, 7)), (3, (5, 6, 5))])
def test_shat_storage_reduces_to_vertex_storage_in_one_material(oracle, dim, nv):
    """With one entry pressure S hat = S (Eq. (hSw), first case): storage and
    M of the S hat variant equal rho Phi V S of Eqs. (dsW),(dpN)."""
    p = I.random_problem(dim, nv, 33, stress=True)
    p["pd"][:] = 755.0
    m0 = oracle.Model(p)
    phiv = oracle.phiv(m0)
    Sn = p["u0"][1::2]
    p["scheme"] = 1
    m1 = oracle.Model(p)
    st = oracle.storage(m1, p["u0"])
    np.testing.assert_allclose(st[:, 1], p["rho_n"] * phiv * Sn, rtol=0, atol=1e-14 * p["rho_n"] * phiv.max())
    np.testing.assert_allclose(st[:, 0], p["rho_w"] * phiv * (1 - Sn), rtol=0,
                               atol=1e-14 * p["rho_w"] * phiv.max())
    _, _, md0 = oracle.assemble(m0, p["u0"])
    _, _, md1 = oracle.assemble(m1, p["u0"])
    np.testing.assert_allclose(md1, md0, rtol=1e-14, atol=0)


@pytest.mark.parametrize("scheme", [0, 1])
def test_mass_matrix_is_the_derivative_of_the_storage(oracle, scheme):
    """M = d m / d S_n (Sec. 4), vertex by vertex, against central differences
    of the storage terms; vertices where one-sided differences disagree (the S
    hat cap inside the step) are skipped."""
    p = I.random_problem(3, (5, 5, 4), 34, stress=True, dirichlet=False)
    p["scheme"] = scheme
    m = oracle.Model(p)
    u = p["u0"]
    _, _, md = oracle.assemble(m, u)
    d = 1e-7
    up, um = u.copy(), u.copy()
    up[1::2] += d
    um[1::2] -= d
    st0, stp, stm = oracle.storage(m, u), oracle.storage(m, up), oracle.storage(m, um)
    fwd, bwd, cen = (stp - st0) / d, (st0 - stm) / d, (stp - stm) / (2 * d)
    ok = np.all(np.abs(fwd - bwd) <= 1e-4 * np.abs(md).max(), axis=1)
    assert ok.mean() > 0.9
    np.testing.assert_allclose(cen[ok], md[ok], rtol=0, atol=1e-6 * np.abs(md).max())


def test_shat_storage_entry_pressure_barrier(oracle):
    """Eq. (hSw), second case: where p_d(N) >= p_dmin J(S_w) the sub-control
    volume holds S_w = 1 - S_nr, i.e. no NAPL.  At S_n = 0.2 (S_e = 0.667) the
    lens sub-volumes around an interface vertex (p_d 1163 against 755) are at
    the cap, so m_n,i = rho_n S_n,i times the pore volume of the sand
    sub-volumes only, and m_w takes the rest."""
    p = I.random_problem(3, (7, 7, 6), 35)
    p["u0"][1::2] = 0.2
    p["scheme"] = 1
    m = oracle.Model(p)
    st = oracle.storage(m, p["u0"])
    W = _cell_weights(p)
    pdm = oracle.pdmin(m)
    mixed = 0
    for v, cells in enumerate(W):
        sand = sum(w for c, w in cells if p["pd"][c] == pdm[v])
        total = sum(w for c, w in cells)
        if sand < total:
            mixed += 1
        assert st[v, 1] == pytest.approx(p["rho_n"] * 0.2 * sand, rel=1e-14, abs=1e-300)
        assert st[v, 0] == pytest.approx(p["rho_w"] * (total - 0.2 * sand), rel=1e-14)
    assert mixed > 10


# ---------------------------------------------------------------- implicit Euler + Newton
def test_ie_hydrostatic_state_is_stationary(oracle):
    """Exact hydrostatic p_w, S_n = 0: R(u_old) = 0 to rounding, so the step
    takes no Newton iteration and returns the state."""
    p = I.random_problem(2, (17, 17), 21)
    n, h = p["n"], p["h"]
    nvx = int(np.prod(n))
    vert = ((np.arange(nvx) // n[0]) % n[1]) * h[1]
    u = np.zeros(2 * nvx)
    u[0::2] = I.P_TOP + p["rho_w"] * I.GRAV * (1.0 - vert)
    m = oracle.Model(p)
    u1, info = oracle.ie_step(m, u, 100.0, nlevels=3)
    assert info["status"] == 0 and info["newton"] == 0
    assert np.array_equal(u1, u)


def test_ie_affine_problem_takes_one_newton_step(oracle):
    """With S_n = 0 everywhere no NAPL moves (k_rn(1) = 0 with zero slope) and
    the water residual is affine in p_w (uniform S: the same k_rw at every
    vertex, a fixed capillary term): one Newton step solves the implicit Euler
    equations up to the linear solver's tolerance."""
    p = I.random_problem(2, (17, 17), 22)
    p["u0"][1::2] = 0.0
    m = oracle.Model(p)
    u1, info = oracle.ie_step(m, p["u0"], 50.0, nlevels=3, rtol=1e-9, atol=0.0, lin_rtol=1e-13)
    assert info["status"] == 0 and info["newton"] == 1, info
    assert info["res"] <= 1e-9 * info["res0"]
    assert np.all(u1[1::2] == 0.0)


@pytest.mark.parametrize("scheme", [0, 1])
def test_ie_napl_mass_balance(oracle, scheme):
    """Every implicit Euler step is a discrete balance: with a NAPL source and
    no NAPL Dirichlet rows, sum_i (m_n,i(u1) - m_n,i(u0)) = H sum_i q_n,i up to
    the Newton residual, also with the nonlinear S hat storage."""
    p = I.dnapl_infiltration(9)
    p["scheme"] = scheme
    m = oracle.Model(p)
    H = 20.0
    u1, info = oracle.ie_step(m, p["u0"], H, nlevels=3, atol=0.0, rtol=1e-13, lin_rtol=1e-14, max_newton=30)
    assert info["status"] == 0, info
    dm = oracle.storage(m, u1)[:, 1].sum() - oracle.storage(m, p["u0"])[:, 1].sum()
    q = p["q_in"][1::2].sum() * H
    assert abs(dm - q) <= 1e-9 * q


def _consistent_start(oracle, m, u):
    """The recipes' noisy p_w does not satisfy the pressure constraint (M has
    no p_w column, so the summed volume balance is algebraic); one short
    implicit Euler step projects the state onto it."""
    u0, inf = oracle.ie_step(m, u, 1e-3, nlevels=2, atol=0.0, rtol=1e-11, lin_rtol=1e-14, max_newton=40)
    assert inf["status"] == 0, inf
    return u0


def test_ie_is_first_order_in_time(oracle):
    """Implicit Euler is first order: successive differences of 16, 32, 64
    and 128 steps over the same interval halve (ratios within [1.8, 2.2])."""
    p = I.random_problem(2, (9, 9), 23)
    m = oracle.Model(p)
    u0 = _consistent_start(oracle, m, p["u0"])
    T, out = 0.5, {}
    for nsteps in (16, 32, 64, 128):
        u = u0.copy()
        for _ in range(nsteps):
            u, inf = oracle.ie_step(m, u, T / nsteps, nlevels=2, atol=0.0, rtol=1e-11, lin_rtol=1e-14, max_newton=40)
            assert inf["status"] == 0, inf
        out[nsteps] = u
    d = [np.abs(out[a][1::2] - out[2 * a][1::2]).max() for a in (16, 32, 64)]
    assert 1.8 <= d[0] / d[1] <= 2.2 and 1.8 <= d[1] / d[2] <= 2.2, d


def test_limex_and_implicit_euler_share_their_limit(oracle):
    """Two independent time integrators of the same semi-discretisation: from a
    consistent state, LIMEX (kappa = 4, two steps) lands within twice implicit
    Euler's own error at 128 steps (its successive difference) of the 128-step
    result, and kappa = 1 (linearly implicit Euler) converges to that limit at
    first order."""
    p = I.random_problem(2, (9, 9), 23)
    m = oracle.Model(p)
    u0 = _consistent_start(oracle, m, p["u0"])
    T = 0.5

    def ie(n):
        u = u0.copy()
        for _ in range(n):
            u, inf = oracle.ie_step(m, u, T / n, nlevels=2, atol=0.0, rtol=1e-11, lin_rtol=1e-14, max_newton=40)
            assert inf["status"] == 0
        return u

    def limex(n, kappa):
        u = u0.copy()
        for _ in range(n):
            u, inf = oracle.limex_step(m, u, T / n, kappa=kappa, tol=1e9, nlevels=2, rtol=1e-14, maxit=400)
            assert inf["status"] == 0
        return u

    a, b = ie(64), ie(128)
    ie_err = np.abs(a[1::2] - b[1::2]).max()
    assert np.abs(limex(2, 4)[1::2] - b[1::2]).max() <= 2.0 * ie_err
    e = [np.abs(limex(n, 1)[1::2] - b[1::2]).max() for n in (2, 8)]
    assert 3.0 <= e[0] / e[1] <= 5.0, e


# ---------------------------------------------------------------- Case 1 (Buckley-Leverett)
def _case1_table():
    rows = {}
    with open(os.path.join(GOLDEN, "case1_error1.txt")) as f:
        for line in f:
            t = line.split()
            if t and t[0] in ("ie", "limex"):
                rows[(t[0], int(t[1]))] = (int(t[2]), float(t[3]), float(t[4]))
    return rows


def test_buckley_leverett_solution_closed_form():
    """The textbook solution used below: with Brooks-Corey lambda = 2 and equal
    viscosities the Welge front saturation is 3/4 (f(S)/S is maximal there),
    and the front speed q f'(S_f)/phi reproduces the paper's v = 1.84e-6 m/s."""
    c = I.CASE1
    q = c["q_out"] / c["rho"]
    _, Sf, xf = H.buckley_leverett_sw(np.array([0.0]), c["T"], q, c["phi"], c["mu"], c["mu"])
    assert Sf == pytest.approx(0.75, abs=1e-4)
    assert xf / c["T"] == pytest.approx(1.84e-6, rel=5e-3)


def test_case1_implicit_euler_errors_match_the_paper(oracle):
    """The whole discretisation against printed numbers: implicit Euler on
    Case 1 with 64 elements at Courant number 0.8 (65 steps in the paper, 64
    here from T / dt rounded up) gives the L1 and L2 errors of Table error1
    within 3%."""
    c = I.CASE1
    rows = _case1_table()
    nx = 64
    p = I.case1_buckley_leverett(nx)
    m = oracle.Model(p)
    nst = int(np.ceil(c["T"] / (0.8 * (c["L"] / nx) / 1.84e-6)))
    u = p["u0"].copy()
    for _ in range(nst):
        u, inf = oracle.ie_step(m, u, c["T"] / nst, nlevels=p["nlevels"], atol=1e-9, rtol=1e-6, lin_rtol=1e-8,
                                max_newton=30)
        assert inf["status"] == 0, inf
    sw = 1.0 - u[1::2].reshape(p["n"][1], p["n"][0])
    assert np.abs(sw - sw[0]).max() <= 1e-9          # one-dimensional flow
    xv = np.arange(nx + 1) * c["L"] / nx
    q = c["q_out"] / c["rho"]
    exact = lambda x: H.buckley_leverett_sw(x, c["T"], q, c["phi"], c["mu"], c["mu"])[0]
    steps, L1, L2 = rows[("ie", nx)]
    assert abs(nst - steps) <= 1
    assert H.lp_error_1d(xv, sw[0], exact, 1) == pytest.approx(L1, rel=0.03)
    assert H.lp_error_1d(xv, sw[0], exact, 2) == pytest.approx(L2, rel=0.03)


def test_ie_line_search_converges_where_plain_newton_fails(oracle):
    """A 1000 s step of the DNAPL-inlet recipe at 9^3: undamped Newton does
    not converge in 40 iterations, backtracking (at most 4 halvings) does, and
    the result solves the implicit Euler equations, checked here from the
    oracle's flux residual and storage rather than the step's own report."""
    p = I.dnapl_infiltration(9)
    m = oracle.Model(p)
    H = 1000.0
    _, plain = oracle.ie_step(m, p["u0"], H, nlevels=2, atol=0.0, rtol=1e-9, lin_rtol=1e-12, max_newton=40)
    assert plain["status"] != 0
    u1, inf = oracle.ie_step(m, p["u0"], H, nlevels=2, atol=0.0, rtol=1e-9, lin_rtol=1e-12, max_newton=40, max_ls=4)
    assert inf["status"] == 0, inf
    F = oracle.assemble(m, u1, jacobian=False)[0]
    dm = oracle.storage(m, u1) - oracle.storage(m, p["u0"])
    R = F - dm.ravel() / H
    R[0::2][p["dir"].astype(bool)] = F[0::2][p["dir"].astype(bool)]
    assert np.linalg.norm(R) <= 1e-9 * inf["res0"] * 1.0000001


# ---------------------------------------------------------------- adaptive LIMEX runs
def test_limex_run_applies_the_step_control_policy(oracle):
    """rfo_limex_run from a consistent state (tol 1e-3, H0 = 50 s, H_max =
    600 s, t_end = 3000 s): accepted steps have eps <= tol and rejected ones
    eps > tol; a rejected step is retried with a smaller H; the step after one
    accepted right after a rejection is not larger (hold); H never exceeds
    H_max; the last step lands on t_end.  Replaying the recorded steps with
    rfo_limex_step gives the same state bit for bit, so the run is exactly a
    composition of steps."""
    p = I.random_problem(2, (9, 9), 23)
    m = oracle.Model(p)
    u0 = _consistent_start(oracle, m, p["u0"])
    tol, H_max, t_end = 1e-3, 600.0, 3000.0
    u, info, hist = oracle.limex_run(m, u0, 50.0, t_end=t_end, H_max=H_max, tol=tol, kappa=3, nlevels=2, rtol=1e-12)
    assert info["status"] == 0 and info["steps"] == len(hist)
    H, eps, acc = hist[:, 0], hist[:, 1], hist[:, 2].astype(bool)
    assert info["rejected"] >= 2 and info["accepted"] == acc.sum() and info["rejected"] == (~acc).sum()
    assert np.all(eps[acc] <= tol) and np.all(eps[~acc] > tol)
    for k in range(len(hist) - 1):
        if not acc[k]:
            assert H[k + 1] < H[k]
        if acc[k] and k > 0 and not acc[k - 1] and k + 1 < len(hist) - 1:
            assert H[k + 1] <= H[k]
    assert H.max() <= H_max and (H == H_max).any()
    assert info["t"] == pytest.approx(t_end, rel=1e-12)
    assert H[acc].sum() == pytest.approx(t_end, rel=1e-12)
    # replay
    v = u0.copy()
    for k in range(len(hist)):
        v2, inf = oracle.limex_step(m, v, H[k], kappa=3, tol=tol, nlevels=2, rtol=1e-12)
        assert inf["accepted"] == acc[k] and inf["eps"] == eps[k]
        v = v2
    assert np.array_equal(v, u)


# ---------------------------------------------------------------- FP32 emulation of the V-cycle
@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("case", ["2d-lens", "3d-random"])
def test_fp32_vcycle_emulation_tracks_the_fp64_vcycle(oracle, case, smoother):
    """The float V-cycle (float storage and sums) is the FP64 V-cycle up to
    single-precision rounding: per component within 2e-6 of the largest
    value (a dropped or misplaced term would move it by O(1)); as a
    stationary iteration on the constant-coefficient Poisson stencil it
    contracts like the FP64 cycle until the float floor."""
    prob = I.lens_square_2d() if case == "2d-lens" else I.random_problem(3, (17, 17, 17), 5)
    m = oracle.Model(prob)
    F, J, md = oracle.assemble(m, prob["u0"])
    A = oracle.make_A(J, md, 2.0 / prob["H"])
    L = 4 if case == "2d-lens" else 3
    gm = oracle.GMG(m.dim, m.n, A, prob["dir"], L, smoother=smoother)
    g32 = oracle.GMG32(gm)
    b = np.random.default_rng(2).standard_normal(2 * m.nv).astype(np.float32).astype(np.float64)
    x64, x32 = gm.vcycle(b), g32.vcycle(b)
    for a in range(2):
        assert np.abs(x32[a::2] - x64[a::2]).max() <= 2e-6 * np.abs(x64[a::2]).max(), a


def test_fp32_vcycle_emulation_converges_on_poisson(oracle):
    dim, nv = 2, (33, 33)
    p = _poisson_problem(dim, nv)
    m = oracle.Model(p)
    F, J, md = oracle.assemble(m, p["u0"])
    A = oracle.make_A(J, md, 0.1)
    gm = oracle.GMG(dim, m.n, A, p["dir"], 4, smoother=0)
    g32 = oracle.GMG32(gm)
    x = np.random.default_rng(3).standard_normal(2 * m.nv)
    x[0::2][p["dir"].astype(bool)] = 0.0
    rs = []
    for _ in range(5):
        r = -oracle.spmv(dim, m.n, A, x)
        rs.append(np.linalg.norm(r))
        x = x + g32.vcycle(r)
    rates = [rs[k + 1] / rs[k] for k in range(1, 4)]
    assert max(rates) <= 0.15, rates


# ---------------------------------------------------------------- Case 2 (extended Buckley-Leverett)
def _case2_table():
    rows, jump = {}, None
    with open(os.path.join(GOLDEN, "case2_error2.txt")) as f:
        for line in f:
            t = line.split()
            if t and t[0] in ("ie", "limex"):
                rows[(t[0], int(t[1]))] = (int(t[2]), float(t[3]), float(t[4]))
            elif t and t[0] == "interface_jump":
                jump = (float(t[1]), float(t[2]))
    return rows, jump


def _case2_exact(x):
    c = I.CASE2
    return H.extended_buckley_leverett_sw(x, c["T"], c["q_out"] / c["rho"], c["phi"], c["mu_w"], c["mu_n"],
                                          c["laws"][0], c["laws"][1], c["x_if"])


def test_extended_buckley_leverett_solution():
    """The reference solution used for Case 2: with the two media's laws as
    printed (k_rn taken as 0 past its first root) the saturation jumps at the
    interface from 0.52 to 0.48, the values the paper gives; with the same law
    on both sides it is the textbook one-medium solution."""
    c = I.CASE2
    _, jump = _case2_table()
    s = _case2_exact(np.array([c["x_if"] - 1e-9, c["x_if"] + 1e-9]))
    assert s[0] == pytest.approx(jump[0], abs=5e-3) and s[1] == pytest.approx(jump[1], abs=5e-3)
    bc = (1.0, 1.0, 4.0, 1.0, 1.0, 1.0)            # Brooks-Corey lambda = 2 written as a polynomial law
    x = np.linspace(0.0, 300.0, 6001)
    q, t = 3e-7, 1500 * 86400.0
    one = H.extended_buckley_leverett_sw(x, t, q, 0.2, 1e-3, 1e-3, bc, bc, 150.0)
    ref = H.buckley_leverett_sw(x, t, q, 0.2, 1e-3, 1e-3)[0]
    assert np.abs(one - ref).sum() * (x[1] - x[0]) <= 0.05


def test_case2_laws_reach_every_use_of_k_r(oracle):
    """Per-cell laws in the assembly: a law table of Brooks-Corey rows gives
    bitwise the assembly without one; polynomial rows equal to the
    Brooks-Corey lambda = 2 laws (k_rw = S^4, k_rn = (1 - S)^2 (1 - S^2)) give
    it up to rounding; and a cell's law changes F only in the rows of its own
    corners (the upwinded k_rw, k_rw at the face and k_rn of S hat all come
    from the face's cell)."""
    p = I.random_problem(2, (9, 7), 11)
    m0 = oracle.Model(p)
    F0, J0, _ = oracle.assemble(m0, p["u0"])
    nc = p["K"].size
    for row, exact in (((0.0,) * 6, True), ((1.0, 1.0, 4.0, 1.0, 1.0, 1.0), False)):
        q = dict(p, kr_laws=np.array([row]), cell_law=np.zeros(nc, np.uint8))
        F1, J1, _ = oracle.assemble(oracle.Model(q), p["u0"])
        if exact:
            assert np.array_equal(F0, F1) and np.array_equal(J0, J1)
        else:
            assert np.abs(F1 - F0).max() <= 1e-13 * np.abs(F0).max()
            assert np.abs(J1 - J0).max() <= 1e-13 * np.abs(J0).max()
    law = np.zeros(nc, np.uint8)
    cell = 3 + 8 * 2                                  # cell (3, 2) of the 8 x 6 cells
    law[cell] = 1
    q = dict(p, kr_laws=np.array([(0.0,) * 6, I.CASE2["laws"][0]]), cell_law=law)
    F2 = oracle.assemble(oracle.Model(q), p["u0"], jacobian=False)[0]
    changed = np.nonzero(np.abs(F2 - F0).reshape(-1, 2).max(axis=1))[0]
    corners = {(3 + a) + 9 * (2 + b) for a in (0, 1) for b in (0, 1)}
    assert len(changed) > 0 and set(changed.tolist()) <= corners


def test_case2_polynomial_law_derivatives(oracle):
    """dk_r/dS_e of the polynomial laws by central differences away from the
    roots, k_rn = 0 from its first root on (law 1: 1.652 S^2 = 1, S = 0.7780;
    law 2: 1.25 S = 1, S = 0.8), and both laws clamped outside [0, 1]."""
    p = I.case2_extended_buckley_leverett(8)
    m = oracle.Model(p)
    for cell, root in ((0, 1.0 / np.sqrt(1.652)), (7, 0.8)):
        for S in (0.1, 0.3, 0.55, 0.7, 0.95):
            v = oracle.kr_law(m, cell, S)
            d = 1e-6
            fd = (oracle.kr_law(m, cell, S + d) - oracle.kr_law(m, cell, S - d)) / (2 * d)
            assert v[1] == pytest.approx(fd[0], rel=1e-6, abs=1e-12)
            if abs(S - root) > 1e-3:
                assert v[3] == pytest.approx(fd[2], rel=1e-6, abs=1e-12)
            assert (v[2] == 0.0) == (S >= root)
        lo, hi = oracle.kr_law(m, cell, -0.2), oracle.kr_law(m, cell, 1.3)
        assert np.array_equal(lo, oracle.kr_law(m, cell, 0.0) * [1, 0, 1, 0])
        assert np.array_equal(hi, oracle.kr_law(m, cell, 1.0) * [1, 0, 1, 0])


def test_case2_implicit_euler_errors_match_the_paper(oracle):
    """The discretisation with per-medium laws against printed numbers:
    implicit Euler on Case 2 with 64 elements and the paper's 65 steps gives
    the L1 and L2 errors of Table error2 within 3%."""
    c = I.CASE2
    rows, _ = _case2_table()
    nx = 64
    steps, L1, L2 = rows[("ie", nx)]
    p = I.case2_extended_buckley_leverett(nx)
    m = oracle.Model(p)
    u = p["u0"].copy()
    for _ in range(steps):
        u, inf = oracle.ie_step(m, u, c["T"] / steps, nlevels=p["nlevels"], atol=1e-9, rtol=1e-6, lin_rtol=1e-8,
                                max_newton=30)
        assert inf["status"] == 0, inf
    sw = 1.0 - u[1::2].reshape(p["n"][1], p["n"][0])
    assert np.abs(sw - sw[0]).max() <= 1e-9          # one-dimensional flow
    xv = np.arange(nx + 1) * c["L"] / nx
    assert H.lp_error_1d(xv, sw[0], _case2_exact, 1) == pytest.approx(L1, rel=0.03)
    assert H.lp_error_1d(xv, sw[0], _case2_exact, 2) == pytest.approx(L2, rel=0.03)
