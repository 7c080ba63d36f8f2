"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element
by element, on seeded inputs that span several thread blocks and ragged tails.

Tolerances:
  FP64 kernels: 1e-12 relative to the row's largest entry (Jacobian, Galerkin
    operators) or to the largest magnitude of the compared vector; the two
    sides sum in different orders, so bitwise equality is not expected.
  FP32 preconditioner kernels: inputs are rounded to FP32 identically on both
    sides; the bound is 64 u32 (|A||x| + |b|) per component, u32 = 2^-24, i.e.
    a few rounding errors of every term of the 27-block row sum.
  Solves: both sides converge to a true relative residual <= 1e-12; the
    solutions then agree to cond(A) * 1e-12, checked as 1e-8 relative in p_w
    increments and 1e-9 absolute in S_n increments.
"""
import numpy as np
import pytest

import oracle as O
from paper_2506_04763_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rf = pytest.importorskip("paper_2506_04763_gb300")

CASES = {
    "2d-lens-33": lambda: I.lens_square_2d(),
    "2d-17x13-stress": lambda: I.random_problem(2, (17, 13), 3, stress=True),
    "3d-9x7x5-stress": lambda: I.random_problem(3, (9, 7, 5), 4, stress=True),
    "3d-17cube": lambda: I.random_problem(3, (17, 17, 17), 5),
    "3d-33x17x9-nodir": lambda: I.random_problem(3, (33, 17, 9), 6, dirichlet=False),
    "2d-even-10x8": lambda: I.random_problem(2, (10, 8), 8),
    # the full-size workload's recipe at 33^3: far-field S_n ~ 1e-13 gives k_rn
    # entries far below the FP32 normal range
    "3d-lenses-33": lambda: I.lognormal_lenses_box(33),
    # each cell with one of Brooks-Corey and the two polynomial k_r laws of Case 2
    "2d-17x13-stress-laws": lambda: I.mixed_kr_laws(I.random_problem(2, (17, 13), 3, stress=True), 21),
    "3d-17x9x13-laws": lambda: I.mixed_kr_laws(I.random_problem(3, (17, 9, 13), 9), 22),
}
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _grid(prob):
    return rf.Grid(prob)


def _assembled(prob):
    g = _grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    torch.cuda.synchronize()
    return g, F.cpu().numpy()


def _levels(prob):
    n = prob["n"][0]
    L = 1
    m = [t for t in prob["n"][:prob["dim"]]]
    while all((t - 1) % 2 == 0 and t >= 3 for t in m) and L < 4:
        m = [(t - 1) // 2 + 1 for t in m]
        L += 1
    return L


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("case", list(CASES))
def test_assembly_matches_oracle(case):
    prob = CASES[case]()
    g, F = _assembled(prob)
    J, md = g.export_jacobian()
    m = O.Model(prob)
    F_o, J_o, md_o = O.assemble(m, prob["u0"])
    for a in range(2):
        rows = np.abs(J_o[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2)) + 1e-300
        err = np.abs(J[:, :, 2 * a:2 * a + 2] - J_o[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2))
        assert np.all(err <= 1e-12 * rows), (case, a, (err / rows).max())
        sc = np.abs(F_o[a::2]).max()
        assert np.abs(F[a::2] - F_o[a::2]).max() <= 1e-12 * sc
    np.testing.assert_allclose(md, md_o, rtol=1e-14, atol=0)
    g.close()


@pytest.mark.parametrize("case", ["3d-9x7x5-stress", "2d-17x13-stress-laws", "3d-17x9x13-laws"])
def test_vertex_and_element_assembly_agree(case, monkeypatch):
    """The one-thread-per-vertex assembly (RF_ASM_VERTEX=1) evaluates every
    face from both ends with the element kernel's face arithmetic, per-medium
    laws included: F, J and M agree to the rounding of their different
    summation orders."""
    prob = CASES[case]()
    out = []
    for mode in ("0", "1"):
        monkeypatch.setenv("RF_ASM_VERTEX", mode)
        g, F = _assembled(prob)
        J, md = g.export_jacobian()
        out.append((F, J, md))
        g.close()
    (F0, J0, m0), (F1, J1, m1) = out
    for a in range(2):
        rows = np.abs(J0[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2)) + 1e-300
        err = np.abs(J1[:, :, 2 * a:2 * a + 2] - J0[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2))
        assert np.all(err <= 1e-13 * rows), (a, (err / rows).max())
        assert np.abs(F1[a::2] - F0[a::2]).max() <= 1e-13 * np.abs(F0[a::2]).max()
    np.testing.assert_allclose(m1, m0, rtol=1e-14, atol=0)


def test_assembly_host_and_device_pointers_agree():
    prob = CASES["3d-9x7x5-stress"]()
    g = _grid(prob)
    F_host = np.zeros(2 * g.nv)
    g.assemble(np.ascontiguousarray(prob["u0"]), True, F_host)
    u = torch.tensor(prob["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    torch.cuda.synchronize()
    assert np.array_equal(F.cpu().numpy(), F_host)
    g.close()


# ------------------------------------------------------------------ outer operator
@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "3d-9x7x5-stress"])
def test_fp64_spmv_matches_oracle(case):
    prob = CASES[case]()
    g, F = _assembled(prob)
    shift = 0.1
    g.gmg_setup([shift], rf.gmg_opts(_levels(prob), precision="fp64"))
    m = O.Model(prob)
    _, J_o, md_o = O.assemble(m, prob["u0"])
    A = O.make_A(J_o, md_o, shift)
    x = np.random.default_rng(1).standard_normal(2 * g.nv) * np.tile([1e3, 0.1], g.nv)
    y = g.apply(rf.RF_OP_SPMV, 0, 0, x)
    y_o = O.spmv(m.dim, m.n, A, x)
    for a in range(2):
        scale = np.abs(A[:, :, 2 * a:2 * a + 2]).max() * np.abs(x).max()
        assert np.abs(y[a::2] - y_o[a::2]).max() <= 1e-13 * scale
    g.close()


# ------------------------------------------------------------------ multigrid pieces
def _setup_both(prob, precision, smoother, levels=None):
    g, F = _assembled(prob)
    shift = 1.0 / prob["H"]
    L = levels or _levels(prob)
    g.gmg_setup([shift, 2 * shift], rf.gmg_opts(L, smoother, precision=precision))
    m = O.Model(prob)
    _, J_o, md_o = O.assemble(m, prob["u0"])
    A = O.make_A(J_o, md_o, 2 * shift)
    gm = O.GMG(m.dim, m.n, A, prob["dir"], L, smoother=O.JACOBI if smoother == "jacobi" else O.GS8)
    return g, F, m, A, gm


@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "3d-33x17x9-nodir"])
def test_galerkin_levels_match_oracle(case):
    prob = CASES[case]()
    g, F, m, A, gm = _setup_both(prob, "fp64", "jacobi")
    assert gm.nlevels == _levels(prob)
    for level in range(gm.nlevels):
        Ag, dims = g.export_level(level, 1)
        Ao = gm.level_matrix(level)
        assert dims == gm.level_dims(level)
        for a in range(2):
            rows = np.abs(Ao[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2)) + 1e-300
            err = np.abs(Ag[:, :, 2 * a:2 * a + 2] - Ao[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2))
            assert np.all(err <= 1e-12 * rows), (level, a, (err / rows).max())
    g.close()


def _unit(prec):
    return 2.0 ** -53 if prec == "fp64" else U32


def _rel_bound(Ao, x, b, dim, n, prec):
    """Residual r = b - A x, per component: 64 u (|A||x| + |b|)."""
    return 64.0 * _unit(prec) * (O.spmv(dim, n, np.abs(Ao), np.abs(x)) + np.abs(b)) + 1e-300


def _centre(dim):
    return 13 if dim == 3 else 4


def _bmul(M, v):
    """Per-vertex 2x2 blocks M [nv, 2, 2] times pairs v [2 nv]."""
    return np.einsum("vab,vb->va", M, v.reshape(-1, 2)).ravel()


def _diag_blocks(dim, A):
    D = A[:, _centre(dim), :].reshape(-1, 2, 2)
    Di = np.linalg.inv(D)
    return np.abs(Di), np.einsum("vab,vbc,vcd->vad", np.abs(Di), np.abs(D), np.abs(Di))


def _jacobi_bound(dim, n, A, b, x, xout, omega, prec, absA=None):
    """x_out = x + omega D^-1 (b - A x), per component: the residual's bound
    through |D^-1|, the rounding of D^-1 itself (|D^-1||D||D^-1| |r|, first
    order), and the final update's rounding."""
    u = _unit(prec)
    aDi, K = _diag_blocks(dim, A)
    absA = np.abs(A) if absA is None else absA
    r = b - O.spmv(dim, n, A, x)
    e_r = O.spmv(dim, n, absA, np.abs(x)) + np.abs(b)
    return 64.0 * u * (omega * (_bmul(aDi, e_r) + _bmul(K, np.abs(r))) + np.abs(x) + np.abs(xout)) + 1e-300


def _gs_bound(dim, n, A, b, x_in, x_out, prec, absA_off=None):
    """Forward multicolour sweep, per component.  A vertex's error is its own
    rounding (as in _jacobi_bound) plus |D^-1| times the errors of the
    neighbours the sweep has already updated (earlier colours), accumulated
    colour by colour in the smoother's order."""
    from tests._helpers import colour
    u = _unit(prec)
    aDi, K = _diag_blocks(dim, A)
    Aoff = A.copy()
    Aoff[:, _centre(dim)] = 0.0
    absAoff = np.abs(Aoff) if absA_off is None else absA_off
    col = np.repeat(colour(dim, n), 2)
    E = np.zeros_like(x_in)
    xcur = x_in.copy()
    for c in range(1 << dim):
        sel = col == c
        r = b - O.spmv(dim, n, Aoff, xcur)
        own = 64.0 * u * (_bmul(aDi, O.spmv(dim, n, absAoff, np.abs(xcur)) + np.abs(b)) + _bmul(K, np.abs(r))
                          + np.abs(x_out))
        prop = _bmul(aDi, O.spmv(dim, n, absAoff, E))
        E[sel] = (own + prop)[sel]
        xcur[sel] = x_out[sel]
    return E + 1e-300


def _within(got, ref, bound):
    err = np.abs(got - ref)
    return np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("smoother", ["jacobi", "gs8"])
@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "2d-17x13-stress"])
def test_level_kernels_match_oracle(case, smoother, precision):
    """Residual, one smoothing sweep and both transfers on every smoothed
    level, each against a per-component rounding bound of its own arithmetic
    (so an error confined to the small S_n rows cannot hide behind the p_w
    rows)."""
    prob = CASES[case]()
    g, F, m, A, gm = _setup_both(prob, precision, smoother)
    rng = np.random.default_rng(5)
    rnd = np.float32 if precision == "fp32" else np.float64
    u = _unit(precision)
    for level in range(gm.nlevels - 1):
        n = gm.level_dims(level)
        nv = int(np.prod(n))
        Ao = gm.level_matrix(level)
        Ao32 = Ao.astype(np.float32).astype(np.float64) if precision == "fp32" else Ao
        b = rng.standard_normal(2 * nv).astype(rnd).astype(np.float64)
        x = rng.standard_normal(2 * nv).astype(rnd).astype(np.float64)
        # residual
        r = g.apply(rf.RF_OP_RESIDUAL, level, 1, b, x)[:2 * nv]
        r_o = O.residual(m.dim, n, Ao32, b, x)
        ok, q = _within(r, r_o, _rel_bound(Ao32, x, b, m.dim, n, precision))
        assert ok, ("residual", level, q)
        # one smoothing sweep (the GPU's D^-1 is the rounded inverse of the
        # FP64 diagonal block; the bound covers both sides' roundings of it)
        sm = g.apply(rf.RF_OP_SMOOTH, level, 1, b, x)[:2 * nv]
        if smoother == "jacobi":
            sm_o = O.jacobi(m.dim, n, Ao32, b, x, 0.8)
            bound = _jacobi_bound(m.dim, n, Ao32, b, x, sm_o, 0.8, precision)
        else:
            sm_o = O.gs_sweep(m.dim, n, Ao32, b, x, True)
            bound = _gs_bound(m.dim, n, Ao32, b, x, sm_o, precision)
        ok, q = _within(sm, sm_o, bound)
        assert ok, ("smoother", level, q)
        # transfers
        nc = gm.level_dims(level + 1)
        nvc = int(np.prod(nc))
        dmf = prob["dir"] if level == 0 else _mask_chain(prob, m, gm, level)
        dmc = _mask_chain(prob, m, gm, level + 1)
        rc = g.apply(rf.RF_OP_RESTRICT, level, 1, b)[:2 * nvc]
        rc_o = O.restrict(m.dim, n, dmf, nc, dmc, b)
        ok, q = _within(rc, rc_o, 64.0 * u * O.restrict(m.dim, n, dmf, nc, dmc, np.abs(b)) + 1e-300)
        assert ok, ("restrict", level, q)
        xc = rng.standard_normal(2 * nvc).astype(rnd).astype(np.float64)
        pr = g.apply(rf.RF_OP_PROLONG, level, 1, xc, x)[:2 * nv]
        pr_o = O.prolong_add(m.dim, n, dmf, nc, dmc, xc, x)
        pbound = 64.0 * u * (np.abs(x) + O.prolong_add(m.dim, n, dmf, nc, dmc, np.abs(xc), np.zeros_like(x))) + 1e-300
        ok, q = _within(pr, pr_o, pbound)
        assert ok, ("prolong", level, q)
    g.close()


def _fp16_dequantised(J):
    """The finest level's FP16 storage as the kernels define it: per vertex and
    entry position q, scale = max over the stencil of |J_q| (as FP32; 1 when
    below the smallest normal float), stored value = half(J_q / scale)
    rounded to nearest, used as float(half) * scale in FP32."""
    mx = np.abs(J).max(axis=1)                                   # [nv, 4]
    sc = np.where(mx >= 1.17549435e-38, mx.astype(np.float32), np.float32(1.0)).astype(np.float32)
    h = (J / sc[:, None, :].astype(np.float64)).astype(np.float16)
    return (h.astype(np.float32) * sc[:, None, :]).astype(np.float64)


@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "3d-9x7x5-stress", "3d-lenses-33"])
def test_fp16_storage_kernels_match_oracle(case):
    """FP16 storage of the finest level (per-position FP32 row scales): the
    residual, a block-Jacobi sweep and a forward 8-colour GS sweep against the
    oracle applied to the same dequantised matrix, per component, to the FP32
    accumulation bound.  The smoothers' D^-1 is that of the unquantised FP64
    diagonal block, as in the kernels."""
    prob = CASES[case]()
    g, F = _assembled(prob)
    shift = 1.0 / prob["H"]
    L = _levels(prob)
    m = O.Model(prob)
    _, J_o, md_o = O.assemble(m, prob["u0"])
    dim, n = m.dim, m.n
    c = _centre(dim)
    Jq = _fp16_dequantised(J_o)
    Aq = O.make_A(Jq, md_o, shift)                 # quantised J, exact shift*M
    Ax = O.make_A(J_o, md_o, shift)                # the FP64 operator (its diagonal feeds D^-1)
    absA = np.abs(Jq)                              # |J| and |shift M| apart: the kernels add them in FP32
    absA[:, c, 1] += shift * np.abs(md_o[:, 0])
    absA[:, c, 3] += shift * np.abs(md_o[:, 1])
    rng = np.random.default_rng(9)
    nv = g.nv
    b = rng.standard_normal(2 * nv).astype(np.float32).astype(np.float64)
    x = rng.standard_normal(2 * nv).astype(np.float32).astype(np.float64)
    for smoother in ("jacobi", "gs8"):
        g.gmg_setup([shift], rf.gmg_opts(L, smoother, precision="fp16"))
        r = g.apply(rf.RF_OP_RESIDUAL, 0, 0, b, x)
        r_o = O.residual(dim, n, Aq, b, x)
        bound = 64.0 * U32 * (O.spmv(dim, n, absA, np.abs(x)) + np.abs(b)) + 1e-300
        ok, q = _within(r, r_o, bound)
        assert ok, ("residual", smoother, q)
        sm = g.apply(rf.RF_OP_SMOOTH, 0, 0, b, x)
        Amix = Aq.copy()
        Amix[:, c] = Ax[:, c]                      # quantised off-diagonal, FP64 diagonal block
        if smoother == "jacobi":
            D = Ax[:, c, :].reshape(-1, 2, 2)
            sm_o = x + 0.8 * _bmul(np.linalg.inv(D), r_o)
            bound = _jacobi_bound(dim, n, Amix, b, x, sm_o, 0.8, "fp32", absA=absA)
        else:
            sm_o = O.gs_sweep(dim, n, Amix, b, x, True)
            absoff = absA.copy()
            absoff[:, c] = 0.0
            bound = _gs_bound(dim, n, Amix, b, x, sm_o, "fp32", absA_off=absoff)
        ok, q = _within(sm, sm_o, bound)
        assert ok, ("smoother", smoother, q)
    g.close()


def _mask_chain(prob, m, gm, level):
    dm = np.asarray(prob["dir"], np.uint8)
    n = m.n
    for l in range(1, level + 1):
        nc = gm.level_dims(l)
        v = np.arange(int(np.prod(nc)))
        I_, J_, K_ = v % nc[0], (v // nc[0]) % nc[1], v // (nc[0] * nc[1])
        dm = dm[2 * I_ + n[0] * (2 * J_ + n[1] * (2 * K_ if m.dim == 3 else 0))]
        n = nc
    return dm


@pytest.mark.parametrize("smoother", ["jacobi", "gs8"])
@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube"])
def test_vcycle_and_coarse_solve_match_oracle(case, smoother):
    prob = CASES[case]()
    g, F, m, A, gm = _setup_both(prob, "fp64", smoother)
    b = np.random.default_rng(2).standard_normal(2 * g.nv)
    x = g.apply(rf.RF_OP_VCYCLE, 0, 1, b)
    x_o = gm.vcycle(b)
    for a in range(2):   # per component
        assert np.abs(x[a::2] - x_o[a::2]).max() <= 1e-9 * np.abs(x_o[a::2]).max(), a
    L = gm.nlevels - 1
    nc = gm.level_dims(L)
    bc = np.random.default_rng(3).standard_normal(2 * int(np.prod(nc)))
    xc = g.apply(rf.RF_OP_COARSE, L, 1, bc)[:len(bc)]
    Ac = __import__("tests._helpers", fromlist=["x"]).stencil_to_dense(m.dim, nc, gm.level_matrix(L))
    xc_o = np.linalg.solve(Ac, bc)
    assert np.abs(xc - xc_o).max() <= 1e-10 * np.abs(xc_o).max()
    g.close()


@pytest.mark.parametrize("smoother", ["jacobi", "gs8"])
@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "3d-lenses-33"])
def test_fp32_vcycle_matches_fp32_emulation(case, smoother):
    """The whole FP32 V-cycle against the oracle's FP32 emulation (the same
    hierarchy with float storage and float sums): per component within 2e-6
    of the largest value, and within the same bound of the FP64 V-cycle."""
    prob = CASES[case]()
    g, F, m, A, gm = _setup_both(prob, "fp32", smoother)
    g32 = O.GMG32(gm)
    b = np.random.default_rng(2).standard_normal(2 * g.nv).astype(np.float32).astype(np.float64)
    x = g.apply(rf.RF_OP_VCYCLE, 0, 1, b)
    x32, x64 = g32.vcycle(b), gm.vcycle(b)
    for a in range(2):
        sc = np.abs(x64[a::2]).max()
        assert np.abs(x[a::2] - x32[a::2]).max() <= 2e-6 * sc, (a, np.abs(x[a::2] - x32[a::2]).max() / sc)
        assert np.abs(x[a::2] - x64[a::2]).max() <= 2e-6 * sc, (a, np.abs(x[a::2] - x64[a::2]).max() / sc)
    g.close()


def _tail_env(monkeypatch, mode):
    """RF_TAIL_MODE / RF_TAIL_SMEM of a tail form: the cluster with the FP32
    GS levels' matrices in shared memory (the default), the cluster reading
    them from global memory, or the cooperative launch."""
    monkeypatch.setenv("RF_TAIL_MODE", "coop" if mode == "coop" else "cluster")
    monkeypatch.setenv("RF_TAIL_SMEM", "0" if mode == "cluster-global" else "1")


@pytest.mark.parametrize("mode", ["cluster", "cluster-global", "coop"])
@pytest.mark.parametrize("smoother", ["jacobi", "gs8"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["3d-17cube", "3d-lenses-33", "2d-lens-33"])
def test_vcycle_tail_matches_oracle(case, precision, smoother, mode, monkeypatch):
    """The one-launch execution of the small levels (RF_TAIL_NV; one
    thread-block cluster, with the FP32 GS levels' matrices in its shared
    memory or not, or a cooperative launch with bounded grid barriers)
    computes the V-cycle of one launch per phase bit for bit (the same
    arithmetic per vertex in the same order, the coarsest solve summed in
    the coarse kernel's order), and so the oracle's V-cycle."""
    prob = CASES[case]()
    out = {}
    for tail in ("0", "100000"):
        monkeypatch.setenv("RF_TAIL_NV", tail)
        _tail_env(monkeypatch, mode)
        g, F, m, A, gm = _setup_both(prob, precision, smoother)
        b = np.random.default_rng(2).standard_normal(2 * g.nv)
        out[tail] = g.apply(rf.RF_OP_VCYCLE, 0, 1, b)
        g.close()
    assert np.array_equal(out["0"], out["100000"])
    x, x_o = out["100000"], gm.vcycle(b)
    tol = 1e-9 if precision == "fp64" else 1e-4
    for a in range(2):   # per component
        assert np.abs(x[a::2] - x_o[a::2]).max() <= tol * np.abs(x_o[a::2]).max(), a


@pytest.mark.parametrize("mode", ["cluster", "cluster-global", "coop"])
@pytest.mark.parametrize("precision,smoother", [("fp32", "gs8"), ("fp64", "jacobi"), ("fp16", "gs8")])
def test_solve_with_one_launch_tail(precision, smoother, mode, monkeypatch):
    """Solves with the small levels in one launch, captured in the
    iteration's CUDA graph and replayed every iteration, are bitwise those of
    the launch-per-phase V-cycle."""
    prob = CASES["3d-lenses-33"]()
    out = {}
    _tail_env(monkeypatch, mode)
    for tail in ("0", "100000"):
        monkeypatch.setenv("RF_TAIL_NV", tail)
        g, F = _assembled(prob)
        g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(_levels(prob), smoother, precision=precision))
        b = torch.tensor(F, device="cuda")
        x = torch.empty_like(b)
        info = g.solve(0, b, x, rtol=1e-11, max_it=300)
        torch.cuda.synchronize()
        assert info["status"] == 0, info
        out[tail] = (x.cpu().numpy(), info)
        g.close()
    (x0, i0), (x1, i1) = out["0"], out["100000"]
    assert i0 == i1 and np.array_equal(x0, x1)


def test_grid_barrier_completes_and_times_out():
    """The bounded grid barrier of the cooperative tail (rf_barrier_check):
    1000 rounds over every co-resident block complete; a barrier that expects
    one block more than the launch has never completes, so every wait gives
    up after its limit and the call returns RF_ETIMEOUT instead of hanging;
    the context stays usable (the next check completes)."""
    import time
    st, blocks = rf.rf_barrier_check(1000, 0, 1.0)
    assert st == rf.RF_OK and blocks >= 152, (st, blocks)
    t0 = time.perf_counter()
    st, _ = rf.rf_barrier_check(3, 1, 0.2)
    dt = time.perf_counter() - t0
    assert st == rf.RF_ETIMEOUT, st
    assert 0.15 <= dt <= 5.0, dt
    st, _ = rf.rf_barrier_check(10, 0, 1.0)
    assert st == rf.RF_OK
    for bad in ((0, 0, 1.0), (1, 2, 1.0), (1, 0, 0.0), (1, 0, 11.0)):
        assert rf.rf_barrier_check(*bad)[0] == rf.RF_EINVAL


# ------------------------------------------------------------------ solves
@pytest.mark.parametrize("precision,smoother", [("fp64", "jacobi"), ("fp32", "jacobi"), ("fp32", "gs8"),
                                                ("fp16", "gs8"), ("fp64", "gs8")])
@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "3d-9x7x5-stress", "2d-even-10x8", "3d-lenses-33"])
def test_solve_matches_oracle(case, precision, smoother):
    prob = CASES[case]()
    g, F = _assembled(prob)
    shift = 1.0 / prob["H"]
    L = _levels(prob)
    g.gmg_setup([shift], rf.gmg_opts(L, smoother, precision=precision))
    b = torch.tensor(F, device="cuda")
    x = torch.empty_like(b)
    info = g.solve(0, b, x, rtol=1e-12, max_it=300)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["relres"] <= 1e-12, info
    m = O.Model(prob)
    _, J_o, md_o = O.assemble(m, prob["u0"])
    A = O.make_A(J_o, md_o, shift)
    gm = O.GMG(m.dim, m.n, A, prob["dir"], L)
    x_o, inf_o = O.bicgstab(m.dim, m.n, A, gm, F, rtol=1e-13, maxit=400)
    assert inf_o["status"] == 0
    xs = x.cpu().numpy()
    # the oracle's own residual of the GPU solution
    r = F - O.spmv(m.dim, m.n, A, xs)
    assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(F)
    p_scale = np.abs(prob["u0"][0::2]).max()
    assert np.abs(xs[0::2] - x_o[0::2]).max() <= 1e-8 * p_scale
    assert np.abs(xs[1::2] - x_o[1::2]).max() <= 1e-9
    g.close()


@pytest.mark.parametrize("precision,smoother", [("fp32", "gs8"), ("fp64", "jacobi"), ("fp16", "gs8")])
def test_autotuned_block_sizes_give_identical_solves(precision, smoother, tmp_path, monkeypatch):
    """The autotuner only changes the thread-block size of the smoothing and
    residual kernels; every vertex's arithmetic is the same, so the solve is
    bitwise identical.  Its choices are appended to the RF_TUNE_CACHE file."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("RF_TUNE_CACHE", str(cache))
    prob = I.random_problem(3, (25, 13, 9), 11 + len(precision) + len(smoother))
    shift = 1.0 / prob["H"]
    L = _levels(prob)
    xs = []
    for tune in (False, True):
        g, F = _assembled(prob)
        g.gmg_setup([shift], rf.gmg_opts(L, smoother, precision=precision, autotune=tune))
        b = torch.tensor(F, device="cuda")
        x = torch.empty_like(b)
        info = g.solve(0, b, x, rtol=1e-11, max_it=300)
        torch.cuda.synchronize()
        assert info["status"] == 0, info
        xs.append(x.cpu().numpy())
        g.close()
    assert np.array_equal(xs[0], xs[1])
    if cache.exists():
        import json
        for line in cache.read_text().splitlines():
            e = json.loads(line)
            assert e["block"] in (64, 128, 256, 512), e


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("case", ["2d-lens-33", "3d-17cube", "3d-9x7x5-stress", "3d-lenses-33"])
def test_solve_with_double_fp32_operator_matches_oracle(case, precision):
    """RF_OUTER_DF32: the iteration's operator applications in double-FP32;
    the FP64 true residual still decides convergence."""
    prob = CASES[case]()
    g, F = _assembled(prob)
    shift = 1.0 / prob["H"]
    L = _levels(prob)
    g.gmg_setup([shift], rf.gmg_opts(L, "gs8", precision=precision))
    b = torch.tensor(F, device="cuda")
    x = torch.empty_like(b)
    info = g.solve(0, b, x, rtol=1e-12, max_it=300, outer="df32")
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["relres"] <= 1e-12, info
    m = O.Model(prob)
    _, J_o, md_o = O.assemble(m, prob["u0"])
    A = O.make_A(J_o, md_o, shift)
    xs = x.cpu().numpy()
    r = F - O.spmv(m.dim, m.n, A, xs)
    assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(F)
    g.close()


def test_solve_host_buffers_and_zero_rhs():
    prob = CASES["2d-lens-33"]()
    g, F = _assembled(prob)
    g.gmg_setup([0.1], rf.gmg_opts(4, precision="fp32"))
    x_host = np.zeros(2 * g.nv)
    info = g.solve(0, np.ascontiguousarray(F), x_host, rtol=1e-10)
    assert info["status"] == 0
    b = torch.tensor(F, device="cuda")
    x = torch.empty_like(b)
    g.solve(0, b, x, rtol=1e-10)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), x_host)
    z = np.zeros(2 * g.nv)
    x0 = np.ones(2 * g.nv)
    info = g.solve(0, z, x0)
    assert info["status"] == 0 and np.all(x0 == 0.0)
    g.close()


def test_invalid_arguments_are_rejected():
    prob = CASES["2d-lens-33"]()
    g = _grid(prob)
    with pytest.raises(rf.RFError) as e:
        g.solve(0, np.zeros(2 * g.nv), np.zeros(2 * g.nv))
    assert e.value.status == rf.RF_EINVAL
    with pytest.raises(rf.RFError):
        g.gmg_setup([0.1], rf.gmg_opts(4))       # no Jacobian yet
    u = torch.tensor(prob["u0"], device="cuda")
    g.assemble(u, True, None)
    with pytest.raises(rf.RFError):
        g.gmg_setup([0.1], rf.gmg_opts(0))
    with pytest.raises(rf.RFError):
        g.gmg_setup([0.1] * 5, rf.gmg_opts(2))
    g.gmg_setup([0.1], rf.gmg_opts(2))
    with pytest.raises(rf.RFError):
        g.solve(3, np.zeros(2 * g.nv), np.zeros(2 * g.nv))
    nc = prob["K"].size
    good = np.array([I.CASE2["laws"][0]])
    for laws, cells in ((np.zeros((5, 6)), np.zeros(nc)),                  # more than RF_MAX_KR_LAWS
                        (good, np.ones(nc)),                                # a cell names a missing law
                        (np.array([[2.0, 1, 1, 1, 1, 1]]), np.zeros(nc)),   # unknown kind
                        (np.array([[1.0, 1, 2.5, 1, 1, 1]]), np.zeros(nc)), # n_w not whole
                        (np.array([[1.0, -1, 2, 1, 1, 1]]), np.zeros(nc))): # a_w < 0
        with pytest.raises(rf.RFError) as e:
            g.set_kr_laws(laws, cells)
        assert e.value.status == rf.RF_EINVAL
    dev_laws = torch.tensor(good.ravel(), device="cuda")
    with pytest.raises(rf.RFError) as e:                                    # device pointers
        rf._check(rf.lib().rf_grid_set_kr_laws(g.handle, 1, dev_laws.data_ptr(), np.zeros(nc, np.uint8).ctypes.data,
                                               None))
    assert e.value.status == rf.RF_EINVAL
    g.set_kr_laws(good, np.zeros(nc))                                       # valid: drops J
    with pytest.raises(rf.RFError):
        g.gmg_setup([0.1], rf.gmg_opts(2))
    g.close()


def test_nonfinite_state_is_reported():
    prob = CASES["2d-lens-33"]()
    g, F = _assembled(prob)
    g.gmg_setup([0.1], rf.gmg_opts(4))
    b = F.copy()
    b[10] = np.nan
    with pytest.raises(rf.RFError) as e:
        g.solve(0, b, np.zeros_like(b))
    assert e.value.status == rf.RF_ENONFINITE
    g.close()


# ------------------------------------------------------------------ LIMEX
@pytest.mark.parametrize("kappa", [1, 2, 4])
def test_limex_step_matches_oracle(kappa):
    prob = I.random_problem(2, (17, 17), 31)
    H = 5.0
    g = _grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    info = g.limex_step(u, H, kappa=kappa, tol=1e9, gmg=rf.gmg_opts(3, precision="fp64"), rtol=1e-13, max_it=300)
    torch.cuda.synchronize()
    m = O.Model(prob)
    u_o, inf_o = O.limex_step(m, prob["u0"], H, kappa=kappa, tol=1e9, nlevels=3, rtol=1e-13, maxit=400)
    assert info["accepted"] == 1 and inf_o["accepted"] == 1
    assert info["solves"] == inf_o["solves"] == kappa * (kappa + 1) // 2
    us = u.cpu().numpy()
    assert np.abs(us[0::2] - u_o[0::2]).max() <= 1e-9 * np.abs(u_o[0::2]).max()
    assert np.abs(us[1::2] - u_o[1::2]).max() <= 1e-9
    if kappa > 1:
        assert info["eps"] == pytest.approx(inf_o["eps"], rel=1e-5)
        assert info["H_new"] == pytest.approx(inf_o["H_new"], rel=1e-5)
    g.close()


def _sequential_env(monkeypatch):
    """The step with its columns one after another (no batched rounds)."""
    monkeypatch.setenv("RF_LIMEX_BATCH", "0")
    monkeypatch.setenv("RF_LIMEX_CONCURRENT", "0")


def test_batched_ensemble_equals_sequential_steps(monkeypatch):
    """rf_limex_step_batched groups the problems of equal shape and solves the
    columns of all members of a group in shared batched rounds; every member's
    result is bitwise the one of its own step with sequential columns."""
    probs = [I.random_problem(3, (17, 17, 17), 41), I.random_problem(3, (9, 9, 9), 42),
             I.random_problem(2, (33, 33), 43), I.random_problem(3, (33, 17, 9), 44),
             I.random_problem(3, (17, 9, 9), 45), I.random_problem(3, (17, 17, 17), 46),
             I.random_problem(3, (9, 9, 9), 47), I.random_problem(3, (17, 17, 17), 49)]
    gm = [rf.gmg_opts(_levels(p), "jacobi", precision="fp32") for p in probs]
    seq = []
    _sequential_env(monkeypatch)
    for p, o in zip(probs, gm):
        g = _grid(p)
        u = torch.tensor(p["u0"], device="cuda")
        info = g.limex_step(u, 5.0, kappa=3, tol=1e9, gmg=o, rtol=1e-11)
        torch.cuda.synchronize()
        seq.append((u.cpu().numpy(), info))
        g.close()
    monkeypatch.delenv("RF_LIMEX_BATCH")
    monkeypatch.delenv("RF_LIMEX_CONCURRENT")
    grids = [_grid(p) for p in probs]
    us = [torch.tensor(p["u0"], device="cuda") for p in probs]
    for rep in range(2):   # the second call re-captures after the new set-ups
        for u, p in zip(us, probs):
            u.copy_(torch.tensor(p["u0"], device="cuda"))
        st, infos = rf.limex_step_batched(grids, us, 5.0, kappa=3, tol=1e9, gmg=gm, rtol=1e-11, max_concurrent=3)
        torch.cuda.synchronize()
        first_bad = next((i["status"] for _, i in seq if i["status"] != 0), 0)
        assert st == first_bad
        assert sum(i["status"] == 0 for _, i in seq) >= 6
        for (u_s, i_s), u_b, i_b in zip(seq, us, infos):
            assert i_b["status"] == i_s["status"]
            assert np.array_equal(u_s, u_b.cpu().numpy())
            assert i_b["iterations"] == i_s["iterations"] and i_b["eps"] == i_s["eps"]
            assert i_b["solves"] == i_s["solves"]
    for g in grids:
        g.close()


def test_adaptive_limex_conserves_napl_mass():
    """DNAPL infiltration recipe (Neumann NAPL inlet on top, Dirichlet p_w
    elsewhere) at 33^3: over adaptive LIMEX steps the NAPL mass grows exactly
    by the injected mass (every stage is a divergence-form balance, the
    extrapolation weights sum to one), up to the linear solves' residuals."""
    prob = I.dnapl_infiltration(33)
    g = _grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    m0 = g.phase_mass(u)[1]
    q = prob["q_in"][1::2].sum()
    t, hist = g.limex_run(u, 10.0, steps=4, tol=1e-3, gmg=rf.gmg_opts(prob["nlevels"], "gs8", precision="fp32"),
                          rtol=1e-12, max_it=400)
    torch.cuda.synchronize()
    m1 = g.phase_mass(u)[1]
    assert sum(h["accepted"] for h in hist) == 4 and t > 0
    err = abs(m1 - m0 - q * t) / m1
    assert err <= 1e-10, err
    g.close()


def test_limex_rejects_and_keeps_state():
    prob = I.random_problem(2, (17, 17), 32)
    g = _grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    u0 = u.clone()
    info = g.limex_step(u, 50.0, kappa=3, tol=1e-12, gmg=rf.gmg_opts(3, precision="fp32"))
    torch.cuda.synchronize()
    assert info["accepted"] == 0 and info["H_new"] < 50.0
    assert torch.equal(u, u0)
    g.close()


@pytest.mark.parametrize("precision,smoother,outer", [("fp64", "jacobi", "fp64"), ("fp32", "gs8", "fp64"),
                                                      ("fp16", "gs8", "fp64"), ("fp32", "gs8", "df32"),
                                                      ("fp32", "jacobi", "fp64")])
def test_limex_column_schedules_are_bitwise_equal(precision, smoother, outer, monkeypatch):
    """The LIMEX columns one after another, side by side on column grids (own
    vectors and streams), and in batched rounds (every active column's solve
    in the same launches, the shared J read once on the finest level) perform
    the same operations per column: the steps are bitwise equal."""
    prob = I.random_problem(3, (17, 17, 9), 44)
    modes = {"sequential": {"RF_LIMEX_BATCH": "0", "RF_LIMEX_CONCURRENT": "0"},
             "concurrent": {"RF_LIMEX_BATCH": "0", "RF_LIMEX_CONCURRENT": "1"},
             "batched": {"RF_LIMEX_BATCH": "1"}}
    out = {}
    for mode, env in modes.items():
        for k in ("RF_LIMEX_BATCH", "RF_LIMEX_CONCURRENT"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        g = _grid(prob)
        u = torch.tensor(prob["u0"], device="cuda")
        info = None
        for _ in range(2):   # second step reuses the column grids after a new set-up
            info = g.limex_step(u, 5.0, kappa=4, tol=1e9, gmg=rf.gmg_opts(3, smoother, precision=precision),
                                rtol=1e-11, max_it=300, outer=outer)
            assert info["status"] == 0, info
        torch.cuda.synchronize()
        out[mode] = (u.cpu().numpy(), info)
        g.close()
    for mode in ("concurrent", "batched"):
        assert np.array_equal(out["sequential"][0], out[mode][0]), mode
        assert out["sequential"][1]["iterations"] == out[mode][1]["iterations"], mode
        assert out["sequential"][1]["eps"] == out[mode][1]["eps"], mode


@pytest.mark.parametrize("dim,nv", [(2, (2, 2)), (2, (3, 2)), (3, (2, 2, 2)), (3, (3, 2, 3))])
def test_smallest_grids_assemble_and_solve(dim, nv):
    """Degenerate sizes: one element (2^d vertices) and one-element-thick
    grids; a one-level hierarchy is the dense coarsest solve itself.  (Dirichlet
    p_w on the top face: without any, the pressure is fixed only up to a
    constant and A = M/h - J is singular.)"""
    prob = I.random_problem(dim, nv, 45)
    g, F = _assembled(prob)
    J, md = g.export_jacobian()
    m = O.Model(prob)
    F_o, J_o, md_o = O.assemble(m, prob["u0"])
    assert np.abs(J - J_o).max() <= 1e-12 * np.abs(J_o).max()
    assert np.abs(F - F_o).max() <= 1e-12 * np.abs(F_o).max()
    shift = 1.0 / prob["H"]
    g.gmg_setup([shift], rf.gmg_opts(1, "jacobi", precision="fp64"))
    b = torch.tensor(F, device="cuda")
    x = torch.empty_like(b)
    info = g.solve(0, b, x, rtol=1e-12, max_it=50)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["iterations"] <= 2, info
    A = O.make_A(J_o, md_o, shift)
    r = F - O.spmv(m.dim, m.n, A, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(F)
    g.close()


def test_coarsest_level_size_limit_is_enforced():
    """A hierarchy whose coarsest level would exceed 4096 unknowns is refused
    at set-up (the dense inverse is sized for that), not run."""
    prob = I.random_problem(3, (17, 17, 17), 46)
    g, _ = _assembled(prob)
    with pytest.raises(rf.RFError) as e:
        g.gmg_setup([0.1], rf.gmg_opts(1))   # 17^3 x 2 = 9826 unknowns on one level
    assert e.value.status == rf.RF_EINVAL
    g.gmg_setup([0.1], rf.gmg_opts(2))       # 9^3 x 2 = 1458: fine
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plane_and_point_transfers_are_bitwise_equal(precision, monkeypatch):
    """The plane-indexed restriction / prolongation kernels gather the same
    values, apply the same masks and weights and sum in the same order as the
    per-point kernels (RF_TRANSFER_POINT=1): transfers on every level and a
    whole solve agree bitwise."""
    prob = I.random_problem(3, (17, 13, 9), 48)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("RF_TRANSFER_POINT", mode)
        g, F = _assembled(prob)
        g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(3, "gs8", precision=precision))
        res = []
        dims = [(17, 13, 9), (9, 7, 5), (5, 4, 3)]   # vertex-nested: n -> (n - 1) / 2 + 1
        for level in range(2):
            nv, nvc = int(np.prod(dims[level])), int(np.prod(dims[level + 1]))
            r = np.random.default_rng(7 + level).standard_normal(2 * nv)
            res.append(g.apply(rf.RF_OP_RESTRICT, level, 0, r)[:2 * nvc])
            xc = np.random.default_rng(9 + level).standard_normal(2 * nvc)
            x = np.random.default_rng(11 + level).standard_normal(2 * nv)
            res.append(g.apply(rf.RF_OP_PROLONG, level, 0, xc, x)[:2 * nv])
        b = torch.tensor(F, device="cuda")
        x = torch.empty_like(b)
        info = g.solve(0, b, x, rtol=1e-12, max_it=200)
        torch.cuda.synchronize()
        res.append(x.cpu().numpy())
        out[mode] = (res, info)
        g.close()
    assert out["0"][1] == out["1"][1] and out["0"][1]["status"] == 0
    for a, b_ in zip(out["0"][0], out["1"][0]):
        assert np.array_equal(a, b_)


def test_limex_run_matches_oracle_run():
    """rf_limex_run against the oracle's rfo_limex_run (same policy: hold
    after a rejection, H_max, landing on t_end) from a consistent state: the
    same accept / reject sequence, the step sizes and the final state."""
    prob = I.random_problem(2, (9, 9), 23)
    m = O.Model(prob)
    u0, inf = O.ie_step(m, prob["u0"], 1e-3, nlevels=2, atol=0.0, rtol=1e-11, lin_rtol=1e-14, max_newton=40)
    assert inf["status"] == 0
    kw = dict(t_end=3000.0, H_max=600.0, tol=1e-3, kappa=3)
    u_o, info_o, hist_o = O.limex_run(m, u0, 50.0, nlevels=2, rtol=1e-12, **kw)
    assert info_o["status"] == 0 and info_o["rejected"] >= 2
    g = _grid(prob)
    u = torch.tensor(u0, device="cuda")
    t, hist = g.limex_run(u, 50.0, gmg=rf.gmg_opts(2, "jacobi", precision="fp64"), rtol=1e-12, max_it=300, **kw)
    torch.cuda.synchronize()
    assert g.last_run["status"] == 0
    assert [h["accepted"] for h in hist] == [int(a) for a in hist_o[:, 2]]
    np.testing.assert_allclose([h["H"] for h in hist], hist_o[:, 0], rtol=1e-7)
    np.testing.assert_allclose([h["eps"] for h in hist], hist_o[:, 1], rtol=1e-5)
    assert t == pytest.approx(info_o["t"], rel=1e-12)
    us = u.cpu().numpy()
    assert np.abs(us[0::2] - u_o[0::2]).max() <= 1e-8 * np.abs(u_o[0::2]).max()
    assert np.abs(us[1::2] - u_o[1::2]).max() <= 1e-9
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_reversed_gs_colour_launches_are_bitwise_equal(precision, monkeypatch):
    """Multicolour Gauss-Seidel sweeps whose colour launches alternate the
    block order (the default; RF_GS_ZIGZAG=0 keeps every launch in order)
    update each vertex from the same neighbour values: a solve and a batched
    LIMEX step (the batched and shared-J smoother kernels) are bitwise equal."""
    prob = I.random_problem(3, (17, 13, 25), 52)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("RF_GS_ZIGZAG", mode)
        monkeypatch.setenv("RF_LIMEX_BATCH", "1")
        g, F = _assembled(prob)
        g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(3, "gs8", precision=precision))
        b = torch.tensor(F, device="cuda")
        x = torch.empty_like(b)
        sinfo = g.solve(0, b, x, rtol=1e-11, max_it=300)
        u = torch.tensor(prob["u0"], device="cuda")
        linfo = g.limex_step(u, 5.0, kappa=3, tol=1e9, gmg=rf.gmg_opts(3, "gs8", precision=precision),
                             rtol=1e-11, max_it=300)
        torch.cuda.synchronize()
        assert sinfo["status"] == 0 and linfo["status"] == 0, (mode, sinfo, linfo)
        out[mode] = (x.cpu().numpy(), sinfo, u.cpu().numpy(), linfo["iterations"], linfo["eps"])
        g.close()
    a, b_ = out["0"], out["1"]
    assert np.array_equal(a[0], b_[0]) and a[1] == b_[1]
    assert np.array_equal(a[2], b_[2]) and a[3:] == b_[3:]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("shape,dim,tail", [((17, 13, 25), 3, "0"), ((33, 9, 17), 3, "default"),
                                            ((9, 17, 5), 3, "0"), ((65, 33), 2, "0")])
def test_colour_pair_launches_are_bitwise_equal(precision, shape, dim, tail, monkeypatch):
    """Colours (0,py,pz) and (1,py,pz) reach each other only on their own
    x-line, so the GS launches that sweep such a pair in one kernel (a block
    barrier between the even- and the odd-x run of each line; the default)
    update every vertex from the same neighbour values as one launch per
    colour (RF_GS_PAIRS=0).  Whole solves (forward sweeps from zero, forward
    and backward sweeps on every smoothed level) and one forward sweep of
    each smoothed level are bitwise equal.  The shapes cover 2D and 3D,
    several line lengths, and the small levels launched one by one
    (RF_TAIL_NV=0) or in the one-launch tail."""
    prob = I.random_problem(dim, shape if dim == 3 else shape + (1,), 61)
    levels = _levels(prob)
    assert levels >= 2
    dims = [tuple(prob["n"][:dim])]
    for _ in range(levels - 1):
        dims.append(tuple((t - 1) // 2 + 1 for t in dims[-1]))
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("RF_GS_PAIRS", mode)
        if tail == "0":
            monkeypatch.setenv("RF_TAIL_NV", "0")
        else:
            monkeypatch.delenv("RF_TAIL_NV", raising=False)
        g, F = _assembled(prob)
        g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(levels, "gs8", precision=precision))
        b = torch.tensor(F, device="cuda")
        x = torch.empty_like(b)
        sinfo = g.solve(0, b, x, rtol=1e-11, max_it=300)
        torch.cuda.synchronize()
        assert sinfo["status"] == 0, (mode, sinfo)
        rng = np.random.default_rng(7)
        sweeps = []
        for lev in range(levels - 1):
            nv = int(np.prod(dims[lev]))
            bl = rng.standard_normal(2 * nv)
            xl = rng.standard_normal(2 * nv)
            sweeps.append(g.apply(rf.RF_OP_SMOOTH, lev, 0, bl, xl)[:2 * nv])
        out[mode] = (x.cpu().numpy(), sinfo["iterations"], sweeps)
        g.close()
    a, c = out["0"], out["1"]
    assert a[1] == c[1] and np.array_equal(a[0], c[0])
    for lev, (s0, s1) in enumerate(zip(a[2], c[2])):
        assert np.array_equal(s0, s1), lev


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_colour_pair_launches_in_batched_paths_are_bitwise_equal(precision, monkeypatch):
    """The colour-pair GS launches of the batched kernels: a LIMEX step whose
    columns run in batched rounds on one shared Jacobian (the shared-matrix
    kernels) and an ensemble step over grids of equal and unequal shapes (the
    per-system batched kernels) are bitwise those of one launch per colour."""
    one = I.random_problem(3, (17, 13, 25), 62)
    probs = [I.random_problem(3, (17, 17, 17), 63), I.random_problem(3, (17, 17, 17), 64),
             I.random_problem(3, (9, 9, 9), 65), I.random_problem(2, (33, 33), 66)]
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("RF_GS_PAIRS", mode)
        monkeypatch.setenv("RF_LIMEX_BATCH", "1")
        g = _grid(one)
        u = torch.tensor(one["u0"], device="cuda")
        info = g.limex_step(u, 5.0, kappa=3, tol=1e9, gmg=rf.gmg_opts(_levels(one), "gs8", precision=precision),
                            rtol=1e-11, max_it=300)
        torch.cuda.synchronize()
        assert info["status"] == 0, (mode, info)
        res = [(u.cpu().numpy(), info["iterations"], info["eps"])]
        g.close()
        monkeypatch.delenv("RF_LIMEX_BATCH")
        grids = [_grid(p) for p in probs]
        us = [torch.tensor(p["u0"], device="cuda") for p in probs]
        gm = [rf.gmg_opts(_levels(p), "gs8", precision=precision) for p in probs]
        st, infos = rf.limex_step_batched(grids, us, 5.0, kappa=3, tol=1e9, gmg=gm, rtol=1e-11, max_concurrent=2)
        torch.cuda.synchronize()
        res += [(v.cpu().numpy(), i["iterations"], i["eps"], i["status"]) for v, i in zip(us, infos)]
        for gg in grids:
            gg.close()
        out[mode] = res
    for a, c in zip(out["0"], out["1"]):
        assert np.array_equal(a[0], c[0]) and a[1:] == c[1:]


def test_host_buffers_pinned_pageable_and_device_agree():
    """State and solution vectors may be device memory, page-locked host
    memory (read and written by the permutation kernels over the CPU-GPU
    interconnect) or pageable host memory (staged with copies): a solve and a
    LIMEX step give bitwise the same results for all three."""
    prob = I.random_problem(3, (17, 9, 13), 71)
    g, F = _assembled(prob)
    g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(_levels(prob), "gs8", precision="fp32"))
    n = F.size
    pinned_b = torch.empty(n, dtype=torch.float64, pin_memory=True)
    pinned_x = torch.empty(n, dtype=torch.float64, pin_memory=True)
    pinned_b.copy_(torch.from_numpy(F))
    xs = {}
    b_pg, x_pg = F.copy(), np.full(n, np.nan)
    info = g.solve(0, b_pg, x_pg, rtol=1e-11, max_it=300)
    assert info["status"] == 0
    xs["pageable"] = x_pg
    pinned_x.fill_(float("nan"))
    info = g.solve(0, pinned_b.numpy(), pinned_x.numpy(), rtol=1e-11, max_it=300)
    assert info["status"] == 0
    xs["pinned"] = pinned_x.numpy().copy()
    b_d = torch.tensor(F, device="cuda")
    x_d = torch.full_like(b_d, float("nan"))
    info = g.solve(0, b_d, x_d, rtol=1e-11, max_it=300)
    torch.cuda.synchronize()
    assert info["status"] == 0
    xs["device"] = x_d.cpu().numpy()
    assert np.array_equal(xs["pageable"], xs["pinned"]) and np.array_equal(xs["pageable"], xs["device"])
    g.close()
    us = {}
    for kind in ("pageable", "pinned", "device"):
        g = _grid(prob)
        if kind == "pageable":
            u = prob["u0"].copy()
        elif kind == "pinned":
            u = torch.empty(n, dtype=torch.float64, pin_memory=True)
            u.copy_(torch.from_numpy(prob["u0"]))
            u = u.numpy()
        else:
            u = torch.tensor(prob["u0"], device="cuda")
        info = g.limex_step(u, 5.0, kappa=2, tol=1e9, gmg=rf.gmg_opts(_levels(prob), "gs8", precision="fp32"),
                            rtol=1e-11, max_it=300)
        torch.cuda.synchronize()
        assert info["status"] == 0, (kind, info)
        us[kind] = u.cpu().numpy() if kind == "device" else np.array(u, copy=True)
        g.close()
    assert np.array_equal(us["pageable"], us["pinned"]) and np.array_equal(us["pageable"], us["device"])


def test_shared_memory_tails_of_grids_of_different_sizes():
    """Grids whose one-launch tails keep different amounts of matrix data in
    shared memory share the tail kernel: a solve on the larger grid after the
    smaller grid's set-up (and the other way round) succeeds and repeats its
    first result bit for bit."""
    big = CASES["3d-lenses-33"]()        # tail from 17^3: ~169 KB per CTA
    small = CASES["3d-17cube"]()         # tail from 9^3: ~24 KB per CTA
    grids, res = {}, {}
    for name, prob in (("big", big), ("small", small)):
        g, F = _assembled(prob)
        g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(_levels(prob), "gs8", precision="fp32"))
        grids[name] = (g, torch.tensor(F, device="cuda"))
    for rep in range(2):
        for name in ("big", "small"):
            g, b = grids[name]
            x = torch.empty_like(b)
            info = g.solve(0, b, x, rtol=1e-11, max_it=300)
            torch.cuda.synchronize()
            assert info["status"] == 0, (name, info)
            if rep == 0:
                res[name] = (x.cpu().numpy(), info["iterations"])
            else:
                assert np.array_equal(res[name][0], x.cpu().numpy()) and res[name][1] == info["iterations"]
    for g, _ in grids.values():
        g.close()
