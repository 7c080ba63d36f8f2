"""Full-size checks on the 257^3 benchmark workload, in the launch configuration
bench.py times (FP32 GMG, 7 levels, 8-colour GS), on outputs the oracle can
compute one by one.

The Jacobian row of vertex v depends only on the state and materials within
two cells of v (the faces of its elements, and p_dmin of their corners), so
the oracle assembles a 5x5x5-vertex sub-box around each sampled vertex and its
centre row must equal the GPU row of the full grid.  The solve is checked by
a property that holds at any size: every component of the oracle's residual
b - A x of the GPU solution x is bounded by the norm the solver guarantees,
|r_v| <= rtol |b|_2 (each component is at most the 2-norm).
"""
import numpy as np
import pytest

import oracle as O
from paper_2506_04763_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rf = pytest.importorskip("paper_2506_04763_gb300")

NV = 257


@pytest.fixture(scope="module")
def big():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    prob = I.lognormal_lenses_box(NV)
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    torch.cuda.synchronize()
    yield prob, g, F
    g.close()
    torch.cuda.empty_cache()


def _samples(prob, count=48, seed=0):
    n = prob["n"]
    rng = np.random.default_rng(seed)
    pts = [(int(rng.integers(0, n[0])), int(rng.integers(0, n[1])), int(rng.integers(0, n[2]))) for _ in range(count)]
    # corners, faces, the Dirichlet top and the NAPL blob under it
    pts += [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (n[0] // 2, n[1] // 2, n[2] - 1),
            (n[0] // 2, n[1] // 2, n[2] - 2), (n[0] // 2, n[1] // 2, n[2] - 9), (0, n[1] // 2, n[2] // 2)]
    # vertices on lens boundaries (p_d jumps): pick cells whose p_d differs from a neighbour's
    pd = prob["pd"].reshape(n[2] - 1, n[1] - 1, n[0] - 1)
    jump = np.argwhere(pd[:, :, 1:] != pd[:, :, :-1])
    for c in jump[rng.choice(len(jump), size=min(12, len(jump)), replace=False)]:
        pts.append((int(c[2]) + 1, int(c[1]), int(c[0])))
    return pts


def _subbox(prob, i, j, k, halo=2):
    """Sub-problem of vertices [c-halo, c+halo] per axis (clipped)."""
    n = prob["n"]
    lo = [max(0, c - halo) for c in (i, j, k)]
    hi = [min(n[a] - 1, c + halo) for a, c in enumerate((i, j, k))]
    sn = tuple(hi[a] - lo[a] + 1 for a in range(3))
    vz, vy, vx = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1), np.arange(lo[0], hi[0] + 1),
                             indexing="ij")
    vids = (vx + n[0] * (vy + n[1] * vz)).ravel()
    cz, cy, cx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]), indexing="ij")
    cids = (cx + (n[0] - 1) * (cy + (n[1] - 1) * cz)).ravel()
    u = np.empty(2 * len(vids))
    u[0::2] = prob["u0"][2 * vids]
    u[1::2] = prob["u0"][2 * vids + 1]
    sub = dict(prob)
    sub.update(n=sn, K=prob["K"][cids], phi=prob["phi"][cids], pd=prob["pd"][cids], dir=prob["dir"][vids],
               pw_dir=prob["pw_dir"][vids], u0=u, q_in=None)
    centre = (i - lo[0]) + sn[0] * ((j - lo[1]) + sn[1] * (k - lo[2]))
    return sub, centre, vids, lo, sn


def test_fullsize_jacobian_rows_match_oracle(big):
    prob, g, F = big
    n = prob["n"]
    pts = _samples(prob)
    verts = np.array([i + n[0] * (j + n[1] * k) for i, j, k in pts], np.int64)
    Jg, mdg = g.export_rows(verts)
    Fg = F.cpu().numpy()
    for r, (i, j, k) in enumerate(pts):
        sub, c, vids, lo, sn = _subbox(prob, i, j, k)
        Fo, Jo, mdo = O.assemble(O.Model(sub), sub["u0"])
        row = np.zeros((27, 4))
        for b in range(27):
            dx, dy, dz = b % 3 - 1, (b // 3) % 3 - 1, b // 9 - 1
            ii, jj, kk = i + dx, j + dy, k + dz
            if 0 <= ii < n[0] and 0 <= jj < n[1] and 0 <= kk < n[2]:
                row[b] = Jo[c, b]
        for a in range(2):
            scale = np.abs(row[:, 2 * a:2 * a + 2]).max() + 1e-300
            assert np.abs(Jg[r, :, 2 * a:2 * a + 2] - row[:, 2 * a:2 * a + 2]).max() <= 1e-12 * scale, (i, j, k, a)
        np.testing.assert_allclose(mdg[r], mdo[c], rtol=1e-14)
        fsc = np.abs(Fo).max() + 1e-300
        assert np.abs(Fg[2 * verts[r]:2 * verts[r] + 2] - Fo[2 * c:2 * c + 2]).max() <= 1e-12 * fsc, (i, j, k)


def test_fullsize_fp32_solve_residual_rows_and_fp64_agreement(big):
    prob, g, F = big
    n = prob["n"]
    shift = 1.0 / prob["H"]
    L = I.levels_for(NV)
    x = torch.empty_like(F)
    g.gmg_setup([shift], rf.gmg_opts(L, "gs8", precision="fp32"))
    info = g.solve(0, F, x, rtol=1e-10, max_it=100)
    assert info["status"] == 0 and info["relres"] <= 1e-10
    xs = x.cpu().numpy()
    b = F.cpu().numpy()
    bnorm = np.linalg.norm(b)
    for (i, j, k) in _samples(prob, count=24, seed=1):
        sub, c, vids, lo, sn = _subbox(prob, i, j, k)
        Fo, Jo, mdo = O.assemble(O.Model(sub), sub["u0"])
        A = O.make_A(Jo, mdo, shift)
        xsub = np.empty(2 * len(vids))
        xsub[0::2] = xs[2 * vids]
        xsub[1::2] = xs[2 * vids + 1]
        Ax = O.spmv(3, sn, A, xsub)
        v = i + n[0] * (j + n[1] * k)
        r = b[2 * v:2 * v + 2] - Ax[2 * c:2 * c + 2]
        assert np.abs(r).max() <= 1.01e-10 * bnorm, (i, j, k, r)
    # the all-FP64 preconditioner gives the same solution to the target tolerances
    g.gmg_setup([shift], rf.gmg_opts(L, "gs8", precision="fp64"))
    x64 = torch.empty_like(F)
    info64 = g.solve(0, F, x64, rtol=1e-10, max_it=100)
    assert info64["status"] == 0
    d = (x - x64).abs().cpu().numpy()
    assert d[0::2].max() <= 1e-8 * np.abs(prob["u0"][0::2]).max()
    assert d[1::2].max() <= 1e-7
