"""Whole-grid oracle parity on the benchmark's recipe (lognormal K seed 2 plus
six low-K lenses, h = 10 s, b = F(u0)), in the configuration bench.py times:
FP64 BiCGSTAB preconditioned by an FP32 V(2,2) cycle with 8-colour block
Gauss-Seidel, x0 = 0, true relative residual <= 1e-10.

At 129^3 vertices (4.3M unknowns) every output is compared with the oracle's:
F and every Jacobian entry (1e-12 of the row's largest entry), and the
solution against the oracle's FP64 BiCGSTAB-GMG solve taken to 1e-13, so that
the difference measures the GPU solution's own error.  Per component:
  p_w: relative to max |p_w| of the state (the reading of the target's
       "1e-8 relative"), and, printed beside it, relative to max |increment|;
  S_n: absolute (target 1e-7).
The same comparison at the benchmark's full 257^3 (34M unknowns) runs when
RF_ORACLE_257=1: the oracle then needs ~45 GB of host memory and minutes.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2506_04763_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rf = pytest.importorskip("paper_2506_04763_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    O.set_threads(len(os.sched_getaffinity(0)))


def _gpu_solve(prob, L):
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(L, "gs8", precision="fp32"))
    x = torch.empty_like(F)
    info = g.solve(0, F, x, rtol=1e-10, max_it=100)
    torch.cuda.synchronize()
    return g, F.cpu().numpy(), x.cpu().numpy(), info


def _compare(nv, check_jacobian):
    prob = I.lognormal_lenses_box(nv)
    L = I.levels_for(nv)
    g, Fg, xg, info = _gpu_solve(prob, L)
    assert info["status"] == 0 and info["relres"] <= 1e-10, info
    Jg = g.export_jacobian()[0] if check_jacobian else None
    g.close()
    del g
    torch.cuda.empty_cache()
    m = O.Model(prob)
    F_o, J_o, md_o = O.assemble(m, prob["u0"])
    for a in range(2):
        sc = np.abs(F_o[a::2]).max()
        assert np.abs(Fg[a::2] - F_o[a::2]).max() <= 1e-12 * sc, a
    if check_jacobian:
        for a in range(2):
            rows = np.abs(J_o[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2)) + 1e-300
            err = np.abs(Jg[:, :, 2 * a:2 * a + 2] - J_o[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2))
            assert np.all(err <= 1e-12 * rows), (a, (err / rows).max())
        del Jg
    A = O.make_A(J_o, md_o, 1.0 / prob["H"])
    del J_o
    gm = O.GMG(3, m.n, A, prob["dir"], L, smoother=O.GS8)
    x_o, inf_o = O.bicgstab(3, m.n, A, gm, F_o, rtol=1e-13, maxit=100)
    assert inf_o["status"] == 0, inf_o
    del gm
    # the oracle's residual of the GPU solution
    r = F_o - O.spmv(3, m.n, A, xg)
    relres_o = np.linalg.norm(r) / np.linalg.norm(F_o)
    dp = np.abs(xg[0::2] - x_o[0::2]).max()
    ds = np.abs(xg[1::2] - x_o[1::2]).max()
    p_state = np.abs(prob["u0"][0::2]).max()
    p_incr = np.abs(x_o[0::2]).max()
    res = dict(nv=nv, dofs=2 * nv ** 3, gpu_iterations=info["iterations"], gpu_relres=info["relres"],
               oracle_relres_of_gpu_solution=relres_o, oracle_iterations=inf_o["iterations"],
               p_err_rel_state=dp / p_state, p_err_rel_increment=dp / p_incr, s_err_abs=ds,
               max_abs_p_increment=p_incr, max_abs_s_increment=np.abs(x_o[1::2]).max())
    print("ORACLE-PARITY " + " ".join("%s=%.6g" % (k, v) for k, v in res.items()))
    assert relres_o <= 1.01e-10
    assert dp <= 1e-8 * p_state
    assert ds <= 1e-7
    return res


def test_whole_grid_parity_129():
    res = _compare(129, check_jacobian=True)
    # the increment itself to 1e-6 (measured ~1e-8: see the printed line)
    assert res["p_err_rel_increment"] <= 1e-6


@pytest.mark.skipif(os.environ.get("RF_ORACLE_257") != "1", reason="opt-in: RF_ORACLE_257=1 (45 GB host, minutes)")
def test_whole_grid_parity_257():
    _compare(257, check_jacobian=False)
