"""Validation of the GPU time integrators on the paper's Case 1
(Buckley-Leverett, Sec. 6, Tables case1 / error1) against the textbook
fractional-flow solution, next to the paper's printed error norms.

Implicit Euler runs at Courant number 0.8 as in the paper; LIMEX with TOL 5e-2,
rho 0.25, dt0 = 1 s, dt_max = 100 days.  The errors must sit within 10%
(implicit Euler) and 25% (LIMEX, whose step sequence depends on the error
estimator's norm) of the printed ones, and fall under refinement at rates
(log2 ratios) within 0.15 of the printed rates.
"""
import os

import numpy as np
import pytest

from paper_2506_04763_gb300 import inputs as I
from tests import _helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rf = pytest.importorskip("paper_2506_04763_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "case1_error1.txt")


def _table():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            t = line.split()
            if t and t[0] in ("ie", "limex"):
                rows[(t[0], int(t[1]))] = (int(t[2]), float(t[3]), float(t[4]))
    return rows


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _errors(prob, u, nx):
    c = I.CASE1
    sw = 1.0 - u[1::2].reshape(prob["n"][1], prob["n"][0])
    # the flow is one-dimensional up to the solvers' tolerances (LIMEX with
    # TOL 5e-2 lets the colour order of the smoother leave ~1e-3 across rows)
    assert np.abs(sw - sw.mean(axis=0)).max() <= 1e-2
    xv = np.arange(nx + 1) * c["L"] / nx
    q = c["q_out"] / c["rho"]
    exact = lambda x: H.buckley_leverett_sw(x, c["T"], q, c["phi"], c["mu"], c["mu"])[0]
    s = sw.mean(axis=0)
    return H.lp_error_1d(xv, s, exact, 1), H.lp_error_1d(xv, s, exact, 2)


def _run(nx, scheme):
    c = I.CASE1
    prob = I.case1_buckley_leverett(nx)
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    gm = rf.gmg_opts(prob["nlevels"], "gs8", precision="fp64")
    if scheme == "ie":
        nst = int(np.ceil(c["T"] / (0.8 * (c["L"] / nx) / 1.84e-6)))
        for _ in range(nst):
            info = g.ie_step(u, c["T"] / nst, atol=1e-9, rtol=1e-6, max_newton=30, gmg=gm, lin_rtol=1e-8, max_it=300)
            assert info["status"] == 0, info
        steps = nst
    else:
        t, hist = g.limex_run(u, 1.0, t_end=c["T"], tol=5e-2, rho=0.25, H_max=100 * 86400.0, gmg=gm, rtol=1e-8,
                              max_it=300, max_rejects=100000)
        assert t == pytest.approx(c["T"], rel=1e-12)
        steps = len(hist)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    g.close()
    return steps, _errors(prob, out, nx)


@pytest.mark.parametrize("scheme,sizes,tol", [("ie", (64, 128, 256), 0.10), ("limex", (64, 128), 0.25)])
def test_case1_errors_and_rates_match_the_paper(scheme, sizes, tol):
    rows = _table()
    res = {nx: _run(nx, scheme) for nx in sizes}
    print(scheme, {nx: (r[0], round(r[1][0], 3), round(r[1][1], 3)) for nx, r in res.items()})
    for nx in sizes:
        steps, (L1, L2) = res[nx]
        _, pL1, pL2 = rows[(scheme, nx)]
        assert L1 == pytest.approx(pL1, rel=tol) and L2 == pytest.approx(pL2, rel=tol), (nx, L1, L2)
    for a, b in zip(sizes, sizes[1:]):
        for k in (0, 1):
            rate = np.log2(res[a][1][k] / res[b][1][k])
            prate = np.log2(rows[(scheme, a)][1 + k] / rows[(scheme, b)][1 + k])
            assert abs(rate - prate) <= 0.15, (scheme, a, k, rate, prate)
