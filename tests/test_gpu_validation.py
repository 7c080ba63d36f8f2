"""Validation of the GPU time integrators on the paper's Cases 1 and 2 (Sec.
6): Buckley-Leverett (Tables case1 / error1) against the textbook
fractional-flow solution, and the extended Buckley-Leverett problem through two
media with their own polynomial relative permeabilities (Tables case2 /
error2) against its solution by characteristics, next to the paper's printed
error norms.

Implicit Euler runs at Courant number 0.8 as in the paper (Case 2: the printed
step counts); LIMEX with rho 0.25, dt0 = 1 s, dt_max = 100 days and TOL 5e-2
(Case 1) or 1e-2 (Case 2).  The errors must sit within 10% (implicit Euler)
and 25% (LIMEX) of the printed ones, and fall under refinement at rates (log2
ratios) within 0.15 (implicit Euler) or 0.25 (LIMEX) of the printed rates.
LIMEX's step sequence follows its error estimate, whose scaled norm the paper
leaves open: the printed runs take 5-8 times the steps taken here, so the
time-discretisation share of the error, and with it the rate, differs more
(the printed LIMEX L1 rates of Case 2 themselves range from 0.70 to 0.46).
"""
import os

import numpy as np
import pytest

from paper_2506_04763_gb300 import inputs as I
from tests import _helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rf = pytest.importorskip("paper_2506_04763_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name="case1_error1.txt"):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
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


def _case1_exact(x):
    c = I.CASE1
    return H.buckley_leverett_sw(x, c["T"], c["q_out"] / c["rho"], c["phi"], c["mu"], c["mu"])[0]


def _case2_exact(x):
    c = I.CASE2
    return H.extended_buckley_leverett_sw(x, c["T"], c["q_out"] / c["rho"], c["phi"], c["mu_w"], c["mu_n"],
                                          c["laws"][0], c["laws"][1], c["x_if"])


CASES = {
    1: dict(c=I.CASE1, make=I.case1_buckley_leverett, exact=_case1_exact, tol=5e-2, table="case1_error1.txt"),
    2: dict(c=I.CASE2, make=I.case2_extended_buckley_leverett, exact=_case2_exact, tol=1e-2,
            table="case2_error2.txt"),
}


def _errors(case, prob, u, nx):
    c = CASES[case]["c"]
    sw = 1.0 - u[1::2].reshape(prob["n"][1], prob["n"][0])
    # the flow is one-dimensional up to the solvers' tolerances (LIMEX with
    # TOL 5e-2 lets the colour order of the smoother leave ~1e-3 across rows)
    assert np.abs(sw - sw.mean(axis=0)).max() <= 1e-2
    xv = np.arange(nx + 1) * c["L"] / nx
    s = sw.mean(axis=0)
    ex = CASES[case]["exact"]
    return H.lp_error_1d(xv, s, ex, 1), H.lp_error_1d(xv, s, ex, 2)


def _run(nx, scheme, case=1):
    cs = CASES[case]
    c = cs["c"]
    prob = cs["make"](nx)
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    gm = rf.gmg_opts(prob["nlevels"], "gs8", precision="fp64")
    if scheme == "ie":
        if case == 1:
            nst = int(np.ceil(c["T"] / (0.8 * (c["L"] / nx) / 1.84e-6)))
        else:
            nst = _table(cs["table"])[("ie", nx)][0]
        for _ in range(nst):
            info = g.ie_step(u, c["T"] / nst, atol=1e-9, rtol=1e-6, max_newton=30, gmg=gm, lin_rtol=1e-8, max_it=300)
            assert info["status"] == 0, info
        steps = nst
    else:
        t, hist = g.limex_run(u, 1.0, t_end=c["T"], tol=cs["tol"], rho=0.25, H_max=100 * 86400.0, gmg=gm,
                              rtol=1e-8, max_it=300, max_rejects=100000)
        assert t == pytest.approx(c["T"], rel=1e-12)
        steps = len(hist)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    g.close()
    return steps, _errors(case, prob, out, nx)


@pytest.mark.parametrize("case", [1, 2])
@pytest.mark.parametrize("scheme,sizes,tol,rtol", [("ie", (64, 128, 256), 0.10, 0.15),
                                                   ("limex", (64, 128), 0.25, 0.25)])
def test_errors_and_rates_match_the_paper(case, scheme, sizes, tol, rtol):
    rows = _table(CASES[case]["table"])
    res = {nx: _run(nx, scheme, case) for nx in sizes}
    print("case", case, scheme, {nx: (r[0], round(r[1][0], 3), round(r[1][1], 3)) for nx, r in res.items()})
    for nx in sizes:
        steps, (L1, L2) = res[nx]
        _, pL1, pL2 = rows[(scheme, nx)]
        assert L1 == pytest.approx(pL1, rel=tol) and L2 == pytest.approx(pL2, rel=tol), (nx, L1, L2)
    for a, b in zip(sizes, sizes[1:]):
        for k in (0, 1):
            rate = np.log2(res[a][1][k] / res[b][1][k])
            prate = np.log2(rows[(scheme, a)][1 + k] / rows[(scheme, b)][1 + k])
            assert abs(rate - prate) <= rtol, (scheme, a, k, rate, prate)
