"""GPU implicit Euler + Newton (rf_ie_step) against the oracle's rfo_ie_step.

Both sides converge Newton to a relative residual of 1e-10 with linear solves
to 1e-13; the solutions then agree to the Newton tolerance times the problem's
conditioning, checked as 1e-8 relative in p_w and 1e-9 absolute in S_n, and
the Newton iteration counts agree exactly.
"""
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


CASES = {
    "2d-17": lambda: I.random_problem(2, (17, 17), 41),
    "3d-9x9x5": lambda: I.random_problem(3, (9, 9, 5), 42),
    "3d-infiltration-17": lambda: I.dnapl_infiltration(17),
}


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("case", list(CASES))
def test_ie_step_matches_oracle(case, scheme):
    prob = CASES[case]()
    prob["scheme"] = scheme
    H = 20.0
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    info = g.ie_step(u, H, atol=0.0, rtol=1e-10, max_newton=30, gmg=rf.gmg_opts(2, precision="fp64"),
                     lin_rtol=1e-13, max_it=400)
    torch.cuda.synchronize()
    u_o, inf_o = O.ie_step(O.Model(prob), prob["u0"], H, atol=0.0, rtol=1e-10, max_newton=30, nlevels=2,
                           lin_rtol=1e-13, lin_maxit=400)
    assert info["status"] == 0 and inf_o["status"] == 0, (info, inf_o)
    assert info["newton"] == inf_o["newton"]
    assert info["res0"] == pytest.approx(inf_o["res0"], rel=1e-10)
    us = u.cpu().numpy()
    assert np.abs(us[0::2] - u_o[0::2]).max() <= 1e-8 * np.abs(u_o[0::2]).max()
    assert np.abs(us[1::2] - u_o[1::2]).max() <= 1e-9
    g.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_ie_conserves_napl_mass(scheme):
    """DNAPL inlet at 33^3: each implicit Euler step changes the NAPL mass by H
    times the injection, with the scheme's own storage (also the nonlinear S
    hat storage), up to H times the NAPL rows' Newton residual (bounded by
    sqrt(nv) ||R||_2).  The residual norm mixes kg/s rows with the Dirichlet
    rows' p_dir - p_w (Pa), whose rounding floor (~1e-11 Pa per row) is why
    the Newton tolerance is 1e-8 here."""
    prob = I.dnapl_infiltration(33)
    prob["scheme"] = scheme
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    m0 = g.phase_mass(u)[1]
    q = prob["q_in"][1::2].sum()
    H, steps, bound = 10.0, 3, 0.0
    for _ in range(steps):
        info = g.ie_step(u, H, atol=0.0, rtol=1e-8, max_newton=30,
                         gmg=rf.gmg_opts(prob["nlevels"], "gs8", precision="fp32"), lin_rtol=1e-12, max_it=400)
        assert info["status"] == 0, info
        bound += H * np.sqrt(g.nv) * info["res"]
    m1 = g.phase_mass(u)[1]
    assert abs(m1 - m0 - q * H * steps) <= bound + 1e-12 * q * H * steps
    assert bound <= 1e-5 * q * H * steps
    g.close()


def test_ie_nonconvergence_keeps_the_state():
    prob = CASES["2d-17"]()
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    info = g.ie_step(u, 20.0, atol=0.0, rtol=1e-14, max_newton=1, gmg=rf.gmg_opts(2, precision="fp64"))
    torch.cuda.synchronize()
    assert info["status"] == rf.RF_ENOTCONV and info["newton"] == 1
    assert np.array_equal(u.cpu().numpy(), prob["u0"])
    g.close()


@pytest.mark.parametrize("case,H", [("2d-17", 1000.0), ("3d-infiltration-9", 1000.0)])
def test_ie_line_search_matches_oracle(case, H):
    """Steps where the undamped Newton iteration fails and backtracking (at
    most 4 halvings) converges: same Newton count and solution on both sides."""
    prob = I.dnapl_infiltration(9) if case == "3d-infiltration-9" else CASES[case]()
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    info = g.ie_step(u, H, atol=0.0, rtol=1e-9, max_newton=40, gmg=rf.gmg_opts(2, precision="fp64"),
                     lin_rtol=1e-12, max_it=400, max_ls=4)
    torch.cuda.synchronize()
    u_o, inf_o = O.ie_step(O.Model(prob), prob["u0"], H, atol=0.0, rtol=1e-9, max_newton=40, nlevels=2,
                           lin_rtol=1e-12, lin_maxit=400, max_ls=4)
    assert info["status"] == 0 and inf_o["status"] == 0, (info, inf_o)
    assert info["newton"] == inf_o["newton"]
    us = u.cpu().numpy()
    assert np.abs(us[0::2] - u_o[0::2]).max() <= 1e-8 * np.abs(u_o[0::2]).max()
    assert np.abs(us[1::2] - u_o[1::2]).max() <= 1e-8
    g.close()
