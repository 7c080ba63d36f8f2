"""The exact hydrostatic state on the GPU (pin P5 and the upwind tie of
Sec. 3.2, Eqs. up_krw / up_krn: "tie >= 0 -> own vertex").

At hydrostatic p_w every water potential difference G(p_n) - rho_w g_k is zero
up to rounding, so the sign of T_w on each face is decided by rounding alone.
The kernels evaluate each face with the oracle's operation order and no fused
multiply-add, so they must take the same upwind, cap and clamp decisions:
the Jacobian rows match the oracle to 1e-12 of the row here too.  With
S_n = 0 the state is an equilibrium (F = 0 to rounding, and a LIMEX step
leaves it unchanged); with S_n = 0.3 and one entry pressure the water fluxes
tie on every face while the NAPL sinks.
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


def _hydrostatic(prob, sn):
    dim, n, h = prob["dim"], prob["n"], prob["h"]
    nv = int(np.prod(n))
    v = np.arange(nv)
    vert = ((v // n[0]) % n[1]) * h[1] if dim == 2 else (v // (n[0] * n[1])) * h[2]
    u = np.empty(2 * nv)
    u[0::2] = I.P_TOP + prob["rho_w"] * I.GRAV * (1.0 - vert)
    u[1::2] = sn
    prob = dict(prob)
    prob["u0"] = u
    prob["q_in"] = None
    return prob


def _case(name):
    if name == "lenses-33":
        return _hydrostatic(I.lognormal_lenses_box(33), 0.0)
    if name == "random-3d-17":
        return _hydrostatic(I.random_problem(3, (17, 17, 17), 21), 0.0)
    if name == "lens-2d-33":
        return _hydrostatic(I.lens_square_2d(), 0.0)
    if name == "one-pd-sn0.3":
        p = I.random_problem(3, (17, 13, 9), 22)
        p["pd"] = np.full_like(p["pd"], I.SAND["pd"])
        return _hydrostatic(p, 0.3)
    raise KeyError(name)


def _flux_scale(p):
    return p["K"].max() * p["rho_w"] ** 2 * I.GRAV / p["mu_w"] * p["h"][0] ** (p["dim"] - 1)


@pytest.mark.parametrize("case", ["lenses-33", "random-3d-17", "lens-2d-33", "one-pd-sn0.3"])
def test_hydrostatic_jacobian_rows_and_residual_match_oracle(case):
    p = _case(case)
    g = rf.Grid(p)
    u = torch.tensor(p["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()
    J, md = g.export_jacobian()
    F_o, J_o, md_o = O.assemble(O.Model(p), p["u0"])
    for a in range(2):
        rows = np.abs(J_o[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2)) + 1e-300
        err = np.abs(J[:, :, 2 * a:2 * a + 2] - J_o[:, :, 2 * a:2 * a + 2]).max(axis=(1, 2))
        assert np.all(err <= 1e-12 * rows), (case, a, (err / rows).max())
    np.testing.assert_allclose(md, md_o, rtol=1e-14, atol=0)
    flux = _flux_scale(p)
    # the water balance is zero to rounding on both sides (every T_w ties)
    assert np.abs(Fg[0::2]).max() <= 1e-11 * flux, np.abs(Fg[0::2]).max() / flux
    assert np.abs(F_o[0::2]).max() <= 1e-11 * flux
    if case == "one-pd-sn0.3":
        # NAPL sinks under buoyancy: a real flux, equal on both sides
        sc = np.abs(F_o[1::2]).max()
        assert sc > 1e-6 * flux
        assert np.abs(Fg[1::2] - F_o[1::2]).max() <= 1e-12 * sc
    else:
        assert np.abs(Fg[1::2]).max() <= 1e-11 * flux
    g.close()


@pytest.mark.parametrize("precision,smoother", [("fp64", "jacobi"), ("fp32", "gs8")])
@pytest.mark.parametrize("case", ["lenses-33", "random-3d-17"])
def test_hydrostatic_limex_step_leaves_the_state_unchanged(case, precision, smoother):
    p = _case(case)
    g = rf.Grid(p)
    u = torch.tensor(p["u0"], device="cuda")
    L = I.levels_for(p["n"][0]) if case == "lenses-33" else 3
    info = g.limex_step(u, 10.0, kappa=4, tol=1e-3, gmg=rf.gmg_opts(L, smoother, precision=precision), rtol=1e-12,
                        max_it=300)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["accepted"] == 1, info
    us = u.cpu().numpy()
    np.testing.assert_allclose(us[0::2], p["u0"][0::2], rtol=1e-12, atol=0)
    assert np.abs(us[1::2]).max() <= 1e-12
    g.close()
