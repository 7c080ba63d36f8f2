"""The workloads end to end against the oracle: the 65^3 lognormal cube (one
full FP64 LIMEX step) and one member of each size of the 64-realisation
ensemble (one LIMEX step with FP32 multigrid inside FP64 BiCGSTAB, at 33^3,
49^3, 65^3 and 97^3; the oracle runs with OpenMP on the host cores).  The
257^3 / 385^3 configurations are checked in test_gpu_oracle_fullsize.py and by
sampled rows and invariants in test_gpu_fullsize.py and test_gpu_parity.py.

Both sides solve every stage to a true relative residual of 1e-12; the LIMEX
results then agree to 1e-8 relative in p_w and 1e-9 absolute in S_n (the
extrapolation weights amplify the solvers' differences by at most ~30), and
the error estimates to 1e-5 relative.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2506_04763_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
rf = pytest.importorskip("paper_2506_04763_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    O.set_threads(len(os.sched_getaffinity(0)))


def _limex_parity(prob, precision, smoother, H=10.0):
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    info = g.limex_step(u, H, kappa=4, tol=1e9, gmg=rf.gmg_opts(prob["nlevels"], smoother, precision=precision),
                        rtol=1e-12, max_it=400)
    torch.cuda.synchronize()
    sm = O.GS8 if smoother == "gs8" else O.JACOBI
    u_o, inf_o = O.limex_step(O.Model(prob), prob["u0"], H, kappa=4, tol=1e9, nlevels=prob["nlevels"], smoother=sm,
                              rtol=1e-12, maxit=400)
    assert info["status"] == 0 and inf_o["status"] == 0, (info, inf_o)
    assert info["solves"] == inf_o["solves"] == 10
    us = u.cpu().numpy()
    assert np.abs(us[0::2] - u_o[0::2]).max() <= 1e-8 * np.abs(u_o[0::2]).max()
    assert np.abs(us[1::2] - u_o[1::2]).max() <= 1e-9
    assert info["eps"] == pytest.approx(inf_o["eps"], rel=1e-5)
    g.close()
    return info, inf_o


def test_lognormal_cube_65_limex_step_matches_oracle():
    """65^3 lognormal field (seed 1), kappa = 4, H = 10 s, FP64
    throughout with 5-level block-Jacobi multigrid."""
    info, inf_o = _limex_parity(I.lognormal_cube_65(), "fp64", "jacobi")
    print("65^3 LIMEX step: GPU iterations", info["iterations"], "oracle", inf_o["iterations"])


@pytest.mark.parametrize("seed,nvert", [(100, 33), (116, 49), (132, 65), (148, 97)])
def test_ensemble_member_limex_step_matches_oracle(seed, nvert):
    """Ensemble members (seed order: 33^3 for seeds 100..115, 49^3 for
    116..131, 65^3 for 132..147, 97^3 for 148..163): one LIMEX step with FP32
    multigrid inside FP64 BiCGSTAB."""
    _limex_parity(I.ensemble_member(seed, nvert), "fp32", "jacobi")
