"""Failure paths of the C ABI, each made on the host (no GPU fault is made):

  - an allocator callback that returns NULL -> RF_ENOMEM, and every buffer
    the library did get is handed back (during grid creation and during the
    multigrid set-up);
  - a solve limited to max_it = 2 -> RF_ENOTCONV with the info filled in;
  - a tolerance below what FP64 can attain (1e-20): the recursive residual
    passes, the true residual check fails, the iteration restarts from the
    current x, and after the restart limit the solve ends with
    RF_EBREAKDOWN ("a breakdown that a restart did not cure").
"""
import ctypes

import numpy as np
import pytest

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


class CountingAllocator:
    """PyTorch's caching allocator behind an rf_allocator that records every
    live buffer and returns NULL once `budget` allocations have been served."""

    def __init__(self, budget=None):
        self.budget = budget
        self.served = 0
        self.live = {}
        self.bad_frees = []
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            if self.budget is not None and self.served >= self.budget:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
            self.served += 1
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, nbytes, stream, ctx):
            # (an exception would not leave a ctypes callback: record instead)
            if self.live.pop(ptr, None) != int(nbytes):
                self.bad_frees.append(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.handle = rf.rf_allocator(rf.ALLOC_FN(_alloc), rf.FREE_FN(_free), None)


def test_allocator_null_during_grid_creation_returns_enomem_and_frees_all():
    prob = I.random_problem(3, (17, 17, 17), 5)
    full = CountingAllocator()
    g = rf.Grid(prob, allocator=full.handle)
    n_create = full.served
    g.close()
    assert n_create > 10 and not full.live
    for budget in (0, 1, n_create // 2, n_create - 1):
        A = CountingAllocator(budget)
        with pytest.raises(rf.RFError) as e:
            rf.Grid(prob, allocator=A.handle)
        assert e.value.status == rf.RF_ENOMEM, budget
        assert A.served == budget and not A.live and not A.bad_frees, (budget, len(A.live))


def test_allocator_null_during_multigrid_setup_returns_enomem_and_keeps_the_grid():
    prob = I.random_problem(3, (17, 17, 17), 6)
    A = CountingAllocator()
    g = rf.Grid(prob, allocator=A.handle)
    u = torch.tensor(prob["u0"], device="cuda")
    g.assemble(u, True, None)
    torch.cuda.synchronize()
    grid_bufs = dict(A.live)
    base = A.served
    g.gmg_setup([0.1], rf.gmg_opts(3, "gs8", precision="fp32"))
    n_setup = A.served - base
    assert n_setup > 5
    for extra in (0, n_setup // 2, n_setup - 1):
        A.budget = A.served + extra
        with pytest.raises(rf.RFError) as e:
            g.gmg_setup([0.1], rf.gmg_opts(3, "gs8", precision="fp32"))
        assert e.value.status == rf.RF_ENOMEM, extra
        assert A.live == grid_bufs, extra            # the hierarchy's buffers went back
    A.budget = None                                    # the grid is still usable
    g.gmg_setup([0.1], rf.gmg_opts(3, "gs8", precision="fp32"))
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    g.gmg_setup([0.1], rf.gmg_opts(3, "gs8", precision="fp32"))
    x = torch.empty_like(u)
    assert g.solve(0, F, x, rtol=1e-10)["status"] == rf.RF_OK
    g.close()
    assert not A.live and not A.bad_frees


def _solve_raw(g, b, x, rtol, max_it):
    opts = rf.rf_solve_opts(float(rtol), int(max_it), rf.RF_OUTER_FP64)
    info = rf.rf_solve_info()
    st = rf.lib().rf_solve(g.handle, 0, b.data_ptr(), x.data_ptr(), ctypes.byref(opts), ctypes.byref(info), g.stream)
    torch.cuda.synchronize()
    return st, info


def test_iteration_limit_returns_enotconv_with_info():
    prob = I.random_problem(3, (33, 17, 17), 7)
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(3, "jacobi", precision="fp32"))
    x = torch.full_like(u, float("nan"))
    st, info = _solve_raw(g, F, x, 1e-14, 2)
    assert st == rf.RF_ENOTCONV and info.status == rf.RF_ENOTCONV
    assert info.iterations == 2 and np.isfinite(info.relres) and 1e-14 < info.relres < 1.0
    xs = x.cpu().numpy()
    assert np.all(np.isfinite(xs)) and np.abs(xs).max() > 0     # the iterate is returned
    assert "no convergence" in rf.rf_last_error()
    g.close()


def test_unattainable_tolerance_ends_in_breakdown_after_restarts():
    prob = I.random_problem(3, (17, 17, 17), 8)
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    F = torch.empty_like(u)
    g.assemble(u, True, F)
    g.gmg_setup([1.0 / prob["H"]], rf.gmg_opts(3, "gs8", precision="fp64"))
    x = torch.empty_like(u)
    st, info = _solve_raw(g, F, x, 1e-20, 1000)
    assert st == rf.RF_EBREAKDOWN and info.status == rf.RF_EBREAKDOWN, (st, info.status, info.iterations)
    assert info.restarts == 21 and info.iterations < 1000
    assert np.isfinite(info.relres) and info.relres < 1e-12      # x is the converged iterate
    assert np.all(np.isfinite(x.cpu().numpy()))
    g.close()
