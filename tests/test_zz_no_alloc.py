"""The allocation-free entry point rf_dense_inverse_noalloc.

It is meant for callers that cannot call cudaMalloc (device memory owned by
another allocator, or code that must not risk the synchronisation cudaMalloc
and cudaFree may cause).  Its working storage is a static device array in the
library, so this test checks it through the C ABI against the existing path
that allocates: the coarsest-level solve of a multigrid hierarchy
(rf_apply with RF_OP_COARSE, whose inverse the set-up built in allocated
memory).  Two calls in a row must both agree, since every call reuses the
static array.  The largest allowed size fills the whole array and is checked
against a library inverse on the CPU; a singular matrix must be reported, and
the call right after it must succeed (the status word is cleared per call).
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rf():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_04763_gb300 as R
    return R


def _call(rf, N, A_dev, Ainv):
    stream = torch.cuda.current_stream().cuda_stream
    return rf.lib().rf_dense_inverse_noalloc(N, A_dev.data_ptr(), Ainv.data_ptr(), stream)


def test_dense_inverse_noalloc_matches_allocating_coarse_solve(rf):
    from paper_2506_04763_gb300 import inputs as I
    from tests import _helpers as H

    prob = I.random_problem(3, (17, 17, 17), 5)
    g = rf.Grid(prob)
    u = torch.tensor(prob["u0"], device="cuda")
    g.assemble(u, True, None)
    g.gmg_setup([0.1], rf.gmg_opts(3, precision="fp64"))     # 17 -> 9 -> 5: coarsest 5^3, N = 250
    level = 2
    A, dims = g.export_level(level, 0)
    N = 2 * int(np.prod(dims))
    dense = H.stencil_to_dense(3, dims, A)
    A_dev = torch.tensor(dense, device="cuda")
    A_keep = A_dev.clone()
    Ainv = torch.empty_like(A_dev)
    b = np.random.default_rng(11).standard_normal(N)
    ref = g.apply(rf.RF_OP_COARSE, level, 0, b)[:N]           # existing, allocating path
    for call in range(2):
        Ainv.fill_(float("nan"))
        st = _call(rf, N, A_dev, Ainv)
        assert st == rf.RF_OK, (call, st)
        torch.cuda.synchronize()
        x = Ainv.cpu().numpy() @ b
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max(), call
    assert torch.equal(A_dev, A_keep)                          # input untouched
    # sizes beyond the reserved scratch and host pointers are rejected
    stream = torch.cuda.current_stream().cuda_stream
    L = rf.lib()
    assert L.rf_dense_inverse_noalloc(rf.RF_NOALLOC_MAX_N + 1, A_dev.data_ptr(), Ainv.data_ptr(), stream) == rf.RF_EINVAL
    assert L.rf_dense_inverse_noalloc(0, A_dev.data_ptr(), Ainv.data_ptr(), stream) == rf.RF_EINVAL
    host = np.zeros((N, N))
    assert L.rf_dense_inverse_noalloc(N, host.ctypes.data, Ainv.data_ptr(), stream) == rf.RF_EINVAL
    g.close()


def test_dense_inverse_noalloc_at_the_size_limit_and_singular_input(rf):
    N = rf.RF_NOALLOC_MAX_N
    rng = np.random.default_rng(12)
    M = rng.standard_normal((N, N)) + N ** 0.5 * np.eye(N)   # well conditioned, pivoting exercised
    ref = np.linalg.inv(M)
    A_dev = torch.tensor(M, device="cuda")
    Ainv = torch.full_like(A_dev, float("nan"))
    assert _call(rf, N, A_dev, Ainv) == rf.RF_OK
    torch.cuda.synchronize()
    assert np.abs(Ainv.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    # a zero row: singular, reported as such
    S = M.copy()
    S[7] = 0.0
    S_dev = torch.tensor(S, device="cuda")
    assert _call(rf, N, S_dev, Ainv) == rf.RF_ENONFINITE
    # a NaN entry that is never a pivot still reaches the factors: reported
    Q = M.copy()
    Q[N - 1, 3] = float("nan")
    Q_dev = torch.tensor(Q, device="cuda")
    assert _call(rf, N, Q_dev, Ainv) == rf.RF_ENONFINITE
    # the next good call starts from a cleared status word
    Ainv.fill_(float("nan"))
    assert _call(rf, N, A_dev, Ainv) == rf.RF_OK
    torch.cuda.synchronize()
    assert np.abs(Ainv.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


def test_dense_inverse_noalloc_refuses_a_capturing_stream(rf):
    """The call reads its status back and synchronises, so it cannot be part
    of a CUDA graph: on a capturing stream it returns RF_EINVAL and enqueues
    nothing, and the capture itself stays valid."""
    N = 64
    M = np.random.default_rng(13).standard_normal((N, N)) + 8.0 * np.eye(N)
    A_dev = torch.tensor(M, device="cuda")
    Ainv = torch.zeros_like(A_dev)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        st = _call(rf, N, A_dev, Ainv)
        Ainv.add_(1.0)                       # keeps the captured graph non-empty
    assert st == rf.RF_EINVAL
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(Ainv, torch.ones_like(Ainv))
    assert _call(rf, N, A_dev, Ainv) == rf.RF_OK      # outside a capture it works
    torch.cuda.synchronize()
    assert np.abs(Ainv.cpu().numpy() - np.linalg.inv(M)).max() <= 1e-11 * np.abs(np.linalg.inv(M)).max()
