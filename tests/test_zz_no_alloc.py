"""The allocation-free entry point rf_dense_inverse_noalloc.

It is meant for callers that cannot call cudaMalloc (device memory owned by
another allocator, or code that must not risk the synchronisation cudaMalloc
and cudaFree may cause).  Its working storage is a static device array in the
library, so this test checks it through the C ABI against the existing path
that allocates: the coarsest-level solve of a multigrid hierarchy
(rf_apply with RF_OP_COARSE, whose inverse the set-up built in allocated
memory).  Two calls in a row must both agree, since every call reuses the
static array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_dense_inverse_noalloc_matches_allocating_coarse_solve():
    import __graft_entry__ as G
    G.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_04763_gb300 as rf
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
    stream = torch.cuda.current_stream().cuda_stream
    L = rf.lib()
    for call in range(2):
        Ainv.fill_(float("nan"))
        st = L.rf_dense_inverse_noalloc(N, A_dev.data_ptr(), Ainv.data_ptr(), stream)
        assert st == rf.RF_OK, (call, st)
        torch.cuda.synchronize()
        x = Ainv.cpu().numpy() @ b
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max(), call
    assert torch.equal(A_dev, A_keep)                          # input untouched
    # sizes beyond the reserved scratch and host pointers are rejected
    assert L.rf_dense_inverse_noalloc(rf.RF_NOALLOC_MAX_N + 1, A_dev.data_ptr(), Ainv.data_ptr(), stream) == rf.RF_EINVAL
    host = np.zeros((N, N))
    assert L.rf_dense_inverse_noalloc(N, host.ctypes.data, Ainv.data_ptr(), stream) == rf.RF_EINVAL
    g.close()
