"""snect_foldin_static: the fold-in entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc (a process working inside another
framework's memory budget, a serving loop that must not stall on the allocator, code that
keeps every device buffer pre-reserved): they pass the frozen factors, the query and the
output row as their own device buffers, and the library works in a fixed device array of its
own.  This test calls it through the C ABI twice in a row and checks each result against
snect_foldin (the context-based entry point) within the fold-in tolerance of the other tests
(1e-3 relative, norm-wise).  The file is collected last so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import snect_synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-3


def test_static_foldin_matches_context_foldin_twice(gpu_lib):
    import torch

    import paper_1711_08095_gb300 as snect

    m = S.serving_model(I=(600, 2000, 5), J=(16, 16, 5))
    G, (U1, U2, U3) = m.G, m.U
    idx = np.array([[0, 0, 0], [1, 1, 1]], np.int32)
    ctx = snect.Snect((U1.shape[0], U2.shape[0], U3.shape[0]), G.shape, idx, np.zeros(2, np.float32),
                      np.zeros((0, 2), np.int32), np.zeros(0, np.float32), G, m.U, lam=m.lam, lam_g=0.0,
                      lr=0.01, batch=1)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dG, dU2, dU3 = dev(G), dev(U2), dev(U3)
    stream = torch.cuda.current_stream().cuda_stream
    lib = snect.load()
    for q, size in ((1, 9000), (2, 5000)):  # two calls in a row, different sizes
        jk, x, _ = S.serving_query(m, q=q, size=size)
        want = ctx.foldin(jk, x)
        djk, dx = dev(jk), dev(x)
        du = torch.full((G.shape[0],), float("nan"), device="cuda")
        rc = lib.snect_foldin_static(dG.data_ptr(), dU2.data_ptr(), dU3.data_ptr(), U2.shape[0], U3.shape[0],
                                     G.shape[0], G.shape[1], G.shape[2], djk.data_ptr(), dx.data_ptr(),
                                     jk.shape[0], ctypes.c_float(m.lam), du.data_ptr(), stream)
        assert rc == 0, lib.snect_last_error(None).decode()
        got = du.cpu().numpy()
        assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want), (q, got, want)
    # a query above the fixed limit is refused with a clear error, and nothing runs
    big = 1 << 20
    rc = lib.snect_foldin_static(dG.data_ptr(), dU2.data_ptr(), dU3.data_ptr(), U2.shape[0], U3.shape[0],
                                 G.shape[0], G.shape[1], G.shape[2], djk.data_ptr(), dx.data_ptr(), big + 1,
                                 ctypes.c_float(m.lam), du.data_ptr(), stream)
    assert rc == -1 and b"1,048,576" in lib.snect_last_error(None)
    ctx.close()
