"""snect_foldin_static: the fold-in entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc (a process working inside another
framework's memory budget, a serving loop that must not stall on the allocator, code that
keeps every device buffer pre-reserved): they pass the frozen factors, the query and the
output row as their own device buffers, and the library works in a fixed device array of its
own.  These tests call it through the C ABI, two calls in a row per core shape, and check
each result against the FP64 oracle's fold-in (Eq. 9 with the ridge term) and against
snect_foldin (the context-based entry point), within the fold-in tolerance of the other
tests (1e-3 relative, norm-wise).  The core shapes span the accepted range up to 32 x 32 x 5
(J1*J2*J3 = 5,120, the largest core the entry point accepts) and the queries reach 75,000
cells, the largest query of the serving workload.  The file is collected last so that a run
stopping at the first failure has run every other test first; it also passes alone in a
fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-3
EINVAL = -1


def _call(lib, dG, dU2, dU3, shape, djk, dx, n, lam, du, stream):
    (I2, I3), (J1, J2, J3) = shape
    return lib.snect_foldin_static(dG.data_ptr(), dU2.data_ptr(), dU3.data_ptr(), I2, I3, J1, J2, J3,
                                   djk.data_ptr(), dx.data_ptr(), n, ctypes.c_float(lam), du.data_ptr(), stream)


@pytest.mark.parametrize("J", [(16, 16, 5), (32, 32, 5)])
def test_static_foldin_matches_oracle_twice(J, gpu_lib):
    import torch

    import paper_1711_08095_gb300 as snect

    m = S.serving_model(I=(600, 15000, 5), J=J)
    G, (U1, U2, U3) = m.G, m.U
    idx = np.array([[0, 0, 0], [1, 1, 1]], np.int32)
    ctx = snect.Snect((U1.shape[0], U2.shape[0], U3.shape[0]), G.shape, idx, np.zeros(2, np.float32),
                      np.zeros((0, 2), np.int32), np.zeros(0, np.float32), G, m.U, lam=m.lam, lam_g=0.0,
                      lr=0.01, batch=1)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dG, dU2, dU3 = dev(G), dev(U2), dev(U3)
    stream = torch.cuda.current_stream().cuda_stream
    lib = snect.load()
    shape = ((U2.shape[0], U3.shape[0]), G.shape)
    for q, size in ((1, 75000), (2, 5000)):  # two calls in a row, the largest query first
        jk, x, _ = S.serving_query(m, q=q, size=size)
        want = oracle.foldin(G, U2, U3, jk, x, m.lam)
        djk, dx = dev(jk), dev(x)
        du = torch.full((G.shape[0],), float("nan"), device="cuda")
        rc = _call(lib, dG, dU2, dU3, shape, djk, dx, jk.shape[0], m.lam, du, stream)
        assert rc == 0, lib.snect_last_error(None).decode()
        got = du.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want), (J, q, got, want)
        ref = ctx.foldin(jk, x)
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(want), (J, q)
    # a query above the fixed limit is refused with a clear error, and nothing runs
    big = 1 << 20
    rc = _call(lib, dG, dU2, dU3, shape, djk, dx, big + 1, m.lam, du, stream)
    assert rc == EINVAL and b"1,048,576" in lib.snect_last_error(None)
    ctx.close()


def test_static_foldin_device_errors_zero_the_row(gpu_lib):
    """The two errors only the GPU can see: a cell outside the factors, and a normal matrix
    that is not positive definite (lambda = 0 and every cell's w = 0, from a zero gene row).
    Both return SNECT_EINVAL with their message, and the output row is left at zero."""
    import torch

    import paper_1711_08095_gb300 as snect

    m = S.serving_model(I=(300, 2000, 5), J=(16, 16, 5))
    G, (_, U2, U3) = m.G, m.U
    U2 = U2.copy()
    U2[7] = 0.0
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dG, dU2, dU3 = dev(G), dev(U2), dev(U3)
    stream = torch.cuda.current_stream().cuda_stream
    lib = snect.load()
    shape = ((U2.shape[0], U3.shape[0]), G.shape)
    jk, x, _ = S.serving_query(m, q=11, size=3000)
    jk = jk.copy()
    jk[1234, 0] = U2.shape[0]  # a gene index one past the end
    du = torch.full((G.shape[0],), float("nan"), device="cuda")
    rc = _call(lib, dG, dU2, dU3, shape, dev(jk), dev(x), jk.shape[0], m.lam, du, stream)
    assert rc == EINVAL and b"out of range" in lib.snect_last_error(None)
    assert np.array_equal(du.cpu().numpy(), np.zeros(G.shape[0], np.float32))
    jk0 = np.array([[7, k] for k in range(5)], np.int32)  # gene 7's row is zero: every w = 0
    x0 = np.ones(5, np.float32)
    du.fill_(float("nan"))
    rc = _call(lib, dG, dU2, dU3, shape, dev(jk0), dev(x0), 5, 0.0, du, stream)
    assert rc == EINVAL and b"positive definite" in lib.snect_last_error(None)
    assert np.array_equal(du.cpu().numpy(), np.zeros(G.shape[0], np.float32))
    # a good call right after the failing ones gives the oracle's row
    jk, x, _ = S.serving_query(m, q=12, size=4000)
    du.fill_(float("nan"))
    rc = _call(lib, dG, dU2, dU3, shape, dev(jk), dev(x), jk.shape[0], m.lam, du, stream)
    assert rc == 0, lib.snect_last_error(None).decode()
    want = oracle.foldin(G, U2, U3, jk, x, m.lam)
    assert np.linalg.norm(du.cpu().numpy() - want) <= TOL * np.linalg.norm(want)
