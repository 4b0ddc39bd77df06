"""GPU fold-in (Eq. 9) and top-k search (Sec. 3.2.1) against the FP64 oracle.

Fold-in: the GPU sums the J1 x J1 Gram in FP32 (fixed order) and solves in FP64; against the
oracle's FP64 solve the row must agree to 1e-3 relative (norm-wise): the Gram's FP32 sum over
up to 75,000 cells carries ~1e-6 relative error, amplified by the system's condition number.
Top-k: the GPU scores in FP32; the returned rows must be a valid top-k under the oracle's FP64
scores within 1e-5, in non-increasing order, and equal to the oracle's rows wherever the
oracle's consecutive scores differ by more than that.
"""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(gpu_lib):
    import paper_1711_08095_gb300 as snect

    m = S.serving_model(I=(1200, 3000, 5), J=(16, 16, 5))
    G, U = m.G, m.U
    # a context holding the frozen factors (entries are irrelevant for serving)
    idx = np.array([[0, 0, 0], [1, 1, 1]], np.int32)
    c = snect.Snect(m.U[0].shape[0:1] + m.U[1].shape[0:1] + m.U[2].shape[0:1], G.shape, idx,
                    np.zeros(2, np.float32), np.zeros((0, 2), np.int32), np.zeros(0, np.float32), G, U,
                    lam=m.lam, lam_g=0.0, lr=0.01, batch=1)
    yield m, c
    c.close()


@pytest.mark.parametrize("n", [1, 17, 256, 4097, 15000])
def test_foldin_matches_oracle(served, n):
    m, c = served
    jk, x, u_true = S.serving_query(m, q=n, size=n)
    got = c.foldin(jk, x)
    want = oracle.foldin(m.G, m.U[1], m.U[2], jk, x, m.lam)
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want), (got, want)
    if n >= 4097:  # many cells: the fold-in recovers the planted row up to the noise
        assert np.linalg.norm(got - u_true) <= 0.1 * np.linalg.norm(u_true)


def test_foldin_matches_oracle_at_the_largest_query(gpu_lib):
    """The serving workload's largest query: 75,000 cells (every (gene, platform) pair of a
    15,000 x 5 model), 293 partial-sum CTAs of 256 cells."""
    import paper_1711_08095_gb300 as snect

    m = S.serving_model(I=(600, 15000, 5), J=(16, 16, 5))
    idx = np.array([[0, 0, 0], [1, 1, 1]], np.int32)
    c = snect.Snect((600, 15000, 5), m.G.shape, idx, np.zeros(2, np.float32), np.zeros((0, 2), np.int32),
                    np.zeros(0, np.float32), m.G, m.U, lam=m.lam, lam_g=0.0, lr=0.01, batch=1)
    jk, x, u_true = S.serving_query(m, q=75, size=75000)
    got = c.foldin(jk, x)
    c.close()
    want = oracle.foldin(m.G, m.U[1], m.U[2], jk, x, m.lam)
    assert jk.shape[0] == 75000
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want), (got, want)
    assert np.linalg.norm(got - u_true) <= 0.1 * np.linalg.norm(u_true)


def test_foldin_is_the_same_alone_and_repeated(served):
    m, c = served
    jk, x, _ = S.serving_query(m, q=3, size=9000)
    a = c.foldin(jk, x)
    jk2, x2, _ = S.serving_query(m, q=4, size=3000)
    c.foldin(jk2, x2)
    b = c.foldin(jk, x)
    assert np.array_equal(a, b)


def check_topk(m, c, k):
    jk, x, _ = S.serving_query(m, q=100 + k, size=5000)
    u = c.foldin(jk, x)
    idx, sc = c.topk(u, k)
    U1 = m.U[0].astype(np.float64)
    ref = (U1 @ u.astype(np.float64)) / (np.linalg.norm(U1, axis=1) * np.linalg.norm(u.astype(np.float64)))
    oi, osc = oracle.topk(U1, u, k)
    tol = 1e-5
    assert np.all(np.diff(sc) <= 0)
    assert np.allclose(sc, ref[idx], atol=tol)
    assert len(set(idx.tolist())) == k
    assert ref[idx].min() >= osc[-1] - tol
    for t in range(k):
        sep = (t == 0 or osc[t - 1] - osc[t] > tol) and (t == k - 1 or osc[t] - osc[t + 1] > tol)
        if sep:
            assert idx[t] == oi[t]


@pytest.mark.parametrize("k", [1, 10, 64])
def test_topk_matches_oracle(served, k):
    check_topk(*served, k)


def test_bad_queries_are_rejected(served):
    import paper_1711_08095_gb300 as snect

    m, c = served
    jk, x, _ = S.serving_query(m, q=7, size=100)
    bad = jk.copy()
    bad[5, 0] = m.U[1].shape[0]
    with pytest.raises(snect.SnectError):
        c.foldin(bad, x)
    for col, v in ((0, -1), (1, -1), (1, m.U[2].shape[0])):  # gene below, platform either side
        bad = jk.copy()
        bad[99, col] = v  # the last cell of the last CTA
        with pytest.raises(snect.SnectError):
            c.foldin(bad, x)
    xn = x.copy()
    xn[3] = np.inf
    with pytest.raises(snect.SnectError):
        c.foldin(jk, xn)
    with pytest.raises(snect.SnectError):
        c.topk(np.ones(16, np.float32), 0)
    # the context still works after rejected calls
    assert np.isfinite(c.foldin(jk, x)).all()
