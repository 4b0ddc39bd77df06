"""Downstream analyses on the GPU against the FP64 oracle, through the C ABI.

Personalised subtype matrix (Sec. 3.3): S = G x1 u, its row norms and the column norms of
S x3 U3, for a batch of patient profiles in one launch; every value within
1e-5 (|oracle| + rms) (FP32 sums of at most 32 terms against FP64).

k-means stratification of the patient profiles (Sec. 3.1.1): the assignment is an integer
decision, so both sides take it in FP64 in the same operation order (reading R14); the
assignments, the centroids and the number of updates must be bit-identical to the oracle's
Lloyd run from the same initial centroids, on planted clusters (which the run must recover)
and on overlapping ones that take many passes; the inertia within 1e-12 relative (the GPU
adds the rows' distances in another order).
"""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu


def frozen_ctx(G, U):
    import paper_1711_08095_gb300 as snect

    I = tuple(u.shape[0] for u in U)
    idx = np.array([[0, 0, 0], [1, 1, 1]], np.int32)
    return snect.Snect(I, G.shape, idx, np.zeros(2, np.float32), np.zeros((0, 2), np.int32),
                       np.zeros(0, np.float32), G, U, lam=0.01, lam_g=0.0, lr=0.01, batch=1)


def close(got, want):
    got = np.asarray(got, np.float64)
    rms = float(np.sqrt(np.mean(want * want)))
    return float((np.abs(got - want) / (np.abs(want) + rms + 1e-30)).max())


@pytest.mark.parametrize("J,I3", [((16, 16, 5), 5), ((32, 32, 5), 5), ((3, 7, 4), 9)])
def test_subtype_matches_oracle(J, I3, gpu_lib):
    m = S.serving_model(I=(700, 2000, I3), J=J)
    c = frozen_ctx(m.G, m.U)
    prof = np.concatenate([m.U[0], c.foldin(*S.serving_query(m, q=1, size=3000)[:2])[None]])  # 701 profiles
    Sg, rg, pg = c.subtype(prof)
    c.close()
    for i in (0, 1, 350, 699, 700):
        So, ro, po = oracle.subtype(m.G, m.U[2], prof[i])
        assert close(Sg[i], So) <= 1e-5 and close(rg[i], ro) <= 1e-5 and close(pg[i], po) <= 1e-5, i
    # every profile (checked in bulk against the oracle's definition, row by row)
    want = np.stack([oracle.subtype(m.G, m.U[2], u)[2] for u in prof])
    assert close(pg, want) <= 1e-5


@pytest.mark.parametrize("n,d,k,spread,recover", [(4500, 16, 13, 0.05, True), (3001, 10, 13, 0.9, False),
                                                   (1000, 32, 128, 0.5, False), (257, 5, 1, 0.3, False)])
def test_kmeans_bit_identical_to_oracle(n, d, k, spread, recover, gpu_lib):
    X, labels, init = S.clustered_profiles(n, d, k, spread=spread, seed=11)
    G = np.ones((d, 2, 1), np.float32)
    U = [X, np.ones((3, 2), np.float32), np.ones((2, 1), np.float32)]
    c = frozen_ctx(G, U)
    a, cent, upd, inertia = c.kmeans(init, 200)
    c.close()
    ao, co, uo, io = oracle.kmeans(X, init, 200)
    assert np.array_equal(a, ao) and np.array_equal(cent, co) and upd == uo, (upd, uo)
    assert abs(inertia - io) <= 1e-12 * io
    if recover:
        assert np.array_equal(a, labels)
    print("k-means n=%d d=%d k=%d: %d updates, inertia %.6g" % (n, d, k, upd, inertia))
