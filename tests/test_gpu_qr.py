"""QR orthogonalisation post-pass on the GPU (snect_qr_post) against the FP64 oracle's
Householder QR: the same Q and R up to the signs of R's rows (Q's columns), predictions
unchanged, orthonormal factors; a mode with J_n > I_n is kept on both sides."""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu


def ctx(p, batch=0):
    import paper_1711_08095_gb300 as snect

    return snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                       batch=batch)


def sign_fix(Q, R):
    """Flips columns of Q and rows of R so that R has a nonnegative diagonal."""
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s, R * s[:, None]


@pytest.mark.parametrize("shape", [((30, 40, 6), (5, 4, 3)), ((4500, 15000, 5), (10, 10, 5))])
def test_qr_post_matches_oracle(shape, gpu_lib):
    I, J = shape
    if I[0] > 1000:  # the paper-scale shape, after an epoch of the fast mode
        p = S.config2(n_patients=4500, nnz=2_000_000, n_edges=20_000)
        c = ctx(p)
        c.epoch(1)
    else:
        p = S.tiny_problem(seed=7, I=I, J=J)
        c = ctx(p, batch=64)
    G0, U0 = c.get_factors()
    skipped = c.qr_post()
    G1, U1 = c.get_factors()
    c.close()
    assert skipped == 0
    P = oracle.Params(G0, U0)
    assert oracle.qr_post(p.I, P) == 0
    for n in range(3):
        Uo = np.asarray(U0[n], np.float64)
        Qg, Rg = sign_fix(np.asarray(U1[n], np.float64), np.asarray(U1[n], np.float64).T @ Uo)
        Qo, Ro = sign_fix(P.U[n], P.U[n].T @ Uo)
        assert np.abs(Qg.T @ Qg - np.eye(p.J[n])).max() < 1e-5
        assert np.abs(Qg - Qo).max() < 1e-4 * max(1.0, np.abs(Qo).max())
        assert np.abs(Rg - Ro).max() < 1e-4 * np.abs(Ro).max()
    # x~ unchanged (gauge invariance), checked on sampled entries
    s = p.idx[: min(5000, p.idx.shape[0])]
    before = oracle.predict(oracle.Params(G0, U0), s)
    after = oracle.predict(oracle.Params(G1, U1), s)
    assert np.abs(after - before).max() <= 1e-4 * max(1.0, np.abs(before).max())


def test_qr_post_keeps_a_mode_wider_than_tall(gpu_lib):
    p = S.config1(J_fit=(5, 5, 5))  # J3 = 5 > I3 = 4 platforms
    c = ctx(p, batch=1024)
    G0, U0 = c.get_factors()
    skipped = c.qr_post()
    G1, U1 = c.get_factors()
    c.close()
    assert skipped == 1 << 2
    assert np.array_equal(U1[2], U0[2])
    for n in range(2):
        assert np.abs(U1[n].T.astype(np.float64) @ U1[n] - np.eye(p.J[n])).max() < 1e-5
