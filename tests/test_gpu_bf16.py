"""BF16 precision form of the fast sweep (tcgen05 tensor cores, FP32 accumulation and FP32
master factors), through the C ABI.

The precision form refits config 1's tensor at core ranks 16 x 16 x 5 and 32 x 32 x 5.  It is
judged against the FP32 fast sweep from the same start: test RMSE within 1% ("equal RMSE"),
and its distance from the FP64 oracle's sequential run is reported (objective, test RMSE,
principal angles between factor column spaces).
"""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu


def ctx(p, precision, **kw):
    import paper_1711_08095_gb300 as snect

    return snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                       batch=0, precision=precision, **kw)


def max_principal_angle(X, Y):
    qx, _ = np.linalg.qr(np.asarray(X, np.float64))
    qy, _ = np.linalg.qr(np.asarray(Y, np.float64))
    s = np.clip(np.linalg.svd(qx.T @ qy, compute_uv=False), -1.0, 1.0)
    return float(np.degrees(np.arccos(s.min())))


@pytest.mark.parametrize("J,tc", [((16, 16, 5), False), ((16, 16, 5), True), ((32, 32, 5), False),
                                  ((16, 32, 5), False)])
def test_bf16_reaches_fp32_rmse_on_config1_refit(J, tc, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p = S.config1(J_fit=J)
    out = {}
    bf = snect.BF16_TC if tc else snect.BF16
    for prec in (snect.FP32, bf):
        c = ctx(p, prec)
        c.epoch(p.epochs)
        out[prec] = (c.loss(p.test_idx, p.test_val), c.get_factors())
        c.close()
    l32, (G32, U32) = out[snect.FP32]
    l16, (G16, U16) = out[bf]
    assert np.isfinite(l16["total"])
    assert l16["rmse_test"] <= 1.01 * l32["rmse_test"], (l16["rmse_test"], l32["rmse_test"])
    # distance from the FP64 oracle's sequential run (reported, loosely bounded)
    P = oracle.Params(p.G0, p.U0)
    for _ in range(p.epochs):
        oracle.sgd_epoch(p.I, P, p.lam, p.lam_g, p.lr, p.idx, p.val, p.edges, p.w)
    ro = oracle.rmse(P, p.test_idx, p.test_val)
    finite = all(np.isfinite(u).all() for u in P.U) and np.isfinite(ro)
    angles = [max_principal_angle(U16[n], P.U[n]) for n in range(2)] if finite else None
    # reported: the sequential per-entry SGD at lr 0.01 is itself unstable at some of these
    # over-parameterised ranks (its factors leave the finite range), the fast mode's damped
    # wave steps are not
    print("J=%s rmse_test bf16 %.4f fp32 %.4f oracle %s; max principal angle vs oracle (deg) %s"
          % (J, l16["rmse_test"], l32["rmse_test"], "%.4f" % ro if finite else "non-finite",
             ["%.1f" % a for a in angles] if angles else "n/a"))
    if finite:
        assert l16["rmse_test"] <= 1.2 * ro


@pytest.mark.parametrize("tc", [False, True])
def test_bf16_sweep_matches_fp32_sweep_after_one_epoch(tc, gpu_lib):
    """One epoch from the same start on a paper-shaped problem: the two forms' factors agree
    to BF16 rounding of the contraction inputs (relative 5e-2 of each matrix's scale)."""
    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=200, nnz=300_000, n_edges=10_000, J_fit=(16, 16, 5))
    res = []
    for prec in (snect.FP32, snect.BF16_TC if tc else snect.BF16):
        c = ctx(p, prec)
        c.epoch(1)
        res.append(c.get_factors())
        c.close()
    (G32, U32), (G16, U16) = res
    for a, b in zip([G32] + U32, [G16] + U16):
        scale = float(np.sqrt(np.mean(a.astype(np.float64) ** 2)))
        assert np.abs(a - b).max() <= 5e-2 * scale + 1e-6, np.abs(a - b).max() / scale


def test_bf16_needs_fast_mode_and_tensor_core_ranks(gpu_lib):
    import paper_1711_08095_gb300 as snect

    p = S.config1(J_fit=(10, 10, 5))
    with pytest.raises(snect.SnectError):
        ctx(p, snect.BF16)
    p = S.config1(J_fit=(16, 16, 5))
    with pytest.raises(snect.SnectError):
        snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                    batch=1024, precision=snect.BF16)
