"""Batched form: several independent decompositions stepped together (snect_batch_*), through
the C ABI.

A batch runs, per wave, one sweep launch over every problem (CTAs allotted by entries, the
launch shape autotuned at the first epoch) and one launch of every problem's wave-end steps.  Each problem must end where it ends when run alone: the
fast sweep accumulates with atomics, so the comparison is to FP32 rounding after one epoch
and on test RMSE after several.
"""
import numpy as np
import pytest

import snect_synth as S

pytestmark = pytest.mark.gpu


def ctx(p, lam_g=None, **kw):
    import paper_1711_08095_gb300 as snect

    return snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam,
                       lam_g=p.lam_g if lam_g is None else lam_g, lr=p.lr, batch=0, **kw)


@pytest.fixture(scope="module")
def cohorts():
    # three cohorts of different sizes, each refit for two graph weights
    ps = [S.config2(seed=40 + c, n_patients=n, nnz=z, n_edges=10_000, J_fit=(16, 16, 5))
          for c, (n, z) in enumerate([(100, 150_000), (150, 220_000), (230, 400_000)])]
    return [(p, lg) for p in ps for lg in (0.01, 0.3)]


def run(cohorts, epochs, batched, **kw):
    import paper_1711_08095_gb300 as snect

    cs = [ctx(p, lam_g=lg, **kw) for p, lg in cohorts]
    if batched:
        b = snect.Batch(cs)
        b.epoch(epochs)
        t = b.tuning()
        assert t["ctas_per_sm"] >= 2 and t["sweep_ms"] > 0, t  # the autotuner ran
        b.close()
    else:
        for c in cs:
            c.epoch(epochs)
    out = [(c.get_factors(), c.loss(p.test_idx, p.test_val)) for c, (p, _) in zip(cs, cohorts)]
    for c in cs:
        c.close()
    return out


def test_batch_matches_separate_runs_after_one_epoch(cohorts, gpu_lib):
    alone, batched = run(cohorts, 1, False), run(cohorts, 1, True)
    for ((Ga, Ua), _), ((Gb, Ub), _) in zip(alone, batched):
        for a, b in zip([Ga] + Ua, [Gb] + Ub):
            scale = float(np.sqrt(np.mean(a.astype(np.float64) ** 2)))
            assert np.isfinite(b).all()
            assert np.abs(a - b).max() <= 1e-3 * scale + 1e-6, np.abs(a - b).max() / scale


def test_bf16_batch_matches_separate_bf16_runs(cohorts, gpu_lib):
    """Contexts whose sweep gathers gene rows in BF16 batch together; the batch keeps each
    context's BF16 copy current (wave ends and network passes)."""
    import paper_1711_08095_gb300 as snect

    alone = run(cohorts, 2, False, precision=snect.BF16)
    batched = run(cohorts, 2, True, precision=snect.BF16)
    for ((Ga, Ua), la), ((Gb, Ub), lb) in zip(alone, batched):
        for a, b in zip([Ga] + Ua, [Gb] + Ub):
            scale = float(np.sqrt(np.mean(a.astype(np.float64) ** 2)))
            assert np.abs(a - b).max() <= 1e-3 * scale + 1e-6, np.abs(a - b).max() / scale
        assert abs(lb["rmse_test"] - la["rmse_test"]) <= 1e-3 * la["rmse_test"]


def test_batch_reaches_separate_rmse(cohorts, gpu_lib):
    alone, batched = run(cohorts, 10, False), run(cohorts, 10, True)
    for (_, la), (_, lb) in zip(alone, batched):
        assert np.isfinite(lb["total"])
        assert abs(lb["rmse_test"] - la["rmse_test"]) <= 0.01 * la["rmse_test"], (la, lb)


def test_batch_of_one_equals_epoch(cohorts, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p, lg = cohorts[0]
    c = ctx(p, lam_g=lg)
    l0 = c.loss(p.test_idx, p.test_val)
    b = snect.Batch([c])
    b.epoch(3)
    b.close()
    l1 = c.loss(p.test_idx, p.test_val)
    c.close()
    assert np.isfinite(l1["total"]) and l1["total"] < l0["total"]


def test_batch_rejects_mismatched_contexts(cohorts, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p, _ = cohorts[0]
    q = S.config2(seed=49, n_patients=100, nnz=150_000, n_edges=10_000, J_fit=(10, 10, 5))
    a, b = ctx(p), ctx(q)
    with pytest.raises(snect.SnectError):
        snect.Batch([a, b])  # different core ranks
    d = snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                    batch=1024)
    with pytest.raises(snect.SnectError):
        snect.Batch([a, d])  # deterministic mode
    e = ctx(p, wave=4096)
    with pytest.raises(snect.SnectError):
        snect.Batch([a, e])  # different number of waves
    for c in (a, b, d, e):
        c.close()
