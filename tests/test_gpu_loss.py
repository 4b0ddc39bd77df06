"""The objective of a fast-mode context against the oracle's (Eq. 3 in the per-entry L2 form
of Sec. 2.3.2, plus the graph term): data, regulariser, graph and total, and both RMSEs, at
the initial parameters and at the GPU's own factors after two epochs.

Each prediction is the product of the entry's gene row with its (patient, platform) row
W[i][k] = Gc_k^T a_i, formed once per call (or, when there are more such rows than training
entries, with Gc_k in the kernel).  Every compiled rank triple is driven, and runtime ranks
(3 x 7 x 4) through the generic kernel.  The test entries are checked as the kernel reads
them: a bad index or value is an error and leaves the context usable.
"""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 predictions, FP64 squares and sums


def _test_entries(p, memory):
    import torch

    if memory == "pageable":
        return p.test_idx, p.test_val
    out = []
    for a in (p.test_idx, p.test_val):
        t = torch.from_numpy(np.ascontiguousarray(a))
        out.append(t.cuda() if memory == "device" else t.pin_memory())
    return tuple(out)


def _check(got, p, G, U):
    P = oracle.Params(G, U)
    want = oracle.loss(p.I, P, p.lam, p.lam_g, p.idx, p.val, p.edges, p.w)
    for k in ("data", "reg", "graph", "total"):
        assert abs(got[k] - want[k]) <= TOL * abs(want[k]), (k, got[k], want[k])
    for k, (idx, val) in (("rmse_train", (p.idx, p.val)), ("rmse_test", (p.test_idx, p.test_val))):
        rm = oracle.rmse(P, idx, val)
        assert abs(got[k] - rm) <= TOL * rm, (k, got[k], rm)


@pytest.mark.parametrize("memory", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("J", [(5, 5, 2), (10, 10, 5), (16, 16, 5), (32, 32, 5), (3, 7, 4)])
def test_fast_mode_objective_matches_oracle(J, memory, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=150, nnz=200_000, n_edges=10_000, J_fit=J)
    c = snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr, batch=0)
    ti, tv = _test_entries(p, memory)
    _check(c.loss(ti, tv), p, p.G0, p.U0)
    c.epoch(2)
    G, U = c.get_factors()
    _check(c.loss(ti, tv), p, G, U)
    c.close()


@pytest.mark.parametrize("memory", ["pageable", "device"])
@pytest.mark.parametrize("case", ["index", "nan"])
def test_bad_test_entries_are_rejected(case, memory, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=60, n_genes=2000, nnz=40_000, n_edges=3_000)
    c = snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr, batch=0)
    ti, tv = p.test_idx.copy(), p.test_val.copy()
    if case == "index":
        ti[1234, 1] = p.I[1]
    else:
        tv[77] = np.nan
    q = S.Problem(**{**p.__dict__, "test_idx": ti, "test_val": tv})
    with pytest.raises(snect.SnectError) as ei:
        c.loss(*_test_entries(q, memory))
    assert ei.value.code == -1
    _check(c.loss(p.test_idx, p.test_val), p, p.G0, p.U0)  # still usable
    c.close()


@pytest.mark.parametrize("memory", ["pageable", "device"])
def test_objective_without_the_row_table(memory, gpu_lib):
    """20,000 patients x 5 platforms are more (patient, platform) rows than the 39,600
    training entries: the loss kernels form the products with Gc_k themselves instead of
    reading the per-row table W[i][k] = Gc_k^T a_i."""
    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=20_000, n_genes=1_000, nnz=44_000, n_edges=3_000)
    assert p.I[0] * p.I[2] > p.nnz
    c = snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr, batch=0)
    ti, tv = _test_entries(p, memory)
    _check(c.loss(ti, tv), p, p.G0, p.U0)
    c.epoch(2)
    G, U = c.get_factors()
    _check(c.loss(ti, tv), p, G, U)
    c.close()
