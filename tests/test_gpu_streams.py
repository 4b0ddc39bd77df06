"""A context on a caller's non-blocking stream, through the C ABI.

Every set-up step, allocation and copy of a context is ordered on the stream it was given
(its device buffers come from the library's memory pool in stream order), so a context
created on a non-blocking stream -- one that does not synchronise with the legacy default
stream -- must give bit for bit the factors a context on the default stream gives (deterministic mode,
two epochs; the objective, reduced with FP64 atomics, to 1e-12), also for a second context
set up right after the first is destroyed (which reuses the pool's memory).
"""
import numpy as np
import pytest

import snect_synth as S

pytestmark = pytest.mark.gpu


def run(p, stream):
    import paper_1711_08095_gb300 as snect

    c = snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                    batch=p.batch, stream=stream)
    c.epoch(2)
    l = c.loss(p.test_idx, p.test_val)
    G, U = c.get_factors()
    c.close()
    return l, G, U


def test_non_blocking_stream_matches_default_stream(gpu_lib):
    import torch

    p = S.config1()
    ref = run(p, None)
    s = torch.cuda.Stream()  # created non-blocking with respect to the legacy default stream
    with torch.cuda.stream(s):
        for _ in range(2):  # the second set-up reuses the memory the first returned
            got = run(p, s.cuda_stream)
            for a, b in zip([got[1]] + got[2], [ref[1]] + ref[2]):
                assert np.array_equal(a, b)
            # the objective's FP64 sums are reduced with atomics: equal to rounding
            for k, v in ref[0].items():
                assert abs(got[0][k] - v) <= 1e-12 * abs(v), (k, got[0][k], v)


def test_fast_mode_on_a_non_blocking_stream(gpu_lib):
    import torch

    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=150, nnz=200_000, n_edges=10_000)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                        batch=0, stream=s.cuda_stream)
        l0 = c.loss(p.test_idx, p.test_val)
        c.epoch(3)
        l1 = c.loss(p.test_idx, p.test_val)
        c.close()
    assert np.isfinite(l1["total"]) and l1["rmse_test"] < l0["rmse_test"]
