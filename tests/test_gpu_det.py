"""GPU parity of the deterministic mini-batch sweep, the network pass and the objective
against the FP64 oracle, through the C ABI.

Tolerances (FP32 on the GPU against FP64 in the oracle):
  * one step from the same state: every value v of G, U1, U2, U3 within
    |v_gpu - v_oracle| <= 1e-5 * (|v_oracle| + rms(tensor))   (1e-5 relative; the rms term
    keeps values that cross zero from dividing by ~0);
  * free-running epochs: every objective term within 1e-4 relative per epoch.
"""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
LOSS_TOL = 1e-4


def ctx(p, batch=None, **kw):
    import paper_1711_08095_gb300 as snect

    return snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                       batch=p.batch if batch is None else batch, **kw)


def assert_close(gpu, ora, tol, what=""):
    gpu = np.asarray(gpu, np.float64)
    ora = np.asarray(ora, np.float64)
    s = float(np.sqrt(np.mean(ora * ora))) if ora.size else 0.0
    err = np.abs(gpu - ora) / (np.abs(ora) + s + 1e-30)
    assert err.max() <= tol, "%s: max rel err %.3g at %s" % (what, err.max(), np.unravel_index(err.argmax(), err.shape))


def assert_params_close(gpu_params, P, tol, what=""):
    G, U = gpu_params
    assert_close(G, P.G, tol, what + " G")
    for n in range(3):
        assert_close(U[n], P.U[n], tol, what + " U%d" % (n + 1))


def step_parity(p, batches, gpu_lib, batch=None):
    B = p.batch if batch is None else batch
    c = ctx(p, batch=B)
    cnt = oracle.counts(p.I, p.idx)
    n_b = (p.nnz + B - 1) // B
    for b in batches:
        b = b % n_b
        G, U = c.get_factors()
        P = oracle.Params(G, U)
        oracle.batch_step(p.I, P, p.lam, p.lr, p.idx, p.val, b * B, min(B, p.nnz - b * B), cnt, p.nnz)
        c.batches(b, 1)
        assert_params_close(c.get_factors(), P, STEP_TOL, "batch %d" % b)
    # network pass from the same state
    G, U = c.get_factors()
    P = oracle.Params(G, U)
    oracle.edge_pass(p.I[1], P, p.lam_g, p.lr, p.edges, p.w)
    c.edge_pass()
    assert_params_close(c.get_factors(), P, STEP_TOL, "network pass")
    c.close()


def test_one_step_parity_config1_first_epoch(gpu_lib):
    p = S.config1()
    step_parity(p, range((p.nnz + p.batch - 1) // p.batch), gpu_lib)


@pytest.mark.parametrize("J", [(2, 3, 2), (3, 7, 4), (5, 5, 2), (10, 10, 5), (16, 16, 5), (32, 32, 5)])
def test_one_step_parity_core_shapes(J, gpu_lib):
    """Compile-time ranks (5,5,2), (10,10,5), (16,16,5), (32,32,5) and the runtime-rank
    kernel; 18,000 entries in batches of 1,024 (17 full batches and a ragged one of 592)."""
    p = S.config1(J_fit=J)
    step_parity(p, [0, 1, 9, -1], gpu_lib)


def test_single_entry_batches_are_textbook_sgd(gpu_lib):
    p = S.tiny_problem(seed=3, I=(6, 7, 3), J=(3, 2, 2), density=0.7, n_edges=5)
    step_parity(p, range(12), gpu_lib, batch=1)


def test_one_batch_larger_than_the_problem(gpu_lib):
    p = S.tiny_problem(seed=4, I=(6, 7, 3), J=(3, 2, 2), density=0.7, n_edges=5)
    step_parity(p, [0, 0, 0], gpu_lib, batch=4096)


def test_network_pass_hub_rows(gpu_lib):
    """Rows above 128 neighbours take the chunked (affine-composition) pass; rows at or below
    take the sequential walk.  Hubs of degree 600, 129 and 128 against the oracle's walk."""
    import paper_1711_08095_gb300 as snect

    rng = np.random.default_rng(21)
    I, J = (3, 700, 2), (2, 5, 2)
    edges = [(0, j) for j in range(1, 601)] + [(650, j) for j in range(1, 130)] + \
            [(699, j) for j in range(200, 328)]
    extra = set()
    while len(extra) < 400:
        a, b = sorted(rng.integers(1, 650, size=2).tolist())
        if a != b and (a, b) not in extra:
            extra.add((a, b))
    edges = np.array(edges + sorted(extra), np.int32)
    edges = edges[rng.permutation(len(edges))]
    w = rng.uniform(0.5, 1.0, len(edges)).astype(np.float32)
    G0, U0 = S.init_params(I, J, 3)
    idx = np.array([[0, 0, 0]], np.int32)
    c = snect.Snect(I, J, idx, np.zeros(1, np.float32), edges, w, G0, U0, lam=0.01, lam_g=2.0, lr=0.05, batch=1)
    P = oracle.Params(G0, U0)
    for _ in range(3):
        oracle.edge_pass(I[1], P, 2.0, 0.05, edges, w)
        c.edge_pass()
    _, U = c.get_factors()
    assert_close(U[1], P.U[1], STEP_TOL, "network pass with hubs")
    c.close()


def test_loss_terms_match_oracle(gpu_lib):
    p = S.config1()
    c = ctx(p)
    got = c.loss(p.test_idx, p.test_val)
    P = oracle.Params(p.G0, p.U0)
    want = oracle.loss(p.I, P, p.lam, p.lam_g, p.idx, p.val, p.edges, p.w)
    for k in ("data", "reg", "graph", "total"):
        assert abs(got[k] - want[k]) <= 1e-6 * abs(want[k]), k
    assert abs(got["rmse_train"] - oracle.rmse(P, p.idx, p.val)) <= 1e-6
    assert abs(got["rmse_test"] - oracle.rmse(P, p.test_idx, p.test_val)) <= 1e-6
    c.close()


def test_free_running_epochs_config1(gpu_lib):
    """Config 1 end to end: 20 epochs, per-epoch objective within 1e-4 of the oracle's."""
    p = S.config1()
    c = ctx(p)
    P = oracle.Params(p.G0, p.U0)
    for ep in range(p.epochs):
        c.epoch(1)
        oracle.epoch(p.I, P, p.lam, p.lam_g, p.lr, p.batch, p.idx, p.val, p.edges, p.w)
        got = c.loss(p.test_idx, p.test_val)
        want = oracle.loss(p.I, P, p.lam, p.lam_g, p.idx, p.val, p.edges, p.w)
        for k in ("data", "reg", "graph", "total"):
            assert abs(got[k] - want[k]) <= LOSS_TOL * abs(want[k]), (ep, k, got[k], want[k])
        rm = oracle.rmse(P, p.test_idx, p.test_val)
        assert abs(got["rmse_test"] - rm) <= LOSS_TOL * rm, (ep, got["rmse_test"], rm)
    c.close()


def test_deterministic_mode_is_bitwise_reproducible(gpu_lib):
    p = S.config1()
    outs = []
    for _ in range(2):
        c = ctx(p)
        c.epoch(3)
        outs.append(c.get_factors())
        c.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for n in range(3):
        assert np.array_equal(outs[0][1][n], outs[1][1][n])


def test_unobserved_rows_and_empty_graph(gpu_lib):
    """Rows with no training entry never move (they have no entry term); with no edges (or
    lambda_g = 0) the network pass changes nothing."""
    p = S.tiny_problem(seed=6, I=(9, 11, 4), J=(2, 3, 2), density=0.35, n_edges=1)
    p.edges = np.zeros((0, 2), np.int32)
    p.w = np.zeros(0, np.float32)
    c = ctx(p, batch=16)
    c.epoch(2)
    G, U = c.get_factors()
    P = oracle.Params(p.G0, p.U0)
    for _ in range(2):
        oracle.epoch(p.I, P, p.lam, p.lam_g, p.lr, 16, p.idx, p.val, p.edges, p.w)
    for n in range(3):
        unseen = np.setdiff1d(np.arange(p.I[n]), p.idx[:, n])
        assert np.array_equal(U[n][unseen], p.U0[n][unseen])
    assert_params_close((G, U), P, 1e-4, "two epochs")
    c.close()


def test_host_and_device_inputs_give_the_same_context(gpu_lib):
    import torch

    p = S.config1()
    a = ctx(p)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    import paper_1711_08095_gb300 as snect

    b = snect.Snect(p.I, p.J, dev(p.idx), dev(p.val), dev(p.edges), dev(p.w), dev(p.G0), [dev(u) for u in p.U0],
                    lam=p.lam, lam_g=p.lam_g, lr=p.lr, batch=p.batch)
    a.epoch(2)
    b.epoch(2)
    ga, gb = a.get_factors(), b.get_factors()
    assert np.array_equal(ga[0], gb[0])
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["index", "nan", "self_loop", "dup_edge", "rank", "batch"])
def test_invalid_inputs_are_rejected(case, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p = S.tiny_problem(seed=8, I=(5, 6, 3), J=(2, 2, 2), density=0.8, n_edges=4)
    kw = dict(lam=p.lam, lam_g=p.lam_g, lr=p.lr, batch=8)
    idx, val, edges, J = p.idx.copy(), p.val.copy(), p.edges.copy(), p.J
    if case == "index":
        idx[3, 1] = p.I[1]
    elif case == "nan":
        val[2] = np.nan
    elif case == "self_loop":
        edges[1, 1] = edges[1, 0]
    elif case == "dup_edge":
        edges[2] = edges[0][::-1]
    elif case == "rank":
        J = (0, 2, 2)
    elif case == "batch":
        kw["batch"] = 5000
    with pytest.raises(snect.SnectError) as ei:
        snect.Snect(p.I, J, idx, val, edges, p.w, p.G0, p.U0, **kw)
    assert ei.value.code == -1
