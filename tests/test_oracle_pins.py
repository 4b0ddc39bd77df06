"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Every expected value here comes from a different route than the oracle's own code: the
mode-1 matricization identity X_(1) = U1 G_(1) (U3 kron U2)^T (Kolda & Bader, the reference
the paper cites for tensor operations), the Laplacian trace form of the graph term
(f_g = 1/2 tr(B^T L B), the commented-out form next to the graph regulariser, Sec. 2.3.1),
central finite differences of the objective, closed forms of the network recurrence,
least squares by numpy.linalg.lstsq, sorting, and convergence to the noise floor.
"""
import math

import numpy as np
import pytest

import oracle
import snect_synth as S


# ---------------------------------------------------------------------------------------
# independent routes
def xhat_kron(G, U, idx):
    """x~ at idx from X_(1) = U1 G_(1) (U3 kron U2)^T, G_(1)[p, q + J2 r] = g_pqr."""
    J1, J2, J3 = G.shape
    G1 = np.transpose(G, (0, 2, 1)).reshape(J1, J3 * J2)
    X1 = U[0] @ G1 @ np.kron(U[2], U[1]).T  # (I1, I2*I3), column j + I2 k
    I2 = U[1].shape[0]
    return X1[idx[:, 0], idx[:, 1] + I2 * idx[:, 2]]


def laplacian(I2, edges, w):
    Y = np.zeros((I2, I2))
    for (u, v), y in zip(edges, w):
        Y[u, v] += y
        Y[v, u] += y
    return np.diag(Y.sum(1)) - Y


def objective(G, U, idx, val, lam, lam_g, edges, w, I):
    """dict(data, reg, graph, total) via the matricization identity and tr(B^T L B)."""
    r = val - xhat_kron(G, U, idx)
    data = 0.5 * float(r @ r)
    reg = float((G * G).sum())
    for n in range(3):
        seen = np.unique(idx[:, n])
        reg += float((U[n][seen] ** 2).sum())
    reg *= 0.5 * lam
    L = laplacian(I[1], edges, w)
    graph = 0.5 * float(np.trace(U[1].T @ L @ U[1]))
    return dict(data=data, reg=reg, graph=graph, total=data + reg + lam_g * graph)


def fd_grad(fun, arrays, h=1e-6):
    """Central differences of fun(arrays) w.r.t. every element of every array."""
    out = []
    for a in range(len(arrays)):
        g = np.zeros_like(arrays[a])
        for ix in np.ndindex(arrays[a].shape):
            old = arrays[a][ix]
            arrays[a][ix] = old + h
            fp = fun(arrays)
            arrays[a][ix] = old - h
            fm = fun(arrays)
            arrays[a][ix] = old
            g[ix] = (fp - fm) / (2 * h)
        out.append(g)
    return out


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.fixture(scope="module")
def tiny():
    return S.tiny_problem(seed=3)


# ---------------------------------------------------------------------------------------
# model and objective (Eq. 2, Eq. 3, Sec. 2.3.2 per-entry L2 form, graph regulariser)
def test_predict_matches_matricization_identity(tiny):
    P = oracle.Params(tiny.G0, tiny.U0)
    got = oracle.predict(P, tiny.idx)
    want = xhat_kron(P.G, P.U, tiny.idx)
    assert rel_err(got, want) < 1e-13


def test_predict_rank_one_and_matrix_special_cases():
    rng = np.random.default_rng(0)
    # J = (1,1,1): x~ = g a b c
    G = rng.standard_normal((1, 1, 1))
    U = [rng.standard_normal((4, 1)), rng.standard_normal((5, 1)), rng.standard_normal((3, 1))]
    idx = np.array([[1, 2, 0], [3, 4, 2], [0, 0, 1]], np.int32)
    got = oracle.predict(oracle.Params(G, U), idx)
    want = G[0, 0, 0] * U[0][idx[:, 0], 0] * U[1][idx[:, 1], 0] * U[2][idx[:, 2], 0]
    assert np.allclose(got, want, rtol=1e-14)
    # I3 = J3 = 1: x~_ij = c * (U1 G[:,:,0] U2^T)_ij, a plain matrix product
    G = rng.standard_normal((3, 2, 1))
    U = [rng.standard_normal((6, 3)), rng.standard_normal((7, 2)), np.array([[1.7]])]
    idx = np.array([[i, j, 0] for i in range(6) for j in range(7)], np.int32)
    got = oracle.predict(oracle.Params(G, U), idx)
    M = 1.7 * U[0] @ G[:, :, 0] @ U[1].T
    assert np.allclose(got, M.reshape(-1), rtol=1e-13)


def test_loss_matches_independent_objective(tiny):
    P = oracle.Params(tiny.G0, tiny.U0)
    got = oracle.loss(tiny.I, P, tiny.lam, tiny.lam_g, tiny.idx, tiny.val, tiny.edges, tiny.w)
    want = objective(P.G, P.U, tiny.idx, tiny.val.astype(np.float64), tiny.lam, tiny.lam_g, tiny.edges,
                     tiny.w.astype(np.float64), tiny.I)
    for k in want:
        assert abs(got[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k])), k


def test_graph_term_zero_for_identical_neighbours():
    I2, J2 = 6, 3
    U2 = np.random.default_rng(1).standard_normal((I2, J2))
    U2[2] = U2[4] = U2[5] = U2[0]
    edges = np.array([[0, 2], [2, 4], [4, 5]], np.int32)
    w = np.array([1.0, 0.5, 2.0])
    P = oracle.Params(np.ones((1, J2, 1)), [np.ones((1, 1)), U2, np.ones((1, 1))])
    l = oracle.loss((1, I2, 1), P, 0.0, 1.0, np.zeros((0, 3), np.int32), np.zeros(0), edges, w)
    assert l["graph"] == 0.0
    before = U2.copy()
    oracle.edge_pass(I2, P, 1.0, 0.3, edges, w)
    assert np.array_equal(P.U[1], before)


def test_gauge_invariance():
    p = S.tiny_problem(seed=5)
    P = oracle.Params(p.G0, p.U0)
    base = oracle.predict(P, p.idx)
    R = np.array([[2.0, 0.3], [-0.4, 1.1]])
    Q = P.copy()
    Q.U[0] = P.U[0] @ R
    Q.G = np.einsum("tp,pqr->tqr", np.linalg.inv(R), P.G)
    assert rel_err(oracle.predict(Q, p.idx), base) < 1e-12


# ---------------------------------------------------------------------------------------
# gradients (gradient equation, Sec. 2.3.2) and the mini-batch step (Alg. 1 lines 4-8)
def test_full_batch_step_is_gradient_descent_on_f(tiny):
    """One batch holding every entry (no network pass) is theta - lr * grad(data + reg)."""
    P0 = oracle.Params(tiny.G0, tiny.U0)
    P1 = P0.copy()
    oracle.batch_step(tiny.I, P1, tiny.lam, tiny.lr, tiny.idx, tiny.val, 0, tiny.nnz)
    val = tiny.val.astype(np.float64)

    def f(arrs):
        o = objective(arrs[0], arrs[1:], tiny.idx, val, tiny.lam, 0.0, tiny.edges, tiny.w, tiny.I)
        return o["data"] + o["reg"]

    grads = fd_grad(f, [P0.G.copy()] + [u.copy() for u in P0.U])
    for a, (before, after) in enumerate(zip([P0.G] + P0.U, [P1.G] + P1.U)):
        step = (before - after) / tiny.lr
        assert rel_err(step, grads[a]) < 1e-6, a


def test_single_entry_step_is_per_entry_sgd(tiny):
    """A batch of one entry is the per-entry step with the SGD-form L2 terms:
    f_e = 1/2 (x - x~)^2 + lambda/2 (||G||^2/|Omega| + sum_n ||u_{i_n}||^2 / |Omega^{n,i_n}|)."""
    cnt = oracle.counts(tiny.I, tiny.idx)
    e = 4
    P0 = oracle.Params(tiny.G0, tiny.U0)
    P1 = P0.copy()
    oracle.batch_step(tiny.I, P1, tiny.lam, tiny.lr, tiny.idx, tiny.val, e, 1, cnt, tiny.nnz)
    t = tiny.idx[e]
    x = float(tiny.val[e])

    def fe(arrs):
        G, U = arrs[0], arrs[1:]
        xt = xhat_kron(G, U, tiny.idx[e:e + 1])[0]
        reg = (G * G).sum() / tiny.nnz + sum((U[n][t[n]] ** 2).sum() / cnt[n][t[n]] for n in range(3))
        return 0.5 * (x - xt) ** 2 + 0.5 * tiny.lam * reg

    grads = fd_grad(fe, [P0.G.copy()] + [u.copy() for u in P0.U])
    for a, (before, after) in enumerate(zip([P0.G] + P0.U, [P1.G] + P1.U)):
        step = (before - after) / tiny.lr
        assert np.abs(step - grads[a]).max() < 1e-6 * max(1.0, np.abs(grads[a]).max()), a


def test_batch_step_sums_entry_gradients_at_batch_start(tiny):
    cnt = oracle.counts(tiny.I, tiny.idx)
    P0 = oracle.Params(tiny.G0, tiny.U0)
    total = [np.zeros_like(x) for x in [P0.G] + P0.U]
    for e in range(3, 11):
        Pe = P0.copy()
        oracle.batch_step(tiny.I, Pe, tiny.lam, tiny.lr, tiny.idx, tiny.val, e, 1, cnt, tiny.nnz)
        for a, (b, x) in enumerate(zip([P0.G] + P0.U, [Pe.G] + Pe.U)):
            total[a] += x - b
    Pb = P0.copy()
    oracle.batch_step(tiny.I, Pb, tiny.lam, tiny.lr, tiny.idx, tiny.val, 3, 8, cnt, tiny.nnz)
    for a, (b, x) in enumerate(zip([P0.G] + P0.U, [Pb.G] + Pb.U)):
        assert np.allclose(x - b, total[a], rtol=1e-12, atol=1e-15), a


def test_data_grad_sums_are_the_gradient_of_the_range_data_term(tiny):
    """The summed data-term gradients of a range of entries (the quantity a fast-mode wave
    accumulates) are the gradient of 1/2 sum_range (x - x~)^2 w.r.t. every row and the core:
    central differences of the objective, with the platform rows' and the core's sums
    included; the per-(row, platform) entry counts equal a brute-force count."""
    P0 = oracle.Params(tiny.G0, tiny.U0)
    lo, n = 3, 11
    idx, val = tiny.idx[lo:lo + n], tiny.val[lo:lo + n].astype(np.float64)
    got = oracle.data_grad_sums(tiny.I, P0, tiny.idx, tiny.val, lo, n)

    def f(arrs):
        r = val - xhat_kron(arrs[0], arrs[1:], idx)
        return 0.5 * float(r @ r)

    grads = fd_grad(f, [P0.G.copy()] + [u.copy() for u in P0.U])
    for key, g in zip(("gG", "gA", "gB", "gC"), grads):
        assert rel_err(got[key], g) < 1e-6, key
    nA = np.zeros((tiny.I[0], tiny.I[2]))
    nB = np.zeros((tiny.I[1], tiny.I[2]))
    for i, j, k in idx:
        nA[i, k] += 1
        nB[j, k] += 1
    assert np.array_equal(got["nA"], nA) and np.array_equal(got["nB"], nB)


def test_data_grad_sums_match_a_batch_step_without_l2(tiny):
    """With lambda = 0 one mini-batch step moves each touched row by -lr times its summed
    data-term gradient (reading R2), which ties the two oracle routes together."""
    P0 = oracle.Params(tiny.G0, tiny.U0)
    P1 = P0.copy()
    oracle.batch_step(tiny.I, P1, 0.0, tiny.lr, tiny.idx, tiny.val, 2, 9)
    got = oracle.data_grad_sums(tiny.I, P0, tiny.idx, tiny.val, 2, 9)
    for key, b, a in zip(("gG", "gA", "gB", "gC"), [P0.G] + P0.U, [P1.G] + P1.U):
        assert np.allclose((b - a) / tiny.lr, got[key], rtol=1e-10, atol=1e-13), key


# ---------------------------------------------------------------------------------------
# network pass (Alg. 1 line 10)
def test_edge_pass_on_a_matching_is_a_gradient_step_on_the_graph_term():
    """With every gene in at most one edge the row-owned pass equals a full gradient step
    on lambda_g f_g (the per-edge gradient lambda_g y (u_k1 - u_k2), both endpoints)."""
    rng = np.random.default_rng(7)
    I2, J2 = 8, 3
    U2 = rng.standard_normal((I2, J2))
    edges = np.array([[0, 3], [5, 1], [2, 7]], np.int32)
    w = np.array([0.7, 1.0, 0.4])
    lam_g, lr = 0.9, 0.2
    P = oracle.Params(np.ones((1, J2, 1)), [np.ones((1, 1)), U2.copy(), np.ones((1, 1))])
    oracle.edge_pass(I2, P, lam_g, lr, edges, w)
    L = laplacian(I2, edges, w)
    grad = fd_grad(lambda arrs: lam_g * 0.5 * np.trace(arrs[0].T @ L @ arrs[0]), [U2.copy()])[0]
    assert np.allclose(P.U[1], U2 - lr * grad, rtol=1e-8, atol=1e-9)


def test_edge_pass_star_graph_closed_form():
    """Centre 3 with leaves 0, 1, 5, 6: the centre's row-owned walk in ascending order has the
    closed form u' = prod(1-a_s) u + sum_s a_s prod_{t>s}(1-a_t) s_s; each leaf moves once."""
    rng = np.random.default_rng(9)
    I2, J2 = 7, 2
    U2 = rng.standard_normal((I2, J2))
    leaves = [6, 0, 5, 1]
    edges = np.array([[3, l] if t % 2 else [l, 3] for t, l in enumerate(leaves)], np.int32)
    w = np.array([0.5, 1.0, 0.8, 0.3])
    lam_g, lr = 0.5, 0.4
    P = oracle.Params(np.ones((1, J2, 1)), [np.ones((1, 1)), U2.copy(), np.ones((1, 1))])
    oracle.edge_pass(I2, P, lam_g, lr, edges, w)
    order = sorted(range(4), key=lambda t: leaves[t])
    alphas = [lr * lam_g * w[t] for t in order]
    nbrs = [leaves[t] for t in order]
    want_c = np.prod([1 - a for a in alphas]) * U2[3]
    for s, (a, l) in enumerate(zip(alphas, nbrs)):
        want_c = want_c + a * np.prod([1 - b for b in alphas[s + 1:]]) * U2[l]
    assert np.allclose(P.U[1][3], want_c, rtol=1e-13)
    for t, l in enumerate(leaves):
        a = lr * lam_g * w[t]
        assert np.allclose(P.U[1][l], (1 - a) * U2[l] + a * U2[3], rtol=1e-13)
    assert np.array_equal(P.U[1][[2, 4]], U2[[2, 4]])  # isolated genes do not move


# ---------------------------------------------------------------------------------------
# whole training
def test_epoch_is_batches_then_network_pass():
    p = S.tiny_problem(seed=11, I=(5, 6, 3), J=(2, 2, 2), density=0.8, n_edges=6)
    A = oracle.Params(p.G0, p.U0)
    oracle.epoch(p.I, A, p.lam, p.lam_g, p.lr, 7, p.idx, p.val, p.edges, p.w)
    B = oracle.Params(p.G0, p.U0)
    for s in range(0, p.nnz, 7):
        oracle.batch_step(p.I, B, p.lam, p.lr, p.idx, p.val, s, min(7, p.nnz - s))
    oracle.edge_pass(p.I[1], B, p.lam_g, p.lr, p.edges, p.w)
    for x, y in zip([A.G] + A.U, [B.G] + B.U):
        assert np.array_equal(x, y)


def test_sequential_epoch_equals_batches_of_one():
    p = S.tiny_problem(seed=12, I=(5, 6, 3), J=(2, 3, 2), density=0.8, n_edges=6)
    A = oracle.Params(p.G0, p.U0)
    oracle.sgd_epoch(p.I, A, p.lam, p.lam_g, p.lr, p.idx, p.val, p.edges, p.w)
    B = oracle.Params(p.G0, p.U0)
    oracle.epoch(p.I, B, p.lam, p.lam_g, p.lr, 1, p.idx, p.val, p.edges, p.w)
    for x, y in zip([A.G] + A.U, [B.G] + B.U):
        assert np.allclose(x, y, rtol=1e-13, atol=1e-15)


def test_sgd_reaches_noise_floor_on_planted_tensor():
    rng = np.random.default_rng(0)
    I, J, sigma = (30, 40, 3), (2, 2, 2), 0.05
    G, U = S.planted_model(I, J, 11)
    cells = np.array([(i, j, k) for i in range(I[0]) for j in range(I[1]) for k in range(I[2])], np.int32)
    idx = cells[rng.random(len(cells)) < 0.7]
    idx = idx[rng.permutation(len(idx))]
    x = xhat_kron(G, U, idx) + sigma * rng.standard_normal(len(idx))
    nt = len(idx) // 10
    te, tr, xte, xtr = idx[:nt], idx[nt:], x[:nt], x[nt:]
    G0, U0 = S.init_params(I, J, 5)
    P = oracle.Params(G0, U0)
    none = np.zeros((0, 2), np.int32)
    for _ in range(80):
        oracle.sgd_epoch(I, P, 1e-3, 0.0, 0.02, tr, xtr, none, np.zeros(0))
    assert oracle.rmse(P, tr, xtr) < 1.1 * sigma
    assert oracle.rmse(P, te, xte) < 1.2 * sigma


def test_config1_epoch_loss_is_monotone():
    """The summed-Jacobi mini-batch reading at batch 1,024 is stable on config 1."""
    p = S.config1()
    P = oracle.Params(p.G0, p.U0)
    prev = oracle.loss(p.I, P, p.lam, p.lam_g, p.idx, p.val, p.edges, p.w)["total"]
    for _ in range(20):
        oracle.epoch(p.I, P, p.lam, p.lam_g, p.lr, p.batch, p.idx, p.val, p.edges, p.w)
        cur = oracle.loss(p.I, P, p.lam, p.lam_g, p.idx, p.val, p.edges, p.w)["total"]
        assert cur < prev
        prev = cur


# ---------------------------------------------------------------------------------------
# QR post-pass (Alg. 1 line 15)
def test_qr_post_pass_keeps_predictions_and_orthonormalises():
    p = S.tiny_problem(seed=2, I=(6, 7, 4), J=(3, 2, 2))
    P = oracle.Params(p.G0, p.U0)
    before = oracle.predict(P, p.idx)
    oracle.qr_post(p.I, P)
    assert rel_err(oracle.predict(P, p.idx), before) < 1e-12
    for n in range(3):
        assert np.allclose(P.U[n].T @ P.U[n], np.eye(p.J[n]), atol=1e-12)
        # same column space as numpy's QR (Q determined up to column signs)
        Qn, _ = np.linalg.qr(np.asarray(p.U0[n], np.float64))
        assert np.allclose(np.abs(Qn.T @ P.U[n]), np.eye(p.J[n]), atol=1e-10)


def test_qr_post_pass_keeps_a_mode_wider_than_tall():
    # config 1's shape: J3 = 5 platforms' worth of columns but only 4 platform rows; that mode
    # has no 5 orthonormal columns and keeps its factor, the others are orthonormalised
    p = S.tiny_problem(seed=3, I=(8, 9, 4), J=(3, 2, 5))
    P = oracle.Params(p.G0, p.U0)
    before = oracle.predict(P, p.idx)
    skipped = oracle.qr_post(p.I, P)
    assert skipped == 1 << 2
    assert np.array_equal(P.U[2], np.asarray(p.U0[2], np.float64))
    for n in range(2):
        assert np.allclose(P.U[n].T @ P.U[n], np.eye(p.J[n]), atol=1e-12)
    assert rel_err(oracle.predict(P, p.idx), before) < 1e-12


def test_qr_post_pass_r_is_the_cholesky_factor_up_to_signs():
    # U = Q R with Q orthonormal means U^T U = R^T R: the oracle's R (recovered as Q^T U)
    # is the Cholesky factor of the Gram matrix up to the signs of its rows
    p = S.tiny_problem(seed=5, I=(12, 10, 6), J=(4, 3, 2))
    P = oracle.Params(p.G0, p.U0)
    oracle.qr_post(p.I, P)
    for n in range(3):
        U0 = np.asarray(p.U0[n], np.float64)
        R = P.U[n].T @ U0
        assert np.allclose(np.tril(R, -1), 0.0, atol=1e-12)
        L = np.linalg.cholesky(U0.T @ U0)
        assert np.allclose(np.abs(R), np.abs(L.T), atol=1e-10)


# ---------------------------------------------------------------------------------------
# fold-in (Eq. 9) and top-k (Sec. 3.2.1)
def _fold_problem(seed, n, noise, J=(4, 3, 2), I2=30, I3=3):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(J)
    B = rng.standard_normal((I2, J[1]))
    C = rng.standard_normal((I3, J[2]))
    cells = rng.choice(I2 * I3, size=n, replace=False)
    jk = np.stack([cells // I3, cells % I3], 1).astype(np.int32)
    W = np.einsum("pqr,nq,nr->np", G, B[jk[:, 0]], C[jk[:, 1]])
    u = rng.standard_normal(J[0])
    x = W @ u + noise * rng.standard_normal(n)
    return G, B, C, jk, x, u, W


def test_foldin_matches_lstsq_with_ridge():
    G, B, C, jk, x, _, W = _fold_problem(1, 40, 0.3)
    lam = 0.7
    A = np.vstack([W, math.sqrt(lam) * np.eye(W.shape[1])])
    rhs = np.concatenate([x, np.zeros(W.shape[1])])
    want = np.linalg.lstsq(A, rhs, rcond=None)[0]
    got = oracle.foldin(G, B, C, jk, x, lam)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-12)


def test_foldin_recovers_planted_row_exactly_without_noise():
    G, B, C, jk, x, u, _ = _fold_problem(2, 25, 0.0)
    got = oracle.foldin(G, B, C, jk, x, 0.0)
    assert np.allclose(got, u, rtol=1e-9, atol=1e-11)


def test_topk_matches_sorted_cosine():
    rng = np.random.default_rng(4)
    U1 = rng.standard_normal((50, 5))
    U1[7] = 0.0  # zero row scores 0
    U1[11] = U1[3]  # exact tie with row 3: the lower index wins
    u = U1[3] + 0.01 * rng.standard_normal(5)
    sc = (U1 @ u) / np.maximum(np.linalg.norm(U1, axis=1) * np.linalg.norm(u), 1e-300)
    sc[7] = 0.0
    order = sorted(range(50), key=lambda i: (-sc[i], i))[:10]
    idx, s = oracle.topk(U1, u, 10)
    assert list(idx) == order
    assert np.allclose(s, sc[order], rtol=1e-12)
    assert list(idx[:2]) == [3, 11]


# ---------------------------------------------------------------------------------------
# the lock-free form of Alg. 1 with one worker (Sec. 2.3.3, reading R13)
def test_hogwild_entries_only_is_the_sequential_epoch(tiny):
    P0 = oracle.Params(tiny.G0, tiny.U0)
    P1, P2 = P0.copy(), P0.copy()
    none = np.zeros((0, 2), np.int32)
    oracle.sgd_epoch(tiny.I, P1, tiny.lam, tiny.lam_g, tiny.lr, tiny.idx, tiny.val, none, np.zeros(0))
    oracle.hogwild_epoch(tiny.I, P2, tiny.lam, tiny.lam_g, tiny.lr, tiny.idx, tiny.val, none, np.zeros(0),
                         np.arange(tiny.nnz))
    for a, b in zip([P1.G] + P1.U, [P2.G] + P2.U):
        assert np.array_equal(a, b)


def test_hogwild_edges_on_a_matching_are_the_network_pass():
    """Disjoint edges: each edge item is the row-owned pass's update of both endpoints."""
    I2, J2 = 6, 3
    rng = np.random.default_rng(5)
    U2 = rng.standard_normal((I2, J2))
    edges = np.array([[0, 3], [4, 1], [2, 5]], np.int32)
    w = np.array([0.7, 1.0, 0.5])
    lam_g, lr = 0.4, 0.3
    A = oracle.Params(np.ones((1, J2, 1)), [np.zeros((1, 1)), U2.copy(), np.zeros((1, 1))])
    B = oracle.Params(np.ones((1, J2, 1)), [np.zeros((1, 1)), U2.copy(), np.zeros((1, 1))])
    oracle.edge_pass(I2, A, lam_g, lr, edges, w)
    no = np.zeros((0, 3), np.int32)
    oracle.hogwild_epoch((1, I2, 1), B, 0.0, lam_g, lr, no, np.zeros(0), edges, w, np.array([1, 0, 2]))
    assert np.allclose(A.U[1], B.U[1], rtol=1e-14, atol=1e-15)


def test_hogwild_interleaving_matters(tiny):
    """An edge visited between entries changes what later entries see."""
    P0 = oracle.Params(tiny.G0, tiny.U0)
    n, m = tiny.nnz, tiny.edges.shape[0]
    a, b = P0.copy(), P0.copy()
    first = np.concatenate([np.arange(n), n + np.arange(m)])
    mixed = np.concatenate([n + np.arange(m), np.arange(n)])
    oracle.hogwild_epoch(tiny.I, a, tiny.lam, 5.0, tiny.lr, tiny.idx, tiny.val, tiny.edges, tiny.w, first)
    oracle.hogwild_epoch(tiny.I, b, tiny.lam, 5.0, tiny.lr, tiny.idx, tiny.val, tiny.edges, tiny.w, mixed)
    assert not np.allclose(a.U[0], b.U[0])


# ---------------------------------------------------------------------------------------
# personalised subtype matrix (Sec. 3.3)
def test_subtype_unit_profile_is_a_core_slice():
    rng = np.random.default_rng(8)
    G = rng.standard_normal((4, 3, 2))
    U3 = rng.standard_normal((5, 2))
    for p in range(4):
        S, rn, pn = oracle.subtype(G, U3, np.eye(4)[p])
        assert np.array_equal(S, G[p])
        assert np.allclose(rn, np.sqrt((G[p] ** 2).sum(1)), rtol=1e-14)


def test_subtype_reproduces_the_patient_slice_and_its_norms():
    """b_j^T S c_k is the patient's predicted cell (Eq. 2 by the matricization identity); with
    orthonormal U2 and U3 the row norms of S and the platform norms are those of U2^T X_i U3
    and of the columns of the patient's predicted gene x platform slice X_i."""
    rng = np.random.default_rng(9)
    J = (4, 3, 2)
    I = (5, 7, 4)
    G = rng.standard_normal(J)
    U = [rng.standard_normal((I[n], J[n])) for n in range(3)]
    U[1] = np.linalg.qr(U[1])[0]
    U[2] = np.linalg.qr(U[2])[0]
    i = 2
    S, rn, pn = oracle.subtype(G, U[2], U[0][i])
    jj, kk = np.meshgrid(np.arange(I[1]), np.arange(I[2]), indexing="ij")
    idx = np.stack([np.full(jj.size, i), jj.ravel(), kk.ravel()], 1)
    Xi = xhat_kron(G, U, idx).reshape(I[1], I[2])
    assert np.allclose(U[1] @ S @ U[2].T, Xi, rtol=1e-12, atol=1e-12)
    assert np.allclose(pn, np.linalg.norm(Xi, axis=0), rtol=1e-12)
    assert np.allclose(rn, np.linalg.norm(U[1].T @ Xi @ U[2], axis=1), rtol=1e-12)


# ---------------------------------------------------------------------------------------
# k-means stratification of the patient profiles (Sec. 3.1.1, reading R14)
def test_kmeans_recovers_planted_clusters_at_a_fixed_point():
    X, labels, init = S.clustered_profiles(600, 10, 13, spread=0.05, seed=3)
    a, cent, it, inertia = oracle.kmeans(X, init, 100)
    assert np.array_equal(a, labels) and it < 100
    Xd = X.astype(np.float64)
    D = ((Xd[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(np.argmin(D, 1), a)  # each row at its nearest centroid
    for c in range(13):
        assert np.allclose(cent[c], Xd[a == c].mean(0), rtol=1e-12, atol=1e-15)  # centroid = mean
    assert abs(inertia - D[np.arange(600), a].sum()) <= 1e-12 * inertia


def test_kmeans_matches_scipy_lloyd():
    from scipy.cluster.vq import kmeans2

    X, _, init = S.clustered_profiles(500, 8, 5, spread=0.6, seed=4)
    a, cent, it, _ = oracle.kmeans(X, init, 200)
    c2, l2 = kmeans2(X.astype(np.float64), init.copy(), iter=it + 1, minit="matrix")
    assert np.array_equal(a, l2)
    assert np.allclose(cent, c2, rtol=1e-10, atol=1e-12)


def test_kmeans_one_cluster_and_monotone_inertia():
    X, _, init = S.clustered_profiles(300, 6, 4, spread=0.8, seed=5)
    a, cent, it, _ = oracle.kmeans(X, X[:1].astype(np.float64), 10)
    assert it == 1 and not a.any() and np.allclose(cent[0], X.astype(np.float64).mean(0), rtol=1e-12)
    prev = np.inf
    for m in range(1, 8):
        inertia = oracle.kmeans(X, init, m)[3]
        assert inertia <= prev * (1 + 1e-12)
        prev = inertia
