"""Seeded synthetic inputs shaped like the SNeCT workloads (patient x gene x platform).

This module is the only code shared by the CUDA library's tests/benchmarks and the
CPU oracle.  It draws random numbers and lays them out; it does not implement any
step of the decomposition (no prediction, gradient, update, loss, fold-in or search).
The observed values of a planted problem are produced by the planted Tucker model
X = G x1 U1 x2 U2 x3 U3 (the model of Eq. 2, Sec. 2.2), evaluated here with a
library contraction (numpy.einsum) plus Gaussian noise, because a planted tensor is
what the synthetic stand-ins for PanCan12 are.

The PanCan12 tensor (4,555 x 14,351 x 5, Sec. 2.1.1) and the PathwayCommons gene
network (665,429 associations, Sec. 2.1.2) are not available; every generator below
stands in for them with the shapes, sparsity and degree structure the paper states.

Conventions shared by both sides:
  * indices are 0-based int32, an entry is the triple (i, j, k) = (patient, gene, platform);
  * the core G is a dense J1 x J2 x J3 array, row-major (last index fastest);
  * a factor matrix U_n is dense I_n x J_n, row-major;
  * the gene network is an undirected edge list, each edge stored once, no self loops,
    with positive weights y.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "Problem",
    "init_params",
    "planted_model",
    "erdos_renyi_edges",
    "chung_lu_edges",
    "tiny_problem",
    "config1",
    "config2",
    "config4_cohorts",
    "ServingModel",
    "serving_model",
    "serving_query",
    "poisson_arrivals",
    "interleaved_order",
    "clustered_profiles",
]


@dataclasses.dataclass
class Problem:
    """One decomposition problem: observed entries, gene network, hyper-parameters, init."""

    I: tuple  # tensor dims (I1, I2, I3)
    J: tuple  # core ranks used for the fit (J1, J2, J3)
    idx: np.ndarray  # (nnz, 3) int32 training entries, in the order the sweep visits them
    val: np.ndarray  # (nnz,) float32
    test_idx: np.ndarray  # (n_test, 3) int32
    test_val: np.ndarray  # (n_test,) float32
    edges: np.ndarray  # (m, 2) int32, undirected, each once
    w: np.ndarray  # (m,) float32 edge weights y
    G0: np.ndarray  # (J1, J2, J3) float32 initial core
    U0: List[np.ndarray]  # [(I_n, J_n) float32] initial factors
    lam: float
    lam_g: float
    lr: float
    epochs: int
    batch: int  # deterministic mini-batch size (0 = unordered fast mode)
    noise: float
    truth: Optional[tuple] = None  # (G, [U1, U2, U3]) of the planted model, float64

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])


def init_params(I, J, seed):
    """Random initial core and factors (Alg. 1 line 1 says "randomly"; the reading used is
    G iid N(0,1) and U_n iid N(0, 1/J_n), i.e. standard deviation 1/sqrt(J_n))."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(tuple(J)).astype(np.float32)
    U = [(rng.standard_normal((I[n], J[n])) / math.sqrt(J[n])).astype(np.float32) for n in range(3)]
    return G, U


def planted_model(I, J, seed):
    """Planted Tucker model: core iid N(0,1), factors iid N(0, 1/J_n), float64."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(tuple(J))
    U = [rng.standard_normal((I[n], J[n])) / math.sqrt(J[n]) for n in range(3)]
    return G, U


def _planted_values(truth, idx, chunk=1 << 21):
    """Noise-free planted values at the cells idx, via a (gene, platform) table and einsum."""
    G, (A, B, C) = truth
    I2, I3 = B.shape[0], C.shape[0]
    # table[j, k, p] = sum_{q, r} G[p, q, r] B[j, q] C[k, r]
    table = np.einsum("pqr,jq,kr->jkp", G, B, C, optimize=True).reshape(I2 * I3, -1)
    out = np.empty(idx.shape[0], dtype=np.float64)
    for s in range(0, idx.shape[0], chunk):
        e = min(s + chunk, idx.shape[0])
        i = idx[s:e, 0].astype(np.int64)
        jk = idx[s:e, 1].astype(np.int64) * I3 + idx[s:e, 2]
        out[s:e] = np.einsum("np,np->n", A[i], table[jk])
    return out


def erdos_renyi_edges(n, m, seed, weight_range=None):
    """G(n, m): m distinct undirected edges drawn uniformly, no self loops."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if m > total:
        raise ValueError("too many edges")
    codes = rng.choice(total, size=m, replace=False)
    # decode the upper-triangle code into (u, v), u < v: row u holds the codes
    # starts[u] .. starts[u] + n - 2 - u
    r = np.arange(n, dtype=np.int64)
    starts = r * n - r * (r + 1) // 2
    u = np.searchsorted(starts, codes, side="right") - 1
    v = codes - starts[u] + u + 1
    e = np.stack([u, v], axis=1).astype(np.int32)
    if weight_range is None:
        w = np.ones(m, dtype=np.float32)
    else:
        w = rng.uniform(weight_range[0], weight_range[1], size=m).astype(np.float32)
    return e, w


def chung_lu_edges(n, m, exponent, seed, weight_range=(0.5, 1.0)):
    """Chung-Lu graph with m distinct undirected edges, expected degree of the node of
    rank r proportional to r^(-1/(exponent-1)) (power-law degrees with that exponent);
    rank -> node through one seeded permutation; weights uniform in weight_range."""
    rng = np.random.default_rng(seed)
    wts = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (exponent - 1.0))
    p = wts / wts.sum()
    perm = rng.permutation(n)
    have = np.zeros(0, dtype=np.int64)
    while have.size < m:
        need = int((m - have.size) * 1.3) + 1024
        a = rng.choice(n, size=need, p=p)
        b = rng.choice(n, size=need, p=p)
        keep = a != b
        lo = np.minimum(a[keep], b[keep])
        hi = np.maximum(a[keep], b[keep])
        codes = lo.astype(np.int64) * n + hi
        # first occurrences only, in draw order, so the result does not depend on sorting
        merged = np.concatenate([have, codes])
        _, first = np.unique(merged, return_index=True)
        have = merged[np.sort(first)]
    have = have[:m]
    e = np.stack([perm[have // n], perm[have % n]], axis=1).astype(np.int32)
    w = rng.uniform(weight_range[0], weight_range[1], size=m).astype(np.float32)
    return e, w


def _split(idx, val, frac_test, rng):
    n = idx.shape[0]
    perm = rng.permutation(n)
    n_test = int(round(n * frac_test))
    te, tr = perm[:n_test], perm[n_test:]
    return idx[tr], val[tr], idx[te], val[te]


def tiny_problem(I=(4, 5, 3), J=(2, 3, 2), density=0.6, n_edges=4, seed=0, lam=0.05, lam_g=0.3,
                 lr=0.05, batch=0):
    """A few dozen cells of a small tensor, for brute-force and finite-difference checks."""
    rng = np.random.default_rng(seed)
    cells = np.array([(i, j, k) for i in range(I[0]) for j in range(I[1]) for k in range(I[2])], dtype=np.int32)
    keep = rng.random(cells.shape[0]) < density
    idx = cells[keep]
    idx = idx[rng.permutation(idx.shape[0])]
    val = rng.standard_normal(idx.shape[0]).astype(np.float32)
    edges, w = erdos_renyi_edges(I[1], n_edges, seed + 1, weight_range=(0.5, 1.0))
    G0, U0 = init_params(I, J, seed + 2)
    return Problem(I=tuple(I), J=tuple(J), idx=idx, val=val, test_idx=idx[:0], test_val=val[:0],
                   edges=edges, w=w, G0=G0, U0=U0, lam=lam, lam_g=lam_g, lr=lr, epochs=1,
                   batch=batch if batch else idx.shape[0], noise=0.0)


def config1(seed=1, J_fit=(5, 5, 2)):
    """Tiny plain-FP32 problem: 200 x 300 x 4 tensor, 20,000 observed cells drawn uniformly
    without replacement from a planted Tucker tensor with core 5 x 5 x 2, noise sigma 0.05;
    Erdos-Renyi gene graph with 1,500 unit-weight edges; lambda 0.01, lambda_g 0.1, lr 0.01,
    20 epochs in fixed-order mini-batches of 1,024; seeded 90/10 train/test split.
    J_fit sets the core ranks of the fit (the precision form refits this tensor at 16x16x5
    and 32x32x5)."""
    I, Jp = (200, 300, 4), (5, 5, 2)
    rng = np.random.default_rng(seed)
    truth = planted_model(I, Jp, seed * 1000 + 1)
    total = I[0] * I[1] * I[2]
    codes = rng.choice(total, size=20000, replace=False)
    idx = np.stack([codes // (I[1] * I[2]), (codes // I[2]) % I[1], codes % I[2]], axis=1).astype(np.int32)
    val = (_planted_values(truth, idx) + 0.05 * rng.standard_normal(idx.shape[0])).astype(np.float32)
    tr_i, tr_v, te_i, te_v = _split(idx, val, 0.1, rng)
    edges, w = erdos_renyi_edges(I[1], 1500, seed * 1000 + 2)
    G0, U0 = init_params(I, J_fit, seed * 1000 + 3)
    return Problem(I=I, J=tuple(J_fit), idx=tr_i, val=tr_v, test_idx=te_i, test_val=te_v, edges=edges,
                   w=w, G0=G0, U0=U0, lam=0.01, lam_g=0.1, lr=0.01, epochs=20, batch=1024, noise=0.05,
                   truth=truth)


def _zipf_patient_platform_cells(n_patients, n_genes, n_platforms, nnz, rng, zipf_s=1.1,
                                 platforms_lo=3, platforms_hi=5):
    """Each patient sits on a uniform random 3..5 of the platforms; nnz cells are split as
    evenly as possible over the (patient, platform) pairs; inside a pair the genes are drawn
    without replacement with probability proportional to Zipf(zipf_s) rank weights
    (Efraimidis-Spirakis keys log(u)/w), rank -> gene through one seeded permutation."""
    n_on = rng.integers(platforms_lo, platforms_hi + 1, size=n_patients)
    pairs = []
    for p in range(n_patients):
        plats = np.sort(rng.choice(n_platforms, size=n_on[p], replace=False))
        pairs.extend((p, k) for k in plats)
    pairs = np.array(pairs, dtype=np.int64)
    n_pairs = pairs.shape[0]
    base, extra = divmod(nnz, n_pairs)
    if base + (1 if extra else 0) > n_genes:
        raise ValueError("more cells per (patient, platform) pair than genes")
    per_pair = np.full(n_pairs, base, dtype=np.int64)
    per_pair[rng.permutation(n_pairs)[:extra]] += 1
    inv_w = np.arange(1, n_genes + 1, dtype=np.float64) ** zipf_s  # 1 / w_rank
    gene_of_rank = rng.permutation(n_genes)
    out_i = np.empty(nnz, dtype=np.int32)
    out_j = np.empty(nnz, dtype=np.int32)
    out_k = np.empty(nnz, dtype=np.int32)
    pos = 0
    chunk = max(1, (1 << 23) // n_genes)
    for s in range(0, n_pairs, chunk):
        e = min(s + chunk, n_pairs)
        keys = np.log(rng.random((e - s, n_genes))) * inv_w  # larger key = picked first
        for m in np.unique(per_pair[s:e]):
            rows = np.nonzero(per_pair[s:e] == m)[0]
            if m == 0:
                continue
            top = np.argpartition(-keys[rows], m - 1, axis=1)[:, :m]
            top = np.sort(top, axis=1)
            cnt = rows.size * m
            out_i[pos:pos + cnt] = np.repeat(pairs[s + rows, 0], m)
            out_k[pos:pos + cnt] = np.repeat(pairs[s + rows, 1], m)
            out_j[pos:pos + cnt] = gene_of_rank[top].reshape(-1)
            pos += cnt
    assert pos == nnz
    return np.stack([out_i, out_j, out_k], axis=1)


def config2(seed=2, n_patients=4500, n_genes=15000, n_platforms=5, nnz=30_000_000, n_edges=300_000,
            J_true=(10, 10, 5), J_fit=(10, 10, 5), noise=0.1, lam=0.01, lam_g=0.1, lr=0.01, epochs=10,
            shuffle=True):
    """Paper-like plain-FP32 problem: 4,500 x 15,000 x 5 tensor, 30M observed cells (each
    patient on a random 3-5 platforms, genes Zipf(1.1)-sampled within them), values from a
    planted Tucker model with core 10 x 10 x 5 plus N(0, 0.1^2) noise; gene graph of 300,000
    edges with power-law degrees (exponent 2.2), weights U(0.5, 1); 10 epochs; 90/10 split.
    The sizes are parameters so that smaller problems of the same structure can be drawn.
    The training entries are returned in one seeded random order (the sweep's visit order)."""
    I = (n_patients, n_genes, n_platforms)
    rng = np.random.default_rng(seed)
    truth = planted_model(I, J_true, seed * 1000 + 1)
    idx = _zipf_patient_platform_cells(n_patients, n_genes, n_platforms, nnz, rng)
    val = _planted_values(truth, idx)
    val += noise * rng.standard_normal(val.shape[0])
    val = val.astype(np.float32)
    tr_i, tr_v, te_i, te_v = _split(idx, val, 0.1, rng)  # the split permutes: random visit order
    if not shuffle:
        o = np.lexsort((tr_i[:, 2], tr_i[:, 1], tr_i[:, 0]))
        tr_i, tr_v = tr_i[o], tr_v[o]
    edges, w = chung_lu_edges(n_genes, n_edges, 2.2, seed * 1000 + 2)
    G0, U0 = init_params(I, J_fit, seed * 1000 + 3)
    return Problem(I=I, J=tuple(J_fit), idx=np.ascontiguousarray(tr_i), val=tr_v,
                   test_idx=np.ascontiguousarray(te_i), test_val=te_v, edges=edges, w=w, G0=G0, U0=U0,
                   lam=lam, lam_g=lam_g, lr=lr, epochs=epochs, batch=0, noise=noise, truth=truth)


def config4_cohorts(seed=4, n_cohorts=12, scale=1.0, J_fit=(16, 16, 5), n_lambda=8):
    """Batched form: cohorts of round(linspace(150, 1100)) patients x 15,000 genes x 5 platforms
    with round(geomspace(0.4M, 8M)) cells each (times `scale`), generated like config2, each
    refit for the n_lambda graph weights geomspace(1e-3, 1).  Returns (cohorts, lambda_g grid)."""
    pats = np.round(np.linspace(150, 1100, n_cohorts)).astype(int)
    nnzs = np.round(np.geomspace(0.4e6, 8e6, n_cohorts) * scale).astype(int)
    cohorts = [config2(seed=seed * 100 + c, n_patients=int(pats[c]), nnz=int(nnzs[c]), n_edges=300_000,
                       J_true=(10, 10, 5), J_fit=J_fit, epochs=1)
               for c in range(n_cohorts)]
    return cohorts, np.geomspace(1e-3, 1.0, n_lambda)


@dataclasses.dataclass
class ServingModel:
    """A frozen planted model that fold-in queries are served against."""

    G: np.ndarray  # (J1, J2, J3) float32
    U: List[np.ndarray]  # [(I_n, J_n) float32]
    lam: float
    noise: float


def serving_model(seed=5, I=(4500, 15000, 5), J=(16, 16, 5), lam=0.01, noise=0.1):
    """Planted model of the paper-like shape at core 16 x 16 x 5, frozen for serving."""
    G, U = planted_model(I, J, seed * 1000 + 1)
    return ServingModel(G=G.astype(np.float32), U=[u.astype(np.float32) for u in U], lam=lam, noise=noise)


def serving_query(model: ServingModel, q, size=None, lo=5000, hi=75000, seed=5):
    """One new-patient query: a planted patient row u ~ N(0, 1/J1), observed at `size` distinct
    (gene, platform) cells drawn uniformly (size log-uniform in [lo, hi] if not given), values
    = planted value + N(0, noise^2).  Returns (jk (n, 2) int32, val (n,) float32, u_true)."""
    rng = np.random.default_rng([seed, q])
    G, (_, B, C) = model.G, model.U
    I2, I3 = B.shape[0], C.shape[0]
    if size is None:
        size = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    size = min(size, I2 * I3)
    cells = np.sort(rng.choice(I2 * I3, size=size, replace=False))
    jk = np.stack([cells // I3, cells % I3], axis=1).astype(np.int32)
    u = rng.standard_normal(G.shape[0]) / math.sqrt(G.shape[0])
    x = np.einsum("p,pqr,nq,nr->n", u, G.astype(np.float64), B[jk[:, 0]].astype(np.float64),
                  C[jk[:, 1]].astype(np.float64), optimize=True)
    x += model.noise * rng.standard_normal(size)
    return jk, x.astype(np.float32), u


def poisson_arrivals(n, rate, seed=5):
    """Arrival times (seconds) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.default_rng([seed, 7])
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def interleaved_order(nnz, m, seed=6):
    """A random interleaving of nnz entries and m network edges (Alg. 1 picks both in random
    order): a permutation of 0 .. nnz + m - 1, where t < nnz is entry t of the visit order and
    t >= nnz is edge t - nnz.  int32."""
    rng = np.random.default_rng([seed, nnz, m])
    return rng.permutation(nnz + m).astype(np.int32)


def clustered_profiles(n, d, k, spread=0.05, seed=7):
    """Patient profiles with planted clusters (the stratification of Sec. 3.1.1 runs k-means
    on the rows of U1): k centres iid N(0, 1/d) per coordinate, each row a centre plus
    N(0, spread^2 / d) noise, cluster sizes uneven (Dirichlet weights).  Returns (X (n, d)
    float32, labels (n,) int32, init (k, d) float64: one seeded random member of each cluster,
    the initial centroids)."""
    rng = np.random.default_rng([seed, n, d, k])
    centres = rng.standard_normal((k, d)) / math.sqrt(d)
    wts = rng.dirichlet(np.full(k, 2.0))
    labels = rng.choice(k, size=n, p=wts).astype(np.int32)
    labels[:k] = np.arange(k, dtype=np.int32)  # every cluster has a member
    X = (centres[labels] + spread / math.sqrt(d) * rng.standard_normal((n, d))).astype(np.float32)
    init = np.stack([X[rng.choice(np.flatnonzero(labels == c))] for c in range(k)]).astype(np.float64)
    return X, labels, init
