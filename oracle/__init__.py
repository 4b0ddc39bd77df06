"""SNeCT CPU oracle (FP64) -- TEST INFRASTRUCTURE ONLY.

Python access to ``snect_oracle.c``, a plain single-threaded FP64 restatement of the
network-constrained Tucker SGD method of Choi & Sael (arXiv 1711.08095): the model of
Eq. 2, the objective of Eq. 3 with the graph term and the per-entry form of Sec. 2.3.2,
the gradient equation, Alg. 1 (entry updates, network updates, QR post-pass), fold-in of
Eq. 9 and top-k search (Sec. 3.2.1).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline arm may use
this package.  It does not import, and is not imported by, the CUDA library.  The
readings of points the paper leaves open are listed at the top of ``snect_oracle.c``.

Every function takes and returns numpy arrays; parameters are converted to float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snect_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force=False):
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_foldin.restype = ctypes.c_int
            lib.oracle_qr_post.restype = ctypes.c_int
            lib.oracle_kmeans.restype = ctypes.c_int
            _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


class Params:
    """Core and factors in float64, updated in place by the oracle's steps."""

    def __init__(self, G, U):
        self.G = np.array(G, dtype=np.float64, order="C")
        self.U = [np.array(u, dtype=np.float64, order="C") for u in U]

    @property
    def J(self):
        return tuple(self.G.shape)

    def copy(self):
        return Params(self.G, self.U)


def predict(params: Params, idx):
    """x~ at each entry (Eq. 2 entrywise)."""
    lib = _load()
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    out = np.empty(idx.shape[0], dtype=np.float64)
    lib.oracle_predict(Jp, params.G.ctypes.data_as(_f64p), *(u.ctypes.data_as(_f64p) for u in params.U),
                       ip, ctypes.c_int64(idx.shape[0]), out.ctypes.data_as(_f64p))
    return out


def counts(I, idx):
    """Training counts |Omega^{n,i}| per mode."""
    lib = _load()
    I, Ip = _i32(I)
    idx, ip = _i32(idx)
    c = [np.zeros(int(I[m]) + 1, dtype=np.int64) for m in range(3)]
    lib.oracle_counts(Ip, ip, ctypes.c_int64(idx.shape[0]), *(x.ctypes.data_as(_i64p) for x in c))
    return [x[:int(I[m])] for m, x in enumerate(c)]


def loss(I, params: Params, lam, lam_g, idx, val, edges, w):
    """dict(data, reg, graph, total): Eq. 3 + L2 form of Sec. 2.3.2 + f_g, f_opt = f + lam_g f_g."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    val, vp = _f64(val)
    edges, ep = _i32(edges.reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32))
    w, wp = _f64(w)
    out = np.zeros(4, dtype=np.float64)
    lib.oracle_loss(Ip, Jp, ctypes.c_double(lam), ctypes.c_double(lam_g), params.G.ctypes.data_as(_f64p),
                    *(u.ctypes.data_as(_f64p) for u in params.U), ip, vp, ctypes.c_int64(idx.shape[0]),
                    ep, wp, ctypes.c_int64(edges.shape[0]), out.ctypes.data_as(_f64p))
    return dict(data=out[0], reg=out[1], graph=out[2], total=out[3])


def rmse(params: Params, idx, val):
    if len(val) == 0:
        return 0.0
    r = predict(params, idx) - np.asarray(val, dtype=np.float64)
    return float(np.sqrt(np.mean(r * r)))


def batch_step(I, params: Params, lam, lr, idx, val, start, length, cnt=None, n_omega=None):
    """One mini-batch step (Alg. 1 lines 4-8, summed Jacobi reading) on entries
    [start, start+length) of the visit order; counts default to those of all of idx."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    val, vp = _f64(val)
    if cnt is None:
        cnt = counts(I, idx)
    if n_omega is None:
        n_omega = idx.shape[0]
    cnt = [np.ascontiguousarray(c, dtype=np.int64) for c in cnt]
    lib.oracle_batch_step(Ip, Jp, ctypes.c_double(lam), ctypes.c_double(lr), params.G.ctypes.data_as(_f64p),
                          *(u.ctypes.data_as(_f64p) for u in params.U), ip, vp, ctypes.c_int64(start),
                          ctypes.c_int64(length), *(c.ctypes.data_as(_i64p) for c in cnt),
                          ctypes.c_int64(n_omega))


def data_grad_sums(I, params: Params, idx, val, start, length):
    """The data-term part of the gradient equation (Sec. 2.3.2) summed over entries
    [start, start+length) of the visit order, all at the same parameters: dict of gA (I1 x J1),
    gB (I2 x J2), gC (I3 x J3), gG (J1 x J2 x J3), and the range's entries per (patient,
    platform) nA (I1 x I3) and per (gene, platform) nB (I2 x I3)."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    val, vp = _f64(val)
    out = dict(gA=np.empty((I[0], J[0])), gB=np.empty((I[1], J[1])), gC=np.empty((I[2], J[2])),
               gG=np.empty(tuple(J)), nA=np.empty((I[0], I[2])), nB=np.empty((I[1], I[2])))
    lib.oracle_data_grad_sums(Ip, Jp, params.G.ctypes.data_as(_f64p), *(u.ctypes.data_as(_f64p) for u in params.U),
                              ip, vp, ctypes.c_int64(start), ctypes.c_int64(length),
                              *(out[k].ctypes.data_as(_f64p) for k in ("gA", "gB", "gC", "gG", "nA", "nB")))
    return out


def edge_pass(I2, params: Params, lam_g, lr, edges, w):
    """Network-term pass over the gene factor (Alg. 1 line 10, row-owned reading)."""
    lib = _load()
    edges, ep = _i32(edges.reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32))
    w, wp = _f64(w)
    lib.oracle_edge_pass(ctypes.c_int32(I2), ctypes.c_int32(params.J[1]), ctypes.c_double(lam_g),
                         ctypes.c_double(lr), params.U[1].ctypes.data_as(_f64p), ep, wp,
                         ctypes.c_int64(edges.shape[0]))


def epoch(I, params: Params, lam, lam_g, lr, batch, idx, val, edges, w):
    """One epoch: batches of `batch` in order (ragged last), then one network pass."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    val, vp = _f64(val)
    edges, ep = _i32(edges.reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32))
    w, wp = _f64(w)
    lib.oracle_epoch(Ip, Jp, ctypes.c_double(lam), ctypes.c_double(lam_g), ctypes.c_double(lr),
                     ctypes.c_int64(batch), params.G.ctypes.data_as(_f64p),
                     *(u.ctypes.data_as(_f64p) for u in params.U), ip, vp, ctypes.c_int64(idx.shape[0]),
                     ep, wp, ctypes.c_int64(edges.shape[0]))


def sgd_epoch(I, params: Params, lam, lam_g, lr, idx, val, edges, w):
    """One sequential per-entry SGD epoch (Alg. 1 with one worker), then one network pass."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    val, vp = _f64(val)
    edges, ep = _i32(edges.reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32))
    w, wp = _f64(w)
    lib.oracle_sgd_epoch(Ip, Jp, ctypes.c_double(lam), ctypes.c_double(lam_g), ctypes.c_double(lr),
                         params.G.ctypes.data_as(_f64p), *(u.ctypes.data_as(_f64p) for u in params.U), ip, vp,
                         ctypes.c_int64(idx.shape[0]), ep, wp, ctypes.c_int64(edges.shape[0]))


def foldin(G, U2, U3, jk, x, ridge):
    """Closed-form fold-in of one new patient row (Eq. 9 with ridge term)."""
    lib = _load()
    G, Gp = _f64(G)
    U2, bp = _f64(U2)
    U3, cp = _f64(U3)
    jk, jp = _i32(jk)
    x, xp = _f64(x)
    J, Jp = _i32(G.shape)
    u = np.zeros(G.shape[0], dtype=np.float64)
    rc = lib.oracle_foldin(Jp, Gp, bp, cp, jp, xp, ctypes.c_int64(x.shape[0]), ctypes.c_double(ridge),
                           u.ctypes.data_as(_f64p))
    if rc != 0:
        raise np.linalg.LinAlgError("fold-in normal matrix is not positive definite")
    return u


def topk(U1, u, k):
    """Top-k rows of U1 by cosine similarity to u: (indices int64, scores float64)."""
    lib = _load()
    U1, Ap = _f64(U1)
    u, up = _f64(u)
    k = int(min(k, U1.shape[0]))
    idx = np.zeros(k, dtype=np.int64)
    sc = np.zeros(k, dtype=np.float64)
    lib.oracle_topk(Ap, ctypes.c_int64(U1.shape[0]), ctypes.c_int32(U1.shape[1]), up, ctypes.c_int32(k),
                    idx.ctypes.data_as(_i64p), sc.ctypes.data_as(_f64p))
    return idx, sc


def qr_post(I, params: Params):
    """Alg. 1's QR post-pass in place: U_n <- Q_n, G <- G x_n R_n for every mode with
    J_n <= I_n; a mode with J_n > I_n keeps its factor (reading R12).  Returns the bit mask
    of the modes kept."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    return int(lib.oracle_qr_post(Ip, Jp, params.G.ctypes.data_as(_f64p),
                                  *(u.ctypes.data_as(_f64p) for u in params.U)))


def hogwild_epoch(I, params: Params, lam, lam_g, lr, idx, val, edges, w, order):
    """Alg. 1 lines 3-13 with one worker in a given interleaved order of entries and edges
    (order[t] < nnz: entry order[t]; otherwise edge order[t] - nnz), reading R13."""
    lib = _load()
    I, Ip = _i32(I)
    J, Jp = _i32(params.J)
    idx, ip = _i32(idx)
    val, vp = _f64(val)
    edges, ep = _i32(edges.reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32))
    w, wp = _f64(w)
    order = np.ascontiguousarray(order, dtype=np.int64)
    lib.oracle_hogwild_epoch(Ip, Jp, ctypes.c_double(lam), ctypes.c_double(lam_g), ctypes.c_double(lr),
                             params.G.ctypes.data_as(_f64p), *(u.ctypes.data_as(_f64p) for u in params.U), ip, vp,
                             ctypes.c_int64(idx.shape[0]), ep, wp, ctypes.c_int64(edges.shape[0]),
                             order.ctypes.data_as(_i64p), ctypes.c_int64(order.shape[0]))


def subtype(G, U3, u):
    """Personalised subtype matrix S = G x1 u (J2 x J3), its row norms (J2) and the column
    norms of S x3 U3 (I3) (Sec. 3.3)."""
    lib = _load()
    G, Gp = _f64(G)
    U3, cp = _f64(U3)
    u, up = _f64(u)
    J, Jp = _i32(G.shape)
    S = np.zeros((G.shape[1], G.shape[2]))
    rn = np.zeros(G.shape[1])
    pn = np.zeros(U3.shape[0])
    lib.oracle_subtype(Jp, ctypes.c_int32(U3.shape[0]), Gp, cp, up, S.ctypes.data_as(_f64p),
                       rn.ctypes.data_as(_f64p), pn.ctypes.data_as(_f64p))
    return S, rn, pn


def kmeans(X, init, max_iter=100):
    """Lloyd's k-means of the rows of X from the initial centroids (Sec. 3.1.1, reading R14):
    (assignment int32, centroids float64, centroid updates made, inertia)."""
    lib = _load()
    X, xp = _f64(X)
    cent = np.array(init, dtype=np.float64, order="C")
    n, d = X.shape
    k = cent.shape[0]
    assign = np.zeros(n, dtype=np.int32)
    inertia = ctypes.c_double()
    it = lib.oracle_kmeans(xp, ctypes.c_int64(n), ctypes.c_int32(d), ctypes.c_int32(k),
                           cent.ctypes.data_as(_f64p), ctypes.c_int32(max_iter),
                           assign.ctypes.data_as(_i32p), ctypes.byref(inertia))
    return assign, cent, int(it), inertia.value
