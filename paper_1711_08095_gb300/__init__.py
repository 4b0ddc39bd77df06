"""GB300 SNeCT: network-constrained Tucker decomposition by SGD on one GPU.

Thin Python binding of the C ABI in ``include/snect.h`` (library ``libsnect.so``, built
from ``csrc/`` by ``build.py``).  Every computation runs in the library's CUDA kernels;
this module only marshals arguments.  Importing the package does not need a GPU;
creating a context does, and there is no CPU fallback: if the library is missing or no
GPU is visible the calls raise.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA memory); the
library copies them during the call.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

__all__ = ["Config", "LossTerms", "Snect", "SnectError", "load", "lib_path", "EXPORTS", "FP32", "BF16", "BF16_TC"]

FP32 = 0
BF16 = 1
BF16_TC = 2

# every symbol include/snect.h declares
EXPORTS = (
    "snect_init",
    "snect_epoch",
    "snect_batches",
    "snect_edge_pass",
    "snect_loss",
    "snect_get_factors",
    "snect_set_factors",
    "snect_foldin",
    "snect_topk",
    "snect_foldin_static",
    "snect_qr_post",
    "snect_batch_create",
    "snect_batch_epoch",
    "snect_batch_tuning",
    "snect_batch_launch_count",
    "snect_batch_last_error",
    "snect_batch_destroy",
    "snect_serve_start",
    "snect_serve_submit",
    "snect_serve_poll",
    "snect_serve_stats",
    "snect_serve_stop",
    "snect_set_sweep_timing",
    "snect_sweep_times",
    "snect_subtype",
    "snect_kmeans",
    "snect_hogwild_epoch",
    "snect_kernel_times",
    "snect_wave_grads",
    "snect_launch_count",
    "snect_last_error",
    "snect_destroy",
)


class SnectError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("snect error %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_int32 * 3),
        ("J", ctypes.c_int32 * 3),
        ("lambda_", ctypes.c_float),
        ("lambda_g", ctypes.c_float),
        ("lr", ctypes.c_float),
        ("batch", ctypes.c_int32),
        ("wave", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class LossTerms(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_double),
        ("reg", ctypes.c_double),
        ("graph", ctypes.c_double),
        ("total", ctypes.c_double),
        ("rmse_train", ctypes.c_double),
        ("rmse_test", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libsnect.so (optionally building it first) and declares the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError("libsnect.so is not built; run paper_1711_08095_gb300.build.build() "
                          "(or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    sig = {
        "snect_init": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(Config), P, P, i64, P, P, i64, P, P, P, P, P]),
        "snect_epoch": (ctypes.c_int, [P, i32]),
        "snect_batches": (ctypes.c_int, [P, i64, i64]),
        "snect_edge_pass": (ctypes.c_int, [P]),
        "snect_loss": (ctypes.c_int, [P, P, P, i64, ctypes.POINTER(LossTerms)]),
        "snect_get_factors": (ctypes.c_int, [P, P, P, P, P]),
        "snect_set_factors": (ctypes.c_int, [P, P, P, P, P]),
        "snect_foldin": (ctypes.c_int, [P, P, P, i64, P]),
        "snect_topk": (ctypes.c_int, [P, P, i32, P, P]),
        "snect_serve_start": (ctypes.c_int, [P, i32, i64, i32, ctypes.POINTER(P)]),
        "snect_serve_submit": (ctypes.c_int, [P, P, P, i64, i32, ctypes.POINTER(ctypes.c_int64)]),
        "snect_serve_poll": (ctypes.c_int, [P, i64, i32, P, P, P, ctypes.POINTER(ctypes.c_double)]),
        "snect_serve_stats": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64)]),
        "snect_serve_stop": (ctypes.c_int, [P]),
        "snect_qr_post": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32)]),
        "snect_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(P), i32, P]),
        "snect_batch_epoch": (ctypes.c_int, [P, i32]),
        "snect_batch_tuning": (ctypes.c_int, [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                              ctypes.POINTER(ctypes.c_double)]),
        "snect_batch_launch_count": (ctypes.c_int64, [P]),
        "snect_batch_last_error": (ctypes.c_char_p, [P]),
        "snect_batch_destroy": (None, [P]),
        "snect_foldin_static": (ctypes.c_int, [P, P, P, i32, i32, i32, i32, i32, P, P, i64, ctypes.c_float, P, P]),
        "snect_set_sweep_timing": (ctypes.c_int, [P, ctypes.c_int32]),
        "snect_sweep_times": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64)]),
        "snect_subtype": (ctypes.c_int, [P, P, i64, P, P, P]),
        "snect_kmeans": (ctypes.c_int, [P, i32, P, i32, P, P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]),
        "snect_hogwild_epoch": (ctypes.c_int, [P, P, i64, i32, i32]),
        "snect_kernel_times": (ctypes.c_int, [P, P, P]),
        "snect_wave_grads": (ctypes.c_int, [P, i64, P, P, P, P, P, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]),
        "snect_launch_count": (ctypes.c_int64, [P]),
        "snect_last_error": (ctypes.c_char_p, [P]),
        "snect_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, keep: list, dtype) -> Optional[int]:
    """Address of a contiguous array of the given numpy dtype (numpy or torch)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch

        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        keep.append(a)
        return a.data_ptr() if a.numel() else None
    arr = np.ascontiguousarray(a, dtype=dtype)
    keep.append(arr)
    return arr.ctypes.data if arr.size else None


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Snect:
    """One decomposition problem resident on the GPU (a snect_ctx)."""

    def __init__(self, I: Sequence[int], J: Sequence[int], idx, val, edges, w, G0, U0, *, lam: float,
                 lam_g: float, lr: float, batch: int = 0, wave: int = 0, stream=None, precision: int = FP32):
        self._lib = load()
        cfg = Config()
        cfg.I[:] = [int(x) for x in I]
        cfg.J[:] = [int(x) for x in J]
        cfg.lambda_, cfg.lambda_g, cfg.lr = float(lam), float(lam_g), float(lr)
        cfg.batch, cfg.wave, cfg.precision, cfg.seed = int(batch), int(wave), int(precision), 0
        self.I, self.J = tuple(cfg.I), tuple(cfg.J)
        keep = []
        nnz = int(val.shape[0])
        m = int(w.shape[0])
        h = ctypes.c_void_p()
        st = _current_stream() if stream is None else stream
        rc = self._lib.snect_init(ctypes.byref(h), ctypes.byref(cfg), _ptr(idx, keep, np.int32),
                                  _ptr(val, keep, np.float32), nnz, _ptr(edges, keep, np.int32),
                                  _ptr(w, keep, np.float32), m, _ptr(G0, keep, np.float32),
                                  _ptr(U0[0], keep, np.float32), _ptr(U0[1], keep, np.float32),
                                  _ptr(U0[2], keep, np.float32), st)
        if rc != 0:
            raise SnectError(rc, self._lib.snect_last_error(None).decode())
        self._h = h
        self.nnz, self.m = nnz, m

    # -- helpers --------------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise SnectError(rc, self._lib.snect_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.snect_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path -------------------------------------------------------------------------
    def epoch(self, n: int = 1):
        self._check(self._lib.snect_epoch(self._h, int(n)))

    def batches(self, first: int, count: int = 1):
        self._check(self._lib.snect_batches(self._h, int(first), int(count)))

    def edge_pass(self):
        self._check(self._lib.snect_edge_pass(self._h))

    def loss(self, test_idx=None, test_val=None) -> dict:
        keep = []
        out = LossTerms()
        n = 0 if test_val is None else int(test_val.shape[0])
        self._check(self._lib.snect_loss(self._h, _ptr(test_idx, keep, np.int32) if n else None,
                                         _ptr(test_val, keep, np.float32) if n else None, n,
                                         ctypes.byref(out)))
        return out.as_dict()

    def get_factors(self):
        G = np.empty(self.J, dtype=np.float32)
        U = [np.empty((self.I[n], self.J[n]), dtype=np.float32) for n in range(3)]
        self._check(self._lib.snect_get_factors(self._h, G.ctypes.data, U[0].ctypes.data, U[1].ctypes.data,
                                                U[2].ctypes.data))
        return G, U

    def set_factors(self, G=None, U=(None, None, None)):
        keep = []
        self._check(self._lib.snect_set_factors(self._h, _ptr(G, keep, np.float32), _ptr(U[0], keep, np.float32),
                                                _ptr(U[1], keep, np.float32), _ptr(U[2], keep, np.float32)))

    def foldin(self, jk, val) -> np.ndarray:
        keep = []
        u = np.empty(self.J[0], dtype=np.float32)
        self._check(self._lib.snect_foldin(self._h, _ptr(jk, keep, np.int32), _ptr(val, keep, np.float32),
                                           int(val.shape[0]), u.ctypes.data))
        return u

    def topk(self, u, k: int = 10):
        keep = []
        idx = np.empty(k, dtype=np.int32)
        sc = np.empty(k, dtype=np.float32)
        self._check(self._lib.snect_topk(self._h, _ptr(u, keep, np.float32), int(k), idx.ctypes.data,
                                         sc.ctypes.data))
        return idx, sc

    def set_sweep_timing(self, mode: int):
        """Sweep launches timed per epoch: 0 none (default), 1 the middle one, -1 all, 2 every
        kernel of the epoch (see kernel_times)."""
        self._check(self._lib.snect_set_sweep_timing(self._h, int(mode)))

    def sweep_times(self):
        """(summed ms, launches, entries) of the timed sweep kernels of the most recent epoch."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        e = ctypes.c_int64()
        self._check(self._lib.snect_sweep_times(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(e)))
        return ms.value, n.value, e.value

    def subtype(self, u):
        """Personalised subtype analysis (Sec. 3.3) of profiles u ((n, J1) or (J1,)): (S (n, J2,
        J3), row norms (n, J2), platform norms (n, I3))."""
        keep = []
        u2 = u if hasattr(u, "data_ptr") else np.ascontiguousarray(u, np.float32)
        n = int(u2.shape[0]) if len(u2.shape) == 2 else 1
        J, I = self.J, self.I
        S = np.empty((n, J[1], J[2]), np.float32)
        rn = np.empty((n, J[1]), np.float32)
        pn = np.empty((n, I[2]), np.float32)
        self._check(self._lib.snect_subtype(self._h, _ptr(u2, keep, np.float32), n, S.ctypes.data, rn.ctypes.data,
                                            pn.ctypes.data))
        return S, rn, pn

    def kmeans(self, init, max_iter: int = 100):
        """k-means of the rows of U1 (Sec. 3.1.1) from initial centroids init (k x J1):
        (assignment int32, centroids float64, centroid updates, inertia)."""
        init = np.ascontiguousarray(init, np.float64)
        k = int(init.shape[0])
        assign = np.empty(self.I[0], np.int32)
        cent = np.empty((k, self.J[0]), np.float64)
        upd = ctypes.c_int32()
        inertia = ctypes.c_double()
        self._check(self._lib.snect_kmeans(self._h, k, init.ctypes.data, int(max_iter), assign.ctypes.data,
                                           cent.ctypes.data, ctypes.byref(upd), ctypes.byref(inertia)))
        return assign, cent, upd.value, inertia.value

    def hogwild_epoch(self, order, P: int, n: int = 1):
        """n epochs of the lock-free form of Alg. 1 with P workers over one interleaved order of
        entries and edges (snect_hogwild_epoch)."""
        keep = []
        n_items = int(order.shape[0])
        self._check(self._lib.snect_hogwild_epoch(self._h, _ptr(order, keep, np.int32), n_items, int(P), int(n)))

    def kernel_times(self):
        """Under timing mode 2: {class: (summed ms, launches)} of the most recent epoch for the
        entry sweeps, the wave ends (or deterministic apply kernels) and the network pass."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        self._check(self._lib.snect_kernel_times(self._h, ms, n))
        return {k: (ms[t], n[t]) for t, k in enumerate(("sweep", "wave_end", "network_pass"))}

    def wave_grads(self, w: int):
        """One wave's entry sweep alone at the current parameters (snect_wave_grads): dict of
        gA (I1 x J1), gB (I2 x J2), M (I3 x J1 x J2), nA (I1 x I3), nB (I2 x I3) and the wave's
        entry range (first, count) in the visit order."""
        I, J = self.I, self.J
        out = dict(gA=np.empty((I[0], J[0]), np.float32), gB=np.empty((I[1], J[1]), np.float32),
                   M=np.empty((I[2], J[0], J[1]), np.float32), nA=np.empty((I[0], I[2]), np.float32),
                   nB=np.empty((I[1], I[2]), np.float32))
        first, count = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.snect_wave_grads(self._h, int(w), *(out[k].ctypes.data for k in
                                                                  ("gA", "gB", "M", "nA", "nB")),
                                               ctypes.byref(first), ctypes.byref(count)))
        out["first"], out["count"] = first.value, count.value
        return out

    def serve(self, n_slots: int = 8, mem_budget_bytes: int = 1 << 30, max_cells: int = 75_000):
        """Starts a continuous-batching fold-in + top-k server on this context's factors."""
        return Server(self, n_slots, mem_budget_bytes, max_cells)

    def qr_post(self):
        """QR orthogonalisation post-pass in place; returns the bit mask of modes left as they
        were (J_n > I_n)."""
        sk = ctypes.c_int32(0)
        self._check(self._lib.snect_qr_post(self._h, ctypes.byref(sk)))
        return int(sk.value)

    @property
    def launches(self) -> int:
        return int(self._lib.snect_launch_count(self._h))

    @property
    def handle(self):
        return self._h


class Server:
    """A running snect_server (see snect_serve_* in include/snect.h)."""

    def __init__(self, ctx: "Snect", n_slots: int, mem_budget_bytes: int, max_cells: int):
        self._lib = ctx._lib
        self._ctx = ctx
        self.J1 = ctx.J[0]
        h = ctypes.c_void_p()
        rc = self._lib.snect_serve_start(ctx.handle, int(n_slots), int(mem_budget_bytes), int(max_cells),
                                         ctypes.byref(h))
        if rc != 0:
            raise SnectError(rc, self._lib.snect_last_error(ctx.handle).decode())
        self._h = h

    def submit(self, jk, val, k: int = 10) -> int:
        jk = np.ascontiguousarray(jk, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float32)
        t = ctypes.c_int64()
        rc = self._lib.snect_serve_submit(self._h, jk.ctypes.data, val.ctypes.data, int(val.shape[0]), int(k),
                                          ctypes.byref(t))
        if rc != 0:
            raise SnectError(rc, "submit rejected (size, k, or server stopping)")
        return t.value

    def poll(self, ticket: int, k: int = 10, wait: bool = True):
        """(u, idx, score, latency_ms) of a finished ticket, or None if not finished and not waiting."""
        u = np.empty(self.J1, np.float32)
        idx = np.empty(k, np.int32)
        sc = np.empty(k, np.float32)
        lat = ctypes.c_double()
        rc = self._lib.snect_serve_poll(self._h, int(ticket), 1 if wait else 0, u.ctypes.data, idx.ctypes.data,
                                        sc.ctypes.data, ctypes.byref(lat))
        if rc == -5 and not wait:
            return None
        if rc != 0:
            raise SnectError(rc, "request %d failed" % ticket)
        return u, idx, sc, lat.value

    def stats(self):
        a, c, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._lib.snect_serve_stats(self._h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(m))
        return dict(admitted=a.value, completed=c.value, max_concurrent=m.value)

    def stop(self):
        if getattr(self, "_h", None):
            self._lib.snect_serve_stop(self._h)
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class Batch:
    """Several fast-mode contexts stepped together (snect_batch_*): one graph per epoch."""

    def __init__(self, ctxs: Sequence["Snect"], stream=None):
        self._lib = load()
        self._ctxs = list(ctxs)  # kept alive while the batch exists
        arr = (ctypes.c_void_p * len(self._ctxs))(*[c.handle.value for c in self._ctxs])
        h = ctypes.c_void_p()
        st = _current_stream() if stream is None else stream
        rc = self._lib.snect_batch_create(ctypes.byref(h), arr, len(self._ctxs), st)
        if rc != 0:
            raise SnectError(rc, self._lib.snect_batch_last_error(None).decode())
        self._h = h

    def epoch(self, n: int = 1):
        rc = self._lib.snect_batch_epoch(self._h, int(n))
        if rc != 0:
            raise SnectError(rc, self._lib.snect_batch_last_error(self._h).decode())

    @property
    def launches(self) -> int:
        return int(self._lib.snect_batch_launch_count(self._h))

    def tuning(self):
        """The autotuner's choice: dict(ctas_per_sm, oversubscription, min_entries_per_warp,
        sweep_ms)."""
        a, o, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ms = ctypes.c_double()
        self._lib.snect_batch_tuning(self._h, ctypes.byref(a), ctypes.byref(o), ctypes.byref(m), ctypes.byref(ms))
        return dict(ctas_per_sm=a.value, oversubscription=o.value, min_entries_per_warp=m.value, sweep_ms=ms.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.snect_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
