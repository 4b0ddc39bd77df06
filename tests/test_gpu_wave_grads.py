"""The fast sweep checked element by element: what one wave's sweep accumulates.

Inside a fast-mode wave every entry's gradient is evaluated at the wave-start parameters
and summed (the gradient equation of Sec. 2.3.2, data term; each row's L2 term is added once
at the wave end).  So what the sweep kernel accumulates before the wave's end step is a
plain, order-free quantity: per patient row, per gene row and per platform the summed
data-term gradients, and per platform M_k = sum r a b^T, from which the core's data-term
gradient is sum_k M_k o c_k and platform row k's is G_(3) vec(M_k).  The FP64 oracle sums
the same per-entry gradients (oracle.data_grad_sums, pinned by finite differences), so every
value is compared: |gpu - oracle| <= tol (|oracle| + rms), tol 1e-5 for the FP32 sweeps.  The
counts of each row's entries per platform in the wave (the row steps' weights) are integers
and must match exactly.

Every compiled path of the sweep is driven: the lane-group and the warp-per-unit per-run
sweeps (5x5x2, 10x10x5, 16x16x5), the tile-claiming variant (16x16x5 with 20 platforms, every platform's
Gc beyond the shared-memory budget), the variant that counts with atomics (64 platforms,
1,024-entry waves), the per-entry sweep (32x32x5, and runtime ranks 3x7x4), and the two BF16
forms, BF16 gene-row gathers and the tensor-core sweep (norm-wise within 8 units of BF16
roundoff, each element within 32: their operands are rounded to BF16).  Each at the initial
parameters and again after two epochs, on the first, a middle and the last (ragged) wave.
"""
import numpy as np
import pytest

import oracle
import snect_synth as S

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
# BF16 keeps 8 significant bits: unit roundoff u = 2^-8.  The BF16 sweeps round gathered rows
# (and, on the tensor cores, a and Gc = G x3 c) to BF16 before their J-term products, so each
# product carries up to 2u of relative error and a sum of J terms of mixed sign up to
# 2u sum|terms|, several times |sum| at J = 16, and a row's sum over its entries adds such
# errors of either sign.  The BF16 forms are therefore held norm-wise, per output (patient
# rows, gene rows, core, platform rows): ||gpu - oracle|| <= 8u ||oracle||, with every single
# element within 32u (|oracle| + rms) as a guard against a systematic error.
U_BF16 = 2.0 ** -8
TOL_BF16 = 32 * U_BF16
TOL_BF16_NORM = 8 * U_BF16


def close(got, want, tol):
    got = np.asarray(got, np.float64)
    rms = float(np.sqrt(np.mean(want * want))) if want.size else 0.0
    err = np.abs(got - want) / (np.abs(want) + rms + 1e-30)
    return float(err.max()) if err.size else 0.0


def normwise(got, want):
    got = np.asarray(got, np.float64)
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30))


def check_waves(p, tol, precision=0, wave=0, epochs_between=2, entries=None):
    import paper_1711_08095_gb300 as snect

    idx, val = entries if entries is not None else (p.idx, p.val)
    c = snect.Snect(p.I, p.J, idx, val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                    batch=0, wave=wave, precision=precision)
    report = []
    for stage in range(2):
        if stage:
            c.epoch(epochs_between)
        G, U = c.get_factors()
        P = oracle.Params(G, U)
        first = c.wave_grads(0)
        n_waves = -(-p.nnz // first["count"]) if first["count"] else 0
        n_waves += n_waves & 1
        for w in sorted({0, n_waves // 2, n_waves - 1}):
            got = c.wave_grads(w)
            want = oracle.data_grad_sums(p.I, P, p.idx, p.val, got["first"], got["count"])
            assert got["count"] > 0 and got["first"] + got["count"] <= p.nnz
            M = got["M"].astype(np.float64)
            gG = np.einsum("kpq,kr->pqr", M, U[2].astype(np.float64))
            gC = np.einsum("pqr,kpq->kr", G.astype(np.float64), M)
            errs = {"gA": close(got["gA"], want["gA"], tol), "gB": close(got["gB"], want["gB"], tol),
                    "gG": close(gG, want["gG"], tol), "gC": close(gC, want["gC"], tol)}
            report.append((stage, w, errs))
            assert max(errs.values()) <= tol, (p.J, stage, w, errs, report)
            if precision:
                nw = {"gA": normwise(got["gA"], want["gA"]), "gB": normwise(got["gB"], want["gB"]),
                      "gG": normwise(gG, want["gG"]), "gC": normwise(gC, want["gC"])}
                assert max(nw.values()) <= TOL_BF16_NORM, (p.J, stage, w, nw)
            assert np.array_equal(got["nA"], want["nA"].astype(np.float32)), (stage, w, "nA")
            assert np.array_equal(got["nB"], want["nB"].astype(np.float32)), (stage, w, "nB")
    # the diagnostic leaves the factors alone
    G2, U2 = c.get_factors()
    assert np.array_equal(G2, G) and all(np.array_equal(a, b) for a, b in zip(U2, U))
    c.close()
    print("wave-gradient parity", p.J, p.I, ["%d/%d %s" % (s, w, {k: "%.1e" % v for k, v in e.items()})
                                              for s, w, e in report])


@pytest.fixture(params=["lanes", "warp"])
def sweep_kernel(request, monkeypatch):
    """The two complete sweep kernels for compile-time ranks up to 16: the lane-group kernel
    (the default) and the warp-per-unit kernel (SNECT_SWEEP_KERNEL=warp, read at set-up)."""
    if request.param == "warp":
        monkeypatch.setenv("SNECT_SWEEP_KERNEL", "warp")
    else:
        monkeypatch.delenv("SNECT_SWEEP_KERNEL", raising=False)
    return request.param


@pytest.mark.parametrize("J", [(5, 5, 2), (10, 10, 5), (16, 16, 5)])
def test_static_partition_sweep(J, sweep_kernel, gpu_lib):
    p = S.config2(n_patients=150, nnz=200_000, n_edges=10_000, J_fit=J)
    check_waves(p, TOL32)


def test_tile_claiming_sweep_many_platforms(gpu_lib):
    p = S.config2(n_patients=120, n_genes=3000, n_platforms=20, nnz=200_000, n_edges=5_000, J_true=(5, 5, 2),
                  J_fit=(16, 16, 5))
    check_waves(p, TOL32)


def test_count_atomics_sweep_small_waves(gpu_lib):
    """With 1,024-entry waves on 64 platforms the per-wave count table would outgrow the
    entries, so the sweep counts each row's entries per platform with atomics."""
    p = S.config2(n_patients=120, n_genes=3000, n_platforms=64, nnz=100_000, n_edges=5_000, J_true=(5, 5, 2),
                  J_fit=(5, 5, 2))
    check_waves(p, TOL32, wave=1024)


@pytest.mark.parametrize("J", [(32, 32, 5), (3, 7, 4)])
def test_per_entry_sweep(J, gpu_lib):
    p = S.config2(n_patients=100, n_genes=3000, nnz=100_000, n_edges=5_000, J_fit=J)
    check_waves(p, TOL32)


@pytest.mark.parametrize("form", ["bf16_gather", "bf16_tensor_cores"])
def test_bf16_sweeps(form, gpu_lib):
    """SNECT_BF16 at 16 x 16 x 5 gathers the gene rows from their BF16 copy (the lane-group
    kernel); SNECT_BF16_TC runs the dense per-entry contractions on tcgen05."""
    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=150, nnz=200_000, n_edges=10_000, J_fit=(16, 16, 5))
    check_waves(p, TOL_BF16, precision=snect.BF16 if form == "bf16_gather" else snect.BF16_TC)


def _inputs(p, memory):
    """The training entries in the given kind of memory; "+1" views start 4 bytes past a
    16-byte boundary."""
    import torch

    if memory == "pageable":
        return p.idx, p.val
    off = 1 if memory.endswith("+1") else 0
    kw = dict(device="cuda") if memory.startswith("device") else dict(pin_memory=True)
    out = []
    for a in (p.idx, p.val):
        flat = torch.from_numpy(np.ascontiguousarray(a).reshape(-1))
        buf = torch.empty(flat.numel() + off, dtype=flat.dtype, **kw)
        buf[off:].copy_(flat)
        out.append(buf[off:].view(a.shape))
    return tuple(out)


@pytest.mark.parametrize("memory", ["pageable", "pinned", "device", "pinned+1", "device+1"])
def test_set_up_reads_the_entries_where_they_are(memory, gpu_lib):
    """The counting form of the set-up packs, validates, counts and orders the entries in one
    pass that reads them where the caller has them; aligned inputs arrive as 16-byte vector
    loads, the "+1" views through the scalar loads.  200,003 entries: the last 128-entry chunk
    is ragged, and the waves (1,999 entries) do not divide the chunks."""
    p = S.config2(n_patients=150, nnz=222_226, n_edges=10_000)
    assert p.nnz % 128 != 0
    check_waves(p, TOL32, wave=1999, entries=_inputs(p, memory))


def test_set_up_radix_form_for_large_bucket_tables(gpu_lib):
    """20,000 patients x 5 platforms x 196 waves of 1,024 entries are 19.6M (wave, platform,
    patient) buckets, above the counting form's limit: the set-up sorts the entries by radix
    instead (and the wave table exceeds its budget, so the sweep counts with atomics)."""
    p = S.config2(n_patients=20_000, n_genes=1_000, nnz=222_000, n_edges=3_000, J_true=(5, 5, 2),
                  J_fit=(5, 5, 2))
    check_waves(p, TOL32, wave=1024)


@pytest.mark.parametrize("memory", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("case", ["index", "nan"])
def test_set_up_rejects_invalid_entries(memory, case, gpu_lib):
    import paper_1711_08095_gb300 as snect

    p = S.config2(n_patients=60, n_genes=2000, nnz=40_000, n_edges=3_000)
    idx, val = p.idx.copy(), p.val.copy()
    if case == "index":
        idx[12_345, 2] = p.I[2]
    else:
        val[33_333] = np.inf
    q = S.Problem(**{**p.__dict__, "idx": idx, "val": val})
    with pytest.raises(snect.SnectError) as ei:
        snect.Snect(p.I, p.J, *_inputs(q, memory), p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr,
                    batch=0)
    assert ei.value.code == -1
