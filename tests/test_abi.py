"""The C ABI library builds, loads and exports every entry point include/snect.h declares.
No compute call is made here (no GPU needed)."""
import os
import re

import pytest

import paper_1711_08095_gb300 as snect

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "snect.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(snect_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert header_symbols() == sorted(snect.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    lib = snect.load(build_if_missing=True)
    for name in header_symbols():
        assert hasattr(lib, name), name
    # exported with C linkage (no C++ mangling) from the in-tree library
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", snect.lib_path()], capture_output=True, text=True).stdout
    defined = set(re.findall(r"\bT (snect_\w+)", out))
    assert set(header_symbols()) <= defined


def test_config_struct_layout_matches_header():
    # int32 I[3], J[3]; float lambda, lambda_g, lr; int32 batch, wave, precision; uint64 seed
    assert snect.Config.seed.offset == 48
    assert snect.LossTerms.rmse_test.offset == 40


def test_oracle_is_not_imported_by_the_library_package():
    src = ""
    pkg = os.path.join(ROOT, "paper_1711_08095_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src += open(os.path.join(dirpath, f)).read()
    assert "import oracle" not in src and "from oracle" not in src and "snect_oracle" not in src


def test_null_handles_are_rejected_before_any_device_work():
    """Every entry point taking a context checks it first: a null handle returns SNECT_EINVAL
    (no CUDA call is made, so this runs without a GPU)."""
    import ctypes

    lib = snect.load(build_if_missing=True)
    EINVAL = -1
    d = ctypes.c_double()
    n = ctypes.c_int64()
    assert lib.snect_epoch(None, 1) == EINVAL
    assert lib.snect_batches(None, 0, 1) == EINVAL
    assert lib.snect_edge_pass(None) == EINVAL
    assert lib.snect_loss(None, None, None, 0, None) == EINVAL
    assert lib.snect_get_factors(None, None, None, None, None) == EINVAL
    assert lib.snect_set_factors(None, None, None, None, None) == EINVAL
    assert lib.snect_qr_post(None, None) == EINVAL
    assert lib.snect_foldin(None, None, None, 1, None) == EINVAL
    assert lib.snect_topk(None, None, 1, None, None) == EINVAL
    assert lib.snect_set_sweep_timing(None, 1) == EINVAL
    assert lib.snect_sweep_times(None, ctypes.byref(d), ctypes.byref(n), None) == EINVAL
    assert lib.snect_launch_count(None) == 0
    lib.snect_destroy(None)
    out = ctypes.c_void_p()
    assert lib.snect_init(ctypes.byref(out), None, None, None, 0, None, None, 0, None, None, None, None,
                          None) == EINVAL
    assert b"null" in lib.snect_last_error(None)


def test_without_a_gpu_the_product_path_fails_loudly():
    """No CPU fallback: where no CUDA device can be used, building a context raises the
    library's error instead of computing anything on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import snect_synth as S

    p = S.config2(n_patients=20, n_genes=50, nnz=500, n_edges=30)
    with pytest.raises(snect.SnectError):
        snect.Snect(p.I, p.J, p.idx, p.val, p.edges, p.w, p.G0, p.U0, lam=p.lam, lam_g=p.lam_g, lr=p.lr, batch=0)
