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
