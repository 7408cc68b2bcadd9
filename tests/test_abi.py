"""The C-ABI library loads and exports every entry point include/*.h declares
(no GPU needed: no compute call is made here), and the host-side error
paths that need no device behave."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2506_10399_gb300 import build
    build.build()
    from paper_2506_10399_gb300 import _native
    return _native


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(fg_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(native):
    names = declared_symbols()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = names - exported
    assert not missing, missing
    for n in names:
        assert hasattr(native.lib, n)


def test_binding_declares_every_symbol(native):
    assert declared_symbols() == set(native.SIGS)


def test_null_arguments_are_rejected_without_a_device(native):
    # argument checks that happen before any device work
    assert native.lib.fg_ctx_create(None, None, None) == -1
    assert native.lib.fg_ctx_destroy(None) == 0
    assert native.lib.fg_plan_destroy(None) == 0
    assert native.lib.fg_keys_destroy(None) == 0
    assert native.lib.fg_last_error(None)


def test_oracle_is_never_imported_by_the_library():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|#include\s+[<\"][^>\"]*oracle", re.M)
    for path in glob.glob(os.path.join(ROOT, "paper_2506_10399_gb300", "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
            assert not pat.search(open(path).read()), path
