"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function declared in include/lre.h; the binding covers all of them."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "lre.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lre_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if subprocess.call(["which", "nvcc"], stdout=subprocess.DEVNULL) != 0 and \
            not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1602_08604_gb300 import build, lre
    build.build()
    return lre.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["lre_create", "lre_destroy", "lre_estimate", "lre_parity_sums", "lre_assemble",
                 "lre_project", "lre_histogram", "lre_sync", "lre_status_string"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only",
                                   os.path.join(ROOT, "paper_1602_08604_gb300", "liblre.so")], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    from paper_1602_08604_gb300 import lre
    bound = {name for name, _, _ in lre.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings_without_gpu(lib):
    from paper_1602_08604_gb300 import lre
    assert lre.lre_status_string(0) == "ok"
    assert "shots" in lre.lre_status_string(3)


def test_arguments_rejected_before_any_device_work(lib):
    import ctypes
    # NULL context and NULL out-pointer are rejected synchronously
    assert lib.lre_estimate(None, None, 0, None, 1, 3, None, None, None) == 1
    assert lib.lre_create(None, 0) == 1
    assert lib.lre_sync(None, None) == 1
    assert lib.lre_profile_count(None) == 0
    n = ctypes.c_size_t()
    assert lib.lre_workspace_size(None, 4, 0, 0, ctypes.byref(n)) == 1
    j = ctypes.c_int(-1)
    assert lib.lre_batch_schedule(None, ctypes.byref(j), None, None, None) == 1
    assert j.value == -1
