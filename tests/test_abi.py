"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(krr_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1805_00569_gb300 import build
    path = build.build() if build.stale() else build.LIB
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_symbols()
    for n in ("krr_partition", "krr_fit_batch", "krr_predict", "krr_select", "krr_ctx_create",
              "krr_ctx_destroy", "krr_model_free"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_no_oracle_in_the_product():
    """The CUDA path shares no code with the oracle and never loads it."""
    pkg = os.path.join(ROOT, "paper_1805_00569_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(f).read()
            assert "import oracle" not in text and "from oracle" not in text and "krr_oracle" not in text, f


def test_library_targets_sm103a_only():
    from paper_1805_00569_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_device_fails_loudly(lib):
    """Without a CUDA device the C ABI refuses a context (status, no handle)
    and the binding raises: nothing falls back to the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p(1)
    lib.krr_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]
    rc = lib.krr_ctx_create(ctypes.byref(h), 0, None, 0)
    assert rc != 0 and h.value is None
    import paper_1805_00569_gb300 as krr
    with pytest.raises(krr.KrrError):
        krr.krr_ctx_create()
