"""Host-side checks of the C-ABI library (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
include/transec.h declares; without a GPU it must refuse to create a context with
a status code instead of crashing.
"""

import os
import re

import pytest

import paper_2208_02783_gb300 as pkg
from paper_2208_02783_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(transec_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = pkg.load(path)
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(binding.EXPORTED) >= declared


def test_status_strings_and_version():
    pkg.load()
    assert pkg.transec_version() >= 10000
    assert pkg.transec_status_string(0) == "ok"
    assert "maxit" in pkg.transec_status_string(-4)


def test_create_without_gpu_returns_status():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.TransecError) as ei:
        pkg.transec_create(4, 4, 8, 0.5, 0.5, 0.5, 2)
    assert ei.value.status in (pkg.ECUDA, pkg.EINVAL)


def test_invalid_geometry_rejected_before_device_use():
    with pytest.raises(pkg.TransecError) as ei:
        pkg.transec_create(4, 4, 8, 0.5, 0.5, 0.5, 3)  # odd order
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.TransecError):
        pkg.transec_create(0, 4, 8, 0.5, 0.5, 0.5, 2)


def test_network_and_fgmres_arguments_rejected_before_device_use():
    import ctypes as C

    lib = pkg.load()
    out = C.c_void_p()
    # the network needs every dimension a positive multiple of 4 (two 2x poolings)
    for dims in ((6, 8, 8), (8, 8, 2), (0, 8, 8), (8, -4, 8)):
        assert lib.transec_unet_create(C.byref(out), 0, *dims, 0) == pkg.EINVAL
        assert out.value is None
    assert lib.transec_unet_create(None, 0, 8, 8, 8, 0) == pkg.EINVAL
    n = C.c_longlong()
    assert lib.transec_unet_n_params(None, C.byref(n)) == pkg.EINVAL
    assert lib.transec_unet_dims(None, None, None, None) == pkg.EINVAL
    assert lib.transec_unet_forward(None, None, None, 0) == pkg.EINVAL
    assert lib.transec_unet_train_step(None, None, None, 0.0, None, None, 0) == pkg.EINVAL
    assert lib.transec_unet_train_operator(None, None, 1, 10, 0.0, 1.0, 1e-3, 0, None) == pkg.EINVAL
    assert lib.transec_fgmres_columns(None, None, 2, 1, None, None, None, 30, 100, None, None, None,
                                      None) == pkg.EINVAL
    assert lib.transec_shifted_column(None, 1, None, 0, 0, None, None, None, None) == pkg.EINVAL
    lib.transec_unet_destroy(None)  # ignored
