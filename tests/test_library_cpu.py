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
