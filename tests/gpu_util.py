"""Helpers shared by the GPU tests: skip without CUDA, build once, make contexts."""

import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def library():
    from paper_2208_02783_gb300 import build
    import paper_2208_02783_gb300 as pkg

    pkg.load(build.build())
    return pkg


def context(inst, **solver):
    pkg = library()
    return pkg.Transec.from_instance(inst, device=0, **solver)
