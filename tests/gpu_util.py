"""Shared helpers of the GPU tests: build/load the engine once, fail loudly."""
import os

import pytest


def engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5072_gb300 import build
    if not os.path.exists(build.SO):
        build.build()
    import paper_1204_5072_gb300 as eng
    eng.load()
    return eng
