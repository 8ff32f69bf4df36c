"""CPU-side checks of the C ABI: the shared library builds, loads and exports every
symbol include/iedg.h declares; calls without a GPU fail loudly."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "iedg.h")).read()
    return sorted(set(re.findall(r"\b(iedg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1605_01020_gb300 import build, iedg
    build.build()
    lib = iedg.load()
    names = _declared()
    assert set(names) == set(iedg.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_no_gpu_means_error_not_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1605_01020_gb300 import iedg
    from paper_1605_01020_gb300 import workloads as W
    wl = W.config(1, N=2)
    with pytest.raises(Exception):
        iedg.mesh_from_workload(wl)
