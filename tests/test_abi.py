"""CPU-side checks of the C ABI: the shared library builds, loads and exports every
symbol include/iedg.h declares; calls without a GPU fail loudly."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "iedg.h")).read()
    return sorted(set(re.findall(r"\b(iedg_[a-z0-9_]+)\s*\(", src)))


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


@pytest.mark.parametrize("d,N,levels", [(2, 5, (1, 2, 3)), (3, 3, (2, 3, 4)), (3, 4, (1, 4))])
def test_mixed_slot_counts_match_the_mesh_builder(d, N, levels):
    """The binding checks ragged sizes before handing pointers to the library; its
    slot count must agree with the mesh builder's slot lists for every element."""
    import numpy as np
    from paper_1605_01020_gb300 import workloads as W
    from paper_1605_01020_gb300.iedg import _slot_count
    probs = np.full(len(levels), 1.0 / len(levels))
    orders = W.mixed_orders([N] * d, 3, levels=levels, probs=probs)
    mesh = W.structured_mesh_mixed(d, N, orders)
    for e in range(mesh.n_elem):
        assert len(mesh.elem_trace[e]) == _slot_count(d, int(mesh.orders[e]), tuple(mesh.face_degree[e].tolist()))
        assert len(mesh.node_xyz[e]) == (int(mesh.orders[e]) + 1) ** d


def test_mixed_mesh_without_gpu_is_an_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1605_01020_gb300 import iedg
    from paper_1605_01020_gb300 import workloads as W
    orders = W.mixed_orders([3, 3], 1, levels=(1, 2), probs=(0.5, 0.5))
    mesh = W.structured_mesh_mixed(2, 3, orders)
    with pytest.raises(Exception):
        iedg.MixedOrderMesh(mesh.node_xyz, mesh.elem_trace, mesh.n_trace, mesh.orders, mesh.face_degree)
