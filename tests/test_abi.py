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


def test_descriptor_checks_come_before_the_device():
    """Without a GPU, iedg_create_mesh still validates the descriptor first: unknown
    precision or stabilisation codes are UNSUPPORTED, every valid code (FP64, mixed,
    mixed with TF32 or BF16 Schur operands) reaches the device check and fails there
    with IEDG_ERR_CUDA; no handle is returned either way."""
    import ctypes
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1605_01020_gb300 import build, iedg
    from paper_1605_01020_gb300 import workloads as W
    build.build()
    lib = iedg.load()
    wl = W.config(1, N=2)
    X = np.ascontiguousarray(wl.mesh.node_xyz, dtype=np.float64)
    ET = np.ascontiguousarray(wl.mesh.elem_trace, dtype=np.int64)

    def create(precision, stab=0, dim=2, order=wl.mesh.p, quad_extra=2, n_elem=X.shape[0], gamma=1.4, flags=0):
        desc = iedg.MeshDesc(dim, order, quad_extra, precision, n_elem, wl.mesh.n_trace, X.ctypes.data,
                             ET.ctypes.data, gamma, 0.72, 1e3, 0.2, 0.0, stab, flags)
        h = ctypes.c_void_p()
        rc = lib.iedg_create_mesh(ctypes.byref(desc), ctypes.c_void_p(0), ctypes.byref(h))
        assert not h.value
        return rc

    for prec in (iedg.PRECISION_FP64, iedg.PRECISION_MIXED, iedg.PRECISION_MIXED_TF32, iedg.PRECISION_MIXED_BF16):
        assert create(prec) == -2, prec
    assert create(4) == -6
    assert create(-1) == -6
    assert create(0, stab=2) == -6
    # degenerate and out-of-range descriptors
    assert create(0, dim=4) == -1                 # dimension
    assert create(0, order=4) == -6               # 2D orders 1..3
    assert create(0, order=0) == -6
    assert create(0, quad_extra=0) == -6
    assert create(0, n_elem=0) == -1              # empty mesh
    assert create(1, flags=iedg.FLAG_MASS_SCALING) == -2    # valid: fails only for want of a device
    assert create(0, flags=iedg.FLAG_MASS_SCALING) == -1    # mass scaling is for the mixed forms
    assert create(1, flags=4) == -1                         # unknown flag
    assert create(0, gamma=1.0) == -1             # physical parameters


def test_autotune_candidates_keep_the_precision():
    """Schedules change how, never what: handles with TF32 / BF16 Schur operands are
    offered only the tensor-core LU; FP32 handles the FFMA form and both tensor-core forms
    (deferred Schur complement, every trailing update); FP64 handles the DFMA
    forms plus the exact-splitting tensor-core form (persistent grid, panel 16)."""
    from paper_1605_01020_gb300 import autotune
    for prec in (2, 3):
        c = autotune.candidates(prec, 3)
        assert c and all(s["lu_tensor"] == 1 for s in c)
    c1 = autotune.candidates(1, 3)
    assert {s["lu_tensor"] for s in c1} == {0, 1, 2}
    c0 = autotune.candidates(0, 3)
    assert {s["lu_tensor"] for s in c0} == {0, 1}
    assert all(s["lu_persistent"] == 1 and s["lu_panel"] == 16 for s in c0 if s["lu_tensor"] == 1)
    assert len({tuple(sorted(s.items())) for s in c0}) == len(c0)
