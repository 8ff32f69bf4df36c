"""Failure handling of the element-local path, with every failure made on the host
(nothing here faults, traps or hangs the GPU):
  - a NaN in one element's state comes back IEDG_ELEM_NONFINITE;
  - an element whose block is made singular by a zero row (injected between assembly
    and the LU) comes back IEDG_ELEM_SINGULAR;
  - the mixed forms' FP64 refinement cut to zero correction steps leaves the FP32
    solve unrefined: those elements are condensed again in FP64 in the same call
    (IEDG_ELEM_FALLBACK, the FP64 path's results) while fallback slots last, and keep
    IEDG_ELEM_REFINE beyond them;
  - a tensor-core completion wait that is allowed no poll gives up: its CTA drains the
    MMAs in flight, frees its tensor memory and flags its elements (the mixed forms
    then fall back to FP64, the FP64 form reports IEDG_ELEM_TIMEOUT), and the next call
    with the normal limit works and gives the usual results.
Every other element must stay IEDG_ELEM_OK, and clearing the injection restores
normal operation on the same handle."""
import numpy as np
import pytest

from paper_1605_01020_gb300 import workloads as W
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def _wl():
    """3D p=3 on 2^3 cells (8 elements, 320 u-unknowns each: several tensor-core K chunks)."""
    return W.config(2, N=2)


def _mesh(wl, precision):
    from paper_1605_01020_gb300 import iedg
    return iedg.mesh_from_workload(wl, precision=precision)


def _assemble(mesh, st, u=None):
    u = dev(st.u) if u is None else u
    K, R = mesh.assemble_condensed(u, dev(st.q), dev(st.uhat))
    return K, R, mesh.element_status()


@pytest.mark.parametrize("precision,lu_tensor", [(0, 0), (1, 0), (1, 1), (1, 2)])
def test_nan_state_is_flagged_nonfinite(precision, lu_tensor):
    from paper_1605_01020_gb300 import iedg
    wl = _wl()
    st = wl.state
    mesh = _mesh(wl, precision)
    mesh.set_schedule(lu_tensor=lu_tensor)
    u = st.u.copy()
    u[5, 17, 2] = np.nan
    _, _, status = _assemble(mesh, st, dev(u))
    assert status[5] == iedg.ELEM_NONFINITE, status
    assert (np.delete(status, 5) == iedg.ELEM_OK).all(), status
    _, _, status = _assemble(mesh, st)
    assert (status == iedg.ELEM_OK).all(), status


@pytest.mark.parametrize("precision,lu_tensor", [(0, 0), (1, 0), (1, 2), (2, 1)])
def test_zero_row_is_flagged_singular(precision, lu_tensor):
    from paper_1605_01020_gb300 import iedg
    wl = _wl()
    st = wl.state
    mesh = _mesh(wl, precision)
    mesh.set_schedule(lu_tensor=lu_tensor)
    K0, R0, status = _assemble(mesh, st)
    assert (status == iedg.ELEM_OK).all()
    mesh.set_fault_injection(zero_row_elem=3, zero_row=101)
    _, _, status = _assemble(mesh, st)
    assert status[3] == iedg.ELEM_SINGULAR, status
    assert (np.delete(status, 3) == iedg.ELEM_OK).all(), status
    mesh.set_fault_injection()
    K1, R1, status = _assemble(mesh, st)
    assert (status == iedg.ELEM_OK).all()
    assert np.array_equal(host(K1), host(K0)) and np.array_equal(host(R1), host(R0))


def _fp64_reference(wl):
    """K, R, du, dq of the FP64 path on the same inputs."""
    st = wl.state
    mesh = _mesh(wl, 0)
    K, R = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat))
    du, dq = mesh.back_substitute(dev(st.duhat))
    out = [host(t) for t in (K, R, du, dq)]
    mesh.close()
    return out


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", [1, 3])
def test_unrefined_elements_fall_back_to_fp64(precision):
    """Refinement cut to zero correction steps: every element misses 1e-10, is condensed
    again in FP64 in the same call and reports IEDG_ELEM_FALLBACK; K, R and the updates
    are then the FP64 path's."""
    from paper_1605_01020_gb300 import iedg
    wl = _wl()
    st = wl.state
    ref = _fp64_reference(wl)
    mesh = _mesh(wl, precision)
    mesh.set_fault_injection(refine_iters=0)
    K, R, status = _assemble(mesh, st)
    du, dq = mesh.back_substitute(dev(st.duhat))
    assert (status == iedg.ELEM_FALLBACK).all(), status
    for got, want in zip((K, R, du, dq), ref):
        assert _rel(host(got), want) <= 1e-12
    mesh.set_fault_injection()
    K, R, status = _assemble(mesh, st)
    assert (status == iedg.ELEM_OK).all(), status


def test_fallback_slots_run_out():
    """64 elements miss the refinement tolerance and 32 fallback slots exist: the 32
    lowest element ids are condensed again in FP64, the others keep IEDG_ELEM_REFINE."""
    from paper_1605_01020_gb300 import iedg
    wl = W.config(2, N=4)
    st = wl.state
    mesh = _mesh(wl, 1)
    mesh.set_fault_injection(refine_iters=0)
    _, _, status = _assemble(mesh, st)
    assert (status[:32] == iedg.ELEM_FALLBACK).all() and (status[32:] == iedg.ELEM_REFINE).all(), status


@pytest.mark.parametrize("precision,lu_tensor", [(1, 1), (1, 2), (2, 1), (0, 1)])
def test_tensor_core_wait_gives_up_and_recovers(precision, lu_tensor):
    """Every completion wait allowed no poll: the tensor-core LU factors nothing and flags
    its elements; on the mixed forms the FP64 fallback condenses them again in the same
    call (IEDG_ELEM_FALLBACK, the FP64 path's results), the FP64 form reports
    IEDG_ELEM_TIMEOUT.  The next call with the normal limit gives the usual results."""
    from paper_1605_01020_gb300 import iedg
    wl = _wl()
    st = wl.state
    mesh = _mesh(wl, precision)
    mesh.set_schedule(lu_tensor=lu_tensor)
    K0, R0, status = _assemble(mesh, st)
    assert (status == iedg.ELEM_OK).all()
    mesh.set_fault_injection(tc_wait_limit=-1)
    K, R, status = _assemble(mesh, st)
    if precision == 0:
        assert (status == iedg.ELEM_TIMEOUT).all(), status
    else:
        assert (status == iedg.ELEM_FALLBACK).all(), status
        ref = _fp64_reference(wl)
        du, dq = mesh.back_substitute(dev(st.duhat))
        for got, want in zip((K, R, du, dq), ref):
            assert _rel(host(got), want) <= 1e-12
    mesh.set_fault_injection()
    K1, R1, status = _assemble(mesh, st)
    assert (status == iedg.ELEM_OK).all(), status
    assert np.array_equal(host(K1), host(K0)) and np.array_equal(host(R1), host(R0))


def test_fault_injection_rejects_bad_values():
    from paper_1605_01020_gb300 import iedg
    wl = _wl()
    mesh = _mesh(wl, 0)
    for kw in (dict(zero_row_elem=8), dict(zero_row_elem=0, zero_row=320), dict(refine_iters=17),
               dict(tc_wait_limit=-2)):
        with pytest.raises(iedg.IedgError):
            mesh.set_fault_injection(**kw)
