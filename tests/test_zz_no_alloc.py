"""The allocation-free residual entry point (iedg_eval_residual_static) against the
regular one (iedg_eval_residual), called through the C ABI.

Callers that cannot allocate device memory at the point of the call (framework-owned
memory pools, real-time loops, plug-ins without allocation rights) use the static
variant; it must give the same residual, also when called twice in a row (its scratch
array is shared and keeps the previous call's contents), and must refuse meshes whose
scratch would not fit."""
import ctypes

import numpy as np
import pytest

from paper_1605_01020_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11          # the FP64 parity tolerance of the other GPU tests


def _lib_and_mesh(wl):
    from __graft_entry__ import build
    build()
    from paper_1605_01020_gb300 import iedg
    return iedg.load(), iedg.mesh_from_workload(wl)


def _cases():
    wl1 = W.config(1)
    st1 = W.make_state(wl1.mesh, W.fourier_perturbed_field(2, 0.2, 11), 12, noise=0.01, uref_shift=0.01)
    wl2 = W.config(2, N=3)
    return [W.Workload("2D p=2 8x8 noisy", wl1.mesh, st1, wl1.params), wl2]


@pytest.mark.parametrize("idx", [0, 1])
def test_static_residual_matches_regular_twice(idx):
    import torch
    wl = _cases()[idx]
    lib, mesh = _lib_and_mesh(wl)
    st = wl.state
    dev = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float64, device="cuda")
    u, uh, q, ur = dev(st.u), dev(st.uhat), dev(st.q), dev(st.u_ref)
    ref = mesh.eval_residual(u, uh, q=q, u_ref=ur)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        r_u = torch.full_like(ref["r_u"], float("nan"))
        r_fl = torch.full_like(ref["r_fl"], float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.iedg_eval_residual_static(mesh._h, u.data_ptr(), uh.data_ptr(), q.data_ptr(),
                                           None if ur is None else ur.data_ptr(), r_u.data_ptr(),
                                           r_fl.data_ptr(), ctypes.c_void_p(stream))
        assert rc == 0, lib.iedg_last_error(mesh._h).decode()
        torch.cuda.synchronize()
        if call == 1:
            # the first call only looks up the scratch array's device address; from then
            # on a call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before, "the static entry point allocated device memory"
        for got, want in ((r_u, ref["r_u"]), (r_fl, ref["r_fl"])):
            g, w = got.cpu().numpy(), want.cpu().numpy()
            scale = max(np.abs(w).max(), np.abs(ref["r_u"].cpu().numpy()).max())
            assert np.isfinite(g).all()
            assert np.abs(g - w).max() <= TOL * scale, f"call {call}"


def test_static_residual_rejects_meshes_beyond_the_limit():
    import torch
    from paper_1605_01020_gb300 import iedg
    lib = iedg.load()
    # 2D p=3: Nb * m = 12 * 4 = 48 scratch doubles per element; 210^2 elements exceed 2^21
    mesh_w = W.structured_mesh(2, 210, 3)
    assert mesh_w.n_elem * 48 > (1 << 21)
    st = W.make_state(mesh_w, W.freestream_field(2, 0.2), 1)
    wl = W.Workload("big 2D", mesh_w, st, dict(gamma=1.4, Pr=0.72, Re=100.0, Minf=0.2, alpha=0.0))
    _, mesh = _lib_and_mesh(wl)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    u, uh, q = dev(st.u), dev(st.uhat), dev(st.q)
    r_fl = torch.zeros(mesh.T, mesh.m, dtype=torch.float64, device="cuda")
    rc = lib.iedg_eval_residual_static(mesh._h, u.data_ptr(), uh.data_ptr(), q.data_ptr(), None, None,
                                       r_fl.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert "static limit" in lib.iedg_last_error(mesh._h).decode()
