"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs.  Tolerance for the FP64 path: max |x - x_oracle| / max |x_oracle|
<= 1e-11 per output array (K per BSR block row); index structures bit-exact."""
import numpy as np
import pytest

from oracle import iedg as oiedg
from oracle import lowprec
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import problem
from gpu_helpers import bsr_row_err, dev, fro_ratio, host, lib_mesh, oracle_K_rows, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _case(name):
    if name == "cfg1":
        return W.config(1)
    if name == "cfg1-noisy":
        wl = W.config(1)
        st = W.make_state(wl.mesh, W.fourier_perturbed_field(2, 0.2, 1001), 1002, noise=0.01, uref_shift=0.01)
        return W.Workload(wl.name + " + nodal noise", wl.mesh, st, wl.params)
    if name == "p3-2cube":
        return W.config(2, N=2)
    if name == "p2-curved":
        wl = W.config(3, N=2)
        mesh = W.structured_mesh(3, 3, 2, mapping=W.stretched_mapping(77, ratio=10.0))
        st = W.make_state(mesh, W.taylor_green_field(0.3), 78, noise=0.01, uref_shift=0.01)
        prm = dict(wl.params, Re=200.0)
        return W.Workload("3D p=2 3^3 curved", mesh, st, prm)
    if name == "2d-p3-steady":
        mesh = W.structured_mesh(2, (3, 4), 3)
        st = W.make_state(mesh, W.fourier_perturbed_field(2, 0.3, 5, amp=0.05), 6, noise=0.01)
        prm = dict(gamma=1.4, Pr=0.72, Re=100.0, Minf=0.3, alpha=0.0)
        return W.Workload("2D p=3 3x4 steady", mesh, st, prm)
    if name == "p4-2cube":
        mesh = W.structured_mesh(3, 2, 4, mapping=W.stretched_mapping(91, ratio=4.0))
        st = W.make_state(mesh, W.broadband_field(0.3, 92), 93, noise=0.005)
        prm = dict(gamma=1.4, Pr=0.72, Re=2.5e5, Minf=0.3, alpha=W.dirk_alpha())
        return W.Workload("3D p=4 2^3 curved", mesh, st, prm)
    if name == "2d-p1":
        mesh = W.structured_mesh(2, 4, 1)
        st = W.make_state(mesh, W.fourier_perturbed_field(2, 0.3, 7, amp=0.05), 8, noise=0.01, uref_shift=0.01)
        prm = dict(gamma=1.4, Pr=0.72, Re=100.0, Minf=0.3, alpha=W.dirk_alpha())
        return W.Workload("2D p=1 4x4", mesh, st, prm)
    if name.endswith("-roe"):
        wl = _case(name[:-4])
        return W.Workload(wl.name + " (Roe)", wl.mesh, wl.state, dict(wl.params, stab=1))
    raise KeyError(name)


CASES = ["cfg1", "cfg1-noisy", "p3-2cube", "p2-curved", "2d-p3-steady", "2d-p1", "p4-2cube",
         "cfg1-noisy-roe", "p3-2cube-roe", "p2-curved-roe"]


@pytest.mark.parametrize("name", CASES)
def test_residual_parity(name):
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    Rq, Ru, Rh, Rfl = pb.residual(st.u, st.q, st.uhat, st.u_ref)
    mesh = lib_mesh(wl)
    out = mesh.eval_residual(dev(st.u), dev(st.uhat), q=dev(st.q), u_ref=dev(st.u_ref))
    assert rel_err(host(out["r_q"]), Rq) <= TOL
    assert rel_err(host(out["r_u"]), Ru) <= TOL
    assert rel_err(host(out["r_fl"]), Rfl, floor=np.abs(Rh).max()) <= TOL


@pytest.mark.parametrize("name", ["cfg1", "p2-curved"])
def test_lifted_gradient_parity(name):
    """q = NULL: q from R_q = 0 (Eq. IEDG a), then R_q vanishes."""
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    q_o = pb.solve_q(st.u, st.uhat)
    mesh = lib_mesh(wl)
    out = mesh.eval_residual(dev(st.u), dev(st.uhat), q=None)
    assert rel_err(host(out["q"]), q_o) <= TOL
    assert np.abs(host(out["r_q"])).max() <= 1e-12 * np.abs(q_o).max()
    Rq, Ru, Rh, Rfl = pb.residual(st.u, q_o, st.uhat)
    assert rel_err(host(out["r_u"]), Ru) <= TOL
    assert rel_err(host(out["r_fl"]), Rfl, floor=np.abs(Rh).max()) <= TOL


@pytest.mark.parametrize("name", CASES)
def test_trace_pattern_bit_exact(name):
    wl = _case(name)
    mesh = lib_mesh(wl)
    rp, col = mesh.trace_pattern()
    rp_o, col_o = oiedg.bsr_pattern(wl.mesh.elem_trace, wl.mesh.n_trace)
    assert np.array_equal(host(rp), rp_o)
    assert np.array_equal(host(col).astype(np.int64), col_o)


@pytest.mark.parametrize("name", CASES)
def test_condensed_parity(name):
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    mesh = lib_mesh(wl)
    K_d, R_d = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat), u_ref=dev(st.u_ref))
    assert bsr_row_err(row_ptr, host(K_d), vals, range(wl.mesh.n_trace)) <= TOL
    assert rel_err(host(R_d), R, floor=np.abs(np.array(Re)).max()) <= TOL
    assert (mesh.element_status() == 0).all()
    # back-substitution
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    du_o = np.zeros_like(st.u)
    dq_o = np.zeros_like(st.q)
    for e in range(E):
        du_o[e], dq_o[e] = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, st.u_ref)
    assert rel_err(host(du_d), du_o) <= TOL
    assert rel_err(host(dq_d), dq_o) <= TOL


@pytest.mark.parametrize("name", ["cfg1-noisy", "p3-2cube", "p2-curved", "2d-p3-steady", "p4-2cube", "p3-2cube-roe"])
def test_condensed_parity_tensor_schur(name):
    """FP64 form with the Schur complement on the tensor cores (exact splitting of the
    FP64 operands, lu_tensor = 1): same tolerance against the oracle as the DFMA form."""
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    mesh = lib_mesh(wl)
    mesh.set_schedule(lu_tensor=1)
    K_d, R_d = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat), u_ref=dev(st.u_ref))
    assert bsr_row_err(row_ptr, host(K_d), vals, range(wl.mesh.n_trace)) <= TOL
    assert rel_err(host(R_d), R, floor=np.abs(np.array(Re)).max()) <= TOL
    assert (mesh.element_status() == 0).all()
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    du_o = np.zeros_like(st.u)
    dq_o = np.zeros_like(st.q)
    for e in range(E):
        du_o[e], dq_o[e] = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, st.u_ref)
    assert rel_err(host(du_d), du_o) <= TOL
    assert rel_err(host(dq_d), dq_o) <= TOL


def test_back_substitute_before_assembly_is_an_error():
    from paper_1605_01020_gb300 import iedg
    wl = _case("cfg1")
    mesh = lib_mesh(wl)
    with pytest.raises(iedg.IedgError) as ei:
        mesh.back_substitute(dev(wl.state.duhat))
    assert ei.value.code == -5


def test_inverted_element_rejected():
    from paper_1605_01020_gb300 import iedg
    wl = _case("cfg1")
    X = wl.mesh.node_xyz.copy()
    X[3] = X[3][:, ::-1]          # swap x and y of one element: detJ < 0
    with pytest.raises(iedg.IedgError) as ei:
        iedg.Mesh(X, wl.mesh.elem_trace, wl.mesh.n_trace, wl.mesh.p, **{k: wl.params[k] for k in ("gamma", "Pr", "Re", "Minf", "alpha")})
    assert ei.value.code == -4


def _cond1(pb, st, els):
    """1-norm condition numbers of the q-eliminated interior blocks A~ of `els`."""
    return [float(np.linalg.cond(pb.qelim(pb.element_blocks(e, st.u, st.q, st.uhat))[0], 1)) for e in els]


@pytest.mark.parametrize("cfg", [2, 3])
def test_full_size_p3_sampled(cfg):
    """The 3D p=3 16^3 workloads at full size (config 3: stretched and sheared, aspect
    up to 50), in the launch configuration the benchmark times: sampled block rows of
    K and R, sampled element updates, all within 1e-11 in FP64; the 1-norm condition
    numbers of the sampled elements' A~ are printed beside the errors."""
    wl = W.config(cfg)
    st = wl.state
    mesh = lib_mesh(wl)
    u, q, uh = dev(st.u), dev(st.q), dev(st.uhat)
    res = mesh.eval_residual(u, uh, q=q)
    K_d, R_d = mesh.assemble_condensed(u, q, uh)
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    K_h, R_h = host(K_d), host(R_d)
    assert np.isfinite(K_h).all() and (mesh.element_status() == 0).all()
    pb = problem(wl.mesh, wl.params)
    rng = np.random.default_rng(0)
    rows = rng.choice(wl.mesh.n_trace, 3, replace=False)
    row_ptr, col, vals, R, els, re_max = oracle_K_rows(pb, wl.mesh, st, rows)
    kerr = bsr_row_err(row_ptr, K_h, vals, rows)
    rerr = rel_err(R_h[rows], R[rows], floor=re_max)
    # residual on the touched elements and trace rows
    Rq, Ru, Rh, Rfl = pb.residual(st.u, st.q, st.uhat, els=els)
    ruerr = rel_err(host(res["r_u"])[els], Ru)
    rqerr = rel_err(host(res["r_q"])[els], Rq)
    duerr = dqerr = 0.0
    for e in els[:2]:
        du_o, dq_o = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat)
        duerr = max(duerr, rel_err(host(du_d[e]), du_o))
        dqerr = max(dqerr, rel_err(host(dq_d[e]), dq_o))
    cond = _cond1(pb, st, els[:2])
    print(f"config {cfg} FP64: K {kerr:.2e}  R {rerr:.2e}  R_u {ruerr:.2e}  R_q {rqerr:.2e}  "
          f"du {duerr:.2e}  dq {dqerr:.2e}  cond1(A~) {max(cond):.2e}")
    assert max(kerr, rerr, ruerr, rqerr, duerr, dqerr) <= TOL


# ---------------------------------------------------------------- mixed precision
# FP32 element matrix and partial LU, FP64 refinement.  Bounds: K is an FP32
# Schur complement, error <= kappa(A~) * 6e-8, checked at 1e-4 relative per block
# row; R and the updates du, dq are refined to FP64 and checked at 1e-10.
TOL_MIXED_K = 1e-4
TOL_MIXED = 1e-10


# Schur complement with TF32 / BF16 operands (one product, FP32 accumulation): K is
# checked against the oracle's condensation with the same operands rounded
# (oracle/lowprec.py) by the ratio ||K - K_rounded|| / ||K_rounded - K_exact||.  A
# device that skipped the rounding scores 1, one that rounded another way (e.g. TF32
# by truncation) about 1.7; the device rounds FP32 operands that carry the FP32 LU's
# error (a few 1e-6 relative), so some entries round to the other neighbour, which a
# CPU model of FP32 operands puts at 0.01 - 0.17.  The error against the exact K is
# printed.  R, du, dq are refined to FP64 as before.
LOW_FMT = {2: "tf32", 3: "bf16"}
LOW_RATIO = 0.35


def _mixed_mesh(wl, precision=1):
    from paper_1605_01020_gb300 import iedg
    return iedg.mesh_from_workload(wl, precision=precision)


@pytest.mark.parametrize("lu_tensor", [0, 1, 2])
@pytest.mark.parametrize("name", ["cfg1-noisy", "p3-2cube", "p2-curved", "2d-p3-steady", "2d-p1", "p4-2cube",
                                  "p3-2cube-roe", "p2-curved-roe"])
def test_mixed_condensed_parity(name, lu_tensor):
    """FP32 element matrix and partial LU in its three forms (FFMA updates; the Schur
    complement deferred to one tensor-core GEMM; every trailing update on the tensor
    cores), FP64 refinement: against the FP64 oracle."""
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    mesh = _mixed_mesh(wl)
    mesh.set_schedule(lu_tensor=lu_tensor)
    K_d, R_d = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat), u_ref=dev(st.u_ref))
    kerr = bsr_row_err(row_ptr, host(K_d), vals, range(wl.mesh.n_trace))
    rerr = rel_err(host(R_d), R, floor=np.abs(np.array(Re)).max())
    assert (mesh.element_status() == 0).all()
    assert kerr <= TOL_MIXED_K, kerr
    assert rerr <= TOL_MIXED, rerr
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    du_o = np.zeros_like(st.u)
    dq_o = np.zeros_like(st.q)
    for e in range(E):
        du_o[e], dq_o[e] = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, st.u_ref)
    assert rel_err(host(du_d), du_o) <= TOL_MIXED
    assert rel_err(host(dq_d), dq_o) <= TOL_MIXED


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("name", ["cfg1-noisy", "p3-2cube", "p2-curved", "p4-2cube"])
def test_mass_scaled_parity(name, precision):
    """Mixed forms on the system scaled by the element mass matrix (S = I (x) L^-1,
    M = L L^T, applied to the u-block): the FP32 form's K against the plain K at the
    FP32 bound, the TF32 / BF16 forms against the oracle's rounded-operand condensation
    of the scaled system; R, du, dq refined to FP64 with the scaled factors."""
    from paper_1605_01020_gb300 import iedg
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    mesh = iedg.mesh_from_workload(wl, precision=precision, flags=iedg.FLAG_MASS_SCALING)
    K_d, R_d = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat), u_ref=dev(st.u_ref))
    K_h = host(K_d)
    rows = range(wl.mesh.n_trace)
    kerr = bsr_row_err(row_ptr, K_h, vals, rows)
    rerr = rel_err(host(R_d), R, floor=np.abs(np.array(Re)).max())
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    du_o = np.zeros_like(st.u)
    dq_o = np.zeros_like(st.q)
    for e in range(E):
        du_o[e], dq_o[e] = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, st.u_ref)
    msg = f"{name} precision {precision} mass-scaled: K {kerr:.2e}  R {rerr:.2e}"
    assert (mesh.element_status() == 0).all()
    if precision == 1:
        assert kerr <= TOL_MIXED_K, msg
    else:
        Kl = [lowprec.condense_rounded(pb, pb.element_blocks(e, st.u, st.q, st.uhat, st.u_ref), LOW_FMT[precision],
                                       mass_scaled=True)[0] for e in range(E)]
        _, _, vals_low, _ = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Kl), np.array(Re))
        ratio = fro_ratio(row_ptr, K_h, vals_low, vals, rows)
        msg += f" (vs scaled rounded-operand oracle: {ratio:.3f} of the rounding's effect)"
        assert ratio <= LOW_RATIO, msg
    print(msg)
    assert rerr <= TOL_MIXED, msg
    assert rel_err(host(du_d), du_o) <= TOL_MIXED
    assert rel_err(host(dq_d), dq_o) <= TOL_MIXED


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("name", ["cfg1-noisy", "p3-2cube", "p2-curved", "p4-2cube", "p3-2cube-roe"])
def test_low_precision_schur_parity(name, precision):
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    Kl = [lowprec.condense_rounded(pb, pb.element_blocks(e, st.u, st.q, st.uhat, st.u_ref), LOW_FMT[precision])[0]
          for e in range(E)]
    _, _, vals_low, _ = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Kl), np.array(Re))
    mesh = _mixed_mesh(wl, precision)
    K_d, R_d = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat), u_ref=dev(st.u_ref))
    K_h = host(K_d)
    rows = range(wl.mesh.n_trace)
    kerr = bsr_row_err(row_ptr, K_h, vals, rows)
    ratio = fro_ratio(row_ptr, K_h, vals_low, vals, rows)
    rerr = rel_err(host(R_d), R, floor=np.abs(np.array(Re)).max())
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    du_o = np.zeros_like(st.u)
    dq_o = np.zeros_like(st.q)
    for e in range(E):
        du_o[e], dq_o[e] = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, st.u_ref)
    print(f"{name} precision {precision}: K {kerr:.2e} (vs rounded-operand oracle: {ratio:.3f} of the "
          f"rounding's effect)  R {rerr:.2e}")
    assert (mesh.element_status() == 0).all()
    assert ratio <= LOW_RATIO, ratio
    assert rerr <= TOL_MIXED, rerr
    assert rel_err(host(du_d), du_o) <= TOL_MIXED
    assert rel_err(host(dq_d), dq_o) <= TOL_MIXED


@pytest.mark.parametrize("quad_extra", [1, 3])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["p2-curved", "p3-2cube", "2d-p3-steady"])
def test_quad_extra_parity(name, precision, quad_extra):
    """Fewer (p + 1) and more (p + 3) Gauss points per direction than the default: the
    work buffers of the point, assembly and refinement kernels change shape."""
    from paper_1605_01020_gb300 import iedg
    wl = _case(name)
    st = wl.state
    pb = problem(wl.mesh, wl.params, quad_extra=quad_extra)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    mesh = iedg.mesh_from_workload(wl, precision=precision, quad_extra=quad_extra)
    K_d, R_d = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat), u_ref=dev(st.u_ref))
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    du_o = np.zeros_like(st.u)
    dq_o = np.zeros_like(st.q)
    for e in range(E):
        du_o[e], dq_o[e] = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, st.u_ref)
    tk, tr = (TOL, TOL) if precision == 0 else (TOL_MIXED_K, TOL_MIXED)
    assert (mesh.element_status() == 0).all()
    assert bsr_row_err(row_ptr, host(K_d), vals, range(wl.mesh.n_trace)) <= tk
    assert rel_err(host(R_d), R, floor=np.abs(np.array(Re)).max()) <= tr
    assert rel_err(host(du_d), du_o) <= tr
    assert rel_err(host(dq_d), dq_o) <= tr


@pytest.mark.parametrize("cfg,precision,lu_tensor,scaled", [(2, 1, 1, 0), (2, 1, 2, 0), (3, 1, 0, 0), (3, 1, 2, 0),
                                                           (3, 2, 1, 0), (3, 3, 1, 0), (3, 1, 0, 1), (3, 2, 1, 1),
                                                           (3, 3, 1, 1)])
def test_mixed_full_size_sampled(cfg, precision, lu_tensor, scaled):
    """The 16^3 p=3 workloads (config 3: stretched and sheared, aspect up to 50) in the
    mixed forms at full size (FP32 Schur complement; on config 3 also TF32 and BF16
    operands): sampled block rows of K and R, sampled updates."""
    wl = W.config(cfg)
    st = wl.state
    from paper_1605_01020_gb300 import iedg
    mesh = iedg.mesh_from_workload(wl, precision=precision, flags=iedg.FLAG_MASS_SCALING if scaled else 0)
    mesh.set_schedule(lu_tensor=lu_tensor)
    u, q, uh = dev(st.u), dev(st.q), dev(st.uhat)
    K_d, R_d = mesh.assemble_condensed(u, q, uh)
    du_d, dq_d = mesh.back_substitute(dev(st.duhat))
    status = mesh.element_status()
    K_h, R_h = host(K_d), host(R_d)
    pb = problem(wl.mesh, wl.params)
    rng = np.random.default_rng(cfg)
    rows = rng.choice(wl.mesh.n_trace, 2, replace=False)
    row_ptr, col, vals, R, els, re_max = oracle_K_rows(pb, wl.mesh, st, rows)
    kerr = bsr_row_err(row_ptr, K_h, vals, rows)
    rerr = rel_err(R_h[rows], R[rows], floor=re_max)
    ratio = None
    if precision in LOW_FMT:
        kfun = lambda e: lowprec.condense_rounded(pb, pb.element_blocks(e, st.u, st.q, st.uhat),
                                                  LOW_FMT[precision], mass_scaled=bool(scaled))[0]
        vals_low = oracle_K_rows(pb, wl.mesh, st, rows, kfun=kfun)[2]
        ratio = fro_ratio(row_ptr, K_h, vals_low, vals, rows)
    e = els[0]
    du_o, dq_o = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat)
    duerr, dqerr = rel_err(host(du_d[e]), du_o), rel_err(host(dq_d[e]), dq_o)
    cond = _cond1(pb, st, [e])
    print(f"config {cfg} precision {precision} lu_tensor {lu_tensor} mass-scaled {scaled}: K {kerr:.2e}  R {rerr:.2e}  du {duerr:.2e}  dq {dqerr:.2e}  "
          f"cond1(A~) {max(cond):.2e}  flagged {int((status != 0).sum())}"
          + ("" if ratio is None else f"  K vs rounded-operand oracle {ratio:.3f} of the rounding's effect"))
    assert (status == 0).all()
    if ratio is None:
        assert kerr <= TOL_MIXED_K
    else:
        assert ratio <= LOW_RATIO
    assert rerr <= TOL_MIXED and duerr <= TOL_MIXED and dqerr <= TOL_MIXED


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_captured_step_matches_eager(precision):
    """The whole element-local step (residual with lifting, condensation,
    back-substitution) captured once in a CUDA graph and replayed gives the same
    outputs as eager calls (the library launches only on the caller's stream and
    allocates nothing per call)."""
    import torch
    from paper_1605_01020_gb300 import iedg
    wl = _case("p3-2cube")
    st = wl.state
    mesh = iedg.mesh_from_workload(wl, precision=precision)
    E, Np, m, d, T = mesh.E, mesh.Np, mesh.m, mesh.d, mesh.T
    u, uh, duh = dev(st.u), dev(st.uhat), dev(st.duhat)
    f64 = torch.float64
    bufs = dict(q=torch.empty(E, Np, m, d, dtype=f64, device="cuda"),
                rq=torch.empty(E, Np, m, d, dtype=f64, device="cuda"),
                ru=torch.empty(E, Np, m, dtype=f64, device="cuda"), rfl=torch.empty(T, m, dtype=f64, device="cuda"),
                K=torch.empty(mesh.nnzb, m, m, dtype=f64, device="cuda"), R=torch.empty(T, m, dtype=f64, device="cuda"),
                du=torch.empty(E, Np, m, dtype=f64, device="cuda"), dq=torch.empty(E, Np, m, d, dtype=f64, device="cuda"))

    def step():
        mesh.eval_residual(u, uh, q=None, q_out=bufs["q"], r_q=bufs["rq"], r_u=bufs["ru"], r_fl=bufs["rfl"])
        mesh.assemble_condensed(u, bufs["q"], uh, K=bufs["K"], R=bufs["R"])
        mesh.back_substitute(duh, bufs["du"], bufs["dq"])

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()                                    # warm-up (kernel attributes set outside capture)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in bufs.items()}
    for v in bufs.values():
        v.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for v in bufs.values():
        v.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for k in bufs:
        assert torch.equal(bufs[k], eager[k]), k
