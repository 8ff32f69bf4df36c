"""GPU parity on meshes with domain boundaries (iedg_create_mesh_bc; far-field and
no-slip adiabatic wall faces with discontinuous traces, Sec. 2.1) against the
oracle's MixedProblem with face kinds.  Tolerances as in the other parity tests."""
import numpy as np
import pytest

from oracle import iedg as oiedg
from oracle import physics
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import ref_element
from gpu_helpers import bsr_row_err, dev, host, rel_err

pytestmark = pytest.mark.gpu
TOL, TOL_MIXED_K, TOL_MIXED = 1e-11, 1e-4, 1e-10


def _uniform(d, v, M=0.3, gamma=1.4):
    rho, p = 1.0, 1.0 / (gamma * M ** 2)
    v = np.asarray(v, dtype=np.float64)
    return np.concatenate([[rho], rho * v, [p / (gamma - 1) + 0.5 * rho * v @ v]])


def _case(name):
    if name.startswith("2d"):
        d, N, levels, boundary, seed = 2, 4, (1, 2, 3), (1, 2), 21
        field = W.fourier_perturbed_field(2, 0.3, 22, amp=0.05)
    else:
        d, N, levels, boundary, seed = 3, 2, (2, 3), (1, 2, 0), 23
        field = W.taylor_green_field(0.3)
    probs = np.full(len(levels), 1.0 / len(levels))
    orders = W.mixed_orders([N] * d, seed, levels=levels, probs=probs)
    mesh = W.structured_mesh_mixed(d, N, orders, boundary=boundary)
    st = W.make_state_mixed(mesh, field, seed + 1, noise=0.01)
    ub = _uniform(d, [0.5, 0.05, 0.0][:d])
    stab = 1 if name.endswith("roe") else 0
    prm = physics.Params(gamma=1.4, Pr=0.72, Re=200.0, Minf=0.3, alpha=W.dirk_alpha(), stab=stab)
    return mesh, st, ub, prm


def _lib(mesh, prm, ub, precision=0):
    from paper_1605_01020_gb300 import iedg
    return iedg.MixedOrderMesh(mesh.node_xyz, mesh.elem_trace, mesh.n_trace, mesh.orders, mesh.face_degree,
                               gamma=prm.gamma, Pr=prm.Pr, Re=prm.Re, Minf=prm.Minf, alpha=prm.alpha,
                               precision=precision, stab=prm.stab, face_kind=mesh.face_kind, u_far=ub)


def _problem(mesh, prm, ub):
    refs = {int(p): ref_element(mesh.d, int(p)) for p in set(mesh.orders.tolist())}
    return oiedg.MixedProblem(refs, mesh, prm, ub=ub)


def _cat(xs):
    return np.concatenate([np.asarray(x) for x in xs])


CASES = ["2d", "3d", "2d-roe", "3d-roe"]


@pytest.mark.parametrize("name", CASES)
def test_boundary_residual_parity(name):
    mesh, st, ub, prm = _case(name)
    pb = _problem(mesh, prm, ub)
    Rq, Ru, Rh, Rfl = pb.residual(st.u, st.q, st.uhat)
    lm = _lib(mesh, prm, ub)
    out = lm.eval_residual(dev(_cat(st.u)), dev(st.uhat), q=dev(_cat(st.q)))
    assert rel_err(host(out["r_q"]), _cat(Rq)) <= TOL
    assert rel_err(host(out["r_u"]), _cat(Ru)) <= TOL
    assert rel_err(host(out["r_fl"]), Rfl, floor=max(np.abs(r).max() for r in Rh)) <= TOL


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_boundary_condensed_parity(name, precision):
    mesh, st, ub, prm = _case(name)
    pb = _problem(mesh, prm, ub)
    E = mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble_ragged(mesh.elem_trace, mesh.n_trace, Ke, Re)
    du_o, dq_o = zip(*[pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat) for e in range(E)])
    lm = _lib(mesh, prm, ub, precision)
    K_d, R_d = lm.assemble_condensed(dev(_cat(st.u)), dev(_cat(st.q)), dev(st.uhat))
    du_d, dq_d = lm.back_substitute(dev(st.duhat))
    tk, tr = (TOL, TOL) if precision == 0 else (TOL_MIXED_K, TOL_MIXED)
    assert bsr_row_err(row_ptr, host(K_d), vals, range(mesh.n_trace)) <= tk
    assert rel_err(host(R_d), R, floor=max(np.abs(r).max() for r in Re)) <= tr
    assert (lm.element_status() == 0).all()
    assert rel_err(host(du_d), _cat(du_o)) <= tr
    assert rel_err(host(dq_d), _cat(dq_o)) <= tr


def test_boundary_kind_validation():
    from paper_1605_01020_gb300 import iedg
    mesh, st, ub, prm = _case("2d")
    fk = mesh.face_kind.copy()
    with pytest.raises(iedg.IedgError):          # far-field faces without u_far
        iedg.MixedOrderMesh(mesh.node_xyz, mesh.elem_trace, mesh.n_trace, mesh.orders, mesh.face_degree,
                            face_kind=fk)
    fk[0, 0] = 7
    with pytest.raises(iedg.IedgError):
        iedg.MixedOrderMesh(mesh.node_xyz, mesh.elem_trace, mesh.n_trace, mesh.orders, mesh.face_degree,
                            face_kind=fk, u_far=ub)
