"""GPU parity on meshes with mixed polynomial orders (iedg_create_mesh_mixed) against
the oracle's MixedProblem: faces between elements of the same order carry the
continuous trace, faces between different orders private nodes of degree
max(p_L, p_R).  Same tolerances as the uniform parity tests: FP64 path 1e-11 per
output array (K per BSR block row), mixed path K 1e-4 and R, du, dq 1e-10; index
structures bit-exact."""
import numpy as np
import pytest

from oracle import iedg as oiedg
from oracle import lowprec, physics
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import ref_element
from gpu_helpers import bsr_row_err, dev, fro_ratio, host, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-11
TOL_MIXED_K = 1e-4
TOL_MIXED = 1e-10


def _case(name):
    if name == "2d-123":
        d, N, levels, probs, seed = 2, 4, (1, 2, 3), (0.3, 0.4, 0.3), 11
        field, alpha = W.fourier_perturbed_field(2, 0.3, 5, amp=0.05), W.dirk_alpha()
    elif name == "3d-234":
        d, N, levels, probs, seed = 3, 2, (2, 3, 4), (0.3, 0.5, 0.2), 12
        field, alpha = W.taylor_green_field(0.3), W.dirk_alpha()
    elif name == "3d-23-steady":
        d, N, levels, probs, seed = 3, 2, (2, 3), (0.5, 0.5), 13
        field, alpha = W.broadband_field(0.3, 14), 0.0
    elif name == "3d-234-roe":
        mesh, st, u_ref, prm = _case("3d-234")
        prm.stab = 1
        return mesh, st, u_ref, prm
    elif name == "3d-234-4cube":
        d, N, levels, probs, seed = 3, 4, (2, 3, 4), (0.3, 0.5, 0.2), 15
        field, alpha = W.taylor_green_field(0.2), W.dirk_alpha()
    else:
        raise KeyError(name)
    orders = W.mixed_orders([N] * d, seed, levels=levels, probs=probs)
    mesh = W.structured_mesh_mixed(d, N, orders)
    st = W.make_state_mixed(mesh, field, seed + 100, noise=0.01)
    rng = np.random.default_rng(seed + 200)
    u_ref = [u + 0.01 * np.abs(u).max() * rng.uniform(-1, 1, u.shape) for u in st.u] if alpha else None
    prm = physics.Params(gamma=1.4, Pr=0.72, Re=200.0 if d == 3 else 100.0, Minf=0.3, alpha=alpha)
    return mesh, st, u_ref, prm


def _problem(mesh, prm):
    refs = {int(p): ref_element(mesh.d, int(p)) for p in set(mesh.orders.tolist())}
    return oiedg.MixedProblem(refs, mesh, prm)


def _lib(mesh, prm, precision=0):
    from paper_1605_01020_gb300 import iedg
    return iedg.MixedOrderMesh(mesh.node_xyz, mesh.elem_trace, mesh.n_trace, mesh.orders, mesh.face_degree,
                               gamma=prm.gamma, Pr=prm.Pr, Re=prm.Re, Minf=prm.Minf, alpha=prm.alpha,
                               precision=precision, stab=prm.stab)


def _cat(xs):
    return np.concatenate([np.asarray(x) for x in xs])


CASES = ["2d-123", "3d-234", "3d-23-steady", "3d-234-roe"]


@pytest.mark.parametrize("name", CASES)
def test_element_sizes_and_pattern(name):
    mesh, st, u_ref, prm = _case(name)
    lm = _lib(mesh, prm)
    npe, nbe = lm.element_sizes()
    assert np.array_equal(npe, [len(x) for x in mesh.node_xyz])
    assert np.array_equal(nbe, [len(t) for t in mesh.elem_trace])
    rp, col = lm.trace_pattern()
    Ke0 = [np.zeros((len(t), 1, len(t), 1)) for t in mesh.elem_trace]
    Re0 = [np.zeros((len(t), 1)) for t in mesh.elem_trace]
    rp_o, col_o, _, _ = oiedg.assemble_ragged(mesh.elem_trace, mesh.n_trace, Ke0, Re0)
    assert np.array_equal(host(rp), rp_o)
    assert np.array_equal(host(col).astype(np.int64), col_o)


@pytest.mark.parametrize("name", CASES)
def test_mixed_orders_residual_parity(name):
    mesh, st, u_ref, prm = _case(name)
    pb = _problem(mesh, prm)
    Rq, Ru, Rh, Rfl = pb.residual(st.u, st.q, st.uhat, u_ref)
    lm = _lib(mesh, prm)
    out = lm.eval_residual(dev(_cat(st.u)), dev(st.uhat), q=dev(_cat(st.q)),
                           u_ref=None if u_ref is None else dev(_cat(u_ref)))
    assert rel_err(host(out["r_q"]), _cat(Rq)) <= TOL
    assert rel_err(host(out["r_u"]), _cat(Ru)) <= TOL
    assert rel_err(host(out["r_fl"]), Rfl, floor=max(np.abs(r).max() for r in Rh)) <= TOL


@pytest.mark.parametrize("name", ["2d-123", "3d-234"])
def test_mixed_orders_lifted_gradient(name):
    mesh, st, u_ref, prm = _case(name)
    pb = _problem(mesh, prm)
    q_o = pb.solve_q(st.u, st.uhat)
    lm = _lib(mesh, prm)
    out = lm.eval_residual(dev(_cat(st.u)), dev(st.uhat), q=None)
    assert rel_err(host(out["q"]), _cat(q_o)) <= TOL
    Rq, Ru, Rh, Rfl = pb.residual(st.u, q_o, st.uhat)
    assert rel_err(host(out["r_u"]), _cat(Ru)) <= TOL
    assert rel_err(host(out["r_fl"]), Rfl, floor=max(np.abs(r).max() for r in Rh)) <= TOL


def _oracle_condensed(mesh, st, u_ref, pb):
    E = mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat, u_ref) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble_ragged(mesh.elem_trace, mesh.n_trace, Ke, Re)
    du, dq = zip(*[pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, u_ref) for e in range(E)])
    return row_ptr, vals, R, max(np.abs(r).max() for r in Re), _cat(du), _cat(dq)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", [0, 1, 3])
def test_mixed_orders_condensed_parity(name, precision):
    mesh, st, u_ref, prm = _case(name)
    pb = _problem(mesh, prm)
    row_ptr, vals, R, re_max, du_o, dq_o = _oracle_condensed(mesh, st, u_ref, pb)
    lm = _lib(mesh, prm, precision)
    K_d, R_d = lm.assemble_condensed(dev(_cat(st.u)), dev(_cat(st.q)), dev(st.uhat),
                                     u_ref=None if u_ref is None else dev(_cat(u_ref)))
    du_d, dq_d = lm.back_substitute(dev(st.duhat))
    tk, tr = (TOL, TOL) if precision == 0 else (TOL_MIXED_K, TOL_MIXED)
    if precision == 3:
        # BF16 Schur operands: against the oracle's condensation with rounded operands
        # (ratio bound as in test_gpu_parity)
        Kl = [lowprec.condense_rounded(pb.pbs[e], pb.element_blocks(e, st.u, st.q, st.uhat, u_ref), "bf16")[0]
              for e in range(mesh.n_elem)]
        Re0 = [np.zeros((len(t), pb.m)) for t in mesh.elem_trace]
        vals_low = oiedg.assemble_ragged(mesh.elem_trace, mesh.n_trace, Kl, Re0)[2]
        assert fro_ratio(row_ptr, host(K_d), vals_low, vals, range(mesh.n_trace)) <= 0.5
    else:
        assert bsr_row_err(row_ptr, host(K_d), vals, range(mesh.n_trace)) <= tk
    assert rel_err(host(R_d), R, floor=re_max) <= tr
    assert (lm.element_status() == 0).all()
    assert rel_err(host(du_d), du_o) <= tr
    assert rel_err(host(dq_d), dq_o) <= tr


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_orders_schedules_agree(precision):
    mesh, st, u_ref, prm = _case("3d-234")
    lm = _lib(mesh, prm, precision)
    args = (dev(_cat(st.u)), dev(_cat(st.q)), dev(st.uhat))
    kw = dict(u_ref=None if u_ref is None else dev(_cat(u_ref)))
    ref = None
    for sched in ({"lu_persistent": 1}, {"lu_persistent": 0}, {"lu_persistent": 1, "asm_chunk": 16},
                  {"lu_persistent": 1, "lu_tensor": 1}, {"lu_persistent": 1, "lu_tensor": 0},
                  *([{"lu_persistent": 1, "lu_tensor": 2}, {"lu_persistent": 0, "lu_tensor": 2}]
                    if precision == 1 else []),
                  {"lu_persistent": 1, "asm_chunk_by_order": [0, 32, 8, 16]}):
        lm.set_schedule(**sched)
        K, R = lm.assemble_condensed(*args, **kw)
        du, dq = lm.back_substitute(dev(st.duhat))
        out = [host(t) for t in (K, R, du, dq)]
        if ref is None:
            ref = out
            continue
        tk = 1e-11 if precision == 0 else 1e-4
        assert rel_err(out[0], ref[0]) <= tk, sched
        for a, b in zip(out[1:], ref[1:]):
            assert rel_err(a, b) <= (1e-11 if precision == 0 else 1e-10), sched


def test_mixed_orders_4cube_sampled():
    """64 elements of orders 2, 3, 4: every element's condensed blocks and updates
    against the oracle for a sample of elements (all orders represented)."""
    mesh, st, u_ref, prm = _case("3d-234-4cube")
    pb = _problem(mesh, prm)
    lm = _lib(mesh, prm)
    K_d, R_d = lm.assemble_condensed(dev(_cat(st.u)), dev(_cat(st.q)), dev(st.uhat),
                                     u_ref=None if u_ref is None else dev(_cat(u_ref)))
    du_d, dq_d = lm.back_substitute(dev(st.duhat))
    K_d, du_d, dq_d = host(K_d), host(du_d), host(dq_d)
    rp = host(lm.trace_pattern()[0])
    col = host(lm.trace_pattern()[1]).astype(np.int64)
    assert (lm.element_status() == 0).all()
    off = np.concatenate([[0], np.cumsum([len(x) for x in mesh.node_xyz])])
    sample = [int(np.flatnonzero(mesh.orders == p)[0]) for p in (2, 3, 4)]
    for e in sample:
        du_o, dq_o = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat, u_ref)
        assert rel_err(du_d[off[e]:off[e + 1]], du_o) <= TOL
        assert rel_err(dq_d[off[e]:off[e + 1]], dq_o) <= TOL
    # one trace row fully: the sum over its elements
    r0 = int(mesh.elem_trace[sample[2]][0])
    els = [e for e in range(mesh.n_elem) if r0 in set(mesh.elem_trace[e].tolist())]
    vals = np.zeros((rp[r0 + 1] - rp[r0], pb.m, pb.m))
    for e in els:
        Ke, _ = pb.condense_qelim(e, st.u, st.q, st.uhat, u_ref)
        tr = mesh.elem_trace[e].tolist()
        s = tr.index(r0)
        for t in range(len(tr)):
            k = int(np.searchsorted(col[rp[r0]:rp[r0 + 1]], tr[t]))
            vals[k] += Ke[s, :, t, :]
    got = K_d[rp[r0]:rp[r0 + 1]]
    assert np.abs(got - vals).max() / np.abs(vals).max() <= TOL
