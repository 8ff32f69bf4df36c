"""Pins of the oracle's mixed-order reading (elements of different orders; faces
between different orders carry private trace nodes of degree max(p_L, p_R)):
partition of unity of the trace basis on every face, free-stream preservation,
discrete conservation, Jacobian blocks against finite differences, and the
condensed solve against the uncondensed global solve."""
import numpy as np
import pytest

from oracle import iedg, physics
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import ref_element


def _mixed(d, N, levels, probs, seed):
    orders = W.mixed_orders([N] * d, seed, levels=levels, probs=probs)
    mesh = W.structured_mesh_mixed(d, N, orders)
    return mesh


def _problem(mesh, alpha=0.0, Re=100.0, Minf=0.3):
    refs = {int(p): ref_element(mesh.d, int(p)) for p in set(mesh.orders.tolist())}
    prm = physics.Params(gamma=1.4, Pr=0.72, Re=Re, Minf=Minf, alpha=alpha)
    return iedg.MixedProblem(refs, mesh, prm)


@pytest.mark.parametrize("d,N,levels", [(2, 4, (1, 2, 3)), (3, 2, (2, 3, 4))])
def test_trace_basis_partition_of_unity_and_slots(d, N, levels):
    mesh = _mixed(d, N, levels, (0.3, 0.4, 0.3), 11)
    assert (mesh.face_degree > 0).any() and (mesh.face_degree == 0).any()
    pb = _problem(mesh)
    for e, p in enumerate(pb.pbs):
        assert p.fmu.shape[2] == len(mesh.elem_trace[e])
        np.testing.assert_allclose(p.fmu.sum(-1), 1.0, atol=1e-13)
    # every private face node is shared by exactly the two elements of its face,
    # every trace node is used by at least one element
    cnt = np.zeros(mesh.n_trace, dtype=int)
    for tr in mesh.elem_trace:
        np.add.at(cnt, tr, 1)
    assert cnt.min() >= 1


@pytest.mark.parametrize("d,N,levels", [(2, 4, (1, 2, 3)), (3, 2, (2, 3, 4))])
def test_mixed_free_stream_preservation(d, N, levels):
    mesh = _mixed(d, N, levels, (0.3, 0.4, 0.3), 12)
    pb = _problem(mesh, alpha=W.dirk_alpha())
    f = W.freestream_field(d, 0.3)
    u = [f(X) for X in mesh.node_xyz]
    q = [np.zeros(x.shape + (d,)) for x in u]
    uh = f(np.zeros((mesh.n_trace, d)))
    Rq, Ru, Rh, Rfl = pb.residual(u, q, uh)
    scale = np.abs(uh).max()
    assert max(np.abs(r).max() for r in Rq) < 1e-12 * scale
    assert max(np.abs(r).max() for r in Ru) < 1e-12 * scale
    assert np.abs(Rfl).max() < 1e-12 * scale


def test_mixed_discrete_conservation():
    mesh = _mixed(2, 4, (1, 2, 3), (0.3, 0.4, 0.3), 13)
    st = W.make_state_mixed(mesh, W.fourier_perturbed_field(2, 0.3, 3, amp=0.05), 4, noise=0.01)
    pb = _problem(mesh, alpha=0.0)
    Rq, Ru, Rh, Rfl = pb.residual(st.u, st.q, st.uhat)
    lhs = sum(r.sum(0) for r in Ru) - Rfl.sum(0)
    np.testing.assert_allclose(lhs, 0.0, atol=1e-12 * max(np.abs(r).max() for r in Ru))
    assert max(np.abs(r).max() for r in Ru) > 1e-4


@pytest.mark.parametrize("d", [2, 3])
def test_mixed_jacobian_blocks_match_finite_differences(d):
    if d == 2:
        mesh = _mixed(2, 4, (1, 2, 3), (0.3, 0.4, 0.3), 14)
        field = W.fourier_perturbed_field(2, 0.3, 5, amp=0.05)
    else:
        # 3D faces: two tangential directions, private nodes of degree 2 on the faces
        # between orders 1 and 2 (tensor products of the 1D Gauss-Lobatto Lagrange basis)
        mesh = _mixed(3, 2, (1, 2), (0.5, 0.5), 16)
        field = W.taylor_green_field(0.3)
    st = W.make_state_mixed(mesh, field, 6, noise=0.01)
    pb = _problem(mesh, alpha=W.dirk_alpha())
    e = int(np.argmax((mesh.face_degree > 0).sum(1)))           # an element with private faces
    sub = pb.pbs[e]
    m, d = pb.m, mesh.d
    u_ref = [x.copy() for x in st.u]                              # fixed reference state
    blk = pb.element_blocks(e, st.u, st.q, st.uhat, u_ref)
    A, B, C, D, F, G = sub.full_system(blk)
    Np, Nb = sub.ref.Np, sub.Nb

    def res(u_e, q_e, uh):
        Rq, Ru, Rh, _ = sub.residual(u_e[None], q_e[None], uh, u_ref[e][None])
        rns = np.concatenate([np.transpose(Rq[0], (1, 2, 0)).reshape(-1), Ru[0].T.reshape(-1)])
        return rns, Rh[0].T.reshape(-1)

    nq = m * d * Np
    rng = np.random.default_rng(0)
    for c in rng.choice(m * Nb, min(10, m * Nb), replace=False):
        i, s = c // Nb, c % Nb
        t = mesh.elem_trace[e][s]
        h = 1e-6 * max(1.0, abs(st.uhat[t, i]))
        up, um = st.uhat.copy(), st.uhat.copy()
        up[t, i] += h
        um[t, i] -= h
        (rp, gp), (rm, gm) = res(st.u[e], st.q[e], up), res(st.u[e], st.q[e], um)
        np.testing.assert_allclose((rp - rm) / (2 * h), B[:, c], rtol=1e-6, atol=2e-7 * np.abs(B).max())
        np.testing.assert_allclose((gp - gm) / (2 * h), D[:, c], rtol=1e-6, atol=2e-7 * np.abs(D).max())
    for c in rng.choice(m * Np, 8, replace=False):
        i, a = c // Np, c % Np
        h = 1e-6 * max(1.0, abs(st.u[e][a, i]))
        up, um = st.u[e].copy(), st.u[e].copy()
        up[a, i] += h
        um[a, i] -= h
        (rp, gp), (rm, gm) = res(up, st.q[e], st.uhat), res(um, st.q[e], st.uhat)
        np.testing.assert_allclose((rp - rm) / (2 * h), A[:, nq + c], rtol=1e-6, atol=2e-7 * np.abs(A).max())
        np.testing.assert_allclose((gp - gm) / (2 * h), C[:, nq + c], rtol=1e-6, atol=2e-7 * np.abs(C).max())


def test_mixed_condensed_solve_equals_global_solve():
    mesh = _mixed(2, 3, (1, 2, 3), (0.3, 0.4, 0.3), 15)
    st = W.make_state_mixed(mesh, W.fourier_perturbed_field(2, 0.3, 7, amp=0.05), 8, noise=0.01)
    pb = _problem(mesh, alpha=W.dirk_alpha())
    m = pb.m
    E = mesh.n_elem
    blks = [pb.element_blocks(e, st.u, st.q, st.uhat) for e in range(E)]
    sizes = [blk["A_qq"].shape[0] + blk["A_uu"].shape[0] for blk in blks]
    off = np.concatenate([[0], np.cumsum(sizes)])
    nt = mesh.n_trace * m
    n = off[-1] + nt
    J = np.zeros((n, n))
    rhs = np.zeros(n)
    for e, blk in enumerate(blks):
        A, B, C, D, F, G = pb.pbs[e].full_system(blk)
        z = slice(off[e], off[e + 1])
        Nb = pb.pbs[e].Nb
        tr = mesh.elem_trace[e]
        gidx = np.array([off[-1] + tr[s] * m + i for i in range(m) for s in range(Nb)])
        J[z, z] = A
        J[z, gidx] += B
        for r, gr in enumerate(gidx):
            J[gr, z] += C[r]
            J[gr, gidx] += D[r]
            rhs[gr] += G[r]
        rhs[z] = F
    x = np.linalg.solve(J, rhs)
    dU_ref = x[off[-1]:].reshape(mesh.n_trace, m)
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat) for e in range(E)])
    row_ptr, col, vals, R = iedg.assemble_ragged(mesh.elem_trace, mesh.n_trace, Ke, Re)
    Kd = np.zeros((nt, nt))
    for r in range(mesh.n_trace):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            Kd[r * m:(r + 1) * m, col[k] * m:(col[k] + 1) * m] = vals[k]
    dU = np.linalg.solve(Kd, R.reshape(-1)).reshape(mesh.n_trace, m)
    assert np.abs(dU - dU_ref).max() <= 1e-10 * np.abs(dU_ref).max()
    for e in range(E):
        du, dq = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, dU)
        zz = x[off[e]:off[e + 1]]
        Np = pb.pbs[e].ref.Np
        du_ref = zz[m * 2 * Np:].reshape(m, Np).T
        assert np.abs(du - du_ref).max() <= 1e-10 * np.abs(du_ref).max()
