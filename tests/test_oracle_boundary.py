"""Pins of the oracle with domain boundaries (Sec. 2.1: traces discontinuous on the
boundary faces, the trace equation takes the boundary flux bhat there): far-field
(inflow/outflow) faces keep a free stream exactly, walls keep a fluid at rest
exactly, every Newton block equals finite differences of the residual on elements
with boundary faces, and the condensed solve equals the uncondensed global solve."""
import numpy as np
import pytest

from oracle import iedg, physics
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import ref_element

GAMMA = 1.4


def _mesh(d, N, levels, boundary, seed):
    probs = np.full(len(levels), 1.0 / len(levels))
    orders = W.mixed_orders([N] * d, seed, levels=levels, probs=probs)
    return W.structured_mesh_mixed(d, N, orders, boundary=boundary)


def _problem(mesh, ub, alpha=0.0, Re=100.0, stab=0):
    refs = {int(p): ref_element(mesh.d, int(p)) for p in set(mesh.orders.tolist())}
    prm = physics.Params(gamma=GAMMA, Pr=0.72, Re=Re, Minf=0.3, alpha=alpha, stab=stab)
    return iedg.MixedProblem(refs, mesh, prm, ub=ub)


def _uniform(d, v):
    rho, p = 1.0, 1.0 / (GAMMA * 0.3 ** 2)
    v = np.asarray(v, dtype=np.float64)
    return np.concatenate([[rho], rho * v, [p / (GAMMA - 1) + 0.5 * rho * v @ v]])


@pytest.mark.parametrize("stab", [0, 1])
@pytest.mark.parametrize("d,N,levels,boundary", [(2, 4, (1, 2), (1, 1)), (3, 2, (1, 2), (1, 1, 0))])
def test_free_stream_with_far_field_boundaries(d, N, levels, boundary, stab):
    mesh = _mesh(d, N, levels, boundary, 3)
    assert (mesh.face_kind == physics.FACE_FARFIELD).any()
    ub = _uniform(d, [0.6, 0.3, 0.1][:d])
    pb = _problem(mesh, ub, alpha=W.dirk_alpha(), stab=stab)
    u = [np.tile(ub, (len(x), 1)) for x in mesh.node_xyz]
    q = [np.zeros(x.shape + (d,)) for x in u]
    uh = np.tile(ub, (mesh.n_trace, 1))
    Rq, Ru, Rh, Rfl = pb.residual(u, q, uh)
    scale = np.abs(ub).max()
    assert max(np.abs(r).max() for r in Ru) < 1e-12 * scale
    assert np.abs(Rfl).max() < 1e-12 * scale


@pytest.mark.parametrize("d,N,levels,boundary", [(2, 4, (1, 2), (1, 2)), (3, 2, (1, 2), (2, 2, 1))])
def test_rest_state_with_walls(d, N, levels, boundary):
    mesh = _mesh(d, N, levels, boundary, 4)
    assert (mesh.face_kind == physics.FACE_WALL).any()
    ub = _uniform(d, np.zeros(d))
    pb = _problem(mesh, ub)
    u = [np.tile(ub, (len(x), 1)) for x in mesh.node_xyz]
    q = [np.zeros(x.shape + (d,)) for x in u]
    uh = np.tile(ub, (mesh.n_trace, 1))
    uh[:, 1:d + 1] = 0.0
    Rq, Ru, Rh, Rfl = pb.residual(u, q, uh)
    assert max(np.abs(r).max() for r in Ru) < 1e-12 * np.abs(ub).max()
    assert np.abs(Rfl).max() < 1e-12 * np.abs(ub).max()


@pytest.mark.parametrize("stab", [0, 1])
@pytest.mark.parametrize("d", [2, 3])
def test_boundary_element_blocks_match_finite_differences(d, stab):
    if d == 2:
        mesh = _mesh(2, 3, (1, 2), (1, 2), 5)
        field = W.fourier_perturbed_field(2, 0.3, 9, amp=0.05)
    else:
        mesh = _mesh(3, 2, (1, 2), (1, 2, 0), 6)
        field = W.taylor_green_field(0.3)
    st = W.make_state_mixed(mesh, field, 10, noise=0.01)
    ub = _uniform(d, [0.5, 0.1, 0.0][:d])
    pb = _problem(mesh, ub, alpha=W.dirk_alpha(), Re=50.0, stab=stab)
    e = int(np.argmax((mesh.face_kind != 0).sum(1)))
    assert (mesh.face_kind[e] == 1).any() or (mesh.face_kind[e] == 2).any()
    sub = pb.pbs[e]
    m = pb.m
    u_ref = [x.copy() for x in st.u]
    blk = pb.element_blocks(e, st.u, st.q, st.uhat, u_ref)
    A, B, C, D, F, G = sub.full_system(blk)
    Np, Nb = sub.ref.Np, sub.Nb

    def res(u_e, q_e, uh):
        Rq, Ru, Rh, _ = sub.residual(u_e[None], q_e[None], uh, u_ref[e][None])
        rns = np.concatenate([np.transpose(Rq[0], (1, 2, 0)).reshape(-1), Ru[0].T.reshape(-1)])
        return rns, Rh[0].T.reshape(-1)

    r0, g0 = res(st.u[e], st.q[e], st.uhat)
    np.testing.assert_allclose(G, -g0, rtol=0, atol=0)
    nq = m * d * Np
    rng = np.random.default_rng(0)
    for c in rng.choice(m * Nb, min(14, m * Nb), replace=False):
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
    for c in rng.choice(nq, 8, replace=False):
        i, j, a = c // (d * Np), (c // Np) % d, c % Np
        h = 1e-6
        qp, qm = st.q[e].copy(), st.q[e].copy()
        qp[a, i, j] += h
        qm[a, i, j] -= h
        (rp, gp), (rm, gm) = res(st.u[e], qp, st.uhat), res(st.u[e], qm, st.uhat)
        np.testing.assert_allclose((rp - rm) / (2 * h), A[:, c], rtol=1e-6, atol=2e-7 * np.abs(A).max())
        np.testing.assert_allclose((gp - gm) / (2 * h), C[:, c], rtol=1e-6, atol=2e-7 * np.abs(C).max())


def test_boundary_condensed_solve_equals_global_solve():
    mesh = _mesh(2, 3, (1, 2, 3), (1, 2), 7)
    st = W.make_state_mixed(mesh, W.fourier_perturbed_field(2, 0.3, 11, amp=0.05), 12, noise=0.01)
    pb = _problem(mesh, _uniform(2, [0.5, 0.0]), alpha=W.dirk_alpha())
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
