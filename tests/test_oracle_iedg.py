"""Pins of the oracle's discretisation (Eq. IEDG a-c, Newton system, Eq. LS):
geometry identities, free-stream preservation, discrete conservation, Jacobian
blocks against finite differences of the residual, condensation against the
uncondensed global solve, and the trace-matrix structure."""
import numpy as np
import pytest

from oracle import iedg
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import global_dense_system, problem


def _params(alpha=0.0, Re=1e3, Minf=0.2):
    return dict(gamma=1.4, Pr=0.72, Re=Re, Minf=Minf, alpha=alpha)


@pytest.mark.parametrize("d,p,curved", [(2, 2, False), (2, 3, True), (3, 2, False), (3, 2, True)])
def test_geometry_identities(d, p, curved):
    mapping = W.stretched_mapping(5, ratio=8.0) if curved else None
    mesh = W.structured_mesh(d, 3, p, mapping=mapping)
    pb = problem(mesh, _params())
    geo = pb.geo
    # total volume of the periodic unit box (the map is measure-preserving on average)
    assert abs(geo.w.sum() - 1.0) < 1e-12
    # closed element surfaces: sum of n dS vanishes per element
    nds = np.einsum("efg,efgj->ej", geo.wf, geo.nf)
    assert np.abs(nds).max() < 1e-14
    # Gauss divergence theorem on each basis function: int dphi_a/dx_j = oint phi_a n_j
    vol = np.einsum("eg,ejga->eja", geo.w, geo.gphi)
    srf = np.einsum("efg,efgj,fga->eja", geo.wf, geo.nf, pb.ref.fphi)
    assert np.abs(vol - srf).max() < 1e-13
    # unit outward normals
    np.testing.assert_allclose(np.linalg.norm(geo.nf, axis=-1), 1.0, atol=1e-14)


@pytest.mark.parametrize("d,p,curved", [(2, 2, False), (2, 3, True), (3, 2, False), (3, 3, True)])
def test_free_stream_preservation(d, p, curved):
    mapping = W.stretched_mapping(6, ratio=8.0) if curved else None
    n = 2 if d == 3 else 3
    mesh = W.structured_mesh(d, n, p, mapping=mapping)
    prm = _params(alpha=W.dirk_alpha())
    pb = problem(mesh, prm)
    f = W.freestream_field(d, 0.2)
    u = f(mesh.node_xyz)
    uh = f(np.zeros((mesh.n_trace, d)))
    q = np.zeros(u.shape + (d,))
    Rq, Ru, Rh, Rfl = pb.residual(u, q, uh)
    scale = np.abs(u).max()
    assert np.abs(Rq).max() < 1e-12 * scale
    assert np.abs(Ru).max() < 1e-12 * scale
    assert np.abs(Rfl).max() < 1e-12 * scale


def test_discrete_conservation():
    """sum_{e,a} R_u[e,a,i] - sum_t R_fl[t,i] = alpha int (u - u_ref)_i - int s_i,
    since the element basis and the trace basis are partitions of unity."""
    wl = W.config(1, N=4)
    st = W.make_state(wl.mesh, W.fourier_perturbed_field(2, 0.2, 3), 4, noise=0.01, uref_shift=0.01)
    src = lambda x: np.stack([np.sin(2 * np.pi * x[..., 0]) + 0.3 * (i + 1) for i in range(4)], -1)
    pb = problem(wl.mesh, _params(alpha=W.dirk_alpha()), source=src)
    Rq, Ru, Rh, Rfl = pb.residual(st.u, st.q, st.uhat, st.u_ref)
    ref = pb.ref
    uq = np.einsum("ga,eai->egi", ref.phi, st.u - st.u_ref)
    rhs = pb.prm.alpha * np.einsum("eg,egi->i", pb.geo.w, uq) - np.einsum("eg,egi->i", pb.geo.w, src(pb.geo.xq))
    lhs = Ru.sum((0, 1)) - Rfl.sum(0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-11)
    assert np.abs(Ru.sum((0, 1))).max() > 1e-3       # the identity is not trivially 0 = 0


@pytest.mark.parametrize("stab", [0, 1])
@pytest.mark.parametrize("d,p", [(2, 2), (3, 2)])
def test_jacobian_blocks_match_finite_differences(d, p, stab):
    """Every block of the Newton matrix equals the central difference of the residual
    (Sec. 2.2.1): columns for q, u of one element and for its trace unknowns; with the
    Lax-Friedrichs (stab 0) and the Roe-type (stab 1) stabilisation."""
    if d == 2:
        mesh = W.structured_mesh(2, 3, p)
        field = W.fourier_perturbed_field(2, 0.3, 7, amp=0.05)
    else:
        mesh = W.structured_mesh(3, 2, p)
        field = W.taylor_green_field(0.3)
    st = W.make_state(mesh, field, 8, noise=0.01, uref_shift=0.01)
    prm = dict(_params(alpha=W.dirk_alpha(), Re=50.0), stab=stab)
    pb = problem(mesh, prm)
    e = 1
    m, Np, Nb = pb.m, pb.ref.Np, pb.ref.Nb
    blk = pb.element_blocks(e, st.u, st.q, st.uhat, st.u_ref)
    A, B, C, D, F, G = pb.full_system(blk)

    def res(u, q, uh):
        Rq, Ru, Rh, _ = pb.residual(u, q, uh, st.u_ref, els=[e])
        rns = np.concatenate([np.transpose(Rq[0], (1, 2, 0)).reshape(-1), Ru[0].T.reshape(-1)])
        return rns, Rh[0].T.reshape(-1)

    r0, g0 = res(st.u, st.q, st.uhat)
    np.testing.assert_allclose(F, -r0, rtol=0, atol=0)
    np.testing.assert_allclose(G, -g0, rtol=0, atol=0)
    rng = np.random.default_rng(0)
    cols_q = rng.choice(m * d * Np, 12, replace=False)
    cols_u = rng.choice(m * Np, 12, replace=False)
    cols_t = rng.choice(m * Nb, 12, replace=False)
    nq = m * d * Np
    for c in cols_q:
        i, j, a = c // (d * Np), (c // Np) % d, c % Np
        h = 1e-6
        qp, qm = st.q.copy(), st.q.copy()
        qp[e, a, i, j] += h
        qm[e, a, i, j] -= h
        (rp, gp), (rm, gm) = res(st.u, qp, st.uhat), res(st.u, qm, st.uhat)
        np.testing.assert_allclose((rp - rm) / (2 * h), A[:, c], rtol=1e-6, atol=2e-7 * np.abs(A).max())
        np.testing.assert_allclose((gp - gm) / (2 * h), C[:, c], rtol=1e-6, atol=2e-7 * np.abs(C).max())
    for c in cols_u:
        i, a = c // Np, c % Np
        h = 1e-6 * max(1.0, abs(st.u[e, a, i]))
        up, um = st.u.copy(), st.u.copy()
        up[e, a, i] += h
        um[e, a, i] -= h
        (rp, gp), (rm, gm) = res(up, st.q, st.uhat), res(um, st.q, st.uhat)
        np.testing.assert_allclose((rp - rm) / (2 * h), A[:, nq + c], rtol=1e-6, atol=2e-7 * np.abs(A).max())
        np.testing.assert_allclose((gp - gm) / (2 * h), C[:, nq + c], rtol=1e-6, atol=2e-7 * np.abs(C).max())
    for c in cols_t:
        i, s = c // Nb, c % Nb
        t = mesh.elem_trace[e, s]
        h = 1e-6 * max(1.0, abs(st.uhat[t, i]))
        up, um = st.uhat.copy(), st.uhat.copy()
        up[t, i] += h
        um[t, i] -= h
        (rp, gp), (rm, gm) = res(st.u, st.q, up), res(st.u, st.q, um)
        np.testing.assert_allclose((rp - rm) / (2 * h), B[:, c], rtol=1e-6, atol=2e-7 * np.abs(B).max())
        np.testing.assert_allclose((gp - gm) / (2 * h), D[:, c], rtol=1e-6, atol=2e-7 * np.abs(D).max())


@pytest.mark.parametrize("cfg,els", [(1, [0, 5, 63]), (2, [0, 2000])])
def test_full_and_qelim_condensation_agree(cfg, els):
    wl = W.config(cfg, N=(None if cfg == 1 else 3))
    pb = problem(wl.mesh, wl.params)
    st = wl.state
    for e in els:
        if e >= wl.mesh.n_elem:
            e = wl.mesh.n_elem - 1
        K1, R1 = pb.condense_full(e, st.u, st.q, st.uhat)
        K2, R2 = pb.condense_qelim(e, st.u, st.q, st.uhat)
        assert np.abs(K1 - K2).max() <= 1e-12 * np.abs(K1).max()
        assert np.abs(R1 - R2).max() <= 1e-12 * np.abs(R1).max()
        du1, dq1 = pb.back_substitute_full(e, st.u, st.q, st.uhat, st.duhat)
        du2, dq2 = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, st.duhat)
        assert np.abs(du1 - du2).max() <= 1e-11 * np.abs(du1).max()
        assert np.abs(dq1 - dq2).max() <= 1e-11 * np.abs(dq1).max()


@pytest.mark.parametrize("d,p", [(2, 2), (2, 3)])
def test_condensed_solve_equals_uncondensed_global_solve(d, p):
    """Solving K dU = R (Eq. LS) and back-substituting reproduces the dense solve
    of the full Newton system [A B; C D] [dZ; dU] = [F; G]."""
    mesh = W.structured_mesh(d, 2, p)
    st = W.make_state(mesh, W.fourier_perturbed_field(d, 0.3, 9, amp=0.05), 10, noise=0.01)
    pb = problem(mesh, _params(alpha=W.dirk_alpha(), Re=100.0))
    J, rhs, nz = global_dense_system(pb, st.u, st.q, st.uhat)
    x = np.linalg.solve(J, rhs)
    E, m = mesh.n_elem, pb.m
    dU_ref = x[E * nz:].reshape(mesh.n_trace, m)
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat) for e in range(E)])
    row_ptr, col, vals, R = iedg.assemble(mesh.elem_trace, mesh.n_trace, np.array(Ke), np.array(Re))
    Kd = np.zeros((mesh.n_trace * m, mesh.n_trace * m))
    for r in range(mesh.n_trace):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            Kd[r * m:(r + 1) * m, col[k] * m:(col[k] + 1) * m] = vals[k]
    dU = np.linalg.solve(Kd, R.reshape(-1)).reshape(mesh.n_trace, m)
    assert np.abs(dU - dU_ref).max() <= 1e-10 * np.abs(dU_ref).max()
    for e in range(E):
        du, dq = pb.back_substitute_qelim(e, st.u, st.q, st.uhat, dU)
        z = x[e * nz:(e + 1) * nz]
        nq = m * d * pb.ref.Np
        dq_ref = z[:nq].reshape(m, d, -1).transpose(2, 0, 1)
        du_ref = z[nq:].reshape(m, -1).T
        assert np.abs(du - du_ref).max() <= 1e-10 * np.abs(du_ref).max()
        assert np.abs(dq - dq_ref).max() <= 1e-9 * np.abs(dq_ref).max()


def _brute_force_nnzb(elem_trace):
    pairs = set()
    for tr in elem_trace.tolist():
        for a in tr:
            for b in tr:
                pairs.add((a, b))
    return len(pairs)


@pytest.mark.parametrize("d,n,p", [(2, 8, 2), (2, 3, 3), (3, 2, 2), (3, 3, 3)])
def test_trace_numbering_and_bsr_pattern(d, n, p):
    mesh = W.structured_mesh(d, n, p)
    # structured periodic count: (pN)^d - N^d (p-1)^d face-lattice nodes
    assert mesh.n_trace == (p * n) ** d - n ** d * (p - 1) ** d
    row_ptr, col = iedg.bsr_pattern(mesh.elem_trace, mesh.n_trace)
    assert row_ptr[-1] == _brute_force_nnzb(mesh.elem_trace)
    for r in range(mesh.n_trace):
        c = col[row_ptr[r]:row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0) and r in c
    # structurally symmetric
    pairs = set(zip(np.repeat(np.arange(mesh.n_trace), np.diff(row_ptr)).tolist(), col.tolist()))
    assert all((c, r) in pairs for r, c in pairs)


def test_config1_sizes():
    """Sizes of the 2D p=2 8x8 workload: 192 trace nodes, 3008 blocks."""
    wl = W.config(1)
    row_ptr, col = iedg.bsr_pattern(wl.mesh.elem_trace, wl.mesh.n_trace)
    assert wl.mesh.n_trace == 192 and row_ptr[-1] == 3008
