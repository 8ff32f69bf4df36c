"""DIRK(3,3) time steps on the GPU (Sec. 2.1 time discretisation, Newton on the
condensed trace system per stage) with the minimal-residual initial guess (Eq.
MinRes2): agreement with an oracle-driven step, discrete conservation over the steps,
and the guess never worse than the previous solution."""
import numpy as np
import pytest

from oracle import geometry
from oracle import iedg as oiedg
from paper_1605_01020_gb300 import timestep
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import problem, ref_element
from gpu_helpers import dev, host, rel_err

pytestmark = pytest.mark.gpu
DT = 0.005


def _setup(d=2):
    """2D: config 1's recipe on 4 x 4 cells.  3D: the Taylor-Green vortex (config 2's
    field and parameters) on 2^3 cells at p = 2."""
    if d == 2:
        wl = W.config(1, N=4)
        st = W.make_state(wl.mesh, W.fourier_perturbed_field(2, 0.2, 41, amp=0.05), 42, noise=0.005)
    else:
        wl2 = W.config(2, N=2)
        mesh = W.structured_mesh(3, 2, 2)
        st = W.make_state(mesh, W.taylor_green_field(0.2), 43, noise=0.005)
        wl = W.Workload("3D TGV p=2 2^3", mesh, st, wl2.params)
    assert abs(wl.params["alpha"] * timestep.GAMMA_DIRK * DT - 1) < 1e-12
    return wl, st


def _oracle_stage(pb, mesh, u, q, uh, u_ref, tol):
    """Newton with the oracle's condensed system and a dense trace solve."""
    m = pb.m
    for _ in range(10):
        Rq, Ru, Rh, Rfl = pb.residual(u, q, uh, u_ref)
        if max(np.abs(Rq).max(), np.abs(Ru).max(), np.abs(Rfl).max()) <= tol:
            return u, q, uh
        E = mesh.n_elem
        Ke, Re = zip(*[pb.condense_qelim(e, u, q, uh, u_ref) for e in range(E)])
        rp, col, vals, R = oiedg.assemble(mesh.elem_trace, mesh.n_trace, np.array(Ke), np.array(Re))
        T = mesh.n_trace
        D = np.zeros((T * m, T * m))
        for r in range(T):
            for k in range(rp[r], rp[r + 1]):
                D[r * m:(r + 1) * m, col[k] * m:(col[k] + 1) * m] = vals[k]
        dU = np.linalg.solve(D, R.reshape(-1)).reshape(T, m)
        du = np.zeros_like(u)
        dq = np.zeros_like(q)
        for e in range(E):
            du[e], dq[e] = pb.back_substitute_qelim(e, u, q, uh, dU, u_ref)
        u, q, uh = u + du, q + dq, uh + dU
    raise AssertionError("oracle Newton did not converge")


@pytest.mark.parametrize("d", [2, 3])
def test_dirk_step_matches_oracle_and_conserves(d):
    from paper_1605_01020_gb300 import iedg
    wl, st = _setup(d)
    mesh = iedg.mesh_from_workload(wl)
    u = dev(st.u)
    uh = dev(st.uhat)
    q = mesh.eval_residual(u, uh, q=None)["q"]
    stepper = timestep.Stepper(mesh, DT, newton_tol=1e-11)
    u1, q1, uh1, its = stepper.step(u, q, uh, use_mr=False)
    assert all(1 <= i <= 6 for i in its), its
    # the same step driven by the oracle (independent restatement of the stage formulas)
    pb = problem(wl.mesh, wl.params)
    A, g = timestep.dirk33(), timestep.GAMMA_DIRK
    uo, qo, uho = st.u.copy(), host(q).copy(), st.uhat.copy()
    un = uo.copy()
    stages = []
    tol = 1e-11 * stepper.rscale
    for i in range(3):
        u_ref = un.copy()
        for j in range(i):
            u_ref = u_ref + (A[i, j] / g) * (stages[j][0] - stages[j][1])
        uo, qo, uho = _oracle_stage(pb, wl.mesh, uo, qo, uho, u_ref, tol)
        stages.append((uo, u_ref))
    assert rel_err(host(u1), uo) <= 1e-9
    assert rel_err(host(uh1), uho) <= 1e-9
    assert rel_err(host(q1), qo) <= 1e-8
    # discrete conservation: sum_e sum_a (sum_g w_g phi_a(g)) u_a is the same before and after
    ref = ref_element(d, wl.mesh.p)
    geo = geometry.Geometry(ref, wl.mesh.node_xyz)
    mvec = np.einsum("eg,ga->ea", geo.w, ref.phi)
    tot0 = np.einsum("ea,eai->i", mvec, st.u)
    tot1 = np.einsum("ea,eai->i", mvec, host(u1))
    assert np.abs(tot1 - tot0).max() <= 1e-10 * np.abs(tot0).max()
    assert np.abs(host(u1) - st.u).max() > 1e-6          # the state did move


def test_minimal_residual_guess():
    """The guess combines the latest solution of the step with the stage's solutions
    at the two previous steps; its residual is never above that of the latest
    solution, and the converged steps are the same with and without it."""
    from paper_1605_01020_gb300 import iedg
    wl, st = _setup()
    mesh = iedg.mesh_from_workload(wl)
    u = dev(st.u)
    uh = dev(st.uhat)
    q = mesh.eval_residual(u, uh, q=None)["q"]
    s_mr = timestep.Stepper(mesh, DT, newton_tol=1e-11)
    s_pl = timestep.Stepper(mesh, DT, newton_tol=1e-11)
    a = (u, q, uh)
    b = (u, q, uh)
    for n in range(4):
        a = s_mr.step(*a, use_mr=True)[:3]
        b = s_pl.step(*b, use_mr=False)[:3]
    assert rel_err(host(a[0]), host(b[0])) <= 1e-9           # same solutions either way
    # residual of the guess for stage 0 of the next step
    u_ref = a[0]
    (gu, gq, guh), beta = s_mr.mr_guess(0, u_ref, a)
    r_mr = float(s_mr.residual_vector(gu, gq, guh, u_ref).norm())
    r_last = float(s_mr.residual_vector(*a, u_ref).norm())
    assert beta is not None and len(beta) == 3
    assert r_mr <= r_last
