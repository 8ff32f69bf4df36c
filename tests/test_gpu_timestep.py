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


def alexander_tableau():
    """Alexander's L-stable, stiffly accurate three-stage DIRK, stated here apart from
    the stepper: gamma is the root in (0.4, 0.5) of 6 g^3 - 18 g^2 + 9 g - 1 = 0 (the
    condition that makes the stability function vanish at infinity with b = last row),
    c = (gamma, (1 + gamma) / 2, 1), a_21 = c_2 - gamma, and b_1, b_2 follow from the
    order conditions sum b = 1, sum b c = 1/2 with b_3 = gamma."""
    roots = np.roots([6.0, -18.0, 9.0, -1.0])
    g = float([r.real for r in roots if abs(r.imag) < 1e-12 and 0.4 < r.real < 0.5][0])
    c2 = (1.0 + g) / 2.0
    b12 = np.linalg.solve(np.array([[1.0, 1.0], [g, c2]]), np.array([1.0 - g, 0.5 - g]))
    A = np.array([[g, 0.0, 0.0], [c2 - g, g, 0.0], [b12[0], b12[1], g]])
    return A, g


def test_own_tableau_satisfies_third_order_conditions():
    A, g = alexander_tableau()
    b, c = A[2], A.sum(axis=1)
    assert abs(b.sum() - 1) < 1e-13 and abs(b @ c - 0.5) < 1e-13
    assert abs(b @ c ** 2 - 1 / 3) < 1e-13 and abs(b @ A @ c - 1 / 6) < 1e-13


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
    assert abs(wl.params["alpha"] * alexander_tableau()[1] * DT - 1) < 1e-12
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
    A, g = alexander_tableau()
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


def test_temporal_order_three():
    """Alexander's scheme is third order: on a smooth 2D state, the GPU stepper's error
    at t = 0.04 against a run with a quarter of the smallest step falls like dt^3 as dt
    halves (same mesh and order, so only the time error changes); the observed rate
    approaches 3 from below as dt shrinks (2.0 and 2.7 from dt = 0.02 to 0.005)."""
    from paper_1605_01020_gb300 import iedg
    wl0 = W.config(1, N=4)
    st = W.make_state(wl0.mesh, W.fourier_perturbed_field(2, 0.2, 41, amp=0.05), 42, noise=0.0)
    _, g = alexander_tableau()
    T_END = 0.04

    def run(dt):
        n = int(round(T_END / dt))
        wl = W.Workload("2D p=2 4x4 smooth", wl0.mesh, st, dict(wl0.params, alpha=1.0 / (g * dt)))
        mesh = iedg.mesh_from_workload(wl)
        u, uh = dev(st.u), dev(st.uhat)
        q = mesh.eval_residual(u, uh, q=None)["q"]
        stepper = timestep.Stepper(mesh, dt, newton_tol=1e-12)
        state = (u, q, uh)
        for _ in range(n):
            state = stepper.step(*state, use_mr=False)[:3]
        out = host(state[0]).copy()
        mesh.close()
        return out

    dts = [0.01, 0.005, 0.0025]
    ref = run(dts[-1] / 4)
    errs = [np.abs(run(dt) - ref).max() for dt in dts]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print("errors", errs, "rates", rates)
    assert errs[-1] < errs[0]
    assert min(rates) >= 2.5 and rates[-1] >= 2.7, (errs, rates)
