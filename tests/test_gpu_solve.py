"""GPU trace solve (GMRES with iterated classical Gram-Schmidt, block-Jacobi left
preconditioning, Sec. 2.2.2) and a whole Newton loop on the GPU."""
import numpy as np
import pytest

from paper_1605_01020_gb300 import workloads as W
from gpu_helpers import dev, host, rel_err

pytestmark = pytest.mark.gpu


def _dense(mesh, K):
    rp, col = (host(t) for t in mesh.trace_pattern())
    Kh = host(K)
    m = mesh.m
    D = np.zeros((mesh.T * m, mesh.T * m))
    for r in range(mesh.T):
        for k in range(rp[r], rp[r + 1]):
            D[r * m:(r + 1) * m, col[k] * m:(col[k] + 1) * m] = Kh[k]
    return D


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_trace_solve_matches_dense_solve(name):
    from paper_1605_01020_gb300 import iedg
    if name == "2d":
        wl = W.config(1)
        st = W.make_state(wl.mesh, W.fourier_perturbed_field(2, 0.2, 21), 22, noise=0.01)
        wl = W.Workload("2d", wl.mesh, st, wl.params)
    else:
        wl = W.config(2, N=3)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl)
    K, R = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat))
    dU, its, rr = mesh.trace_solve(K, R, restart=30, max_iter=600, rtol=1e-12)
    assert rr <= 1e-12 and its < 600
    ref = np.linalg.solve(_dense(mesh, K), host(R).reshape(-1)).reshape(mesh.T, mesh.m)
    assert rel_err(host(dU), ref) <= 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_loop_converges(precision):
    """One implicit stage solved by Newton on the GPU: residual, condensed Jacobian,
    GMRES trace solve, back-substitution, update; the residual must drop
    quadratically (to round-off in at most four steps from a 1 % perturbation)."""
    import torch
    from paper_1605_01020_gb300 import iedg
    wl = W.config(1)
    st = W.make_state(wl.mesh, W.fourier_perturbed_field(2, 0.2, 31), 32, noise=0.01)
    mesh = iedg.mesh_from_workload(wl, precision=precision)
    u_ref = dev(st.u)
    rng = np.random.default_rng(5)
    u = dev(st.u * (1 + 0.01 * rng.uniform(-1, 1, st.u.shape)))
    uh = dev(st.uhat)
    q = mesh.eval_residual(u, uh, q=None)["q"]          # start with R_q = 0
    norms = []
    for it in range(6):
        res = mesh.eval_residual(u, uh, q=q, u_ref=u_ref)
        nrm = max(float(res["r_u"].abs().max()), float(res["r_fl"].abs().max()), float(res["r_q"].abs().max()))
        norms.append(nrm)
        if nrm < 1e-11 * norms[0]:
            break
        K, R = mesh.assemble_condensed(u, q, uh, u_ref=u_ref)
        dU, its, rr = mesh.trace_solve(K, R, rtol=1e-12, max_iter=800)
        du, dq = mesh.back_substitute(dU)
        u = u + du
        q = q + dq
        uh = uh + dU
    assert norms[-1] < 1e-10 * norms[0], norms
    assert len(norms) <= 6, norms


def _bilu_case(name):
    if name == "2d":
        return W.config(1)
    return W.config(2, N=2)


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_bilu0_matches_oracle(name):
    """BILU(0) in multicolour order (Sec. 2.2.2): colouring bit-exact, factors and the
    preconditioner solve within 1e-11 of the oracle on the same K."""
    from oracle import bilu
    from paper_1605_01020_gb300 import iedg
    wl = _bilu_case(name)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl)
    K, R = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat))
    rp, col = (host(t).astype(np.int64) for t in mesh.trace_pattern())
    rank, color = bilu.multicolor_rank(rp, col)
    assert np.array_equal(mesh.trace_colors(), color)
    F_o = bilu.bilu0(rp, col, host(K), rank)
    F = mesh.bilu0_factor(K)
    worst = max(np.abs(host(F)[rp[r]:rp[r + 1]] - F_o[rp[r]:rp[r + 1]]).max() / np.abs(F_o[rp[r]:rp[r + 1]]).max()
                for r in range(mesh.T))
    assert worst <= 1e-11
    x_o = bilu.bilu0_solve(rp, col, F_o, host(R), rank)
    x = mesh.bilu0_apply(F, R)
    assert rel_err(host(x), x_o) <= 1e-11


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_gmres_with_bilu0(name):
    """GMRES with the BILU(0) preconditioner reaches the dense solution and needs no
    more iterations than with block Jacobi."""
    from paper_1605_01020_gb300 import iedg
    wl = W.config(1) if name == "2d" else W.config(2, N=3)
    st = wl.state
    mesh = iedg.mesh_from_workload(wl)
    K, R = mesh.assemble_condensed(dev(st.u), dev(st.q), dev(st.uhat))
    dU_j, its_j, rr_j = mesh.trace_solve(K, R, restart=30, max_iter=800, rtol=1e-12)
    mesh.set_trace_precond(iedg.PREC_BILU0)
    dU_b, its_b, rr_b = mesh.trace_solve(K, R, restart=30, max_iter=800, rtol=1e-12)
    assert rr_b <= 1e-12 and its_b <= its_j, (its_b, its_j)
    ref = np.linalg.solve(_dense(mesh, K), host(R).reshape(-1)).reshape(mesh.T, mesh.m)
    assert rel_err(host(dU_b), ref) <= 1e-8
