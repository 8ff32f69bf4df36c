"""Manufactured-solution convergence of the oracle's discretisation (2D periodic,
one implicit stage with alpha = 1 and u_ref = u_ex at the nodes, so the manufactured
u_ex solves alpha (u - u_ex) + div F(u, grad u) - s = 0; a purely steady periodic
problem has a singular Jacobian because total mass, momentum and energy are then
undetermined): Newton on Eq. NLS through the condensed system Eq. LS,
then ||u_h - u_ex||_L2 must fall like h^(p+1) (optimal rate of the IEDG family for
smooth solutions; Re = 1000 keeps the problem in the convection-dominated
regime of the paper's flows, where the continuous-trace (EDG) family shows its
asymptotic rate on these small meshes).  This pins the weak form (Eq. IEDG a-c), the numerical flux,
the Newton blocks and the condensation/back-substitution all together."""
import numpy as np
import pytest

from oracle import iedg, physics
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import problem

G = 1.4
P0 = 1.0 / (G * 0.5 ** 2)
TP = 2 * np.pi


def exact(x):
    """Conserved u_ex [..., 4] and its gradient [..., 4, 2] on the unit torus."""
    X, Y = x[..., 0], x[..., 1]
    rho = 1 + 0.1 * np.sin(TP * X) * np.sin(TP * Y)
    drho = np.stack([0.1 * TP * np.cos(TP * X) * np.sin(TP * Y), 0.1 * TP * np.sin(TP * X) * np.cos(TP * Y)], -1)
    vx = 0.6 + 0.1 * np.cos(TP * Y)
    dvx = np.stack([0 * X, -0.1 * TP * np.sin(TP * Y)], -1)
    vy = 0.2 + 0.1 * np.sin(TP * X)
    dvy = np.stack([0.1 * TP * np.cos(TP * X), 0 * X], -1)
    p = P0 * (1 + 0.05 * np.cos(TP * (X + Y)))
    dp = np.stack([-P0 * 0.05 * TP * np.sin(TP * (X + Y))] * 2, -1)
    u = np.stack([rho, rho * vx, rho * vy, p / (G - 1) + 0.5 * rho * (vx ** 2 + vy ** 2)], -1)
    du = np.stack([drho,
                   vx[..., None] * drho + rho[..., None] * dvx,
                   vy[..., None] * drho + rho[..., None] * dvy,
                   dp / (G - 1) + 0.5 * (vx ** 2 + vy ** 2)[..., None] * drho
                   + rho[..., None] * (vx[..., None] * dvx + vy[..., None] * dvy)], -2)
    return u, du


def make_source(prm):
    """s = div F(u_ex, grad u_ex), by 4th-order central differences of the analytic flux."""
    def flux_at(x):
        u, du = exact(x)
        F, _, _ = physics.flux_with_jacobians(u, du, prm, 2)
        return F

    def src(x):
        h = 1e-3
        s = 0.0
        for j in range(2):
            e = np.zeros(2)
            e[j] = h
            dF = (-flux_at(x + 2 * e) + 8 * flux_at(x + e) - 8 * flux_at(x - e) + flux_at(x - 2 * e)) / (12 * h)
            s = s + dF[..., :, j]
        return s
    return src


def solve_mms(n, p, Re=1000.0):
    mesh = W.structured_mesh(2, n, p)
    prm = dict(gamma=G, Pr=0.72, Re=Re, Minf=0.5, alpha=1.0)
    pb0 = problem(mesh, prm)
    pb = problem(mesh, prm, source=make_source(pb0.prm))
    m = 4
    u, q = exact(mesh.node_xyz)
    u_ref = u.copy()
    xt = np.zeros((mesh.n_trace, 2))
    xt[mesh.elem_trace.reshape(-1)] = mesh.node_xyz[:, mesh.bnodes].reshape(-1, 2)
    uh = exact(xt)[0]
    E = mesh.n_elem
    for it in range(10):
        Ke, Re_ = zip(*[pb.condense_qelim(e, u, q, uh, u_ref) for e in range(E)])
        row_ptr, col, vals, R = iedg.assemble(mesh.elem_trace, mesh.n_trace, np.array(Ke), np.array(Re_))
        Kd = np.zeros((mesh.n_trace * m,) * 2)
        for r in range(mesh.n_trace):
            for k in range(row_ptr[r], row_ptr[r + 1]):
                Kd[r * m:(r + 1) * m, col[k] * m:(col[k] + 1) * m] = vals[k]
        dU = np.linalg.solve(Kd, R.reshape(-1)).reshape(mesh.n_trace, m)
        for e in range(E):
            du, dq = pb.back_substitute_qelim(e, u, q, uh, dU, u_ref)
            u[e] += du
            q[e] += dq
        uh = uh + dU
        if np.abs(dU).max() < 1e-10:
            break
    assert np.abs(dU).max() < 1e-8, "Newton did not converge"
    ue, _ = exact(pb.geo.xq)
    uhq = np.einsum("ga,eai->egi", pb.ref.phi, u)
    return np.sqrt(np.einsum("eg,egi->", pb.geo.w, (uhq - ue) ** 2))


@pytest.mark.slow
@pytest.mark.parametrize("p,ns", [(1, (8, 16)), (2, (8, 16)), (3, (4, 8))])
def test_mms_convergence_rate(p, ns):
    errs = [solve_mms(n, p) for n in ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] >= p + 0.8, (errs, rates)
