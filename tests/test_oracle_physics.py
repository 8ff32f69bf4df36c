"""Pins of the oracle's pointwise physics (Sec. 2.1 flux definitions, Eq. IEDG d)
against closed forms, exact invariants and finite differences."""
import numpy as np
import pytest

from oracle import physics

PRM = physics.Params(gamma=1.4, Pr=0.72, Re=100.0, Minf=0.3)


def _state(d, rng):
    rho = 1.0 + 0.2 * rng.random()
    v = rng.normal(size=d) * 0.5
    p = 3.0 + rng.random()
    u = np.concatenate([[rho], rho * v, [p / 0.4 + 0.5 * rho * v @ v]])
    q = rng.normal(size=(d + 2, d))
    return u, q


@pytest.mark.parametrize("d", [2, 3])
def test_euler_flux_homogeneity_and_eigenvalues(d):
    """Inviscid flux is homogeneous of degree 1: (dF/du) u = F (exact for Euler);
    the normal Jacobian has eigenvalues v.n (d-fold) and v.n +- c."""
    rng = np.random.default_rng(d)
    u, _ = _state(d, rng)
    q0 = np.zeros((d + 2, d))
    F, Fu, Fq = physics.flux_with_jacobians(u[None], q0[None], PRM, d)
    np.testing.assert_allclose(np.einsum("ijk,k->ij", Fu[0], u), F[0], rtol=1e-13, atol=1e-13)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    An = np.einsum("ijk,j->ik", Fu[0], n)
    ev = np.sort(np.linalg.eigvals(An).real)
    rho = u[0]
    v = u[1:d + 1] / rho
    p = 0.4 * (u[-1] - 0.5 * rho * v @ v)
    c = np.sqrt(1.4 * p / rho)
    vn = v @ n
    np.testing.assert_allclose(ev, np.sort([vn - c] + [vn] * d + [vn + c]), atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_viscous_flux_linear_in_q(d):
    rng = np.random.default_rng(10 + d)
    u, q = _state(d, rng)
    F, Fu, Fq = physics.flux_with_jacobians(u[None], q[None], PRM, d)
    F0, _, _ = physics.flux_with_jacobians(u[None], 0 * q[None], PRM, d)
    np.testing.assert_allclose(np.einsum("ijkl,kl->ij", Fq[0], q), F[0] - F0[0], rtol=1e-12, atol=1e-13)


def test_shear_stress_closed_form():
    """Fluid at rest with d(rho v_x)/dy = s: tau_xy = s / Re, no heat flux."""
    d, s = 3, 0.7
    p0 = 2.0
    u = np.array([1.0, 0, 0, 0, p0 / 0.4])
    q = np.zeros((5, 3))
    q[1, 1] = s
    F = physics.flux(list(u), [list(r) for r in q], PRM, d)
    assert abs(F[1][1] - (-s / PRM.Re)) < 1e-15
    assert abs(F[2][0] - (-s / PRM.Re)) < 1e-15
    assert abs(F[1][0] - p0) < 1e-14 and abs(F[2][1] - p0) < 1e-14
    assert all(abs(F[4][j]) < 1e-15 for j in range(d))


def test_heat_flux_is_dissipative():
    """Fluid at rest, rho = 1, d(rho E)/dx_j = g_j: e = E, energy flux
    = -(gamma / (Re Pr)) g_j (heat flows down the temperature gradient)."""
    d = 3
    g = np.array([0.3, -0.2, 0.5])
    u = np.array([1.0, 0, 0, 0, 5.0])
    q = np.zeros((5, 3))
    q[4] = g
    F = physics.flux(list(u), [list(r) for r in q], PRM, d)
    kappa = PRM.gamma / (PRM.Re * PRM.Pr)
    for j in range(d):
        assert abs(F[4][j] - (-kappa * g[j])) < 1e-15


@pytest.mark.parametrize("d", [2, 3])
def test_dual_jacobians_match_finite_differences(d):
    rng = np.random.default_rng(20 + d)
    u, q = _state(d, rng)
    F, Fu, Fq = physics.flux_with_jacobians(u[None], q[None], PRM, d)
    h = 1e-6
    for k in range(d + 2):
        du = np.zeros(d + 2)
        du[k] = h * max(1.0, abs(u[k]))
        Fp, _, _ = physics.flux_with_jacobians((u + du)[None], q[None], PRM, d)
        Fm, _, _ = physics.flux_with_jacobians((u - du)[None], q[None], PRM, d)
        np.testing.assert_allclose((Fp - Fm)[0] / (2 * du[k]), Fu[0][:, :, k], rtol=1e-6, atol=1e-7)
    for k in range(d + 2):
        for l in range(d):
            dq = np.zeros((d + 2, d))
            dq[k, l] = h
            Fp, _, _ = physics.flux_with_jacobians(u[None], (q + dq)[None], PRM, d)
            Fm, _, _ = physics.flux_with_jacobians(u[None], (q - dq)[None], PRM, d)
            np.testing.assert_allclose((Fp - Fm)[0] / (2 * h), Fq[0][:, :, k, l], rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("d", [2, 3])
def test_lax_friedrichs_flux(d):
    rng = np.random.default_rng(30 + d)
    uh, q = _state(d, rng)
    u, _ = _state(d, rng)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    f, fuh, fu, fq = physics.numerical_flux_with_jacobians(uh[None], u[None], q[None], n[None], PRM, d)
    F, _, Fq = physics.flux_with_jacobians(uh[None], q[None], PRM, d)
    rho = uh[0]
    v = uh[1:d + 1] / rho
    p = 0.4 * (uh[-1] - 0.5 * rho * v @ v)
    lam = abs(v @ n) + np.sqrt(1.4 * p / rho)
    np.testing.assert_allclose(f[0], F[0] @ n + lam * (u - uh), rtol=1e-14, atol=1e-13)
    np.testing.assert_allclose(fu[0], lam * np.eye(d + 2), atol=1e-14)
    np.testing.assert_allclose(fq[0], np.einsum("ijkl,j->ikl", Fq[0], n), atol=1e-14)
    # consistency: u = uhat gives the physical normal flux
    f2, *_ = physics.numerical_flux_with_jacobians(uh[None], uh[None], q[None], n[None], PRM, d)
    np.testing.assert_allclose(f2[0], F[0] @ n, rtol=1e-14, atol=1e-13)
    # d fhat / d uhat by central differences
    h = 1e-6
    for k in range(d + 2):
        du = np.zeros(d + 2)
        du[k] = h * max(1.0, abs(uh[k]))
        fp, *_ = physics.numerical_flux_with_jacobians((uh + du)[None], u[None], q[None], n[None], PRM, d)
        fm, *_ = physics.numerical_flux_with_jacobians((uh - du)[None], u[None], q[None], n[None], PRM, d)
        np.testing.assert_allclose((fp - fm)[0] / (2 * du[k]), fuh[0][:, k], rtol=1e-6, atol=1e-7)


PRM_ROE = physics.Params(gamma=1.4, Pr=0.72, Re=100.0, Minf=0.3, stab=1)


def _normal_jacobian(uh, n, d):
    q0 = np.zeros((d + 2, d))
    _, Fu, _ = physics.flux_with_jacobians(uh[None], q0[None], PRM, d)
    return np.einsum("ijk,j->ik", Fu[0], n)


@pytest.mark.parametrize("d", [2, 3])
def test_roe_matrix_is_the_absolute_value_of_the_normal_jacobian(d):
    """S = |A_n(uhat)| = R |Lambda| R^-1 from numpy's eigen-decomposition of the
    dual-number Jacobian A_n; for supersonic flow along n every eigenvalue is
    positive and S = A_n; S is applied by the closed form of the oracle."""
    rng = np.random.default_rng(40 + d)
    for trial in range(4):
        uh, _ = _state(d, rng)
        n = rng.normal(size=d)
        n /= np.linalg.norm(n)
        if trial == 3:                         # supersonic along n
            rho = uh[0]
            p = 0.4 * (uh[-1] - 0.5 * uh[1:d + 1] @ uh[1:d + 1] / rho)
            c = np.sqrt(1.4 * p / rho)
            v = 2.5 * c * n
            uh = np.concatenate([[rho], rho * v, [p / 0.4 + 0.5 * rho * v @ v]])
        An = _normal_jacobian(uh, n, d)
        lam, R = np.linalg.eig(An)
        absA = np.real(R @ np.diag(np.abs(lam)) @ np.linalg.inv(R))
        S = np.stack([np.array(physics.roe_dissipation(uh, np.eye(d + 2)[k], n, PRM_ROE, d)) for k in range(d + 2)], 1)
        np.testing.assert_allclose(S, absA, rtol=1e-10, atol=1e-10 * np.abs(absA).max())
        if trial == 3:
            np.testing.assert_allclose(S, An, rtol=1e-12, atol=1e-12 * np.abs(An).max())


@pytest.mark.parametrize("d", [2, 3])
def test_roe_flux_consistency_and_jacobians(d):
    rng = np.random.default_rng(50 + d)
    uh, q = _state(d, rng)
    u, _ = _state(d, rng)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    f, fuh, fu, fq = physics.numerical_flux_with_jacobians(uh[None], u[None], q[None], n[None], PRM_ROE, d)
    F, _, Fq = physics.flux_with_jacobians(uh[None], q[None], PRM_ROE, d)
    S = np.stack([np.array(physics.roe_dissipation(uh, np.eye(d + 2)[k], n, PRM_ROE, d)) for k in range(d + 2)], 1)
    np.testing.assert_allclose(f[0], F[0] @ n + S @ (u - uh), rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(fu[0], S, rtol=1e-13, atol=1e-13 * np.abs(S).max())
    np.testing.assert_allclose(fq[0], np.einsum("ijkl,j->ikl", Fq[0], n), atol=1e-14)
    f2, *_ = physics.numerical_flux_with_jacobians(uh[None], uh[None], q[None], n[None], PRM_ROE, d)
    np.testing.assert_allclose(f2[0], F[0] @ n, rtol=1e-14, atol=1e-13)
    h = 1e-6
    for k in range(d + 2):
        du = np.zeros(d + 2)
        du[k] = h * max(1.0, abs(uh[k]))
        fp, *_ = physics.numerical_flux_with_jacobians((uh + du)[None], u[None], q[None], n[None], PRM_ROE, d)
        fm, *_ = physics.numerical_flux_with_jacobians((uh - du)[None], u[None], q[None], n[None], PRM_ROE, d)
        np.testing.assert_allclose((fp - fm)[0] / (2 * du[k]), fuh[0][:, k], rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("d", [2, 3])
def test_normal_jacobian_apply_matches_dual_jacobian(d):
    rng = np.random.default_rng(60 + d)
    uh, _ = _state(d, rng)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    An = _normal_jacobian(uh, n, d)
    for k in range(d + 2):
        x = np.eye(d + 2)[k]
        np.testing.assert_allclose(np.array(physics.normal_jacobian_apply(uh, x, n, PRM, d)), An[:, k],
                                   rtol=1e-13, atol=1e-13 * np.abs(An).max())


def _bflux(uh, u, q, n, d, kind, ub, prm=PRM):
    b, buh, bu, bq = physics.boundary_flux_with_jacobians(uh[None], u[None], q[None], n[None], prm, d, kind, ub)
    return b[0], buh[0], bu[0], bq[0]


@pytest.mark.parametrize("d", [2, 3])
def test_farfield_boundary_flux(d):
    """Upwinding of the far-field flux: free stream gives zero; with u = u_b only the
    A_n (uhat - u) part is left; supersonic outflow ignores u_b and supersonic inflow
    ignores u (every wave leaves, resp. enters, through the face)."""
    rng = np.random.default_rng(70 + d)
    uh, q = _state(d, rng)
    u, _ = _state(d, rng)
    ub, _ = _state(d, rng)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    K = physics.FACE_FARFIELD
    b, *_ = _bflux(uh, uh, q, n, d, K, uh)
    assert np.abs(b).max() < 1e-12 * np.abs(uh).max()
    An = _normal_jacobian(uh, n, d)
    b, *_ = _bflux(uh, u, q, n, d, K, u)
    np.testing.assert_allclose(b, An @ (uh - u), rtol=1e-12, atol=1e-12 * np.abs(An).max())
    rho = uh[0]
    p = 0.4 * (uh[-1] - 0.5 * uh[1:d + 1] @ uh[1:d + 1] / rho)
    c = np.sqrt(1.4 * p / rho)
    for sgn in (1.0, -1.0):
        v = sgn * 2.5 * c * n
        us = np.concatenate([[rho], rho * v, [p / 0.4 + 0.5 * rho * v @ v]])
        As = _normal_jacobian(us, n, d)
        b, *_ = _bflux(us, u, q, n, d, K, ub)
        ref = As @ (us - u) if sgn > 0 else As @ (us - ub)
        np.testing.assert_allclose(b, ref, rtol=1e-10, atol=1e-10 * np.abs(As).max())


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("d", [2, 3])
def test_boundary_flux_jacobians_by_finite_differences(d, kind):
    rng = np.random.default_rng(80 + d + 10 * kind)
    uh, q = _state(d, rng)
    u, _ = _state(d, rng)
    ub, _ = _state(d, rng)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    b, buh, bu, bq = _bflux(uh, u, q, n, d, kind, ub)
    if kind == physics.FACE_WALL:
        f, *_ = physics.numerical_flux_with_jacobians(uh[None], u[None], q[None], n[None], PRM, d)
        np.testing.assert_allclose(b, np.concatenate([[uh[0] - u[0]], uh[1:d + 1], [f[0][-1]]]), rtol=1e-14)
    h = 1e-6
    for k in range(d + 2):
        e = np.zeros(d + 2)
        e[k] = h * max(1.0, abs(uh[k]))
        bp, *_ = _bflux(uh + e, u, q, n, d, kind, ub)
        bm, *_ = _bflux(uh - e, u, q, n, d, kind, ub)
        np.testing.assert_allclose((bp - bm) / (2 * e[k]), buh[:, k], rtol=1e-6, atol=1e-6)
        e = np.zeros(d + 2)
        e[k] = h * max(1.0, abs(u[k]))
        bp, *_ = _bflux(uh, u + e, q, n, d, kind, ub)
        bm, *_ = _bflux(uh, u - e, q, n, d, kind, ub)
        np.testing.assert_allclose((bp - bm) / (2 * e[k]), bu[:, k], rtol=1e-6, atol=1e-6)
    for k in range(d + 2):
        for l in range(d):
            dq = np.zeros_like(q)
            dq[k, l] = h
            bp, *_ = _bflux(uh, u, q + dq, n, d, kind, ub)
            bm, *_ = _bflux(uh, u, q - dq, n, d, kind, ub)
            np.testing.assert_allclose((bp - bm) / (2 * h), bq[:, k, l], rtol=1e-6, atol=1e-7)
