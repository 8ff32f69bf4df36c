"""Host logic of the time stepper (no GPU): the DIRK(3,3) tableau of Sec. 2.1 and the
Levenberg-Marquardt solver of the minimal-residual guess (Eq. MinRes2)."""
import numpy as np

from paper_1605_01020_gb300 import timestep


def test_dirk33_tableau_order_conditions():
    A = timestep.dirk33()
    b = A[-1]
    c = A.sum(1)
    g = timestep.GAMMA_DIRK
    assert np.allclose(np.diag(A), g)
    # third order: sum b = 1, b.c = 1/2, b.c^2 = 1/3, b.A.c = 1/6
    assert abs(b.sum() - 1) < 1e-14
    assert abs(b @ c - 0.5) < 1e-14
    assert abs(b @ c ** 2 - 1 / 3) < 1e-13
    assert abs(b @ A @ c - 1 / 6) < 1e-13
    # L-stability: stability function R(z) -> 0 as z -> -inf (stiffly accurate, A invertible)
    z = -1e8
    R = 1 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))
    assert abs(R) < 1e-6
    assert abs(c[-1] - 1) < 1e-14


def test_levenberg_marquardt_linear_least_squares():
    rng = np.random.default_rng(0)
    Z = rng.standard_normal((40, 3))
    t = rng.standard_normal(40)
    beta, phi, evals = timestep.levenberg_marquardt(lambda b: Z @ b - t, [1.0, 0.0, 0.0])
    ref = np.linalg.lstsq(Z, t, rcond=None)[0]
    assert np.abs(beta - ref).max() < 1e-6
    assert abs(phi - np.sum((Z @ ref - t) ** 2)) < 1e-10


def test_levenberg_marquardt_nonlinear_never_worse_than_the_start():
    # Rosenbrock-like residual; LM only accepts decreases
    resid = lambda b: np.array([10 * (b[1] - b[0] ** 2), 1 - b[0]])
    start = np.array([-1.2, 1.0])
    beta, phi, _ = timestep.levenberg_marquardt(resid, start, max_iter=200)
    assert phi <= np.sum(resid(start) ** 2)
    assert np.abs(beta - 1).max() < 1e-4
