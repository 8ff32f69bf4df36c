"""Implicit time stepping on top of the element-local library: the DIRK stages of
Sec. 2.1 (Alexander's L-stable three-stage scheme), each stage solved by Newton's
method with the condensed trace system (Eq. NLS, Eq. LS), and the minimal-residual
initial guess of Sec. 2.2 (Eq. MinRes2, Levenberg-Marquardt with finite-difference
gradients).  Host-side driver only: every residual, Jacobian, trace solve and
back-substitution is a call into libiedg.so through the binding.

Stage equations.  With M du/dt + R_sp(u) = 0 (R_sp the spatial residual of Eq.
IEDG b) and a DIRK tableau with a_ii = gamma, stage i solves
    alpha M (U_i - u_ref_i) + R_sp(U_i) = 0,   alpha = 1 / (gamma dt),
    u_ref_i = u^n + sum_{j<i} (a_ij / gamma) (U_j - u_ref_j),
because the converged stage j gives M^-1 R_sp(U_j) = -alpha (U_j - u_ref_j); the
trace and gradient equations (Eq. IEDG a, c) hold at every stage.  The scheme is
stiffly accurate, so u^{n+1} = U_3 (with its q and uhat).
"""
import numpy as np

GAMMA_DIRK = 0.435866521508459


def dirk33():
    """Butcher matrix of Alexander's L-stable, stiffly accurate DIRK(3,3)."""
    g = GAMMA_DIRK
    b1 = -(6 * g * g - 16 * g + 1) / 4
    b2 = (6 * g * g - 20 * g + 5) / 4
    return np.array([[g, 0.0, 0.0],
                     [(1 - g) / 2, g, 0.0],
                     [b1, b2, g]])


def levenberg_marquardt(resid, beta0, h=1e-7, max_iter=12, mu0=1e-3):
    """Minimise |resid(beta)|^2 over beta (a few unknowns) by Levenberg-Marquardt
    with forward-difference gradients (one residual per unknown and iteration).
    resid returns a 1D array-like supporting dot products (numpy or torch).
    Returns (beta, |r(beta)|^2, evaluations)."""
    beta = np.array(beta0, dtype=np.float64)
    s = len(beta)
    r = resid(beta)
    phi = float(_dot(r, r))
    evals = 1
    mu = mu0
    for _ in range(max_iter):
        cols = []
        for j in range(s):
            hj = h * max(1.0, abs(beta[j]))
            bp = beta.copy()
            bp[j] += hj
            cols.append((resid(bp) - r) / hj)
            evals += 1
        JtJ = np.array([[float(_dot(cols[a], cols[b])) for b in range(s)] for a in range(s)])
        Jtr = np.array([float(_dot(cols[a], r)) for a in range(s)])
        improved = False
        for _ in range(8):
            A = JtJ + mu * np.diag(np.maximum(np.diag(JtJ), 1e-300))
            step = np.linalg.solve(A, -Jtr)
            rn = resid(beta + step)
            evals += 1
            phin = float(_dot(rn, rn))
            if phin < phi:
                beta, r, phi = beta + step, rn, phin
                mu = max(mu / 10.0, 1e-12)
                improved = True
                break
            mu *= 10.0
        if not improved or np.abs(step).max() < 1e-12 * max(1.0, np.abs(beta).max()):
            break
    return beta, phi, evals


def _dot(a, b):
    try:
        return (a * b).sum()
    except TypeError:
        return np.dot(a, b)


class Stepper:
    """DIRK(3,3) time stepping of one mesh handle (uniform or mixed orders).  State:
    torch tensors u, q, uhat on the device in the binding's layouts."""

    def __init__(self, mesh, dt, newton_tol=1e-10, max_newton=8, gmres_rtol=1e-12, mr_history=2):
        # the handle's implicit-stage coefficient must be 1 / (gamma dt)
        a = getattr(mesh, "alpha", None)
        if a is not None and abs(a * GAMMA_DIRK * dt - 1.0) > 1e-12:
            raise ValueError("the mesh handle must be created with alpha = 1 / (GAMMA_DIRK dt)")
        self.mesh, self.dt = mesh, dt
        self.A = dirk33()
        self.newton_tol, self.max_newton, self.gmres_rtol = newton_tol, max_newton, gmres_rtol
        self.mr_history = mr_history
        self.history = [[] for _ in range(3)]   # converged (u, q, uhat) per stage, newest first
        self.newton_iters = []
        self.alpha = 1.0 / (GAMMA_DIRK * dt)
        self.rscale = None        # residual size that sets the Newton tolerance (first one met)

    def residual_vector(self, u, q, uh, u_ref):
        import torch
        out = self.mesh.eval_residual(u, uh, q=q, u_ref=u_ref)
        return torch.cat([out["r_q"].reshape(-1), out["r_u"].reshape(-1), out["r_fl"].reshape(-1)])

    def newton(self, u, q, uh, u_ref):
        """Newton on one stage from (u, q, uh); returns the solution and iterations."""
        mesh = self.mesh
        for it in range(self.max_newton + 1):
            r = self.residual_vector(u, q, uh, u_ref)
            nrm = float(r.abs().max())
            if self.rscale is None:
                self.rscale = max(nrm, 1e-300)
            if nrm <= self.newton_tol * self.rscale:
                return u, q, uh, it
            K, R = mesh.assemble_condensed(u, q, uh, u_ref=u_ref)
            dU, _, _ = mesh.trace_solve(K, R, rtol=self.gmres_rtol, max_iter=2000)
            du, dq = mesh.back_substitute(dU)
            u, q, uh = u + du, q + dq, uh + dU
        raise RuntimeError(f"Newton did not converge in {self.max_newton} iterations (|R| = {nrm:.3e})")

    def mr_guess(self, stage, u_ref, fallback):
        """Eq. MinRes2: the initial guess as the combination minimising the residual (LM,
        finite-difference gradients) of the stage's solutions at previous time steps
        and, as the first member (the DIRK adaptation: the paper's scheme combines
        previous time steps), `fallback`, the latest solution of this time step.  LM
        starts from `fallback` alone, so the guess is never worse than it."""
        hist = [fallback] + self.history[stage][:self.mr_history]
        if len(hist) == 1:
            return fallback, None

        def combo(beta):
            u = sum(float(b) * z[0] for b, z in zip(beta, hist))
            q = sum(float(b) * z[1] for b, z in zip(beta, hist))
            uh = sum(float(b) * z[2] for b, z in zip(beta, hist))
            return u, q, uh

        def resid(beta):
            u, q, uh = combo(beta)
            return self.residual_vector(u, q, uh, u_ref)

        beta0 = np.zeros(len(hist))
        beta0[0] = 1.0                                     # start from the last solution
        beta, _, _ = levenberg_marquardt(resid, beta0)
        return combo(beta), beta

    def step(self, u, q, uh, use_mr=True):
        """One time step; returns (u, q, uh) at t + dt and the stage iterations."""
        A, g = self.A, GAMMA_DIRK
        stages = []
        its = []
        cur = (u, q, uh)
        for i in range(3):
            u_ref = u.clone()
            for j in range(i):
                Uj, urj = stages[j][0], stages[j][3]
                u_ref = u_ref + (A[i, j] / g) * (Uj - urj)
            guess = self.mr_guess(i, u_ref, cur)[0] if use_mr else cur
            Ui, qi, uhi, it = self.newton(*guess, u_ref)
            stages.append((Ui, qi, uhi, u_ref))
            its.append(it)
            cur = (Ui, qi, uhi)
            self.history[i].insert(0, (Ui, qi, uhi))
            del self.history[i][self.mr_history:]
        self.newton_iters.append(its)
        return cur[0], cur[1], cur[2], its
