"""Pointwise compressible Navier-Stokes physics for the oracle (test infrastructure only).

Sec. 2.1 (Eq. NS and the definitions that follow it): u = (rho, rho v_j, rho E),
q = grad u, flux F(u, q) = inviscid - viscous, with
    tau_ij = (1/Re) (d_j v_i + d_i v_j - 2/3 delta_ij d_k v_k),
    p      = (gamma - 1) rho (E - v_k v_k / 2).
Readings (the paper is silent or garbled there):
  * T is the specific internal energy e = E - v_k v_k / 2 (c_v = 1), so the
    conductivity is gamma / (Re Pr);
  * the heat-flux term is taken with the dissipative sign: the energy flux is
        v_j (rho E + p) - v_i tau_ij - (gamma / (Re Pr)) d_j e .
Numerical flux (Eq. IEDG d): fhat = F(uhat, q) . n + S (u - uhat) with the
Lax-Friedrichs choice S = lambda I, lambda = |vhat . n| + chat evaluated at uhat.

Jacobians are taken by forward-mode dual numbers (class Dual), independent of any
hand-derived formula.
"""
import numpy as np


class Dual:
    """Forward-mode dual number: value v (any shape S) and tangent t (shape S + (n,))."""

    __slots__ = ("v", "t")

    def __init__(self, v, t):
        self.v = np.asarray(v, dtype=np.float64)
        self.t = np.asarray(t, dtype=np.float64)

    @staticmethod
    def const(v, n):
        v = np.asarray(v, dtype=np.float64)
        return Dual(v, np.zeros(v.shape + (n,)))

    def _lift(self, o):
        if isinstance(o, Dual):
            return o
        o = np.asarray(o, dtype=np.float64)
        return Dual(o, np.zeros(o.shape + (self.t.shape[-1],)))

    def __add__(self, o):
        o = self._lift(o)
        return Dual(self.v + o.v, self.t + o.t)

    __radd__ = __add__

    def __sub__(self, o):
        o = self._lift(o)
        return Dual(self.v - o.v, self.t - o.t)

    def __rsub__(self, o):
        return self._lift(o) - self

    def __neg__(self):
        return Dual(-self.v, -self.t)

    def __mul__(self, o):
        o = self._lift(o)
        return Dual(self.v * o.v, self.t * o.v[..., None] + o.t * self.v[..., None])

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = self._lift(o)
        inv = 1.0 / o.v
        return Dual(self.v * inv,
                    (self.t - o.t * (self.v * inv)[..., None]) * inv[..., None])

    def __rtruediv__(self, o):
        return self._lift(o) / self

    def sqrt(self):
        s = np.sqrt(self.v)
        return Dual(s, self.t * (0.5 / s)[..., None])

    def abs(self):
        # d|x|/dx = sign(x), with sign(0) := 0
        return Dual(np.abs(self.v), self.t * np.sign(self.v)[..., None])


def seed(values):
    """Turn a list of k value arrays (same shape) into k Duals with unit tangents."""
    k = len(values)
    out = []
    for i, v in enumerate(values):
        v = np.asarray(v, dtype=np.float64)
        t = np.zeros(v.shape + (k,))
        t[..., i] = 1.0
        out.append(Dual(v, t))
    return out


class Params:
    """stab: 0 = Lax-Friedrichs S = lambda I, 1 = Roe-type S = |A_n(uhat)| (Sec. 2.1)."""

    def __init__(self, gamma=1.4, Pr=0.72, Re=1.0e3, Minf=0.2, alpha=0.0, stab=0):
        self.gamma, self.Pr, self.Re, self.Minf, self.alpha = gamma, Pr, Re, Minf, alpha
        self.stab = stab


def flux(u, q, prm, d):
    """Navier-Stokes flux F[i][j] (list of lists, m x d) for conserved u[i] and
    gradients q[i][j] = d u_i / d x_j (Sec. 2.1).  Works on floats, arrays or Duals."""
    m = d + 2
    g = prm.gamma
    rho = u[0]
    rE = u[m - 1]
    v = [u[1 + i] / rho for i in range(d)]
    E = rE / rho
    vv = v[0] * v[0]
    for i in range(1, d):
        vv = vv + v[i] * v[i]
    e = E - 0.5 * vv
    p = (g - 1.0) * rho * e
    # primitive gradients
    dv = [[(q[1 + i][j] - v[i] * q[0][j]) / rho for j in range(d)] for i in range(d)]
    dE = [(q[m - 1][j] - E * q[0][j]) / rho for j in range(d)]
    de = []
    for j in range(d):
        t = dE[j]
        for k in range(d):
            t = t - v[k] * dv[k][j]
        de.append(t)
    div = dv[0][0]
    for k in range(1, d):
        div = div + dv[k][k]
    inv_re = 1.0 / prm.Re
    tau = [[None] * d for _ in range(d)]
    for i in range(d):
        for j in range(d):
            t = dv[i][j] + dv[j][i]
            if i == j:
                t = t - (2.0 / 3.0) * div
            tau[i][j] = inv_re * t
    kappa = g / (prm.Re * prm.Pr)
    F = [[None] * d for _ in range(m)]
    for j in range(d):
        F[0][j] = u[1 + j]
        for i in range(d):
            t = u[1 + i] * v[j] - tau[i][j]
            if i == j:
                t = t + p
            F[1 + i][j] = t
        t = v[j] * (rE + p) - kappa * de[j]
        for i in range(d):
            t = t - v[i] * tau[i][j]
        F[m - 1][j] = t
    return F


def pressure(u, prm, d):
    m = d + 2
    rho = u[0]
    vv = (u[1] / rho) * (u[1] / rho)
    for i in range(1, d):
        vv = vv + (u[1 + i] / rho) * (u[1 + i] / rho)
    return (prm.gamma - 1.0) * (u[m - 1] - 0.5 * rho * vv)


def lf_lambda(uh, n, prm, d):
    """Lax-Friedrichs coefficient lambda = |vhat . n| + chat, chat^2 = gamma phat / rhohat."""
    rho = uh[0]
    vn = (uh[1] / rho) * n[0]
    for j in range(1, d):
        vn = vn + (uh[1 + j] / rho) * n[j]
    p = pressure(uh, prm, d)
    c = (prm.gamma * p / rho).sqrt() if isinstance(p, Dual) else np.sqrt(prm.gamma * p / rho)
    return (vn.abs() if isinstance(vn, Dual) else np.abs(vn)) + c


def _abs(x):
    return x.abs() if isinstance(x, Dual) else np.abs(x)


def roe_dissipation(uh, du, n, prm, d):
    """|A_n(uhat)| du, A_n = d(F_inv . n)/du the normal Jacobian of the Euler flux at
    uhat (the Roe-type stabilisation tensor of Sec. 2.1).  Written from the
    eigen-decomposition of A_n: eigenvalues v_n - c, v_n (d-fold), v_n + c; the
    acoustic wave strengths of du are a_-+ = (dp -+ c rho dv_n) / (2 c^2) with the
    linearised jumps dp = (gamma-1)(d(rhoE) - v.d(rho v) + |v|^2/2 drho) and
    rho dv_n = n.d(rho v) - v_n drho, eigenvectors r_-+ = (1, v -+ c n, H -+ c v_n),
    and every other wave travels at v_n, so
        |A_n| du = |v_n| du + (|v_n - c| - |v_n|) a_- r_- + (|v_n + c| - |v_n|) a_+ r_+ .
    Works on floats, arrays or Duals (|x|' = sign(x), sign(0) := 0)."""
    rho = uh[0]
    v = [uh[1 + j] / rho for j in range(d)]
    p = pressure(uh, prm, d)
    c2 = prm.gamma * p / rho
    c = c2.sqrt() if isinstance(c2, Dual) else np.sqrt(c2)
    H = (uh[d + 1] + p) / rho
    vn = v[0] * n[0]
    q2 = v[0] * v[0]
    for j in range(1, d):
        vn = vn + v[j] * n[j]
        q2 = q2 + v[j] * v[j]
    vdm = v[0] * du[1]
    ndm = du[1] * n[0]
    for j in range(1, d):
        vdm = vdm + v[j] * du[1 + j]
        ndm = ndm + du[1 + j] * n[j]
    dp = (prm.gamma - 1.0) * (du[d + 1] - vdm + 0.5 * q2 * du[0])
    rdvn = ndm - vn * du[0]
    am = (dp - c * rdvn) / (2.0 * c2)
    ap = (dp + c * rdvn) / (2.0 * c2)
    l0 = _abs(vn)
    wm = (_abs(vn - c) - l0) * am
    wp = (_abs(vn + c) - l0) * ap
    out = [l0 * du[0] + wm + wp]
    for j in range(d):
        out.append(l0 * du[1 + j] + wm * (v[j] - c * n[j]) + wp * (v[j] + c * n[j]))
    out.append(l0 * du[d + 1] + wm * (H - c * vn) + wp * (H + c * vn))
    return out


def normal_jacobian_apply(uh, x, n, prm, d):
    """A_n(uhat) x with A_n = d(F_inv . n)/du the normal Jacobian of the Euler flux at
    uhat, from the differentials of rho v_n, rho v v_n + p n, (rho E + p) v_n:
    dp = (gamma-1)(x_E - v.x_m + |v|^2/2 x_rho), H = (rho E + p)/rho."""
    rho = uh[0]
    v = [uh[1 + j] / rho for j in range(d)]
    p = pressure(uh, prm, d)
    H = (uh[d + 1] + p) / rho
    vn = v[0] * n[0]
    q2 = v[0] * v[0]
    vdm = v[0] * x[1]
    ndm = x[1] * n[0]
    for j in range(1, d):
        vn = vn + v[j] * n[j]
        q2 = q2 + v[j] * v[j]
        vdm = vdm + v[j] * x[1 + j]
        ndm = ndm + x[1 + j] * n[j]
    dp = (prm.gamma - 1.0) * (x[d + 1] - vdm + 0.5 * q2 * x[0])
    out = [ndm]
    for j in range(d):
        out.append(x[1 + j] * vn + v[j] * ndm - v[j] * vn * x[0] + dp * n[j])
    out.append((x[d + 1] + dp) * vn + H * (ndm - vn * x[0]))
    return out


FACE_INTERIOR, FACE_FARFIELD, FACE_WALL = 0, 1, 2


def boundary_flux(uh, u, q, n, prm, d, kind, ub):
    """Boundary flux bhat of the trace equation on a boundary face (Eq. IEDG c).
    Far field (inflow/outflow, Sec. 2.1): bhat = (A_n + |A_n|)/2 (uhat - u)
    + (A_n - |A_n|)/2 (uhat - u_b), A_n and |A_n| at uhat, u_b the given state.
    No-slip adiabatic wall: bhat = (rhohat - rho, rho vhat, fhat_E): the trace density
    follows the interior, the trace velocity vanishes, and the normal energy flux
    (the energy row of the numerical flux, pure heat flux at a no-slip wall) is zero."""
    m = d + 2
    if kind == FACE_FARFIELD:
        a = [uh[i] - u[i] for i in range(m)]
        b = [uh[i] - ub[i] for i in range(m)]
        Aa = normal_jacobian_apply(uh, a, n, prm, d)
        Ab = normal_jacobian_apply(uh, b, n, prm, d)
        Sa = roe_dissipation(uh, a, n, prm, d)
        Sb = roe_dissipation(uh, b, n, prm, d)
        return [0.5 * (Aa[i] + Sa[i]) + 0.5 * (Ab[i] - Sb[i]) for i in range(m)]
    if kind == FACE_WALL:
        fh = numerical_flux(uh, u, q, n, prm, d)
        return [uh[0] - u[0]] + [uh[1 + j] for j in range(d)] + [fh[m - 1]]
    raise ValueError(f"unknown boundary kind {kind}")


def boundary_flux_with_jacobians(uh, u, q, n, prm, d, kind, ub):
    """Face points of one boundary kind: bhat [..., m] and its derivatives in uhat, u
    [..., m, m] and q [..., m, m, d] (dual numbers, like numerical_flux_with_jacobians)."""
    m = d + 2
    shp = u.shape[:-1]
    vals = ([uh[..., i] for i in range(m)] + [u[..., i] for i in range(m)]
            + [q[..., i, j] for i in range(m) for j in range(d)])
    duals = seed(vals)
    uhd = duals[:m]
    ud = duals[m:2 * m]
    qd = [[duals[2 * m + i * d + j] for j in range(d)] for i in range(m)]
    nn = [n[..., j] for j in range(d)]
    ubl = [np.broadcast_to(np.asarray(ub[i], dtype=np.float64), shp) for i in range(m)]
    bh = boundary_flux(uhd, ud, qd, nn, prm, d, kind, ubl)
    b = np.zeros(shp + (m,))
    buh = np.zeros(shp + (m, m))
    bu = np.zeros(shp + (m, m))
    bq = np.zeros(shp + (m, m, d))
    for i in range(m):
        bi = bh[i] if isinstance(bh[i], Dual) else Dual.const(bh[i], 2 * m + m * d)
        b[..., i] = bi.v
        buh[..., i, :] = bi.t[..., :m]
        bu[..., i, :] = bi.t[..., m:2 * m]
        bq[..., i, :, :] = bi.t[..., 2 * m:].reshape(shp + (m, d))
    return b, buh, bu, bq


def numerical_flux(uh, u, q, n, prm, d):
    """fhat_i = F_ij(uhat, q) n_j + S(uhat) (u - uhat)_i  (Eq. IEDG d); S = lambda I
    (Lax-Friedrichs, lambda = |vhat.n| + chat) or |A_n(uhat)| (Roe), by prm.stab."""
    m = d + 2
    F = flux(uh, q, prm, d)
    du = [u[i] - uh[i] for i in range(m)]
    if getattr(prm, "stab", 0) == 1:
        sdu = roe_dissipation(uh, du, n, prm, d)
    else:
        lam = lf_lambda(uh, n, prm, d)
        sdu = [lam * du[i] for i in range(m)]
    out = []
    for i in range(m):
        t = F[i][0] * n[0]
        for j in range(1, d):
            t = t + F[i][j] * n[j]
        out.append(t + sdu[i])
    return out


def flux_with_jacobians(u, q, prm, d):
    """Volume points.  u: [..., m], q: [..., m, d].
    Returns F [..., m, d], dF/du [..., m, d, m], dF/dq [..., m, d, m, d]."""
    m = d + 2
    shp = u.shape[:-1]
    vals = [u[..., i] for i in range(m)] + [q[..., i, j] for i in range(m) for j in range(d)]
    duals = seed(vals)
    ud = duals[:m]
    qd = [[duals[m + i * d + j] for j in range(d)] for i in range(m)]
    F = flux(ud, qd, prm, d)
    Fv = np.zeros(shp + (m, d))
    Fu = np.zeros(shp + (m, d, m))
    Fq = np.zeros(shp + (m, d, m, d))
    for i in range(m):
        for j in range(d):
            Fv[..., i, j] = F[i][j].v
            Fu[..., i, j, :] = F[i][j].t[..., :m]
            Fq[..., i, j, :, :] = F[i][j].t[..., m:].reshape(shp + (m, d))
    return Fv, Fu, Fq


def numerical_flux_with_jacobians(uh, u, q, n, prm, d):
    """Face points.  uh, u: [..., m], q: [..., m, d], n: [..., d] (unit).
    Returns fhat [..., m], d/duhat [..., m, m], d/du [..., m, m], d/dq [..., m, m, d]."""
    m = d + 2
    shp = u.shape[:-1]
    vals = ([uh[..., i] for i in range(m)] + [u[..., i] for i in range(m)]
            + [q[..., i, j] for i in range(m) for j in range(d)])
    duals = seed(vals)
    uhd = duals[:m]
    ud = duals[m:2 * m]
    qd = [[duals[2 * m + i * d + j] for j in range(d)] for i in range(m)]
    nn = [n[..., j] for j in range(d)]
    fh = numerical_flux(uhd, ud, qd, nn, prm, d)
    f = np.zeros(shp + (m,))
    fuh = np.zeros(shp + (m, m))
    fu = np.zeros(shp + (m, m))
    fq = np.zeros(shp + (m, m, d))
    for i in range(m):
        f[..., i] = fh[i].v
        fuh[..., i, :] = fh[i].t[..., :m]
        fu[..., i, :] = fh[i].t[..., m:2 * m]
        fq[..., i, :, :] = fh[i].t[..., 2 * m:].reshape(shp + (m, d))
    return f, fuh, fu, fq
