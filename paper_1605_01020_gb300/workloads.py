"""Seeded synthetic meshes and flow states shaped like the paper's workloads.

This module generates INPUTS only (mesh coordinates, element-to-trace maps, nodal
states).  It holds none of the method's arithmetic: no basis, quadrature, flux,
residual or Jacobian.  Both the CUDA library's tests and the CPU oracle's tests
draw their inputs from here.

Meshes are structured, periodic, tensor-product (quads in 2D, hexes in 3D).  The
element nodes are placed at the Gauss-Lobatto-Legendre positions of degree p
(here computed with numpy.polynomial, independently of the library and of the
oracle) of the logical cell, then pushed through an optional smooth mapping.
Trace ("high-order face") nodes are the lattice nodes lying on element faces;
periodic faces are identified, so every face is interior.  Trace ids are assigned
in lexicographic order (x fastest) of the global lattice position; an element's
trace slots are its boundary nodes in lexicographic local order.
"""
import itertools
from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial import legendre as npleg

GAMMA = 1.4
DIRK33_A11 = 0.435866521508459      # diagonal coefficient of Alexander's L-stable DIRK(3,3)
DT_STAR = 0.005                      # non-dimensional time step of the paper's runs


def dirk_alpha(dt=DT_STAR, a11=DIRK33_A11):
    return 1.0 / (a11 * dt)


def gll_positions(p):
    """-1, roots of P_p', +1 (node placement only)."""
    if p == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(p + 1)
    c[p] = 1.0
    r = np.sort(np.real(npleg.legroots(npleg.legder(c))))
    return np.concatenate([[-1.0], r, [1.0]])


def _multi(n, d):
    return [tuple(reversed(t)) for t in itertools.product(range(n), repeat=d)]


@dataclass
class Mesh:
    d: int
    p: int
    N: tuple
    node_xyz: np.ndarray        # [E, Np, d]
    elem_trace: np.ndarray      # [E, Nb] int64
    n_trace: int
    bnodes: np.ndarray          # local node index of each trace slot
    extent: tuple = field(default=None)

    @property
    def n_elem(self):
        return self.node_xyz.shape[0]


def structured_mesh(d, N, p, extent=None, mapping=None):
    """Periodic structured mesh with N[r] cells in direction r on [0, extent[r])."""
    N = tuple(int(n) for n in (N if np.ndim(N) else [N] * d))
    extent = tuple(extent) if extent is not None else (1.0,) * d
    assert all(n >= 2 for n in N), "at least two cells per direction"
    xi = gll_positions(p)
    nodes = _multi(p + 1, d)
    cells = _multi(max(N), d)
    cells = [c for c in cells if all(c[r] < N[r] for r in range(d))]
    cells.sort(key=lambda c: tuple(reversed(c)))           # x fastest
    E = len(cells)
    Np = len(nodes)
    X = np.zeros((E, Np, d))
    bnodes = np.array([a for a, ai in enumerate(nodes) if any(t in (0, p) for t in ai)], dtype=np.int64)
    L = [N[r] * p for r in range(d)]                        # lattice size per direction
    lattice = np.zeros((E, len(bnodes), d), dtype=np.int64)
    for e, c in enumerate(cells):
        for a, ai in enumerate(nodes):
            for r in range(d):
                X[e, a, r] = (c[r] + 0.5 * (1.0 + xi[ai[r]])) * extent[r] / N[r]
        for s, a in enumerate(bnodes):
            ai = nodes[a]
            lattice[e, s] = [(c[r] * p + ai[r]) % L[r] for r in range(d)]
    if mapping is not None:
        X = mapping(X)
    # number the face-lattice nodes lexicographically (x fastest)
    strides = np.cumprod([1] + L[:-1])
    key = (lattice * strides).sum(-1)
    uniq, inv = np.unique(key.reshape(-1), return_inverse=True)
    elem_trace = inv.reshape(E, len(bnodes)).astype(np.int64)
    return Mesh(d, p, N, X, elem_trace, len(uniq), bnodes, extent)


def stretched_mapping(seed, ratio=50.0, shear=0.3):
    """Smooth periodic-compatible map: y = eta - (beta / 2pi) sin(2 pi eta) with
    (1 + beta) / (1 - beta) = ratio (boundary-layer-like grading), plus sinusoidal
    shears of x and z.  detJ = 1 - beta cos(2 pi eta) > 0."""
    rng = np.random.default_rng(seed)
    ph1, ph2 = rng.uniform(0, 2 * np.pi, 2)
    beta = (ratio - 1.0) / (ratio + 1.0)

    def mapping(X):
        Y = X.copy()
        xi, eta = X[..., 0], X[..., 1]
        Y[..., 1] = eta - beta / (2 * np.pi) * np.sin(2 * np.pi * eta)
        Y[..., 0] = xi + shear / (2 * np.pi) * np.sin(2 * np.pi * eta + ph1)
        if X.shape[-1] == 3:
            Y[..., 2] = X[..., 2] + shear / (2 * np.pi) * np.sin(2 * np.pi * xi + ph2)
        return Y
    return mapping


# ----------------------------------------------------------------------- states
def conserved_from_primitive(rho, vel, p, gamma=GAMMA):
    d = len(vel)
    ke = 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ke], axis=-1)


def freestream_field(d, Minf, gamma=GAMMA):
    pinf = 1.0 / (gamma * Minf ** 2)

    def f(x):
        one = np.ones(x.shape[:-1])
        vel = [one] + [0.0 * one for _ in range(d - 1)]
        return conserved_from_primitive(one, vel, pinf * one, gamma)
    return f


def fourier_perturbed_field(d, Minf, seed, amp=0.01, kmax=3, gamma=GAMMA):
    """Free stream (rho = 1, v = e_x, p = 1 / (gamma M^2)) plus, per conserved
    variable i, amp * sigma_i * mean_k a_k sin(2 pi k.x + phi_k) over k in [1..kmax]^d."""
    rng = np.random.default_rng(seed)
    base = freestream_field(d, Minf, gamma)
    m = d + 2
    ks = np.array(list(itertools.product(range(1, kmax + 1), repeat=d)), dtype=np.float64)
    a = rng.uniform(0.5, 1.0, (m, len(ks)))
    ph = rng.uniform(0, 2 * np.pi, (m, len(ks)))
    rhoE = base(np.zeros((1, d)))[0, -1]
    sigma = np.ones(m)
    sigma[-1] = rhoE

    def f(x):
        u = base(x)
        arg = 2 * np.pi * np.einsum("...r,kr->...k", x, ks)
        for i in range(m):
            u[..., i] += amp * sigma[i] * np.mean(a[i] * np.sin(arg + ph[i]), axis=-1)
        return u
    return f


def taylor_green_field(M0=0.2, gamma=GAMMA):
    """3D Taylor-Green vortex on x' = 2 pi x (velocity amplitude 1, Mach M0)."""
    p0 = 1.0 / (gamma * M0 ** 2)

    def f(x):
        X, Y, Z = (2 * np.pi * x[..., r] for r in range(3))
        u = np.sin(X) * np.cos(Y) * np.cos(Z)
        v = -np.cos(X) * np.sin(Y) * np.cos(Z)
        w = 0.0 * X
        p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
        rho = p / p0
        return conserved_from_primitive(rho, [u, v, w], p, gamma)
    return f


def broadband_field(Minf, seed, rms=0.05, kmin=1, kmax=8, gamma=GAMMA):
    """Mach-Minf free stream along x plus a solenoidal random Fourier velocity field
    over integer wavevectors 1 <= |k| <= kmax, shell energy ~ |k|^(-5/3), scaled to
    `rms` of U_inf; rho = 1, p = p_inf."""
    rng = np.random.default_rng(seed)
    pinf = 1.0 / (gamma * Minf ** 2)
    ks = [k for k in itertools.product(range(-kmax, kmax + 1), repeat=3)
          if kmin ** 2 <= k[0] ** 2 + k[1] ** 2 + k[2] ** 2 <= kmax ** 2 and k > (0, 0, 0)]
    ks = np.array(ks, dtype=np.float64)
    kn = np.linalg.norm(ks, axis=1)
    # random amplitude direction projected perpendicular to k (solenoidal)
    a = rng.normal(size=(len(ks), 3))
    a -= (np.einsum("kr,kr->k", a, ks) / kn ** 2)[:, None] * ks
    a /= np.linalg.norm(a, axis=1)[:, None]
    shell = np.round(kn).astype(int)
    counts = np.bincount(shell)
    amp = np.sqrt(kn ** (-5.0 / 3.0) / counts[shell])
    ph = rng.uniform(0, 2 * np.pi, len(ks))
    # per-component rms: <|v|^2> = scale^2 sum amp^2 / 2, shared by 3 components
    scale = rms / np.sqrt(np.sum(amp ** 2) / 6.0)

    coef = (np.exp(1j * ph) * amp * scale)[:, None] * a        # complex amplitude of each wave
    kint = ks.astype(np.int64) + kmax

    def velocity(x):
        """sum_k sin(2 pi k.x + phi_k) amp_k scale a_k.  Points on a tensor grid of
        coordinates (structured meshes: few distinct values per direction) are summed
        direction by direction as Im sum_k c_k e^(2 pi i kx x) e^(2 pi i ky y) e^(2 pi i kz z)
        over the grid and gathered; other point sets are summed directly."""
        pts = x.reshape(-1, 3)
        uniq = [np.unique(pts[:, r]) for r in range(3)]
        if np.prod([len(v) for v in uniq]) <= 8 * len(pts):
            nk = 2 * kmax + 1
            C = np.zeros((nk, nk, nk, 3), dtype=np.complex128)
            C[kint[:, 0], kint[:, 1], kint[:, 2]] = coef
            E = [np.exp(2j * np.pi * np.outer(v, np.arange(-kmax, kmax + 1))) for v in uniq]
            G = np.einsum("ia,abcr->ibcr", E[0], C)
            G = np.einsum("jb,ibcr->ijcr", E[1], G)
            G = np.einsum("lc,ijcr->ijlr", E[2], G).imag
            idx = [np.searchsorted(uniq[r], pts[:, r]) for r in range(3)]
            return G[idx[0], idx[1], idx[2]].reshape(x.shape)
        arg = 2 * np.pi * np.einsum("...r,kr->...k", x, ks) + ph
        s = np.sin(arg) * amp * scale
        return np.einsum("...k,kr->...r", s, a)

    def f(x):
        vel = velocity(x)
        one = np.ones(x.shape[:-1])
        return conserved_from_primitive(one, [1.0 + vel[..., 0], vel[..., 1], vel[..., 2]],
                                        pinf * one, gamma)
    return f


def fd_gradient(field, x, h=1e-5):
    """Central-difference gradient of a conserved field at physical points x:
    returns [..., m, d] (input-generation only)."""
    d = x.shape[-1]
    cols = []
    for r in range(d):
        dx = np.zeros(d)
        dx[r] = h
        cols.append((field(x + dx) - field(x - dx)) / (2 * h))
    return np.stack(cols, axis=-1)


@dataclass
class State:
    u: np.ndarray           # [E, Np, m]
    q: np.ndarray           # [E, Np, m, d]
    uhat: np.ndarray        # [n_trace, m]
    u_ref: np.ndarray       # [E, Np, m] or None
    duhat: np.ndarray       # [n_trace, m]  (stand-in trace increment for back-substitution)


def make_state(mesh, field, seed, noise=0.0, uref_shift=0.0, gamma=GAMMA):
    """u = field at the element nodes (+ per-node noise noise * sigma_i * U(-1, 1)),
    q = central-difference gradient of the smooth field at the nodes, uhat = mean of
    u over the element nodes that share each trace node, u_ref = u shifted by a small
    seeded amount (None when uref_shift == 0), duhat = seeded small increment."""
    rng = np.random.default_rng(seed)
    X = mesh.node_xyz
    u = field(X)
    m = u.shape[-1]
    sigma = np.ones(m)
    sigma[-1] = np.abs(u[..., -1]).mean()
    if noise:
        u = u + noise * sigma * rng.uniform(-1.0, 1.0, u.shape)
    q = fd_gradient(field, X)
    acc = np.zeros((mesh.n_trace, m))
    cnt = np.zeros(mesh.n_trace)
    ub = u[:, mesh.bnodes, :]
    np.add.at(acc, mesh.elem_trace.reshape(-1), ub.reshape(-1, m))
    np.add.at(cnt, mesh.elem_trace.reshape(-1), 1.0)
    uhat = acc / cnt[:, None]
    u_ref = None
    if uref_shift:
        u_ref = u + uref_shift * sigma * rng.uniform(-1.0, 1.0, u.shape)
    duhat = 1e-3 * sigma * rng.uniform(-1.0, 1.0, (mesh.n_trace, m))
    return State(u, q, uhat, u_ref, duhat)


# ---------------------------------------------------------------------- configs
@dataclass
class Workload:
    name: str
    mesh: Mesh
    state: State
    params: dict


def config(index, seed=None, N=None):
    """The synthetic workloads (1-based index).  `N` overrides the cell count for
    scaled-down test variants of the same recipe."""
    seed = 1000 + index if seed is None else seed
    alpha = dirk_alpha()
    if index == 1:
        n = N or 8
        mesh = structured_mesh(2, n, 2)
        field = fourier_perturbed_field(2, 0.2, seed)
        st = make_state(mesh, field, seed + 1)
        prm = dict(gamma=GAMMA, Pr=0.72, Re=1.0e3, Minf=0.2, alpha=alpha)
        return Workload(f"2D NS p=2 {n}x{n} periodic quads", mesh, st, prm)
    if index in (2, 3):
        n = N or 16
        mapping = stretched_mapping(seed) if index == 3 else None
        mesh = structured_mesh(3, n, 3, mapping=mapping)
        field = taylor_green_field(0.2)
        st = make_state(mesh, field, seed + 1, noise=0.01)
        prm = dict(gamma=GAMMA, Pr=0.72, Re=2.5e5, Minf=0.2, alpha=alpha)
        tag = " stretched/sheared (aspect 1-50)" if index == 3 else ""
        return Workload(f"3D NS p=3 {n}^3 periodic hexes{tag}", mesh, st, prm)
    if index == 4:
        shape = (N, N, 2 * N) if N else (16, 16, 32)
        orders = mixed_orders(shape, seed, levels=(2, 3, 4), probs=(0.3, 0.5, 0.2))
        mesh = structured_mesh_mixed(3, shape, orders, extent=(1.0, 1.0, 2.0))
        st = make_state_mixed(mesh, taylor_green_field(0.2), seed + 1, noise=0.01)
        prm = dict(gamma=GAMMA, Pr=0.72, Re=2.5e5, Minf=0.2, alpha=alpha)
        E = int(np.prod(shape))
        return Workload(f"3D NS mixed orders p in {{2,3,4}} (0.3/0.5/0.2) {shape[0]}x{shape[1]}x{shape[2]} "
                        f"periodic hexes ({E} elements)", mesh, st, prm)
    if index == 5:
        n = N or 24
        mesh = structured_mesh(3, n, 4)
        field = broadband_field(0.3, seed)
        st = make_state(mesh, field, seed + 1)
        prm = dict(gamma=GAMMA, Pr=0.72, Re=2.5e5, Minf=0.3, alpha=alpha)
        return Workload(f"3D NS p=4 {n}^3 periodic hexes", mesh, st, prm)
    raise ValueError(f"no synthetic workload {index}")


# ------------------------------------------------------------------ mixed orders
@dataclass
class MixedMesh:
    """Structured periodic mesh whose elements have different polynomial orders.

    face_degree[e][f] = 0 for a face shared with an element of the same order (the
    trace there is the continuous one of the uniform case), else the degree of the
    face's private trace nodes, max(p_e, p_neighbour).  An element's trace slots are
    its boundary nodes that lie on at least one same-order face (lexicographic), then
    the private nodes of each other face in face order (-x, +x, -y, +y, -z, +z),
    (q+1)^(d-1) of them, first tangential direction fastest."""
    d: int
    N: tuple
    orders: np.ndarray          # [E]
    node_xyz: list              # per element [Np_e, d]
    elem_trace: list            # per element [Nb_e] int64
    face_degree: np.ndarray     # [E, 2d]
    n_trace: int
    extent: tuple = field(default=None)
    face_kind: np.ndarray = field(default=None)   # [E, 2d] 0 interior, 1 far field, 2 wall (None: all interior)

    @property
    def n_elem(self):
        return len(self.orders)


def structured_mesh_mixed(d, N, orders, extent=None, boundary=None):
    """boundary[r]: 0 = periodic in direction r (default), else the kind of the two
    domain faces normal to r (1 far field, 2 no-slip wall); a domain-boundary face
    carries private trace nodes of the element's own degree."""
    N = tuple(int(n) for n in (N if np.ndim(N) else [N] * d))
    extent = tuple(extent) if extent is not None else (1.0,) * d
    boundary = tuple(boundary) if boundary is not None else (0,) * d
    orders = np.asarray(orders, dtype=np.int64)
    cells = [c for c in _multi(max(N), d) if all(c[r] < N[r] for r in range(d))]
    cells.sort(key=lambda c: tuple(reversed(c)))
    index = {c: i for i, c in enumerate(cells)}
    E = len(cells)
    assert len(orders) == E
    nf = 2 * d
    face_degree = np.zeros((E, nf), dtype=np.int64)
    face_kind = np.zeros((E, nf), dtype=np.int64)
    for e, c in enumerate(cells):
        for f in range(nf):
            r, side = divmod(f, 2)
            nb = list(c)
            nb[r] = nb[r] + (1 if side else -1)
            if boundary[r] and not (0 <= nb[r] < N[r]):
                face_degree[e, f] = orders[e]
                face_kind[e, f] = boundary[r]
                continue
            nb[r] %= N[r]
            pe, pn = orders[e], orders[index[tuple(nb)]]
            face_degree[e, f] = 0 if pe == pn else max(pe, pn)
    node_xyz, keys = [], []
    for e, c in enumerate(cells):
        p = int(orders[e])
        xi = gll_positions(p)
        nodes = _multi(p + 1, d)
        X = np.array([[(c[r] + 0.5 * (1.0 + xi[ai[r]])) * extent[r] / N[r] for r in range(d)] for ai in nodes])
        node_xyz.append(X)
        ek = []
        edg_faces = [f for f in range(nf) if face_degree[e, f] == 0]
        for a, ai in enumerate(nodes):
            on_edg = any(ai[f // 2] == (p if f % 2 else 0) for f in edg_faces)
            if on_edg:
                # lattice position (wrapped in the periodic directions only)
                pos = tuple((c[r] * p + ai[r]) % (N[r] * p) if not boundary[r] else c[r] * p + ai[r]
                            for r in range(d))
                ek.append(("E", p, tuple(reversed(pos))))
        for f in range(nf):
            q = int(face_degree[e, f])
            if q == 0:
                continue
            r, side = divmod(f, 2)
            if face_kind[e, f]:
                # domain boundary: the face belongs to this element alone
                for j in range((q + 1) ** (d - 1)):
                    ek.append(("H", e, nf + f, j))
                continue
            # the face is owned by the cell on its -r side; key = (that cell, r)
            owner = list(c)
            if not side:
                owner[r] = (owner[r] - 1) % N[r]
            okey = index[tuple(owner)]
            for j in range((q + 1) ** (d - 1)):
                ek.append(("H", okey, r, j))
        keys.append(ek)
    allkeys = sorted({k for ek in keys for k in ek}, key=lambda k: (k[0] != "E", k[1:]))
    gid = {k: i for i, k in enumerate(allkeys)}
    elem_trace = [np.array([gid[k] for k in ek], dtype=np.int64) for ek in keys]
    return MixedMesh(d, N, orders, node_xyz, elem_trace, face_degree, len(allkeys), extent,
                     face_kind if face_kind.any() else None)


def make_state_mixed(mesh, field, seed, noise=0.0):
    """State on a MixedMesh (per-element lists): u, q as in make_state, uhat = mean
    over the element slots sharing each trace node of the element's value at the
    slot's position: the field there plus the same per-value noise as u (as in
    make_state, where uhat averages the noisy nodal values), so that no trace value
    sits exactly on a symmetry zero of the field (e.g. rho w = 0 of the Taylor-Green
    field, where |vhat . n| of the Lax-Friedrichs lambda has its kink)."""
    rng = np.random.default_rng(seed)
    m = mesh.d + 2
    us, qs = [], []
    acc = np.zeros((mesh.n_trace, m))
    cnt = np.zeros(mesh.n_trace)
    for e in range(mesh.n_elem):
        X = mesh.node_xyz[e]
        u = field(X)
        if noise:
            sigma = np.ones(m)
            sigma[-1] = np.abs(u[..., -1]).mean()
            u = u + noise * sigma * rng.uniform(-1.0, 1.0, u.shape)
        us.append(u)
        qs.append(fd_gradient(field, X))
        pos = _slot_positions(mesh, e)
        val = field(pos)
        if noise:
            val = val + noise * sigma * rng.uniform(-1.0, 1.0, val.shape)
        np.add.at(acc, mesh.elem_trace[e], val)
        np.add.at(cnt, mesh.elem_trace[e], 1.0)
    uhat = acc / cnt[:, None]
    duhat = 1e-3 * rng.uniform(-1.0, 1.0, (mesh.n_trace, m))
    return State(us, qs, uhat, None, duhat)


def _slot_positions(mesh, e):
    """Physical positions of element e's trace slots (axis-aligned cells only)."""
    d, p = mesh.d, int(mesh.orders[e])
    X = mesh.node_xyz[e]
    lo, hi = X.min(0), X.max(0)
    nodes = _multi(p + 1, d)
    edg_faces = [f for f in range(2 * d) if mesh.face_degree[e, f] == 0]
    out = []
    for a, ai in enumerate(nodes):
        if any(ai[f // 2] == (p if f % 2 else 0) for f in edg_faces):
            out.append(X[a])
    for f in range(2 * d):
        q = int(mesh.face_degree[e, f])
        if q == 0:
            continue
        r, side = divmod(f, 2)
        others = [s for s in range(d) if s != r]
        xi = gll_positions(q)
        for idx in _multi(q + 1, d - 1):
            x = np.zeros(d)
            x[r] = hi[r] if side else lo[r]
            for t, s in enumerate(others):
                x[s] = lo[s] + 0.5 * (1 + xi[idx[t]]) * (hi[s] - lo[s])
            out.append(x)
    return np.array(out)


def mixed_orders(shape, seed, levels=(2, 3, 4), probs=(0.3, 0.5, 0.2)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.array(levels), size=int(np.prod(shape)), p=np.array(probs))
