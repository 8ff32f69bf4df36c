"""Reference element for the oracle (test infrastructure only).

The IEDG spaces Q_h^k, V_h^k, M_h^k of Sec. 2.1 are polynomial spaces of degree k
on each element; the paper defers their construction to its reference [Nguyen:093].
Reading used here (the paper defers the construction): tensor-product Q_k spaces on quads/hexes,
nodal Lagrange basis at the Gauss-Lobatto-Legendre ("high-order") nodes, element
and face integrals by tensor Gauss-Legendre rules with n_q1 = k + quad_extra points
per direction.

Local numbering: node a = i_0 + (p+1) i_1 + (p+1)^2 i_2 (first index fastest),
volume point g likewise over the n_q1 Gauss points.  Face f = 2 r + side is the
face xi_r = -1 (side 0) or +1 (side 1); its points run over the remaining
directions in increasing order, first fastest.
"""
import itertools
import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (Bonnet)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative from (1-x^2) P_n' = n (P_{n-1} - x P_n), valid off x = +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    return p1, dp


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton iteration,
    weights 2 / ((1 - x^2) P_n'(x)^2).  Exact for polynomials of degree 2n-1."""
    i = np.arange(n)
    x = np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        pn, dpn = legendre(n, x)
        dx = pn / dpn
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dpn = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dpn * dpn)
    order = np.argsort(x)
    return x[order], w[order]


def gauss_lobatto(p):
    """p+1 Gauss-Lobatto-Legendre nodes: -1, the roots of P_p', +1, with weights
    2 / (p (p+1) P_p(x)^2).  The interior roots come from Newton's method on
    q(x) = P_p'(x), using the Legendre ODE for q'(x)."""
    if p == 1:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    m = p - 1
    # Chebyshev-Gauss-Lobatto interior points as starting guesses
    x = -np.cos(np.pi * np.arange(1, p) / p)
    for _ in range(100):
        pn, dpn = legendre(p, x)
        # Legendre ODE: (1-x^2) P'' = 2x P' - p(p+1) P
        d2 = (2 * x * dpn - p * (p + 1) * pn) / (1 - x * x)
        dx = dpn / d2
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    assert len(x) == m
    xs = np.concatenate([[-1.0], np.sort(x), [1.0]])
    pn, _ = legendre(p, xs)
    w = 2.0 / (p * (p + 1) * pn * pn)
    return xs, w


def lagrange(nodes, x):
    """Lagrange basis l_j(x) = prod_{k != j} (x - x_k) / (x_j - x_k) and its
    derivative, written as products.  Returns (L, dL), shape [len(x), len(nodes)]."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for j in range(n):
        others = [k for k in range(n) if k != j]
        for k in others:
            L[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
        for mm in others:
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[mm]))
            for k in others:
                if k != mm:
                    term = term * (x - nodes[k]) / (nodes[j] - nodes[k])
            dL[:, j] += term
    return L, dL


class RefElement:
    """Tensor reference element [-1,1]^d of degree p with n_q1 = p + quad_extra
    Gauss points per direction.

    Attributes (all float64):
      phi   [Nq, Np]      basis at volume points
      dphi  [d, Nq, Np]   reference derivatives d/dxi_r at volume points
      wq    [Nq]          volume weights
      xq    [Nq, d]       volume points
      fphi  [2d, Nfq, Np] basis at the face points of each face
      fdphi [2d, d, Nfq, Np]
      fw    [Nfq]         face weights (same for all faces)
      fxq   [2d, Nfq, d]  face points in reference coordinates
      nref  [2d, d]       reference outward normals
      bnodes [Nb]         boundary (trace) nodes in lexicographic order = trace slots
    """

    def __init__(self, d, p, quad_extra=2):
        self.d, self.p = d, p
        self.nq1 = p + quad_extra
        self.np1 = p + 1
        self.Np = (p + 1) ** d
        self.Nq = self.nq1 ** d
        self.Nfq = self.nq1 ** (d - 1)
        self.nodes1, self.lobatto_w = gauss_lobatto(p)
        self.xq1, self.wq1 = gauss_legendre(self.nq1)
        L, dL = lagrange(self.nodes1, self.xq1)           # [nq1, p+1]
        Le, dLe = lagrange(self.nodes1, np.array([-1.0, 1.0]))
        # exact endpoint values: the GLL set contains +-1, so l_j(+-1) is 0 or 1
        Le = np.zeros((2, p + 1))
        Le[0, 0] = 1.0
        Le[1, p] = 1.0

        # multi-indices, first index fastest
        def multi(n, dim):
            return [tuple(reversed(t)) for t in itertools.product(range(n), repeat=dim)]

        self.node_idx = multi(p + 1, d)                     # [Np] tuples
        self.qp_idx = multi(self.nq1, d)
        self.phi = np.ones((self.Nq, self.Np))
        self.dphi = np.ones((d, self.Nq, self.Np))
        for g, gi in enumerate(self.qp_idx):
            for a, ai in enumerate(self.node_idx):
                for r in range(d):
                    self.phi[g, a] *= L[gi[r], ai[r]]
                    for s in range(d):
                        self.dphi[s, g, a] *= (dL if s == r else L)[gi[r], ai[r]]
        self.wq = np.array([np.prod([self.wq1[gi[r]] for r in range(d)]) for gi in self.qp_idx])
        self.xq = np.array([[self.xq1[gi[r]] for r in range(d)] for gi in self.qp_idx])

        nf = 2 * d
        fidx = multi(self.nq1, d - 1) if d > 1 else [()]
        self.fw = np.array([np.prod([self.wq1[t] for t in fi]) for fi in fidx])
        self.fphi = np.ones((nf, self.Nfq, self.Np))
        self.fdphi = np.ones((nf, d, self.Nfq, self.Np))
        self.fxq = np.zeros((nf, self.Nfq, d))
        self.nref = np.zeros((nf, d))
        for f in range(nf):
            r, side = divmod(f, 2)
            self.nref[f, r] = 1.0 if side else -1.0
            others = [s for s in range(d) if s != r]
            for gf, fi in enumerate(fidx):
                xi = np.zeros(d)
                xi[r] = 1.0 if side else -1.0
                for t, s in enumerate(others):
                    xi[s] = self.xq1[fi[t]]
                self.fxq[f, gf] = xi
                for a, ai in enumerate(self.node_idx):
                    for s in range(d):
                        if s == r:
                            v, dv = Le[side, ai[s]], dLe[side, ai[s]]
                        else:
                            k = fi[others.index(s)]
                            v, dv = L[k, ai[s]], dL[k, ai[s]]
                        self.fphi[f, gf, a] *= v
                        for s2 in range(d):
                            self.fdphi[f, s2, gf, a] *= (dv if s2 == s else v)
        self.bnodes = np.array([a for a, ai in enumerate(self.node_idx)
                                if any(t == 0 or t == p for t in ai)], dtype=np.int64)
        self.Nb = len(self.bnodes)
        # face -> its nodes (those with index 0 / p in direction r)
        self.face_nodes = []
        for f in range(nf):
            r, side = divmod(f, 2)
            self.face_nodes.append(np.array([a for a, ai in enumerate(self.node_idx)
                                             if ai[r] == (p if side else 0)], dtype=np.int64))
