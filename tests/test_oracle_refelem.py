"""Pins of the oracle's reference element against closed forms and published tables."""
import os

import numpy as np
import pytest

from oracle import refelem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_tables.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        kind, n, x, w = line.split()
        rows.setdefault((kind, int(n)), []).append((float(x), float(w)))
    return rows


def test_quadrature_matches_published_tables():
    for (kind, n), pts in _table().items():
        x, w = (refelem.gauss_legendre(n) if kind == "gauss" else refelem.gauss_lobatto(n - 1))
        xt, wt = np.array(pts).T
        np.testing.assert_allclose(x, xt, atol=1e-15)
        np.testing.assert_allclose(w, wt, atol=1e-15)


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = refelem.gauss_legendre(n)
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # and not beyond: degree 2n is integrated with an error
    assert abs(np.dot(w, x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("p", range(1, 7))
def test_lobatto_nodes_and_exactness(p):
    x, w = refelem.gauss_lobatto(p)
    assert x[0] == -1.0 and x[-1] == 1.0
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    if p > 1:
        c = np.zeros(p + 1)
        c[p] = 1.0
        roots = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)))
        np.testing.assert_allclose(x[1:-1], roots, atol=1e-14)
    for k in range(2 * p):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", range(1, 6))
def test_lagrange_interpolation(p):
    nodes, _ = refelem.gauss_lobatto(p)
    L, dL = refelem.lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(p + 1), atol=1e-14)
    x = np.linspace(-1, 1, 17)
    L, dL = refelem.lagrange(nodes, x)
    np.testing.assert_allclose(L.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dL.sum(1), 0.0, atol=1e-11)
    rng = np.random.default_rng(0)
    c = rng.normal(size=p + 1)                  # random degree-p polynomial
    poly = np.polynomial.Polynomial(c)
    np.testing.assert_allclose(L @ poly(nodes), poly(x), atol=1e-12)
    np.testing.assert_allclose(dL @ poly(nodes), poly.deriv()(x), atol=1e-10)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 2), (3, 3), (3, 4)])
def test_tensor_tables(d, p):
    ref = refelem.RefElement(d, p)
    assert ref.Np == (p + 1) ** d
    assert ref.Nb == (p + 1) ** d - (p - 1) ** d
    np.testing.assert_allclose(ref.phi.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(ref.dphi.sum(2), 0.0, atol=1e-11)
    assert abs(ref.wq.sum() - 2.0 ** d) < 1e-13
    assert abs(ref.fw.sum() - 2.0 ** (d - 1)) < 1e-13
    # face tables are the volume basis evaluated at the face points
    for f in range(2 * d):
        np.testing.assert_allclose(ref.fphi[f].sum(1), 1.0, atol=1e-13)
        off = np.setdiff1d(np.arange(ref.Np), ref.face_nodes[f])
        assert np.all(ref.fphi[f][:, off] == 0.0)
    # a polynomial of degree p per direction is reproduced at the volume points,
    # and its derivative too
    rng = np.random.default_rng(1)
    coef = rng.normal(size=(p + 1,) * d)
    nodes = np.array([[ref.nodes1[t] for t in ai] for ai in ref.node_idx])

    def poly(X):
        out = np.zeros(len(X))
        for idx in np.ndindex(*coef.shape):
            out += coef[idx] * np.prod([X[:, r] ** idx[r] for r in range(d)], axis=0)
        return out

    def dpoly(X, s):
        out = np.zeros(len(X))
        for idx in np.ndindex(*coef.shape):
            if idx[s] == 0:
                continue
            t = coef[idx] * idx[s]
            out += t * np.prod([X[:, r] ** (idx[r] - (1 if r == s else 0)) for r in range(d)], axis=0)
        return out

    np.testing.assert_allclose(ref.phi @ poly(nodes), poly(ref.xq), atol=1e-11)
    for s in range(d):
        np.testing.assert_allclose(ref.dphi[s] @ poly(nodes), dpoly(ref.xq, s), atol=1e-9)
    # the volume rule integrates degree 2 n_q1 - 1 per direction exactly
    k = 2 * ref.nq1 - 1
    mono = np.prod(ref.xq ** (k - 1), axis=1)   # odd-1 = even power per direction
    exact = (2.0 / k) ** d
    assert abs(np.dot(ref.wq, mono) - exact) < 1e-12
