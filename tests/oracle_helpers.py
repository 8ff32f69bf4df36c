"""Glue between the synthetic workloads and the oracle (tests only)."""
import numpy as np

from oracle import geometry, iedg, physics, refelem

_REF = {}


def ref_element(d, p, quad_extra=2):
    key = (d, p, quad_extra)
    if key not in _REF:
        _REF[key] = refelem.RefElement(d, p, quad_extra)
    return _REF[key]


def problem(mesh, params, quad_extra=2, source=None):
    ref = ref_element(mesh.d, mesh.p, quad_extra)
    assert np.array_equal(ref.bnodes, mesh.bnodes)
    geo = geometry.Geometry(ref, mesh.node_xyz)
    prm = physics.Params(**{k: params[k] for k in ("gamma", "Pr", "Re", "Minf", "alpha")},
                         stab=params.get("stab", 0))
    return iedg.Problem(ref, geo, mesh.elem_trace, mesh.n_trace, prm, source)


def global_dense_system(pb, u, q, uhat, u_ref=None):
    """Uncondensed global Newton matrix [A B; C D] and right-hand side [F; G] for a
    tiny mesh, unknowns ordered element by element then trace (i-major per node)."""
    E, m = pb.geo.E, pb.m
    blks = [pb.element_blocks(e, u, q, uhat, u_ref) for e in range(E)]
    nz = blks[0]["A_qq"].shape[0] + blks[0]["A_uu"].shape[0]
    nt = pb.n_trace * m
    n = E * nz + nt
    J = np.zeros((n, n))
    rhs = np.zeros(n)
    Nb = pb.ref.Nb
    for e, blk in enumerate(blks):
        A, B, C, D, F, G = pb.full_system(blk)
        z = slice(e * nz, (e + 1) * nz)
        # trace columns of element e: local (i, s) -> global trace t*m + i
        tr = pb.elem_trace[e]
        gidx = np.array([E * nz + tr[s] * m + i for i in range(m) for s in range(Nb)])
        J[z, z] = A
        J[z, gidx] += B
        for r, gr in enumerate(gidx):
            J[gr, z] += C[r]
            J[gr, gidx] += D[r]
            rhs[gr] += G[r]
        rhs[z] = F
    return J, rhs, nz
