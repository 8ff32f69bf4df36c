"""Isoparametric element geometry for the oracle (test infrastructure only).

Sec. 3.1: the map from the reference element to each physical element is
polynomial of the same degree p as the approximation (p = k), x(xi) = sum_a x_a
phi_a(xi) over the element's nodal coordinates x_a.

For element e and volume point g:  J[i, r] = d x_i / d xi_r,  detJ,  Jinv = J^-1,
physical basis gradients d phi_a / d x_j = sum_r dphi_r[g, a] Jinv[r, j],
weights w = W_g detJ.
For face point (f, gf): the area-scaled outward normal is cof(J) nref W_f with
cof(J) = detJ J^-T; wf = |cof(J) nref| W_f and n = cof(J) nref / |cof(J) nref|.
"""
import numpy as np


class Geometry:
    def __init__(self, ref, node_xyz):
        """ref: RefElement; node_xyz: [E, Np, d]."""
        d = ref.d
        X = np.asarray(node_xyz, dtype=np.float64)
        self.E = X.shape[0]
        # volume points
        J = np.einsum("rga,eai->egir", ref.dphi, X)          # [E, Nq, d, d]
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("element with detJ <= 0")
        Jinv = np.linalg.inv(J)                                # [E, Nq, d(r), d(i)]
        self.detJ = detJ
        self.w = detJ * ref.wq[None, :]                        # [E, Nq]
        self.Jinv = Jinv
        # physical gradients dphi/dx_j at volume points: [E, d(j), Nq, Np]
        self.gphi = np.einsum("rga,egrj->ejga", ref.dphi, Jinv)
        self.xq = np.einsum("ga,eai->egi", ref.phi, X)
        # faces
        nf = 2 * d
        Jf = np.einsum("frga,eai->efgir", ref.fdphi, X)      # [E, nf, Nfq, d, d]
        detf = np.linalg.det(Jf)
        cof = detf[..., None, None] * np.swapaxes(np.linalg.inv(Jf), -1, -2)
        nds = np.einsum("efgij,fj->efgi", cof, ref.nref)     # [E, nf, Nfq, d]
        mag = np.linalg.norm(nds, axis=-1)
        self.wf = mag * ref.fw[None, None, :]                  # [E, nf, Nfq]
        self.nf = nds / mag[..., None]                         # unit normals
        self.xf = np.einsum("fga,eai->efgi", ref.fphi, X)
        # mass matrix M_ab = sum_g w phi_a phi_b
        self.M = np.einsum("eg,ga,gb->eab", self.w, ref.phi, ref.phi)
