"""IEDG residuals, Newton blocks, static condensation and trace assembly
(oracle, test infrastructure only).

Weak form (Eq. IEDG a-c), test functions r = phi_a e_(i,j), w = phi_a e_i,
mu = mu_t e_i.  With w = W_g detJ at volume points, wf = W_f |n dS| at face points:

  R_q[a,i,j] =  sum_g w q_ij phi_a + sum_g w u_i dphi_a/dx_j
               - sum_faces sum_gf wf uhat_i n_j phi_a                        (IEDG a)
  R_u[a,i]   =  alpha sum_g w (u - u_ref)_i phi_a - sum_g w F_ij dphi_a/dx_j
               + sum_faces sum_gf wf fhat_i phi_a - sum_g w s_i phi_a         (IEDG b)
  R_fl[t,i]  =  sum_elements sum_faces sum_gf wf fhat_i mu_t                  (IEDG c)

Readings (where the paper leaves a choice open): the DIRK stage (Sec. 2.1) enters
as alpha M (u - u_ref) with alpha = 1 / (a_ii dt); the trace space is continuous
across interior and periodic faces, its basis on a face being the element basis
restricted to that face (trace slot s <-> boundary node bnodes[s]); the source s
is a given function of position (used by the manufactured-solution test only).

Newton system (Sec. 2.2.1): [A B; C D] [dZ; dU] = [F; G] with Z = (q, u),
A = dR_NS/dZ, B = dR_NS/dU, C = dR_FL/dZ, D = dR_FL/dU, F = -R_NS, G = -R_FL.
A is block diagonal over elements, so (Eq. LS)
  K = D - C A^-1 B,   R = G - C A^-1 F,   dZ = A^-1 (F - B dU).
Element unknown ordering used here: q first, index (i d + j) Np + a; then u,
index n_q + i Np + a.  Trace unknowns: i Nb + s.  Outputs are reshaped to
node-major layouts at the end: K_e[s, i, t, k], R_e[s, i], du[a, i], dq[a, i, j].
"""
import numpy as np
import scipy.linalg

from . import physics


class Problem:
    def __init__(self, ref, geo, elem_trace, n_trace, prm, source=None, fmu=None, fkind=None, ub=None):
        """ref: RefElement, geo: Geometry, elem_trace [E, Nb] global trace ids,
        prm: physics.Params, source: optional callable x[..., d] -> s[..., m],
        fmu: trace basis at the face points [nf, Nfq, Nb] shared by the elements
        (default: the element basis restricted to the faces, mu_s = phi_bnodes[s]),
        fkind: [E, nf] face kinds (physics.FACE_*; None = every face interior): on a
        boundary face the trace equation takes the boundary flux bhat (Eq. IEDG c),
        ub: the far-field state u_b [m]."""
        self.ref, self.geo, self.prm = ref, geo, prm
        self.fkind = None if fkind is None else np.asarray(fkind, dtype=np.int64).reshape(geo.E, 2 * ref.d)
        self.ub = None if ub is None else np.asarray(ub, dtype=np.float64)
        self.d = ref.d
        self.m = ref.d + 2
        self.elem_trace = np.asarray(elem_trace, dtype=np.int64)
        self.n_trace = int(n_trace)
        self.fmu = ref.fphi[:, :, ref.bnodes] if fmu is None else np.asarray(fmu)   # [nf, Nfq, Nb]
        self.Nb = self.fmu.shape[2]
        self.source = source

    # ------------------------------------------------------------------ points
    def points(self, els, u, q, uhat):
        """Interpolate the element states to volume and face points."""
        ref = self.ref
        ue, qe = u[els], q[els]
        uh_e = uhat[self.elem_trace[els]]                       # [E, Nb, m]
        P = {}
        P["u"] = np.einsum("ga,eai->egi", ref.phi, ue, optimize=True)
        P["q"] = np.einsum("ga,eaij->egij", ref.phi, qe, optimize=True)
        P["uf"] = np.einsum("fga,eai->efgi", ref.fphi, ue, optimize=True)
        P["qf"] = np.einsum("fga,eaij->efgij", ref.fphi, qe, optimize=True)
        P["uhf"] = np.einsum("fgs,esi->efgi", self.fmu, uh_e, optimize=True)
        return P

    # --------------------------------------------------------------- residual
    def residual(self, u, q, uhat, u_ref=None, els=None):
        """Returns R_q [E, Np, m, d], R_u [E, Np, m], Rhat_e [E, Nb, m] (each element's
        own contribution to R_fl) and R_fl [n_trace, m] (sum over all elements)."""
        ref, geo, prm, d, m = self.ref, self.geo, self.prm, self.d, self.m
        if els is None:
            els = np.arange(geo.E)
        els = np.asarray(els)
        P = self.points(els, u, q, uhat)
        w, gphi = geo.w[els], geo.gphi[els]
        wf, nf = geo.wf[els], geo.nf[els]
        F, _, _ = physics.flux_with_jacobians(P["u"], P["q"], prm, d)
        fh, _, _, _ = physics.numerical_flux_with_jacobians(P["uhf"], P["uf"], P["qf"], nf, prm, d)
        Rq = (np.einsum("eg,egij,ga->eaij", w, P["q"], ref.phi, optimize=True)
              + np.einsum("eg,egi,ejga->eaij", w, P["u"], gphi, optimize=True)
              - np.einsum("efg,efgi,efgj,fga->eaij", wf, P["uhf"], nf, ref.fphi, optimize=True))
        Ru = (-np.einsum("eg,egij,ejga->eai", w, F, gphi, optimize=True)
              + np.einsum("efg,efgi,fga->eai", wf, fh, ref.fphi, optimize=True))
        if prm.alpha != 0.0:
            uref_pts = P["u"] if u_ref is None else np.einsum("ga,eai->egi", ref.phi, u_ref[els], optimize=True)
            Ru = Ru + prm.alpha * np.einsum("eg,egi,ga->eai", w, P["u"] - uref_pts, ref.phi, optimize=True)
        if self.source is not None:
            s = self.source(geo.xq[els])
            Ru = Ru - np.einsum("eg,egi,ga->eai", w, s, ref.phi, optimize=True)
        Rhat_e = np.einsum("efg,efgi,fgs->esi", wf, self._trace_flux(els, P, nf, fh), self.fmu, optimize=True)
        Rfl = np.zeros((self.n_trace, m))
        np.add.at(Rfl, self.elem_trace[els].reshape(-1), Rhat_e.reshape(-1, m))
        return Rq, Ru, Rhat_e, Rfl

    def _trace_flux(self, els, P, nf, fh):
        """The flux of the trace equation: fhat on interior faces, bhat on boundary
        faces (values only)."""
        if self.fkind is None or not (self.fkind[els] != 0).any():
            return fh
        out = fh.copy()
        for kind in (physics.FACE_FARFIELD, physics.FACE_WALL):
            mask = self.fkind[els] == kind
            if mask.any():
                b, _, _, _ = physics.boundary_flux_with_jacobians(
                    P["uhf"][mask], P["uf"][mask], P["qf"][mask], nf[mask], self.prm, self.d, kind, self.ub)
                out[mask] = b
        return out

    def geometric_blocks(self, e):
        """Mass M, B_j[a,b] = sum_g w dphi_a/dx_j phi_b, E_j[a,t] = sum wf n_j phi_a mu_t."""
        ref, geo = self.ref, self.geo
        M = geo.M[e]
        Bj = np.einsum("g,jga,gb->jab", geo.w[e], geo.gphi[e], ref.phi, optimize=True)
        Ej = np.einsum("fg,fgj,fga,fgt->jat", geo.wf[e], geo.nf[e], ref.fphi, self.fmu, optimize=True)
        return M, Bj, Ej

    def solve_q(self, u, uhat):
        """q with R_q = 0 on every element: q_ij = M^-1 (E_j uhat_i - B_j u_i)."""
        E, Np, m, d = self.geo.E, self.ref.Np, self.m, self.d
        q = np.zeros((E, Np, m, d))
        for e in range(E):
            M, Bj, Ej = self.geometric_blocks(e)
            uh_e = uhat[self.elem_trace[e]]
            for j in range(d):
                q[e, :, :, j] = np.linalg.solve(M, Ej[j] @ uh_e - Bj[j] @ u[e])
        return q

    # ------------------------------------------------------------ Newton blocks
    def element_blocks(self, e, u, q, uhat, u_ref=None):
        """Dense Newton blocks of element e in the ordering of the module docstring.
        Returns dict with A_qq, A_qu, B_q, A_uq, A_uu, B_u, C_q, C_u, D, F_q, F_u, G."""
        ref, geo, prm, d, m = self.ref, self.geo, self.prm, self.d, self.m
        Np, Nb = ref.Np, self.Nb
        els = np.array([e])
        P = self.points(els, u, q, uhat)
        _, Fu, Fq = physics.flux_with_jacobians(P["u"][0], P["q"][0], prm, d)
        _, fuh, fu, fq = physics.numerical_flux_with_jacobians(
            P["uhf"][0], P["uf"][0], P["qf"][0], geo.nf[e], prm, d)
        w, gphi, wf = geo.w[e], geo.gphi[e], geo.wf[e]
        phi, fphi, fmu = ref.phi, ref.fphi, self.fmu
        M, Bj, Ej = self.geometric_blocks(e)
        I_m = np.eye(m)
        I_d = np.eye(d)
        blk = {}
        # q-equation rows (IEDG a): linear, geometry only
        blk["A_qq"] = np.einsum("ik,jl,ab->ijaklb", I_m, I_d, M, optimize=True).reshape(m * d * Np, m * d * Np)
        blk["A_qu"] = np.einsum("ik,jab->ijakb", I_m, Bj, optimize=True).reshape(m * d * Np, m * Np)
        blk["B_q"] = -np.einsum("ik,jat->ijakt", I_m, Ej, optimize=True).reshape(m * d * Np, m * Nb)
        # u-equation rows (IEDG b)
        A_uq = (-np.einsum("g,jga,gijkl,gb->iaklb", w, gphi, Fq, phi, optimize=True)
                + np.einsum("fg,fga,fgikl,fgb->iaklb", wf, fphi, fq, fphi, optimize=True))
        A_uu = (-np.einsum("g,jga,gijk,gb->iakb", w, gphi, Fu, phi, optimize=True)
                + np.einsum("fg,fga,fgik,fgb->iakb", wf, fphi, fu, fphi, optimize=True))
        A_uu = A_uu + prm.alpha * np.einsum("ik,ab->iakb", I_m, M, optimize=True)
        blk["A_uq"] = A_uq.reshape(m * Np, m * d * Np)
        blk["A_uu"] = A_uu.reshape(m * Np, m * Np)
        blk["B_u"] = np.einsum("fg,fga,fgik,fgt->iakt", wf, fphi, fuh, fmu, optimize=True).reshape(m * Np, m * Nb)
        # trace rows (IEDG c): bhat and its derivatives on boundary faces
        if self.fkind is not None and (self.fkind[e] != 0).any():
            fuh, fu, fq = fuh.copy(), fu.copy(), fq.copy()
            for f in range(2 * d):
                kind = int(self.fkind[e, f])
                if kind == physics.FACE_INTERIOR:
                    continue
                _, buh, bu, bq = physics.boundary_flux_with_jacobians(
                    P["uhf"][0, f], P["uf"][0, f], P["qf"][0, f], geo.nf[e][f], prm, d, kind, self.ub)
                fuh[f], fu[f], fq[f] = buh, bu, bq
        blk["C_q"] = np.einsum("fg,fgs,fgikl,fgb->isklb", wf, fmu, fq, fphi, optimize=True).reshape(m * Nb, m * d * Np)
        blk["C_u"] = np.einsum("fg,fgs,fgik,fgb->iskb", wf, fmu, fu, fphi, optimize=True).reshape(m * Nb, m * Np)
        blk["D"] = np.einsum("fg,fgs,fgik,fgt->iskt", wf, fmu, fuh, fmu, optimize=True).reshape(m * Nb, m * Nb)
        Rq, Ru, Rhat_e, _ = self.residual(u, q, uhat, u_ref, els=els)
        blk["F_q"] = -np.transpose(Rq[0], (1, 2, 0)).reshape(-1)        # (i, j, a)
        blk["F_u"] = -np.transpose(Ru[0], (1, 0)).reshape(-1)         # (i, a)
        blk["G"] = -np.transpose(Rhat_e[0], (1, 0)).reshape(-1)          # (i, s)
        blk["M"], blk["Bj"], blk["Ej"] = M, Bj, Ej
        return blk

    def full_system(self, blk):
        A = np.block([[blk["A_qq"], blk["A_qu"]], [blk["A_uq"], blk["A_uu"]]])
        B = np.vstack([blk["B_q"], blk["B_u"]])
        C = np.hstack([blk["C_q"], blk["C_u"]])
        F = np.concatenate([blk["F_q"], blk["F_u"]])
        return A, B, C, blk["D"], F, blk["G"]

    def _to_node_major(self, Kc, Rc):
        m, Nb = self.m, self.Nb
        K = Kc.reshape(m, Nb, m, Nb).transpose(1, 0, 3, 2)   # [s, i, t, k]
        R = Rc.reshape(m, Nb).T                               # [s, i]
        return K, R

    # -------------------------------------------------------------- condensation
    def condense_full(self, e, u, q, uhat, u_ref=None):
        """Definition: K_e = D - C A^-1 B, R_e = G - C A^-1 F with the dense element
        block A factored by LU with partial pivoting (LAPACK getrf: largest |a|,
        first index on ties)."""
        blk = self.element_blocks(e, u, q, uhat, u_ref)
        A, B, C, D, F, G = self.full_system(blk)
        lu = scipy.linalg.lu_factor(A)
        X = scipy.linalg.lu_solve(lu, np.column_stack([B, F]))
        K = D - C @ X[:, :-1]
        R = G - C @ X[:, -1]
        return self._to_node_major(K, R)

    def qelim(self, blk):
        """Exact elimination of q (A_qq = M (x) I): dq_kl = M^-1 F_q,kl - G_l du_k + H_l dU_k
        with G_l = M^-1 B_l, H_l = M^-1 E_l.  Returns At, Bt, Ct, Dt, Ft, Gt."""
        m, d = self.m, self.d
        Np, Nb = self.ref.Np, self.Nb
        M = blk["M"]
        Gl = np.stack([np.linalg.solve(M, blk["Bj"][j]) for j in range(d)])    # [d, Np, Np]
        Hl = np.stack([np.linalg.solve(M, blk["Ej"][j]) for j in range(d)])    # [d, Np, Nb]
        Fq = blk["F_q"].reshape(m, d, Np)
        MFq = np.stack([[np.linalg.solve(M, Fq[k, l]) for l in range(d)] for k in range(m)])
        A_uq = blk["A_uq"].reshape(m * Np, m, d, Np)
        C_q = blk["C_q"].reshape(m * Nb, m, d, Np)
        At = blk["A_uu"] - np.einsum("rklc,lcb->rkb", A_uq, Gl, optimize=True).reshape(m * Np, m * Np)
        Bt = blk["B_u"] + np.einsum("rklc,lct->rkt", A_uq, Hl, optimize=True).reshape(m * Np, m * Nb)
        Ft = blk["F_u"] - np.einsum("rklc,klc->r", A_uq, MFq, optimize=True)
        Ct = blk["C_u"] - np.einsum("rklc,lcb->rkb", C_q, Gl, optimize=True).reshape(m * Nb, m * Np)
        Dt = blk["D"] + np.einsum("rklc,lct->rkt", C_q, Hl, optimize=True).reshape(m * Nb, m * Nb)
        Gt = blk["G"] - np.einsum("rklc,klc->r", C_q, MFq, optimize=True)
        return At, Bt, Ct, Dt, Ft, Gt, Gl, Hl, MFq

    def condense_qelim(self, e, u, q, uhat, u_ref=None):
        """Same K_e, R_e through the q-eliminated element system:
        K_e = Dt - Ct At^-1 Bt, R_e = Gt - Ct At^-1 Ft."""
        blk = self.element_blocks(e, u, q, uhat, u_ref)
        At, Bt, Ct, Dt, Ft, Gt = self.qelim(blk)[:6]
        lu = scipy.linalg.lu_factor(At)
        X = scipy.linalg.lu_solve(lu, np.column_stack([Bt, Ft]))
        K = Dt - Ct @ X[:, :-1]
        R = Gt - Ct @ X[:, -1]
        return self._to_node_major(K, R)

    # ------------------------------------------------------------ back-substitution
    def back_substitute_full(self, e, u, q, uhat, duhat, u_ref=None):
        """dZ_e = A^-1 (F - B dU_e).  Returns du [Np, m], dq [Np, m, d]."""
        m, d, Np = self.m, self.d, self.ref.Np
        blk = self.element_blocks(e, u, q, uhat, u_ref)
        A, B, C, D, F, G = self.full_system(blk)
        dU = duhat[self.elem_trace[e]].T.reshape(-1)          # (i, s)
        dZ = np.linalg.solve(A, F - B @ dU)
        nq = m * d * Np
        dq = dZ[:nq].reshape(m, d, Np).transpose(2, 0, 1)
        du = dZ[nq:].reshape(m, Np).T
        return du, dq

    def back_substitute_qelim(self, e, u, q, uhat, duhat, u_ref=None):
        m, d, Np = self.m, self.d, self.ref.Np
        blk = self.element_blocks(e, u, q, uhat, u_ref)
        At, Bt, Ct, Dt, Ft, Gt, Gl, Hl, MFq = self.qelim(blk)
        dU = duhat[self.elem_trace[e]]                         # [Nb, m]
        du = np.linalg.solve(At, Ft - Bt @ dU.T.reshape(-1)).reshape(m, Np)   # [k, b]
        dq = np.zeros((Np, m, d))
        for k in range(m):
            for l in range(d):
                dq[:, k, l] = MFq[k, l] - Gl[l] @ du[k] + Hl[l] @ dU[:, k]
        return du.T, dq


# ------------------------------------------------------------------ trace matrix
def bsr_pattern(elem_trace, n_trace):
    """Block compressed rows of K (Sec. 2.2.2): one block row per trace node, a block
    (r, c) for every pair of trace nodes that share an element, columns sorted."""
    et = np.asarray(elem_trace, dtype=np.int64)
    rows = np.repeat(et, et.shape[1], axis=1).reshape(-1)
    cols = np.tile(et, (1, et.shape[1])).reshape(-1)
    key = np.unique(rows * n_trace + cols)
    r = key // n_trace
    c = key % n_trace
    row_ptr = np.zeros(n_trace + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, c.astype(np.int64)


def bsr_find(row_ptr, col, r, c):
    lo, hi = row_ptr[r], row_ptr[r + 1]
    k = lo + np.searchsorted(col[lo:hi], c)
    assert col[k] == c
    return k


def assemble(elem_trace, n_trace, K_e, R_e, els=None):
    """K = sum_e P_e^T K_e P_e, R = sum_e P_e^T R_e, summed in element order.
    K_e [E, Nb, m, Nb, m] (s, i, t, k); returns values [nnzb, m, m] and R [n_trace, m]."""
    et = np.asarray(elem_trace, dtype=np.int64)
    row_ptr, col = bsr_pattern(et, n_trace)
    m = K_e.shape[2]
    vals = np.zeros((len(col), m, m))
    R = np.zeros((n_trace, m))
    els = range(len(K_e)) if els is None else els
    for n, e in enumerate(els):
        tr = et[e]
        for s in range(len(tr)):
            R[tr[s]] += R_e[n][s]
            for t in range(len(tr)):
                vals[bsr_find(row_ptr, col, tr[s], tr[t])] += K_e[n][s, :, t, :]
    return row_ptr, col, vals, R


# ------------------------------------------------------------------ mixed orders
def face_trace_basis(ref, face_degree):
    """Trace basis of one element at its face points, [nf, Nfq, Nb_e], for the
    mixed-order reading: on a face shared with an element of the same order
    (face_degree 0) the trace is the continuous one, mu_s = phi_a restricted to the
    face for the element's boundary nodes a on such faces; a face shared with an
    element of another order q carries (q+1)^(d-1) private nodes at the Gauss-Lobatto
    points of degree q in the face's tangential coordinates (first fastest), with
    the degree-q Lagrange basis, and every other slot vanishes on it.  Slots: the
    boundary nodes on same-order faces (lexicographic), then each private face in
    face order."""
    from . import refelem as re
    d, nf = ref.d, 2 * ref.d
    edg = [f for f in range(nf) if face_degree[f] == 0]
    nodes = [a for a, ai in enumerate(ref.node_idx)
             if any(ai[f // 2] == (ref.p if f % 2 else 0) for f in edg)]
    cols = []
    for a in nodes:
        c = np.zeros((nf, ref.Nfq))
        for f in edg:
            c[f] = ref.fphi[f][:, a]
        cols.append(c)
    for f in range(nf):
        q = int(face_degree[f])
        if q == 0:
            continue
        r = f // 2
        others = [s for s in range(d) if s != r]
        gl, _ = re.gauss_lobatto(q)
        Ls = [re.lagrange(gl, ref.fxq[f][:, s])[0] for s in others]     # [Nfq, q+1] each
        idx = [tuple(reversed(t)) for t in np.ndindex(*([q + 1] * (d - 1)))]
        for j in idx:
            c = np.zeros((nf, ref.Nfq))
            v = np.ones(ref.Nfq)
            for t in range(d - 1):
                v = v * Ls[t][:, j[t]]
            c[f] = v
            cols.append(c)
    return np.stack(cols, axis=-1)


class MixedProblem:
    """Elements of different orders sharing one trace space (see face_trace_basis);
    each element is an independent single-element Problem with its own reference
    element, geometry and trace basis."""

    def __init__(self, refs, mesh, prm, source=None, ub=None):
        """refs: {p: RefElement}; mesh: workloads.MixedMesh (face_kind None: every face
        interior); prm: physics.Params; ub: far-field state for far-field faces."""
        from .geometry import Geometry
        self.mesh, self.prm = mesh, prm
        self.m = mesh.d + 2
        self.n_trace = mesh.n_trace
        self.pbs = []
        for e in range(mesh.n_elem):
            ref = refs[int(mesh.orders[e])]
            geo = Geometry(ref, mesh.node_xyz[e][None])
            fmu = face_trace_basis(ref, mesh.face_degree[e])
            fk = None if getattr(mesh, "face_kind", None) is None else mesh.face_kind[e][None]
            self.pbs.append(Problem(ref, geo, mesh.elem_trace[e][None], mesh.n_trace, prm, source, fmu, fk, ub))

    def residual(self, u, q, uhat, u_ref=None):
        """Per-element lists R_q, R_u, Rhat_e and the assembled R_fl."""
        Rq, Ru, Rh = [], [], []
        Rfl = np.zeros((self.n_trace, self.m))
        for e, pb in enumerate(self.pbs):
            ur = None if u_ref is None else u_ref[e][None]
            a, b, c, f = pb.residual(u[e][None], q[e][None], uhat, ur)
            Rq.append(a[0]); Ru.append(b[0]); Rh.append(c[0])
            Rfl += f
        return Rq, Ru, Rh, Rfl

    def solve_q(self, u, uhat):
        return [pb.solve_q(u[e][None], uhat)[0] for e, pb in enumerate(self.pbs)]

    def condense_qelim(self, e, u, q, uhat, u_ref=None):
        ur = None if u_ref is None else u_ref[e][None]
        return self.pbs[e].condense_qelim(0, u[e][None], q[e][None], uhat, ur)

    def condense_full(self, e, u, q, uhat, u_ref=None):
        ur = None if u_ref is None else u_ref[e][None]
        return self.pbs[e].condense_full(0, u[e][None], q[e][None], uhat, ur)

    def back_substitute_qelim(self, e, u, q, uhat, duhat, u_ref=None):
        ur = None if u_ref is None else u_ref[e][None]
        return self.pbs[e].back_substitute_qelim(0, u[e][None], q[e][None], uhat, duhat, ur)

    def element_blocks(self, e, u, q, uhat, u_ref=None):
        ur = None if u_ref is None else u_ref[e][None]
        return self.pbs[e].element_blocks(0, u[e][None], q[e][None], uhat, ur)


def assemble_ragged(elem_trace, n_trace, K_e, R_e):
    """K = sum_e P_e^T K_e P_e, R = sum_e P_e^T R_e for elements with different slot
    counts (lists), summed in element order; returns row_ptr, col, values, R."""
    pairs = set()
    for tr in elem_trace:
        for a in tr.tolist():
            for b in tr.tolist():
                pairs.add((a, b))
    keys = np.array(sorted(r * n_trace + c for r, c in pairs), dtype=np.int64)
    r_, c_ = keys // n_trace, keys % n_trace
    row_ptr = np.zeros(n_trace + 1, dtype=np.int64)
    np.add.at(row_ptr, r_ + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    col = c_.astype(np.int64)
    m = R_e[0].shape[1]
    vals = np.zeros((len(col), m, m))
    R = np.zeros((n_trace, m))
    for e, tr in enumerate(elem_trace):
        for s in range(len(tr)):
            R[tr[s]] += R_e[e][s]
            for t in range(len(tr)):
                vals[bsr_find(row_ptr, col, tr[s], tr[t])] += K_e[e][s, :, t, :]
    return row_ptr, col, vals, R
