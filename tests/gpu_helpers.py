"""Shared pieces of the GPU parity tests: building/loading the CUDA library,
moving workload arrays to the device, oracle reference values and the error
norms the tolerances are stated in."""
import numpy as np

from oracle import iedg as oiedg


def lib_mesh(wl):
    from paper_1605_01020_gb300 import iedg
    return iedg.mesh_from_workload(wl)


def dev(x):
    import torch
    return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_err(x, ref, floor=0.0):
    """max |x - ref| / max(max |ref|, floor) (the norm of the tolerances).  `floor`
    is the size of the per-element terms an assembled output is summed from, for
    outputs that cancel to round-off (e.g. R_FL of a continuous state)."""
    x, ref = np.asarray(x), np.asarray(ref)
    scale = max(np.abs(ref).max(), floor)
    return np.abs(x - ref).max() / (scale if scale > 0 else 1.0)


def bsr_row_err(row_ptr, vals, ref_vals, rows):
    """Per block row: max |K - K_o| / max |K_o| over the row, worst over `rows`."""
    worst = 0.0
    for r in rows:
        a, b = row_ptr[r], row_ptr[r + 1]
        s = np.abs(ref_vals[a:b]).max()
        worst = max(worst, np.abs(vals[a:b] - ref_vals[a:b]).max() / s)
    return worst


def oracle_K_rows(pb, mesh, st, rows, u_ref=None, kfun=None):
    """Oracle BSR values restricted to the block rows `rows` (sums over the elements
    touching each row, in element order), plus R on those rows.  kfun(e), if given,
    replaces the element's condensed block K_e."""
    row_ptr, col = oiedg.bsr_pattern(mesh.elem_trace, mesh.n_trace)
    m = pb.m
    vals = np.zeros((len(col), m, m))
    R = np.zeros((mesh.n_trace, m))
    rows = set(int(r) for r in rows)
    els = sorted({e for e in range(mesh.n_elem) if rows & set(mesh.elem_trace[e].tolist())})
    re_max = 0.0
    for e in els:
        Ke, Re = pb.condense_qelim(e, st.u, st.q, st.uhat, u_ref)
        if kfun is not None:
            Ke = kfun(e)
        re_max = max(re_max, np.abs(Re).max())
        tr = mesh.elem_trace[e]
        for s in range(len(tr)):
            if int(tr[s]) not in rows:
                continue
            R[tr[s]] += Re[s]
            for t in range(len(tr)):
                vals[oiedg.bsr_find(row_ptr, col, tr[s], tr[t])] += Ke[s, :, t, :]
    return row_ptr, col, vals, R, els, re_max


def fro_ratio(row_ptr, vals, ref_vals, exact_vals, rows):
    """||K - K_ref||_F / ||K_ref - K_exact||_F over the block rows `rows`: how far the
    device result is from the rounded-operand oracle, against the rounding's own size."""
    num = den = 0.0
    for r in rows:
        sl = slice(row_ptr[r], row_ptr[r + 1])
        num += float(((vals[sl] - ref_vals[sl]) ** 2).sum())
        den += float(((ref_vals[sl] - exact_vals[sl]) ** 2).sum())
    return (num / den) ** 0.5 if den > 0 else float("inf")
