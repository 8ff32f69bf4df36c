"""Block incomplete LU with zero fill-in, BILU(0), of the block compressed-row trace
matrix K (Sec. 2.2.2: m x m blocks, the factors keep the pattern of K), and the
preconditioner solve with its factors.  Test infrastructure only (see oracle/__init__).

Definition, for an elimination order of the trace nodes (a rank per node): L is block
unit lower triangular and U block upper triangular in that order, both with the
pattern of K, such that (L U)_ij = K_ij for every block (i, j) of the pattern.
Computed row by row in the order, for row i and each neighbour k ranked before i in
increasing rank,
    L_ik = A_ik U_kk^-1,   A_ij -= L_ik U_kj  for every j ranked after k that is in
                           the patterns of rows i and k,
where A is row i as updated so far.  The factors are stored in place of K: blocks of
neighbours ranked before i hold L_ik, the others U_ij.

Orders: the natural order of the trace nodes, or the multicolour order (greedy
colouring of the node graph, nodes visited in natural order, each taking the
smallest colour no earlier neighbour has; then nodes sorted by colour, ties by
index).  Nodes of one colour share no block, so the rows of a colour can be factored
and solved together.  (The paper reorders with minimum discarded fill; any order
gives a BILU(0).)
"""
import numpy as np


def _find(row_ptr, col, r, c):
    lo, hi = row_ptr[r], row_ptr[r + 1]
    k = lo + np.searchsorted(col[lo:hi], c)
    return k if (k < hi and col[k] == c) else -1


def greedy_colors(row_ptr, col):
    """Colour of every trace node (see the module docstring)."""
    T = len(row_ptr) - 1
    color = np.full(T, -1, dtype=np.int64)
    for t in range(T):
        used = {int(color[c]) for c in col[row_ptr[t]:row_ptr[t + 1]] if c < t}
        c = 0
        while c in used:
            c += 1
        color[t] = c
    return color


def multicolor_rank(row_ptr, col):
    color = greedy_colors(row_ptr, col)
    order = np.lexsort((np.arange(len(color)), color))
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    return rank, color


def bilu0(row_ptr, col, vals, rank=None):
    """Factors of BILU(0) in the layout of `vals` [nnzb, m, m] for the elimination
    order `rank` (None: natural order)."""
    F = np.array(vals, dtype=np.float64, copy=True)
    T = len(row_ptr) - 1
    rank = np.arange(T) if rank is None else np.asarray(rank)
    for i in sorted(range(T), key=lambda t: rank[t]):
        lo, hi = row_ptr[i], row_ptr[i + 1]
        ents = sorted(range(lo, hi), key=lambda kk: rank[col[kk]])
        for q, kk in enumerate(ents):
            k = col[kk]
            if rank[k] >= rank[i]:
                break
            dk = _find(row_ptr, col, k, k)
            F[kk] = F[kk] @ np.linalg.inv(F[dk])
            for jj in ents[q + 1:]:
                pos = _find(row_ptr, col, k, col[jj])
                if pos >= 0:
                    F[jj] -= F[kk] @ F[pos]
    return F


def bilu0_solve(row_ptr, col, F, r, rank=None):
    """x = U^-1 L^-1 r with the factors of bilu0 (r [T, m])."""
    T = len(row_ptr) - 1
    rank = np.arange(T) if rank is None else np.asarray(rank)
    order = sorted(range(T), key=lambda t: rank[t])
    y = np.array(r, dtype=np.float64, copy=True)
    for i in order:
        for kk in range(row_ptr[i], row_ptr[i + 1]):
            if rank[col[kk]] < rank[i]:
                y[i] -= F[kk] @ y[col[kk]]
    x = np.zeros_like(y)
    for i in reversed(order):
        s = y[i].copy()
        d = -1
        for jj in range(row_ptr[i], row_ptr[i + 1]):
            j = col[jj]
            if j == i:
                d = jj
            elif rank[j] > rank[i]:
                s -= F[jj] @ x[j]
        x[i] = np.linalg.solve(F[d], s)
    return x


def lu_product_on_pattern(row_ptr, col, F, rank=None):
    """(L U)_ij for every block (i, j) of the pattern, from the stored factors."""
    T = len(row_ptr) - 1
    rank = np.arange(T) if rank is None else np.asarray(rank)
    m = F.shape[1]
    out = np.zeros_like(F)
    for i in range(T):
        for jj in range(row_ptr[i], row_ptr[i + 1]):
            j = col[jj]
            s = np.zeros((m, m))
            # sum over k ranked no later than both i and j of L_ik U_kj, L_ii = I
            for kk in range(row_ptr[i], row_ptr[i + 1]):
                k = col[kk]
                if rank[k] > min(rank[i], rank[j]):
                    continue
                pos = _find(row_ptr, col, k, j)
                if pos < 0:
                    continue
                s += (np.eye(m) if k == i else F[kk]) @ F[pos]
            out[jj] = s
    return out
