"""Pins of the oracle's BILU(0) (Sec. 2.2.2, block ILU with zero fill-in and m x m
blocks): its defining property (L U = K on the pattern), exactness when the pattern
is closed under elimination, and the solve inverting L U exactly."""
import numpy as np
import pytest

from oracle import bilu
from oracle import iedg as oiedg
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import problem


def _dense(row_ptr, col, blocks):
    T = len(row_ptr) - 1
    m = blocks.shape[1]
    D = np.zeros((T * m, T * m))
    for r in range(T):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            D[r * m:(r + 1) * m, col[k] * m:(col[k] + 1) * m] = blocks[k]
    return D


def _condensed_K(N=4):
    wl = W.config(1, N=N)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    E = wl.mesh.n_elem
    Ke, Re = zip(*[pb.condense_qelim(e, st.u, st.q, st.uhat) for e in range(E)])
    row_ptr, col, vals, R = oiedg.assemble(wl.mesh.elem_trace, wl.mesh.n_trace, np.array(Ke), np.array(Re))
    return row_ptr, col, vals, R


def test_lu_product_equals_K_on_the_pattern():
    row_ptr, col, vals, _ = _condensed_K()
    F = bilu.bilu0(row_ptr, col, vals)
    P = bilu.lu_product_on_pattern(row_ptr, col, F)
    assert np.abs(P - vals).max() <= 1e-12 * np.abs(vals).max()
    # and it is not the exact factorisation: fill-in was dropped somewhere
    D = _dense(row_ptr, col, vals)
    x = np.random.default_rng(0).standard_normal(D.shape[0])
    y = bilu.bilu0_solve(row_ptr, col, F, (D @ x).reshape(-1, vals.shape[1])).reshape(-1)
    assert np.abs(y - x).max() > 1e-8


def test_exact_lu_when_the_pattern_is_closed():
    """Block tridiagonal pattern: elimination creates no fill, so BILU(0) is the block
    LU without pivoting and the preconditioner solve is the exact solve."""
    rng = np.random.default_rng(1)
    T, m = 9, 5
    rows, cols = [], []
    for i in range(T):
        for j in (i - 1, i, i + 1):
            if 0 <= j < T:
                rows.append(i)
                cols.append(j)
    row_ptr = np.zeros(T + 1, dtype=np.int64)
    np.add.at(row_ptr, np.array(rows) + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    col = np.array(cols, dtype=np.int64)
    vals = rng.standard_normal((len(col), m, m))
    for i in range(T):
        vals[oiedg.bsr_find(row_ptr, col, i, i)] += 8.0 * np.eye(m)
    F = bilu.bilu0(row_ptr, col, vals)
    b = rng.standard_normal((T, m))
    x = bilu.bilu0_solve(row_ptr, col, F, b)
    ref = np.linalg.solve(_dense(row_ptr, col, vals), b.reshape(-1)).reshape(T, m)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_solve_inverts_L_times_U():
    row_ptr, col, vals, _ = _condensed_K(N=3)
    F = bilu.bilu0(row_ptr, col, vals)
    T, m = len(row_ptr) - 1, vals.shape[1]
    Lb = np.zeros_like(F)
    Ub = np.zeros_like(F)
    for i in range(T):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            if col[k] < i:
                Lb[k] = F[k]
            else:
                Ub[k] = F[k]
                if col[k] == i:
                    Lb[k] = np.eye(m)
    LU = _dense(row_ptr, col, Lb) @ _dense(row_ptr, col, Ub)
    x = np.random.default_rng(2).standard_normal((T, m))
    y = bilu.bilu0_solve(row_ptr, col, F, (LU @ x.reshape(-1)).reshape(T, m))
    assert np.abs(y - x).max() <= 1e-10 * np.abs(x).max()


def test_multicolor_order_is_a_colouring_and_bilu_holds():
    """Greedy colouring: adjacent trace nodes (sharing a block) never share a colour, so
    every row's earlier-ranked neighbours have smaller colours; BILU(0) in that order
    keeps L U = K on the pattern and its solve inverts L U."""
    row_ptr, col, vals, _ = _condensed_K(N=4)
    rank, color = bilu.multicolor_rank(row_ptr, col)
    T, m = len(row_ptr) - 1, vals.shape[1]
    for i in range(T):
        nb = col[row_ptr[i]:row_ptr[i + 1]]
        nb = nb[nb != i]
        assert (color[nb] != color[i]).all()
        assert ((rank[nb] < rank[i]) == (color[nb] < color[i])).all()
    assert color.max() + 1 < T // 3          # far fewer colours than nodes
    F = bilu.bilu0(row_ptr, col, vals, rank)
    P = bilu.lu_product_on_pattern(row_ptr, col, F, rank)
    assert np.abs(P - vals).max() <= 1e-12 * np.abs(vals).max()
    Lb = np.zeros_like(F)
    Ub = np.zeros_like(F)
    for i in range(T):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            if rank[col[k]] < rank[i]:
                Lb[k] = F[k]
            else:
                Ub[k] = F[k]
                if col[k] == i:
                    Lb[k] = np.eye(m)
    LU = _dense(row_ptr, col, Lb) @ _dense(row_ptr, col, Ub)
    x = np.random.default_rng(3).standard_normal((T, m))
    y = bilu.bilu0_solve(row_ptr, col, F, (LU @ x.reshape(-1)).reshape(T, m), rank)
    assert np.abs(y - x).max() <= 1e-10 * np.abs(x).max()
