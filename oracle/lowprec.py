"""Static condensation with the operands of the Schur complement rounded to a lower
precision (oracle, test infrastructure only; see oracle/__init__).

The condensed block of an element is K = D~ - C~ A~^-1 B~ (Eq. LS, q eliminated).
With the LU of A~ by partial pivoting, P^T A~ = L U (largest |a| in the column),
the partial LU of the bordered matrix [A~ B~; C~ D~] leaves
    W = C~ U^-1         in the trace rows' u-columns (the multipliers), and
    Z = L^-1 P^T B~     in the u-rows' trace columns,
with W Z = C~ A~^-1 B~, so K = D~ - W Z.  The low-precision form takes
    K_low = D~ - rho(W) rho(Z),
rho rounding every operand entry to the target format; the products and their sum
are formed here in FP64 (the tensor core accumulates in FP32, a difference far
below the operand rounding).  The paper has no precision discussion: this is the
reading of a Schur-complement GEMM with rounded operands and wide accumulation.

Mass-matrix scaling (a reading: the paper has no precision discussion; "scaling by
the element mass matrix" is read as a symmetric scaling of the u-block by the inverse
Cholesky factor of the element mass matrix M = L L^T, per conserved component): the
u-block A~ (dominated by the implicit stage's alpha M) becomes S A~ S^T with
S = I_m (x) L^-1, B~ becomes S B~ and C~ becomes C~ S^T.  The Schur complement is
unchanged in exact arithmetic; the factors W, Z of the scaled system are the ones
rounded.

Formats (values first rounded to FP32 with round-to-nearest-even, as the FP32
operands a device holds):
  TF32: 10 explicit mantissa bits, round to nearest, ties away from zero;
  BF16:  7 explicit mantissa bits, round to nearest, ties to even.
Unit roundoffs 2^-11 (TF32) and 2^-8 (BF16).
"""
import numpy as np
import scipy.linalg

UNIT_ROUNDOFF = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def round_tf32(x):
    """Nearest TF32 value, ties away from zero (on the FP32 bit pattern: add half an
    ulp of the 10-bit mantissa to the magnitude, clear the 13 dropped bits)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def round_bf16(x):
    """Nearest BF16 value, ties to even (add 0x7FFF plus the lowest kept bit, clear
    the 16 dropped bits)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


ROUNDING = {"tf32": round_tf32, "bf16": round_bf16, None: lambda x: np.asarray(x, dtype=np.float64)}


def schur_operands(At, Bt, Ct):
    """W = C~ U^-1 and Z = L^-1 P^T B~ of the partial LU with partial pivoting."""
    P, L, U = scipy.linalg.lu(At)                       # At = P L U
    W = scipy.linalg.solve_triangular(U.T, Ct.T, lower=True).T
    Z = scipy.linalg.solve_triangular(L, P.T @ Bt, lower=True, unit_diagonal=True)
    return W, Z


def mass_scaling(M, m):
    """S = I_m (x) L^-1 with M = L L^T (Cholesky factor of the element mass matrix), one
    diagonal block per conserved component of the component-major u-unknowns."""
    Linv = scipy.linalg.solve_triangular(np.linalg.cholesky(M), np.eye(M.shape[0]), lower=True)
    return np.kron(np.eye(m), Linv)


def scale_system(S, At, Bt, Ct):
    """The element system scaled symmetrically on its u-block: S A~ S^T, S B~, C~ S^T
    (the trace block D~ is unchanged).  The Schur complement is the same:
    C~ S^T (S A~ S^T)^-1 S B~ = C~ A~^-1 B~."""
    return S @ At @ S.T, S @ Bt, Ct @ S.T


def condense_rounded(sub, blk, fmt, mass_scaled=False):
    """K_low of one element in the node-major layout [s, i, t, k] and the first-order
    bound |W| |Z| of the rounding error's terms (same layout).  sub: the element's
    oracle Problem (its qelim and layout); blk: its element_blocks; fmt: "tf32",
    "bf16" or None (no rounding: K itself).  mass_scaled: W and Z are those of the
    system scaled by the element mass matrix (scale_system with mass_scaling)."""
    At, Bt, Ct, Dt = sub.qelim(blk)[:4]
    if mass_scaled:
        At, Bt, Ct = scale_system(mass_scaling(blk["M"], sub.m), At, Bt, Ct)
    W, Z = schur_operands(At, Bt, Ct)
    rho = ROUNDING[fmt]
    K = Dt - rho(W) @ rho(Z)
    bound = np.abs(W) @ np.abs(Z)
    m, Nb = sub.m, sub.Nb
    to_nm = lambda X: X.reshape(m, Nb, m, Nb).transpose(1, 0, 3, 2)
    return to_nm(K), to_nm(bound)
