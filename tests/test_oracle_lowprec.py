"""Pins of the oracle's low-precision condensation (oracle/lowprec.py): the rounding
functions against their IEEE definitions (ties, the library's BF16 conversion), the
W, Z operands against the plain Schur complement, and the error of the rounded form
against its first-order bound."""
import numpy as np
import pytest
import scipy.linalg

from oracle import lowprec
from paper_1605_01020_gb300 import workloads as W
from oracle_helpers import problem


def test_round_bf16_ties_and_library():
    one = 1.0
    ulp = 2.0 ** -7
    assert lowprec.round_bf16(one + ulp / 2) == one                    # tie, even neighbour below
    assert lowprec.round_bf16(one + 3 * ulp / 2) == one + 2 * ulp      # tie, even neighbour above
    assert lowprec.round_bf16(-(one + 3 * ulp / 2)) == -(one + 2 * ulp)
    assert lowprec.round_bf16(one + ulp / 2 + 2.0 ** -20) == one + ulp
    torch = pytest.importorskip("torch")
    scale = 10.0 ** np.random.default_rng(1).integers(-6, 6, 20000)
    x = (np.random.default_rng(0).standard_normal(20000) * scale).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert (lowprec.round_bf16(x) == ref).all()


def test_round_tf32_ties_and_bound():
    one = 1.0
    ulp = 2.0 ** -10
    assert lowprec.round_tf32(one + ulp / 2) == one + ulp               # tie, away from zero
    assert lowprec.round_tf32(-(one + ulp / 2)) == -(one + ulp)
    assert lowprec.round_tf32(one + 3 * ulp / 2) == one + 2 * ulp
    assert lowprec.round_tf32(one + ulp / 2 - 2.0 ** -20) == one
    x = np.random.default_rng(2).standard_normal(20000).astype(np.float32)
    r = lowprec.round_tf32(x)
    assert (np.abs(r - x) <= 2.0 ** -11 * np.abs(x) * (1 + 1e-7)).all()
    assert (r.astype(np.float32).view(np.uint32) & 0x1FFF == 0).all()   # 13 low bits dropped


@pytest.fixture(scope="module")
def element():
    wl = W.config(1)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    e = 5
    blk = pb.element_blocks(e, st.u, st.q, st.uhat, st.u_ref)
    Ke, _ = pb.condense_qelim(e, st.u, st.q, st.uhat, st.u_ref)
    return pb, blk, Ke


def test_operands_reproduce_the_schur_complement(element):
    """No rounding: D~ - W Z is the condensed block of the plain definition, W the
    multipliers (W U = C~) and Z the eliminated right block (P L Z = B~)."""
    pb, blk, Ke = element
    K, _ = lowprec.condense_rounded(pb, blk, None)
    assert np.abs(K - Ke).max() <= 1e-12 * np.abs(Ke).max()
    At, Bt, Ct = pb.qelim(blk)[:3]
    Wm, Zm = lowprec.schur_operands(At, Bt, Ct)
    P, L, U = scipy.linalg.lu(At)
    assert np.abs(Wm @ U - Ct).max() <= 1e-12 * np.abs(Ct).max()
    assert np.abs(P @ L @ Zm - Bt).max() <= 1e-12 * np.abs(Bt).max()


@pytest.mark.parametrize("fmt", ["tf32", "bf16"])
def test_rounded_error_within_first_order_bound(element, fmt):
    """|K_low - K| <= (2u + u^2) |W| |Z| entrywise (the operands rounded, nothing
    else), and the error is not zero (the rounding is applied)."""
    pb, blk, Ke = element
    K, bound = lowprec.condense_rounded(pb, blk, fmt)
    u = lowprec.UNIT_ROUNDOFF[fmt]
    err = np.abs(K - Ke)
    assert (err <= (2 * u + u * u) * bound * (1 + 1e-6) + 1e-14 * np.abs(Ke).max()).all()
    assert err.max() > 0.01 * u * bound.max()


def test_rounded_condensation_on_a_mixed_order_element():
    """The per-element form used for meshes of mixed orders: with no rounding it is the
    element's condensed block, with BF16 rounding it moves within the bound."""
    from oracle import iedg as oiedg
    from oracle import physics
    from oracle_helpers import ref_element
    orders = W.mixed_orders([3, 3], 5, levels=(1, 2, 3), probs=(0.3, 0.4, 0.3))
    mesh = W.structured_mesh_mixed(2, 3, orders)
    st = W.make_state_mixed(mesh, W.fourier_perturbed_field(2, 0.3, 6, amp=0.05), 7, noise=0.01)
    refs = {int(p): ref_element(2, int(p)) for p in set(mesh.orders.tolist())}
    prm = physics.Params(gamma=1.4, Pr=0.72, Re=100.0, Minf=0.3, alpha=W.dirk_alpha())
    pb = oiedg.MixedProblem(refs, mesh, prm)
    for e in range(mesh.n_elem):
        blk = pb.element_blocks(e, st.u, st.q, st.uhat)
        Ke, _ = pb.condense_qelim(e, st.u, st.q, st.uhat)
        K0, _ = lowprec.condense_rounded(pb.pbs[e], blk, None)
        assert np.abs(K0 - Ke).max() <= 1e-12 * np.abs(Ke).max()
        Kb, bound = lowprec.condense_rounded(pb.pbs[e], blk, "bf16")
        u = lowprec.UNIT_ROUNDOFF["bf16"]
        assert (np.abs(Kb - Ke) <= (2 * u + u * u) * bound * (1 + 1e-6) + 1e-14 * np.abs(Ke).max()).all()


def test_mass_scaling_of_the_mass_block_is_the_identity(element):
    """S (M (x) I) S^T = I and S^T S = I (x) M^-1 for S = I (x) L^-1, M = L L^T: the
    scaling turns the implicit stage's mass term into alpha I."""
    pb, blk, _ = element
    M = blk["M"]
    S = lowprec.mass_scaling(M, pb.m)
    MM = np.kron(np.eye(pb.m), M)
    n = MM.shape[0]
    assert np.abs(S @ MM @ S.T - np.eye(n)).max() <= 1e-12
    assert np.abs(S.T @ S @ MM - np.eye(n)).max() <= 1e-10
    assert np.abs(np.triu(S, 1)).max() == 0.0                      # lower triangular


def test_mass_scaled_system_has_the_same_schur_complement(element):
    """No rounding: the scaled system condenses to the plain K (Eq. LS is invariant
    under the u-block scaling)."""
    pb, blk, Ke = element
    K, _ = lowprec.condense_rounded(pb, blk, None, mass_scaled=True)
    assert np.abs(K - Ke).max() <= 1e-12 * np.abs(Ke).max()


@pytest.mark.parametrize("fmt", ["tf32", "bf16"])
def test_mass_scaled_rounded_error_within_first_order_bound(element, fmt):
    pb, blk, Ke = element
    K, bound = lowprec.condense_rounded(pb, blk, fmt, mass_scaled=True)
    u = lowprec.UNIT_ROUNDOFF[fmt]
    err = np.abs(K - Ke)
    assert (err <= (2 * u + u * u) * bound * (1 + 1e-6) + 1e-14 * np.abs(Ke).max()).all()
    assert err.max() > 0.01 * u * bound.max()


def test_mass_scaling_lowers_the_interior_conditioning():
    """On a 3D p=3 element of the Taylor-Green recipe the scaled u-block is better
    conditioned than A~ (1-norm condition numbers; measured about 28x lower)."""
    wl = W.config(2, N=2)
    st = wl.state
    pb = problem(wl.mesh, wl.params)
    blk = pb.element_blocks(3, st.u, st.q, st.uhat)
    At, Bt, Ct = pb.qelim(blk)[:3]
    As = lowprec.scale_system(lowprec.mass_scaling(blk["M"], pb.m), At, Bt, Ct)[0]
    assert np.linalg.cond(As, 1) * 5 < np.linalg.cond(At, 1)
