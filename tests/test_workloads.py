"""The synthetic input recipes: the fields and maps have the properties their
descriptions state (periodicity, solenoidal velocity, spectrum support and rms,
stretching ratio, positive Jacobians, order proportions).  Input generation only:
none of this is method arithmetic."""
import numpy as np
import pytest

from paper_1605_01020_gb300 import workloads as W


def _vel(field, x):
    u = field(x)
    return u[..., 1:4] / u[..., :1]


def test_broadband_field_is_periodic_solenoidal_with_the_stated_rms():
    f = W.broadband_field(0.3, 7)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (4000, 3))
    v = _vel(f, x) - np.array([1.0, 0.0, 0.0])
    # periodic on the unit cube (integer wavevectors)
    for r in range(3):
        e = np.zeros(3)
        e[r] = 1.0
        assert np.abs(_vel(f, x + e) - _vel(f, x)).max() < 1e-12
    # solenoidal: central-difference divergence far below the velocity gradients
    h = 1e-5
    div = np.zeros(len(x))
    gnorm = np.zeros(len(x))
    for r in range(3):
        e = np.zeros(3)
        e[r] = h
        dv = (_vel(f, x + e) - _vel(f, x - e)) / (2 * h)
        div += dv[:, r]
        gnorm += (dv ** 2).sum(-1)
    assert np.abs(div).max() < 1e-6 * np.sqrt(gnorm.max())
    # 5 % rms per component of the free-stream speed (sampling error ~ 2 %)
    rms = np.sqrt((v ** 2).mean(0))
    assert np.all(np.abs(rms - 0.05) < 0.006), rms
    # density and pressure of the free stream
    u = f(x)
    assert np.allclose(u[..., 0], 1.0)


def test_broadband_spectrum_support_and_slope():
    """Shell energies of the field's Fourier coefficients: nonzero only for
    1 <= |k| <= 8 and proportional to |k|^(-5/3) (shells of equal radius)."""
    f = W.broadband_field(0.3, 3)
    n = 20
    g = (np.arange(n) + 0.5) / n
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1)
    v = _vel(f, X) - np.array([1.0, 0.0, 0.0])
    vh = np.fft.fftn(v, axes=(0, 1, 2)) / n ** 3
    k = np.fft.fftfreq(n, 1.0 / n)
    K = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    E = (np.abs(vh) ** 2).sum(-1)
    shell = np.round(K).astype(int)
    Es = np.bincount(shell.ravel(), weights=E.ravel())
    assert Es[0] < 1e-20 and Es[9:].sum() < 1e-20 * Es.sum()
    ratios = Es[1:9] / (np.arange(1, 9) ** (-5.0 / 3.0))
    assert ratios.max() / ratios.min() < 1.5     # random phases and the rounding of |k| to shells


def test_stretched_mapping_ratio_and_jacobian():
    mp = W.stretched_mapping(5, ratio=50.0)
    eta = np.linspace(0, 1, 20001)
    X = np.stack([np.full_like(eta, 0.3), eta, np.full_like(eta, 0.7)], axis=-1)
    Y = mp(X)
    dy = np.gradient(Y[:, 1], eta)
    assert abs(dy.max() / dy.min() - 50.0) < 0.05
    rng = np.random.default_rng(1)
    P = rng.uniform(0, 1, (2000, 3))
    h = 1e-6
    J = np.stack([(mp(P + h * e) - mp(P - h * e)) / (2 * h) for e in np.eye(3)], axis=-1)
    assert (np.linalg.det(J) > 0).all()
    for r in range(3):                              # periodic-compatible map
        e = np.zeros(3)
        e[r] = 1.0
        assert np.abs(mp(P + e) - mp(P) - e).max() < 1e-12


def test_taylor_green_field():
    f = W.taylor_green_field(0.2)
    x = np.random.default_rng(2).uniform(0, 1, (500, 3))
    u = f(x)
    rho = u[..., 0]
    p = (1.4 - 1) * (u[..., 4] - 0.5 * (u[..., 1:4] ** 2).sum(-1) / rho)
    p0 = 1.0 / (1.4 * 0.2 ** 2)
    assert np.allclose(rho, p / p0, rtol=1e-12)
    assert np.abs(u[..., 3]).max() < 1e-14                      # w = 0


def test_mixed_order_draw_proportions():
    """The mixed-order batch's draw (16 x 16 x 32 cells, seed 1000 + 4): 2376 / 4110 /
    1706 elements of orders 2 / 3 / 4, within sampling error of 0.3 / 0.5 / 0.2."""
    orders = W.mixed_orders((16, 16, 32), 1004, levels=(2, 3, 4), probs=(0.3, 0.5, 0.2))
    counts = np.bincount(np.asarray(orders).ravel(), minlength=5)[2:5]
    assert counts.tolist() == [2376, 4110, 1706]
    assert np.all(np.abs(counts / 8192 - np.array([0.3, 0.5, 0.2])) < 0.02), counts
