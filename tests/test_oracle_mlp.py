"""Pins of the FP64 surrogate oracle: the analytic gradient equals central
finite differences of the loss; the output map inverts the target map."""
import numpy as np
import pytest

import oracle


def random_params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return rng.normal(size=oracle.mlp_nparam()) * scale


def test_parameter_count():
    assert oracle.mlp_nparam() == 64 * 4 + 64 + 64 * 64 + 64 + 8 * 64 + 8 == 5000


def test_gradient_equals_finite_differences():
    rng = np.random.default_rng(3)
    p = random_params(1)
    f = rng.normal(size=(7, 4))
    z = rng.integers(0, 8, size=7)
    t = rng.normal(size=7)
    loss, g = oracle.mlp_loss_grad(p, f, z, t)
    idx = np.concatenate([np.arange(0, 256, 17), np.arange(256, 320, 9),
                          np.arange(320, 4416, 97), np.arange(4416, 4480, 7),
                          np.arange(4480, 4992, 23), np.arange(4992, 5000)])
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, f, z, t)[0] - oracle.mlp_loss_grad(pm, f, z, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_forward_consistent_with_loss():
    rng = np.random.default_rng(4)
    p = random_params(2)
    f = rng.normal(size=(11, 4))
    z = rng.integers(0, 8, size=11)
    t = rng.normal(size=11)
    y = oracle.mlp_forward(p, f)
    loss, _ = oracle.mlp_loss_grad(p, f, z, t)
    assert loss == pytest.approx(np.mean((y[np.arange(11), z] - t) ** 2), rel=1e-12)


@pytest.mark.parametrize("nu", [0.0, 1e-12, 3.7e-9, 1e-3, 0.5, 7.0, 2e4])
def test_output_map_inverts_target(nu):
    assert oracle.mlp_rate_from_output(oracle.mlp_target(nu)) == pytest.approx(nu, rel=1e-9,
                                                                              abs=1e-24)
    assert oracle.mlp_target(0.0) == -1.0
    assert oracle.mlp_target(1e-20) == pytest.approx(-1.0, abs=1e-8)  # soft floor at 1e-12


def test_features_definition_points():
    """The field enters relative to F0 = (2 Ip)^(3/2) (atomic units) and the
    temperature relative to Ip: scaling Ip by 4 and the field by 8, or Ip and
    T_e by 2, leaves the features unchanged; at F = F0 the field feature is
    (0 + 1.4)/1.5.  The atomic field in the paper's unit a = eE/(m_e omega c)
    follows from SI constants."""
    e_au_paper = 5.14220674763e11 * 1.602176634e-19 / (
        9.1093837015e-31 * 299792458.0 * 2 * np.pi * 299792458.0 / 0.8e-6)
    hartree = 27.211386245988
    # hydrogen-like Ip = E_h / 2: F0 = 1 atomic unit
    f = oracle.mlp_features(e_au_paper, 8, 10 ** 19.5, 0.5 * hartree * 10 ** -0.2,
                            0.5 * hartree)
    np.testing.assert_allclose(f, [1.4 / 1.5, 1.0, 0.0, 0.0], atol=1e-9)
    a = oracle.mlp_features(0.05, 3, 1e21, 40.0, 60.0)
    b = oracle.mlp_features(0.4, 3, 1e21, 80.0, 240.0)
    c = oracle.mlp_features(0.4, 3, 1e21, 160.0, 240.0)
    assert a[0] == pytest.approx(b[0], abs=1e-12)
    assert a[3] == pytest.approx(c[3], abs=1e-12)
    f = oracle.mlp_features(0.0, 0, 0.0, 0.0, 15.0)  # floors: 1e-6, 1e15 cm^-3, 0.1 eV
    g = oracle.mlp_features(1e-6, 0, 1e15, 0.1, 15.0)
    np.testing.assert_allclose(f, g, atol=1e-15)
    assert f[2] == pytest.approx((15 - 19.5) / 4.5) and f[1] == 0.0
    # the other ends of the normalised ranges: F = 10^0.1 F0, n_e = 1e24 cm^-3 and
    # T_e = 10^2.8 Ip each map to +1
    f = oracle.mlp_features(e_au_paper * 10 ** 0.1, 8, 1e24, 0.5 * hartree * 10 ** 2.8,
                            0.5 * hartree)
    np.testing.assert_allclose(f, [1.0, 1.0, 1.0, 1.0], atol=1e-9)
