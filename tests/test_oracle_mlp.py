"""Pins of the learned starting-density model's oracle (oracle.mlp): the
back-propagated gradient against central finite differences of the loss,
closed forms of the forward pass, the descriptors' normalisation, and the
first Adam step."""
import numpy as np
import pytest

from oracle import mlp
from paper_2112_08639_gb300 import inputs


def _small(seed=0, n_in=3, hidden=6, P=40):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(n_in, hidden, seed=seed)
    for k in p:                     # nonzero biases so every term is exercised
        if k.startswith("b"):
            p[k] = rng.normal(size=p[k].shape) * 0.3
    X = rng.uniform(0.0, 2.0, size=(P, n_in))
    rho = rng.uniform(0.01, 0.2, size=P)
    return p, X, rho


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    p, X, rho = _small(seed)
    Ne, dV = 3.0, 0.7
    L, g = mlp.loss_and_grad(p, X, rho, Ne, dV)
    assert L == pytest.approx(mlp.loss(p, X, rho, Ne, dV), rel=1e-14)
    eps = 1e-6
    for k in mlp.LAYER_NAMES:
        num = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += eps
            lp = mlp.loss(q, X, rho, Ne, dV)
            q[k][idx] -= 2 * eps
            lm = mlp.loss(q, X, rho, Ne, dV)
            num[idx] = (lp - lm) / (2 * eps)
        err = np.max(np.abs(num - g[k])) / max(np.max(np.abs(g[k])), 1e-12)
        assert err < 1e-6, (k, err)


def test_zero_weights_give_the_uniform_density():
    """With every weight zero the output is the same at every point, so the
    normalised density is exactly uniform, Ne / (P dV)."""
    p, X, _ = _small(2)
    for k in ("W1", "W2", "W3", "w4"):
        p[k] = np.zeros_like(p[k])
    rho = mlp.predict(p, X, 5.0, 0.25)
    np.testing.assert_allclose(rho, 5.0 / (len(X) * 0.25), rtol=1e-14)


def test_forward_of_a_hand_network():
    """One unit per layer, written out by hand."""
    p = {"W1": np.array([[0.5]]), "b1": np.array([0.1]), "W2": np.array([[-1.2]]),
         "b2": np.array([0.3]), "W3": np.array([[2.0]]), "b3": np.array([-0.4]),
         "w4": np.array([1.5]), "b4": np.array([0.2])}
    x = 0.8
    h1 = np.tanh(0.5 * x + 0.1)
    h2 = np.tanh(-1.2 * h1 + 0.3)
    h3 = np.tanh(2.0 * h2 - 0.4)
    y = np.log1p(np.exp(1.5 * h3 + 0.2))
    a = mlp.forward(p, np.array([[x]]))
    assert a["y"][0] == pytest.approx(y, rel=1e-15)


def test_prediction_holds_ne_electrons_and_is_positive():
    p, X, _ = _small(3, P=200)
    rho = mlp.predict(p, X, 7.0, 0.05)
    assert np.all(rho > 0)
    assert rho.sum() * 0.05 == pytest.approx(7.0, rel=1e-14)


def test_descriptors_have_unit_mean_and_follow_the_atoms():
    cfg = inputs.C1
    pos = inputs.fcc_positions(1, disp_sigma=0.2, seed=1)
    d = mlp.descriptors(cfg.n, cfg.L, pos)
    # before the compression each feature has mean 1: the grid sum of a
    # Gaussian is its integral up to aliasing, which is tiny while w is
    # above the spacing (h = 0.43 bohr)
    np.testing.assert_allclose(np.expm1(d).mean(0)[2:], 1.0, rtol=1e-6)
    assert np.all(d >= 0)
    # a lattice-vector shift of every atom leaves them unchanged
    d2 = mlp.descriptors(cfg.n, cfg.L, pos + cfg.L * np.array([1, -2, 0]))
    np.testing.assert_allclose(d2, d, rtol=1e-12, atol=1e-14)


def test_first_adam_step_moves_each_parameter_by_lr():
    p, X, rho = _small(4)
    _, g = mlp.loss_and_grad(p, X, rho, 3.0, 0.7)
    q = {k: v.copy() for k, v in p.items()}
    opt = mlp.Adam(q, lr=1e-2, eps=0.0)
    opt.step(q, g)
    for k in p:
        nz = g[k] != 0
        np.testing.assert_allclose((p[k] - q[k])[nz], 1e-2 * np.sign(g[k][nz]), rtol=1e-12)


def test_training_lowers_the_loss():
    """Target: the density of another network of the same shape."""
    p, X, _ = _small(5, P=100)
    q, _, _ = _small(6, P=100)
    rho = mlp.predict(q, X, 3.0, 0.7)
    L0, _ = mlp.loss_and_grad(p, X, rho, 3.0, 0.7)
    opt = mlp.Adam(p, lr=1e-2)
    for _ in range(200):
        _, g = mlp.loss_and_grad(p, X, rho, 3.0, 0.7)
        opt.step(p, g)
    assert mlp.loss(p, X, rho, 3.0, 0.7) < 0.05 * L0
