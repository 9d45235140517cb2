"""Pins of the FP64 oracle of the learned point proposal (no GPU).

Analytic backpropagation against central finite differences, Adam's first
step against its closed form, the features against closed forms on analytic
densities, and the candidate rule against a plain sort."""
import numpy as np
import pytest

from oracle import mlp_oracle as ML


def batch(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 3))
    y = (rng.uniform(size=n) < 0.2).astype(float)
    return x, y


def test_parameter_count():
    assert ML.NPARAM == 8641


@pytest.mark.parametrize("seed", [1, 2])
def test_backprop_equals_finite_differences(seed):
    """Every one of the 8,641 partial derivatives, central differences h = 1e-6."""
    p = ML.init_params(seed)
    p[ML.NPARAM - 1] = 0.3           # nonzero output bias
    x, y = batch(7, seed)
    L, g = ML.loss_grad(p, x, y, pos_weight=5.0)
    assert abs(L - ML.loss(p, x, y, 5.0)) < 1e-15
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(ML.NPARAM):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (ML.loss(p + e, x, y, 5.0) - ML.loss(p - e, x, y, 5.0)) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-8 * max(np.abs(g).max(), 1e-3)


def test_silu_derivative():
    a = np.linspace(-8, 8, 41)
    h = 1e-6
    fd = (ML.silu(a + h) - ML.silu(a - h)) / (2 * h)
    assert np.abs(fd - ML.silu_grad(a)).max() < 1e-9


def test_loss_limits():
    """BCE with logits: a confident right answer costs ~0, a wrong one ~|z|
    (times pos_weight for a missed positive); z = 0 costs log 2 per class."""
    p = np.zeros(ML.NPARAM)
    x = np.zeros((2, 3))
    p[-1] = 0.0
    assert abs(ML.loss(p, x, np.array([1.0, 0.0]), 1.0) - np.log(2)) < 1e-15
    p[-1] = 40.0
    assert ML.loss(p, x[:1], np.array([1.0]), 3.0) < 1e-15
    assert abs(ML.loss(p, x[:1], np.array([0.0]), 3.0) - 40.0) < 1e-12
    p[-1] = -40.0
    assert abs(ML.loss(p, x[:1], np.array([1.0]), 3.0) - 120.0) < 1e-12


def test_first_adam_step_is_a_signed_step():
    """At t = 1 the bias-corrected ratio m/sqrt(v) is g/|g|: every parameter
    with g != 0 moves by lr (up to eps), against its gradient."""
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = ML.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr=1e-3, eps=0.0)
    assert np.allclose(p1 - p, -1e-3 * np.sign(g), atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_gradient_of_a_plane_wave_density():
    """rho = 2 + cos(2 pi x / L) on a cubic grid: |grad rho| by central
    differences equals (2 pi / L) |sin| times sin(2 pi / g) / (2 pi / g)."""
    L, g = 7.0, 24
    lat = np.eye(3) * L
    x = np.arange(g) / g
    rho = np.broadcast_to((2.0 + np.cos(2 * np.pi * x))[:, None, None], (g, g, g)).ravel()
    got = ML.grad_norm(rho, (g, g, g), lat)
    exact = np.broadcast_to((2 * np.pi / L * np.abs(np.sin(2 * np.pi * x)))[:, None, None], (g, g, g)).ravel()
    factor = np.sin(2 * np.pi / g) / (2 * np.pi / g)
    assert np.abs(got - exact * factor).max() < 1e-12


def test_nearest_centre_minimum_image():
    lat = np.diag([4.0, 5.0, 6.0])
    d = ML.nearest_centre((4, 5, 6), lat, np.array([[0.0, 0.0, 0.0]]))
    # the point at fractional (0.75, 0, 0) is 1 bohr from the image at (4, 0, 0)
    idx = (3 * 5 + 0) * 6 + 0
    assert abs(d[idx] - 1.0) < 1e-14
    assert abs(d[0]) < 1e-14
    # the farthest point of the grid sits at fractional (0.5, 0.4, 0.5)
    assert abs(d.max() - np.sqrt(2.0 ** 2 + 2.0 ** 2 + 3.0 ** 2)) < 1e-12


def test_top_candidates_ties():
    s = np.array([0.5, 0.9, 0.5, 0.1, 0.9, 0.5])
    assert ML.top_candidates(s, 3).tolist() == [0, 1, 4]
    assert ML.top_candidates(s, 4).tolist() == [0, 1, 2, 4]
