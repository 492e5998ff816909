"""CPU tests of the gradient-based fitting driver: the normalised descent with an
acceptance test converges on known goals (a quadratic; a quadratic whose
gradient carries noise), and the log-scale parameter map keeps class ratios."""
import numpy as np

from paper_1502_02908_gb300 import fitting as F
from paper_1502_02908_gb300 import workloads as W


def test_descent_finds_the_minimum_of_a_quadratic():
    A = np.array([[3.0, 0.5], [0.5, 1.0]])
    x_star = np.array([0.3, -0.2])

    def fg(x):
        d = x - x_star
        return float(d @ A @ d), 2 * A @ d

    r = F.gradient_descent(fg, [1.0, 1.0], step=0.5, iterations=60)
    assert np.linalg.norm(r.x - x_star) < 1e-3
    assert r.f < 1e-6
    assert all(b[2] <= a[2] for a, b in zip(r.history, r.history[1:]))      # never increases


def test_descent_tolerates_gradient_noise():
    rng = np.random.default_rng(3)
    x_star = np.array([-0.4, 0.25])

    def fg(x):
        d = x - x_star
        g = 2 * d + rng.normal(0.0, 0.3 * (np.linalg.norm(d) + 1e-3), size=2)   # 30 % noise
        return float(d @ d), g

    r = F.gradient_descent(fg, [0.5, 0.5], step=0.3, iterations=80)
    assert np.linalg.norm(r.x - x_star) < 0.02


def test_scaled_params_keep_class_ratios():
    w = W.sise3_national(N=50, T=5, n_events=0, R=2)
    p = F.scaled_params(w.params, [np.log(2.0), np.log(0.5)])
    np.testing.assert_allclose(p.upsilon, 2.0 * w.params.upsilon)
    np.testing.assert_allclose(p.gamma, 0.5 * w.params.gamma)
    np.testing.assert_array_equal(p.beta, w.params.beta)
