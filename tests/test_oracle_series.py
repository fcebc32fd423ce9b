"""The analytical solution of the 2D reaction-diffusion verification case
(Eq. analytical2Dverification with Eq. Analytical_PeDa, Sec. 3.1) checked
against the boundary-value problem it solves."""
import math

import numpy as np
import pytest

from oracle import analytic


@pytest.mark.parametrize("peda", [0.1, 1.0, 100.0])
def test_beta_roots(peda):
    b = 80.0
    beta = analytic.beta_roots(peda, b, 100)
    t = beta * b
    assert np.allclose(t * np.tan(t), peda, rtol=1e-9)
    assert np.all(np.diff(beta) > 0)


@pytest.mark.parametrize("peda", [0.1, 1.0, 100.0])
def test_series_solves_the_problem(peda):
    a, b, c0, ceq = 100.0, 80.0, 1.0, 0.2
    D = 0.08
    k_r = peda * D / b
    h = 1e-3
    xs = np.linspace(5.0, 95.0, 7)
    ys = np.linspace(5.0, 75.0, 7)
    X, Y = np.meshgrid(xs, ys)
    f = lambda x, y: analytic.series_2d(x, y, a, b, peda, c0, ceq)
    lap = (f(X + h, Y) + f(X - h, Y) + f(X, Y + h) + f(X, Y - h) - 4 * f(X, Y)) / h**2
    assert np.abs(lap).max() < 1e-5
    # zero gradient at y = 0 and x = a
    assert np.abs((f(xs, np.full_like(xs, h)) - f(xs, np.full_like(xs, -h))) / (2 * h)).max() < 1e-8
    assert np.abs((f(np.full_like(ys, a + h), ys) - f(np.full_like(ys, a - h), ys)) / (2 * h)).max() < 1e-8
    # first-order reaction at y = b: -D dC/dy = k_r (C - C_eq)
    dcdy = (f(xs, np.full_like(xs, b + h)) - f(xs, np.full_like(xs, b - h))) / (2 * h)
    assert np.allclose(-D * dcdy, k_r * (f(xs, np.full_like(xs, b)) - ceq), rtol=1e-5, atol=1e-12)
    # Dirichlet C = c0 at x = 0 away from the corners (truncated series)
    assert np.abs(f(np.zeros(5), np.linspace(10, 60, 5)) - c0).max() < 2e-2
