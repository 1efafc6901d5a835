"""Pins for oracle.bspline: the Cox-de Boor shapes against closed forms and moments."""
import numpy as np
import pytest

from oracle import bspline


def closed_form(t, p):
    """Textbook piecewise polynomials of the centred cardinal B-splines (degrees 1-4)."""
    a = np.abs(np.asarray(t, dtype=np.float64))
    if p == 1:
        return np.where(a < 1, 1 - a, 0.0)
    if p == 2:
        return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    if p == 3:
        return np.where(a < 1, 2 / 3 - a * a + 0.5 * a ** 3,
                        np.where(a < 2, (2 - a) ** 3 / 6, 0.0))
    if p == 4:
        return np.where(
            a < 0.5, (115 - 120 * a ** 2 + 48 * a ** 4) / 192,
            np.where(a < 1.5, (55 + 20 * a - 120 * a ** 2 + 80 * a ** 3 - 16 * a ** 4) / 96,
                     np.where(a < 2.5, (5 - 2 * a) ** 4 / 384, 0.0)))
    raise ValueError(p)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cox_de_boor_matches_closed_form(p):
    t = np.linspace(-3.2, 3.2, 2001)
    np.testing.assert_allclose(bspline.cardinal_bspline(t, p), closed_form(t, p), atol=2e-15)


def test_quadratic_offset_form():
    # w_{-1} = (1/2)(1/2 - d)^2, w_0 = 3/4 - d^2, w_{+1} = (1/2)(1/2 + d)^2 for the
    # nearest node i0 = floor(xi + 1/2) and d = xi - i0 (Birdsall & Langdon 8.8).
    rng = np.random.default_rng(0)
    xi = rng.uniform(0, 50, 500)
    i0, w = bspline.node_weights(xi, 2)
    ic = np.floor(xi + 0.5).astype(int)
    d = xi - ic
    np.testing.assert_array_equal(i0, ic - 1)
    np.testing.assert_allclose(w[:, 0], 0.5 * (0.5 - d) ** 2, atol=1e-15)
    np.testing.assert_allclose(w[:, 1], 0.75 - d * d, atol=1e-15)
    np.testing.assert_allclose(w[:, 2], 0.5 * (0.5 + d) ** 2, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_partition_of_unity_and_first_moment(p):
    rng = np.random.default_rng(p)
    xi = rng.uniform(0, 100, 4000)
    i0, w = bspline.node_weights(xi, p)
    nodes = i0[:, None] + np.arange(p + 1)[None, :]
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose((w * (nodes - xi[:, None])).sum(axis=1), 0.0, atol=1e-13)
    assert np.all(w >= -1e-16)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_second_moment_is_spline_variance(p):
    # B-splines of degree >= 2 reproduce quadratics: sum_i (i - xi)^2 W_p(xi - i)
    # equals the variance of a sum of p+1 independent U(-1/2, 1/2), (p+1)/12.
    rng = np.random.default_rng(10 + p)
    xi = rng.uniform(0, 100, 4000)
    i0, w = bspline.node_weights(xi, p)
    nodes = i0[:, None] + np.arange(p + 1)[None, :]
    np.testing.assert_allclose((w * (nodes - xi[:, None]) ** 2).sum(axis=1), (p + 1) / 12,
                               atol=1e-12)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_unit_integral(p):
    t = np.linspace(-3, 3, 600001)
    integral = np.trapezoid(bspline.cardinal_bspline(t, p), t)
    assert abs(integral - 1.0) < 1e-9
