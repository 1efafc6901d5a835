"""Pins for oracle.steppers: printed coefficients, closed-form amplification factors,
equilibria and exactness on manufactured solutions."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import steppers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s):
    return Fraction(s)


# ------------------------------------------------------------ coefficients --

def test_bdf2_matches_printed_coefficients():
    with open(os.path.join(GOLDEN, "bdf2_printed.json")) as f:
        g = json.load(f)
    a, beta = steppers.bdf_coefficients(2)
    C = steppers.bdf_second_derivative_coefficients(a)
    assert a == [_frac(s) for s in g["first_derivative_numerator"]]
    assert beta == _frac(g["beta"])
    assert C == [_frac(s) for s in g["second_derivative_numerator"]]


def test_bdf3_textbook():
    # 11/6 u^{n+1} - 3 u^n + 3/2 u^{n-1} - 1/3 u^{n-2} = dt f   (Hairer-Wanner table)
    a, beta = steppers.bdf_coefficients(3)
    assert beta == Fraction(6, 11)
    assert a == [1, Fraction(-18, 11), Fraction(9, 11), Fraction(-2, 11)]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_table1_C_is_self_convolution(k):
    a, _ = steppers.bdf_coefficients(k)
    C = steppers.bdf_second_derivative_coefficients(a)
    conv = np.convolve(np.array([float(x) for x in a]), np.array([float(x) for x in a]))
    np.testing.assert_allclose([float(x) for x in C], conv, atol=1e-12)
    # Table 1 end rows: C_{2k} = a_k a_k, C_{2k-1} = 2 a_{k-1} a_k
    assert C[2 * k] == a[k] * a[k]
    assert C[2 * k - 1] == 2 * a[k - 1] * a[k]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_bdf_exact_on_polynomials(k):
    a, beta = steppers.bdf_coefficients(k)
    dt = 0.1
    t = 1.0 - dt * np.arange(k + 1)          # t^{n+1}, t^n, ...
    for r in range(k + 1):
        u = t ** r
        d = sum(float(a[j]) * u[j] for j in range(k + 1)) / (float(beta) * dt)
        exact = r * t[0] ** (r - 1) if r > 0 else 0.0
        assert abs(d - exact) < 1e-9


def test_printed_dirk2_tableau_and_reading():
    with open(os.path.join(GOLDEN, "dirk2_printed.json")) as f:
        g = json.load(f)
    pr = steppers.DIRK2_AS_PRINTED
    assert pr["A"] == [[float(_frac(x)) for x in row] for row in g["A"]]
    assert pr["b"] == [float(_frac(x)) for x in g["b"]]
    assert pr["c"] == [float(_frac(x)) for x in g["c"]]
    # As printed the row sums are not c (the internal-consistency condition fails) ...
    assert not np.allclose(np.sum(pr["A"], axis=1), pr["c"])
    # ... while the reading used satisfies it.
    for tab in (steppers.DIRK2_QIN_ZHANG, steppers.DIRK3_MIDPOINT):
        np.testing.assert_allclose(np.sum(tab["A"], axis=1), tab["c"], atol=1e-15)


# ------------------------------------------------------- transfer matrices --

def _stability_function(tab, w):
    A = np.array(tab["A"], dtype=complex)
    b = np.array(tab["b"], dtype=complex)
    s = len(b)
    return 1.0 + w * b @ np.linalg.solve(np.eye(s) - w * A, np.ones(s))


def _bdf_transfer(k, K, c, dt):
    a, beta = steppers.bdf_coefficients(k)
    C = steppers.bdf_second_derivative_coefficients(a)
    n = 2 * k
    M = np.zeros((n, n))
    for col in range(n):
        hist = [np.zeros(1) for _ in range(n)]
        hist[col][0] = 1.0
        new = steppers.bdf_wave_update(hist, np.zeros(1), K, c, dt, beta, C)
        M[0, col] = new[0]
        if col + 1 < n:
            M[col + 1, col] = 1.0
    return M


@pytest.mark.parametrize("K", [0.3, 4.0, 150.0, 3.0e4])
def test_bdf1_amplification(K):
    c, dt = 1.0, 0.05
    th = c * np.sqrt(K) * dt
    ev = np.sort_complex(np.linalg.eigvals(_bdf_transfer(1, K, c, dt)))
    expect = np.sort_complex(np.array([1 / (1 + 1j * th), 1 / (1 - 1j * th)]))
    np.testing.assert_allclose(ev, expect, atol=1e-13)


@pytest.mark.parametrize("K", [0.3, 4.0, 150.0, 3.0e4])
def test_bdf2_amplification(K):
    c, dt = 1.0, 0.05
    th = c * np.sqrt(K) * dt
    roots = []
    for sgn in (+1, -1):
        r = np.sqrt(1 + sgn * 2j * th)
        roots += [1 / (2 + r), 1 / (2 - r)]
    ev = np.sort_complex(np.linalg.eigvals(_bdf_transfer(2, K, c, dt)))
    np.testing.assert_allclose(ev, np.sort_complex(np.array(roots)), atol=1e-12)


@pytest.mark.parametrize("k", [3, 4])
def test_bdfk_amplification_from_characteristic_polynomial(k):
    # D^2 u + w^2 u = 0 factors as (D - i w)(D + i w): z solves
    # sum_j a_j z^{k-j} = (+-) i w beta dt z^k.
    c, dt, K = 1.0, 0.05, 40.0
    a, beta = steppers.bdf_coefficients(k)
    w = c * np.sqrt(K)
    roots = []
    for sgn in (+1, -1):
        poly = np.array([float(x) for x in a], dtype=complex)
        poly[0] -= sgn * 1j * w * float(beta) * dt
        roots += list(np.roots(poly))
    ev = np.sort_complex(np.linalg.eigvals(_bdf_transfer(k, K, c, dt)))
    np.testing.assert_allclose(ev, np.sort_complex(np.array(roots)), atol=1e-9)


@pytest.mark.parametrize("K", [0.3, 4.0, 150.0, 3.0e4])
def test_cdf2_amplification_unit_modulus(K):
    c, dt = 1.0, 0.05
    M = np.zeros((2, 2))
    for col in range(2):
        u = [np.zeros(1), np.zeros(1)]
        u[col][0] = 1.0
        M[0, col] = steppers.cdf2_wave_update(u[0], u[1], 0.0, 0.0, K, c, dt)[0]
    M[1, 0] = 1.0
    ev = np.linalg.eigvals(M)
    L = 1 + 0.5 * c * c * dt * dt * K
    expect = np.roots([L, -2.0, L])
    np.testing.assert_allclose(np.sort_complex(ev), np.sort_complex(expect), atol=1e-13)
    np.testing.assert_allclose(np.abs(ev), 1.0, atol=1e-13)
    np.testing.assert_allclose(np.cos(np.angle(ev[0])), 1.0 / L, atol=1e-13)


@pytest.mark.parametrize("name", ["qz", "mid3", "printed"])
@pytest.mark.parametrize("K", [0.3, 4.0, 150.0, 3.0e4])
def test_dirk_amplification(name, K):
    tab = {"qz": steppers.DIRK2_QIN_ZHANG, "mid3": steppers.DIRK3_MIDPOINT,
           "printed": steppers.DIRK2_AS_PRINTED}[name]
    c, h = 1.0, 0.05
    M = np.zeros((2, 2))
    for col in range(2):
        uv = [np.zeros(1), np.zeros(1)]
        uv[col][0] = 1.0
        u1, v1 = steppers.dirk_wave_update(uv[0], uv[1], 0.0, 0.0, K, c, h,
                                           tab["A"], tab["b"], tab["c"])
        M[0, col], M[1, col] = u1[0], v1[0]
    th = c * np.sqrt(K) * h
    expect = np.array([_stability_function(tab, 1j * th), _stability_function(tab, -1j * th)])
    ev = np.linalg.eigvals(M)
    np.testing.assert_allclose(np.sort_complex(ev), np.sort_complex(expect), atol=1e-12)
    z = 1j * th
    if name == "qz":
        closed = ((1 + z / 4) / (1 - z / 4)) ** 2
        np.testing.assert_allclose(expect[0], closed, atol=1e-13)
        np.testing.assert_allclose(np.abs(ev), 1.0, atol=1e-12)
    if name == "mid3":
        closed = ((1 + z / 6) / (1 - z / 6)) ** 3
        np.testing.assert_allclose(expect[0], closed, atol=1e-13)
        np.testing.assert_allclose(np.abs(ev), 1.0, atol=1e-12)
    if name == "printed":
        closed = (8 - z * z) / (2 * (2 - z) ** 2)
        np.testing.assert_allclose(expect[0], closed, atol=1e-13)


# ------------------------------------------------------------- equilibria ---

@pytest.mark.parametrize("K", [0.5, 20.0])
def test_static_equilibrium_is_fixed_point(K):
    # u = S/K is the steady solution of (1/c^2) u_tt + K u = S for every stepper.
    c, dt, S = 0.7, 0.03, 2.5 + 1.5j
    u_eq = np.array([S / K])
    for k in (1, 2, 3):
        a, beta = steppers.bdf_coefficients(k)
        C = steppers.bdf_second_derivative_coefficients(a)
        new = steppers.bdf_wave_update([u_eq] * (2 * k), np.array([S]), K, c, dt, beta, C)
        np.testing.assert_allclose(new, u_eq, rtol=1e-13)
    new = steppers.cdf2_wave_update(u_eq, u_eq, S, S, K, c, dt)
    np.testing.assert_allclose(new, u_eq, rtol=1e-13)
    for tab in (steppers.DIRK2_QIN_ZHANG, steppers.DIRK3_MIDPOINT):
        u1, v1 = steppers.dirk_wave_update(u_eq, np.zeros(1), S, S, K, c, dt,
                                           tab["A"], tab["b"], tab["c"])
        np.testing.assert_allclose(u1, u_eq, rtol=1e-13)
        np.testing.assert_allclose(v1, 0.0, atol=1e-13)


# ------------------------------------------------ manufactured solutions ----

def _quad(t):
    return 0.3 - 1.1 * t + 0.7 * t * t


def test_bdf2_and_cdf2_exact_for_quadratic_in_time():
    # u(t) = quadratic; source S = u''/c^2 + K u is then reproduced exactly.
    c, dt, K = 0.9, 0.07, 3.0
    src = lambda t: 1.4 / (c * c) + K * _quad(t)
    a, beta = steppers.bdf_coefficients(2)
    C = steppers.bdf_second_derivative_coefficients(a)
    t_new = 1.0
    hist = [np.array([_quad(t_new - j * dt)]) for j in range(1, 5)]
    new = steppers.bdf_wave_update(hist, np.array([src(t_new)]), K, c, dt, beta, C)
    np.testing.assert_allclose(new, _quad(t_new), rtol=1e-12)
    new = steppers.cdf2_wave_update(np.array([_quad(t_new - dt)]), np.array([_quad(t_new - 2 * dt)]),
                                    src(t_new), src(t_new - 2 * dt), K, c, dt)
    np.testing.assert_allclose(new, _quad(t_new), rtol=1e-12)


def test_bdf1_exact_for_linear_in_time():
    c, dt, K = 1.3, 0.05, 2.0
    u = lambda t: 0.4 + 2.0 * t
    a, beta = steppers.bdf_coefficients(1)
    C = steppers.bdf_second_derivative_coefficients(a)
    hist = [np.array([u(1.0 - dt)]), np.array([u(1.0 - 2 * dt)])]
    new = steppers.bdf_wave_update(hist, np.array([K * u(1.0)]), K, c, dt, beta, C)
    np.testing.assert_allclose(new, u(1.0), rtol=1e-12)


@pytest.mark.parametrize("tab", [steppers.DIRK2_QIN_ZHANG, steppers.DIRK3_MIDPOINT])
def test_dirk_second_order_convergence(tab):
    # Forced wave mode u = sin(w t) + 0.2 t^2 with S = u''/c^2 + K u.
    c, K, w, T = 1.0, 9.0, 1.7, 2.0
    u = lambda t: np.sin(w * t) + 0.2 * t * t
    ud = lambda t: w * np.cos(w * t) + 0.4 * t
    src = lambda t: (-w * w * np.sin(w * t) + 0.4) / (c * c) + K * u(t)
    errs = []
    for nsteps in (40, 80, 160):
        h = T / nsteps
        uu, vv = np.array([u(0.0)]), np.array([ud(0.0)])
        for n in range(nsteps):
            uu, vv = steppers.dirk_wave_update(uu, vv, src(n * h), src((n + 1) * h), K, c, h,
                                               tab["A"], tab["b"], tab["c"])
        errs.append(abs(uu[0] - u(T)))
    assert 3.3 < errs[0] / errs[1] < 4.7
    assert 3.3 < errs[1] / errs[2] < 4.7


def test_continuity_updates():
    rng = np.random.default_rng(3)
    rho = [rng.standard_normal(5) + 1j * rng.standard_normal(5) for _ in range(3)]
    divj = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    dt = 0.02
    for k in (1, 2, 3):
        a, beta = steppers.bdf_coefficients(k)
        new = steppers.bdf_continuity(rho[:k], divj, dt, a, beta)
        lhs = (sum(float(a[j]) * ([new] + rho[:k])[j] for j in range(k + 1))
               / (float(beta) * dt) + divj)
        np.testing.assert_allclose(lhs, 0.0, atol=1e-10)
    new = steppers.cdf2_continuity(rho[0], divj, dt)
    np.testing.assert_allclose((new - rho[0]) / dt + divj, 0.0, atol=1e-10)
    tab = steppers.DIRK2_QIN_ZHANG
    divj_n = rng.standard_normal(5) + 0j
    new = steppers.dirk_continuity(rho[0], divj_n, divj, dt, tab["b"], tab["c"])
    r0, r1 = steppers.dirk_interp_weights(tab["b"], tab["c"])
    assert (r0, r1) == (0.5, 0.5)
    np.testing.assert_allclose(new, rho[0] - dt * (0.5 * divj_n + 0.5 * divj), atol=1e-14)


# ------------------------------------------- CDF-2 semi-implicit / explicit ----

def _transfer(update, K, c, dt):
    """2x2 transfer matrix of a source-free two-level update u^{n+1} = f(u^n, u^{n-1})."""
    M = np.zeros((2, 2))
    for col in range(2):
        u = [np.zeros(1), np.zeros(1)]
        u[col][0] = 1.0
        M[0, col] = update(u[0], u[1], 0.0, K, c, dt)[0]
    M[1, 0] = 1.0
    return M


@pytest.mark.parametrize("K", [0.3, 4.0, 150.0, 3.0e4])
def test_cdf2_semi_implicit_roots_of_printed_equation(K):
    # section 3.1, second form: (u+ - 2u + u-)/(c^2 dt^2) + K (u+ + u-)/2 = S^n; with S = 0
    # the roots of (1/(c dt)^2 + K/2) z^2 - 2/(c dt)^2 z + (1/(c dt)^2 + K/2) are the
    # eigenvalues of the update, on the unit circle for every K
    c, dt = 1.0, 0.05
    h = 1.0 / (c * c * dt * dt)
    expect = np.roots([h + 0.5 * K, -2.0 * h, h + 0.5 * K])
    ev = np.linalg.eigvals(_transfer(steppers.cdf2_semi_implicit_update, K, c, dt))
    np.testing.assert_allclose(np.sort_complex(ev), np.sort_complex(expect), atol=1e-12)
    np.testing.assert_allclose(np.abs(ev), 1.0, atol=1e-12)


@pytest.mark.parametrize("K", [0.3, 4.0, 150.0, 1500.0, 1700.0])
def test_cdf2_explicit_roots_and_stability_limit(K):
    # section 3.1, third form: (u+ - 2u + u-)/(c^2 dt^2) + K u = S^n; roots of
    # z^2 - (2 - (c dt)^2 K) z + 1: unit modulus while (c dt)^2 K <= 4, growth beyond
    c, dt = 1.0, 0.05
    expect = np.roots([1.0, -(2.0 - c * c * dt * dt * K), 1.0])
    ev = np.linalg.eigvals(_transfer(steppers.cdf2_explicit_update, K, c, dt))
    np.testing.assert_allclose(np.sort_complex(ev), np.sort_complex(expect), atol=1e-12)
    if c * c * dt * dt * K <= 4.0:
        np.testing.assert_allclose(np.abs(ev), 1.0, atol=1e-9)
    else:
        assert np.max(np.abs(ev)) > 1.0 + 1e-3


@pytest.mark.parametrize("K", [0.5, 20.0])
def test_cdf2_variants_static_equilibrium(K):
    # u = S/K (the Poisson solution) is a fixed point of both forms
    c, dt, S = 0.7, 0.03, 2.5 + 1.5j
    u_eq = np.array([S / K])
    for upd in (steppers.cdf2_semi_implicit_update, steppers.cdf2_explicit_update):
        np.testing.assert_allclose(upd(u_eq, u_eq, S, K, c, dt), u_eq, rtol=1e-13)
