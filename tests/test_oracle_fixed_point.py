"""Pins for oracle.fixed_point, the bit-exact model of the FP32 form's move and
fixed-point current deposit.

  * fmaf against exact rational arithmetic (fractions.Fraction, correctly rounded to
    float32), on random triples and on constructed ties;
  * the float32 shape weights against the textbook B-spline polynomials (FP64) within
    float32 rounding, summing to one;
  * a contribution is the exact product t W rounded once to the quantum: against exact
    rational arithmetic, on random float32 pairs and on constructed half-quantum ties;
  * the integer sums are exactly independent of the order of the particles;
  * the deposited current against the FP64 oracle deposit (oracle.pic.deposit) within the
    bound set by the quantum and the float32 roundings;
  * the quantum's power of two keeps every contribution below 2^38 quanta and every node
    total below 2^62.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fixed_point as fx
from oracle import pic as opic

from test_oracle_bspline import closed_form


def _round_f32(q):
    """Exact rational q rounded to the nearest float32 (ties to even)."""
    f = np.float32(float(q))  # within one float32 ulp of q; settle by exact comparison
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - q),
                                     int(np.frombuffer(np.float32(c).tobytes(), np.uint32)[0]) & 1))
    return np.float32(best)


def test_fmaf_is_correctly_rounded():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(3000).astype(np.float32)
    b = rng.standard_normal(3000).astype(np.float32) * np.float32(2.0) ** rng.integers(-30, 30, 3000).astype(np.float32)
    c = rng.standard_normal(3000).astype(np.float32) * np.float32(2.0) ** rng.integers(-40, 40, 3000).astype(np.float32)
    got = fx.fmaf(a, b, c)
    for i in range(3000):
        q = Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i]))
        assert got[i] == _round_f32(q), (i, a[i], b[i], c[i])


def test_fmaf_ties_are_settled_by_the_exact_value():
    # a b + c whose float64 sum lands on a float32 midpoint while the exact value does not
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -23)
    a = np.array([one + ulp, one + ulp, one], dtype=np.float32)
    b = np.array([one + ulp, one - ulp, one], dtype=np.float32)
    c = np.array([np.float32(2.0 ** -24), -np.float32(2.0 ** -24), np.float32(2.0 ** -24)],
                 dtype=np.float32)
    got = fx.fmaf(a, b, c)
    for i in range(3):
        q = Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i]))
        assert got[i] == _round_f32(q), i
    # a plain tie (exact value on the midpoint) rounds to even
    assert fx.fmaf(one, one, np.float32(2.0 ** -24)) == one


@pytest.mark.parametrize("p", [2, 3, 4])
def test_float32_weights_match_the_polynomials(p):
    xi = np.random.default_rng(p).uniform(0.0, 64.0, 5000).astype(np.float32)
    i0, w = fx.weights32(xi, p)
    for a in range(p + 1):
        exact = closed_form(xi.astype(np.float64) - (i0 + a), p)
        np.testing.assert_allclose(w[:, a], exact, rtol=0, atol=4e-7)
    np.testing.assert_allclose(w.astype(np.float64).sum(axis=1), 1.0, atol=1e-6)
    # the first node is the one of the FP64 oracle
    ref_i0, _ = opic.bspline.node_weights(xi.astype(np.float64), p)
    assert np.array_equal(i0, ref_i0)


def _rne(q):
    """Exact rational q rounded to the nearest integer, ties to even."""
    f = q.numerator // q.denominator
    r = q - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return f


def test_contribution_is_the_exact_product_rounded_once():
    rng = np.random.default_rng(5)
    scale = 2.0 ** 38
    t = (rng.standard_normal(2000) * 0.7).astype(np.float32)
    w = rng.uniform(0.0, 0.7, 2000).astype(np.float32)
    got = fx.contribution(t, w, scale)
    for i in range(2000):
        q = Fraction(float(t[i])) * Fraction(float(w[i])) * Fraction(2) ** 38
        assert got[i] == _rne(q), i
    # products that fall exactly on half a quantum go to the even integer, and rounding the
    # product to float32 first would move this one by a quantum
    half = np.float32(2.0 ** -39)
    t2 = np.array([3 * half, 5 * half, -3 * half], dtype=np.float32)
    w2 = np.ones(3, dtype=np.float32)
    assert list(fx.contribution(t2, w2, scale)) == [2, 2, -2]
    a, b = np.float32(1 + 2.0 ** -23), np.float32(1 - 2.0 ** -23)   # a b = 1 - 2^-46
    assert fx.contribution(a, b, 2.0 ** 46) == 2 ** 46 - 1
    assert np.rint(np.float64(np.float32(a * b)) * 2.0 ** 46) == 2 ** 46


def _inputs(n, seed, lx=1.0, ly=0.75):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0, lx, n), rng.uniform(0, ly, n), 0.3 * rng.standard_normal(n),
            0.3 * rng.standard_normal(n))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_sums_are_order_independent_and_match_fp64(p):
    nx, ny, lx, ly, dt = 16, 12, 1.0, 0.75, 0.02
    x, y, vx, vy = _inputs(3001, p)
    scale = fx.current_scale(1.0, len(x))
    x1, y1, jx, jy = fx.move_deposit(x, y, vx, vy, dt, lx, ly, nx, ny, p, scale)
    perm = np.random.default_rng(9).permutation(len(x))
    _, _, jx2, jy2 = fx.move_deposit(x[perm], y[perm], vx[perm], vy[perm], dt, lx, ly, nx, ny,
                                     p, scale)
    assert np.array_equal(jx, jx2) and np.array_equal(jy, jy2)
    # against the FP64 deposit of the same float32 positions and velocities: each of the
    # (p+1)^2 contributions a particle makes is off by at most half a quantum plus its float32
    # roundings (about 6 ulp of a value below |v|)
    cfg = opic.Config(nx=nx, ny=ny, lx=lx, ly=ly, dt=dt, p=p, w=1.0)
    v32x, v32y = vx.astype(np.float32).astype(np.float64), vy.astype(np.float32).astype(np.float64)
    ref = opic.deposit(cfg, x1.astype(np.float64), y1.astype(np.float64), v32x) * (cfg.dx * cfg.dy)
    # contributions per node: the particles whose stencil covers it
    i0, _ = fx.weights32((x1 * np.float32(1.0 / cfg.dx)).astype(np.float32), p)
    j0, _ = fx.weights32((y1 * np.float32(1.0 / cfg.dy)).astype(np.float32), p)
    cnt = np.zeros(nx * ny)
    for a in range(p + 1):
        for b in range(p + 1):
            np.add.at(cnt, np.mod(i0 + a, nx) * ny + np.mod(j0 + b, ny), 1.0)
    cnt = cnt.reshape(nx, ny)
    for v64, j in ((v32x, jx), (v32y, jy)):
        ref = opic.deposit(cfg, x1.astype(np.float64), y1.astype(np.float64), v64) * (cfg.dx * cfg.dy)
        bound = cnt * (0.5 / scale + 6 * 2.0 ** -24 * np.max(np.abs(v64)))
        assert np.all(np.abs(j / scale - ref) <= bound)


def test_quantum_bounds():
    for n in (1, 2, 1000, 2 ** 20, 26214400, 2 ** 31 - 1):
        for c in (1.0, 3.0, 0.25):
            s = fx.current_scale(c, n)
            assert c * s <= 2.0 ** 38                      # a contribution |v W W| < c
            assert n * c * s < 2.0 ** 62                   # one contribution per particle and node
            assert np.log2(s) == int(np.log2(s))           # a power of two
