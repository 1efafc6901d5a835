"""Pins for oracle.adjoint, the discrete adjoint of the PIC step.

The adjoint is the transpose of the Jacobian of the forward map oracle.pic.step
(Algorithm 1 with the BDF-k stepper of section 3.2, the CDF-2 forms of section 3.1 or
s-stage DIRK of section 3.3), so it is pinned by things fixed outside it:
  * spline derivatives against the closed-form B-spline polynomials (differentiated by
    hand for p = 2, by central differences for p = 3, 4) and their zero sum;
  * exact transpose identities of the linear pieces (scatter vs gather; the whole field
    solve against oracle.pic.field_solve by the dot-product test), which a dropped term,
    a flipped sign of i k or exchanged DIRK source columns planted in the adjoint break;
  * gradients of the full run against central finite differences of oracle.pic.run,
    for W_B = 1/2 sum B_z^2 dx dy and for the final momenta, per component and along
    random directions, for both v^0 and P^0 as the independent variable;
  * free streaming (zero weight): P stays P^0, so d(sum a.P^N)/dv^0 = (dP/dv)^T a and
    d/dP^0 = a in closed form.
"""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import pic as opic
from oracle import spectral
from oracle import steppers as osteps

from test_oracle_bspline import closed_form


def _cfg(**kw):
    base = dict(nx=16, ny=12, lx=1.0, ly=0.8, dt=0.025, p=3, stepper="bdf", bdf_order=2,
                w=1.0 / 160)
    base.update(kw)
    return opic.Config(**base)


def _beams(n, seed, vd=0.3, vth=0.05, lx=1.0, ly=0.8):
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0, lx, n)
    y0 = rng.uniform(0, ly, n)
    sign = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0)
    vx0 = vth * rng.standard_normal(n)
    vy0 = sign * vd + vth * rng.standard_normal(n)
    return x0, y0, vx0, vy0


# ------------------------------------------------------------------ shapes --

def test_shape_derivative_quadratic_by_hand():
    # w = ((1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2), d = xi - round(xi)
    xi = np.array([3.0, 3.2, 3.49, 2.51, 0.0])
    i0, w, dw = oadj.node_weight_derivatives(xi, 2)
    d = xi - (i0 + 1)
    np.testing.assert_allclose(dw, np.stack([-(0.5 - d), -2.0 * d, 0.5 + d], axis=-1),
                               atol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_shape_derivatives_match_closed_form_and_sum_to_zero(p):
    xi = np.random.default_rng(p).uniform(0.0, 9.0, 400)
    i0, w, dw = oadj.node_weight_derivatives(xi, p)
    h = 1e-6
    for a in range(p + 1):
        t = xi - (i0 + a)
        fd = (closed_form(t + h, p) - closed_form(t - h, p)) / (2 * h)
        np.testing.assert_allclose(dw[:, a], fd, atol=1e-8)
    np.testing.assert_allclose(dw.sum(axis=1), 0.0, atol=1e-14)


def test_gather_grad_is_derivative_of_gather():
    cfg = _cfg(p=4)
    rng = np.random.default_rng(3)
    grid = rng.standard_normal((cfg.nx, cfg.ny))
    x = rng.uniform(0, cfg.lx, 50)
    y = rng.uniform(0, cfg.ly, 50)
    gx, gy = oadj.gather_grad(cfg, x, y, grid)
    h = 1e-6
    fdx = (opic.gather(cfg, x + h, y, grid) - opic.gather(cfg, x - h, y, grid)) / (2 * h)
    fdy = (opic.gather(cfg, x, y + h, grid) - opic.gather(cfg, x, y - h, grid)) / (2 * h)
    np.testing.assert_allclose(gx, fdx, rtol=1e-7, atol=1e-7)
    np.testing.assert_allclose(gy, fdy, rtol=1e-7, atol=1e-7)


def test_scatter_is_transpose_of_gather():
    cfg = _cfg(p=3)
    rng = np.random.default_rng(4)
    x = rng.uniform(0, cfg.lx, 70)
    y = rng.uniform(0, cfg.ly, 70)
    vals = rng.standard_normal(70)
    grid = rng.standard_normal((cfg.nx, cfg.ny))
    lhs = np.sum(oadj.scatter(cfg, x, y, vals) * grid)
    rhs = np.dot(vals, opic.gather(cfg, x, y, grid))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


# ------------------------------------------------------------------ fields --

def _hermitian(rng, cfg):
    return spectral.dft2(rng.standard_normal((cfg.nx, cfg.ny)))


def _pair(a, b):
    return float(np.real(np.sum(np.conj(a) * b)))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_field_adjoint_is_transpose_of_field_solve(k):
    # the field solve is linear in (history, J): <H'_bar, H'> + <F_bar, F> must equal
    # <H_bar, dH> + <J_bar, dJ> for the adjoint (H_bar, J_bar) of (H'_bar, F_bar)
    cfg = _cfg(bdf_order=k)
    rng = np.random.default_rng(10 + k)
    st = opic.State(*[np.zeros(1)] * 8)
    st.hist = {"phi": [_hermitian(rng, cfg) for _ in range(2 * k)],
               "ax": [_hermitian(rng, cfg) for _ in range(2 * k)],
               "ay": [_hermitian(rng, cfg) for _ in range(2 * k)],
               "rho": [_hermitian(rng, cfg) for _ in range(k)]}
    h_in = {key: [v.copy() for v in vals] for key, vals in st.hist.items()}
    jx = rng.standard_normal((cfg.nx, cfg.ny))
    jy = rng.standard_normal((cfg.nx, cfg.ny))
    fields = opic.field_solve(cfg, st, jx, jy)
    hbar_out = {key: [_hermitian(rng, cfg) for _ in vals] for key, vals in st.hist.items()}
    fbar = {name: rng.standard_normal((cfg.nx, cfg.ny)) for name in opic.FIELD_NAMES}
    hbar_in, (jxb, jyb) = oadj.field_adjoint_bdf(cfg, hbar_out, fbar)
    lhs = sum(_pair(hbar_out[key][d], st.hist[key][d]) for key in st.hist
              for d in range(len(st.hist[key])))
    lhs += sum(float(np.sum(fbar[name] * fields[name])) for name in opic.FIELD_NAMES)
    rhs = sum(_pair(hbar_in[key][d], h_in[key][d]) for key in h_in for d in range(len(h_in[key])))
    rhs += float(np.sum(jxb * jx) + np.sum(jyb * jy))
    scale = sum(abs(_pair(hbar_out[key][d], st.hist[key][d])) for key in st.hist
                for d in range(len(st.hist[key])))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def _random_hist(rng, cfg, like):
    return {key: ([_hermitian(rng, cfg) for _ in val] if isinstance(val, list)
                  else _hermitian(rng, cfg)) for key, val in like.items()}


def _pair_hist(a, b):
    return sum(sum(_pair(x, y) for x, y in zip(a[key], b[key])) if isinstance(a[key], list)
               else _pair(a[key], b[key]) for key in a)


OTHER_STEPPERS = [
    ("cdf2-implicit", dict(stepper="cdf2", cdf_form="implicit")),
    ("cdf2-semi", dict(stepper="cdf2", cdf_form="semi")),
    ("cdf2-explicit", dict(stepper="cdf2", cdf_form="explicit")),
    ("dirk2", dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG)),
    ("dirk3", dict(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT)),
]


@pytest.mark.parametrize("name,kw", OTHER_STEPPERS, ids=[c[0] for c in OTHER_STEPPERS])
def test_cdf2_and_dirk_field_adjoints_are_transposes(name, kw):
    # the same dot-product identity for the CDF-2 and DIRK field solves, on a history of
    # random spectra (every level independent, so a dropped or misrouted term shows)
    cfg = _cfg(**kw)
    rng = np.random.default_rng(abs(hash(name)) % 1000)
    st = opic.initial_state(cfg, *_beams(8, seed=1))
    st.hist = _random_hist(rng, cfg, st.hist)
    h_in = {key: ([v.copy() for v in val] if isinstance(val, list) else val.copy())
            for key, val in st.hist.items()}
    jx = rng.standard_normal((cfg.nx, cfg.ny))
    jy = rng.standard_normal((cfg.nx, cfg.ny))
    fields = opic.field_solve(cfg, st, jx, jy)
    hbar_out = _random_hist(rng, cfg, st.hist)
    fbar = {name_: rng.standard_normal((cfg.nx, cfg.ny)) for name_ in opic.FIELD_NAMES}
    adj = oadj.field_adjoint_cdf2 if cfg.stepper == "cdf2" else oadj.field_adjoint_dirk
    hbar_in, (jxb, jyb) = adj(cfg, hbar_out, fbar)
    assert set(hbar_in) == set(h_in)
    lhs = _pair_hist(hbar_out, st.hist)
    lhs += sum(float(np.sum(fbar[f] * fields[f])) for f in opic.FIELD_NAMES)
    rhs = _pair_hist(hbar_in, h_in) + float(np.sum(jxb * jx) + np.sum(jyb * jy))
    scale = abs(_pair_hist(hbar_out, st.hist)) + abs(_pair_hist(hbar_in, h_in))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
    # each block separately: only the current, only one history entry
    for key in h_in:
        zero_out = {k: ([np.zeros_like(v) for v in val] if isinstance(val, list)
                        else np.zeros_like(val)) for k, val in hbar_out.items()}
        zero_out[key] = hbar_out[key]
        nof = {f: np.zeros((cfg.nx, cfg.ny)) for f in opic.FIELD_NAMES}
        hb, (jxb1, jyb1) = adj(cfg, zero_out, nof)
        st.hist = {k: ([v.copy() for v in val] if isinstance(val, list) else val.copy())
                   for k, val in h_in.items()}
        opic.field_solve(cfg, st, jx, jy)
        l1 = _pair_hist(zero_out, st.hist)
        r1 = _pair_hist(hb, h_in) + float(np.sum(jxb1 * jx) + np.sum(jyb1 * jy))
        assert abs(l1 - r1) <= 1e-12 * (abs(l1) + abs(r1) + 1.0), (key, l1, r1)


def _identity_gap(cfg, seed, adjoint=None):
    """(lhs - rhs, scale) of the dot-product identity of one field solve and its adjoint
    on random histories, currents and field adjoints."""
    rng = np.random.default_rng(seed)
    st = opic.initial_state(cfg, *_beams(8, seed=1))
    st.hist = _random_hist(rng, cfg, st.hist)
    h_in = {key: ([v.copy() for v in val] if isinstance(val, list) else val.copy())
            for key, val in st.hist.items()}
    jx = rng.standard_normal((cfg.nx, cfg.ny))
    jy = rng.standard_normal((cfg.nx, cfg.ny))
    fields = opic.field_solve(cfg, st, jx, jy)
    hbar_out = _random_hist(rng, cfg, st.hist)
    fbar = {f: rng.standard_normal((cfg.nx, cfg.ny)) for f in opic.FIELD_NAMES}
    if adjoint is None:
        adjoint = oadj.field_adjoint_cdf2 if cfg.stepper == "cdf2" else oadj.field_adjoint_dirk
    hbar_in, (jxb, jyb) = adjoint(cfg, hbar_out, fbar)
    lhs = _pair_hist(hbar_out, st.hist) + sum(float(np.sum(fbar[f] * fields[f]))
                                              for f in opic.FIELD_NAMES)
    rhs = _pair_hist(hbar_in, h_in) + float(np.sum(jxb * jx) + np.sum(jyb * jy))
    return lhs - rhs, abs(lhs) + abs(rhs)


def test_planted_adjoint_mistakes_break_the_identity(monkeypatch):
    # the dot-product identity is the adjoints' pin: each plausible mistake, planted in a
    # copy of the oracle's adjoint, must break it by far more than its 1e-12 tolerance
    cfg = _cfg(stepper="cdf2", cdf_form="implicit")
    gap, scale = _identity_gap(cfg, 5)
    assert abs(gap) <= 1e-12 * scale

    def dropped_term(c, hb, fb):  # the implicit form's rho^{n-1} source left out
        out, j = oadj.field_adjoint_cdf2(c, hb, fb)
        out["rho_prev"] = np.zeros_like(out["rho_prev"])
        return out, j
    gap, scale = _identity_gap(cfg, 5, dropped_term)
    assert abs(gap) > 1e-6 * scale

    def wrong_sign(c, hb, fb):  # conj(i k) taken as +i k (every k flipped in the adjoint)
        with monkeypatch.context() as m:
            kgrid = spectral.wavenumber_grid
            m.setattr(spectral, "wavenumber_grid",
                      lambda *a: (lambda kx, ky, K: (-kx, -ky, K))(*kgrid(*a)))
            return oadj.field_adjoint_cdf2(c, hb, fb)
    gap, scale = _identity_gap(cfg, 5, wrong_sign)
    assert abs(gap) > 1e-6 * scale

    # DIRK: the S^n and S^{n+1} columns of the stage matrix exchanged (an index mistake)
    dcfg = _cfg(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG)
    _, _, K = spectral.wavenumber_grid(dcfg.nx, dcfg.ny, dcfg.lx, dcfg.ly)
    M = oadj.dirk_matrix(dcfg, K)
    assert np.max(np.abs(M[0][2] - M[0][3])) > 1e-3 * np.max(np.abs(M[0][2]))
    good = oadj.dirk_matrix
    monkeypatch.setattr(oadj, "dirk_matrix",
                        lambda c, k: [[r[0], r[1], r[3], r[2]] for r in good(c, k)])
    gap, scale = _identity_gap(dcfg, 6)
    assert abs(gap) > 1e-6 * scale


def test_dirk_matrix_reproduces_the_stage_loop():
    # the unit-input matrix applied to random inputs equals the stage recurrence itself
    cfg = _cfg(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT)
    _, _, K = spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)
    rng = np.random.default_rng(2)
    u, v, s0, s1 = (_hermitian(rng, cfg) for _ in range(4))
    M = oadj.dirk_matrix(cfg, K)
    A, b, cv = cfg.dirk["A"], cfg.dirk["b"], cfg.dirk["c"]
    uo, vo = osteps.dirk_wave_update(u, v, s0, s1, K, cfg.c, cfg.dt, A, b, cv)
    for r, ref in ((0, uo), (1, vo)):
        got = M[r][0] * u + M[r][1] * v + M[r][2] * s0 + M[r][3] * s1
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.max(np.abs(ref)))
    # K = 0, one stage of the implicit midpoint: k_v = c^2 (S0 + S1)/2, k_u = v + h k_v / 2,
    # so u' = u + h v + (h c)^2 (S0 + S1)/4 and v' = v + h c^2 (S0 + S1)/2
    mid = _cfg(stepper="dirk", dirk={"A": [[0.5]], "b": [1.0], "c": [0.5]}, c=2.0)
    m0 = oadj.dirk_matrix(mid, np.zeros(1))
    h, c2 = mid.dt, mid.c ** 2
    np.testing.assert_allclose([m0[0][i][0] for i in range(4)],
                               [1.0, h, h * h * c2 / 4, h * h * c2 / 4], rtol=1e-14)
    np.testing.assert_allclose([m0[1][i][0] for i in range(4)],
                               [0.0, 1.0, h * c2 / 2, h * c2 / 2], rtol=1e-14, atol=1e-16)


# ------------------------------------------------------------------ whole run --

def _fd(f, h):
    return (f(h) - f(-h)) / (2 * h)


@pytest.mark.parametrize("p,k", [(2, 1), (3, 2), (4, 3)])
def test_magnetic_energy_gradient_matches_finite_differences(p, k):
    cfg = _cfg(p=p, bdf_order=k)
    n, nsteps = 160, 10
    x0, y0, vx0, vy0 = _beams(n, seed=p)
    tape = oadj.record(cfg, x0, y0, vx0, vy0, nsteps)
    g = oadj.gradient(tape)
    gvx, gvy = g["v0"]
    rng = np.random.default_rng(100 + p)
    h = 1e-6
    # components
    for i in rng.choice(n, 4, replace=False):
        for c, gv in ((0, gvx), (1, gvy)):
            def f(e, i=i, c=c):
                v = [vx0.copy(), vy0.copy()]
                v[c][i] += e
                return oadj.objective(cfg, x0, y0, v[0], v[1], nsteps)
            fd = _fd(f, h)
            assert abs(fd - gv[i]) <= 1e-6 * abs(gv[i]) + 1e-13, (i, c, fd, gv[i])
    # random directions in v^0
    for _ in range(2):
        d = rng.standard_normal((2, n))
        fd = _fd(lambda e: oadj.objective(cfg, x0, y0, vx0 + e * d[0], vy0 + e * d[1], nsteps), h)
        ad = float(np.dot(gvx, d[0]) + np.dot(gvy, d[1]))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("name,kw", OTHER_STEPPERS, ids=[c[0] for c in OTHER_STEPPERS])
def test_cdf2_and_dirk_gradients_match_finite_differences(name, kw):
    cfg = _cfg(p=3, **kw)
    n, nsteps = 160, 10
    x0, y0, vx0, vy0 = _beams(n, seed=11)
    tape = oadj.record(cfg, x0, y0, vx0, vy0, nsteps)
    g = oadj.gradient(tape)
    gvx, gvy = g["v0"]
    rng = np.random.default_rng(12)
    h = 1e-6
    for i in rng.choice(n, 3, replace=False):
        def f(e, i=i):
            v = vy0.copy()
            v[i] += e
            return oadj.objective(cfg, x0, y0, vx0, v, nsteps)
        fd = _fd(f, h)
        assert abs(fd - gvy[i]) <= 1e-6 * abs(gvy[i]) + 1e-13, (i, fd, gvy[i])
    d = rng.standard_normal((2, n))
    fd = _fd(lambda e: oadj.objective(cfg, x0, y0, vx0 + e * d[0], vy0 + e * d[1], nsteps), h)
    ad = float(np.dot(gvx, d[0]) + np.dot(gvy, d[1]))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    # the final momenta as the objective
    ax, ay = rng.standard_normal(n), rng.standard_normal(n)
    gm = oadj.gradient(tape, px_bar=ax, py_bar=ay)
    fd = _fd(lambda e: oadj.objective(cfg, x0, y0, vx0 + e * d[0], vy0 + e * d[1], nsteps,
                                      px_bar=ax, py_bar=ay), h)
    ad = float(np.dot(gm["v0"][0], d[0]) + np.dot(gm["v0"][1], d[1]))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_momentum_gradient_with_p0_as_variable():
    cfg = _cfg(p=3, bdf_order=2)
    n, nsteps = 160, 8
    x0, y0, vx0, vy0 = _beams(n, seed=7)
    c2 = cfg.c ** 2
    gam = 1.0 / np.sqrt(1.0 - (vx0 ** 2 + vy0 ** 2) / c2)
    px0, py0 = gam * cfg.m * vx0, gam * cfg.m * vy0
    rng = np.random.default_rng(8)
    ax, ay = rng.standard_normal(n), rng.standard_normal(n)
    tape = oadj.record(cfg, x0, y0, vx0, vy0, nsteps)
    g = oadj.gradient(tape, px_bar=ax, py_bar=ay)
    gpx, gpy = g["p0"]

    def f(e, d):
        vx, vy = oadj.velocity_from_p0(cfg, px0 + e * d[0], py0 + e * d[1])
        return oadj.objective(cfg, x0, y0, vx, vy, nsteps, px_bar=ax, py_bar=ay)
    for _ in range(2):
        d = rng.standard_normal((2, n))
        fd = _fd(lambda e: f(e, d), 1e-6)
        ad = float(np.dot(gpx, d[0]) + np.dot(gpy, d[1]))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    for i in rng.choice(n, 3, replace=False):
        d = np.zeros((2, n))
        d[1, i] = 1.0
        fd = _fd(lambda e: f(e, d), 1e-6)
        assert abs(fd - gpy[i]) <= 1e-6 * abs(gpy[i]), (i, fd, gpy[i])


def test_free_streaming_gradient_closed_form():
    # zero weight: no fields, P^N = P^0 = gamma m v^0
    cfg = _cfg(p=2, bdf_order=2, w=0.0)
    n = 64
    x0, y0, vx0, vy0 = _beams(n, seed=9)
    rng = np.random.default_rng(9)
    ax, ay = rng.standard_normal(n), rng.standard_normal(n)
    tape = oadj.record(cfg, x0, y0, vx0, vy0, 6)
    g = oadj.gradient(tape, px_bar=ax, py_bar=ay)
    c2 = cfg.c ** 2
    gam = 1.0 / np.sqrt(1.0 - (vx0 ** 2 + vy0 ** 2) / c2)
    va = vx0 * ax + vy0 * ay
    ex = gam * cfg.m * (ax + gam ** 2 * vx0 * va / c2)
    ey = gam * cfg.m * (ay + gam ** 2 * vy0 * va / c2)
    np.testing.assert_allclose(g["v0"][0], ex, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(g["v0"][1], ey, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(g["p0"][0], ax, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g["p0"][1], ay, rtol=1e-12, atol=1e-14)
