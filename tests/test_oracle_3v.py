"""Pins for the oracle's 2D-3V and multi-species paths (oracle.pic with vdim = 3 and a
species table).

Section 2.2 writes the particle equations with three-component P and A and each
particle's own charge and mass; section 2.1 sums the densities over species.  On the
plane d/dz = 0, so A_z obeys its own wave equation with source mu0 J_z, P_z is constant
and B = (dA_z/dy, -dA_z/dx, B_z).  Pinned by:
  * reductions: v_z = 0 gives the 2D-2V run exactly; a one-entry species table is the
    single species; splitting particles between two identical species changes nothing;
  * the invariance q -> a q, m -> a m, w -> w / a of one species (same q/m, same q w):
    identical positions, velocities and fields, momenta scaled by a;
  * P_z conserved exactly by every particle;
  * gauge and continuity residuals at roundoff (the theorems of section 3 do not involve
    A_z), Gauss too for BDF-k;
  * the cold transverse plasma oscillation: particles on a uniform lattice streaming
    along z make a uniform J_z, and the k = 0 mode of A_z oscillates with
    w^2 = sum_s w_ps^2 / gamma_s (w_ps^2 = n_s q_s^2 / (eps0 m_s)), so v_z = v0 cos(w t) --
    a check of the z deposit, the A_z update, the 3V push and the species sum;
  * the k = 0 mode has no preferred transverse direction: a uniform stream along z evolves
    exactly like the same stream along x in 2D-2V.
"""
import dataclasses

import numpy as np
import pytest

from oracle import pic, steppers


def _cfg(**kw):
    base = dict(nx=16, ny=12, lx=1.0, ly=0.75, dt=0.02, p=3, stepper="bdf", bdf_order=2,
                w=1.0 / 400)
    base.update(kw)
    return pic.Config(**base)


STEPPERS = [dict(stepper="bdf", bdf_order=2), dict(stepper="cdf2"),
            dict(stepper="dirk", dirk=steppers.DIRK2_QIN_ZHANG)]
IDS = ["bdf2", "cdf2", "dirk2"]


def _particles(n, seed, lx=1.0, ly=0.75, vz_scale=0.2):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, lx, n)
    y = rng.uniform(0, ly, n)
    vx = 0.2 * rng.standard_normal(n) / 2
    vy = 0.2 * rng.standard_normal(n) / 2
    vz = vz_scale * rng.standard_normal(n) / 2
    sp = (np.arange(n) % 2).astype(np.int64)
    return x, y, vx, vy, vz, sp


@pytest.mark.parametrize("kw", STEPPERS, ids=IDS)
def test_zero_vz_reduces_to_2d2v(kw):
    cfg2 = _cfg(**kw)
    cfg3 = dataclasses.replace(cfg2, vdim=3)
    x, y, vx, vy, _, _ = _particles(400, 1)
    a = pic.run(cfg2, x, y, vx, vy, 6)
    b = pic.run(cfg3, x, y, vx, vy, 6, vz0=np.zeros(400))
    for k in ("x", "y", "px", "py", "vx", "vy", "vx_old", "vy_old"):
        np.testing.assert_allclose(getattr(b, k), getattr(a, k), rtol=0, atol=1e-15)
    assert np.all(b.pz == 0.0) and np.all(b.vz == 0.0)
    assert np.all(b.grids["az"] == 0.0)
    for f in ("phi", "ax", "ay", "bz"):
        np.testing.assert_allclose(b.grids[f], a.grids[f], rtol=0, atol=1e-15)


@pytest.mark.parametrize("kw", STEPPERS, ids=IDS)
def test_species_table_reductions(kw):
    cfg = _cfg(**kw, vdim=3)
    x, y, vx, vy, vz, sp = _particles(400, 2)
    ref = pic.run(cfg, x, y, vx, vy, 5, vz0=vz)
    one = dataclasses.replace(cfg, species=((cfg.q, cfg.m, cfg.w),))
    two = dataclasses.replace(cfg, species=((cfg.q, cfg.m, cfg.w), (cfg.q, cfg.m, cfg.w)))
    for c, s in ((one, np.zeros(400, dtype=np.int64)), (two, sp)):
        got = pic.run(c, x, y, vx, vy, 5, vz0=vz, species=s)
        for k in ("x", "y", "px", "py", "pz", "vx", "vy", "vz"):
            np.testing.assert_allclose(getattr(got, k), getattr(ref, k), rtol=0, atol=1e-14)
        for f in ("phi", "ax", "ay", "az", "bz"):
            np.testing.assert_allclose(got.grids[f], ref.grids[f], rtol=0, atol=1e-13)


@pytest.mark.parametrize("kw", STEPPERS, ids=IDS)
def test_charge_mass_weight_scaling_of_a_species(kw):
    # species 1 with (a q, a m, w / a): same q/m and the same charge per macro-particle
    base = _cfg(**kw, vdim=3)
    a = 3.0
    c1 = dataclasses.replace(base, species=((-1.0, 1.0, base.w), (1.0, 4.0, base.w)))
    c2 = dataclasses.replace(base, species=((-1.0, 1.0, base.w), (a, 4.0 * a, base.w / a)))
    x, y, vx, vy, vz, sp = _particles(400, 3)
    r1 = pic.run(c1, x, y, vx, vy, 5, vz0=vz, species=sp)
    r2 = pic.run(c2, x, y, vx, vy, 5, vz0=vz, species=sp)
    for k in ("x", "y", "vx", "vy", "vz"):
        np.testing.assert_allclose(getattr(r2, k), getattr(r1, k), rtol=1e-13, atol=1e-15)
    scale = np.where(sp == 1, a, 1.0)
    for k in ("px", "py", "pz"):
        np.testing.assert_allclose(getattr(r2, k), scale * getattr(r1, k), rtol=1e-13, atol=1e-15)
    for f in ("phi", "ax", "ay", "az", "bz"):
        np.testing.assert_allclose(r2.grids[f], r1.grids[f], rtol=1e-12,
                                   atol=1e-12 * np.max(np.abs(r1.grids[f])))


@pytest.mark.parametrize("kw", STEPPERS, ids=IDS)
def test_pz_is_conserved_and_residuals_vanish(kw):
    cfg = _cfg(**kw, vdim=3, species=((-1.0, 1.0, 1.0 / 400), (1.0, 5.0, 1.0 / 400)))
    x, y, vx, vy, vz, sp = _particles(400, 4, vz_scale=0.4)
    st = pic.initial_state(cfg, x, y, vx, vy, vz0=vz, species=sp)
    pz0 = st.pz.copy()
    for _ in range(6):
        pic.step(cfg, st)
        res = pic.residual_norms(cfg, st)
        scale = np.max(np.abs(st.grids["rho"])) + 1.0
        assert res["gauge"][0] <= 1e-12 * scale, res
        assert res["continuity"][0] <= 1e-12 * scale / cfg.dt, res
        if cfg.stepper == "bdf":
            assert res["gauss"][0] <= 1e-12 * scale, res
    assert np.array_equal(st.pz, pz0)
    assert np.max(np.abs(st.grids["az"])) > 0.0
    e = pic.energies(cfg, st)
    assert e["wb"] > 0 and e["we"] > 0 and e["ke"] > 0


def _lattice(nx, ny, lx, ly, per_axis=2):
    # per_axis^2 particles per cell at fixed offsets: the B-spline sums are uniform
    ix = (np.arange(nx * per_axis) + 0.5) * lx / (nx * per_axis)
    iy = (np.arange(ny * per_axis) + 0.5) * ly / (ny * per_axis)
    X, Y = np.meshgrid(ix, iy, indexing="ij")
    return X.ravel(), Y.ravel()


def _oscillation_frequency(t, v):
    # zero crossings of v (linear interpolation) -> mean half period
    s = np.sign(v)
    idx = np.where(s[:-1] * s[1:] < 0)[0]
    tz = t[idx] - v[idx] * (t[idx + 1] - t[idx]) / (v[idx + 1] - v[idx])
    return np.pi / np.mean(np.diff(tz))


@pytest.mark.parametrize("kw", [dict(stepper="cdf2"), dict(stepper="bdf", bdf_order=2)],
                         ids=["cdf2", "bdf2"])
def test_transverse_plasma_oscillation(kw):
    nx, ny, lx, ly = 8, 8, 1.0, 1.0
    x, y = _lattice(nx, ny, lx, ly)
    n = len(x)
    w = lx * ly / n                      # omega_p = 1 for |q| = m = 1 at this weight
    v0 = 0.01
    dt = 0.02
    # one species: electrons streaming along +z
    cfg = _cfg(nx=nx, ny=ny, lx=lx, ly=ly, dt=dt, p=3, vdim=3, w=w, **kw)
    st = pic.initial_state(cfg, x, y, np.zeros(n), np.zeros(n), vz0=np.full(n, v0))
    t, vz = [], []
    for k in range(700):
        pic.step(cfg, st)
        t.append((k + 1) * dt)
        vz.append(st.vz[0])
    assert np.ptp(st.vz) <= 1e-12 * v0     # the particles move in lockstep
    g0 = 1.0 / np.sqrt(1.0 - v0 * v0)
    wexp = 1.0 / np.sqrt(g0)
    assert abs(_oscillation_frequency(np.array(t), np.array(vz)) / wexp - 1.0) < 2e-3
    # two species: electrons (+z) and ions of mass 4 (-z), equal densities
    sp = (np.arange(n) % 2).astype(np.int64)
    cfg2 = dataclasses.replace(cfg, species=((-1.0, 1.0, 2 * w), (1.0, 4.0, 2 * w)))
    vz0 = np.where(sp == 0, v0, -v0 / 4)
    st = pic.initial_state(cfg2, x, y, np.zeros(n), np.zeros(n), vz0=vz0, species=sp)
    t, ve = [], []
    for k in range(700):
        pic.step(cfg2, st)
        t.append((k + 1) * dt)
        ve.append(st.vz[0])
    # w^2 = w_pe^2/gamma_e + w_pi^2/gamma_i with w_pe^2 = 1 (half the particles at twice
    # the weight) and w_pi^2 = 1/4
    gi = 1.0 / np.sqrt(1.0 - (v0 / 4) ** 2)
    wexp = np.sqrt(1.0 / g0 + 0.25 / gi)
    assert abs(_oscillation_frequency(np.array(t), np.array(ve)) / wexp - 1.0) < 2e-3


@pytest.mark.parametrize("kw", [dict(stepper="cdf2"), dict(stepper="bdf", bdf_order=2),
                                dict(stepper="dirk", dirk=steppers.DIRK2_QIN_ZHANG)],
                         ids=["cdf2", "bdf2", "dirk2"])
def test_uniform_z_stream_matches_uniform_x_stream(kw):
    # the k = 0 mode has no preferred transverse direction: a uniform stream along z
    # (2D-3V, A_z) evolves exactly like the same stream along x (2D-2V, A_x)
    x, y = _lattice(8, 8, 1.0, 1.0)
    n = len(x)
    cfg2 = _cfg(nx=8, ny=8, lx=1.0, ly=1.0, dt=0.02, p=3, w=1.0 / n, **kw)
    cfg3 = dataclasses.replace(cfg2, vdim=3)
    v0 = 0.01
    a = pic.initial_state(cfg2, x, y, np.full(n, v0), np.zeros(n))
    b = pic.initial_state(cfg3, x, y, np.zeros(n), np.zeros(n), vz0=np.full(n, v0))
    for _ in range(60):
        pic.step(cfg2, a)
        pic.step(cfg3, b)
        assert abs(b.vz[0] - a.vx[0]) <= 1e-17 + 1e-14 * abs(a.vx[0])
        assert abs(b.pz[0] - a.px[0]) <= 1e-16
    np.testing.assert_allclose(b.grids["az"], a.grids["ax"], rtol=0, atol=1e-16)
