"""Pins for oracle.pic.energies: the field and kinetic energies against closed forms.

The GPU's diagnostics are compared with oracle.pic.energies, so each of its three sums
is fixed here by something outside the oracle:

  * W_B and W_E of single Fourier modes carried through one field solve, where the
    implicit update of a static history is known in closed form (section 3.2, BDF-1:
    u^{n+1} = u^n / (1 + (c dt)^2 K) with no source), and B = curl A, E = -grad phi - dA/dt
    (section 2.2) give the energies as sums of cos^2 over whole periods;
  * the kinetic energy sum_p w_p m_p c^2 (gamma_p - 1) of particles at chosen speeds, with
    one species and with a species table;
  * the k = 0 cold-plasma oscillation, where all of the initial kinetic energy turns into
    electric field energy and back, so the two exchange equal amounts and their sum stays
    constant as dt -> 0.

c and eps0 differ from 1 throughout, so a misplaced mu0 = 1/(eps0 c^2), eps0 or c^2 changes
the result.
"""
import numpy as np
import pytest

from oracle import pic, spectral, steppers

C, EPS0 = 2.0, 0.5          # mu0 = 1 / (eps0 c^2) = 0.5
NX, NY, LX, LY = 16, 8, 1.3, 0.9


def _cfg(**kw):
    base = dict(nx=NX, ny=NY, lx=LX, ly=LY, dt=0.01, p=2, stepper="bdf", bdf_order=1,
                c=C, eps0=EPS0, w=0.3, m=1.7, q=-1.0)
    base.update(kw)
    return pic.Config(**base)


def _nodes(cfg):
    X = (np.arange(cfg.nx) * cfg.dx)[:, None] * np.ones((1, cfg.ny))
    Y = np.ones((cfg.nx, 1)) * (np.arange(cfg.ny) * cfg.dy)[None, :]
    return X, Y


def _empty_state(cfg, levels):
    e = np.zeros(0)
    st = pic.State(x=e, y=e, px=e, py=e, vx=e, vy=e, vx_old=e, vy_old=e)
    st.hist = levels
    if cfg.vdim == 3:
        st.pz, st.vz, st.vz_old = e, e, e
    return st


def test_single_mode_field_energies_bdf1():
    # History: A_y = a sin(k_x x) and phi = b cos(k_y y) at both BDF-1 levels, rho = 0,
    # no particles (J = 0).  Then rho^{n+1} = 0, and with C = (1, -2, 1)
    #   u^{n+1} = (2 u^n - u^{n-1}) / (1 + g K) = u0 / (1 + g K),  g = (c dt)^2,
    # so B_z = d_x A_y = a k_x cos(k_x x) / (1 + g Kx) and
    #   E_y = -d_y phi - (A_y^{n+1} - A_y^n)/dt
    #       = b k_y sin(k_y y)/(1 + g Ky) + a g Kx sin(k_x x) / ((1 + g Kx) dt).
    # Over whole periods sum cos^2 = sum sin^2 = N/2 and the cross term sums to zero:
    #   W_B = (a k_x/(1 + g Kx))^2 Lx Ly / (4 mu0)
    #   W_E = eps0/2 (Lx Ly/2) [(b k_y/(1 + g Ky))^2 + (a g Kx/((1 + g Kx) dt))^2].
    cfg = _cfg()
    X, Y = _nodes(cfg)
    kx, ky = 2 * np.pi * 2 / LX, 2 * np.pi / LY
    a, b = 0.7, -0.4
    ay0 = spectral.dft2(a * np.sin(kx * X))
    phi0 = spectral.dft2(b * np.cos(ky * Y))
    z = np.zeros((NX, NY), dtype=complex)
    st = _empty_state(cfg, {"phi": [phi0.copy(), phi0.copy()], "ax": [z.copy(), z.copy()],
                            "ay": [ay0.copy(), ay0.copy()], "rho": [z.copy()]})
    zero = np.zeros((NX, NY))
    pic.field_solve(cfg, st, zero, zero)
    e = pic.energies(cfg, st)
    g = (C * cfg.dt) ** 2
    Kx, Ky = kx * kx, ky * ky
    mu0 = 1.0 / (EPS0 * C * C)
    wb = (a * kx / (1 + g * Kx)) ** 2 * LX * LY / (4 * mu0)
    we = 0.5 * EPS0 * (LX * LY / 2) * ((b * ky / (1 + g * Ky)) ** 2
                                       + (a * g * Kx / ((1 + g * Kx) * cfg.dt)) ** 2)
    assert e["wb"] == pytest.approx(wb, rel=1e-12)
    assert e["we"] == pytest.approx(we, rel=1e-12)
    assert e["ke"] == 0.0


def test_curl_free_vector_potential_has_no_magnetic_energy():
    # A = grad psi with psi = s sin(k_x x + k_y y): B_z = d_x A_y - d_y A_x = 0, and the
    # static BDF-1 update scales both components of the mode alike, so B stays zero;
    # W_E = eps0/2 (Lx Ly/2) (s |k| g K/((1 + g K) dt))^2 from -dA/dt alone.
    cfg = _cfg()
    X, Y = _nodes(cfg)
    kx, ky = 2 * np.pi / LX, 2 * np.pi * 2 / LY
    s = 0.2
    ax0 = spectral.dft2(s * kx * np.cos(kx * X + ky * Y))
    ay0 = spectral.dft2(s * ky * np.cos(kx * X + ky * Y))
    z = np.zeros((NX, NY), dtype=complex)
    st = _empty_state(cfg, {"phi": [z.copy(), z.copy()], "ax": [ax0.copy(), ax0.copy()],
                            "ay": [ay0.copy(), ay0.copy()], "rho": [z.copy()]})
    zero = np.zeros((NX, NY))
    pic.field_solve(cfg, st, zero, zero)
    e = pic.energies(cfg, st)
    g, K = (C * cfg.dt) ** 2, kx * kx + ky * ky
    we = 0.5 * EPS0 * (LX * LY / 2) * (s * np.sqrt(K) * g * K / ((1 + g * K) * cfg.dt)) ** 2
    assert e["wb"] < 1e-28 * we
    assert e["we"] == pytest.approx(we, rel=1e-12)


def test_single_mode_field_energies_cdf2():
    # CDF-2 implicit with a static history (u^{n+1/2} = u^{n-1/2} = u0) and no sources:
    #   u^{new} = 2 u0 / (1 + th K) - u0 = u0 (1 - th K)/(1 + th K),  th = (c dt)^2 / 2.
    # The diagnostic E (at t^{n+1/2}) is
    #   -grad (phi^{n+3/2} + phi^{n-1/2})/2 - (A^{n+1} - A^n)/dt,
    # with phi^{n-1/2} = phi0: so E_y = b k_y sin(k_y y) (r_y + 1)/2 - a (r_x - 1) sin(k_x x)/dt,
    # r = (1 - th K)/(1 + th K); B_z = a k_x r_x cos(k_x x).
    cfg = _cfg(stepper="cdf2")
    X, Y = _nodes(cfg)
    kx, ky = 2 * np.pi / LX, 2 * np.pi * 3 / LY
    a, b = -0.25, 0.9
    ay0 = spectral.dft2(a * np.sin(kx * X))
    phi0 = spectral.dft2(b * np.cos(ky * Y))
    z = np.zeros((NX, NY), dtype=complex)
    st = _empty_state(cfg, {"phi": phi0.copy(), "phi_prev": phi0.copy(), "rho": z.copy(),
                            "rho_prev": z.copy(), "ax": z.copy(), "ax_prev": z.copy(),
                            "ay": ay0.copy(), "ay_prev": ay0.copy(), "jx": z.copy(),
                            "jx_prev": z.copy(), "jy": z.copy(), "jy_prev": z.copy()})
    zero = np.zeros((NX, NY))
    pic.field_solve(cfg, st, zero, zero)
    e = pic.energies(cfg, st)
    th = (C * cfg.dt) ** 2 / 2
    rx = (1 - th * kx * kx) / (1 + th * kx * kx)
    ry = (1 - th * ky * ky) / (1 + th * ky * ky)
    mu0 = 1.0 / (EPS0 * C * C)
    wb = (a * kx * rx) ** 2 * LX * LY / (4 * mu0)
    we = 0.5 * EPS0 * (LX * LY / 2) * ((b * ky * (ry + 1) / 2) ** 2
                                       + (a * (rx - 1) / cfg.dt) ** 2)
    assert e["wb"] == pytest.approx(wb, rel=1e-12)
    assert e["we"] == pytest.approx(we, rel=1e-12)


def test_single_mode_field_energies_3v():
    # 2D-3V, BDF-1: A_z = a sin(k_x x) at both levels and no current.  A_z^{n+1} =
    # A_z0/(1 + g K), so B_y = -d_x A_z = -a k_x cos(k_x x)/(1 + g K) (B_x = d_y A_z = 0)
    # and E_z = -(A_z^{n+1} - A_z^n)/dt = a g K sin(k_x x)/((1 + g K) dt).
    cfg = _cfg(vdim=3)
    X, _ = _nodes(cfg)
    kx = 2 * np.pi * 3 / LX
    a = 0.35
    az0 = spectral.dft2(a * np.sin(kx * X))
    z = np.zeros((NX, NY), dtype=complex)
    st = _empty_state(cfg, {"phi": [z.copy(), z.copy()], "ax": [z.copy(), z.copy()],
                            "ay": [z.copy(), z.copy()], "rho": [z.copy()],
                            "az": [az0.copy(), az0.copy()]})
    zero = np.zeros((NX, NY))
    pic.field_solve(cfg, st, zero, zero, jz=zero)
    e = pic.energies(cfg, st)
    g = (C * cfg.dt) ** 2
    K = kx * kx
    mu0 = 1.0 / (EPS0 * C * C)
    assert e["wb"] == pytest.approx((a * kx / (1 + g * K)) ** 2 * LX * LY / (4 * mu0), rel=1e-12)
    assert e["we"] == pytest.approx(0.5 * EPS0 * (LX * LY / 2)
                                    * (a * g * K / ((1 + g * K) * cfg.dt)) ** 2, rel=1e-12)


def _state_with_speeds(cfg, speeds, angles, vz=None):
    v = np.asarray(speeds) * C
    st = _empty_state(cfg, {})
    st.vx, st.vy = v * np.cos(angles), v * np.sin(angles)
    if vz is not None:
        st.vz = np.asarray(vz)
    zero = np.zeros((NX, NY))
    st.grids = {"bz": zero, "ex": zero, "ey": zero, "bx": zero, "by": zero, "ez": zero}
    return st


def test_kinetic_energy_one_species():
    # |v| = 0.6 c: gamma = 5/4; 0.8 c: 5/3; 0: 1.  KE = sum w m c^2 (gamma - 1).
    cfg = _cfg()
    st = _state_with_speeds(cfg, [0.6, 0.8, 0.0, 0.6], [0.3, 2.0, 0.0, -1.1])
    ke = 0.3 * 1.7 * C * C * (0.25 + 2.0 / 3.0 + 0.0 + 0.25)
    e = pic.energies(cfg, st)
    assert e["ke"] == pytest.approx(ke, rel=1e-14)
    assert e["wb"] == 0.0 and e["we"] == 0.0


def test_kinetic_energy_species_table_and_vz():
    # Two species (q, m, w): each particle weighs w_s m_s; in 2D-3V |v| includes v_z.
    tab = ((-1.0, 1.0, 0.5), (1.0, 4.0, 0.25))
    cfg = _cfg(species=tab, vdim=3)
    # (0.6 c in the plane, 0.8 c along z): |v| = c, excluded; use 0.36 c and 0.48 c -> 0.6 c
    st = _state_with_speeds(cfg, [0.36, 0.8, 0.6], [0.0, 1.0, 2.5],
                            vz=np.array([0.48, 0.0, 0.0]) * C)
    st.sp = np.array([0, 1, 1])
    ke = C * C * (0.5 * 1.0 * 0.25 + 0.25 * 4.0 * (2.0 / 3.0) + 0.25 * 4.0 * 0.25)
    assert pic.energies(cfg, st)["ke"] == pytest.approx(ke, rel=1e-14)


def _lattice(nx, ny, lx, ly, sub):
    gx = (np.arange(nx * sub) + 0.5) * lx / (nx * sub)
    gy = (np.arange(ny * sub) + 0.5) * ly / (ny * sub)
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    return X.ravel(), Y.ravel()


@pytest.mark.parametrize("stepper", ["cdf2", "bdf", "dirk"])
def test_uniform_oscillation_exchanges_kinetic_and_electric_energy(stepper):
    # Cold electrons all drifting at v0 along x: the k = 0 mode of A_x oscillates and the
    # whole kinetic energy KE0 = sum w m c^2 (gamma0 - 1) passes into the uniform electric
    # field and back (no B: a uniform A has no curl).  The discrete energies carry an
    # O(dt) error (the IAEM push couples particles and fields at first order), so the
    # checks are on values extrapolated to dt -> 0 from dt and dt/2:
    #   peak-to-peak of KE and of W_E  ->  KE0,   variation of W_E + KE  ->  0.
    nx = ny = 4
    x, y = _lattice(nx, ny, 1.0, 1.0, 2)
    n = len(x)
    v0 = 0.01 * C
    w = EPS0 * 1.0 / n          # omega_pe^2 = n w q^2 / (eps0 m L^2) = 1
    ke0 = n * w * 1.0 * C * C * (1.0 / np.sqrt(1.0 - (v0 / C) ** 2) - 1.0)
    out = []
    for dt in (0.025, 0.0125):
        cfg = pic.Config(nx=nx, ny=ny, lx=1.0, ly=1.0, dt=dt, p=2, stepper=stepper,
                         bdf_order=2, dirk=steppers.DIRK2_QIN_ZHANG, c=C, eps0=EPS0,
                         w=w, m=1.0, q=-1.0)
        st = pic.initial_state(cfg, x, y, np.full(n, v0), np.zeros(n))
        ke, we, wb = [ke0], [], []
        for _ in range(int(round(8.0 / dt))):   # more than one period 2 pi
            pic.step(cfg, st)
            e = pic.energies(cfg, st)
            ke.append(e["ke"])
            we.append(e["we"])
            wb.append(e["wb"])
        ke, we = np.array(ke), np.array(we)
        assert max(wb) < 1e-20 * ke0
        tot = we + 0.5 * (ke[1:] + ke[:-1])     # KE at t^{n+1/2}, where W_E sits
        out.append((np.ptp(ke), np.ptp(we), np.ptp(tot)))
    (k1, e1, t1), (k2, e2, t2) = out
    assert 2 * k2 - k1 == pytest.approx(ke0, rel=0.06)
    assert 2 * e2 - e1 == pytest.approx(ke0, rel=0.06)
    assert abs(2 * t2 - t1) < 0.05 * ke0
    assert t2 < 0.6 * t1                        # the variation falls with dt
