"""Whole PIC step of the gauge-conserving method, FP64 (oracle; test infrastructure only).

Section 4.2 (Algorithm 1) advances, per time step:
  1. positions  x^{n+1} = x^n + v^n dt                        (IAEM, section 4.1)
  2. current    J^{n+1} deposited with x^{n+1} and v^n       (section 4, B-spline shape)
  3. charge     rho from the continuity equation of the stepper in use
  4. potentials phi, A at the new level by the spectral implicit wave solve
  5. gradients  grad phi, grad A computed spectrally
  6. gather     grad phi~, A, grad A at the particles with the same shape
  7. push       v* = 2 v^n - v^{n-1};  P^{n+1} = P^n + q(-grad phi~ + grad A . v*) dt;
                v^{n+1} = c^2 (P - qA) / sqrt(c^2 |P - qA|^2 + (m c^2)^2)
  8. shift the time histories.

Units: the caller fixes c, eps0 (mu0 = 1/(eps0 c^2)), the physical charge q and mass m
of one electron, and the macro-particle weight w: a macro-particle carries charge
w q (what is deposited) and mass w m, so only q/m enters the push.  Grid densities
are per unit area: node (i, j) receives q_p W(x/dx - i) W(y/dy - j) / (dx dy).

Readings of points the paper leaves open (each also listed in the design notes):
  * v^n (not v*) is deposited (section 4: the paper found no difference).
  * Initial state (Algorithm 1 gives only "x^0, P^0, v^0 and the fields"):
    rho^0 = deposited charge with its K = 0 modes set to zero -- the k = 0 mode is
    the uniform neutralising ion background, and the Nyquist-corner modes are the
    ones the spectral divergence cannot reach, so Poisson's equation (and hence the
    residual-free start the theorems assume) can hold exactly;
    phi^0 solves Poisson; A^0 = 0; P^0 = gamma m v^0; every history level of phi, A
    and rho equals its t = 0 value, time derivatives (DIRK) are zero, and the current
    history (CDF J^{n-1}, DIRK J^n) is zero.  v^{-1} is a first-order Taylor step
    back in the t = 0 electric field E^0 = -grad phi^0:
        v^{-1} = v^0 - dt (q/(gamma m)) (E^0 - v^0 (v^0 . E^0)/c^2).
  * BDF continuity uses the form of section 3.2 (the algorithm box prints it with
    other signs); CDF particles use phi~ = (phi^{n+3/2} + phi^{n+1/2})/2.
  * Positions wrap into [0, L) after the move; node indices wrap modulo N.
"""
import dataclasses
from dataclasses import dataclass, field

import numpy as np

from . import bspline, spectral, steppers

FIELD_NAMES = ("dphidx", "dphidy", "ax", "ay", "daxdx", "daxdy", "daydx", "daydy")
# 2D-3V adds the z potential and its in-plane gradient (d/dz = 0 on the plane)
FIELD_NAMES_Z = ("az", "dazdx", "dazdy")


@dataclass
class Config:
    nx: int
    ny: int
    lx: float
    ly: float
    dt: float
    p: int = 2                      # spline degree
    stepper: str = "bdf"            # "bdf" | "cdf2" | "dirk"
    bdf_order: int = 1
    dirk: dict = None               # {"A": [[..]], "b": [..], "c": [..]}
    cdf_form: str = "implicit"      # CDF-2 only: "implicit" | "semi" | "explicit" (section 3.1)
    charge: str = "continuity"      # "continuity" | "deposit" (the naive update of section 5)
    c: float = 1.0
    eps0: float = 1.0
    q: float = -1.0
    m: float = 1.0
    w: float = 1.0                  # macro-particle weight
    vdim: int = 2                   # velocity components: 2 (2D-2V) or 3 (2D-3V)
    species: tuple = None           # ((q, m, w), ...) per species, or None: one species

    def particle_constants(self, sp=None):
        """(q_p = w q, q, m) of each particle.  Section 2.2 writes the equations of motion
        and the densities with the charge q_i and mass m_i of each particle, and section
        2.1 sums the densities over species; with a species table the values come per
        particle from its species index sp, else they are the single species' scalars."""
        if self.species is None:
            return self.w * self.q, self.q, self.m
        tab = np.asarray(self.species, dtype=np.float64)
        sp = np.asarray(sp)
        return tab[sp, 2] * tab[sp, 0], tab[sp, 0], tab[sp, 1]

    @property
    def mu0(self):
        return 1.0 / (self.eps0 * self.c * self.c)

    @property
    def dx(self):
        return self.lx / self.nx

    @property
    def dy(self):
        return self.ly / self.ny


@dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    px: np.ndarray
    py: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vx_old: np.ndarray
    vy_old: np.ndarray
    hist: dict = field(default_factory=dict)
    n: int = 0
    grids: dict = field(default_factory=dict)   # last step's grid quantities
    res: dict = field(default_factory=dict)     # last step's residual spectra
    pz: np.ndarray = None                       # 2D-3V: z momentum and velocities
    vz: np.ndarray = None
    vz_old: np.ndarray = None
    sp: np.ndarray = None                       # species index of each particle


# ------------------------------------------------------- particle <-> mesh ----

def deposit(cfg, x, y, values):
    """Grid density sum_p values_p W(x_p/dx - i) W(y_p/dy - j) / (dx dy).

    Section 2.2 (PIC charge/current densities with shape S) and section 4 (tensor
    product of 1-D B-splines).  A direct loop over the (p+1)^2 stencil offsets,
    each a scatter-add over all particles (numpy bincount).
    """
    nx, ny, p = cfg.nx, cfg.ny, cfg.p
    i0, wx = bspline.node_weights(np.asarray(x) / cfg.dx, p)
    j0, wy = bspline.node_weights(np.asarray(y) / cfg.dy, p)
    grid = np.zeros(nx * ny)
    for a in range(p + 1):
        ii = np.mod(i0 + a, nx)
        for b in range(p + 1):
            jj = np.mod(j0 + b, ny)
            grid += np.bincount(ii * ny + jj, weights=values * wx[:, a] * wy[:, b],
                                minlength=nx * ny)
    return grid.reshape(nx, ny) / (cfg.dx * cfg.dy)


def gather(cfg, x, y, grid):
    """sum_{i,j} grid[i, j] W(x_p/dx - i) W(y_p/dy - j): the same shape as deposit (section 4)."""
    nx, ny, p = cfg.nx, cfg.ny, cfg.p
    i0, wx = bspline.node_weights(np.asarray(x) / cfg.dx, p)
    j0, wy = bspline.node_weights(np.asarray(y) / cfg.dy, p)
    out = np.zeros(len(x))
    for a in range(p + 1):
        ii = np.mod(i0 + a, nx)
        for b in range(p + 1):
            jj = np.mod(j0 + b, ny)
            out += grid[ii, jj] * wx[:, a] * wy[:, b]
    return out


def wrap(x, length):
    """Periodic wrap of a position that moved by less than one period."""
    x = np.where(x >= length, x - length, x)
    return np.where(x < 0.0, x + length, x)


def velocity_from_momentum(cfg, px, py, ax, ay):
    """v = c^2 (P - qA) / sqrt(c^2 |P - qA|^2 + (m c^2)^2) (section 2.2; the velocity update of the IAEM scheme)."""
    ux = px - cfg.q * ax
    uy = py - cfg.q * ay
    c2 = cfg.c * cfg.c
    den = np.sqrt(c2 * (ux * ux + uy * uy) + (cfg.m * c2) ** 2)
    return c2 * ux / den, c2 * uy / den


def iaem_push(cfg, st, g):
    """IAEM momentum and velocity update (section 4.1) with gathered fields g.

    g holds the eight gathered quantities of FIELD_NAMES; (grad A . v*)_l is
    sum_m (d_l A_m) v*_m.  v^{n+1} overwrites v^n and v^n becomes v^{n-1}.
    """
    if cfg.vdim == 3 or cfg.species is not None:
        return iaem_push_general(cfg, st, g)
    dt, q = cfg.dt, cfg.q
    vsx = 2.0 * st.vx - st.vx_old
    vsy = 2.0 * st.vy - st.vy_old
    st.px = st.px + q * dt * (-g["dphidx"] + g["daxdx"] * vsx + g["daydx"] * vsy)
    st.py = st.py + q * dt * (-g["dphidy"] + g["daxdy"] * vsx + g["daydy"] * vsy)
    vx_new, vy_new = velocity_from_momentum(cfg, st.px, st.py, g["ax"], g["ay"])
    st.vx_old, st.vy_old = st.vx, st.vy
    st.vx, st.vy = vx_new, vy_new


# ------------------------------------------------------------ field solve ----

def iaem_push_general(cfg, st, g):
    """The IAEM update of section 4.1 with per-particle charges and masses (section 2.2)
    and, in 2D-3V, three momentum components: (grad A . v*)_l = sum_{m=x,y,z} d_l A_m v*_m
    for l = x, y, and d/dz = 0 leaves P_z unchanged; u = P - q A has three components and
    v = c^2 u / sqrt(c^2 |u|^2 + (m c^2)^2)."""
    _, q, m = cfg.particle_constants(st.sp)
    dt, c2 = cfg.dt, cfg.c * cfg.c
    three = cfg.vdim == 3
    vsx = 2.0 * st.vx - st.vx_old
    vsy = 2.0 * st.vy - st.vy_old
    fx = -g["dphidx"] + g["daxdx"] * vsx + g["daydx"] * vsy
    fy = -g["dphidy"] + g["daxdy"] * vsx + g["daydy"] * vsy
    if three:
        vsz = 2.0 * st.vz - st.vz_old
        fx = fx + g["dazdx"] * vsz
        fy = fy + g["dazdy"] * vsz
    st.px = st.px + q * dt * fx
    st.py = st.py + q * dt * fy
    ux = st.px - q * g["ax"]
    uy = st.py - q * g["ay"]
    u2 = ux * ux + uy * uy
    if three:
        uz = st.pz - q * g["az"]
        u2 = u2 + uz * uz
    den = np.sqrt(c2 * u2 + (m * c2) ** 2)
    st.vx_old, st.vy_old = st.vx, st.vy
    st.vx, st.vy = c2 * ux / den, c2 * uy / den
    if three:
        st.vz_old = st.vz
        st.vz = c2 * uz / den


def _k(cfg):
    return spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)


def _grid_fields(cfg, phi_hat, ax_hat, ay_hat):
    """The eight real mesh fields gathered by the particles (Algorithm 1, gradient step)."""
    kx, ky, _ = _k(cfg)
    spectra = {
        "dphidx": 1j * kx * phi_hat, "dphidy": 1j * ky * phi_hat,
        "ax": ax_hat, "ay": ay_hat,
        "daxdx": 1j * kx * ax_hat, "daxdy": 1j * ky * ax_hat,
        "daydx": 1j * kx * ay_hat, "daydy": 1j * ky * ay_hat,
    }
    return {name: spectral.idft2(s).real for name, s in spectra.items()}


def _grid_fields_z(cfg, az_hat):
    """A_z and its in-plane gradient on the mesh (2D-3V)."""
    kx, ky, _ = _k(cfg)
    spectra = {"az": az_hat, "dazdx": 1j * kx * az_hat, "dazdy": 1j * ky * az_hat}
    return {name: spectral.idft2(s).real for name, s in spectra.items()}


def deposited_charge_hat(cfg, x, y, sp=None):
    """Spectrum of the charge deposited at the given positions, its K = 0 modes removed
    as at t = 0 (reading R15): rho^{n+1} of the naive update that section 5 compares
    against (both rho and J mapped to the mesh with the particle shape)."""
    kx, ky, K = _k(cfg)
    qp = cfg.particle_constants(sp)[0] * np.ones(len(x))
    rho_hat = spectral.dft2(deposit(cfg, x, y, qp))
    rho_hat[K == 0.0] = 0.0
    return rho_hat


def field_solve(cfg, st, jx, jy, rho_dep_hat=None, jz=None):
    """Continuity + implicit wave solve + spectral gradients for the new J (Algorithm 1).

    Updates st.hist, records residual spectra in st.res (before the history shift,
    so every level a residual needs is still there) and returns the eight mesh
    fields the particles gather.  With cfg.charge == "deposit" (BDF-k and DIRK only),
    rho^{n+1} is rho_dep_hat, the deposited charge, instead of the continuity update.
    In 2D-3V (jz given) A_z follows the same stepper with the source mu0 J_z and the
    three A_z fields are returned too; A_z is in neither the continuity equation nor the
    gauge (d/dz = 0), and E_z = -dA_z/dt is the stepper's discrete derivative (BDF: the
    BDF difference, CDF-2: the centred difference at n+1/2, DIRK: -v_Az).
    """
    if cfg.charge == "deposit" and (rho_dep_hat is None or cfg.stepper == "cdf2"):
        raise ValueError("the deposited-charge update needs rho_dep_hat and a BDF or DIRK stepper")
    kx, ky, K = _k(cfg)
    c, dt, eps0, mu0 = cfg.c, cfg.dt, cfg.eps0, cfg.mu0
    h = st.hist
    jx_hat = spectral.dft2(jx)
    jy_hat = spectral.dft2(jy)
    divj = spectral.div_hat(jx_hat, jy_hat, kx, ky)
    res = {}

    if cfg.stepper == "bdf":
        a, beta = steppers.bdf_coefficients(cfg.bdf_order)
        C = steppers.bdf_second_derivative_coefficients(a)
        bdt = float(beta) * dt
        rho_new = steppers.bdf_continuity(h["rho"], divj, dt, a, beta)
        if cfg.charge == "deposit":
            rho_new = rho_dep_hat
        phi_new = steppers.bdf_wave_update(h["phi"], rho_new / eps0, K, c, dt, beta, C)
        ax_new = steppers.bdf_wave_update(h["ax"], mu0 * jx_hat, K, c, dt, beta, C)
        ay_new = steppers.bdf_wave_update(h["ay"], mu0 * jy_hat, K, c, dt, beta, C)
        phis = [phi_new] + h["phi"]
        axs = [ax_new] + h["ax"]
        ays = [ay_new] + h["ay"]
        rhos = [rho_new] + h["rho"]
        dphi = sum(float(a[j]) * phis[j] for j in range(len(a)))
        dax = sum(float(a[j]) * axs[j] for j in range(len(a)))
        day = sum(float(a[j]) * ays[j] for j in range(len(a)))
        drho = sum(float(a[j]) * rhos[j] for j in range(len(a)))
        div_a = spectral.div_hat(ax_new, ay_new, kx, ky)
        # section 3.2: gauge and continuity residuals; Gauss with E^{n+1} = -grad phi - D_BDF A
        res["gauge"] = dphi / (c * c * bdt) + div_a
        res["continuity"] = drho / bdt + divj
        ex_hat = -1j * kx * phi_new - dax / bdt
        ey_hat = -1j * ky * phi_new - day / bdt
        res["gauss"] = spectral.div_hat(ex_hat, ey_hat, kx, ky) - rho_new / eps0
        res["ex"], res["ey"] = ex_hat, ey_hat
        if jz is not None:
            jz_hat = spectral.dft2(jz)
            az_new = steppers.bdf_wave_update(h["az"], mu0 * jz_hat, K, c, dt, beta, C)
            azs = [az_new] + h["az"]
            res["ez"] = -sum(float(a[j]) * azs[j] for j in range(len(a))) / bdt
            h["az"] = azs[:-1]
        h["phi"] = phis[:-1]
        h["ax"] = axs[:-1]
        h["ay"] = ays[:-1]
        h["rho"] = rhos[:-1]
        phi_part = phi_new
        rho_out, phi_out = rho_new, phi_new

    elif cfg.stepper == "cdf2":
        rho_new = steppers.cdf2_continuity(h["rho"], divj, dt)              # rho^{n+3/2}
        if cfg.cdf_form == "implicit":
            phi_new = steppers.cdf2_wave_update(h["phi"], h["phi_prev"], rho_new / eps0,
                                                h["rho_prev"] / eps0, K, c, dt)  # phi^{n+3/2}
            ax_new = steppers.cdf2_wave_update(h["ax"], h["ax_prev"], mu0 * jx_hat,
                                               mu0 * h["jx_prev"], K, c, dt)     # A^{n+1}
            ay_new = steppers.cdf2_wave_update(h["ay"], h["ay_prev"], mu0 * jy_hat,
                                               mu0 * h["jy_prev"], K, c, dt)
        else:  # sources at the middle level: rho^{n+1/2} and J^n
            upd = {"semi": steppers.cdf2_semi_implicit_update,
                   "explicit": steppers.cdf2_explicit_update}[cfg.cdf_form]
            phi_new = upd(h["phi"], h["phi_prev"], h["rho"] / eps0, K, c, dt)
            ax_new = upd(h["ax"], h["ax_prev"], mu0 * h["jx"], K, c, dt)
            ay_new = upd(h["ay"], h["ay_prev"], mu0 * h["jy"], K, c, dt)
        div_a = spectral.div_hat(ax_new, ay_new, kx, ky)
        # section 3.1: eps_1, eps_2 and Gauss at t^{n+1/2} for the implicit scheme
        res["gauge"] = (phi_new - h["phi"]) / (c * c * dt) + div_a
        res["continuity"] = (rho_new - h["rho"]) / dt + divj
        phi_avg = 0.5 * (phi_new + h["phi_prev"])
        ex_hat = -1j * kx * phi_avg - (ax_new - h["ax"]) / dt
        ey_hat = -1j * ky * phi_avg - (ay_new - h["ay"]) / dt
        res["gauss"] = (spectral.div_hat(ex_hat, ey_hat, kx, ky)
                        - 0.5 * (rho_new + h["rho_prev"]) / eps0)
        res["ex"], res["ey"] = ex_hat, ey_hat
        phi_part = 0.5 * (phi_new + h["phi"])                               # phi~ at t^{n+1}
        if jz is not None:
            jz_hat = spectral.dft2(jz)
            if cfg.cdf_form == "implicit":
                az_new = steppers.cdf2_wave_update(h["az"], h["az_prev"], mu0 * jz_hat,
                                                   mu0 * h["jz_prev"], K, c, dt)
            else:
                az_new = upd(h["az"], h["az_prev"], mu0 * h["jz"], K, c, dt)
            res["ez"] = -(az_new - h["az"]) / dt
            h["az_prev"], h["az"] = h["az"], az_new
            h["jz_prev"], h["jz"] = h["jz"], jz_hat
        h["phi_prev"], h["phi"] = h["phi"], phi_new
        h["rho_prev"], h["rho"] = h["rho"], rho_new
        h["ax_prev"], h["ax"] = h["ax"], ax_new
        h["ay_prev"], h["ay"] = h["ay"], ay_new
        h["jx_prev"], h["jx"] = h["jx"], jx_hat
        h["jy_prev"], h["jy"] = h["jy"], jy_hat
        rho_out, phi_out = rho_new, phi_new

    elif cfg.stepper == "dirk":
        A, b, cv = cfg.dirk["A"], cfg.dirk["b"], cfg.dirk["c"]
        divj_n = spectral.div_hat(h["jx"], h["jy"], kx, ky)
        rho_new = steppers.dirk_continuity(h["rho"], divj_n, divj, dt, b, cv)
        if cfg.charge == "deposit":
            rho_new = rho_dep_hat
        phi_new, vphi_new = steppers.dirk_wave_update(
            h["phi"], h["vphi"], h["rho"] / eps0, rho_new / eps0, K, c, dt, A, b, cv)
        ax_new, vax_new = steppers.dirk_wave_update(
            h["ax"], h["vax"], mu0 * h["jx"], mu0 * jx_hat, K, c, dt, A, b, cv)
        ay_new, vay_new = steppers.dirk_wave_update(
            h["ay"], h["vay"], mu0 * h["jy"], mu0 * jy_hat, K, c, dt, A, b, cv)
        r0, r1 = steppers.dirk_interp_weights(b, cv)
        div_a_n = spectral.div_hat(h["ax"], h["ay"], kx, ky)
        div_a = spectral.div_hat(ax_new, ay_new, kx, ky)
        div_va_n = spectral.div_hat(h["vax"], h["vay"], kx, ky)
        div_va = spectral.div_hat(vax_new, vay_new, kx, ky)
        # section 3.3.2: eps_1 (gauge), eps_2 (its time derivative), eps_3 (continuity)
        res["gauge"] = -(phi_new - h["phi"]) - c * c * dt * (r0 * div_a_n + r1 * div_a)
        res["gauge_dt"] = -(vphi_new - h["vphi"]) - c * c * dt * (r0 * div_va_n + r1 * div_va)
        res["continuity"] = -(rho_new - h["rho"]) - dt * (r0 * divj_n + r1 * divj)
        ex_hat = -1j * kx * phi_new - vax_new
        ey_hat = -1j * ky * phi_new - vay_new
        res["gauss"] = spectral.div_hat(ex_hat, ey_hat, kx, ky) - rho_new / eps0
        res["ex"], res["ey"] = ex_hat, ey_hat
        if jz is not None:
            jz_hat = spectral.dft2(jz)
            az_new, vaz_new = steppers.dirk_wave_update(
                h["az"], h["vaz"], mu0 * h["jz"], mu0 * jz_hat, K, c, dt, A, b, cv)
            res["ez"] = -vaz_new
            h.update(az=az_new, vaz=vaz_new, jz=jz_hat)
        h.update(phi=phi_new, vphi=vphi_new, ax=ax_new, vax=vax_new, ay=ay_new,
                 vay=vay_new, rho=rho_new, jx=jx_hat, jy=jy_hat)
        phi_part = phi_new
        rho_out, phi_out = rho_new, phi_new
    else:
        raise ValueError(cfg.stepper)

    st.res = res
    st.grids = {
        "jx": jx, "jy": jy,
        "rho": spectral.idft2(rho_out).real,
        "phi": spectral.idft2(phi_out).real,
        "bz": spectral.idft2(1j * kx * ay_new - 1j * ky * ax_new).real,
        "ex": spectral.idft2(res["ex"]).real,
        "ey": spectral.idft2(res["ey"]).real,
    }
    fields = _grid_fields(cfg, phi_part, ax_new, ay_new)
    if jz is not None:
        az_new = h["az"][0] if cfg.stepper == "bdf" else h["az"]
        st.grids.update(jz=jz, az=spectral.idft2(az_new).real,
                        bx=spectral.idft2(1j * ky * az_new).real,
                        by=spectral.idft2(-1j * kx * az_new).real,
                        ez=spectral.idft2(res["ez"]).real)
        fields.update(_grid_fields_z(cfg, az_new))
    st.grids.update(fields)
    return fields


# ------------------------------------------------------------ init / step ----

def taylor_back_velocity(cfg, vx, vy, ex, ey):
    """v(-dt) to first order for a particle in the field E (B = 0), Algorithm 1 set-up.

    d(gamma m v)/dt = q E gives dv/dt = (q/(gamma m)) (E - v (v . E)/c^2); one explicit
    Taylor step backwards is v - dt dv/dt.
    """
    c2 = cfg.c * cfg.c
    gamma = 1.0 / np.sqrt(1.0 - (vx * vx + vy * vy) / c2)
    vdote = vx * ex + vy * ey
    coef = cfg.dt * cfg.q / (gamma * cfg.m)
    return vx - coef * (ex - vx * vdote / c2), vy - coef * (ey - vy * vdote / c2)


def taylor_back_velocity3(cfg, vx, vy, vz, ex, ey, q, m):
    """The Taylor start of taylor_back_velocity with three velocity components and the
    particles' own charges and masses (E_z = 0 at t = 0: A^0 = 0 and dA_z/dt = 0)."""
    c2 = cfg.c * cfg.c
    gamma = 1.0 / np.sqrt(1.0 - (vx * vx + vy * vy + vz * vz) / c2)
    vdote = vx * ex + vy * ey
    coef = cfg.dt * q / (gamma * m)
    return (vx - coef * (ex - vx * vdote / c2), vy - coef * (ey - vy * vdote / c2),
            vz + coef * vz * vdote / c2)


def initial_state(cfg, x0, y0, vx0, vy0, sample=None, vz0=None, species=None):
    """t = 0 state for Algorithm 1 (readings listed in the module docstring).

    sample: optional particle indices.  The grid quantities always come from every
    particle; with a sample, the particle arrays of the state (and the Taylor start) are
    those of the sampled particles only, each equal to its value without sampling.
    vz0: the z velocities (2D-3V); species: each particle's index into cfg.species.
    """
    general = cfg.vdim == 3 or cfg.species is not None
    if general:
        return _initial_state_general(cfg, x0, y0, vx0, vy0, vz0, species, sample)
    x0 = wrap(np.asarray(x0, dtype=np.float64), cfg.lx)
    y0 = wrap(np.asarray(y0, dtype=np.float64), cfg.ly)
    vx0 = np.asarray(vx0, dtype=np.float64).copy()
    vy0 = np.asarray(vy0, dtype=np.float64).copy()
    n = len(x0)
    kx, ky, K = _k(cfg)
    qp = cfg.w * cfg.q
    rho = deposit(cfg, x0, y0, np.full(n, qp))
    rho_hat = spectral.dft2(rho)
    rho_hat[K == 0.0] = 0.0
    phi_hat = np.where(K > 0.0, rho_hat / (cfg.eps0 * np.where(K > 0.0, K, 1.0)), 0.0)
    ex = spectral.idft2(-1j * kx * phi_hat).real
    ey = spectral.idft2(-1j * ky * phi_hat).real
    if sample is not None:
        x0, y0, vx0, vy0 = x0[sample], y0[sample], vx0[sample], vy0[sample]
    exp_ = gather(cfg, x0, y0, ex)
    eyp = gather(cfg, x0, y0, ey)
    vx_old, vy_old = taylor_back_velocity(cfg, vx0, vy0, exp_, eyp)
    gamma = 1.0 / np.sqrt(1.0 - (vx0 * vx0 + vy0 * vy0) / (cfg.c * cfg.c))
    st = State(x=x0, y=y0, px=gamma * cfg.m * vx0, py=gamma * cfg.m * vy0,
               vx=vx0, vy=vy0, vx_old=vx_old, vy_old=vy_old)
    zero = np.zeros_like(rho_hat)
    if cfg.stepper == "bdf":
        k = cfg.bdf_order
        st.hist = {"phi": [phi_hat.copy() for _ in range(2 * k)],
                   "ax": [zero.copy() for _ in range(2 * k)],
                   "ay": [zero.copy() for _ in range(2 * k)],
                   "rho": [rho_hat.copy() for _ in range(k)]}
    elif cfg.stepper == "cdf2":
        st.hist = {"phi": phi_hat.copy(), "phi_prev": phi_hat.copy(),
                   "rho": rho_hat.copy(), "rho_prev": rho_hat.copy(),
                   "ax": zero.copy(), "ax_prev": zero.copy(),
                   "ay": zero.copy(), "ay_prev": zero.copy(),
                   "jx": zero.copy(), "jx_prev": zero.copy(),
                   "jy": zero.copy(), "jy_prev": zero.copy()}
    elif cfg.stepper == "dirk":
        st.hist = {"phi": phi_hat.copy(), "vphi": zero.copy(), "ax": zero.copy(),
                   "vax": zero.copy(), "ay": zero.copy(), "vay": zero.copy(),
                   "rho": rho_hat.copy(), "jx": zero.copy(), "jy": zero.copy()}
    else:
        raise ValueError(cfg.stepper)
    st.grids = {"rho": spectral.idft2(rho_hat).real, "phi": spectral.idft2(phi_hat).real,
                "ex0": exp_, "ey0": eyp}
    return st


def _initial_state_general(cfg, x0, y0, vx0, vy0, vz0, species, sample):
    """initial_state with per-particle charges and masses and/or three velocity components:
    rho^0 deposits each particle's q_p, P^0 = gamma m v^0 with the particle's mass and the
    three-component gamma, and every A_z level (and its current history) starts at 0."""
    n = len(x0)
    if cfg.species is not None and species is None:
        raise ValueError("a species table needs each particle's species index")
    sp = None if species is None else np.asarray(species).copy()
    vz0 = (np.zeros(n) if vz0 is None else np.asarray(vz0, dtype=np.float64).copy())
    st = initial_state(dataclasses.replace(cfg, vdim=2, species=None), x0, y0, vx0, vy0)
    # rho^0 from every particle's own charge (the single-species set-up above used w q)
    x0 = wrap(np.asarray(x0, dtype=np.float64), cfg.lx)
    y0 = wrap(np.asarray(y0, dtype=np.float64), cfg.ly)
    kx, ky, K = _k(cfg)
    qp, q, m = cfg.particle_constants(sp)
    rho_hat = spectral.dft2(deposit(cfg, x0, y0, qp * np.ones(n)))
    rho_hat[K == 0.0] = 0.0
    phi_hat = np.where(K > 0.0, rho_hat / (cfg.eps0 * np.where(K > 0.0, K, 1.0)), 0.0)
    ex = spectral.idft2(-1j * kx * phi_hat).real
    ey = spectral.idft2(-1j * ky * phi_hat).real
    vx0 = np.asarray(vx0, dtype=np.float64).copy()
    vy0 = np.asarray(vy0, dtype=np.float64).copy()
    if sample is not None:
        x0, y0, vx0, vy0, vz0 = x0[sample], y0[sample], vx0[sample], vy0[sample], vz0[sample]
        if sp is not None:
            sp = sp[sample]
        q = q if np.isscalar(q) else q[sample]
        m = m if np.isscalar(m) else m[sample]
    exp_ = gather(cfg, x0, y0, ex)
    eyp = gather(cfg, x0, y0, ey)
    vxo, vyo, vzo = taylor_back_velocity3(cfg, vx0, vy0, vz0, exp_, eyp, q, m)
    c2 = cfg.c * cfg.c
    gamma = 1.0 / np.sqrt(1.0 - (vx0 * vx0 + vy0 * vy0 + vz0 * vz0) / c2)
    st.x, st.y = x0, y0
    st.px, st.py = gamma * m * vx0, gamma * m * vy0
    st.vx, st.vy, st.vx_old, st.vy_old = vx0, vy0, vxo, vyo
    st.sp = sp
    if cfg.vdim == 3:
        st.pz, st.vz, st.vz_old = gamma * m * vz0, vz0, vzo
    zero = np.zeros_like(rho_hat)
    h = st.hist
    for key in list(h):
        if key.startswith("phi"):
            h[key] = ([phi_hat.copy() for _ in h[key]] if isinstance(h[key], list)
                      else phi_hat.copy())
        elif key.startswith("rho"):
            h[key] = ([rho_hat.copy() for _ in h[key]] if isinstance(h[key], list)
                      else rho_hat.copy())
    if cfg.vdim == 3:
        if cfg.stepper == "bdf":
            h["az"] = [zero.copy() for _ in range(2 * cfg.bdf_order)]
        elif cfg.stepper == "cdf2":
            h.update(az=zero.copy(), az_prev=zero.copy(), jz=zero.copy(), jz_prev=zero.copy())
        else:
            h.update(az=zero.copy(), vaz=zero.copy(), jz=zero.copy())
    st.grids = {"rho": spectral.idft2(rho_hat).real, "phi": spectral.idft2(phi_hat).real,
                "ex0": exp_, "ey0": eyp}
    return st


def step(cfg, st):
    """Advance one time step of Algorithm 1 (section 4.2)."""
    st.x = wrap(st.x + st.vx * cfg.dt, cfg.lx)
    st.y = wrap(st.y + st.vy * cfg.dt, cfg.ly)
    qp = cfg.particle_constants(st.sp)[0]
    jx = deposit(cfg, st.x, st.y, qp * st.vx)
    jy = deposit(cfg, st.x, st.y, qp * st.vy)
    jz = deposit(cfg, st.x, st.y, qp * st.vz) if cfg.vdim == 3 else None
    rho_dep = (deposited_charge_hat(cfg, st.x, st.y, st.sp) if cfg.charge == "deposit"
               else None)
    fields = field_solve(cfg, st, jx, jy, rho_dep, jz=jz)
    names = FIELD_NAMES + (FIELD_NAMES_Z if cfg.vdim == 3 else ())
    g = {name: gather(cfg, st.x, st.y, fields[name]) for name in names}
    iaem_push(cfg, st, g)
    st.n += 1
    return st


def run(cfg, x0, y0, vx0, vy0, nsteps, vz0=None, species=None):
    st = initial_state(cfg, x0, y0, vx0, vy0, vz0=vz0, species=species)
    for _ in range(nsteps):
        step(cfg, st)
    return st


def first_step_sampled(cfg, x0, y0, vx0, vy0, sample):
    """The first step of run(..., 1) for problems too large to push every particle on
    the CPU: the move, the deposit and the field solve use every particle, as in step();
    the gather and the push are done for the particles `sample` only.  The returned
    state holds those particles (in the order of `sample`) and the full grid quantities;
    every value equals the corresponding value of run(..., 1).
    """
    st = initial_state(cfg, x0, y0, vx0, vy0, sample=sample)
    x0 = wrap(np.asarray(x0, dtype=np.float64), cfg.lx)
    y0 = wrap(np.asarray(y0, dtype=np.float64), cfg.ly)
    vx0 = np.asarray(vx0, dtype=np.float64)
    vy0 = np.asarray(vy0, dtype=np.float64)
    x1 = wrap(x0 + vx0 * cfg.dt, cfg.lx)
    y1 = wrap(y0 + vy0 * cfg.dt, cfg.ly)
    qp = cfg.w * cfg.q
    jx = deposit(cfg, x1, y1, qp * vx0)
    jy = deposit(cfg, x1, y1, qp * vy0)
    rho_dep = deposited_charge_hat(cfg, x1, y1) if cfg.charge == "deposit" else None
    fields = field_solve(cfg, st, jx, jy, rho_dep)
    st.x, st.y = x1[sample], y1[sample]
    g = {name: gather(cfg, st.x, st.y, fields[name]) for name in FIELD_NAMES}
    iaem_push(cfg, st, g)
    st.n += 1
    return st


# ------------------------------------------------------------ diagnostics ----

def residual_norms(cfg, st):
    """Grid max-abs and RMS of each residual of the last step (inverse DFT of the spectra)."""
    out = {}
    for name in ("gauge", "gauge_dt", "continuity", "gauss"):
        if name in st.res:
            g = spectral.idft2(st.res[name]).real
            out[name] = (float(np.max(np.abs(g))), float(np.sqrt(np.mean(g * g))))
    return out


def energies(cfg, st):
    """Field and kinetic energies after the last step.

    W_B = sum B_z^2 dx dy / (2 mu0) with B_z = dAy/dx - dAx/dy; W_E = eps0/2 sum |E|^2 dx dy
    with E the stepper's discrete E (section 2.2, E = -grad phi - dA/dt); kinetic
    energy sum_p w m c^2 (gamma - 1) with gamma from v^{n+1}.
    """
    area = cfg.dx * cfg.dy
    bz = st.grids["bz"]
    b2 = bz * bz
    e2 = st.grids["ex"] ** 2 + st.grids["ey"] ** 2
    v2 = st.vx * st.vx + st.vy * st.vy
    if cfg.vdim == 3:   # B_x = dA_z/dy, B_y = -dA_z/dx, E_z = -dA_z/dt
        b2 = b2 + st.grids["bx"] ** 2 + st.grids["by"] ** 2
        e2 = e2 + st.grids["ez"] ** 2
        v2 = v2 + st.vz * st.vz
    wb = float(np.sum(b2) * area / (2.0 * cfg.mu0))
    we = float(0.5 * cfg.eps0 * np.sum(e2) * area)
    gamma = 1.0 / np.sqrt(1.0 - v2 / (cfg.c * cfg.c))
    if cfg.species is None:
        wm = cfg.w * cfg.m
    else:
        tab = np.asarray(cfg.species, dtype=np.float64)
        wm = tab[st.sp, 2] * tab[st.sp, 1]
    ke = float(np.sum(wm * cfg.c * cfg.c * (gamma - 1.0)))
    return {"wb": wb, "we": we, "ke": ke}
