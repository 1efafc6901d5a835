"""Discrete adjoint of the PIC step (oracle; test infrastructure only).

The paper defines the forward method only; the gradient of an objective of the final
state with respect to the initial velocities is the transpose of the Jacobian of the
forward map, applied step by step in reverse.  The forward map is oracle.pic.step
(Algorithm 1, section 4.2) with the charge from the continuity equation and any of the
steppers of section 3: BDF-k (3.2), the three CDF-2 forms (3.1) or s-stage DIRK (3.3).  The objective is

    W_B = 1/2 sum_ij B_z(i, j)^2 dx dy       (magnetic energy, section 5)

at the last level, optionally plus sum_p (Px_bar P_x + Py_bar P_y) of the final
momenta.  Gradients are taken with respect to v^0 (the velocities pic_init receives)
and, equivalently, with respect to P^0 = gamma m v^0 as the independent variable.

Reverse of one step n -> n+1, per particle and per Fourier mode (adjoint of a quantity
z written z_bar; inner products are the plain sums over grid nodes and particles, and
for a spectrum z the pairing Re sum conj(z_bar) dz):

  8. push:    u = P^{n+1} - q A_p,  v^{n+1} = c^2 u / D,  D = sqrt(c^2 |u|^2 + (m c^2)^2)
              u_bar = (c^2/D) (v_bar - c^2 u (u . v_bar)/D^2)
              P_bar <- P_bar + u_bar;  A_p_bar = -q u_bar
              P^{n+1} = P^n + q dt (-grad phi + (grad A) . v*):  grad phi_bar = -q dt P_bar,
              (d_l A_m)_bar = q dt P_bar_l v*_m,  v*_bar_m = q dt sum_l P_bar_l d_l A_m
              v* = 2 v^n - v^{n-1}: v^n_bar += 2 v*_bar, v^{n-1}_bar = -v*_bar
  7. gather:  field_bar(node) += g_bar W(node)  (a deposit); x_bar += g_bar grad_x(gather)
  6. fields:  F = IDFT(M u_hat)  ->  u_hat_bar += conj(M) DFT(F_bar)/N   (conj(i k) = -i k)
  5. stepper: BDF-k u^{n+1} = (g S - sum_d C_d u^{n+1-d})/(C_0 + g K),
              rho^{n+1} = -sum_j a_j rho^{n+1-j} - beta dt i k . J_hat; CDF-2 and DIRK
              likewise linear with real per-mode coefficients (DIRK's from the
              stage recurrence, taken as the Jacobian of the forward stage loop)
  4. J_hat = DFT(J)  ->  J_bar = Re(N IDFT(J_hat_bar))
  3. deposit: J = q_p v^n W(x^{n+1}) / (dx dy): v^n_bar += q_p/(dx dy) gather(J_bar);
              x^{n+1}_bar += q_p/(dx dy) v^n . grad_x gather(J_bar)
  2. move:    x^{n+1} = x^n + dt v^n: x^n_bar = x^{n+1}_bar, v^n_bar += dt x^{n+1}_bar
And at t = 0: P^0 = gamma m v^0 and the Taylor start v^{-1}(v^0, E^0(x^0)).

Spline derivatives use the identity W_p'(t) = W_{p-1}(t + 1/2) - W_{p-1}(t - 1/2) for the
centred cardinal B-spline (W_p is W_{p-1} convolved with the unit box), with the values
from the Cox-de Boor recursion.
"""
from dataclasses import dataclass

import numpy as np

from . import bspline, spectral, steppers
from . import pic as opic


# ---------------------------------------------------------------- shapes ----

def node_weight_derivatives(xi, p):
    """(i0, w, dw): node indices and weights of a degree-p shape at xi = x/dx and the
    derivatives dw[:, a] = d/dxi W_p(xi - (i0 + a)) = W_{p-1}(t + 1/2) - W_{p-1}(t - 1/2),
    t = xi - (i0 + a)."""
    xi = np.asarray(xi, dtype=np.float64)
    i0, w = bspline.node_weights(xi, p)
    t = [xi - (i0 + a) for a in range(p + 1)]
    dw = np.stack([bspline.cardinal_bspline(ta + 0.5, p - 1)
                   - bspline.cardinal_bspline(ta - 0.5, p - 1) for ta in t], axis=-1)
    return i0, w, dw


def gather_grad(cfg, x, y, grid):
    """(d/dx, d/dy) of sum_ij grid[i, j] W(x/dx - i) W(y/dy - j) at each particle."""
    nx, ny, p = cfg.nx, cfg.ny, cfg.p
    i0, wx, dwx = node_weight_derivatives(np.asarray(x) / cfg.dx, p)
    j0, wy, dwy = node_weight_derivatives(np.asarray(y) / cfg.dy, p)
    gx = np.zeros(len(x))
    gy = np.zeros(len(x))
    for a in range(p + 1):
        ii = np.mod(i0 + a, nx)
        for b in range(p + 1):
            jj = np.mod(j0 + b, ny)
            val = grid[ii, jj]
            gx += val * dwx[:, a] * wy[:, b]
            gy += val * wx[:, a] * dwy[:, b]
    return gx / cfg.dx, gy / cfg.dy


def scatter(cfg, x, y, values):
    """sum_p values_p W(x_p/dx - i) W(y_p/dy - j): the transpose of oracle.pic.gather
    (the deposit without its 1/(dx dy))."""
    return opic.deposit(cfg, x, y, values) * (cfg.dx * cfg.dy)


# ---------------------------------------------------------------- forward tape ----

PARTICLE_KEYS = ("x", "y", "px", "py", "vx", "vy", "vx_old", "vy_old")


@dataclass
class Tape:
    cfg: object
    states: list      # states[n]: particle arrays at the start of step n, n = 0..N
    fields: list      # fields[n]: the eight gathered mesh fields of step n (level n+1)
    e0: tuple         # E^0 gathered at x^0 (the Taylor start)
    final: object     # the oracle State after N steps


def _snapshot(st):
    return {k: np.array(getattr(st, k), copy=True) for k in PARTICLE_KEYS}


def record(cfg, x0, y0, vx0, vy0, nsteps):
    """Run oracle.pic for nsteps, keeping every particle state and every step's fields."""
    if cfg.charge != "continuity" or cfg.vdim != 2 or cfg.species is not None:
        raise ValueError("the adjoint covers the continuity charge, 2D-2V, one species")
    st = opic.initial_state(cfg, x0, y0, vx0, vy0)
    e0 = (st.grids["ex0"].copy(), st.grids["ey0"].copy())
    states = [_snapshot(st)]
    fields = []
    for _ in range(nsteps):
        opic.step(cfg, st)
        fields.append({name: st.grids[name].copy() for name in opic.FIELD_NAMES})
        states.append(_snapshot(st))
    return Tape(cfg, states, fields, e0, st)


def magnetic_energy(cfg, st):
    """W_B = 1/2 sum B_z^2 dx dy of the newest level."""
    return 0.5 * float(np.sum(st.grids["bz"] ** 2)) * cfg.dx * cfg.dy


# ---------------------------------------------------------------- adjoint pieces ----

def _gathered_field_adjoints(cfg, fbar):
    """Spectral adjoints of the potentials behind the eight gathered mesh fields: the
    fields are IDFT(i kx u), IDFT(i ky u), IDFT(A) with u = phi~, Ax, Ay, so each gets
    -i k_l DFT(field_bar)/N (conj(i k) = -i k) or DFT(field_bar)/N."""
    kx, ky, _ = spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)
    N = cfg.nx * cfg.ny
    fh = {name: spectral.dft2(fbar[name]) / N for name in opic.FIELD_NAMES}
    phi = -1j * kx * fh["dphidx"] - 1j * ky * fh["dphidy"]
    ax = fh["ax"] - 1j * kx * fh["daxdx"] - 1j * ky * fh["daxdy"]
    ay = fh["ay"] - 1j * kx * fh["daydx"] - 1j * ky * fh["daydy"]
    return phi, ax, ay


def _mesh_current_adjoint(cfg, jx_hat_bar, jy_hat_bar):
    """J_hat = DFT(J) -> J_bar = Re(N IDFT(J_hat_bar))."""
    N = cfg.nx * cfg.ny
    return N * spectral.idft2(jx_hat_bar).real, N * spectral.idft2(jy_hat_bar).real


def field_adjoint_cdf2(cfg, hbar, fbar):
    """Reverse of one CDF-2 field solve (section 3.1; cfg.cdf_form implicit, semi or
    explicit).  hbar: adjoints of the history after the step, with the forward's keys
    (phi, phi_prev, rho, rho_prev, ax, ax_prev, ay, ay_prev, jx, jx_prev, jy, jy_prev);
    returns (the adjoints before the step, the mesh J adjoint).  The particles use
    phi~ = (phi^{n+3/2} + phi^{n+1/2})/2 and A^{n+1}; the shift moves each new level to the
    current slot and the current one to the previous slot."""
    kx, ky, K = spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)
    c, dt, eps0, mu0 = cfg.c, cfg.dt, cfg.eps0, cfg.mu0
    phi_c, ax_c, ay_c = _gathered_field_adjoints(cfg, fbar)
    # adjoints of the new levels and of the levels the step read (after the shift)
    phin = hbar["phi"] + 0.5 * phi_c
    phih = hbar["phi_prev"] + 0.5 * phi_c
    rhon, rhoh = hbar["rho"], hbar["rho_prev"]
    an = {"x": hbar["ax"] + ax_c, "y": hbar["ay"] + ay_c}
    ah = {"x": hbar["ax_prev"], "y": hbar["ay_prev"]}
    jn = {"x": hbar["jx"], "y": hbar["jy"]}
    jh = {"x": hbar["jx_prev"], "y": hbar["jy_prev"]}
    zero = np.zeros_like(phin)
    phip, rhop = zero.copy(), zero.copy()
    ap = {"x": zero.copy(), "y": zero.copy()}
    jp = {"x": zero.copy(), "y": zero.copy()}
    th = 0.5 * c * c * dt * dt
    inv = 1.0 / (1.0 + th * K)
    h2 = c * c * dt * dt
    if cfg.cdf_form == "implicit":
        # u^{n+1} = inv (2 u^n + th (S^{n+1} + S^{n-1})) - u^{n-1}
        phih = phih + 2.0 * inv * phin
        rhon = rhon + (inv * th / eps0) * phin
        rhop = rhop + (inv * th / eps0) * phin
        phip = phip - phin
        for d in ("x", "y"):
            ah[d] = ah[d] + 2.0 * inv * an[d]
            jn[d] = jn[d] + (inv * th * mu0) * an[d]
            jp[d] = jp[d] + (inv * th * mu0) * an[d]
            ap[d] = ap[d] - an[d]
    elif cfg.cdf_form == "semi":
        # u^{n+1} = inv (2 u^n + c^2 dt^2 S^n) - u^{n-1}, S^n = rho^{n+1/2}/eps0, mu0 J^n
        phih = phih + 2.0 * inv * phin
        rhoh = rhoh + (inv * h2 / eps0) * phin
        phip = phip - phin
        for d in ("x", "y"):
            ah[d] = ah[d] + 2.0 * inv * an[d]
            jh[d] = jh[d] + (inv * h2 * mu0) * an[d]
            ap[d] = ap[d] - an[d]
    elif cfg.cdf_form == "explicit":
        # u^{n+1} = 2 u^n - u^{n-1} + c^2 dt^2 (S^n - K u^n)
        phih = phih + (2.0 - h2 * K) * phin
        rhoh = rhoh + (h2 / eps0) * phin
        phip = phip - phin
        for d in ("x", "y"):
            ah[d] = ah[d] + (2.0 - h2 * K) * an[d]
            jh[d] = jh[d] + (h2 * mu0) * an[d]
            ap[d] = ap[d] - an[d]
    else:
        raise ValueError(cfg.cdf_form)
    # rho^{n+3/2} = rho^{n+1/2} - dt (i kx Jx + i ky Jy)
    rhoh = rhoh + rhon
    jn["x"] = jn["x"] + 1j * dt * kx * rhon
    jn["y"] = jn["y"] + 1j * dt * ky * rhon
    out = {"phi": phih, "phi_prev": phip, "rho": rhoh, "rho_prev": rhop,
           "ax": ah["x"], "ax_prev": ap["x"], "ay": ah["y"], "ay_prev": ap["y"],
           "jx": jh["x"], "jx_prev": jp["x"], "jy": jh["y"], "jy_prev": jp["y"]}
    return out, _mesh_current_adjoint(cfg, jn["x"], jn["y"])


def dirk_matrix(cfg, K):
    """The real per-mode matrix of one DIRK wave step (section 3.3.1):
    (u^{n+1}, v^{n+1}) = M (u^n, v^n, S^n, S^{n+1}), M[r][i] evaluated by running the stage
    recurrence steppers.dirk_wave_update on unit inputs (the map is linear in them)."""
    A, b, cv = cfg.dirk["A"], cfg.dirk["b"], cfg.dirk["c"]
    cols = []
    for e in np.eye(4):
        uo, vo = steppers.dirk_wave_update(e[0] + 0.0 * K, e[1] + 0.0 * K, e[2], e[3], K, cfg.c,
                                           cfg.dt, A, b, cv)
        cols.append((uo, vo))
    return [[cols[i][r] for i in range(4)] for r in range(2)]


def field_adjoint_dirk(cfg, hbar, fbar):
    """Reverse of one s-stage DIRK field solve (section 3.3).  hbar: adjoints of the state
    after the step (phi, vphi, ax, vax, ay, vay, rho, jx, jy -- jx, jy the stored J^{n+1});
    returns (the adjoints before the step, the mesh J^{n+1} adjoint)."""
    kx, ky, K = spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)
    dt, eps0, mu0 = cfg.dt, cfg.eps0, cfg.mu0
    r0, r1 = steppers.dirk_interp_weights(cfg.dirk["b"], cfg.dirk["c"])
    M = dirk_matrix(cfg, K)
    phi_c, ax_c, ay_c = _gathered_field_adjoints(cfg, fbar)

    def back(ub, vb):  # transpose of M applied to (u_bar^{n+1}, v_bar^{n+1})
        return [M[0][i] * ub + M[1][i] * vb for i in range(4)]

    p = back(hbar["phi"] + phi_c, hbar["vphi"])
    ax = back(hbar["ax"] + ax_c, hbar["vax"])
    ay = back(hbar["ay"] + ay_c, hbar["vay"])
    # phi's sources rho^n/eps0, rho^{n+1}/eps0; A's mu0 J^n, mu0 J^{n+1}
    rhon = hbar["rho"] + p[3] / eps0
    rho = p[2] / eps0 + rhon                           # rho^{n+1} = rho^n - dt (...)
    jx = mu0 * ax[2] + 1j * dt * r0 * kx * rhon        # J^n (the stored level)
    jy = mu0 * ay[2] + 1j * dt * r0 * ky * rhon
    jxn = hbar["jx"] + mu0 * ax[3] + 1j * dt * r1 * kx * rhon
    jyn = hbar["jy"] + mu0 * ay[3] + 1j * dt * r1 * ky * rhon
    out = {"phi": p[0], "vphi": p[1], "ax": ax[0], "vax": ax[1], "ay": ay[0], "vay": ay[1],
           "rho": rho, "jx": jx, "jy": jy}
    return out, _mesh_current_adjoint(cfg, jxn, jyn)


def field_adjoint_bdf(cfg, hbar, fbar):
    """Reverse of one BDF-k field solve (continuity + wave update + gradient fields).

    hbar: adjoints of the history after the step, {"phi": [L], "ax": [L], "ay": [L],
    "rho": [k]}, newest first (spectra).  fbar: adjoints of the eight real mesh fields
    the step produced.  Returns (hbar before the step, (Jx_bar, Jy_bar)) with J_bar the
    adjoint of the real mesh current J^{n+1}."""
    kx, ky, K = spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)
    a, beta = steppers.bdf_coefficients(cfg.bdf_order)
    C = steppers.bdf_second_derivative_coefficients(a)
    a = [float(v) for v in a]
    C = [float(v) for v in C]
    c, dt, eps0, mu0 = cfg.c, cfg.dt, cfg.eps0, cfg.mu0
    g = (c * float(beta) * dt) ** 2
    bdt = float(beta) * dt
    N = cfg.nx * cfg.ny
    fh = {name: spectral.dft2(fbar[name]) / N for name in opic.FIELD_NAMES}
    # step 6: the fields are IDFT(i kx phi), IDFT(i ky phi), IDFT(A), IDFT(i k_l A_m)
    phi_s = hbar["phi"][0] - 1j * kx * fh["dphidx"] - 1j * ky * fh["dphidy"]
    ax_s = hbar["ax"][0] + fh["ax"] - 1j * kx * fh["daxdx"] - 1j * ky * fh["daxdy"]
    ay_s = hbar["ay"][0] + fh["ay"] - 1j * kx * fh["daydx"] - 1j * ky * fh["daydy"]
    # step 5: u^{n+1} = (g S - sum_d C_d u^{n+1-d}) / (C_0 + g K)
    den = C[0] + g * K
    L = len(C) - 1
    out = {}
    for name, us in (("phi", phi_s), ("ax", ax_s), ("ay", ay_s)):
        old = hbar[name]
        out[name] = [(old[d] if d < L else 0.0) - (C[d] / den) * us for d in range(1, L + 1)]
    rho_s = hbar["rho"][0] + (g / (eps0 * den)) * phi_s
    k = len(a) - 1
    out["rho"] = [(hbar["rho"][j] if j < k else 0.0) - (a[j] / a[0]) * rho_s
                  for j in range(1, k + 1)]
    # rho^{n+1} = (-beta dt (i kx Jx + i ky Jy) - ...)/a_0;  A: g mu0 J/(C_0 + g K)
    jx_hat_bar = (1j * bdt * kx / a[0]) * rho_s + (g * mu0 / den) * ax_s
    jy_hat_bar = (1j * bdt * ky / a[0]) * rho_s + (g * mu0 / den) * ay_s
    # step 4: J_hat = DFT(J)
    jx_bar = N * spectral.idft2(jx_hat_bar).real
    jy_bar = N * spectral.idft2(jy_hat_bar).real
    return out, (jx_bar, jy_bar)


def push_adjoint(cfg, s0, s1, g, abar):
    """Reverse of the IAEM push of step n (section 4.1).

    s0, s1: particle states at the start and end of the step; g: the eight gathered
    values at x^{n+1}; abar: adjoints of s1 (modified copy returned) with the adjoints
    of the gathered values.  Returns (abar_partial, g_bar): abar_partial holds P^n_bar,
    v^{n-1}_bar (in vx_old, vy_old) and the v^n_bar terms from the push (in vx, vy)."""
    q, dt, c2, m = cfg.q, cfg.dt, cfg.c * cfg.c, cfg.m
    ux = s1["px"] - q * g["ax"]
    uy = s1["py"] - q * g["ay"]
    D = np.sqrt(c2 * (ux * ux + uy * uy) + (m * c2) ** 2)
    udv = ux * abar["vx"] + uy * abar["vy"]
    ubx = (c2 / D) * (abar["vx"] - c2 * ux * udv / D ** 2)
    uby = (c2 / D) * (abar["vy"] - c2 * uy * udv / D ** 2)
    pbx = abar["px"] + ubx
    pby = abar["py"] + uby
    vsx = 2.0 * s0["vx"] - s0["vx_old"]
    vsy = 2.0 * s0["vy"] - s0["vy_old"]
    qdt = q * dt
    gbar = {
        "dphidx": -qdt * pbx, "dphidy": -qdt * pby,
        "ax": -q * ubx, "ay": -q * uby,
        "daxdx": qdt * pbx * vsx, "daxdy": qdt * pby * vsx,
        "daydx": qdt * pbx * vsy, "daydy": qdt * pby * vsy,
    }
    vsbx = qdt * (pbx * g["daxdx"] + pby * g["daxdy"])
    vsby = qdt * (pbx * g["daydx"] + pby * g["daydy"])
    out = dict(abar)
    out["px"], out["py"] = pbx, pby
    # the v_old slot of s1 holds v^n; v* = 2 v^n - v^{n-1}
    out["vx"] = abar["vx_old"] + 2.0 * vsbx
    out["vy"] = abar["vy_old"] + 2.0 * vsby
    out["vx_old"], out["vy_old"] = -vsbx, -vsby
    return out, gbar


def adjoint_step(cfg, s0, s1, fields, abar, hbar):
    """Reverse of step n: adjoints of (state s1, history after) -> (state s0, history before)."""
    x1, y1 = s1["x"], s1["y"]
    g = {name: opic.gather(cfg, x1, y1, fields[name]) for name in opic.FIELD_NAMES}
    ab, gbar = push_adjoint(cfg, s0, s1, g, abar)
    # step 7: the gather's transpose is a deposit of g_bar; the positions get the gradient
    fbar = {}
    xb = ab["x"].copy()
    yb = ab["y"].copy()
    for name in opic.FIELD_NAMES:
        fbar[name] = scatter(cfg, x1, y1, gbar[name])
        gx, gy = gather_grad(cfg, x1, y1, fields[name])
        xb = xb + gbar[name] * gx
        yb = yb + gbar[name] * gy
    field_adjoint = {"bdf": field_adjoint_bdf, "cdf2": field_adjoint_cdf2,
                     "dirk": field_adjoint_dirk}[cfg.stepper]
    hbar, (jxb, jyb) = field_adjoint(cfg, hbar, fbar)
    # step 3: J = q_p v^n W(x^{n+1}) / (dx dy)
    s = cfg.w * cfg.q / (cfg.dx * cfg.dy)
    vx, vy = s0["vx"], s0["vy"]
    vbx = ab["vx"] + s * opic.gather(cfg, x1, y1, jxb)
    vby = ab["vy"] + s * opic.gather(cfg, x1, y1, jyb)
    gxx, gxy = gather_grad(cfg, x1, y1, jxb)
    gyx, gyy = gather_grad(cfg, x1, y1, jyb)
    xb = xb + s * (vx * gxx + vy * gyx)
    yb = yb + s * (vx * gxy + vy * gyy)
    # step 2: x^{n+1} = x^n + dt v^n
    vbx = vbx + cfg.dt * xb
    vby = vby + cfg.dt * yb
    out = dict(ab)
    out.update(x=xb, y=yb, vx=vbx, vy=vby)
    return out, hbar


def initial_adjoint(cfg, s0, e0, abar):
    """Gradient with respect to v^0 from the adjoints of the t = 0 state.

    P^0 = gamma m v^0 and v^{-1} = v^0 - kappa (E - v (v . E)/c^2), kappa = dt q/(gamma m),
    with E = E^0(x^0) fixed.  Returns (dJ/dv^0, dJ/dP^0) as pairs of arrays; the second is
    the gradient with P^0 the independent variable (v^0 = c^2 P/sqrt(c^2 |P|^2 + m^2 c^4)).
    """
    c2, m = cfg.c * cfg.c, cfg.m
    vx, vy = s0["vx"], s0["vy"]
    ex, ey = e0
    gam = 1.0 / np.sqrt(1.0 - (vx * vx + vy * vy) / c2)
    # dP/dv = gamma m (I + gamma^2 v v^T / c^2), symmetric
    pvb = vx * abar["px"] + vy * abar["py"]
    gx = abar["vx"] + gam * m * (abar["px"] + gam * gam * vx * pvb / c2)
    gy = abar["vy"] + gam * m * (abar["py"] + gam * gam * vy * pvb / c2)
    # v^{-1}: d/dv [-kappa T], T = E - v (v.E)/c^2, d kappa/dv = -kappa gamma^2 v / c^2,
    # dT/dv = -(v E^T + (v.E) I)/c^2;  transpose applied to w = v^{-1}_bar
    wx, wy = abar["vx_old"], abar["vy_old"]
    kap = cfg.dt * cfg.q / (gam * m)
    vde = vx * ex + vy * ey
    tx = ex - vx * vde / c2
    ty = ey - vy * vde / c2
    tw = tx * wx + ty * wy
    vw = vx * wx + vy * wy
    gx = gx + wx + kap * gam * gam * vx * tw / c2 + (kap / c2) * (ex * vw + vde * wx)
    gy = gy + wy + kap * gam * gam * vy * tw / c2 + (kap / c2) * (ey * vw + vde * wy)
    # dv/dP = (1/(gamma m)) (I - v v^T / c^2), symmetric
    vg = vx * gx + vy * gy
    pgx = (gx - vx * vg / c2) / (gam * m)
    pgy = (gy - vy * vg / c2) / (gam * m)
    return (gx, gy), (pgx, pgy)


def gradient(tape, bz_bar=None, px_bar=None, py_bar=None):
    """dJ/dv^0 and dJ/dP^0 for J = sum bz_bar B_z (final) + sum (px_bar Px + py_bar Py).

    bz_bar defaults to B_z dx dy, the seed of J = W_B.  Returns a dict with "v0" and
    "p0" (each a pair of arrays)."""
    cfg = tape.cfg
    n = len(tape.states[0]["x"])
    fin = tape.final
    if bz_bar is None and px_bar is None and py_bar is None:
        bz_bar = fin.grids["bz"] * (cfg.dx * cfg.dy)
    kx, ky, _ = spectral.wavenumber_grid(cfg.nx, cfg.ny, cfg.lx, cfg.ly)
    zero = np.zeros((cfg.nx, cfg.ny), dtype=np.complex128)
    # adjoints of the history after the last step, with the forward's keys; the newest
    # A (the level B_z is taken from) is ax[0] for BDF-k and ax for CDF-2 and DIRK
    hbar = {key: ([zero.copy() for _ in val] if isinstance(val, list) else zero.copy())
            for key, val in fin.hist.items()}
    if bz_bar is not None:
        # B_z = IDFT(i kx Ay - i ky Ax) of the newest level
        zb = spectral.dft2(np.asarray(bz_bar, dtype=np.float64)) / (cfg.nx * cfg.ny)
        if cfg.stepper == "bdf":
            hbar["ay"][0] = hbar["ay"][0] - 1j * kx * zb
            hbar["ax"][0] = hbar["ax"][0] + 1j * ky * zb
        else:
            hbar["ay"] = hbar["ay"] - 1j * kx * zb
            hbar["ax"] = hbar["ax"] + 1j * ky * zb
    abar = {key: np.zeros(n) for key in PARTICLE_KEYS}
    if px_bar is not None:
        abar["px"] = np.asarray(px_bar, dtype=np.float64).copy()
    if py_bar is not None:
        abar["py"] = np.asarray(py_bar, dtype=np.float64).copy()
    for step in range(len(tape.fields) - 1, -1, -1):
        abar, hbar = adjoint_step(cfg, tape.states[step], tape.states[step + 1],
                                  tape.fields[step], abar, hbar)
    v0, p0 = initial_adjoint(cfg, tape.states[0], tape.e0, abar)
    return {"v0": v0, "p0": p0, "x0_partial": (abar["x"], abar["y"])}


def objective(cfg, x0, y0, vx0, vy0, nsteps, px_bar=None, py_bar=None):
    """J = W_B of the final level (+ final momenta against px_bar, py_bar) by a plain
    forward run of oracle.pic: the function the gradients differentiate."""
    st = opic.run(cfg, x0, y0, vx0, vy0, nsteps)
    if px_bar is None and py_bar is None:
        return magnetic_energy(cfg, st)
    val = 0.0
    if px_bar is not None:
        val += float(np.dot(px_bar, st.px))
    if py_bar is not None:
        val += float(np.dot(py_bar, st.py))
    return val


def velocity_from_p0(cfg, px0, py0):
    """v^0 of a given P^0 with A^0 = 0 (the inverse of P^0 = gamma m v^0)."""
    c2 = cfg.c * cfg.c
    den = np.sqrt(c2 * (px0 * px0 + py0 * py0) + (cfg.m * c2) ** 2)
    return c2 * px0 / den, c2 * py0 / den
