"""Per-mode time steppers for the Lorenz-gauge wave equations (oracle).

Section 3 discretises (1/c^2) u_tt - Laplacian u = S in time only; with the
spectral spatial discretisation every Fourier mode k evolves independently, the
Laplacian becoming -K with K = |k|^2.  All functions here act elementwise on numpy
arrays of modes (complex spectra) and on the scalar K of each mode.

  * BDF-k (section 3.2): first derivative (1/(beta dt)) sum_j a_j u^{n+1-j}, second
    derivative the same operator applied twice, whose coefficients C_i are given by
    the coefficient-reordering Lemma and Table 1 of the paper.
  * CDF-2 implicit (section 3.1): the Crank-Nicolson-averaged centred scheme with
    L = I - alpha^-2 Laplacian, alpha = sqrt(2)/(c dt).
  * s-stage DIRK (section 3.3.1): the wave equation as the first-order system
    d/dt (v, u) = (c^2 (S + Laplacian u), v), each stage solved implicitly with
    L_i = I - (h a_ii c)^2 Laplacian.
"""
from fractions import Fraction
from math import comb

import numpy as np


# ---------------------------------------------------------------- BDF-k ------

def bdf_coefficients(k):
    """BDF-k coefficients (a, beta), normalised so that a[0] = 1.

    Built from the textbook definition of the k-step backward differentiation
    formula, sum_{j=1..k} (1/j) nabla^j u^{n+1} = dt u'(t_{n+1}) with nabla the
    backward difference, so that du/dt ~ (1/(beta dt)) sum_{j=0..k} a_j u^{n+1-j}
    (section 3.2, first-derivative form; the BDF-2 remark prints a = (1, -4/3, 1/3)
    and beta = 2/3).  Exact rationals are returned.
    """
    if k < 1:
        raise ValueError("BDF order must be >= 1")
    alpha = [Fraction(0)] * (k + 1)
    for j in range(1, k + 1):
        for i in range(j + 1):
            alpha[i] += Fraction((-1) ** i * comb(j, i), j)
    a0 = alpha[0]
    return [x / a0 for x in alpha], 1 / a0


def bdf_second_derivative_coefficients(a):
    """C_d, d = 0..2k: coefficients of the twice-applied BDF operator.

    Follows the case formula of the coefficient-reordering Lemma in section 3.2,
    indexed by the distance d = n - i below the newest level:
        C_d = sum_{j=0..d}      a_j a_{d-j}          for d <= k,
        C_d = sum_{j=0..2k-d}   a_{k-j} a_{d-k+j}    for d >  k.
    """
    k = len(a) - 1
    out = []
    for d in range(2 * k + 1):
        if d <= k:
            out.append(sum(a[j] * a[d - j] for j in range(d + 1)))
        else:
            out.append(sum(a[k - j] * a[d - k + j] for j in range(2 * k - d + 1)))
    return out


def bdf_continuity(rho_hist, div_j_new, dt, a, beta):
    """rho^{n+1} from the BDF-k continuity equation (section 3.2).

    (1/(beta dt)) sum_j a_j rho^{n+1-j} + div J^{n+1} = 0, solved for the newest
    level; rho_hist = [rho^n, rho^{n-1}, ...] (newest first).
    """
    rhs = -float(beta) * dt * div_j_new
    for j in range(1, len(a)):
        rhs = rhs - float(a[j]) * rho_hist[j - 1]
    return rhs / float(a[0])


def bdf_wave_update(u_hist, source_new, K, c, dt, beta, C):
    """u^{n+1} of one mode from the BDF-k wave equation (section 3.2).

    (1/(c^2 beta^2 dt^2)) sum_{d=0..2k} C_d u^{n+1-d} + K u^{n+1} = S^{n+1}
    multiplied through by (c beta dt)^2; u_hist = [u^n, u^{n-1}, ...] (2k levels).
    """
    g = (c * float(beta) * dt) ** 2
    rhs = g * source_new
    for d in range(1, len(C)):
        rhs = rhs - float(C[d]) * u_hist[d - 1]
    return rhs / (float(C[0]) + g * K)


# ---------------------------------------------------------------- CDF-2 ------

def cdf2_continuity(rho_half, div_j_new, dt):
    """rho^{n+3/2} = rho^{n+1/2} - dt div J^{n+1} (section 3.1, staggered continuity)."""
    return rho_half - dt * div_j_new


def cdf2_wave_update(u_now, u_prev, s_new, s_old, K, c, dt):
    """Implicit CDF-2 update of one mode (section 3.1).

    L (u^{n+1} + u^{n-1}) = 2 u^n + alpha^-2 (S^{n+1} + S^{n-1}) with
    L = 1 + alpha^-2 K, alpha^-2 = c^2 dt^2 / 2.
    """
    inv_alpha2 = 0.5 * c * c * dt * dt
    return (2.0 * u_now + inv_alpha2 * (s_new + s_old)) / (1.0 + inv_alpha2 * K) - u_prev


def cdf2_semi_implicit_update(u_now, u_prev, s_now, K, c, dt):
    """Semi-implicit CDF-2 update of one mode (section 3.1, the second form): the
    Laplacian averaged over levels n+1 and n-1, the source at level n,

        (u^{n+1} - 2u^n + u^{n-1}) / (c^2 dt^2) + K (u^{n+1} + u^{n-1}) / 2 = S^n,

    so u^{n+1} = (2 u^n + c^2 dt^2 S^n) / (1 + alpha^-2 K) - u^{n-1}, alpha^-2 = c^2 dt^2 / 2.
    """
    inv_alpha2 = 0.5 * c * c * dt * dt
    return (2.0 * u_now + c * c * dt * dt * s_now) / (1.0 + inv_alpha2 * K) - u_prev


def cdf2_explicit_update(u_now, u_prev, s_now, K, c, dt):
    """Explicit CDF-2 update of one mode (section 3.1, the third form): the Laplacian and
    the source at level n,

        (u^{n+1} - 2u^n + u^{n-1}) / (c^2 dt^2) + K u^n = S^n.
    """
    return 2.0 * u_now - u_prev + c * c * dt * dt * (s_now - K * u_now)


# ---------------------------------------------------------------- DIRK -------

# The tableau printed in section 5 for the Qin-Zhang method, exactly as printed.
DIRK2_AS_PRINTED = {
    "A": [[0.5, 0.0], [0.25, 0.5]],
    "b": [0.5, 0.5],
    "c": [0.25, 0.25],
}

# Reading used throughout: the Qin-Zhang 2-stage symplectic DIRK (two implicit
# midpoint half steps), whose row sums equal c and whose stability function has
# modulus one on the imaginary axis.
DIRK2_QIN_ZHANG = {
    "A": [[0.25, 0.0], [0.5, 0.25]],
    "b": [0.5, 0.5],
    "c": [0.25, 0.75],
}

# 3-stage reading: three implicit-midpoint thirds composed (same construction).
DIRK3_MIDPOINT = {
    "A": [[1 / 6, 0.0, 0.0], [1 / 3, 1 / 6, 0.0], [1 / 3, 1 / 3, 1 / 6]],
    "b": [1 / 3, 1 / 3, 1 / 3],
    "c": [1 / 6, 0.5, 5 / 6],
}


def dirk_interp_weights(b, cvec):
    """(R0, R1) with sum_i b_i X^(i) = R0 X^n + R1 X^{n+1} for X^(i) = (1-c_i) X^n + c_i X^{n+1}.

    Section 3.3.1 (the R^{s,n} and R^{s,n+1} of the linear stage interpolation).
    """
    r0 = sum(bi * (1.0 - ci) for bi, ci in zip(b, cvec))
    r1 = sum(bi * ci for bi, ci in zip(b, cvec))
    return r0, r1


def dirk_continuity(rho_n, div_j_n, div_j_new, h, b, cvec):
    """rho^{n+1} = rho^n - h sum_i b_i div J^(i) (section 3.3.1, DIRK continuity)."""
    out = rho_n
    for bi, ci in zip(b, cvec):
        out = out - h * bi * ((1.0 - ci) * div_j_n + ci * div_j_new)
    return out


def dirk_wave_update(u, v, s_n, s_new, K, c, h, A, b, cvec):
    """One s-stage DIRK step of d/dt (v, u) = (c^2 (S - K u), v) for one mode.

    Section 3.3.1.  Stage i uses the stage source S^(i) = (1-c_i) S^n + c_i S^{n+1}
    and the known earlier stages through
        ubar = u^n + h sum_{j<i} a_ij k_j^u,  vbar = v^n + h sum_{j<i} a_ij k_j^v;
    the implicit pair k^u = vbar + h a_ii k^v, k^v = c^2 (S^(i) - K (ubar + h a_ii k^u))
    is solved in closed form with d = 1 + (h a_ii c)^2 K (the per-mode L_i).
    The c^2 on the k^v source follows the first-order system (the stage formula
    printed for k^v omits it; with c = 1 the two agree).
    Returns (u^{n+1}, v^{n+1}).
    """
    s = len(b)
    ku, kv = [], []
    for i in range(s):
        ubar = u
        vbar = v
        for j in range(i):
            ubar = ubar + h * A[i][j] * ku[j]
            vbar = vbar + h * A[i][j] * kv[j]
        src = (1.0 - cvec[i]) * s_n + cvec[i] * s_new
        gam = h * A[i][i]
        d = 1.0 + (gam * c) ** 2 * K
        force = c * c * (src - K * ubar)
        ku.append((vbar + gam * force) / d)
        kv.append((force - gam * c * c * K * vbar) / d)
    u_new = u
    v_new = v
    for i in range(s):
        u_new = u_new + h * b[i] * ku[i]
        v_new = v_new + h * b[i] * kv[i]
    return u_new, v_new
