"""Bit-exact CPU model of the FP32 form's first move and current deposit (test
infrastructure only).

The FP32 form is a build-side design (the paper computes in FP64): positions and
velocities are FP32, and each current contribution q_p v W_x W_y is deposited as an
integer multiple of a power-of-two quantum and summed in int64, so the grid sums are
exact and independent of the order of the particles.  This module restates that
arithmetic -- the position update and current deposit of Algorithm 1 (section 4.2:
x^{n+1} = x^n + v^n dt, then J^{n+1} from x^{n+1} and v^n with the B-spline shape of
section 4) -- in numpy float32 with exact integer sums, so that the GPU's current can be
compared bit for bit:

  * every float32 operation is one IEEE-754 operation rounded to nearest even;
  * a fused multiply-add a b + c is rounded once: the product is exact in float64, the
    sum is formed with its exact error term (Knuth's TwoSum) and rounded to float32 with
    that error deciding a float64 value that falls exactly on a float32 tie;
  * the shape weights are the closed-form piecewise polynomials of the centred cardinal
    B-splines (degrees 2, 3, 4), written in the operation order this form fixes (the
    oracle's FP64 path uses the Cox-de Boor recursion instead);
  * a contribution of node (a, b) is t_a W_y,b with t_a = v W_x,a rounded to float32; it is
    summed as rint(t_a W_y,b 2^s) of the exact product (half to even), i.e. rounded once to
    the quantum: the float64 product of two float32 values is exact, and so is its scaling
    by the power of two 2^s.
"""
import numpy as np

F32 = np.float32


def _two_sum(a, b):
    s = a + b
    bp = s - a
    ap = s - bp
    return s, (a - ap) + (b - bp)


def fmaf(a, b, c):
    """float32 a * b + c with one rounding (arrays or scalars of float32)."""
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    c = np.asarray(c, dtype=np.float32)
    p = a.astype(np.float64) * b.astype(np.float64)          # exact: 24 + 24 bits
    s, err = _two_sum(p, c.astype(np.float64))               # p + c = s + err exactly
    r = s.astype(np.float32)                                 # nearest, ties to even
    # s lies on a float32 tie only if it is the midpoint of its two float32 neighbours;
    # then the sign of err decides (err = 0 keeps the even choice)
    lo = np.where(r.astype(np.float64) <= s, r, np.nextafter(r, np.float32(-np.inf)))
    hi = np.nextafter(lo, np.float32(np.inf))
    mid = 0.5 * (lo.astype(np.float64) + hi.astype(np.float64))
    tie = (s == mid) & (err != 0)
    return np.where(tie & (err > 0), hi, np.where(tie & (err < 0), lo, r)).astype(np.float32)


def wrap32(x, length):
    """Periodic wrap after a move of less than one period, in float32."""
    x = np.asarray(x, dtype=np.float32)
    L = F32(length)
    x = np.where(x >= L, (x - L).astype(np.float32), x)
    return np.where(x < F32(0), (x + L).astype(np.float32), x).astype(np.float32)


def weights32(xi, p):
    """(first node, weights[:, p+1]) of the degree-p shape at xi (float32 arithmetic)."""
    xi = np.asarray(xi, dtype=np.float32)
    h = F32(0.5)
    if p == 2:
        f = np.floor((xi + h).astype(np.float32))
        d = (xi - f).astype(np.float32)
        hm, hp = (h - d).astype(np.float32), (h + d).astype(np.float32)
        w = [h * (hm * hm).astype(np.float32), fmaf(-d, d, F32(0.75)),
             h * (hp * hp).astype(np.float32)]
        i0 = f.astype(np.int64) - 1
    elif p == 3:
        f = np.floor(xi)
        d = (xi - f).astype(np.float32)
        e = (F32(1) - d).astype(np.float32)
        s6, t3 = F32(1.0 / 6.0), F32(2.0 / 3.0)
        d2, e2 = (d * d).astype(np.float32), (e * e).astype(np.float32)
        d3, e3 = (d2 * d).astype(np.float32), (e2 * e).astype(np.float32)
        w = [s6 * e3, fmaf(h, d3, (t3 - d2).astype(np.float32)),
             fmaf(h, e3, (t3 - e2).astype(np.float32)), s6 * d3]
        i0 = f.astype(np.int64) - 1
    elif p == 4:
        def mid(t):  # (55 + 20 t - 120 t^2 + 80 t^3 - 16 t^4) / 96, Horner
            r = fmaf(F32(-16), t, F32(80))
            r = fmaf(r, t, F32(-120))
            r = fmaf(r, t, F32(20))
            r = fmaf(r, t, F32(55))
            return (r * F32(1.0 / 96.0)).astype(np.float32)
        f = np.floor((xi + h).astype(np.float32))
        d = (xi - f).astype(np.float32)
        a = fmaf(F32(-2), d, F32(1))
        b = fmaf(F32(2), d, F32(1))
        a2, b2, d2 = (a * a).astype(np.float32), (b * b).astype(np.float32), (d * d).astype(np.float32)
        s384 = F32(1.0 / 384.0)
        inner = fmaf((F32(48) * d2).astype(np.float32), d2, fmaf(F32(-120), d2, F32(115)))
        w = [s384 * (a2 * a2).astype(np.float32), mid((F32(1) + d).astype(np.float32)),
             (inner * F32(1.0 / 192.0)).astype(np.float32), mid((F32(1) - d).astype(np.float32)),
             s384 * (b2 * b2).astype(np.float32)]
        i0 = f.astype(np.int64) - 2
    else:
        raise ValueError(p)
    return i0, np.stack([np.asarray(v, dtype=np.float32) for v in w], axis=-1)


def current_scale(c, n, rmax=1.0):
    """The power-of-two factor 2^s of the fixed-point current: s = min(38, 62 - ceil(log2 n))
    - ceil(log2 c) - ceil(log2 rmax), so that no contribution exceeds 2^38 quanta and no int64
    node total can reach 2^62 (rmax: largest |q w| of a species table, else 1)."""
    k = 38 if n <= 1 else min(38, 62 - int(np.ceil(np.log2(n))))
    return float(2.0 ** (k - int(np.ceil(np.log2(c))) - int(np.ceil(np.log2(rmax)))))


def contribution(t, w, scale):
    """rint(t w scale) of the exact product of the float32 values t and w (int64)."""
    t = np.asarray(t, dtype=np.float32).astype(np.float64)
    w = np.asarray(w, dtype=np.float32).astype(np.float64)
    return np.rint(t * w * np.float64(scale)).astype(np.int64)


def move_deposit(x, y, vx, vy, dt, lx, ly, nx, ny, p, scale):
    """One move + fixed-point deposit from FP64 inputs rounded to float32.

    Returns (x1, y1, jx, jy): the moved float32 positions and the int64 node sums of
    rint((v W_x) W_y * scale) for each current component (v W_x rounded to float32, the
    product with W_y exact), shape (nx, ny).  The positions are first rounded to float32 and
    wrapped, as at t = 0."""
    x = wrap32(np.asarray(x, dtype=np.float64).astype(np.float32), lx)
    y = wrap32(np.asarray(y, dtype=np.float64).astype(np.float32), ly)
    vx = np.asarray(vx, dtype=np.float64).astype(np.float32)
    vy = np.asarray(vy, dtype=np.float64).astype(np.float32)
    dt32 = F32(dt)
    x1 = wrap32(fmaf(vx, dt32, x), lx)
    y1 = wrap32(fmaf(vy, dt32, y), ly)
    xi = (x1 * F32(1.0 / (lx / nx))).astype(np.float32)
    yj = (y1 * F32(1.0 / (ly / ny))).astype(np.float32)
    i0, wx = weights32(xi, p)
    j0, wy = weights32(yj, p)
    jx = np.zeros(nx * ny, dtype=np.int64)
    jy = np.zeros(nx * ny, dtype=np.int64)
    for a in range(p + 1):
        ii = np.mod(i0 + a, nx)
        tx = (vx * wx[:, a]).astype(np.float32)
        ty = (vy * wx[:, a]).astype(np.float32)
        for b in range(p + 1):
            node = ii * ny + np.mod(j0 + b, ny)
            np.add.at(jx, node, contribution(tx, wy[:, b], scale))
            np.add.at(jy, node, contribution(ty, wy[:, b], scale))
    return x1, y1, jx.reshape(nx, ny), jy.reshape(nx, ny)
