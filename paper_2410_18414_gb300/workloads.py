"""Seeded synthetic initial conditions for the PIC workloads.

This module only draws random numbers: positions and initial velocities of the
macro-electrons, plus the grid/time parameters that describe each workload.  It
holds none of the PIC method's arithmetic, so both the CUDA library and the CPU
oracle can be fed from it.  All draws use numpy's PCG64 with the stated seed.

Workloads (stand-ins for the two experiments of section 5; no dataset exists):
  * drifting_cloud -- a Gaussian electron cloud (sigma = 0.1 about the centre of
    [0,1]^2) drifting with v = (0.1, 0) plus a 0.01 Gaussian spread per component,
    over a uniform neutralising background (cf. section 5.2).
  * weibel -- two counter-streaming electron beams along y with drift +-v_d and an
    isotropic Maxwellian spread u_th in proper velocity u = gamma v, positions
    uniform in the periodic square of side 1.153896 c/omega_pe (cf. section 5.1,
    Table 2).  Particle k is in the +y beam for even k and the -y beam for odd k,
    so any prefix of the arrays is current-neutral to sampling noise.

The macro-particle weight is chosen so that the mean electron density gives
omega_pe = 1 in units c = eps0 = 1, |q| = m = 1:  w = Lx Ly / N_p.
"""
from dataclasses import dataclass

import numpy as np

WEIBEL_L = 1.153896


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    lx: float
    ly: float
    dt: float
    p: int
    stepper: str
    bdf_order: int
    nsteps: int
    x: np.ndarray
    y: np.ndarray
    vx: np.ndarray
    vy: np.ndarray

    @property
    def n(self):
        return len(self.x)

    @property
    def weight(self):
        return self.lx * self.ly / max(self.n, 1)


def _proper_to_velocity(ux, uy):
    # A Maxwellian "in u = gamma v" is sampled in u; the particle velocity is
    # u / sqrt(1 + |u|^2) (c = 1).  This is the sampler's definition.
    g = np.sqrt(1.0 + ux * ux + uy * uy)
    return ux / g, uy / g


def drifting_cloud(n=16384, nx=32, ny=32, seed=1, nsteps=100, stepper="bdf",
                   bdf_order=1, p=2):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.mod(rng.normal(0.5, 0.1, n), 1.0)
    y = np.mod(rng.normal(0.5, 0.1, n), 1.0)
    vx = 0.1 + 0.01 * rng.standard_normal(n)
    vy = 0.01 * rng.standard_normal(n)
    dx = 1.0 / nx
    return Workload("drifting_cloud", nx, ny, 1.0, 1.0, 0.5 * dx, p, stepper, bdf_order,
                    nsteps, x, y, vx, vy)


def weibel(nx=128, ny=128, ppc=64, v_drift=0.5, u_th=0.01, seed=2, p=3,
           stepper="bdf", bdf_order=2, nsteps=2000, n=None, length=WEIBEL_L):
    rng = np.random.Generator(np.random.PCG64(seed))
    if n is None:
        n = nx * ny * ppc
    x = rng.uniform(0.0, length, n)
    y = rng.uniform(0.0, length, n)
    u_d = v_drift / np.sqrt(1.0 - v_drift * v_drift)
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    ux = u_th * rng.standard_normal(n)
    uy = sign * u_d + u_th * rng.standard_normal(n)
    vx, vy = _proper_to_velocity(ux, uy)
    dx = length / nx
    return Workload("weibel", nx, ny, length, length, 0.4 * dx, p, stepper, bdf_order,
                    nsteps, x, y, vx, vy)


# Named workloads with the sizes they are measured at.
def cloud_32(seed=1):
    """32x32 drifting cloud, 16,384 particles, BDF-1, quadratic shapes, dt = dx/2, 100 steps."""
    return drifting_cloud(seed=seed)


def weibel_128(stepper="bdf", bdf_order=2, seed=2):
    """128x128 Weibel, 64 per cell (1,048,576), v_d = 0.5c, u_th = 0.01c, cubic, dt = 0.4 dx."""
    return weibel(128, 128, 64, 0.5, 0.01, seed, 3, stepper, bdf_order, 2000)


def weibel_512(stepper="dirk", seed=3):
    """512x512 Weibel, 100 per cell (26,214,400), v_d = 0.6c, u_th = 0.02c, quartic, dt = 0.4 dx."""
    return weibel(512, 512, 100, 0.6, 0.02, seed, 4, stepper, 2, 500)


def weibel_seeded(nx=128, ny=128, ppc=64, v_drift=0.5, u_th=0.01, seed=2, p=3, eps=1e-3,
                  stepper="bdf", bdf_order=2, nsteps=2000, length=WEIBEL_L):
    """The Weibel set-up with its lowest filamentation mode seeded: the two beams are
    displaced in antiphase along x, x -> x + s (eps / k) cos(k x) for the beam moving along
    s y (s = +-1), k = 2 pi / L, which modulates the beam densities by s eps sin(k x) to first
    order: a current J_y ~ sin(k x) (the growing mode's B_z ~ cos(k x)) with the charge
    density unchanged."""
    wl = weibel(nx, ny, ppc, v_drift, u_th, seed, p, stepper, bdf_order, nsteps, length=length)
    k = 2.0 * np.pi / length
    s = np.where(np.arange(wl.n) % 2 == 0, 1.0, -1.0)
    wl.x = np.mod(wl.x + s * (eps / k) * np.cos(k * wl.x), length)
    wl.name = "weibel_seeded"
    return wl


def weibel_adjoint_128(seed=5):
    """128x128 Weibel, 16 per cell (262,144), v_d = 0.5c, BDF-2, cubic, 200 steps."""
    return weibel(128, 128, 16, 0.5, 0.01, seed, 3, "bdf", 2, 200)


def ensemble_specs(count=256, seed0=1000):
    """Parameters of the batched-ensemble runs: run r draws, from PCG64(seed0 + r), a grid
    of N x N with N uniform in {32, 48, 64, 96, 128}, an integer number of particles per
    cell uniform in 16..64 and a drift uniform in (0.3, 0.7) c; u_th = 0.01 c, cubic
    shapes, BDF-2, dt = 0.4 dx, 300 steps."""
    specs = []
    for r in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + r))
        n_axis = int(rng.choice([32, 48, 64, 96, 128]))
        ppc = int(rng.integers(16, 65))
        v_drift = float(rng.uniform(0.3, 0.7))
        specs.append({"n": n_axis, "ppc": ppc, "v_drift": v_drift, "seed": seed0 + r})
    return specs


def ensemble_run(spec):
    """The particles of one ensemble run (seeded with the run's own seed)."""
    return weibel(spec["n"], spec["n"], spec["ppc"], spec["v_drift"], 0.01, spec["seed"], 3,
                  "bdf", 2, 300)
