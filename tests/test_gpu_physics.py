"""Physics checks on the 128x128 Weibel configuration: the linear growth rate of the
magnetic energy against the cold two-beam filamentation theory (reading R11), from particle
noise and from a seeded single mode.

Two symmetric cold beams of total plasma frequency w_p, speeds +-v0 along y (gamma0),
and a wave vector k along x give the dispersion relation

    w^4 - w^2 (k^2 c^2 + w_p^2 / gamma0) - k^2 c^2 w_p^2 beta0^2 / gamma0 = 0,

whose unstable root grows at Gamma(k)^2 = (sqrt(a^2 + 4 k^2 c^2 w_p^2 beta0^2 / gamma0) - a) / 2
with a = k^2 c^2 + w_p^2 / gamma0 (Gamma -> beta0 w_p / sqrt(gamma0) for large k).  The
magnetic energy of a mode grows at 2 Gamma.  The observable is the energy of B_z in the
four lowest modes k = (m 2 pi / L, 0), m = 1..4 (B_z perturbations vary across the beams),
fitted over t in [2.5, 6.5] w_p^-1, inside the linear phase of the 2000-step run.  The
beams are warm (u_th = 0.01 c) and start from particle noise, so agreement is expected to
about 20%, as the paper reports it (by eye, from its growth-rate figures).
"""
import numpy as np
import pytest

from oracle import steppers as osteps
from paper_2410_18414_gb300 import pic, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(pic.LIB_PATH):
        from paper_2410_18414_gb300 import build
        build.build()
    pic.load_library()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


def cold_filamentation_rate(k, beta0, wp=1.0, c=1.0):
    g0 = 1.0 / np.sqrt(1.0 - beta0 * beta0)
    a = k * k * c * c + wp * wp / g0
    return np.sqrt((np.sqrt(a * a + 4.0 * k * k * c * c * wp * wp * beta0 * beta0 / g0) - a) / 2.0)


def test_cold_rate_limits():
    # large k: beta0 w_p / sqrt(gamma0) (at k c = 1000 w_p within 1e-6 relative); k -> 0:
    # no growth
    g0 = 1.0 / np.sqrt(1.0 - 0.25)
    assert abs(cold_filamentation_rate(1e3, 0.5) / (0.5 / np.sqrt(g0)) - 1.0) < 1e-5
    assert cold_filamentation_rate(1e-6, 0.5) < 1e-5


@pytest.mark.parametrize("stepper,kw", [("bdf", dict(bdf_order=2)), ("cdf2", {}),
                                        ("dirk", dict(dirk=osteps.DIRK2_QIN_ZHANG))],
                         ids=["bdf2", "cdf2", "dirk2"])
def test_weibel_magnetic_growth_rate(device, stepper, kw):
    wl = workloads.weibel_128(stepper=stepper)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper=stepper,
                          weight=wl.weight, precision=pic.FP32_FIX64, sort_interval=8, **kw)
    modes = (1, 2, 3, 4)
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
        t, energy = [], []
        for i in range(200):
            sim.step(10)
            bh = np.fft.fft2(sim.field("bz"))
            t.append((i + 1) * 10 * wl.dt)
            energy.append(sum(abs(bh[m, 0]) ** 2 + abs(bh[-m, 0]) ** 2 for m in modes))
    t, le = np.array(t), np.log(np.array(energy))
    window = (t >= 2.5) & (t <= 6.5)
    rate = np.polyfit(t[window], le[window], 1)[0]
    theory = 2.0 * max(cold_filamentation_rate(2 * np.pi * m / wl.lx, 0.5) for m in modes)
    print(f"{stepper}: magnetic energy growth {rate:.3f}, cold theory {theory:.3f}")
    assert abs(rate / theory - 1.0) < 0.2, (rate, theory)


@pytest.mark.parametrize("stepper,kw,v_drift",
                         [("bdf", dict(bdf_order=2), 0.5), ("bdf", dict(bdf_order=2), 0.6),
                          ("cdf2", {}, 0.5), ("dirk", dict(dirk=osteps.DIRK2_QIN_ZHANG), 0.5)],
                         ids=["bdf2-0.5c", "bdf2-0.6c", "cdf2-0.5c", "dirk2-0.5c"])
def test_seeded_mode_growth_rate(device, stepper, kw, v_drift):
    # The lowest filamentation mode k = 2 pi / L seeded (workloads.weibel_seeded, eps = 1e-2,
    # about ten times the noise in that mode): |B_z(k)| grows at the cold rate Gamma(k)
    # once the seed has projected onto the growing eigenmode.  Fit of ln(|B_z(k, 0)| +
    # |B_z(-k, 0)|) over t in [3, 7.5] w_p^-1, 2 e-folds; measured +2.9% (0.5c) and +1.9%
    # (0.6c) on GB300 (all three steppers agree to 1e-3); bound 10%.
    wl = workloads.weibel_seeded(eps=1e-2, v_drift=v_drift, stepper=stepper)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper=stepper,
                          weight=wl.weight, precision=pic.FP32_FIX64, sort_interval=8, **kw)
    t, amp = [], []
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
        for i in range(420):
            sim.step(5)
            bh = np.fft.fft2(sim.field("bz"))
            t.append((i + 1) * 5 * wl.dt)
            amp.append(abs(bh[1, 0]) + abs(bh[-1, 0]))
    t, la = np.array(t), np.log(np.array(amp))
    window = (t >= 3.0) & (t <= 7.5)
    rate = np.polyfit(t[window], la[window], 1)[0]
    theory = cold_filamentation_rate(2 * np.pi / wl.lx, v_drift)
    print(f"{stepper} {v_drift}c: seeded mode growth {rate:.4f}, cold theory {theory:.4f}")
    assert abs(rate / theory - 1.0) < 0.1, (rate, theory)
