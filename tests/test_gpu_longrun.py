"""Long runs of the FP32 form against the plain FP64 path, compared on what the paper plots
for its Weibel runs (section 5.1): the magnetic energy history and its growth rate, the
electric and kinetic energy histories, and the gauge and continuity residuals over the
whole run.  Single trajectories of the two forms decorrelate (the instability amplifies
the rounding differences), so long runs are compared on these histories, not on states.

The 128x128 Weibel configuration (1,048,576 particles, cubic shapes, dt = 0.4 dx), the
2000 steps of its linear phase, with the diagnostics of every tenth step logged on the
device (pic_diagnostics_history).
"""
import numpy as np
import pytest

from oracle import steppers as osteps
from paper_2410_18414_gb300 import pic, workloads

pytestmark = pytest.mark.gpu

# Bounds, about five times the largest difference measured on GB300 over the three
# steppers (in parentheses; the design notes list both).
RATE_TOL = 1e-4      # W_B growth rate over t in [2.5, 6.5], FP32 / FP64 - 1 (<= 1.7e-5)
WB_TOL = 3e-4        # max |W_B32 / W_B64 - 1| over the linear phase (<= 6.6e-5)
WE_TOL = 6e-4        # max |W_E32 / W_E64 - 1| over the run (<= 1.2e-4)
KE_TOL = 2e-8        # max |KE32 / KE64 - 1| over the run (<= 4.6e-9)
GAUGE_TOL = 1e-11    # gauge_rms / div_a_rms and continuity_rms / rho_rms, every record
                     # (<= 1.3e-12 and 3.5e-14)


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


def history(device, wl, stepper, kw, precision, sort):
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper=stepper,
                          weight=wl.weight, precision=precision, sort_interval=sort, **kw)
    recs = []
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
        sim.set_diagnostics(10)
        for _ in range(4):
            sim.step(wl.nsteps // 4)
            recs += sim.diagnostics_history()
    out = {k: np.array([r[k] for r in recs]) for k in recs[0]}
    out["t"] = out["step"] * wl.dt
    return out


@pytest.mark.parametrize("stepper,kw", [("bdf", dict(bdf_order=2)), ("cdf2", {}),
                                        ("dirk", dict(dirk=osteps.DIRK2_QIN_ZHANG))],
                         ids=["bdf2", "cdf2", "dirk2"])
def test_fp32_form_long_run_histories_match_fp64(device, stepper, kw):
    wl = workloads.weibel_128(stepper=stepper)
    h32 = history(device, wl, stepper, kw, pic.FP32_FIX64, 8)
    h64 = history(device, wl, stepper, kw, pic.FP64, 0)
    assert len(h32["t"]) == len(h64["t"]) == wl.nsteps // 10
    assert np.array_equal(h32["step"], h64["step"])
    t = h32["t"]
    window = (t >= 2.5) & (t <= 6.5)
    rate32 = np.polyfit(t[window], np.log(h32["w_b"][window]), 1)[0]
    rate64 = np.polyfit(t[window], np.log(h64["w_b"][window]), 1)[0]
    d = {
        "rate": abs(rate32 / rate64 - 1.0),
        "w_b": np.max(np.abs(h32["w_b"][t <= 6.5] / h64["w_b"][t <= 6.5] - 1.0)),
        "w_e": np.max(np.abs(h32["w_e"] / h64["w_e"] - 1.0)),
        "ke": np.max(np.abs(h32["kinetic"] / h64["kinetic"] - 1.0)),
    }
    res = {}
    for name, h in (("fp32", h32), ("fp64", h64)):
        res[name] = (np.max(h["gauge_rms"] / h["div_a_rms"]),
                     np.max(h["continuity_rms"] / h["rho_rms"]))
    print(f"{stepper}: W_B rate {rate32:.4f} (FP32) {rate64:.4f} (FP64); differences {d}; "
          f"residuals {res}")
    assert d["rate"] < RATE_TOL
    assert d["w_b"] < WB_TOL
    assert d["w_e"] < WE_TOL
    assert d["ke"] < KE_TOL
    for name, (g, c) in res.items():
        assert g < GAUGE_TOL and c < GAUGE_TOL, (name, g, c)
