"""GPU checks of caller-owned particle arrays (pic_init_bound): a simulation stepping the
caller's CUDA tensors in place gives the same bits as one that copies the particles in
(both forms, BDF-2 and CDF-2), its tensors are the state (no read-back needed), the
velocity pairs exchange roles every step as pic_velocity_slot says, and checkpoints and
ensembles work on it."""
import numpy as np
import pytest

from paper_2410_18414_gb300 import pic, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(pic.LIB_PATH):
        from paper_2410_18414_gb300 import build
        build.build()
    pic.load_library()
    torch.cuda.set_device(0)
    return torch


def _bound(torch, cfg, wl, stream):
    dtype = torch.float32 if cfg.precision == pic.FP32_FIX64 else torch.float64
    arrays = {k: torch.zeros(wl.n, dtype=dtype, device="cuda") for k in pic.Simulation.BOUND_KEYS}
    for k, v in (("x", wl.x), ("y", wl.y), ("vx", wl.vx), ("vy", wl.vy)):
        arrays[k].copy_(torch.tensor(v))  # the storage type's rounding of x^0, v^0
    torch.cuda.synchronize()
    return pic.Simulation.bound(cfg, arrays, stream=stream), arrays


def _state_of_tensors(sim):
    (vx, vy), (vxo, vyo) = sim.velocities()
    a = sim.arrays
    return {"x": a["x"], "y": a["y"], "px": a["px"], "py": a["py"], "vx": vx, "vy": vy,
            "vx_old": vxo, "vy_old": vyo}


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_FIX64], ids=["fp64", "fp32"])
@pytest.mark.parametrize("stepper,kw", [("bdf", dict(bdf_order=2)), ("cdf2", {})],
                         ids=["bdf2", "cdf2"])
def test_bound_tensors_step_like_a_copying_handle(torch_mod, precision, stepper, kw):
    torch = torch_mod
    wl = workloads.weibel(48, 32, 16, 0.5, 0.01, 41, 3)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, stepper=stepper,
                          weight=wl.weight, precision=precision, **kw)
    stream = torch.cuda.current_stream().cuda_stream
    ref = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=stream)
    sim, arrays = _bound(torch, cfg, wl, stream)
    for nsteps, slot in ((1, 1), (2, 1), (4, 1)):  # 1, 3 and 7 steps done
        ref.step(nsteps)
        sim.step(nsteps)
        assert sim.velocity_slot == slot == ref.velocity_slot
        want = ref.particles()
        got = {k: v.double().cpu().numpy() for k, v in _state_of_tensors(sim).items()}
        for k in want:
            assert np.array_equal(got[k], want[k]), (nsteps, k)
        read = sim.particles()  # the library's read-back of the same tensors
        for k in want:
            assert np.array_equal(read[k], want[k]), k
        for f in ("jx", "phi", "ay", "daxdy"):
            assert np.array_equal(sim.field(f), ref.field(f)), f
    ref.step(1)
    sim.step(1)
    assert sim.velocity_slot == 0
    ref.close()
    sim.close()
    # the tensors outlive the handle and keep the last state
    assert torch.isfinite(arrays["px"]).all()


def test_bound_checkpoint_and_ensemble(torch_mod):
    torch = torch_mod
    wl = workloads.weibel(32, 32, 16, 0.5, 0.01, 42, 3)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf", bdf_order=2,
                          weight=wl.weight, precision=pic.FP32_FIX64)
    s1 = torch.cuda.Stream()
    sim, _ = _bound(torch, cfg, wl, s1.cuda_stream)
    solo = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=torch.cuda.Stream().cuda_stream)
    sim.step(3)
    state = sim.save_state()
    other, _ = _bound(torch, cfg, workloads.weibel(32, 32, 16, 0.5, 0.01, 43, 3), s1.cuda_stream)
    other.load_state(state)  # into another bound handle's tensors
    with pic.Ensemble([sim], torch.cuda.Stream().cuda_stream) as ens:
        P = ens.period
        ens.step(P)
    solo.step(3 + P)
    other.step(P)
    for k, v in solo.particles().items():
        assert np.array_equal(sim.particles()[k], v), k
        assert np.array_equal(other.particles()[k], v), k
    for s in (sim, solo, other):
        s.close()


def test_bound_rejects_sorting_and_wrong_tensors(torch_mod):
    torch = torch_mod
    wl = workloads.weibel(16, 16, 8, 0.5, 0.01, 44, 2)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=2, weight=wl.weight,
                          sort_interval=4)
    with pytest.raises(pic.PicError) as e:
        _bound(torch, cfg, wl, None)
    assert e.value.status == 2
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=2, weight=wl.weight,
                          precision=pic.FP32_FIX64)
    arrays = {k: torch.zeros(wl.n, dtype=torch.float64, device="cuda")
              for k in pic.Simulation.BOUND_KEYS}
    with pytest.raises(TypeError):
        pic.Simulation.bound(cfg, arrays)  # FP32 form: float32 tensors


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_FIX64], ids=["fp64", "fp32"])
def test_bound_empty_particle_set(torch_mod, precision):
    torch = torch_mod
    dtype = torch.float32 if precision == pic.FP32_FIX64 else torch.float64
    cfg = pic.make_config(16, 16, 1.0, 1.0, 0.01, p=3, stepper="bdf", bdf_order=2, weight=1.0,
                          precision=precision)
    arrays = {k: torch.zeros(0, dtype=dtype, device="cuda") for k in pic.Simulation.BOUND_KEYS}
    with pic.Simulation.bound(cfg, arrays,
                              stream=torch.cuda.current_stream().cuda_stream) as sim:
        sim.set_diagnostics(1)
        sim.step(3)
        for f in ("jx", "phi", "ax", "dphidx"):
            assert np.max(np.abs(sim.field(f))) == 0.0
        assert sim.residuals()["kinetic"] == 0.0
        assert all(len(v) == 0 for v in sim.particles().values())
