"""Checkpoint and resume (pic_save_state / pic_load_state): a handle loaded with the state
of another steps on exactly as the other does -- bit for bit in both forms, whose current
sums are order-independent integers (int64 in the FP32 form, 128-bit in the FP64 path).
Saved mid sort interval (the sort's order and tile
offsets), after an odd number of CDF-2 steps (its swapped levels), with BDF rings whose
head has moved, and in 2D-3V with species.  Loading into another configuration or from a
truncated string is refused."""
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


FIELDS = ("jx", "jy", "rho", "phi", "ax", "ay", "bz", "dphidx", "daydy")

CASES = [
    ("fp32-bdf2-sorted", dict(stepper="bdf", bdf_order=2, precision=pic.FP32_FIX64,
                              sort_interval=4), 2, 7),
    ("fp32-cdf2", dict(stepper="cdf2", precision=pic.FP32_FIX64), 2, 7),
    ("fp32-dirk2", dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG, precision=pic.FP32_FIX64),
     2, 5),
    ("fp32-bdf3-3v-species", dict(stepper="bdf", bdf_order=3, precision=pic.FP32_FIX64, vdim=3,
                                  species=((-1.0, 1.0, 1.0 / 8192), (1.0, 4.0, 1.0 / 8192))),
     3, 5),
    ("fp64-cdf2", dict(stepper="cdf2"), 3, 5),
    ("fp64-bdf2-sorted", dict(stepper="bdf", bdf_order=2, sort_interval=3), 2, 4),
    ("fp32-bdf2-sorted-species", dict(stepper="bdf", bdf_order=2, precision=pic.FP32_FIX64,
                                      sort_interval=3,
                                      species=((-1.0, 1.0, 1.0 / 8192), (1.0, 4.0, 1.0 / 8192))),
     2, 5),
    ("fp32-cdf2-sorted-3v", dict(stepper="cdf2", precision=pic.FP32_FIX64, sort_interval=2,
                                 vdim=3), 2, 5),
    ("fp64-bdf2-3v", dict(stepper="bdf", bdf_order=2, vdim=3), 2, 4),
]


def _make(device, kw, seed):
    wl = workloads.weibel(32, 32, 8, 0.5, 0.01, seed, 3, nsteps=20)
    kw = dict(kw)
    kw.setdefault("weight", wl.weight)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, **kw)
    extra = {}
    if kw.get("vdim") == 3:
        extra["vz"] = np.random.default_rng(seed).uniform(-0.3, 0.3, wl.n)
    if kw.get("species"):
        extra["species"] = (np.arange(wl.n) % 2).astype(np.int32)
    return pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device, **extra)


def _snapshot(sim, three):
    out = dict(sim.particles())
    out.update({f: sim.field(f) for f in FIELDS + (("az", "jz") if three else ())})
    return out


@pytest.mark.parametrize("name,kw,before,after", CASES, ids=[c[0] for c in CASES])
def test_resume_steps_on_like_the_source(device, name, kw, before, after):
    three = kw.get("vdim") == 3
    a = _make(device, kw, seed=1)
    a.step(before * 2 + 1)
    state = a.save_state()
    a.step(after)
    ref = _snapshot(a, three)
    a.close()
    b = _make(device, kw, seed=2)      # other particles: everything comes from the state
    b.load_state(state)
    assert b.step_count == before * 2 + 1
    b.step(after)
    got = _snapshot(b, three)
    b.close()
    for k, v in ref.items():
        assert np.array_equal(got[k], v), k


def test_load_refuses_other_configurations(device):
    a = _make(device, dict(stepper="bdf", bdf_order=2), seed=1)
    a.step(2)
    state = a.save_state()
    b = _make(device, dict(stepper="bdf", bdf_order=3), seed=1)
    with pytest.raises(pic.PicError) as e:
        b.load_state(state)
    assert e.value.status == 1
    with pytest.raises(pic.PicError) as e:
        a.load_state(state[:len(state) // 2])
    assert e.value.status == 1
    with pytest.raises(pic.PicError) as e:
        a.load_state(b"x" * 200)
    assert e.value.status == 1
    a.load_state(state)              # its own state: accepted
    a.close()
    b.close()


def _make_cfg(device, seed, dt_scale=1.0, species=None, **kw):
    wl = workloads.weibel(32, 32, 8, 0.5, 0.01, seed, 3, nsteps=20)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt * dt_scale, p=3, stepper="bdf",
                          bdf_order=2, weight=wl.weight, species=species, **kw)
    extra = {}
    if species:
        extra["species"] = (np.arange(wl.n) % len(species)).astype(np.int32)
    return pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device, **extra)


def test_load_refuses_other_fp64_parameters(device):
    # Same layout (grid, order, stepper, particle count) but another dt, or one species
    # mass changed: the state belongs to another configuration.
    a = _make_cfg(device, 1)
    a.step(2)
    state = a.save_state()
    b = _make_cfg(device, 1, dt_scale=1.0 + 2.0 ** -40)
    with pytest.raises(pic.PicError) as e:
        b.load_state(state)
    assert e.value.status == 1
    b.close()
    tab = ((-1.0, 1.0, 1.0 / 8192), (1.0, 4.0, 1.0 / 8192))
    c = _make_cfg(device, 1, species=tab)
    c.step(1)
    sstate = c.save_state()
    d = _make_cfg(device, 1, species=((-1.0, 1.0, 1.0 / 8192), (1.0, 4.5, 1.0 / 8192)))
    with pytest.raises(pic.PicError) as e:
        d.load_state(sstate)
    assert e.value.status == 1
    e2 = _make_cfg(device, 2, species=tab)   # the same table: accepted
    e2.load_state(sstate)
    assert e2.step_count == 1
    for s in (a, c, d, e2):
        s.close()


def test_load_refuses_another_tile_width(device):
    # the saved sort order and tile offsets belong to the tiles they were made for
    a = _make_cfg(device, 3, precision=pic.FP32_FIX64, sort_interval=4, tile=4)
    a.step(3)
    state = a.save_state()
    b = _make_cfg(device, 3, precision=pic.FP32_FIX64, sort_interval=4, tile=8)
    with pytest.raises(pic.PicError) as e:
        b.load_state(state)
    assert e.value.status == 1
    c = _make_cfg(device, 4, precision=pic.FP32_FIX64, sort_interval=4, tile=4)
    c.load_state(state)
    a.step(2)
    c.step(2)
    for k, v in a.particles().items():
        assert np.array_equal(c.particles()[k], v), k
    for s in (a, b, c):
        s.close()


def test_diagnostics_log_restarts_at_a_load(device):
    # Records logged before a load are not returned after it, so step numbers never repeat
    # or go backwards.
    a = _make_cfg(device, 1)
    a.set_diagnostics(1)
    a.step(3)
    state = a.save_state()            # saved at step 3
    a.step(4)                         # steps 4..7 logged, not read
    a.load_state(state)               # back to step 3
    a.step(2)                         # steps 4, 5
    steps = [r["step"] for r in a.diagnostics_history()]
    assert steps == [4, 5], steps
    a.close()
