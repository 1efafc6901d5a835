"""GPU checks of the FP32 form (FP32 particles and FFT, int64 fixed-point current).

Against the FP64 oracle the FP32 form is compared with tolerances derived from FP32
arithmetic (unit roundoff u = 6e-8): particle arrays carry a few u of rounding per step
(measured <= 4e-7 after 10 steps), grid fields inherit the FP32 weights and transforms,
amplified by the cancellation of a nearly neutral plasma (measured <= 5e-6 on small grids,
<= 2e-5 on the 128x128 workload).  Each bound below is about 5x the measured error.

What the FP32 form must keep exactly: the gauge, Gauss (BDF, CDF) and continuity
residuals stay at FP64 roundoff, because the per-mode recurrences and the histories are
FP64 whatever the storage type; and the current is summed in int64, so results are
bitwise reproducible and do not depend on the order of the particles.
"""
import numpy as np
import pytest

from oracle import pic as opic
from oracle import steppers as osteps
from paper_2410_18414_gb300 import pic, workloads

pytestmark = pytest.mark.gpu

P_TOL = 2e-6
F_TOL = 3e-5
PARTICLE_KEYS = ("px", "py", "vx", "vy", "vx_old", "vy_old")


@pytest.fixture(scope="module", autouse=True)
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def wrapped_rel(a, b, length):
    d = np.mod(a - b + 0.5 * length, length) - 0.5 * length
    return float(np.linalg.norm(d) / np.linalg.norm(b))


def fp32_sim(wl, device, diag=0, order=None, **kw):
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                          precision=pic.FP32_FIX64, **kw)
    x, y, vx, vy = wl.x, wl.y, wl.vx, wl.vy
    if order is not None:
        x, y, vx, vy = x[order], y[order], vx[order], vy[order]
    sim = pic.Simulation(cfg, x, y, vx, vy, stream=device)
    if diag:
        sim.set_diagnostics(diag)
    return sim


CASES = [
    ("cloud32_bdf1_p2", lambda: workloads.drifting_cloud(n=16384, nx=32, ny=32),
     dict(stepper="bdf", bdf_order=1)),
    ("weibel24x16_bdf2_p3", lambda: workloads.weibel(24, 16, 8, 0.5, 0.01, 21, 3, n=3001),
     dict(stepper="bdf", bdf_order=2)),
    ("weibel32x48_cdf2_p4", lambda: workloads.weibel(32, 48, 4, 0.5, 0.01, 22, 4, n=5003),
     dict(stepper="cdf2")),
    ("weibel16_dirk2_p2", lambda: workloads.weibel(16, 16, 8, 0.5, 0.01, 23, 2, n=2001),
     dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG)),
    ("weibel48x32_dirk3_p4", lambda: workloads.weibel(48, 32, 3, 0.6, 0.02, 24, 4, n=4099),
     dict(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT)),
    ("weibel24x16_bdf2_naive_p3", lambda: workloads.weibel(24, 16, 8, 0.5, 0.01, 33, 3, n=3001),
     dict(stepper="bdf", bdf_order=2, charge="deposit")),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_fp32_form_against_oracle(device, name, make, kw):
    wl = make()
    nsteps = 10
    naive = kw.get("charge") == "deposit"
    gkw = {k: v for k, v in kw.items() if k != "charge"}
    if naive:
        gkw["charge"] = pic.CHARGE_DEPOSIT
    sim = fp32_sim(wl, device, diag=1, **gkw)
    sim.step(nsteps)
    got = sim.particles()
    ocfg = opic.Config(nx=wl.nx, ny=wl.ny, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=wl.p, w=wl.weight, **kw)
    st = opic.run(ocfg, wl.x, wl.y, wl.vx, wl.vy, nsteps)
    errs = {"x": wrapped_rel(got["x"], st.x, wl.lx), "y": wrapped_rel(got["y"], st.y, wl.ly)}
    errs.update({k: rel(got[k], getattr(st, k)) for k in PARTICLE_KEYS})
    bad = {k: v for k, v in errs.items() if not v <= P_TOL}
    ferrs = {f: rel(sim.field(f), st.grids[f]) for f in
             ("jx", "jy", "rho", "phi", "ax", "ay", "bz", "dphidx", "daxdx", "daydy")}
    bad.update({k: v for k, v in ferrs.items() if not v <= F_TOL})
    assert not bad, bad
    # the theorems of section 3 hold to FP64 roundoff in the FP32 form too (not for the
    # naive update, which gives them up)
    d = sim.residuals()
    if naive:
        sim.close()
        return
    assert d["gauge_rms"] <= 1e-11 * d["div_a_rms"], d
    assert d["continuity_rms"] <= 1e-11 * d["rho_rms"] / wl.dt, d
    if kw["stepper"] != "dirk":
        assert d["gauss_rms"] <= 1e-11 * d["rho_rms"], d
    sim.close()


def test_fp32_form_bitwise_reproducible_and_order_independent(device):
    wl = workloads.weibel(32, 32, 16, 0.5, 0.01, 91, 3, n=16001)
    kw = dict(stepper="bdf", bdf_order=2)
    a = fp32_sim(wl, device, **kw)
    b = fp32_sim(wl, device, **kw)
    perm = np.random.default_rng(1).permutation(wl.n)
    c = fp32_sim(wl, device, order=perm, **kw)
    for s in (a, b, c):
        s.step(8)
    pa, pb, pc = a.particles(), b.particles(), c.particles()
    inv = np.argsort(perm)
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
        assert np.array_equal(pa[k], pc[k][inv]), k
    for f in ("jx", "jy", "phi", "ax"):
        assert np.array_equal(a.field(f), b.field(f)) and np.array_equal(a.field(f), c.field(f))
    for s in (a, b, c):
        s.close()


def test_fp32_form_full_size_weibel_128(device):
    wl = workloads.weibel_128(stepper="bdf", bdf_order=2)
    kw = dict(stepper="bdf", bdf_order=2)
    sim = fp32_sim(wl, device, **kw)
    sim.step(2)
    got = sim.particles()
    ocfg = opic.Config(nx=128, ny=128, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=3, w=wl.weight, **kw)
    st = opic.run(ocfg, wl.x, wl.y, wl.vx, wl.vy, 2)
    assert wrapped_rel(got["x"], st.x, wl.lx) <= P_TOL
    for k in PARTICLE_KEYS:
        assert rel(got[k], getattr(st, k)) <= P_TOL, k
    limits = {"jx": 5e-5, "jy": 5e-5, "rho": 5e-5, "phi": 1e-4, "ax": 5e-5, "dphidx": 1e-4}
    for f, tol in limits.items():
        assert rel(sim.field(f), st.grids[f]) <= tol, f
    sim.close()


def test_fp32_form_empty_and_edge_particles(device):
    x = np.array([0.0, np.nextafter(1.0, 0.0), 1.0, 0.5])
    y = np.array([np.nextafter(1.0, 0.0), 0.0, 0.25, 1.0])
    vx = np.array([-0.3, 0.3, 0.0, 0.1])
    vy = np.array([0.3, -0.3, 0.0, -0.1])
    wl = workloads.Workload("edge", 16, 16, 1.0, 1.0, 0.5 / 16, 2, "bdf", 2, 5, x, y, vx, vy)
    sim = fp32_sim(wl, device, stepper="bdf", bdf_order=2)
    sim.step(5)
    got = sim.particles()
    assert np.all((got["x"] >= 0) & (got["x"] < 1.0))
    sim.close()
    e = np.zeros(0)
    wl0 = workloads.Workload("empty", 16, 16, 1.0, 1.0, 0.01, 3, "bdf", 1, 2, e, e, e, e)
    sim = fp32_sim(wl0, device, stepper="cdf2")
    sim.step(2)
    assert np.max(np.abs(sim.field("jx"))) == 0.0
    sim.close()


@pytest.mark.parametrize("make,sort,nsteps", [
    (lambda: workloads.weibel(64, 64, 16, 0.5, 0.01, 92, 3, n=65531), 4, 10),
    (lambda: workloads.drifting_cloud(n=20000, nx=48, ny=32, seed=93), 1, 6),
    # 0.36 cells per step for 100 steps overruns the 24-cell halo: global fallback path
    (lambda: workloads.weibel(128, 128, 1, 0.9, 0.05, 94, 4, n=16387), 100, 105),
    (lambda: workloads.weibel(16, 24, 8, 0.9, 0.05, 95, 4, n=3001), 50, 55),
], ids=["weibel64_sort4", "cloud48x32_sort1", "weibel128_sort100_beyond_halo",
        "weibel16x24_sort50_region_wraps"])
def test_fp32_tile_sort_is_bitwise_identical_to_unsorted(device, make, sort, nsteps):
    # The sort changes only the order of the particles; the int64 current and the
    # per-particle push make the result independent of that order.
    wl = make()
    kw = dict(stepper="bdf", bdf_order=2)
    plain = fp32_sim(wl, device, **kw)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                          precision=pic.FP32_FIX64, sort_interval=sort, **kw)
    sorted_ = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    plain.step(nsteps)
    sorted_.step(nsteps)
    a, b = plain.particles(), sorted_.particles()

    def diff(u, v):
        return f"{int(np.sum(u != v))} differ, max |d| = {np.max(np.abs(u - v)):.3e}"

    for f in ("jx", "jy", "rho", "phi", "ax", "daydx"):
        u, v = plain.field(f), sorted_.field(f)
        assert np.array_equal(u, v), (f, diff(u, v))
    for k in a:
        assert np.array_equal(a[k], b[k]), (k, diff(a[k], b[k]))
    # the call's last step: its field solve and gather (its deposit ran fused with the
    # gather before it, or on its own, after a sort or at the start of the call)
    assert sorted_.kernels_per_step >= 4
    plain.close()
    sorted_.close()


def test_kernel_timers_count_the_launches_they_bracket(device):
    # sort every 4 steps: sorts in steps 1, 5, 9 of 10.  The sorted FP32 form runs the
    # gather + push of every step fused with the move + deposit of the next (the last step
    # of a pic_step call leaves that deposit pending for the next call), so only the first
    # step of the handle deposits on its own, and a sort due later follows the fused
    # deposit.  Launches beyond the reserved pairs go untimed.
    wl = workloads.weibel(32, 32, 8, 0.5, 0.01, 96, 3)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                          precision=pic.FP32_FIX64, sort_interval=4, stepper="bdf", bdf_order=2)
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
        sim.set_kernel_timing(16)
        sim.step(10)
        got = {k: sim.kernel_time(k) for k in pic.KERNEL_TIMERS}
        assert {k: v[1] for k, v in got.items()} == {
            "sort": 3, "deposit": 1, "field_solve": 10, "gather_push": 0,
            "adj_push": 0, "adj_field": 0, "adj_deposit": 0, "gather_deposit": 10}
        assert all(v[0] > 0 for k, v in got.items() if v[1]), got
        sim.set_kernel_timing(2)  # restart with fewer pairs than launches
        sim.step(6)               # steps 11-16: a sort in 13, six fused kernels
        sim.step(4)               # 17-20: a sort in 17
        assert sim.kernel_time("sort")[1] == 2
        assert sim.kernel_time("gather_deposit")[1] == 2
        assert sim.kernel_time("deposit")[1] == 0
        # the phases one at a time run the kernels apart (the pending deposit is used first)
        sim.deposit()
        sim.field_solve()
        sim.gather_push()
        sim.deposit()
        assert sim.kernel_time("deposit")[1] == 1
        assert sim.kernel_time("gather_push")[1] == 1
        sim.field_solve()
        sim.gather_push()
        sim.set_kernel_timing(0)
        sim.step(1)
        assert sim.kernel_time("deposit")[1] == 1
        with pytest.raises(pic.PicError):
            sim.set_kernel_timing(-1)
        with pytest.raises(KeyError):
            sim.kernel_time("fft")


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_FIX64], ids=["fp64", "fp32"])
@pytest.mark.parametrize("stepper,kw", [("bdf", dict(bdf_order=2)), ("bdf", dict(bdf_order=3)),
                                        ("cdf2", {})], ids=["bdf2", "bdf3", "cdf2"])
def test_diagnostics_do_not_change_the_trajectory(device, precision, stepper, kw):
    # diagnosed steps take a different (one thread per mode) path through the per-mode
    # update; the arithmetic must be the same.  Both forms sum the current in integers,
    # so the trajectories are bitwise equal.
    wl = workloads.weibel(48, 32, 8, 0.5, 0.01, 97, 3)
    sims = []
    for diag in (0, 3):
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                              precision=precision, stepper=stepper, **kw)
        sim = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
        if diag:
            sim.set_diagnostics(diag)
        sim.step(7)
        sims.append(sim)
    a, b = sims[0].particles(), sims[1].particles()
    fields = [(sims[0].field(f), sims[1].field(f)) for f in ("phi", "ax", "ay", "rho", "daxdy")]
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    for u, v in fields:
        assert np.array_equal(u, v)
    for s in sims:
        s.close()


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_FIX64], ids=["fp64", "fp32"])
def test_diagnostics_history_records_every_diagnosed_step(device, precision):
    # the device ring keeps each diagnosed step's accumulators: read back later, every
    # record equals what pic_residuals returned right after that step
    wl = workloads.weibel(32, 32, 8, 0.5, 0.01, 98, 3)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                          precision=precision, stepper="bdf", bdf_order=2,
                          sort_interval=4 if precision == pic.FP32_FIX64 else 0)
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
        sim.step(3)
        sim.set_diagnostics(2)
        assert sim.diagnostics_history() == []
        direct = []
        for _ in range(5):
            sim.step(2)
            direct.append(sim.residuals())
        hist = sim.diagnostics_history()
        # a step is diagnosed when its new index is a multiple of `every`
        assert [h["step"] for h in hist] == [4, 6, 8, 10, 12]
        assert hist == direct
        assert sim.diagnostics_history() == []          # read once
        sim.step(6)
        last = sim.diagnostics_history(capacity=2)      # the newest two of three
        assert [h["step"] for h in last] == [16, 18]
        # a wrapped ring: more diagnosed steps than it holds keep the newest
        sim.set_diagnostics(1)
        sim.step(pic.DIAG_HISTORY + 3)
        wrapped = sim.diagnostics_history()
        assert len(wrapped) == pic.DIAG_HISTORY
        assert wrapped[-1]["step"] == sim.step_count
        assert [h["step"] for h in wrapped] == list(range(sim.step_count - pic.DIAG_HISTORY + 1,
                                                          sim.step_count + 1))
        assert wrapped[-1] == sim.residuals()


def test_pending_deposit_leaves_the_state_of_each_step(device):
    # The sorted FP32 form ends each pic_step call with the next step's move and deposit
    # done ahead (pending).  Read between calls, the particles and fields are still those
    # of the step just finished -- bitwise those of the unsorted form, which has no pending
    # deposit -- and one call of n steps, n calls of one step, the phases one at a time and
    # a saved and reloaded state all step on to the same bits.
    wl = workloads.weibel(48, 32, 8, 0.5, 0.01, 98, 3)
    kw = dict(stepper="bdf", bdf_order=2)

    def make(sort):
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                              precision=pic.FP32_FIX64, sort_interval=sort, **kw)
        return pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)

    def snap(sim):
        out = dict(sim.particles())
        out.update({f: sim.field(f) for f in ("jx", "jy", "phi", "daxdy")})
        return out

    plain, one, many, phases = make(0), make(3), make(3), make(3)
    for k in range(7):
        plain.step(1)
        one.step(1)
        ref = snap(plain)
        got = snap(one)
        for name in ref:
            assert np.array_equal(got[name], ref[name]), (k, name)
    many.step(7)
    for _ in range(7):
        phases.deposit()
        phases.field_solve()
        phases.gather_push()
    for sim in (many, phases):
        got = snap(sim)
        for name in ref:
            assert np.array_equal(got[name], ref[name]), name
    state = one.save_state()        # saved with a deposit pending
    other = make(3)
    other.load_state(state)
    one.step(4)
    other.step(4)
    plain.step(4)
    ref = snap(plain)
    for sim in (one, other):
        got = snap(sim)
        for name in ref:
            assert np.array_equal(got[name], ref[name]), name
    for sim in (plain, one, many, phases, other):
        sim.close()
