"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

Tolerance, per particle array and per grid field after the given number of steps (plain
FP64 path): relative L2 error <= 1e-12, and element by element max |a - b| <= 1e-12 max |b|
(so an error confined to a few nodes or particles cannot hide in the norm).  Positions
are compared modulo the period.  Inputs are the seeded workloads of paper_2410_18414_gb300.workloads.
"""
import numpy as np
import pytest

from oracle import pic as opic
from oracle import steppers as osteps
from paper_2410_18414_gb300 import pic, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12
PARTICLE_KEYS = ("px", "py", "vx", "vy", "vx_old", "vy_old")
ORACLE_KEYS = {"vx_old": "vx_old", "vy_old": "vy_old"}
FIELD_KEYS = ("jx", "jy", "rho", "phi", "ax", "ay", "bz", "dphidx", "dphidy", "daxdx", "daxdy",
              "daydx", "daydy")
ORACLE_FIELD = {"gax": "ax", "gay": "ay"}


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import os
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


def maxrel(a, b):
    """max |a - b| over the elements, relative to max |b|."""
    a, b = np.ravel(a), np.ravel(b)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def wrapped_maxrel(a, b, length):
    d = np.mod(a - b + 0.5 * length, length) - 0.5 * length
    if d.size == 0:
        return 0.0
    return float(np.max(np.abs(d)) / max(np.max(np.abs(b)), 1e-300))


# the CDF-2 forms of section 3.1: library stepper name -> (oracle stepper, oracle cdf_form)
CDF_FORMS = {"cdf2": ("cdf2", "implicit"), "cdf2_semi": ("cdf2", "semi"),
             "cdf2_explicit": ("cdf2", "explicit")}


def run_both(wl, device, nsteps, stepper="bdf", bdf_order=1, dirk=None, p=None, diag=0,
             charge=pic.CHARGE_CONTINUITY):
    p = wl.p if p is None else p
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=p, stepper=stepper,
                          bdf_order=bdf_order, dirk=dirk, weight=wl.weight, charge=charge)
    sim = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    if diag:
        sim.set_diagnostics(diag)
    sim.step(nsteps)
    ostepper, form = CDF_FORMS.get(stepper, (stepper, "implicit"))
    ocfg = opic.Config(nx=wl.nx, ny=wl.ny, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=p, stepper=ostepper,
                       bdf_order=bdf_order, dirk=dirk, w=wl.weight, cdf_form=form,
                       charge="deposit" if charge == pic.CHARGE_DEPOSIT else "continuity")
    st = opic.run(ocfg, wl.x, wl.y, wl.vx, wl.vy, nsteps)
    return sim, st, ocfg


def compare(sim, st, wl, fields=FIELD_KEYS, tol=TOL):
    got = sim.particles()
    errs = {"x": wrapped_rel(got["x"], st.x, wl.lx), "y": wrapped_rel(got["y"], st.y, wl.ly),
            "x max": wrapped_maxrel(got["x"], st.x, wl.lx),
            "y max": wrapped_maxrel(got["y"], st.y, wl.ly)}
    for k in PARTICLE_KEYS:
        errs[k] = rel(got[k], getattr(st, k))
        errs[k + " max"] = maxrel(got[k], getattr(st, k))
    for f in fields:
        g, o = sim.field(f), st.grids[ORACLE_FIELD.get(f, f)]
        errs[f] = rel(g, o)
        errs[f + " max"] = maxrel(g, o)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad
    return errs


CASES = [
    # name, workload, nsteps, stepper kwargs
    ("cloud32_bdf1_p2", lambda: workloads.drifting_cloud(n=16384, nx=32, ny=32), 10,
     dict(stepper="bdf", bdf_order=1)),
    ("weibel24x16_bdf2_p3", lambda: workloads.weibel(24, 16, 8, 0.5, 0.01, 21, 3, n=3001), 10,
     dict(stepper="bdf", bdf_order=2)),
    ("weibel32x48_cdf2_p4", lambda: workloads.weibel(32, 48, 4, 0.5, 0.01, 22, 4, n=5003), 10,
     dict(stepper="cdf2")),
    ("weibel16_dirk2_p2", lambda: workloads.weibel(16, 16, 8, 0.5, 0.01, 23, 2, n=2001), 10,
     dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG)),
    ("weibel48x32_dirk3_p4", lambda: workloads.weibel(48, 32, 3, 0.6, 0.02, 24, 4, n=4099), 10,
     dict(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT)),
    ("cloud16_bdf3_p3", lambda: workloads.drifting_cloud(n=2500, nx=16, ny=16, seed=25, p=3), 10,
     dict(stepper="bdf", bdf_order=3)),
    ("cloud96x64_cdf2_p2", lambda: workloads.drifting_cloud(n=7777, nx=96, ny=64, seed=26), 6,
     dict(stepper="cdf2")),
    ("weibel32x24_cdf2semi_p3", lambda: workloads.weibel(32, 24, 8, 0.5, 0.01, 27, 3, n=6001), 10,
     dict(stepper="cdf2_semi")),
    ("weibel24x32_cdf2explicit_p2", lambda: workloads.weibel(24, 32, 8, 0.5, 0.01, 28, 2, n=5999),
     10, dict(stepper="cdf2_explicit")),
    ("weibel16_dirk2printed_p3", lambda: workloads.weibel(16, 16, 8, 0.5, 0.01, 29, 3, n=2047), 10,
     dict(stepper="dirk", dirk=osteps.DIRK2_AS_PRINTED)),
    # the naive update of section 5: rho^{n+1} deposited instead of from continuity
    ("weibel24x16_bdf2_naive_p2", lambda: workloads.weibel(24, 16, 8, 0.5, 0.01, 30, 2, n=3001), 10,
     dict(stepper="bdf", bdf_order=2, charge=pic.CHARGE_DEPOSIT)),
    ("weibel16_dirk2_naive_p3", lambda: workloads.weibel(16, 16, 8, 0.5, 0.01, 31, 3, n=2047), 10,
     dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG, charge=pic.CHARGE_DEPOSIT)),
]


@pytest.mark.parametrize("name,make,nsteps,kw", CASES, ids=[c[0] for c in CASES])
def test_parity_small(device, name, make, nsteps, kw):
    wl = make()
    sim, st, _ = run_both(wl, device, nsteps, **kw)
    compare(sim, st, wl)
    assert sim.step_count == nsteps
    sim.close()


def test_parity_step_phases_match_pic_step(device):
    # pic_deposit + pic_field_solve + pic_gather_push == pic_step(1), bit for bit.
    wl = workloads.weibel(16, 16, 8, 0.5, 0.01, 31, 3, n=2049)
    cfg = pic.make_config(16, 16, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf", bdf_order=2,
                          weight=wl.weight)
    a = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    b = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    for _ in range(3):
        a.deposit()
        a.field_solve()
        a.gather_push()
    b.step(3)
    pa, pb = a.particles(), b.particles()
    for k in ("x", "px", "vy_old"):
        assert rel(pa[k], pb[k]) < 1e-13
    with pytest.raises(pic.PicError):
        a.field_solve()          # out of order: no deposit yet
    a.close()
    b.close()


@pytest.mark.parametrize("stepper,kw", [("bdf", dict(bdf_order=1)), ("bdf", dict(bdf_order=2)),
                                        ("cdf2", {}), ("cdf2_semi", {}),
                                        ("dirk", dict(dirk=osteps.DIRK2_QIN_ZHANG))])
def test_diagnostics_invariants_and_energies(device, stepper, kw):
    wl = workloads.drifting_cloud(n=6000, nx=32, ny=32, seed=41)
    sim, st, ocfg = run_both(wl, device, 12, stepper=stepper, diag=1, **kw)
    d = sim.residuals()
    assert d["step"] == 12
    # time consistency (section 3): gauge and continuity at roundoff for every stepper
    assert d["gauge_rms"] <= 1e-11 * d["div_a_rms"], d
    assert d["continuity_rms"] <= 1e-11 * d["rho_rms"] / wl.dt, d
    if stepper == "dirk":
        assert d["gauge_dt_rms"] <= 1e-11 * d["rho_rms"], d
        assert d["gauss_rms"] > 1e-9 * d["rho_rms"]        # not a theorem for DIRK
    elif stepper == "cdf2_semi":
        # Gauss as the implicit form defines it is not a theorem for the semi-implicit form
        assert d["gauss_rms"] > 1e-9 * d["rho_rms"]
    else:
        assert d["gauss_rms"] <= 1e-11 * d["rho_rms"], d
    e = opic.energies(ocfg, st)
    assert abs(d["w_b"] - e["wb"]) <= 1e-10 * e["wb"]
    assert abs(d["w_e"] - e["we"]) <= 1e-10 * e["we"]
    assert abs(d["kinetic"] - e["ke"]) <= 1e-9 * e["ke"]
    # E of the last diagnosed step is readable and matches the oracle's
    assert rel(sim.field("ex"), st.grids["ex"]) < TOL
    assert rel(sim.field("ey"), st.grids["ey"]) < TOL
    on = opic.residual_norms(ocfg, st)
    assert on["gauge"][1] <= 1e-11 * d["div_a_rms"]
    sim.close()


def test_parity_full_size_weibel_128(device):
    # The 128x128, 64 particles per cell (1,048,576) cubic BDF-2 workload, in the
    # launch configuration the bench times; two steps checked everywhere.
    wl = workloads.weibel_128(stepper="bdf", bdf_order=2)
    sim, st, _ = run_both(wl, device, 2, stepper="bdf", bdf_order=2)
    compare(sim, st, wl, fields=("jx", "jy", "rho", "phi", "ax", "ay", "dphidx", "daydx"))
    sim.close()


def test_initial_fields_match_oracle(device):
    wl = workloads.drifting_cloud(n=4000, nx=32, ny=16, seed=51)
    cfg = pic.make_config(32, 16, wl.lx, wl.ly, wl.dt, p=2, stepper="cdf2", weight=wl.weight)
    sim = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    st = opic.initial_state(opic.Config(nx=32, ny=16, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=2,
                                        stepper="cdf2", w=wl.weight), wl.x, wl.y, wl.vx, wl.vy)
    assert rel(sim.field("rho"), st.grids["rho"]) < TOL
    assert rel(sim.field("phi"), st.grids["phi"]) < TOL
    got = sim.particles()
    assert rel(got["vx_old"], st.vx_old) < TOL and rel(got["px"], st.px) < TOL
    with pytest.raises(pic.PicError) as e:
        sim.field("jx")                # no step yet
    assert e.value.status == 7
    sim.close()


def test_empty_particle_set(device):
    x = np.zeros(0)
    cfg = pic.make_config(16, 16, 1.0, 1.0, 0.01, p=3, stepper="bdf", bdf_order=2, weight=1.0)
    sim = pic.Simulation(cfg, x, x, x, x, stream=device)
    sim.set_diagnostics(1)
    sim.step(3)
    for f in ("jx", "phi", "ax", "dphidx"):
        assert np.max(np.abs(sim.field(f))) == 0.0
    d = sim.residuals()
    assert d["gauge_rms"] == 0.0 and d["kinetic"] == 0.0
    sim.close()


def test_boundary_positions_and_single_particles(device):
    # Particles exactly at 0, just below L and exactly at L (wrapped to 0 by init).
    L = 1.0
    x = np.array([0.0, np.nextafter(L, 0.0), L, 0.5, 0.999999])
    y = np.array([np.nextafter(L, 0.0), 0.0, 0.25, L, 1e-300])
    vx = np.array([-0.3, 0.3, 0.0, 0.1, 0.2])
    vy = np.array([0.3, -0.3, 0.0, -0.1, 0.0])
    wl = workloads.Workload("edge", 16, 16, L, L, 0.5 / 16, 3, "bdf", 2, 5, x, y, vx, vy)
    sim, st, _ = run_both(wl, device, 5, stepper="bdf", bdf_order=2, p=3)
    compare(sim, st, wl, fields=("jx", "jy", "rho", "phi", "ax"))
    sim.close()


def test_superluminal_input_is_reported(device):
    x = np.array([0.1, 0.2])
    cfg = pic.make_config(16, 16, 1.0, 1.0, 0.01, p=2)
    with pytest.raises(pic.PicError) as e:
        pic.Simulation(cfg, x, x, np.array([0.5, 1.5]), np.zeros(2), stream=device)
    assert e.value.status == 4


def test_thin_grids_max_line_length(device):
    # 1024-point lines along x and along y (largest supported transform).
    for nx, ny in ((1024, 8), (8, 1024)):
        wl = workloads.weibel(nx, ny, 1, 0.5, 0.01, 61, 2, n=3003)
        sim, st, _ = run_both(wl, device, 3, stepper="bdf", bdf_order=1, p=2)
        compare(sim, st, wl, fields=("jx", "jy", "phi", "ax", "daydx"))
        sim.close()


def test_device_pointers_accepted(device):
    import torch
    wl = workloads.drifting_cloud(n=1000, nx=16, ny=16, seed=71)
    cfg = pic.make_config(16, 16, wl.lx, wl.ly, wl.dt, p=2, weight=wl.weight)
    t = {k: torch.from_numpy(getattr(wl, k).copy()).cuda() for k in ("x", "y", "vx", "vy")}
    sim = pic.Simulation(cfg, t["x"], t["y"], t["vx"], t["vy"], stream=device)
    sim.step(2)
    out = {k: torch.empty(wl.n, dtype=torch.float64, device="cuda") for k in
           ("x", "y", "px", "py", "vx", "vy", "vx_old", "vy_old")}
    sim.particles(out)
    host = sim.particles()
    assert np.array_equal(out["px"].cpu().numpy(), host["px"])
    jx = torch.empty((16, 16), dtype=torch.float64, device="cuda")
    sim.field("jx", jx)
    assert np.array_equal(jx.cpu().numpy(), sim.field("jx"))
    sim.close()


SORT_CASES = [
    # name, workload, nsteps, sort interval, stepper kwargs
    ("cloud32_sort1_bdf1", lambda: workloads.drifting_cloud(n=16384, nx=32, ny=32), 8, 1,
     dict(stepper="bdf", bdf_order=1)),
    ("weibel96x64_sort4_bdf2_p3", lambda: workloads.weibel(96, 64, 4, 0.5, 0.01, 27, 3, n=24571),
     9, 4, dict(stepper="bdf", bdf_order=2)),
    ("weibel16_sort3_dirk2_p4", lambda: workloads.weibel(16, 16, 8, 0.6, 0.02, 28, 4, n=2047), 7, 3,
     dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG)),
    # sort interval far beyond the halo: particles leave their tile region (global fallback)
    ("weibel8x12_sort40_cdf2", lambda: workloads.weibel(8, 12, 6, 0.9, 0.05, 29, 2, n=577), 45,
     40, dict(stepper="cdf2")),
    # 0.36 cells per step for 100 steps overruns the 24-cell halo: global fallback path
    ("weibel128_sort100_beyond_halo", lambda: workloads.weibel(128, 128, 1, 0.9, 0.05, 30, 2,
                                                              n=2003), 105, 100,
     dict(stepper="bdf", bdf_order=1)),
]


@pytest.mark.parametrize("name,make,nsteps,sort,kw", SORT_CASES, ids=[c[0] for c in SORT_CASES])
def test_parity_with_tile_sort(device, name, make, nsteps, sort, kw):
    wl = make()
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                          sort_interval=sort, **kw)
    sim = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    sim.step(nsteps)
    ocfg = opic.Config(nx=wl.nx, ny=wl.ny, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=wl.p, w=wl.weight, **kw)
    st = opic.run(ocfg, wl.x, wl.y, wl.vx, wl.vy, nsteps)
    compare(sim, st, wl, fields=("jx", "jy", "rho", "phi", "ax", "ay", "dphidx", "daydy"))
    sim.close()


@pytest.mark.parametrize("kw", [dict(stepper="bdf", bdf_order=2),
                                dict(stepper="bdf", bdf_order=1, charge=pic.CHARGE_DEPOSIT),
                                dict(stepper="cdf2", vdim=3)],
                         ids=["bdf2", "bdf1-naive-charge", "cdf2-3v"])
def test_fp64_deposit_is_deterministic(device, kw):
    # The FP64 path sums every deposit (current, J_z, the charge at t = 0 and the naive
    # charge) as 128-bit integers, so the order of the additions cannot change a bit: two
    # runs of one handle configuration, and a run whose tile sort reorders the particles
    # (and so the order of the atomics) every 3 steps, give identical particles and fields.
    wl = workloads.weibel(48, 32, 12, 0.5, 0.01, 33, 3)
    extra = {}
    if kw.get("vdim") == 3:
        extra["vz"] = np.random.default_rng(5).uniform(-0.2, 0.2, wl.n)
    runs = []
    for sort in ((0, 0) if kw.get("vdim") == 3 else (0, 0, 3)):  # 2D-3V runs unsorted
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                              sort_interval=sort, **kw)
        with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device, **extra) as sim:
            sim.step(11)
            f = ("jx", "jy", "rho", "phi", "ax", "ay", "dphidx", "daydy") + \
                (("jz", "az") if kw.get("vdim") == 3 else ())
            runs.append((sim.particles(), {k: sim.field(k) for k in f}))
    for parts, fields in runs[1:]:
        for k, v in runs[0][0].items():
            assert np.array_equal(parts[k], v), k
        for k, v in runs[0][1].items():
            assert np.array_equal(fields[k], v), k


def test_tile_sort_full_size_weibel_128(device):
    wl = workloads.weibel_128(stepper="bdf", bdf_order=2)
    cfg = pic.make_config(128, 128, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf", bdf_order=2,
                          weight=wl.weight, sort_interval=8)
    sim = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device)
    sim.step(2)
    st = opic.run(opic.Config(nx=128, ny=128, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=3, stepper="bdf",
                              bdf_order=2, w=wl.weight), wl.x, wl.y, wl.vx, wl.vy, 2)
    compare(sim, st, wl, fields=("jx", "jy", "phi", "ax", "dphidx"))
    sim.close()


def test_naive_charge_breaks_the_gauge_as_section_5_reports(device):
    # with the deposited charge, the gauge and continuity residuals leave roundoff; with
    # the conserving update they stay there (same workload, same steps)
    wl = workloads.weibel(32, 32, 8, 0.5, 0.01, 32, 2, n=8191)
    out = {}
    for charge in (pic.CHARGE_CONTINUITY, pic.CHARGE_DEPOSIT):
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper="bdf",
                              bdf_order=2, weight=wl.weight, charge=charge)
        with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
            sim.set_diagnostics(1)
            sim.step(20)
            out[charge] = sim.residuals()
    good, naive = out[pic.CHARGE_CONTINUITY], out[pic.CHARGE_DEPOSIT]
    assert good["gauge_rms"] <= 1e-11 * good["div_a_rms"]
    assert naive["gauge_rms"] > 1e-6 * naive["div_a_rms"], naive
    assert naive["continuity_rms"] > 1e-6 * naive["rho_rms"] / wl.dt, naive

