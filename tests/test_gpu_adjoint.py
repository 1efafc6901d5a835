"""GPU checks of the discrete adjoint (pic_adjoint_*) of the FP64 run and the FP32 form.

- Against the oracle's adjoint (oracle.adjoint, pinned on CPU by finite differences
  and transpose identities): small grids, several spline orders and BDF orders, both
  seeds (the magnetic energy W_B and a final-momentum objective), checkpoint intervals
  that leave a ragged last segment.  Measured on GB300: <= 2e-14 relative; bound 1e-11.
  The same for the three CDF-2 forms and DIRK (Qin-Zhang 2-stage, implicit-midpoint
  3-stage), in both record modes, with the fused column pass and the separate mode
  kernel (a grid whose x extent is too large for the column pass's shared memory).
- Checkpoint-interval invariance: K = 1, 3, N give the same gradient (to the roundoff of
  the reverse pass's FP64 field-adjoint atomics, which sum in no fixed order).
- The 128 x 128 Weibel configuration (262,144 particles, v_d = 0.5c, BDF-2, cubic, 200
  steps): the gradient of W_B against central finite differences of the forward run with
  h = 1e-6 along v_d (through u_d = gamma_d v_d) and along 4 random directions in v^0;
  bound 1e-6 relative (measured <= 1.5e-7).  Along 32 random single components of P^0
  the forward's own roundoff limits the finite difference: W_B carries FP64 roundoff
  amplified by 200 steps of the unstable dynamics (identical runs are bit-identical, the
  deposit summing integers, but a perturbed input reshuffles the roundoff of every later
  transform and push), while one particle's derivative is only ~1e-10 against
  W_B = 5.8e-7.  The finite difference then carries an error of about sigma W_B / h;
  measured sigma <= 1.9e-13 at h = 1e-6 and <= 1.3e-12 at h = 1e-4 (truncation
  included).  There h = 1e-4 and the bound is 1e-6 |g| + sigma W_B / h with
  sigma = 4e-12 (about 1e-4 of a typical component).
- The handle is left at the end of the forward run; torch.autograd returns the same
  gradient as the library call.
- The FP32 form's adjoint (unsorted handles) against the oracle's FP64 gradient, for
  BDF-1/2, CDF-2 and DIRK-2, both seeds and both record modes: measured <= 1.4e-6
  relative on GB300, bound 1e-5; its two record modes agree to 1e-6.  On the 128 x 128
  Weibel run (200 steps) against the FP64 adjoint: 1.7e-5 over the whole gradient and
  1.0e-6 along the drift (bounds 2e-4 and 1e-5), the difference of the two trajectories;
  and against central differences of the FP32 run itself (h = 1e-3, the truncation
  error removed by the same difference of the FP64 run, allowance 4e-6 W_B / h for the
  FP32 run's noise floor).
"""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import pic as opic
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _case(p, k, nx, ny, n, seed, stepper="bdf", dirk=None, cdf_form="implicit",
          precision=None):
    rng = np.random.default_rng(seed)
    lx, ly = 1.0, 0.8
    x = rng.uniform(0, lx, n)
    y = rng.uniform(0, ly, n)
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    vx = 0.05 * rng.standard_normal(n)
    vy = sgn * 0.3 + 0.05 * rng.standard_normal(n)
    dt = 0.4 * lx / nx
    w = lx * ly / n
    name = stepper if cdf_form == "implicit" else f"cdf2_{cdf_form}"
    cfg = pic.make_config(nx, ny, lx, ly, dt, p=p, stepper=name, bdf_order=k, dirk=dirk,
                          weight=w, precision=pic.FP64 if precision is None else precision)
    ocfg = opic.Config(nx=nx, ny=ny, lx=lx, ly=ly, dt=dt, p=p, stepper=stepper, bdf_order=k,
                       w=w, dirk=dirk, cdf_form=cdf_form)
    return cfg, ocfg, x, y, vx, vy


def _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K, pb=None, mode="replay"):
    import torch
    area = cfg.lx / cfg.nx * cfg.ly / cfg.ny
    with pic.Simulation(cfg, x, y, vx, vy, stream=device) as sim:
        with pic.Adjoint(sim, nsteps, K, mode=mode) as adj:
            adj.forward()
            bz = torch.empty((cfg.nx, cfg.ny), dtype=torch.float64, device="cuda")
            sim.field("bz", out=bz)
            wb = 0.5 * area * float((bz * bz).sum())
            if pb is None:
                g = adj.backward(bz_bar=(bz * area).contiguous())
            else:
                g = adj.backward(px_bar=torch.tensor(pb[0], device="cuda"),
                                 py_bar=torch.tensor(pb[1], device="cuda"))
            return wb, {key: v.cpu().numpy() for key, v in g.items()}


CASES = [(2, 1, 24, 16, 3000, 13, 5), (3, 2, 32, 32, 4096, 13, 5), (4, 3, 16, 24, 2000, 9, 4)]


@pytest.mark.parametrize("p,k,nx,ny,n,nsteps,K", CASES, ids=["p2-bdf1", "p3-bdf2", "p4-bdf3"])
def test_adjoint_matches_oracle(device, p, k, nx, ny, n, nsteps, K):
    cfg, ocfg, x, y, vx, vy = _case(p, k, nx, ny, n, seed=p)
    tape = oadj.record(ocfg, x, y, vx, vy, nsteps)
    expect = oadj.gradient(tape)
    wb, got = _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K,
                            mode="recompute" if p == 4 else "replay")
    assert abs(wb / oadj.magnetic_energy(ocfg, tape.final) - 1.0) <= 1e-12
    errs = {"vx": rel(got["vx"], expect["v0"][0]), "vy": rel(got["vy"], expect["v0"][1]),
            "px": rel(got["px"], expect["p0"][0]), "py": rel(got["py"], expect["p0"][1])}
    assert max(errs.values()) <= 1e-11, errs
    # final-momentum objective
    rng = np.random.default_rng(20 + p)
    pb = (rng.standard_normal(n), rng.standard_normal(n))
    expect = oadj.gradient(tape, px_bar=pb[0], py_bar=pb[1])
    _, got = _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K, pb=pb)
    errs = {"vx": rel(got["vx"], expect["v0"][0]), "vy": rel(got["vy"], expect["v0"][1]),
            "px": rel(got["px"], expect["p0"][0]), "py": rel(got["py"], expect["p0"][1])}
    assert max(errs.values()) <= 1e-11, errs


OTHER = [
    ("cdf2-implicit", dict(stepper="cdf2"), 3, 32, 24, 3000, 9, 4, "replay"),
    ("cdf2-semi", dict(stepper="cdf2", cdf_form="semi"), 2, 24, 16, 2000, 9, 4, "recompute"),
    # explicit form: c dt |k|_max = 1.7 < 2, inside its stability limit
    ("cdf2-explicit", dict(stepper="cdf2", cdf_form="explicit"), 4, 16, 12, 2000, 8, 3, "replay"),
    ("dirk2", dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG), 3, 32, 32, 3000, 9, 4, "replay"),
    ("dirk3", dict(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT), 2, 24, 24, 2000, 8, 3,
     "recompute"),
    # nx = 1024 exceeds the column pass's shared memory (17 nx complex values): the
    # separate mode kernel runs
    ("cdf2-wide", dict(stepper="cdf2"), 2, 1024, 8, 3000, 4, 2, "replay"),
    ("dirk2-wide", dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG), 2, 1024, 8, 3000, 4, 2,
     "replay"),
]


@pytest.mark.parametrize("name,kw,p,nx,ny,n,nsteps,K,mode", OTHER, ids=[c[0] for c in OTHER])
def test_cdf2_and_dirk_adjoint_match_oracle(device, name, kw, p, nx, ny, n, nsteps, K, mode):
    cfg, ocfg, x, y, vx, vy = _case(p, 1, nx, ny, n, seed=len(name), **kw)
    tape = oadj.record(ocfg, x, y, vx, vy, nsteps)
    expect = oadj.gradient(tape)
    wb, got = _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K, mode=mode)
    assert abs(wb / oadj.magnetic_energy(ocfg, tape.final) - 1.0) <= 1e-12
    errs = {"vx": rel(got["vx"], expect["v0"][0]), "vy": rel(got["vy"], expect["v0"][1]),
            "px": rel(got["px"], expect["p0"][0]), "py": rel(got["py"], expect["p0"][1])}
    assert max(errs.values()) <= 1e-11, errs
    rng = np.random.default_rng(31)
    pb = (rng.standard_normal(n), rng.standard_normal(n))
    expect = oadj.gradient(tape, px_bar=pb[0], py_bar=pb[1])
    _, got = _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K, pb=pb, mode=mode)
    errs = {"vx": rel(got["vx"], expect["v0"][0]), "vy": rel(got["vy"], expect["v0"][1])}
    assert max(errs.values()) <= 1e-11, errs


@pytest.mark.parametrize("mode", ["replay", "recompute"])
def test_checkpoint_interval_invariance(device, mode):
    # the replay mode rebuilds the particle states between checkpoints from the recorded
    # gathered fields (bit for bit the forward's); the recompute mode re-runs the steps
    cfg, _, x, y, vx, vy = _case(3, 2, 32, 32, 4096, seed=3)
    ref = _gpu_gradient(device, cfg, x, y, vx, vy, 13, 5)[1]
    for K in (1, 3, 13, 100):
        got = _gpu_gradient(device, cfg, x, y, vx, vy, 13, K, mode=mode)[1]
        for key in ref:
            assert rel(got[key], ref[key]) <= 1e-12, (mode, K, key)


@pytest.mark.parametrize("kw,mode", [(dict(), "replay"), (dict(stepper="cdf2"), "recompute"),
                                     (dict(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT), "replay")],
                         ids=["bdf2", "cdf2", "dirk3"])
def test_handle_left_at_end_of_forward_run(device, kw, mode):
    # CDF-2 swaps its level pairs every step and the checkpoints hold them by role: after
    # an odd number of steps the buffers in each role differ from those at step 0
    import torch
    cfg, _, x, y, vx, vy = _case(3, 2, 32, 32, 4096, seed=4, **kw)
    with pic.Simulation(cfg, x, y, vx, vy, stream=device) as sim:
        with pic.Adjoint(sim, 9, 3, mode=mode) as adj:
            adj.forward()
            before = sim.particles()
            fields = {f: sim.field(f) for f in ("bz", "jx", "phi", "ay", "dphidx")}
            bz = torch.tensor(fields["bz"], device="cuda")
            adj.backward(bz_bar=bz)
            after = sim.particles()
            assert sim.step_count == 9
            for key in before:
                assert np.array_equal(before[key], after[key]), key
            for f, v in fields.items():
                assert np.array_equal(sim.field(f), v), f
            sim.step(2)  # the handle steps on from there


def test_adjoint_rejects_unsupported_handles(device):
    cfg, _, x, y, vx, vy = _case(3, 2, 32, 32, 512, seed=5)
    for kw in (dict(precision=pic.FP32_FIX64, sort_interval=4), dict(sort_interval=4),
               dict(charge=pic.CHARGE_DEPOSIT)):
        args = dict(p=3, stepper="bdf", bdf_order=2, weight=cfg.weight)
        args.update(kw)
        c = pic.make_config(cfg.nx, cfg.ny, cfg.lx, cfg.ly, cfg.dt, **args)
        with pic.Simulation(c, x, y, vx, vy, stream=device) as sim:
            with pytest.raises(pic.PicError) as e:
                pic.Adjoint(sim, 5)
            assert e.value.status == 2
    with pic.Simulation(cfg, x, y, vx, vy, stream=device) as sim:
        sim.step(1)
        with pytest.raises(pic.PicError) as e:
            pic.Adjoint(sim, 5)
        assert e.value.status == 7


# The FP32 form's adjoint (the step's adjoint in exact arithmetic along the FP32 trajectory,
# particle adjoints in FP32, field adjoints and the reverse field solve in FP64) against the
# oracle's FP64 gradient: the difference is the FP32 trajectory's own departure from the
# FP64 one plus FP32 rounding in the reverse particle arithmetic.
FP32_CASES = [
    ("p2-bdf1", dict(p=2, k=1, nx=24, ny=16, n=3000, seed=2), {}, 6, 3, "replay"),
    ("p3-bdf2", dict(p=3, k=2, nx=32, ny=32, n=4096, seed=3), {}, 6, 4, "recompute"),
    ("p3-cdf2", dict(p=3, k=1, nx=32, ny=24, n=4096, seed=4), dict(stepper="cdf2"), 5, 5,
     "replay"),
    ("p4-dirk2", dict(p=4, k=1, nx=16, ny=24, n=2000, seed=5),
     dict(stepper="dirk", dirk=osteps.DIRK2_QIN_ZHANG), 4, 2, "replay"),
]
FP32_GRAD_TOL = 1e-5


@pytest.mark.parametrize("name,case,kw,nsteps,K,mode", FP32_CASES,
                         ids=[c[0] for c in FP32_CASES])
def test_fp32_form_adjoint_matches_oracle(device, name, case, kw, nsteps, K, mode):
    cfg, ocfg, x, y, vx, vy = _case(**case, **kw, precision=pic.FP32_FIX64)
    tape = oadj.record(ocfg, x, y, vx, vy, nsteps)
    expect = oadj.gradient(tape)
    wb, got = _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K, mode=mode)
    ewb = oadj.magnetic_energy(ocfg, tape.final)
    print(f"{name}: W_B {wb / ewb - 1:.2e}", end="")
    assert abs(wb / ewb - 1.0) <= 1e-5
    # W_B and a final-momentum objective
    rng = np.random.default_rng(30 + case["p"])
    pb = (rng.standard_normal(case["n"]), rng.standard_normal(case["n"]))
    for obj in ("wb", "p"):
        if obj == "p":
            expect = oadj.gradient(tape, px_bar=pb[0], py_bar=pb[1])
            _, got = _gpu_gradient(device, cfg, x, y, vx, vy, nsteps, K, pb=pb, mode=mode)
        for key, ref in (("vx", expect["v0"][0]), ("vy", expect["v0"][1]),
                         ("px", expect["p0"][0]), ("py", expect["p0"][1])):
            r = rel(got[key], ref)
            print(f"  {obj}:{key} {r:.2e}", end="")
            assert r <= FP32_GRAD_TOL, (obj, key, r)
    print()


@pytest.mark.parametrize("p,k,precision", [(2, 1, pic.FP64), (3, 2, pic.FP64), (4, 3, pic.FP64),
                                           (3, 2, pic.FP32_FIX64)],
                         ids=["p2-fp64", "p3-fp64", "p4-fp64", "p3-fp32"])
def test_lean_replay_gives_the_replay_gradient(device, p, k, precision):
    # The lean records keep P and v only; the reverse push gathers A and grad A again from
    # the recorded fields with the forward gather's own operations, so the gradient is the
    # replay mode's up to the order of the field-adjoint atomics; FP64 also against the
    # oracle at the parity bound.
    cfg, ocfg, x, y, vx, vy = _case(p, k, 32, 24, 3001, seed=40 + p, precision=precision)
    _, full = _gpu_gradient(device, cfg, x, y, vx, vy, 7, 3, mode="replay")
    _, lean = _gpu_gradient(device, cfg, x, y, vx, vy, 7, 3, mode="replay_lean")
    tol = 1e-13 if precision == pic.FP64 else 1e-6
    for key in full:
        assert rel(lean[key], full[key]) <= tol, (key, rel(lean[key], full[key]))
    if precision == pic.FP64:
        expect = oadj.gradient(oadj.record(ocfg, x, y, vx, vy, 7))
        assert rel(lean["vx"], expect["v0"][0]) <= 1e-11
        assert rel(lean["py"], expect["p0"][1]) <= 1e-11


def test_fp32_form_adjoint_modes_agree(device):
    # replay (recorded P, v and gathered fields) and recompute (the segment's FP32 steps
    # re-run; the fixed-point current is bit-exact) reverse the same trajectory: they differ
    # only by the order of the FP64 field-adjoint atomics
    cfg, _, x, y, vx, vy = _case(3, 2, 32, 32, 4096, seed=7, precision=pic.FP32_FIX64)
    _, a = _gpu_gradient(device, cfg, x, y, vx, vy, 9, 4, mode="replay")
    _, b = _gpu_gradient(device, cfg, x, y, vx, vy, 9, 4, mode="recompute")
    _, c = _gpu_gradient(device, cfg, x, y, vx, vy, 9, 9, mode="replay")
    for key in a:
        assert rel(a[key], b[key]) <= 1e-6, key
        assert rel(a[key], c[key]) <= 1e-6, key


@pytest.mark.parametrize("precision,mode,tol", [(pic.FP64, "replay", 1e-12),
                                                (pic.FP64, "replay_lean", 1e-12),
                                                (pic.FP32_FIX64, "replay", 1e-6)],
                         ids=["fp64", "fp64-lean", "fp32"])
def test_autograd_matches_library(device, precision, mode, tol):
    import torch
    from paper_2410_18414_gb300 import autograd
    cfg, _, x, y, vx, vy = _case(3, 2, 32, 32, 4096, seed=6, precision=precision)
    vx0 = torch.tensor(vx, device="cuda", requires_grad=True)
    vy0 = torch.tensor(vy, device="cuda", requires_grad=True)
    wb = autograd.magnetic_energy(cfg, x, y, vx0, vy0, 12, checkpoint_every=5, mode=mode)
    (2.5 * wb).backward()
    _, ref = _gpu_gradient(device, cfg, x, y, vx, vy, 12, 12)
    assert rel(vx0.grad.cpu().numpy(), 2.5 * ref["vx"]) <= tol
    assert rel(vy0.grad.cpu().numpy(), 2.5 * ref["vy"]) <= tol


# ------------------------------------------------------------ 128 x 128 Weibel --

@pytest.fixture(scope="module")
def c5(device):
    wl = workloads.weibel_adjoint_128()
    assert (wl.nx, wl.ny, wl.n, wl.p, wl.nsteps) == (128, 128, 262144, 3, 200)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper="bdf",
                          bdf_order=2, weight=wl.weight)
    wb, g = _gpu_gradient(device, cfg, wl.x, wl.y, wl.vx, wl.vy, wl.nsteps, 20)
    return wl, cfg, wb, g


def _wb(device, wl, cfg, vx, vy):
    with pic.Simulation(cfg, wl.x, wl.y, vx, vy, stream=device) as sim:
        sim.step(wl.nsteps)
        bz = sim.field("bz")
    return 0.5 * (wl.lx / wl.nx) * (wl.ly / wl.ny) * float(np.sum(bz * bz))


def _v_of_vd(wl, vd):
    # the workload's draws (weibel(): x, y, then u_x, then the u_y spread), with the drift
    rng = np.random.Generator(np.random.PCG64(5))
    rng.uniform(0.0, wl.lx, wl.n)
    rng.uniform(0.0, wl.ly, wl.n)
    ux = 0.01 * rng.standard_normal(wl.n)
    uy = np.where(np.arange(wl.n) % 2 == 0, 1.0, -1.0) * (vd / np.sqrt(1 - vd * vd)) \
        + 0.01 * rng.standard_normal(wl.n)
    gam = np.sqrt(1.0 + ux * ux + uy * uy)
    return ux / gam, uy / gam


def test_c5_drift_gradient_matches_finite_differences(device, c5):
    wl, cfg, wb, g = c5
    vx, vy = _v_of_vd(wl, 0.5)
    assert np.array_equal(vx, wl.vx) and np.array_equal(vy, wl.vy)
    # P^0_y = m u_y, u_y = +-u_d + spread, du_d/dv_d = gamma_d^3 (m = 1)
    sgn = np.where(np.arange(wl.n) % 2 == 0, 1.0, -1.0)
    adj = (1.0 / np.sqrt(0.75)) ** 3 * float(np.sum(sgn * g["py"]))
    h = 1e-6
    fd = (_wb(device, wl, cfg, *_v_of_vd(wl, 0.5 + h))
          - _wb(device, wl, cfg, *_v_of_vd(wl, 0.5 - h))) / (2 * h)
    assert abs(fd - adj) <= 1e-6 * abs(adj), (fd, adj)


def test_c5_direction_gradients_match_finite_differences(device, c5):
    wl, cfg, wb, g = c5
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal((2, wl.n))
        ad = float(np.dot(g["vx"], d[0]) + np.dot(g["vy"], d[1]))
        fd = (_wb(device, wl, cfg, wl.vx + h * d[0], wl.vy + h * d[1])
              - _wb(device, wl, cfg, wl.vx - h * d[0], wl.vy - h * d[1])) / (2 * h)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.fixture(scope="module")
def c5_32(device, c5):
    wl = c5[0]
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper="bdf",
                          bdf_order=2, weight=wl.weight, precision=pic.FP32_FIX64)
    wb32, g32 = _gpu_gradient(device, cfg, wl.x, wl.y, wl.vx, wl.vy, wl.nsteps, 20)
    return cfg, wb32, g32


def test_c5_fp32_form_adjoint_matches_fp64(device, c5, c5_32):
    # the FP32 form's adjoint of the same 200-step run against the FP64 adjoint: the whole
    # gradient and its projection on the drift direction
    wl, _, wb, g = c5
    _, wb32, g32 = c5_32
    sgn = np.where(np.arange(wl.n) % 2 == 0, 1.0, -1.0)
    d64, d32 = float(np.sum(sgn * g["py"])), float(np.sum(sgn * g32["py"]))
    r = {key: rel(g32[key], g[key]) for key in g}
    print(f"W_B {wb32 / wb - 1:.2e} drift {d32 / d64 - 1:.2e} " +
          " ".join(f"{k} {v:.2e}" for k, v in r.items()))
    assert abs(wb32 / wb - 1.0) <= 1e-5
    assert abs(d32 / d64 - 1.0) <= 1e-5
    for key, v in r.items():
        assert v <= 2e-4, (key, v)


def test_c5_fp32_form_finite_differences(device, c5, c5_32):
    # Central differences of the FP32 form's own forward run against its adjoint.  The FP32
    # run's W_B carries a noise floor sigma relative (FP32 roundoff through 200 steps of the
    # instability; from the spread of central differences over h = 1e-6 .. 1e-3: 1e-7 to
    # 3e-7 along the drift, about 1e-6 along a random direction, which moves every
    # particle's roundoff), so h is 1e-3, and the truncation error of that h is taken out by
    # the same difference of the FP64 run: (fd32 - fd64) must match (adj32 - adj64) within
    # the noise allowance 4e-6 W_B / h (2.3e-9; measured 1.3e-10 along the drift and
    # 5.7e-10 along the direction).
    wl, cfg64, wb, g = c5
    cfg32, wb32, g32 = c5_32
    h = 1e-3
    sgn = np.where(np.arange(wl.n) % 2 == 0, 1.0, -1.0)
    gd = (1.0 / np.sqrt(0.75)) ** 3
    d = np.random.default_rng(13).standard_normal((2, wl.n))
    probes = [
        (lambda s: _v_of_vd(wl, 0.5 + s * h), lambda gr: gd * float(np.sum(sgn * gr["py"]))),
        (lambda s: (wl.vx + s * h * d[0], wl.vy + s * h * d[1]),
         lambda gr: float(np.dot(gr["vx"], d[0]) + np.dot(gr["vy"], d[1]))),
    ]
    for v_at, proj in probes:
        fd = {}
        for name, cfg in (("32", cfg32), ("64", cfg64)):
            fd[name] = (_wb(device, wl, cfg, *v_at(1.0)) - _wb(device, wl, cfg, *v_at(-1.0))) / (2 * h)
        a32, a64 = proj(g32), proj(g)
        err = abs((fd["32"] - fd["64"]) - (a32 - a64))
        print(f"fd32 {fd['32']:.8e} adj32 {a32:.8e} fd64 {fd['64']:.8e} adj64 {a64:.8e} "
              f"residual {err:.2e} (sigma {err * h / wb32:.1e})")
        assert err <= 4e-6 * wb32 / h, (fd, a32, a64)


def test_c5_momentum_components_match_finite_differences(device, c5):
    wl, cfg, wb, g = c5
    gam = 1.0 / np.sqrt(1.0 - (wl.vx ** 2 + wl.vy ** 2))
    px0, py0 = gam * wl.vx, gam * wl.vy
    rng = np.random.default_rng(12)
    h, sigma = 1e-4, 4e-12
    for i in rng.choice(wl.n, 32, replace=False):
        comp = int(rng.integers(2))
        vals = []
        for s in (1.0, -1.0):
            p = [px0.copy(), py0.copy()]
            p[comp][i] += s * h
            den = np.sqrt(p[0] ** 2 + p[1] ** 2 + 1.0)
            vals.append(_wb(device, wl, cfg, p[0] / den, p[1] / den))
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = g["px" if comp == 0 else "py"][i]
        assert abs(fd - ad) <= 1e-6 * abs(ad) + sigma * wb / h, (i, comp, fd, ad)
