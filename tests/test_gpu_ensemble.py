"""GPU checks of ensembles (pic_ensemble_*): independent runs captured into one CUDA
graph and advanced by replaying it must give the results of pic_step on each run, bit for
bit in both forms, whose currents are integer sums; at the benchmarked size (256 runs,
7.0e7 particles) on sampled runs."""
import numpy as np
import pytest

from oracle import steppers as osteps
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# (workload, precision, sort interval, stepper kwargs)
RUNS = [
    (lambda: workloads.weibel(32, 32, 16, 0.4, 0.01, 1001, 3), pic.FP32_FIX64, 8,
     dict(stepper="bdf", bdf_order=2)),
    (lambda: workloads.weibel(48, 32, 24, 0.6, 0.01, 1002, 3), pic.FP32_FIX64, 4,
     dict(stepper="bdf", bdf_order=2)),
    (lambda: workloads.weibel(64, 64, 16, 0.3, 0.01, 1003, 3), pic.FP32_FIX64, 0,
     dict(stepper="cdf2")),
    (lambda: workloads.weibel(24, 24, 8, 0.5, 0.02, 1004, 4), pic.FP64, 0,
     dict(stepper="bdf", bdf_order=3)),
    (lambda: workloads.weibel(32, 48, 8, 0.5, 0.02, 1005, 2), pic.FP32_FIX64, 2,
     dict(stepper="dirk", dirk=osteps.DIRK3_MIDPOINT)),
]


def make(torch, spec, stream=None):
    make_wl, prec, sort, kw = spec
    wl = make_wl()
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, weight=wl.weight,
                          precision=prec, sort_interval=sort, **kw)
    s = stream if stream is not None else torch.cuda.Stream()
    return pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=s.cuda_stream), s


def assert_same(a, b, prec):
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), (k, prec)
    for f in ("jx", "phi", "ay", "daxdy"):
        assert np.array_equal(a.field(f), b.field(f)), (f, prec)


def test_ensemble_matches_runs_stepped_alone(torch_mod):
    torch = torch_mod
    runs = [make(torch, spec) for spec in RUNS]
    solo = [make(torch, spec) for spec in RUNS]
    master = torch.cuda.Stream()
    with pic.Ensemble([r for r, _ in runs], master.cuda_stream) as ens:
        P = ens.period
        # lcm(2, BDF-2 rings 4 and 2, BDF-3 rings 6 and 3, twice the sort intervals 16, 8, 4)
        assert P == 48
        ens.step(2 * P)
        for (r, _), (s, _) in zip(runs, solo):
            s.step(2 * P)
            assert r.step_count == s.step_count == 2 * P
        for (r, _), (s, _), spec in zip(runs, solo, RUNS):
            assert_same(r, s, spec[1])
        # a run may go on alone afterwards; then the graph no longer matches it
        runs[0][0].step(3)
        solo[0][0].step(3)
        assert_same(runs[0][0], solo[0][0], RUNS[0][1])
        with pytest.raises(pic.PicError, match="no longer matches"):
            ens.step(P)
        runs[0][0].step(P - 3)  # back in phase: the graph applies again
        solo[0][0].step(P - 3)
        ens.step(P)
        for (r, _), (s, _) in zip(runs[1:], solo[1:]):
            s.step(P)
        for (r, _), (s, _), spec in zip(runs, solo, RUNS):
            if r is runs[0][0]:
                s.step(P)
            assert_same(r, s, spec[1])
    for r, _ in runs + solo:
        r.close()


def test_ensemble_capture_runs_nothing_and_leaves_runs_unchanged(torch_mod):
    torch = torch_mod
    runs = [make(torch, spec) for spec in RUNS[:2]]
    solo = [make(torch, spec) for spec in RUNS[:2]]
    ens = pic.Ensemble([r for r, _ in runs], torch.cuda.Stream().cuda_stream)
    assert ens.period == 16
    ens.close()  # captured, never launched
    for (r, _), (s, _), spec in zip(runs, solo, RUNS):
        assert r.step_count == 0
        r.step(5)
        s.step(5)
        assert_same(r, s, spec[1])
    for r, _ in runs + solo:
        r.close()


def test_ensemble_rejects_misuse(torch_mod):
    torch = torch_mod
    r0, _ = make(torch, RUNS[0])
    r1, _ = make(torch, RUNS[1])
    master = torch.cuda.Stream().cuda_stream
    with pytest.raises(pic.PicError, match="repeats"):
        pic.Ensemble([r0, r0], master)
    with pytest.raises(pic.PicError, match="stream"):
        pic.Ensemble([r0], 0)
    r1.set_diagnostics(2)
    with pytest.raises(pic.PicError, match="diagnostics"):
        pic.Ensemble([r0, r1], master)
    r1.set_diagnostics(0)
    r1.deposit()
    with pytest.raises(pic.PicError, match="middle of a step"):
        pic.Ensemble([r0, r1], master)
    r1.field_solve()
    r1.gather_push()
    with pic.Ensemble([r0, r1], master) as ens:
        with pytest.raises(pic.PicError, match="multiple"):
            ens.step(ens.period + 1)
        ens.step(0)
    r0.close()
    r1.close()


def test_autotuner_picks_the_fastest_pair_and_caches(torch_mod):
    from paper_2410_18414_gb300 import autotune
    t, s, ms = autotune.tune(32, 20)
    # every tile up to half the grid with every sort interval was probed
    assert set(ms) == {(a, b) for a in (4, 8, 16) for b in (1, 2, 4, 8, 16)}
    assert (t, s) == min(ms, key=ms.get)
    assert autotune.density_class(20) == 16 and autotune.density_class(50) == 64
    assert autotune._cache[(32, 16, 3, pic.FP32_FIX64)] == (t, s)
    assert autotune.tune(32, 18) == (t, s, {})  # same key: from the cache
    assert autotune.candidates(16) == [(a, b) for a in (4, 8) for b in (1, 2, 4, 8, 16)]


def test_tile_width_changes_no_result(torch_mod):
    # the sorted FP32 form sums its current exactly in integers, so the tiling (which
    # regroups the sums) leaves every bit unchanged: tiles 4, 8, 16 and the derived one
    torch = torch_mod
    wl = workloads.weibel(64, 48, 24, 0.5, 0.01, 1021, 3)
    out = []
    for tile in (0, 4, 8, 16):
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf",
                              bdf_order=2, weight=wl.weight, precision=pic.FP32_FIX64,
                              sort_interval=4, tile=tile)
        with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy,
                            stream=torch.cuda.Stream().cuda_stream) as sim:
            sim.step(13)
            out.append((sim.particles(), {f: sim.field(f) for f in ("jx", "jy", "phi", "ay")}))
    for parts, fields in out[1:]:
        for k in parts:
            assert np.array_equal(parts[k], out[0][0][k]), k
        for f in fields:
            assert np.array_equal(fields[f], out[0][1][f]), f


def test_ensemble_matches_the_oracle(torch_mod):
    # An FP64 run and an FP32-form run (sorted, with a fused kernel in every step) stepped
    # together by the graph against the CPU oracle: FP64 to 1e-12, the FP32 form within
    # the bounds of its stated error (3e-5 on fields, 2e-6 on particles after 10 steps).
    from oracle import pic as opic
    torch = torch_mod
    specs = [
        (lambda: workloads.weibel(24, 16, 8, 0.5, 0.01, 1011, 3, n=3001), pic.FP64, 0,
         dict(stepper="bdf", bdf_order=2), dict(stepper="bdf", bdf_order=2), 1e-12, 1e-12),
        (lambda: workloads.weibel(32, 24, 8, 0.5, 0.01, 1012, 2, n=6007), pic.FP32_FIX64, 2,
         dict(stepper="cdf2"), dict(stepper="cdf2"), 3e-5, 2e-6),
    ]
    runs = [make(torch, (m, prec, sort, kw)) for m, prec, sort, kw, _, _, _ in specs]
    master = torch.cuda.Stream()
    with pic.Ensemble([r for r, _ in runs], master.cuda_stream) as ens:
        P = ens.period
        nsteps = P * max(1, -(-10 // P))
        ens.step(nsteps)
    for (r, _), (mk, prec, sort, kw, okw, ftol, ptol) in zip(runs, specs):
        wl = mk()
        ocfg = opic.Config(nx=wl.nx, ny=wl.ny, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=wl.p,
                           w=wl.weight, **okw)
        st = opic.run(ocfg, wl.x, wl.y, wl.vx, wl.vy, nsteps)
        got = r.particles()
        for k in ("px", "py", "vx", "vy", "vx_old", "vy_old"):
            assert rel(got[k], getattr(st, k)) < ptol, (k, rel(got[k], getattr(st, k)))
        for k, L in (("x", wl.lx), ("y", wl.ly)):
            d = np.mod(got[k] - getattr(st, k) + 0.5 * L, L) - 0.5 * L
            assert np.linalg.norm(d) / np.linalg.norm(getattr(st, k)) < ptol, k
        for f in ("jx", "jy", "rho", "phi", "ax", "ay", "bz", "daydx"):
            assert rel(r.field(f), st.grids[f]) < ftol, (f, rel(r.field(f), st.grids[f]))
        r.close()


def test_full_size_ensemble_matches_solo_runs(torch_mod):
    # The benchmarked ensemble at its full size: 256 runs drawn as the benchmark draws them
    # (7.0e7 particles), tile widths and sort intervals from the autotuner, one period
    # replayed as one graph launch; seeded sample runs stepped alone must give the same bits.
    from paper_2410_18414_gb300 import autotune
    torch = torch_mod
    specs = workloads.ensemble_specs()
    tuned = [autotune.tune(sp["n"], sp["ppc"])[:2] for sp in specs]

    def make_run(sp, t_s):
        wl = workloads.ensemble_run(sp)
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf",
                              bdf_order=2, weight=wl.weight, precision=pic.FP32_FIX64,
                              sort_interval=t_s[1], tile=t_s[0])
        return pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy,
                              stream=torch.cuda.Stream().cuda_stream)

    runs = [make_run(sp, ts) for sp, ts in zip(specs, tuned)]
    assert sum(r.n for r in runs) > 6e7
    with pic.Ensemble(runs, torch.cuda.Stream().cuda_stream) as ens:
        P = ens.period
        ens.step(P)
    sample = np.random.default_rng(7).choice(len(specs), 4, replace=False)
    for k in sample:
        solo = make_run(specs[k], tuned[k])
        solo.step(P)
        assert_same(runs[k], solo, pic.FP32_FIX64)
        solo.close()
    for r in runs:
        r.close()
