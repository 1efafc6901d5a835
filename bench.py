#!/usr/bin/env python
"""Throughput of the gauge-conserving spectral PIC step on GB300 (particle-steps/s).

Default workload: the 128x128 relativistic Weibel set-up -- 64 macro-electrons per
cell (1,048,576), counter-streaming beams +-0.5c along y, u_th = 0.01c, cubic
B-splines, dt = 0.4 dx, BDF-2 -- run through the C ABI of libgpic (pic_deposit,
pic_field_solve, pic_gather_push).  Inputs are the seeded synthetic initial
conditions of paper_2410_18414_gb300.workloads, resident in HBM before timing.

Timing: W untimed warm-up steps, then exactly K steps, each bracketed by CUDA
events on the library's stream, with a 256 MiB device write between steps
(outside the events) so that every timed step starts with a cold L2.  With more
than one GPU (torchrun), every rank runs an independent replica (its own seed):
weak scaling, no collective on the data path; the timed region is the max over
ranks.  `--impl reference` times the CPU oracle instead (see run_reference).

One JSON line is printed by rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
STEPPER_NAMES = {"bdf1": ("bdf", 1), "bdf2": ("bdf", 2), "cdf2": ("cdf2", 1), "dirk2": ("dirk", 1),
                 "dirk3": ("dirk", 1)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=list(WORKLOADS) + ["ensemble256", "adjoint128"],
                    default="weibel128",
                    help="weibel128: the headline configuration; weibel512: the large one; "
                         "ensemble256: 256 independent runs in one graph launch per period; "
                         "adjoint128: gradient of the final magnetic energy (the adjoint "
                         "of --adjoint-form)")
    ap.add_argument("--adjoint-form", choices=["fp64", "fp32"], default="fp64",
                    help="adjoint128: the FP64 run or the (unsorted) FP32 form")
    ap.add_argument("--repeats", type=int, default=3,
                    help="adjoint128: timed gradient evaluations per checkpoint interval")
    ap.add_argument("--stepper", choices=list(STEPPER_NAMES), default=None,
                    help="default: the workload's own (bdf2 for weibel128, dirk3 for weibel512)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="form timed for the headline value; the other form is timed beside it")
    ap.add_argument("--sort-interval", type=int, default=8,
                    help="re-sort particles by tile every this many steps (0 = never)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-steppers", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint timing that the default line carries")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the ensemble timing that the default line carries")
    a = ap.parse_args()
    if a.stepper is None:
        a.stepper = WORKLOADS[a.workload]["stepper"] if a.workload in WORKLOADS else "bdf2"
    return a


# ----------------------------------------------------------------- workload --

# Workloads: the 128x128 Weibel (2^20 particles, cubic, BDF-2: the headline) and the
# 512x512 one (26,214,400 particles, quartic, 3-stage DIRK).  seed: the seed of rank 0.
WORKLOADS = {
    "weibel128": dict(n=128, ppc=64, v_drift=0.5, u_th=0.01, p=3, seed=2, stepper="bdf2"),
    "weibel512": dict(n=512, ppc=100, v_drift=0.6, u_th=0.02, p=4, seed=3, stepper="dirk3"),
}


class Ranks:
    """The ranks of a torchrun launch (RANK, WORLD_SIZE, LOCAL_RANK): every rank runs an
    independent replica, so the only collectives are the barriers around a timed region
    and the max of its duration over ranks.  With one rank both are local no-ops.
    backend/device: "nccl"/"cuda" on GPUs, "gloo"/"cpu" for the CPU tests."""

    def __init__(self, backend="nccl", device="cuda"):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def _sync(self):
        if self.device == "cuda":
            import torch
            torch.cuda.synchronize()

    def barrier(self):
        """Synchronize the device, wait for every rank, synchronize again."""
        self._sync()
        if self.dist:
            self.dist.barrier()
        self._sync()

    def max(self, value):
        """The largest of the ranks' values (a float)."""
        if not self.dist:
            return float(value)
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(units_per_rank, world, steps, max_ms):
    """Units (particle-steps) per second of the whole job: every rank's units over the
    slowest rank's time."""
    return units_per_rank * world * steps / (max_ms * 1e-3)


def make_workload(name, rank=0):
    from paper_2410_18414_gb300 import workloads
    w = WORKLOADS[name]
    return workloads.weibel(w["n"], w["n"], w["ppc"], w["v_drift"], w["u_th"], w["seed"] + rank,
                            w["p"], "bdf", 2, 2000)


def dirk_tableau(name):
    # Butcher tableaux of the readings used for DIRK-2 (Qin-Zhang) and DIRK-3.
    if name == "dirk2":
        return {"A": [[0.25, 0.0], [0.5, 0.25]], "b": [0.5, 0.5], "c": [0.25, 0.75]}
    return {"A": [[1 / 6, 0, 0], [1 / 3, 1 / 6, 0], [1 / 3, 1 / 3, 1 / 6]],
            "b": [1 / 3, 1 / 3, 1 / 3], "c": [1 / 6, 0.5, 5 / 6]}


def make_config(wl, stepper_name, precision="fp64", sort_interval=0):
    from paper_2410_18414_gb300 import pic
    stepper, k = STEPPER_NAMES[stepper_name]
    dirk = dirk_tableau(stepper_name) if stepper == "dirk" else None
    prec = pic.FP32_FIX64 if precision == "fp32" else pic.FP64
    return pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=wl.p, stepper=stepper,
                           bdf_order=k, dirk=dirk, weight=wl.weight, precision=prec,
                           sort_interval=sort_interval)


def workload_desc(name, wl, stepper_name):
    w = WORKLOADS[name]
    shape = {2: "quadratic", 3: "cubic", 4: "quartic"}[wl.p]
    return {"workload": f"weibel_{wl.nx}x{wl.ny}_ppc{w['ppc']}_{shape}_{stepper_name}",
            "nx": wl.nx, "ny": wl.ny, "particles_per_gpu": wl.n, "spline_order": wl.p,
            "stepper": stepper_name, "dt": wl.dt, "v_drift": w["v_drift"], "u_th": w["u_th"]}


# --------------------------------------------------- algorithmic op counts --
# Per particle, counted from the arithmetic the method needs (see the design notes):
# weights of one axis for degree p (incl. x/dx), gather: one weight product and 8
# FMAs per node, IAEM push 31 flops; deposit: move 4, per node 2 products + 2 adds.
WEIGHT_FLOPS = {2: 10, 3: 19, 4: 39}


def flops_gather_push(p):
    return 2 * WEIGHT_FLOPS[p] + 17 * (p + 1) ** 2 + 31


def flops_move_deposit(p):
    return 4 + 2 * WEIGHT_FLOPS[p] + 2 * (p + 1) + 4 * (p + 1) ** 2


def bytes_gather_push(rsz):
    return 12 * rsz     # read x, y, Px, Py, v^n, v^{n-1} (8); write Px, Py, v^{n+1} (4)


def bytes_move_deposit(rsz):
    return 6 * rsz      # read x, y, v^n (4); write x, y (2)


def bytes_gather_deposit(rsz):
    # the fused kernel: read x, y, Px, Py, v^n, v^{n-1} (8); write Px, Py, v^{n+1}, x, y (6)
    return 14 * rsz


def flops_gather_deposit(p):
    return flops_gather_push(p) + flops_move_deposit(p)


# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel on a workload, from a
# committed ncu capture (profiles/), with the SHA-1 of the kernel's source file at capture
# time: when the source has changed since, the bench line reports no traffic.
TRAFFIC = {
    # (kernel, workload): (bytes per launch, source file, its SHA-1 prefix, profile)
    ("gather_deposit", "weibel128"): (34.43e6 + 0.017e6, "particles.cu", "9ba05500f8ad",
                                      "profiles/gather_deposit_fused_weibel128.md"),
    ("gather_deposit", "weibel512"): (853.19e6 + 592.23e6, "particles.cu", "9ba05500f8ad",
                                      "profiles/gather_deposit_fused_weibel512.md"),
}


# Shared-memory wavefronts per launch (l1tex__data_pipe_lsu_wavefronts_mem_shared.sum) of the
# fused FP32 kernel, from the same kind of committed capture: the pipe that bounds it.  One
# wavefront per SM clock is the pipe's peak (128 B a clock).
SMEM_WAVEFRONTS = {
    # (kernel, workload): (wavefronts per launch, source file, its SHA-1 prefix, profile)
    ("gather_deposit", "weibel128"): (9.40e6, "particles.cu", "9ba05500f8ad",
                                      "profiles/gather_deposit_fused_weibel128.md"),
}


def source_sha1(name):
    import hashlib
    path = os.path.join(ROOT, "paper_2410_18414_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def traffic_of(kernel, workload):
    entry = TRAFFIC.get((kernel, workload))
    if entry is None:
        return None, "no ncu capture of this kernel on this workload is committed"
    nbytes, src, sha, profile = entry
    if source_sha1(src) != sha:
        return None, f"{src} changed since the capture in {profile}"
    return nbytes, f"ncu capture: {profile}"


def smem_pipe_of(kernel, workload, ms, sm_mhz, nsm):
    """The kernel's shared-memory pipe use: committed wavefronts per launch over the
    event-timed launch, per SM clock at the sampled clock (peak 1.0), or None."""
    entry = SMEM_WAVEFRONTS.get((kernel, workload))
    if entry is None:
        return None
    wf, src, sha, profile = entry
    if source_sha1(src) != sha:
        return {"wavefronts": None, "source": f"{src} changed since the capture in {profile}"}
    per_clk = wf / (ms * 1e-3 * nsm * sm_mhz * 1e6)
    return {"wavefronts": wf, "achieved": per_clk, "peak": 1.0,
            "unit": "wavefronts per SM clock", "frac": per_clk,
            "source": f"ncu capture: {profile}; {nsm} SMs at the measured {sm_mhz:.0f} MHz"}


_FP64 = {}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "hbm_src": "fallback"}
    try:
        with open(path) as f:
            m = json.load(f)
        out["hbm_gbs"] = float(m["hbm_gbs"])
        out["hbm_src"] = "measured"
    except Exception:
        pass
    if "gflops" not in _FP64:   # the FP64 FMA rate, measured once on this device
        try:
            from paper_2410_18414_gb300 import pic
            _FP64["gflops"] = pic.measure_fp64_fma()
            _FP64["src"] = "measured: pic_measure_fp64_fma (FP64 FMA chains on every SM)"
        except Exception as exc:
            _FP64["gflops"] = 1250.0
            _FP64["src"] = f"nominal 1.25 TFLOP/s (measurement failed: {exc})"[:200]
    out["fp64_gflops"] = _FP64["gflops"]
    out["fp64_src"] = _FP64["src"]
    return out


def fp32_peak_gflops(sm_mhz):
    """FP32 FMA peak from the unit counts and the measured clock: 152 SMs x 128 FP32 lanes
    x 2 flops per FMA per cycle."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e9


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle --

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import pic as opic
from paper_2410_18414_gb300 import workloads
wl = workloads.weibel({nx}, {nx}, {ppc}, {v_drift}, {u_th}, {seed}, {p}, "bdf", 2, 2000)


def start(n):
    cfg = opic.Config(nx={nx}, ny={nx}, lx=wl.lx, ly=wl.ly, dt=wl.dt, p={p},
                      stepper={stepper!r}, bdf_order={k}, dirk={dirk!r}, w=wl.lx * wl.ly / n)
    return cfg, opic.initial_state(cfg, wl.x[:n], wl.y[:n], wl.vx[:n], wl.vy[:n])


def one_step_s(n):
    cfg, st = start(n)
    opic.step(cfg, st)
    t0 = time.perf_counter()
    opic.step(cfg, st)
    return time.perf_counter() - t0


n = min({n}, len(wl.x))
budget = {budget_s}
if budget > 0:
    # a step costs a + b n (the grid's transforms plus the particles): size the sample so
    # that warm-up and timed steps fit the budget
    n0, n1 = 1024, min(16384, n)
    t0, t1 = one_step_s(n0), one_step_s(n1)
    b = max((t1 - t0) / (n1 - n0), 1e-9) if n1 > n0 else 1e-9
    a = max(t0 - b * n0, 0.0)
    per_step = budget / max(1, {warmup} + {steps})
    n = int(min(n, max(n0, (per_step - a) / b)))
cfg, st = start(n)
for _ in range({warmup}):
    opic.step(cfg, st)
times = []
for _ in range({steps}):
    t0 = time.perf_counter()
    opic.step(cfg, st)
    times.append(time.perf_counter() - t0)
print(json.dumps({{"times": times, "n": n}}))
"""


def workload_params(workload):
    """WORKLOADS entry, or for the ensemble the parameters of its first run."""
    if workload in WORKLOADS:
        return WORKLOADS[workload]
    from paper_2410_18414_gb300 import workloads
    sp = workloads.ensemble_specs(count=1)[0]
    return dict(n=sp["n"], ppc=sp["ppc"], v_drift=sp["v_drift"], u_th=0.01, p=3,
                seed=sp["seed"], stepper="bdf2")


def run_oracle(workload, stepper_name, n, steps, warmup, budget_s=0.0, threads=1):
    """Per-step times of the oracle on the first n particles of the workload (weight
    rescaled), after `warmup` untimed steps, with `threads` BLAS threads (the oracle's
    transforms are dense matrix products).  budget_s > 0: n is lowered, from a two-size
    probe of the step cost, so that all the steps take about budget_s.  Returns (times, n)."""
    stepper, k = STEPPER_NAMES[stepper_name]
    dirk = dirk_tableau(stepper_name) if stepper == "dirk" else None
    w = workload_params(workload)
    code = ORACLE_SNIPPET.format(root=ROOT, seed=w["seed"], n=n, stepper=stepper, k=k, dirk=dirk,
                                 warmup=warmup, steps=steps, nx=w["n"], ppc=w["ppc"],
                                 v_drift=w["v_drift"], u_th=w["u_th"], p=w["p"],
                                 budget_s=float(budget_s))
    nt = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=nt, OPENBLAS_NUM_THREADS=nt, MKL_NUM_THREADS=nt,
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    if budget_s <= 0 and out["n"] != n:
        raise RuntimeError(f"the workload holds only {out['n']} particles, fewer than {n}")
    return out["times"], out["n"]


def cpu_baseline(workload, stepper_name, threads=1):
    """The oracle as it stands on a sample of the workload: one host thread, or `threads`
    BLAS threads (the host's cores)."""
    n = 262144
    steps = 12
    times, _ = run_oracle(workload, stepper_name, n, steps, 1, threads=threads)
    v = n * len(times) / sum(times)
    w = WORKLOADS[workload]
    total = w["n"] * w["n"] * w["ppc"]
    how = "single thread" if threads == 1 else f"{threads} BLAS threads (all host cores)"
    return {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"numpy FP64 oracle, {how}, {w['n']}x{w['n']} grid with the first "
                      f"{n} of the {total:,} particles (weight rescaled), {steps} timed steps "
                      f"after 1 warm-up, {sum(times):.1f} s"}


ADJOINT_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import adjoint as oadj, pic as opic
from paper_2410_18414_gb300 import workloads
wl = workloads.weibel_adjoint_128()
n, steps = {n}, {steps}
w = wl.lx * wl.ly / n
cfg = opic.Config(nx=wl.nx, ny=wl.ny, lx=wl.lx, ly=wl.ly, dt=wl.dt, p=wl.p, w=w,
                  **json.loads({stepper_kw!r}))
args = (cfg, wl.x[:n], wl.y[:n], wl.vx[:n], wl.vy[:n], steps)
t0 = time.perf_counter(); opic.run(*args); t1 = time.perf_counter()
tape = oadj.record(*args); oadj.gradient(tape); t2 = time.perf_counter()
print(json.dumps({{"forward_s": t1 - t0, "gradient_s": t2 - t1}}))
"""


def run_reference_adjoint(a):
    """The reference arm of `--workload adjoint128`: the oracle's own forward run and its
    recorded run plus reverse sweep (oracle.adjoint), on a bounded sample of the workload
    (128 x 128 grid, the first 8192 of its 262,144 particles with the weight rescaled, 10
    steps), as the same ratio."""
    n, steps = 8192, min(10, max(1, a.steps))
    stepper, k = STEPPER_NAMES[a.stepper]
    kw = dict(stepper=stepper, bdf_order=k)
    if stepper == "dirk":
        kw["dirk"] = dirk_tableau(a.stepper)
    code = ADJOINT_ORACLE_SNIPPET.format(root=ROOT, n=n, steps=steps, stepper_kw=json.dumps(kw))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle adjoint run failed: " + r.stderr[-2000:])
    t = json.loads(r.stdout.strip().splitlines()[-1])
    ratio = t["gradient_s"] / t["forward_s"]
    sample = (f"numpy FP64 oracle, single thread: 128x128 grid, the first {n} of the 262,144 "
              f"particles (weight rescaled), {steps} steps; forward {t['forward_s']:.1f} s, "
              f"recorded run + reverse sweep {t['gradient_s']:.1f} s")
    line = {"metric": "adjoint/forward time", "value": ratio, "unit": "ratio",
            "impl": "reference", "n_gpus": a.gpus, "steps": steps, "warmup": 0,
            "ms_per_step": 1e3 * t["gradient_s"] / steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"weibel_adjoint_128x128_16ppc_cubic_{a.stepper}", "form": "fp64",
                       "sample_particles": n, "parallelism": "replicas"},
            "cpu_baseline": {"value": ratio, "unit": "ratio", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": ratio, "unit": "ratio", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(a):
    """The reference arm: the CPU oracle on the host cores, bounded samples of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if a.workload == "adjoint128":
        run_reference_adjoint(a)
        return
    wp = workload_params(a.workload)
    # every one of the K + W steps runs, each on a sample sized so that they all take
    # about two minutes of one host core
    n = min(131072, wp["n"] * wp["n"] * wp["ppc"])
    times, n = run_oracle(a.workload, a.stepper, n, a.steps, a.warmup, budget_s=120.0)
    total = sum(times)
    value = n * len(times) / total
    if a.workload in WORKLOADS:
        wl_desc = workload_desc(a.workload, make_workload(a.workload), a.stepper)
    else:
        wp = workload_params(a.workload)
        wl_desc = {"workload": "ensemble_256_weibel_cubic_bdf2",
                   "oracle_sample": f"first run: {wp['n']}x{wp['n']}, {wp['ppc']} per cell"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(wl_desc, form="fp64", sample_particles=n, parallelism="replicas"),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"each step: the numpy FP64 oracle on the {wp['n']}x{wp['n']} "
                                       f"grid with the first {n} particles (weight rescaled; the "
                                       f"sample sized so that the {a.warmup} + {a.steps} steps take "
                                       f"about 2 minutes), single thread"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm --

KERNEL_GROUPS = ("sort", "deposit", "field_solve", "gather_push", "gather_deposit")


def time_steps(sim, steps, warmup, stream, flush, count=None, detail=False):
    """Per-step device times (CUDA events on the simulation's stream), one pic_step call
    per step, L2 flushed between steps outside the events.  detail=True also runs the
    library's per-kernel event pairs (pic_set_kernel_timing) around each launch group:
    the sort, the separate deposit, the field solve, the separate gather + push and the
    fused gather + push + next deposit of the sorted FP32 form."""
    import torch
    for _ in range(warmup):
        sim.step(1)
        flush.zero_()
    torch.cuda.synchronize()
    if detail:
        sim.set_kernel_timing(steps + 1)   # the library's per-kernel event pairs, made up front
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for k in range(steps):
        e = ev[k]
        e[0].record(stream)
        sim.step(1)
        e[1].record(stream)
        if count is not None:
            count[0] += sim.kernels_per_step
        flush.zero_()       # cold L2 for the next step (outside the events)
    torch.cuda.synchronize()
    out = {"step_ms": [e[0].elapsed_time(e[1]) for e in ev]}
    if detail:
        kt = {}
        for name in KERNEL_GROUPS:
            ms, nl = sim.kernel_time(name)
            kt[name] = {"launches": nl, "ms_per_launch": ms / nl if nl else None, "ms_total": ms}
        sim.set_kernel_timing(0)
        out["kernels"] = kt
    return out


def run_ensemble(a):
    """The ensemble workload on its own (--workload ensemble256): one JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    line = ensemble_line(ranks, a.steps, a.warmup)
    ranks.close()
    if line is not None:
        print(json.dumps(line))


def ensemble_line(ranks, steps, warmup):
    """256 independent Weibel runs (grid sizes, densities and drifts drawn per run; FP32
    form, BDF-2, cubic), tile widths and sort intervals from the autotuner, advanced
    together by one
    CUDA-graph launch per period (pic_ensemble_step); the same runs stepped on their own
    streams without the graph are timed beside it.  Returns rank 0's line (None on the
    other ranks)."""
    import torch
    from paper_2410_18414_gb300 import autotune, pic, workloads
    rank, world = ranks.rank, ranks.world
    pic.load_library()
    specs = workloads.ensemble_specs(seed0=1000 + 256 * rank)
    t0 = time.perf_counter()
    tuned = [autotune.tune(sp["n"], sp["ppc"])[:2] for sp in specs]
    tune_s = time.perf_counter() - t0

    def build():
        sims, streams = [], []
        for sp, (ti, si) in zip(specs, tuned):
            wl = workloads.ensemble_run(sp)
            cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf",
                                  bdf_order=2, weight=wl.weight, precision=pic.FP32_FIX64,
                                  sort_interval=si, tile=ti)
            st = torch.cuda.Stream()
            sims.append(pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=st.cuda_stream))
            streams.append(st)
        return sims, streams

    def join(master, streams):
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            master.wait_event(ev)

    sims, streams = build()
    n_total = sum(s.n for s in sims)
    master = torch.cuda.Stream()
    t0 = time.perf_counter()
    ens = pic.Ensemble(sims, master.cuda_stream)
    capture_s = time.perf_counter() - t0
    P = ens.period
    full, rest = (steps // P) * P, steps % P
    warm = max(1, -(-warmup // P)) * P         # whole periods keep the runs in phase
    ens.step(warm)
    ranks.barrier()
    clocks = ClockSampler(ranks.local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(master)
    ens.step(full)
    for s in sims:      # the steps left over after whole periods, on the runs' own streams
        if rest:
            s.step(rest)
    join(master, streams)
    e1.record(master)
    e1.synchronize()
    clk = clocks.stop()
    ranks.barrier()
    ms = ranks.max(e0.elapsed_time(e1))
    ens.close()
    for s in sims:
        s.sync()  # reports any latched device error
        s.close()
    # the same runs without the graph: every run's steps enqueued on its own stream
    sims, streams = build()
    for s in sims:
        s.step(warm)
    ranks.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(master)
    for st in streams:         # start after the event above
        st.wait_event(f0)
    for s in sims:
        s.step(steps)
    join(master, streams)
    f1.record(master)
    f1.synchronize()
    ranks.barrier()
    ms_plain = ranks.max(f0.elapsed_time(f1))
    for s in sims:
        s.close()
    if rank != 0:
        return None
    value = whole_job_rate(n_total, world, steps, ms)
    hist = {}
    for ti, si in tuned:
        hist[f"T{ti}_S{si}"] = hist.get(f"T{ti}_S{si}", 0) + 1
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ensemble_256_weibel_cubic_bdf2", "runs": len(specs),
                   "particles_total": n_total, "grid_sizes": sorted({sp["n"] for sp in specs}),
                   "ppc_range": [min(sp["ppc"] for sp in specs), max(sp["ppc"] for sp in specs)],
                   "tile_and_sort_interval": hist, "period": P, "graph_steps": full,
                   "steps_outside_graph": rest, "form": "fp32_fix64",
                   "l2": "no flush: the ensemble's particle state (about 7 GB) is far larger "
                         "than L2", "parallelism": "single"},
        "roofline": {"kernel": "whole step, all runs", "bound": "hbm",
                     "achieved": 56.0 * n_total * steps / (ms * 1e-3) / 1e9,
                     "peak": peaks()["hbm_gbs"], "unit": "GB/s",
                     "frac": 56.0 * n_total * steps / (ms * 1e-3) / 1e9 / peaks()["hbm_gbs"],
                     "traffic": None, "peak_source": peaks()["hbm_src"],
                     "note": "56 B algorithmic per particle-step (the fused gather + push + "
                             "move + deposit: 8 values read, 6 written)"},
        "no_graph": {"ms_per_step": ms_plain / steps,
                     "value": whole_job_rate(n_total, world, steps, ms_plain),
                     "how": "each run's steps enqueued on its own stream, no graph"},
        "ps_per_particle_step": ms * 1e9 / (n_total * steps),
        "autotune_s": tune_s, "capture_s": capture_s,
        "cpu_baseline": None, "e2e": None,
        "gpu_launches": None, "clocks": clk,
    }
    return line


def adjoint_timings(steps, reps, rank=0, stepper="bdf2", form="fp64"):
    """Gradient of the magnetic energy W_B = 1/2 sum B_z^2 dx dy after `steps` (at most 200)
    steps of the 128x128 Weibel run with 16 particles per cell (262,144), cubic, under
    `stepper` (a STEPPER_NAMES key; BDF-2 by default), with respect to every initial
    velocity and momentum, by the library's adjoint of the FP64 run or (form "fp32") of the
    unsorted FP32 form, each against its own plain forward run.
    Timed per whole run with CUDA events (L2 flushed before each run): the plain forward
    run (pic_step), the recording forward run and the reverse sweep, with checkpoints every
    20 steps -- replaying the particle states of each segment from the recorded gathered
    fields (the default), or recomputing each segment's full steps (least memory) -- and
    with one segment of 200 steps; one more sweep runs under the library's adjoint kernel
    timers."""
    import torch
    from paper_2410_18414_gb300 import pic, workloads
    pic.load_library()
    wl = workloads.weibel_adjoint_128(seed=5 + rank)
    cfg = make_config(wl, stepper, precision=form)
    rsz = 4 if form == "fp32" else 8
    N = min(wl.nsteps, steps)
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    area = (wl.lx / wl.nx) * (wl.ly / wl.ny)
    x = torch.tensor(wl.x, device="cuda")
    y = torch.tensor(wl.y, device="cuda")
    vx = torch.tensor(wl.vx, device="cuda")
    vy = torch.tensor(wl.vy, device="cuda")
    bz = torch.empty((wl.nx, wl.ny), dtype=torch.float64, device="cuda")
    out = {k: torch.empty(wl.n, dtype=torch.float64, device="cuda") for k in ("vx", "vy", "px", "py")}

    def once(K, mode="replay"):
        sim = pic.Simulation(cfg, x, y, vx, vy, stream=sid)
        adj = pic.Adjoint(sim, N, K, mode=mode) if K else None
        flush.zero_()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        if adj is None:
            sim.step(N)
        else:
            adj.forward()
        ev[1].record(stream)
        if adj is not None:
            sim.field("bz", out=bz)
            adj.backward(bz_bar=(bz * area).contiguous(), out=out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if adj is not None:
            adj.close()
        sim.close()
        return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    k20 = min(20, N)
    for K, mode in ((0, "replay"), (k20, "replay"), (k20, "recompute"), (k20, "replay_lean"),
                    (N, "replay")):
        once(K, mode)          # warm-up: one of each
    # one instrumented reverse sweep (every step kept): the library's per-kernel event
    # pairs around the three reverse launch groups of every step
    sim = pic.Simulation(cfg, x, y, vx, vy, stream=sid)
    adj = pic.Adjoint(sim, N, N)
    adj.forward()
    sim.field("bz", out=bz)
    flush.zero_()
    torch.cuda.synchronize()
    sim.set_kernel_timing(N + 1)
    adj.backward(bz_bar=(bz * area).contiguous(), out=out)
    kt = {}
    for name in ("adj_push", "adj_field", "adj_deposit"):
        ms, nl = sim.kernel_time(name)
        kt[name] = {"launches": nl, "ms_per_launch": ms / nl if nl else None}
    sim.set_kernel_timing(0)
    adj.close()
    sim.close()
    med = statistics.median
    fwd = med([once(0)[0] for _ in range(reps)])
    t20 = [once(k20) for _ in range(reps)]
    t20r = [once(k20, "recompute") for _ in range(reps)]
    t20l = [once(k20, "replay_lean") for _ in range(reps)]
    tall = [once(N) for _ in range(reps)]
    r20 = (med([t[0] for t in t20]) + med([t[1] for t in t20])) / fwd
    r20r = (med([t[0] for t in t20r]) + med([t[1] for t in t20r])) / fwd
    r20l = (med([t[0] for t in t20l]) + med([t[1] for t in t20l])) / fwd
    rall = (med([t[0] for t in tall]) + med([t[1] for t in tall])) / fwd
    seg = (N + k20 - 1) // k20
    st = 8 * rsz * wl.n          # one particle state
    gf = 8 * rsz * wl.nx * wl.ny  # one step's gather fields
    return {
        "workload": f"weibel_adjoint_128x128_16ppc_cubic_{stepper}", "particles": wl.n,
        "steps_per_run": N, "form": form, "objective": "W_B at the last step",
        "forward_ms": fwd,
        "checkpoint_20": {"mode": "replay", "record_forward_ms": med([t[0] for t in t20]),
                          "backward_ms": med([t[1] for t in t20]), "ratio": r20,
                          "record_bytes": int(N * (80 * wl.n + gf) + (seg + 1 + k20) * st)},
        "checkpoint_20_recompute": {"mode": "recompute",
                                    "record_forward_ms": med([t[0] for t in t20r]),
                                    "backward_ms": med([t[1] for t in t20r]), "ratio": r20r,
                                    "record_bytes": int((seg + 1) * st + k20 * (
                                        80 * wl.n + st + gf))},
        "checkpoint_20_lean": {"mode": "replay_lean",
                               "record_forward_ms": med([t[0] for t in t20l]),
                               "backward_ms": med([t[1] for t in t20l]), "ratio": r20l,
                               "record_bytes": int(N * (32 * wl.n + gf) + (seg + 1 + k20) * st)},
        "keep_all_steps": {"mode": "replay", "record_forward_ms": med([t[0] for t in tall]),
                           "backward_ms": med([t[1] for t in tall]), "ratio": rall,
                           "record_bytes": int(N * (80 * wl.n + st + gf))},
        "kernels": kt,
        "roofline": adjoint_roofline(wl.p, wl.n, kt["adj_push"]["ms_per_launch"], form),
    }


def run_adjoint(a):
    """`--workload adjoint128`: the adjoint timings as their own line.  value = (recording
    forward + reverse sweep) / plain forward with checkpoints every 20 steps."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks()
    rank, world = ranks.rank, ranks.world
    ranks.barrier()
    clocks = ClockSampler(ranks.local)
    clocks.start()
    t = adjoint_timings(a.steps, max(1, a.repeats), rank, a.stepper, a.adjoint_form)
    clk = clocks.stop()
    ranks.barrier()
    # every replica's own ratio; the line reports the slowest rank's
    ratio = ranks.max(t["checkpoint_20"]["ratio"])
    ranks.close()
    if rank != 0:
        return
    line = {
        "metric": "adjoint/forward time", "value": ratio, "unit": "ratio",
        "n_gpus": world, "steps": t["steps_per_run"], "warmup": 1, "repeats": max(1, a.repeats),
        "ms_per_step": t["checkpoint_20"]["backward_ms"] / t["steps_per_run"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if t["form"] == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": t["workload"], "particles": t["particles"],
                   "steps_per_run": t["steps_per_run"], "objective": t["objective"],
                   "gradient": "dW_B/dv0 and dW_B/dP0, every particle", "form": t["form"],
                   "l2": "flushed (256 MiB write) before each timed run", "parallelism": "replicas"},
        "forward_ms": t["forward_ms"], "checkpoint_20": t["checkpoint_20"],
        "checkpoint_20_recompute": t["checkpoint_20_recompute"],
        "checkpoint_20_lean": t["checkpoint_20_lean"],
        "keep_all_steps": t["keep_all_steps"], "kernels": t["kernels"], "roofline": t["roofline"],
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def flops_adj_push(p):
    """FP64 flops per particle of k_adj_push_gather: weights and their derivatives on both
    axes, the reverse push (48), per stencil node the field dot product, the separable
    position-gradient sums, the weight product and the eight deposit operands (29), per
    row the two cross-row sums (4), and the final updates (10).  600 for cubic shapes."""
    w = {2: 10, 3: 19, 4: 39}[p]
    dw = {2: 5, 3: 12, 4: 25}[p]
    return 2 * (w + dw) + 48 + 29 * (p + 1) ** 2 + 4 * (p + 1) + 10


def adjoint_roofline(p, n, ms, form="fp64"):
    """k_adj_push_gather against the FP64 pipe (its FMA rate measured on this device); in
    the FP32 form its particle arithmetic is FP32 (the field-adjoint sums stay FP64) and
    the FP32 peak is the reference."""
    if not ms:
        return None
    pk = peaks()
    achieved = flops_adj_push(p) * n / (ms * 1e-3) / 1e12
    if form == "fp32":
        peak, src = fp32_peak_gflops(2070), "FP32 FMA issue rate at the 2070 MHz maximum SM clock"
        traffic, traffic_src = None, "not captured for the FP32 form"
    else:
        peak, src = pk["fp64_gflops"], pk["fp64_src"]
        traffic, traffic_src = traffic_of("adj_push_gather", "adjoint128")
    return {"kernel": "k_adj_push_gather", "bound": "alu", "achieved": achieved,
            "peak": peak / 1e3, "unit": "TFLOP/s", "frac": achieved * 1e3 / peak,
            "traffic": traffic, "traffic_source": traffic_src, "peak_source": src,
            "note": f"{flops_adj_push(p)} {form.upper()} flops per particle (cubic: 600)"}


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload == "ensemble256":
        run_ensemble(a)
        return
    if a.workload == "adjoint128":
        run_adjoint(a)
        return
    import numpy as np
    import torch
    from paper_2410_18414_gb300 import pic

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ranks = Ranks()
    rank, world = ranks.rank, ranks.world
    pic.load_library()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    wl = make_workload(a.workload, rank)
    cfg = make_config(wl, a.stepper, a.precision, a.sort_interval)
    sim = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=sp)

    ranks.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches = [0]
    t = time_steps(sim, a.steps, a.warmup, stream, flush, launches)
    clk = clocks.stop()
    ranks.barrier()
    sim.sync()
    total_ms = ranks.max(sum(t["step_ms"]))
    n_all = wl.n * world
    value = whole_job_rate(wl.n, world, a.steps, total_ms)
    # per-kernel breakdown: an instrumented run of the same simulation right after the
    # timed region (its extra event records would slow the headline steps)
    nd = min(a.steps, 500)
    t = time_steps(sim, nd, 3, stream, flush, detail=True)

    # roofline of the dominant kernel: per-launch averages of the library's own event
    # pairs around each kernel (same stream, timed region only)
    pk = peaks()
    fp32 = a.precision == "fp32"
    rsz = 4 if fp32 else 8
    p = wl.p
    kt = t["kernels"]
    counts = {
        "gather_deposit": (flops_gather_deposit(p), bytes_gather_deposit(rsz)),
        "gather_push": (flops_gather_push(p), bytes_gather_push(rsz)),
        "deposit": (flops_move_deposit(p), bytes_move_deposit(rsz)),
    }
    kern = {}
    for name, (fl, by) in counts.items():
        if not kt[name]["launches"]:
            continue
        k = {"ms": kt[name]["ms_per_launch"], "launches": kt[name]["launches"],
             "flops": fl * wl.n, "bytes": by * wl.n}
        k["gflops"] = k["flops"] / (k["ms"] * 1e-3) / 1e9
        k["gbs"] = k["bytes"] / (k["ms"] * 1e-3) / 1e9
        k["frac_hbm"] = k["gbs"] / pk["hbm_gbs"]
        if not fp32:
            k["frac_fp64_alu"] = k["gflops"] / pk["fp64_gflops"]
        kern[name] = k
    # the dominant particle kernel: the one with the most time per step
    dom_name = max(kern, key=lambda k: kern[k]["ms"] * kern[k]["launches"])
    dom = kern[dom_name]
    traffic, traffic_src = traffic_of(dom_name, a.workload)
    if fp32:
        sm_mhz = clk.get("sm_mhz") or 2070.0
        roofline = {"kernel": dom_name, "bound": "hbm", "achieved": dom["gbs"],
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": dom["gbs"] / pk["hbm_gbs"],
                    "traffic": traffic, "traffic_source": traffic_src,
                    "peak_source": pk["hbm_src"],
                    "bytes_per_particle": dom["bytes"] / wl.n,
                    "fp32_alu": {"achieved_gflops": dom["gflops"],
                                 "peak_gflops": fp32_peak_gflops(sm_mhz),
                                 "frac": dom["gflops"] / fp32_peak_gflops(sm_mhz),
                                 "flops_per_particle": dom["flops"] / wl.n,
                                 "peak_source": f"152 SMs x 128 FP32 lanes x 2 at the measured "
                                                f"{sm_mhz:.0f} MHz"}}
        nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        smem = smem_pipe_of(dom_name, a.workload, dom["ms"], sm_mhz, nsm)
        if smem is not None:
            roofline["smem_pipe"] = smem
    else:
        roofline = {"kernel": dom_name, "bound": "alu", "achieved": dom["gflops"],
                    "peak": pk["fp64_gflops"], "unit": "GFLOP/s",
                    "frac": dom["gflops"] / pk["fp64_gflops"],
                    "traffic": traffic, "traffic_source": traffic_src,
                    "peak_source": pk["fp64_src"],
                    "hbm": {"achieved_gbs": dom["gbs"], "peak_gbs": pk["hbm_gbs"],
                            "frac": dom["gbs"] / pk["hbm_gbs"], "peak_source": pk["hbm_src"]}}

    # the configuration's whole run (its own step count, whatever --steps says): every
    # step in one pic_step call (the call's steps run back to back, so no L2 flush
    # separates them)
    full_steps = wl.nsteps
    sf = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=sp)
    sf.step(3)
    flush.zero_()
    ranks.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    sf.step(full_steps)
    f1.record(stream)
    f1.synchronize()
    full_ms = ranks.max(f0.elapsed_time(f1))
    sf.sync()
    sf.close()
    full_run = {"steps": full_steps, "ms": full_ms, "ms_per_step": full_ms / full_steps,
                "value": whole_job_rate(wl.n, world, full_steps, full_ms),
                "how": f"the configuration's {full_steps} steps in one pic_step call after 3 "
                       "warm-up steps; L2 not flushed between steps"}

    # the other precision form on the same workload (the metric's comparison)
    other = "fp64" if fp32 else "fp32"
    # (each form at its own best setting: the FP64 path's global FP64 atomics contend more
    # on tile-sorted particles, so it runs unsorted)
    other_sort = a.sort_interval if other == "fp32" else 0
    so = pic.Simulation(make_config(wl, a.stepper, other, other_sort), wl.x, wl.y, wl.vx,
                        wl.vy, stream=sp)
    to = time_steps(so, max(20, a.steps // 4), 5, stream, flush)
    tod = time_steps(so, 50, 2, stream, flush, detail=True)
    so.close()
    other_ms = statistics.mean(to["step_ms"])
    other_form = {"form": other, "ms_per_step": other_ms, "sort_interval": other_sort,
                  "value": wl.n * world / (other_ms * 1e-3),
                  "kernel_ms": {k: v["ms_per_launch"] for k, v in tod["kernels"].items()
                                if v["launches"]}}

    # the same form with the residual and energy diagnostics (a10) on every step
    sd = pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=sp)
    sd.set_diagnostics(1)
    td = time_steps(sd, max(20, a.steps // 4), 5, stream, flush)
    diag_res = sd.residuals()
    sd.close()
    diag_ms = statistics.mean(td["step_ms"])
    with_diagnostics = {"ms_per_step": diag_ms, "value": wl.n * world / (diag_ms * 1e-3),
                        "every": 1, "steps": len(td["step_ms"]),
                        "last_residuals": {k: diag_res[k] for k in
                                           ("gauge_rms", "gauss_rms", "continuity_rms",
                                            "div_a_rms", "rho_rms", "w_b", "w_e", "kinetic")}}

    # other steppers of the same workload (shorter runs)
    by_stepper = {a.stepper: total_ms / a.steps}
    if not a.no_extra_steppers:
        for name in ("bdf2", "cdf2", "dirk2"):
            if name == a.stepper:
                continue
            s2 = pic.Simulation(make_config(wl, name, a.precision, a.sort_interval), wl.x, wl.y,
                                wl.vx, wl.vy, stream=sp)
            t2 = time_steps(s2, max(10, a.steps // 5), 3, stream, flush)
            by_stepper[name] = statistics.mean(t2["step_ms"])
            s2.close()

    # end to end through the public API with pinned host buffers
    host = {k: torch.from_numpy(getattr(wl, k).copy()).pin_memory() for k in ("x", "y", "vx", "vy")}
    outs = {k: torch.empty(wl.n, dtype=torch.float64).pin_memory()
            for k in ("x", "y", "px", "py", "vx", "vy", "vx_old", "vy_old")}
    ranks.barrier()
    t0 = time.perf_counter()
    s3 = pic.Simulation(cfg, host["x"], host["y"], host["vx"], host["vy"], stream=sp)
    s3.step(a.steps)
    s3.particles(outs)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ranks.barrier()
    s3.close()
    e2e = {"value": n_all * a.steps / e2e_s if world == 1 else None, "unit": METRIC,
           "h2d_bytes_per_step": 4 * 8 * wl.n / a.steps,
           "d2h_bytes_per_step": 8 * 8 * wl.n / a.steps,
           "includes": "pic_init from pinned host arrays (incl. device allocation and t=0 solve), "
                       "K steps, read-back of all 8 particle arrays"}
    if world > 1:
        e2e["value"] = n_all * a.steps / ranks.max(e2e_s)

    # the adjoint (the metric's "adjoint/forward time"): the gradient of W_B on the
    # 262,144-particle Weibel workload, FP64, one timed run per checkpoint setting
    adjoint = adjoint32 = None
    if not a.no_adjoint:
        adjoint = adjoint_timings(200, 1, rank)
        adjoint32 = adjoint_timings(200, 1, rank, form="fp32")

    # the batched ensemble (256 independent runs, one graph launch per period)
    ensemble = None
    if not a.no_ensemble:
        eline = ensemble_line(ranks, 300, 20)
        if eline is not None:
            ensemble = {k: eline[k] for k in ("value", "unit", "ms_per_step", "steps", "config",
                                              "roofline", "no_graph", "autotune_s",
                                              "capture_s", "clocks")}

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        for threads in (1, os.cpu_count() or 1):
            try:
                res = cpu_baseline(a.workload, a.stepper, threads)
            except Exception as exc:  # the line still prints; the failure is stated
                res = {"value": None, "unit": METRIC, "cores": threads, "kind": "oracle",
                       "sample": f"failed: {exc}"[:300]}
            if threads == 1:
                cpu = res
            else:
                cpu_all = res

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
            "data": "synthetic",
            "config": dict(workload_desc(a.workload, wl, a.stepper),
                           form="fp32_fix64" if fp32 else "fp64",
                           l2="flushed between timed steps (256 MiB device write)",
                           sort_interval=a.sort_interval,
                           parallelism="replicas" if world > 1 else "single"),
            "roofline": roofline,
            "kernels": {k: {kk: round(vv, 6) if isinstance(vv, float) else vv
                            for kk, vv in v.items()} for k, v in kern.items()},
            "kernel_ms": {k: v["ms_per_launch"] for k, v in kt.items()},
            "kernel_launches": {k: v["launches"] for k, v in kt.items()},
            "detail_steps": nd,
            "full_run": full_run,
            "by_stepper_ms_per_step": by_stepper,
            "other_form": other_form,
            "ratio_vs_other_form": (total_ms / a.steps) and other_ms / (total_ms / a.steps),
            "with_diagnostics": with_diagnostics,
            "adjoint": adjoint, "adjoint_fp32": adjoint32,
            "ensemble": ensemble,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e,
            "gpu_launches": launches[0],
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    ranks.close()


if __name__ == "__main__":
    main()
