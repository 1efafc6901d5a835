"""Sort-interval autotuner for the FP32 form.

The sort interval S trades the cost of a sort (every S steps) against the drift of the
particles away from their sorted cells, which makes the tiled deposit's shared-memory
atomics collide and pushes particles out of their tile's region.  The best S depends on
the grid size, the particles per cell and the shape order, so it is measured: a probe
run of the same grid size, density class and shape is timed for each candidate (CUDA
events around whole periods of steps, so every candidate pays its sorts in full) and the
fastest is kept, cached per key (grid size, density class, shape order, form).  The tile
width needs no tuning: the library derives it from the particle density.
"""
from . import pic, workloads

CANDIDATES = (4, 8, 16)
DENSITY_CLASSES = (16, 32, 64)
_cache = {}


def density_class(ppc):
    """The nearest of DENSITY_CLASSES (particles per cell of the probe run)."""
    return min(DENSITY_CLASSES, key=lambda c: abs(c - ppc))


def tune_sort_interval(n_axis, ppc, p=3, precision=pic.FP32_FIX64, stepper="bdf",
                       bdf_order=2, candidates=CANDIDATES, periods=2):
    """Fastest sort interval for an n_axis x n_axis Weibel-like run (cached)."""
    import torch
    key = (n_axis, density_class(ppc), p, precision)
    if key in _cache:
        return _cache[key]
    wl = workloads.weibel(n_axis, n_axis, key[1], 0.5, 0.01, 7, p, stepper, bdf_order, 0)
    stream = torch.cuda.Stream()
    best = None
    for s in candidates:
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=p, stepper=stepper,
                              bdf_order=bdf_order, weight=wl.weight, precision=precision,
                              sort_interval=s)
        with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=stream.cuda_stream) as sim:
            sim.step(s)  # warm-up, one sort
            steps = periods * max(candidates)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            sim.step(steps)
            ev[1].record(stream)
            ev[1].synchronize()
            ms = ev[0].elapsed_time(ev[1]) / steps
        if best is None or ms < best[1]:
            best = (s, ms)
    _cache[key] = best[0]
    return best[0]
