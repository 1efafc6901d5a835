"""Tile-width and sort-interval autotuner for the sorted FP32 form.

The sort interval S trades the cost of a sort (every S steps) against the drift of the
particles away from their sorted cells, which spreads each CTA's particles over more
shared-memory rows and pushes particles out of their tile's region.  The tile width T
sets how many cells a tile holds: wider tiles mean fewer, fuller tiles and more of the
region in shared memory per CTA, narrower ones a smaller region and more CTAs.  The best
pair depends on the grid size, the particles per cell and the shape order, and on
whether the run has the GPU to itself: a lone small run wants many small CTAs, while runs
stepped together (an ensemble) want the least work per particle.  So it is measured as
throughput under load: several copies of a probe run of the same grid size, density class
and shape (enough for about 4 M particles, at most 16) step concurrently on their own
streams for every candidate pair (CUDA events around whole periods of the longest
interval, so every candidate pays its sorts in full), and the pair with the least time per
step is kept, cached per key (grid size, density class, shape order, form).
"""
from . import pic, workloads

TILES = (4, 8, 16)
SORT_INTERVALS = (1, 2, 4, 8, 16)
DENSITY_CLASSES = (16, 32, 64)
_cache = {}


def density_class(ppc):
    """The nearest of DENSITY_CLASSES (particles per cell of the probe run)."""
    return min(DENSITY_CLASSES, key=lambda c: abs(c - ppc))


def candidates(n_axis, tiles=TILES, sort_intervals=SORT_INTERVALS):
    """The (T, S) pairs probed on an n_axis x n_axis grid: tiles of at most half the grid."""
    return [(t, s) for t in tiles if 2 * t <= n_axis for s in sort_intervals]


def copies_for(n_particles, target=4 << 20, most=16):
    """How many copies of a probe run of n_particles step together in a probe."""
    return max(1, min(most, -(-target // max(1, n_particles))))


def probe_ms(n_axis, ppc, tile, sort_interval, p=3, precision=pic.FP32_FIX64,
             stepper="bdf", bdf_order=2, periods=2, copies=None):
    """ms per step of `copies` concurrent Weibel-like probe runs under (tile,
    sort_interval), each on its own stream: CUDA events around `periods` x 16 steps of
    every copy, after one warm-up interval."""
    import torch
    wl = workloads.weibel(n_axis, n_axis, ppc, 0.5, 0.01, 7, p, stepper, bdf_order, 0)
    copies = copies or copies_for(wl.n)
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=p, stepper=stepper,
                          bdf_order=bdf_order, weight=wl.weight, precision=precision,
                          sort_interval=sort_interval, tile=tile)
    streams = [torch.cuda.Stream() for _ in range(copies)]
    sims = [pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=st.cuda_stream)
            for st in streams]
    try:
        for sim in sims:
            sim.step(sort_interval)  # warm-up, one sort
        torch.cuda.synchronize()
        steps = periods * max(SORT_INTERVALS)
        master = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(master)
        for st in streams:
            st.wait_event(ev[0])
        for sim in sims:
            sim.step(steps)
        for st in streams:
            done = torch.cuda.Event()
            done.record(st)
            master.wait_event(done)
        ev[1].record(master)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / steps
    finally:
        for sim in sims:
            sim.close()


def tune(n_axis, ppc, p=3, precision=pic.FP32_FIX64, stepper="bdf", bdf_order=2,
         tiles=TILES, sort_intervals=SORT_INTERVALS, periods=2):
    """Fastest (tile, sort_interval) for n_axis x n_axis Weibel-like runs (cached).
    Returns (T, S, timings) with timings {(T, S): ms per step} of the probes (empty when
    the pair came from the cache)."""
    key = (n_axis, density_class(ppc), p, precision)
    if key in _cache:
        return _cache[key] + ({},)
    ms = {}
    for t, s in candidates(n_axis, tiles, sort_intervals):
        ms[(t, s)] = probe_ms(n_axis, key[1], t, s, p, precision, stepper, bdf_order,
                              periods)
    best = min(ms, key=ms.get)
    _cache[key] = best
    return best + (ms,)
