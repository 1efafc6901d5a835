"""The FP32 form's first move and fixed-point current, bit for bit against the CPU model
oracle.fixed_point (pinned in tests/test_oracle_fixed_point.py): float32 positions after
the move and every node of J_x, J_y (the int64 sums, read back through the library's
scaling), for p = 2, 3, 4, unsorted (global int64 atomics) and sorted (the tiled pass:
split 32-bit shared sums flushed into int64), on a 48 x 32 grid with a ragged particle
count and particles that cross the periodic edges during the move.  And at the full size
of the benchmarked 128 x 128 run, the fused kernel's move and current (the deposit each
pic_step call leaves pending) from the state it starts from."""
import numpy as np
import pytest

from oracle import fixed_point as fx
from paper_2410_18414_gb300 import pic

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


@pytest.mark.parametrize("sort", [0, 1], ids=["unsorted", "sorted"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_first_move_and_current_bit_exact(device, p, sort):
    nx, ny, lx, ly = 48, 32, 1.0, 0.75
    n = 20011
    rng = np.random.default_rng(100 + p)
    x = rng.uniform(0, lx, n)
    y = rng.uniform(0, ly, n)
    vx = rng.uniform(-0.4, 0.4, n)   # |v| < 0.73 c with the edge offsets below
    vy = rng.uniform(-0.4, 0.4, n)
    # a few hundred particles just inside the edges, moving across them
    e = 300
    x[:e] = lx - rng.uniform(0, 2e-3, e)
    vx[:e] = np.abs(vx[:e]) + 0.2
    y[e:2 * e] = rng.uniform(0, 2e-3, e)
    vy[e:2 * e] = -np.abs(vy[e:2 * e]) - 0.2
    dt = 0.4 * lx / nx
    w, q = lx * ly / n, -1.0
    cfg = pic.make_config(nx, ny, lx, ly, dt, p=p, stepper="bdf", bdf_order=2, weight=w, q=q,
                          precision=pic.FP32_FIX64, sort_interval=sort)
    with pic.Simulation(cfg, x, y, vx, vy, stream=device) as sim:
        sim.step(1)
        got = sim.particles()
        jx, jy = sim.field("jx"), sim.field("jy")
    scale = fx.current_scale(1.0, n)
    x1, y1, ix, iy = fx.move_deposit(x, y, vx, vy, dt, lx, ly, nx, ny, p, scale)
    assert np.array_equal(got["x"], x1.astype(np.float64))
    assert np.array_equal(got["y"], y1.astype(np.float64))
    dx, dy = lx / nx, ly / ny
    out = (1.0 / scale) * (w * q / (dx * dy))    # the library's read-back factor
    assert np.array_equal(jx, out * ix.astype(np.float64)), np.max(np.abs(jx - out * ix))
    assert np.array_equal(jy, out * iy.astype(np.float64)), np.max(np.abs(jy - out * iy))


@pytest.mark.parametrize("nsteps", [5, 8], ids=["mid-interval", "at-a-sort"])
def test_fused_kernel_deposit_bit_exact_at_full_size(device, nsteps):
    # The 128 x 128 Weibel run the benchmark times (2^20 particles, cubic, BDF-2, sorted
    # every 8 steps): every pic_step call ends with the fused kernel, which pushes the
    # particles and then moves them and deposits the next step's current.  That pending
    # deposit, taken by the next pic_deposit, must be the CPU model's move and current
    # from the state the call left (x^n, v^n read back), bit for bit at every node and
    # particle; at a step that is a multiple of 8 the deposit also sorts.
    from paper_2410_18414_gb300 import workloads
    wl = workloads.weibel_128()
    cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=3, stepper="bdf", bdf_order=2,
                          weight=wl.weight, precision=pic.FP32_FIX64, sort_interval=8)
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=device) as sim:
        sim.step(nsteps)
        st = sim.particles()
        sim.deposit()  # the fused kernel's pending move and current
        jx, jy = sim.field("jx"), sim.field("jy")
        sim.field_solve()
        sim.gather_push()
        moved = sim.particles()
    scale = fx.current_scale(1.0, wl.n)
    x1, y1, ix, iy = fx.move_deposit(st["x"], st["y"], st["vx"], st["vy"], wl.dt, wl.lx, wl.ly,
                                     wl.nx, wl.ny, 3, scale)
    assert np.array_equal(moved["x"], x1.astype(np.float64))
    assert np.array_equal(moved["y"], y1.astype(np.float64))
    out = (1.0 / scale) * (wl.weight * -1.0 / ((wl.lx / wl.nx) * (wl.ly / wl.ny)))
    assert np.array_equal(jx, out * ix.astype(np.float64)), np.max(np.abs(jx - out * ix))
    assert np.array_equal(jy, out * iy.astype(np.float64)), np.max(np.abs(jy - out * iy))
