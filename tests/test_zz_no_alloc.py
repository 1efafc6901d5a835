"""The allocation-free move + deposit pass against the regular entry points.

pic_move_deposit_noalloc exists for callers that cannot let the library allocate device
memory (hosts whose GPU memory belongs to their own pool allocator, latency-bound loops
that cannot take cudaMalloc's device-wide synchronisation).  Its scratch is a fixed
array inside the library instead of the simulation handle's buffers, so this test checks
that it computes what pic_init + one step computes for the moved positions and J^{n+1},
on two calls in a row with different particles (the second call must not see the first
call's contents).  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_18414_gb300 import pic, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(pic.LIB_PATH):
        from paper_2410_18414_gb300 import build
        build.build()
    lib = pic.load_library()
    fn = lib.pic_move_deposit_noalloc
    fn.argtypes = ([ctypes.POINTER(pic.PicConfig), ctypes.c_int64] + [ctypes.c_void_p] * 7)
    fn.restype = ctypes.c_int32
    torch.cuda.set_device(0)
    return fn, torch.cuda.current_stream().cuda_stream


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def regular_pass(cfg, wl, stream):
    # pic_init + one step: J^{n+1} and x^{n+1} are final after the deposit phase.
    with pic.Simulation(cfg, wl.x, wl.y, wl.vx, wl.vy, stream=stream) as sim:
        sim.step(1)
        part = sim.particles()
        return part["x"], part["y"], sim.field("jx"), sim.field("jy")


def noalloc_pass(fn, cfg, wl, stream):
    import torch
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(wl, k))).cuda()
           for k in ("x", "y", "vx", "vy")}
    jx = torch.full((cfg.nx, cfg.ny), float("nan"), dtype=torch.float64, device="cuda")
    jy = torch.full((cfg.nx, cfg.ny), float("nan"), dtype=torch.float64, device="cuda")
    st = fn(ctypes.byref(cfg), wl.n, dev["x"].data_ptr(), dev["y"].data_ptr(),
            dev["vx"].data_ptr(), dev["vy"].data_ptr(), jx.data_ptr(), jy.data_ptr(), stream)
    assert st == pic.PIC_OK, st
    return dev["x"].cpu().numpy(), dev["y"].cpu().numpy(), jx.cpu().numpy(), jy.cpu().numpy()


def test_two_calls_match_regular_path(env):
    fn, stream = env
    for seed, p in ((81, 3), (82, 2)):
        wl = workloads.weibel(64, 48, 16, 0.5, 0.01, seed, p, n=64 * 48 * 16 - 5)
        cfg = pic.make_config(wl.nx, wl.ny, wl.lx, wl.ly, wl.dt, p=p, stepper="bdf",
                              bdf_order=2, weight=wl.weight)
        x_r, y_r, jx_r, jy_r = regular_pass(cfg, wl, stream)
        x_n, y_n, jx_n, jy_n = noalloc_pass(fn, cfg, wl, stream)
        np.testing.assert_array_equal(x_n, x_r)
        np.testing.assert_array_equal(y_n, y_r)
        assert rel(jx_n, jx_r) <= TOL and rel(jy_n, jy_r) <= TOL, (rel(jx_n, jx_r), rel(jy_n, jy_r))


def test_rejects_grid_above_limit(env):
    fn, stream = env
    cfg = pic.make_config(1024, 512, 1.0, 1.0, 0.001, p=2)
    z = np.zeros(1)
    st = fn(ctypes.byref(cfg), 1, z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
            z.ctypes.data, z.ctypes.data, stream)
    assert st == 1
