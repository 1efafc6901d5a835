"""Python binding of the C ABI in include/pic.h (argument marshalling only).

Every step of the PIC method runs inside libgpic.so's CUDA kernels; this module only
loads the library, mirrors its structs with ctypes and turns status codes into
exceptions.  It never computes anything of the method itself, and it refuses to run
without the compiled library (there is no CPU fallback).

Arrays may be numpy (host) or torch tensors (host or CUDA): the library's copies use
unified addressing, so a device pointer and a host pointer are both accepted.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the in-tree build; GPIC_LIB names another build of the same library (the host-sanitizer
# build libgpic_asan.so, say)
LIB_PATH = os.environ.get("GPIC_LIB") or os.path.join(_HERE, "libgpic.so")

# pic_status
PIC_OK = 0
STATUS_NAMES = {0: "PIC_OK", 1: "PIC_ERR_INVALID_ARG", 2: "PIC_ERR_UNSUPPORTED", 3: "PIC_ERR_CUDA",
                4: "PIC_ERR_NONFINITE", 5: "PIC_ERR_OVERFLOW", 6: "PIC_ERR_TIMEOUT",
                7: "PIC_ERR_STATE"}
# pic_stepper
STEPPER_BDF, STEPPER_CDF2, STEPPER_DIRK = 0, 1, 2
STEPPER_CDF2_SEMI, STEPPER_CDF2_EXPLICIT = 3, 4
STEPPERS = {"bdf": STEPPER_BDF, "cdf2": STEPPER_CDF2, "dirk": STEPPER_DIRK,
            "cdf2_semi": STEPPER_CDF2_SEMI, "cdf2_explicit": STEPPER_CDF2_EXPLICIT}
# pic_precision
FP64, FP32_FIX64 = 0, 1
# pic_field
FIELDS = {"jx": 0, "jy": 1, "rho": 2, "phi": 3, "ax": 4, "ay": 5, "bz": 6, "ex": 7, "ey": 8,
          "dphidx": 9, "dphidy": 10, "gax": 11, "gay": 12, "daxdx": 13, "daxdy": 14,
          "daydx": 15, "daydy": 16,
          "jz": 17, "az": 18, "bx": 19, "by": 20, "dazdx": 21, "dazdy": 22}
KERNEL_TIMERS = {"sort": 0, "deposit": 1, "field_solve": 2, "gather_push": 3,
                 "adj_push": 4, "adj_field": 5, "adj_deposit": 6, "gather_deposit": 7}


class PicError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("spline_order", ctypes.c_int32), ("stepper", ctypes.c_int32),
        ("bdf_order", ctypes.c_int32), ("dirk_stages", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("sort_interval", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("c", ctypes.c_double), ("eps0", ctypes.c_double), ("dt", ctypes.c_double),
        ("q", ctypes.c_double), ("m", ctypes.c_double), ("weight", ctypes.c_double),
        ("dirk_a", ctypes.c_double * 16), ("dirk_b", ctypes.c_double * 4),
        ("dirk_c", ctypes.c_double * 4),
        ("charge", ctypes.c_int32),
        ("vdim", ctypes.c_int32), ("nspecies", ctypes.c_int32),
        ("tile", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4),
        ("species_q", ctypes.c_double * 4), ("species_m", ctypes.c_double * 4),
        ("species_w", ctypes.c_double * 4),
    ]


class PicParticlesIn(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("vx", ctypes.c_void_p),
                ("vy", ctypes.c_void_p), ("n", ctypes.c_int64), ("vz", ctypes.c_void_p),
                ("species", ctypes.c_void_p)]


class PicParticlesBound(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("x", "y", "px", "py", "vx", "vy", "vx_old",
                                               "vy_old")] + [("n", ctypes.c_int64)]


DIAG_HISTORY = 4096  # PIC_DIAG_HISTORY: records the device ring holds


class PicDiagnostics(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in
                ("gauge_rms", "gauss_rms", "continuity_rms", "gauge_dt_rms", "rho_rms",
                 "div_a_rms", "w_e", "w_b", "kinetic")] + [("step", ctypes.c_int64)]


EXPORTS = ("pic_init", "pic_deposit", "pic_field_solve", "pic_gather_push", "pic_step",
           "pic_set_diagnostics", "pic_residuals", "pic_get_field", "pic_read_particles",
           "pic_sync", "pic_step_count", "pic_kernels_per_step", "pic_last_error", "pic_destroy")

_lib = None


def load_library(path=None):
    """Load libgpic.so (once; path defaults to LIB_PATH).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgpic.so not found at {path}: build it with "
                           "`python -m paper_2410_18414_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "pic_init": ([ctypes.POINTER(PicConfig), ctypes.POINTER(PicParticlesIn), vp,
                      ctypes.POINTER(vp)], i32),
        "pic_init_bound": ([ctypes.POINTER(PicConfig), ctypes.POINTER(PicParticlesBound), vp,
                            ctypes.POINTER(vp)], i32),
        "pic_velocity_slot": ([vp], i32),
        "pic_deposit": ([vp], i32),
        "pic_field_solve": ([vp], i32),
        "pic_gather_push": ([vp], i32),
        "pic_step": ([vp, i32], i32),
        "pic_set_diagnostics": ([vp, i32], i32),
        "pic_residuals": ([vp, ctypes.POINTER(PicDiagnostics)], i32),
        "pic_diagnostics_history": ([vp, ctypes.POINTER(PicDiagnostics), i32,
                                     ctypes.POINTER(i32)], i32),
        "pic_get_field": ([vp, i32, vp], i32),
        "pic_read_particles": ([vp] + [vp] * 8, i32),
        "pic_read_particles_z": ([vp] + [vp] * 4, i32),
        "pic_save_state": ([vp, vp, ctypes.POINTER(ctypes.c_size_t)], i32),
        "pic_load_state": ([vp, vp, ctypes.c_size_t], i32),
        "pic_sync": ([vp], i32),
        "pic_step_count": ([vp], i64),
        "pic_kernels_per_step": ([vp], i32),
        "pic_set_kernel_timing": ([vp, i32], i32),
        "pic_kernel_time": ([vp, i32, dp, ctypes.POINTER(i64)], i32),
        "pic_ensemble_create": ([ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)], i32),
        "pic_ensemble_step": ([vp, i32], i32),
        "pic_ensemble_period": ([vp], i32),
        "pic_ensemble_destroy": ([vp], None),
        "pic_adjoint_create": ([vp, i32, i32, ctypes.POINTER(vp)], i32),
        "pic_adjoint_create_ex": ([vp, i32, i32, i32, ctypes.POINTER(vp)], i32),
        "pic_adjoint_forward": ([vp], i32),
        "pic_adjoint_backward": ([vp] + [vp] * 7, i32),
        "pic_adjoint_checkpoint_every": ([vp], i32),
        "pic_adjoint_destroy": ([vp], None),
        "pic_measure_fp64_fma": ([vp, dp], i32),
        "pic_last_error": ([vp], ctypes.c_char_p),
        "pic_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    del dp
    _lib = lib
    return lib


def _ptr(a, kind="float64"):
    """Raw address of a numpy array or torch tensor (contiguous float64, or int32)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(kind) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"arrays must be contiguous {kind}")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != getattr(torch, kind) or not a.is_contiguous():
            raise TypeError(f"tensors must be contiguous {kind}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


CHARGE_CONTINUITY, CHARGE_DEPOSIT = 0, 1


def make_config(nx, ny, lx, ly, dt, p=2, stepper="bdf", bdf_order=1, dirk=None, c=1.0, eps0=1.0,
                q=-1.0, m=1.0, weight=1.0, precision=FP64, sort_interval=0,
                charge=CHARGE_CONTINUITY, vdim=2, species=None, tile=0):
    """species: optional ((q, m, w), ...) per species (at most 4); particles then carry a
    species index (Simulation(..., species=...)).  tile: the sorted form's tile width T
    (4, 8 or 16; 0 = chosen from the particle density)."""
    cfg = PicConfig()
    cfg.nx, cfg.ny, cfg.lx, cfg.ly, cfg.dt = nx, ny, lx, ly, dt
    cfg.spline_order = p
    cfg.stepper = STEPPERS[stepper] if isinstance(stepper, str) else int(stepper)
    cfg.bdf_order = bdf_order
    cfg.c, cfg.eps0, cfg.q, cfg.m, cfg.weight = c, eps0, q, m, weight
    cfg.precision = precision
    cfg.sort_interval = sort_interval
    cfg.tile = tile
    cfg.charge = charge
    cfg.vdim = vdim
    if species is not None:
        cfg.nspecies = len(species)
        for i, (qs, ms, ws) in enumerate(species):
            cfg.species_q[i], cfg.species_m[i], cfg.species_w[i] = qs, ms, ws
    if dirk is not None:
        s = len(dirk["b"])
        cfg.dirk_stages = s
        for i in range(s):
            for j in range(s):
                cfg.dirk_a[i * s + j] = dirk["A"][i][j]
            cfg.dirk_b[i] = dirk["b"][i]
            cfg.dirk_c[i] = dirk["c"][i]
    return cfg


def measure_fp64_fma(stream=None):
    """The current device's FP64 FMA rate in GFLOP/s (pic_measure_fp64_fma)."""
    lib = load_library()
    out = ctypes.c_double()
    st = lib.pic_measure_fp64_fma(ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if st != PIC_OK:
        raise PicError(st, "pic_measure_fp64_fma failed")
    return out.value


class Simulation:
    """One simulation handle of libgpic (owns its device memory until close())."""

    def __init__(self, cfg, x, y, vx, vy, stream=None, vz=None, species=None):
        """vz: z velocities (2D-3V, cfg.vdim = 3); species: int32 species indices (a config
        with a species table)."""
        self.lib = load_library()
        self.cfg = cfg
        self.n = len(x)
        self._keep = (x, y, vx, vy, vz, species)
        init = PicParticlesIn(_ptr(x), _ptr(y), _ptr(vx), _ptr(vy), self.n, _ptr(vz),
                              _ptr(species, "int32"))
        handle = ctypes.c_void_p()
        st = self.lib.pic_init(ctypes.byref(cfg), ctypes.byref(init),
                               ctypes.c_void_p(stream or 0), ctypes.byref(handle))
        if st != PIC_OK:
            raise PicError(st, self.lib.pic_last_error(None).decode())
        self.h = handle
        self._keep = None

    BOUND_KEYS = ("x", "y", "px", "py", "vx", "vy", "vx_old", "vy_old")

    @classmethod
    def bound(cls, cfg, arrays, stream=None):
        """A simulation that steps the caller's CUDA tensors in place (pic_init_bound):
        `arrays` maps BOUND_KEYS to contiguous CUDA tensors of n values (float64, or
        float32 for the FP32 form); x, y, vx, vy hold x^0 and v^0.  The tensors must live
        as long as the simulation (it keeps references).  velocities() names the pair that
        holds v^n after each step."""
        import torch
        sim = cls.__new__(cls)
        sim.lib = load_library()
        sim.cfg = cfg
        dtype = torch.float32 if cfg.precision == FP32_FIX64 else torch.float64
        n = arrays["x"].numel()
        for k in cls.BOUND_KEYS:
            t = arrays[k]
            if t.dtype != dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise TypeError(f"{k}: a contiguous CUDA {dtype} tensor of {n} values")
        sim.n = n
        sim.arrays = dict(arrays)
        desc = PicParticlesBound(*[arrays[k].data_ptr() for k in cls.BOUND_KEYS], n)
        handle = ctypes.c_void_p()
        st = sim.lib.pic_init_bound(ctypes.byref(cfg), ctypes.byref(desc),
                                    ctypes.c_void_p(stream or 0), ctypes.byref(handle))
        if st != PIC_OK:
            raise PicError(st, sim.lib.pic_last_error(None).decode())
        sim.h = handle
        sim._keep = None
        return sim

    @property
    def velocity_slot(self):
        """0 while (vx, vy) hold v^n, 1 while (vx_old, vy_old) do (pic_velocity_slot)."""
        return int(self.lib.pic_velocity_slot(self.h))

    def velocities(self):
        """Bound simulations: ((vx^n, vy^n), (vx^{n-1}, vy^{n-1})) as the caller's tensors."""
        a = self.arrays
        now, old = (("vx", "vy"), ("vx_old", "vy_old"))
        if self.velocity_slot:
            now, old = old, now
        return (a[now[0]], a[now[1]]), (a[old[0]], a[old[1]])

    def _check(self, st):
        if st != PIC_OK:
            raise PicError(st, self.lib.pic_last_error(self.h).decode())

    def deposit(self):
        self._check(self.lib.pic_deposit(self.h))

    def field_solve(self):
        self._check(self.lib.pic_field_solve(self.h))

    def gather_push(self):
        self._check(self.lib.pic_gather_push(self.h))

    def step(self, nsteps=1):
        self._check(self.lib.pic_step(self.h, nsteps))

    def set_diagnostics(self, every):
        self._check(self.lib.pic_set_diagnostics(self.h, every))

    def residuals(self):
        d = PicDiagnostics()
        self._check(self.lib.pic_residuals(self.h, ctypes.byref(d)))
        return {name: getattr(d, name) for name, _ in PicDiagnostics._fields_}

    def diagnostics_history(self, capacity=DIAG_HISTORY):
        """The diagnostics of every step diagnosed since the previous call (or since
        set_diagnostics), oldest first, as a list of dicts like residuals()."""
        buf = (PicDiagnostics * max(1, capacity))()
        count = ctypes.c_int32(0)
        self._check(self.lib.pic_diagnostics_history(self.h, buf, capacity, ctypes.byref(count)))
        return [{name: getattr(buf[i], name) for name, _ in PicDiagnostics._fields_}
                for i in range(count.value)]

    def field(self, name, out=None):
        if out is None:
            out = np.empty((self.cfg.nx, self.cfg.ny), dtype=np.float64)
        self._check(self.lib.pic_get_field(self.h, FIELDS[name], ctypes.c_void_p(_ptr(out))))
        return out

    def particles(self, out=None):
        """Dict of the eight particle arrays (x, y, px, py, vx, vy, vx_old, vy_old), FP64;
        in 2D-3V also pz, vz, vz_old, and with a species table the species indices."""
        names = ("x", "y", "px", "py", "vx", "vy", "vx_old", "vy_old")
        if out is None:
            out = {k: np.empty(self.n, dtype=np.float64) for k in names}
        ptrs = [ctypes.c_void_p(_ptr(out[k])) if out.get(k) is not None else None for k in names]
        self._check(self.lib.pic_read_particles(self.h, *ptrs))
        three = self.cfg.vdim == 3
        table = self.cfg.nspecies > 0
        if three or table:
            z = {}
            if three:
                z = {k: out.get(k, np.empty(self.n, dtype=np.float64))
                     for k in ("pz", "vz", "vz_old")}
            if table:
                z["species"] = out.get("species", np.empty(self.n, dtype=np.int32))
            ptrs = [ctypes.c_void_p(_ptr(z[k])) if k in z else None
                    for k in ("pz", "vz", "vz_old")]
            ptrs.append(ctypes.c_void_p(_ptr(z["species"], "int32")) if table else None)
            self._check(self.lib.pic_read_particles_z(self.h, *ptrs))
            out.update(z)
        return out

    def save_state(self):
        """The handle's state as bytes (pic_save_state)."""
        size = ctypes.c_size_t(0)
        self._check(self.lib.pic_save_state(self.h, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        self._check(self.lib.pic_save_state(self.h, buf, ctypes.byref(size)))
        return buf.raw[:size.value]

    def load_state(self, state):
        """Restore bytes from save_state of a handle with the same configuration."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        self._check(self.lib.pic_load_state(self.h, buf, len(state)))

    def sync(self):
        self._check(self.lib.pic_sync(self.h))

    @property
    def step_count(self):
        return int(self.lib.pic_step_count(self.h))

    @property
    def kernels_per_step(self):
        return int(self.lib.pic_kernels_per_step(self.h))

    def set_kernel_timing(self, max_launches):
        """Start (max_launches > 0) or stop (0) the library's per-kernel event timers."""
        self._check(self.lib.pic_set_kernel_timing(self.h, max_launches))

    def kernel_time(self, which):
        """(total milliseconds, timed launches) of timer `which` (see KERNEL_TIMERS)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.pic_kernel_time(self.h, KERNEL_TIMERS[which], ctypes.byref(ms),
                                             ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Ensemble:
    """Independent runs advanced together by one CUDA-graph launch per period
    (pic_ensemble_*).  `sims`: Simulation objects, each best on a stream of its own;
    `stream`: the stream the graph is launched on (a CUDA stream handle, not 0)."""

    def __init__(self, sims, stream):
        self.lib = load_library()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.h for s in self.sims])
        e = ctypes.c_void_p()
        st = self.lib.pic_ensemble_create(arr, len(self.sims), ctypes.c_void_p(stream),
                                          ctypes.byref(e))
        if st != PIC_OK:
            raise PicError(st, self.lib.pic_last_error(None).decode())
        self.e = e

    @property
    def period(self):
        return int(self.lib.pic_ensemble_period(self.e))

    def step(self, nsteps):
        st = self.lib.pic_ensemble_step(self.e, nsteps)
        if st != PIC_OK:
            raise PicError(st, self.lib.pic_last_error(None).decode())

    def close(self):
        if getattr(self, "e", None):
            self.lib.pic_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()



class Adjoint:
    """Discrete adjoint of the next `nsteps` steps of a fresh unsorted Simulation (either
    precision, any stepper) (pic_adjoint_*): run forward() once, then backward(...) for the
    gradient of
    J = sum bz_bar B_z + sum (px_bar Px + py_bar Py) of the final state with respect to
    v^0 and, with P^0 = gamma m v^0 independent, to P^0.  Seeds and results are CUDA
    float64 tensors (the library reads and writes device memory)."""

    MODES = {"replay": 0, "recompute": 1, "replay_lean": 2}

    def __init__(self, sim, nsteps, checkpoint_every=None, mode="replay"):
        """mode "replay": the forward pass keeps every step's gathered fields and the backward
        pass replays particle states between checkpoints; "replay_lean": the same with per
        particle only P and v kept (the reverse push gathers the fields again);
        "recompute": it re-runs each segment's full steps (least memory)."""
        self.lib = load_library()
        self.sim = sim
        self.nsteps = int(nsteps)
        a = ctypes.c_void_p()
        k = self.nsteps if checkpoint_every is None else int(checkpoint_every)
        st = self.lib.pic_adjoint_create_ex(sim.h, self.nsteps, k, self.MODES[mode],
                                            ctypes.byref(a))
        if st != PIC_OK:
            raise PicError(st, self.lib.pic_last_error(sim.h).decode())
        self.a = a

    @property
    def checkpoint_every(self):
        return int(self.lib.pic_adjoint_checkpoint_every(self.a))

    def _check(self, st):
        if st != PIC_OK:
            raise PicError(st, self.lib.pic_last_error(self.sim.h).decode())

    def forward(self):
        self._check(self.lib.pic_adjoint_forward(self.a))

    def backward(self, bz_bar=None, px_bar=None, py_bar=None, out=None):
        """Dict of CUDA tensors "vx", "vy" (dJ/dv^0) and "px", "py" (dJ/dP^0)."""
        import torch
        n = self.sim.n
        if out is None:
            out = {k: torch.empty(n, dtype=torch.float64, device="cuda")
                   for k in ("vx", "vy", "px", "py")}
        for t in (bz_bar, px_bar, py_bar, *out.values()):
            if t is not None and not (hasattr(t, "is_cuda") and t.is_cuda):
                raise TypeError("adjoint seeds and outputs must be CUDA float64 tensors")
        vp = ctypes.c_void_p
        args = [vp(_ptr(t)) if t is not None else None
                for t in (bz_bar, px_bar, py_bar, out.get("vx"), out.get("vy"),
                          out.get("px"), out.get("py"))]
        self._check(self.lib.pic_adjoint_backward(self.a, *args))
        return out

    def close(self):
        if getattr(self, "a", None):
            self.lib.pic_adjoint_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
