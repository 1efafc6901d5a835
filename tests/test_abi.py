"""C ABI checks that need no GPU: the library builds, loads, exports every entry
point include/pic.h declares, mirrors its struct layouts, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_2410_18414_gb300 import pic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pic.LIB_PATH):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("libgpic.so not built and no nvcc to build it")
        from paper_2410_18414_gb300 import build
        build.build()
    return pic.load_library()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(pic_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert "pic_init" in decl and "pic_step" in decl
    out = subprocess.run(["nm", "-D", "--defined-only", pic.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pic_\w+)", out))
    missing = [n for n in decl if n not in exported]
    assert not missing, missing
    for n in decl:
        assert getattr(lib, n) is not None


def test_struct_layout_matches_header(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
        "int main(){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(pic_config),"
        " offsetof(pic_config, lx), offsetof(pic_config, dirk_a), offsetof(pic_config, reserved),"
        " sizeof(pic_diagnostics), sizeof(pic_particles_in), offsetof(pic_diagnostics, step),"
        " offsetof(pic_config, charge)); printf(\"%zu\\n\", sizeof(pic_particles_bound));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                             check=True).stdout.split()]
    py_vals = [ctypes.sizeof(pic.PicConfig), pic.PicConfig.lx.offset, pic.PicConfig.dirk_a.offset,
               pic.PicConfig.reserved.offset, ctypes.sizeof(pic.PicDiagnostics),
               ctypes.sizeof(pic.PicParticlesIn), pic.PicDiagnostics.step.offset,
               pic.PicConfig.charge.offset, ctypes.sizeof(pic.PicParticlesBound)]
    assert c_vals == py_vals


def _bad(lib, **kw):
    base = dict(nx=16, ny=16, lx=1.0, ly=1.0, dt=0.01, p=2, stepper="bdf", bdf_order=2)
    base.update(kw)
    x = np.zeros(4)
    with pytest.raises(pic.PicError) as e:
        pic.Simulation(pic.make_config(**base), x, x, x, x)
    return e.value


@pytest.mark.parametrize("kw", [
    dict(nx=7), dict(nx=10), dict(ny=2048), dict(nx=14), dict(p=5), dict(p=1), dict(dt=-1.0),
    dict(dt=2.0), dict(bdf_order=7), dict(bdf_order=0), dict(stepper=9), dict(lx=float("nan")),
    dict(stepper="dirk"),  # zero stages
    dict(charge=2), dict(tile=3), dict(tile=32), dict(tile=-4),
])
def test_invalid_config_is_rejected_without_a_device(lib, kw):
    err = _bad(lib, **kw)
    assert err.status == 1, err


@pytest.mark.parametrize("stepper", ["cdf2", "cdf2_semi", "cdf2_explicit"])
def test_deposited_charge_with_cdf2_is_unsupported(lib, stepper):
    # CDF-2 keeps its charge at half levels; a deposit at x^{n+1} has no place there
    assert _bad(lib, stepper=stepper, charge=pic.CHARGE_DEPOSIT).status == 2


def test_upper_triangular_dirk_rejected(lib):
    tab = {"A": [[0.25, 0.1], [0.5, 0.25]], "b": [0.5, 0.5], "c": [0.25, 0.75]}
    assert _bad(lib, stepper="dirk", dirk=tab).status == 1


def test_null_particle_arrays_rejected(lib):
    cfg = pic.make_config(16, 16, 1.0, 1.0, 0.01)
    init = pic.PicParticlesIn(None, None, None, None, 5)
    h = ctypes.c_void_p()
    st = lib.pic_init(ctypes.byref(cfg), ctypes.byref(init), None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"NULL" in lib.pic_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.pic_step(None, 1) == 1
    assert lib.pic_sync(None) == 1
    assert lib.pic_step_count(None) == -1
    assert lib.pic_set_kernel_timing(None, 8) == 1
    out = ctypes.c_void_p()
    assert lib.pic_ensemble_create(None, 1, ctypes.c_void_p(1), ctypes.byref(out)) == 1
    runs = (ctypes.c_void_p * 1)(None)
    assert lib.pic_ensemble_create(runs, 1, ctypes.c_void_p(1), ctypes.byref(out)) == 1
    assert b"NULL" in lib.pic_last_error(None)
    assert lib.pic_ensemble_step(None, 0) == 1
    assert lib.pic_ensemble_period(None) == 0
    lib.pic_ensemble_destroy(None)
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert lib.pic_kernel_time(None, 0, ctypes.byref(ms), ctypes.byref(n)) == 1
    adj = ctypes.c_void_p()
    assert lib.pic_adjoint_create(None, 10, 5, ctypes.byref(adj)) == 1
    assert not adj.value
    assert lib.pic_adjoint_forward(None) == 1
    assert lib.pic_adjoint_backward(None, None, None, None, None, None, None, None) == 1
    assert lib.pic_adjoint_checkpoint_every(None) == 0
    lib.pic_adjoint_destroy(None)
    size = ctypes.c_size_t(0)
    assert lib.pic_save_state(None, None, ctypes.byref(size)) == 1
    assert lib.pic_load_state(None, None, 0) == 1
    count = ctypes.c_int32(7)
    assert lib.pic_diagnostics_history(None, None, 0, ctypes.byref(count)) == 1
    assert lib.pic_diagnostics_history(None, None, 0, None) == 1
    lib.pic_destroy(None)


def test_3v_and_species_configs_are_validated_without_a_device(lib):
    x = np.zeros(4)
    sp = np.zeros(4, dtype=np.int32)

    def status(cfg, **kw):
        with pytest.raises(pic.PicError) as e:
            pic.Simulation(cfg, x, x, x, x, **kw)
        return e.value.status

    base = dict(nx=16, ny=16, lx=1.0, ly=1.0, dt=0.01, p=2, stepper="bdf", bdf_order=2)
    assert status(pic.make_config(**base, vdim=4)) == 1
    assert status(pic.make_config(**base, vdim=3)) == 1                  # no z velocities
    assert status(pic.make_config(**base, species=((-1.0, 1.0, 1.0),))) == 1   # no indices
    assert status(pic.make_config(**base, species=((-1.0, 0.0, 1.0),)), species=sp) == 1
    assert status(pic.make_config(**base, species=((-1.0, 1.0, -1.0),)), species=sp) == 1
    cfg = pic.make_config(**base)
    cfg.nspecies = 5
    assert status(cfg) == 1


def test_new_struct_fields_match_header(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    src = tmp_path / "layout2.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
        "int main(){printf(\"%zu %zu %zu %zu %zu %zu\\n\", offsetof(pic_config, vdim),"
        " offsetof(pic_config, nspecies), offsetof(pic_config, species_q),"
        " offsetof(pic_config, species_w), offsetof(pic_particles_in, vz),"
        " offsetof(pic_particles_in, species));return 0;}\n")
    exe = tmp_path / "layout2"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                             check=True).stdout.split()]
    assert c_vals == [pic.PicConfig.vdim.offset, pic.PicConfig.nspecies.offset,
                      pic.PicConfig.species_q.offset, pic.PicConfig.species_w.offset,
                      pic.PicParticlesIn.vz.offset, pic.PicParticlesIn.species.offset]


def test_bound_arrays_rejected_without_a_device(lib):
    # pic_init_bound checks its configuration and arrays before any device work: sorted,
    # 2D-3V and species configurations are unsupported, NULL and host arrays refused
    base = dict(nx=16, ny=16, lx=1.0, ly=1.0, dt=0.01, p=2, stepper="bdf", bdf_order=2)
    x = np.zeros(4)
    host = pic.PicParticlesBound(*([x.ctypes.data] * 8), 4)
    nulls = pic.PicParticlesBound(*([None] * 8), 4)

    def status(cfg, desc):
        h = ctypes.c_void_p()
        return lib.pic_init_bound(ctypes.byref(cfg), ctypes.byref(desc), None, ctypes.byref(h))

    assert status(pic.make_config(**base, sort_interval=4), host) == 2
    assert status(pic.make_config(**base, vdim=3), host) == 2
    assert status(pic.make_config(**base, species=((-1.0, 1.0, 1.0),)), host) == 2
    assert status(pic.make_config(**base), nulls) == 1
    assert status(pic.make_config(**base), host) == 1
    assert lib.pic_velocity_slot(None) == -1
