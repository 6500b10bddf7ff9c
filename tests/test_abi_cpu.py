"""The C ABI library on a host without a GPU: exports, constants, validation.

Nothing here launches a kernel.  The library must load, export every entry
point include/fd.h declares, and reject bad arguments with the documented
status codes before touching the device.
"""
import os
import re
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from conftest import ROOT, cuda_available

HEADER = os.path.join(ROOT, "include", "fd.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^\s*(?:fd_status|double|uint64_t|const\s+char\s*\*)\s*\*?\s*(fd_\w+)\s*\(",
                          text, flags=re.M))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("fd_model_create", "fd_step", "fd_run_shot", "fd_gather_traces", "fd_model_destroy"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(fdlib):
    names = header_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", fdlib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(fd_\w+)$", out, flags=re.M))
    assert names <= exported, names - exported
    assert set(fdlib.EXPORTS) == names


def test_cfl_limit_matches_oracle(fdlib, oracle):
    for d in (2, 3):
        assert fdlib.fd_cfl_limit(d) == pytest.approx(oracle.cfl_limit(d), rel=1e-13)
    assert fdlib.fd_cfl_limit(4) < 0


def test_stencil_weights_are_the_taylor_weights_in_fp32(fdlib, oracle):
    w = fdlib.fd_stencil_weights()
    exact = oracle.taylor_coefficients(4)[1:]
    for got, ex in zip(w, exact):
        # within half an FP32 ulp of the exact rational
        ulp = abs(np.spacing(np.float32(float(ex))))
        assert abs(Fraction(float(got)) - ex) <= Fraction(float(ulp)) / 2


def _desc(fd, **kw):
    base = dict(ndim=2, nx=16, ny=1, nz=12, h=10.0, dt=0.002, sponge_width=0, sponge_R=1e-3)
    base.update(kw)
    return fd.make_desc(**base)


@pytest.mark.parametrize("kw", [dict(ndim=4), dict(ndim=2, ny=3), dict(nx=0), dict(nz=-1), dict(h=0.0),
                                dict(dt=-1.0), dict(dt=float("nan")), dict(sponge_width=-2),
                                dict(sponge_width=4, sponge_R=0.0), dict(sponge_width=4, sponge_R=1.0)])
def test_bad_descriptor_is_einval(fdlib, kw):
    d = _desc(fdlib, **kw)
    n = max(d.nx * d.ny * d.nz, 1)
    with pytest.raises(fdlib.FDError) as e:
        fdlib.fd_model_create(d, np.full(n, 2000.0, np.float32)) if d.nx * d.ny * d.nz > 0 else \
            fdlib._check(fdlib._lib.fd_model_create(fdlib.ctypes.byref(d), None, None,
                                                    fdlib.ctypes.byref(fdlib._vp())), "fd_model_create")
    assert e.value.status == fdlib.FD_EINVAL


@pytest.mark.parametrize("bad", [0.0, -5.0, float("nan"), float("inf")])
def test_bad_velocity_is_einval(fdlib, bad):
    d = _desc(fdlib)
    v = np.full(d.nx * d.nz, 2000.0, np.float32)
    v[7] = bad
    with pytest.raises(fdlib.FDError) as e:
        fdlib.fd_model_create(d, v)
    assert e.value.status == fdlib.FD_EINVAL


def test_unstable_time_step_is_ecfl(fdlib):
    lim = fdlib.fd_cfl_limit(3)
    d = fdlib.make_desc(3, 8, 8, 8, 10.0, 1.01 * lim * 10.0 / 3000.0)
    v = np.full(512, 2000.0, np.float32)
    v[100] = 3000.0
    with pytest.raises(fdlib.FDError) as e:
        fdlib.fd_model_create(d, v)
    assert e.value.status == fdlib.FD_ECFL
    assert "Courant" in fdlib.fd_last_error()


def test_null_arguments_are_einval(fdlib):
    assert fdlib._lib.fd_step(None, 1) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_gather_traces(None, None, 0) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_stencil_weights(None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_model_destroy(None) == fdlib.FD_OK
    assert fdlib._lib.fd_set_stream(None, None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_stream_create(0, None, None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_stream_destroy(None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_set_time_fusion(None, 2) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_velocity_from_slowness(None, None, 4, None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_gradient_from_image(None, 1, None, None, 4, None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_batch_create(None, 0, None) == fdlib.FD_EINVAL


@pytest.mark.skipif(cuda_available(), reason="checks the no-device error path")
def test_no_device_is_ecuda(fdlib):
    with pytest.raises(fdlib.FDError) as e:
        fdlib.fd_model_create(_desc(fdlib), np.full(16 * 12, 2000.0, np.float32))
    assert e.value.status in (fdlib.FD_ECUDA, fdlib.FD_ENOMEM)


def _build_c_example(tmp_path):
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2311_05038_b300")
    exe = str(tmp_path / "example_shot")
    cmd = ["gcc", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
           os.path.join(pkg, "csrc", "example_shot.c"), "-L", pkg, "-lfd", f"-Wl,-rpath,{pkg}", "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_compiles_and_links_against_the_header_alone(fdlib, tmp_path):
    """A C caller needs only include/fd.h and libfd.so (no Python, no torch)."""
    assert os.path.exists(_build_c_example(tmp_path))
