"""The oracle's pins have teeth: planted mistakes in the oracle fail them (CPU only).

Each case copies ``oracle/fd_oracle.c``, plants one plausible mistake (a dropped
axis, a wrong sign, a shifted index, a wrong scaling, a wrong time level, a
wrong boundary), compiles the copy, loads it into a private copy of the oracle
module and runs the pins.  At least one pin must fail for every mutant.
"""
import ctypes
import importlib.util
import os
import subprocess

import pytest

import test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fd_oracle.c")

MUTANTS = {
    "drop_y_axis": ("if (ndim == 3) {", "if (ndim == 4) {"),
    "sponge_sign": ("(1.0 - a) * Pold[i]", "(1.0 + a) * Pold[i]"),
    "source_one_step_late": ("wavelet[n] / hd", "wavelet[n > 0 ? n - 1 : 0] / hd"),
    "source_scaled_by_h2": ("wavelet[n] / hd", "wavelet[n] / (h * h)"),
    "stencil_index_shift": ("ix - k, iy, iz));", "ix - k + 1, iy, iz));"),
    "traces_record_old_level": ("traces[(long)s * nrec + r] = Pn[", "traces[(long)s * nrec + r] = P["),
    "clamped_boundary": ("        return 0.0;",
                         "        return P[((iz < 0 ? 0 : iz >= nz ? nz - 1 : iz) * ny"
                         " + (iy < 0 ? 0 : iy >= ny ? ny - 1 : iy)) * nx"
                         " + (ix < 0 ? 0 : ix >= nx ? nx - 1 : ix)];"),
    "centre_term_once": ("    /* z axis */\n    sum += c[0] * centre;", "    /* z axis */"),
}

# pins that take the oracle module as their only argument
PIN_FUNCS = [
    pins.test_operator_is_eighth_order,
    pins.test_operator_is_axis_symmetric_3d,
    pins.test_energy_identity_with_sponge,
    pins.test_green_function_3d,
    pins.test_green_function_2d_and_refinement,
    pins.test_sponge_absorbs_outgoing_wave,
    lambda o: pins.test_energy_is_conserved_without_sponge(o, (14, 12, 18)),
    lambda o: pins.test_reciprocity(o, 3, 4),
    lambda o: pins.test_dense_matrix_brute_force(o, (9, 11), 3),
    lambda o: pins.test_dense_matrix_brute_force(o, (7, 9, 11), 2),
]


def _mutant_module(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) >= 1, f"anchor for {name} not found"
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new, 1))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(src)], check=True)
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}",
                                                  os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._lib = mod._configure(ctypes.CDLL(str(lib)))
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    mod = _mutant_module(tmp_path, name, old, new)
    failed = []
    for fn in PIN_FUNCS:
        try:
            fn(mod)
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(getattr(fn, "__name__", "lambda"))
            break
    assert failed, f"no pin caught mutant {name}"
