"""The oracle's pins catch plausible mistakes: each case plants one mistake in
a copy of bpm_oracle.c (on the CPU, in a temporary directory), builds it, and
runs the pin tests against the mutated copy; at least one pin must fail."""
import ctypes
import os
import subprocess
import sys
import types

import pytest

import oracle
import tests.test_oracle_adaptive as t_ada
import tests.test_oracle_absorption as t_abs
import tests.test_oracle_fft as t_fft
import tests.test_oracle_propagation as t_prop
import tests.test_oracle_synthesis as t_syn

SRC = os.path.join(os.path.dirname(oracle.__file__), "bpm_oracle.c")

MUTATIONS = [
    ("screen sign", "e *= cexp(I * k0 * dz_slice[i] * dz);", "e *= cexp(-I * k0 * dz_slice[i] * dz);"),
    ("missing 1/M of the inverse DFT", "cplx e = E[i] / (double)M;", "cplx e = E[i];"),
    ("screen before diffraction", "        oracle_dft2(nx, ny, (double *)E, -1);\n        for (size_t i = 0; i < M; ++i) E[i] *= H[i];",
     "        if (z > 0) for (size_t i = 0; i < M; ++i) E[i] *= cexp(I * k0 * dn[(size_t)(z - 1) * M + i] * dz) / cexp(I * k0 * dn[(size_t)z * M + i] * dz);\n        oracle_dft2(nx, ny, (double *)E, -1);\n        for (size_t i = 0; i < M; ++i) E[i] *= H[i];"),
    ("evanescent tie kept", "H[(size_t)y * nx + x] = (kz2 > 0) ? cexp(I * sqrt(kz2) * dz) : 0;",
     "H[(size_t)y * nx + x] = (kz2 >= 0) ? cexp(I * sqrt(kz2) * dz) : 0;"),
    ("ky from dx", "        double ky = grid_k(y, ny, dy);\n        for (int x = 0; x < nx; ++x) {\n            double kx = grid_k(x, nx, dx);\n            double kz2 = K * K - kx * kx - ky * ky;",
     "        double ky = grid_k(y, ny, dx);\n        for (int x = 0; x < nx; ++x) {\n            double kx = grid_k(x, nx, dx);\n            double kz2 = K * K - kx * kx - ky * ky;"),
    ("paraxial kz", "H[(size_t)y * nx + x] = (kz2 > 0) ? cexp(I * sqrt(kz2) * dz) : 0;",
     "H[(size_t)y * nx + x] = (kz2 > 0) ? cexp(I * (K - (kx * kx + ky * ky) / (2 * K)) * dz) : 0;"),
    ("DFT twiddle sign in the combine step", "acc += t[a] * root_of_unity((long long)a * (k + (long long)b * m), n, sign);",
     "acc += t[a] * root_of_unity((long long)a * (k + (long long)b * m), n, -sign);"),
    ("emitter amplitude", "double amp = sqrt((double)M / (double)n_pupil);", "double amp = sqrt((double)n_pupil / (double)M);"),
    ("defocus sign", "F[i] *= cexp(-I * sqrt(kz2) * zg);", "F[i] *= cexp(I * sqrt(kz2) * zg);"),
    ("pupil radius from K", "if (kp2 >= kin * kin && kp2 <= kna * kna && K * K - kp2 > 0) ++n_pupil;",
     "if (kp2 >= kin * kin && kp2 <= K * K && K * K - kp2 > 0) ++n_pupil;"),
    ("light-sheet waist", "w0 = lambda / (M_PI * NA);", "w0 = lambda / (2 * M_PI * NA);"),
    ("light-sheet centre", "double xc = (double)(nx / 2) * dx;", "double xc = (double)(nx / 2 + 1) * dx;"),
    ("adapted propagator correction sign", "cexp(I * (kz + delta * k0 * k0 * n0 / kz) * dz)",
     "cexp(I * (kz - delta * k0 * k0 * n0 / kz) * dz)"),
    ("absorption sign", "e *= cexp(I * k0 * d_re[i] * dz) * exp(-k0 * d_im[i] * dz);",
     "e *= cexp(I * k0 * d_re[i] * dz) * exp(k0 * d_im[i] * dz);"),
    ("absorption on the amplitude squared", "e *= cexp(I * k0 * d_re[i] * dz) * exp(-k0 * d_im[i] * dz);",
     "e *= cexp(I * k0 * d_re[i] * dz) * exp(-2 * k0 * d_im[i] * dz);"),
    ("adapted screen keeps the mean", "e *= cexp(I * k0 * (slice[i] - delta) * dz);", "e *= cexp(I * k0 * slice[i] * dz);"),
]

PINS = [
    t_fft.test_dft_matches_numpy, t_prop.test_tilted_plane_wave_closed_form, t_prop.test_evanescent_wave_is_cut,
    t_prop.test_exact_tie_at_kz_zero_is_cut, t_prop.test_uniform_index_is_global_phase,
    t_prop.test_gaussian_beam_matches_angular_spectrum_quadrature,
    t_prop.test_screen_acts_after_diffraction_within_a_slice, t_syn.test_multiplex_equals_direct_sum,
    t_syn.test_each_focus_has_unit_energy, t_syn.test_single_focus_forms_at_its_depth_and_position,
    t_syn.test_light_sheet_focus_profile, t_ada.test_zero_mean_slices_give_reading_a,
    t_ada.test_uniform_slices_tilted_plane_wave_closed_forms, t_ada.test_reading_b_beats_reading_a_in_a_uniform_medium,
    t_abs.test_zero_kappa_is_the_lossless_method, t_abs.test_uniform_kappa_follows_beer_lambert,
]


def _mutated_oracle(tmp_path, find, repl, tag):
    src = open(SRC).read()
    assert src.count(find) >= 1, f"mutation site not found: {tag}"
    csrc = tmp_path / "bpm_oracle.c"
    csrc.write_text(src.replace(find, repl, 1))
    lib = tmp_path / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", str(csrc),
                    "-o", str(lib), "-lm"], check=True)
    init = os.path.join(os.path.dirname(SRC), "__init__.py")
    mod = types.ModuleType(f"oracle_mut_{abs(hash(tag))}")
    mod.__file__ = str(tmp_path / "__init__.py")
    sys.modules[mod.__name__] = mod
    code = open(init).read()
    exec(compile(code, init, "exec"), mod.__dict__)
    mod._LIB_PATH = str(lib)
    mod._SRC = str(csrc)
    mod._lib = None
    return mod


@pytest.mark.parametrize("tag,find,repl", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, monkeypatch, tag, find, repl):
    mod = _mutated_oracle(tmp_path, find, repl, tag)
    failed = []
    for pin in PINS:
        for m in (t_fft, t_prop, t_syn, t_ada, t_abs):
            monkeypatch.setattr(m, "oracle", mod)
        try:
            if pin is t_fft.test_dft_matches_numpy:
                pin(64)
            else:
                pin()
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the mutation '{tag}'"
