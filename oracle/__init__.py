"""FP64 CPU oracle for split-step beam propagation (test infrastructure only).

This package is the slow, plainly written reference that the CUDA library is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never does, and the
two share no code.

Every function follows the Biobeam paper (Weigert, Myers & Kreysing,
arXiv:1706.02261): the method paragraph (beam-propagation model with the exact
propagator, the refractive-index phase screen, multiplexed focused input
fields), and the light-sheet paragraph (the excitation is |E|^2 at every
voxel).  The arithmetic lives in ``bpm_oracle.c`` (compiled with gcc into
``liboracle.so``); :mod:`oracle.mie` holds the scalar Mie series used to check
the physics of a single sphere.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (brute-force DFT, closed forms for plane and tilted
waves, the semigroup property, Parseval / energy, an independent angular-
spectrum quadrature for a Gaussian beam, a direct sum for the multiplexed
synthesis, and the scalar Mie series as a physics report).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bpm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``bpm_oracle.c`` into ``liboracle.so`` with gcc (FP64, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
               "-Wall", _SRC, "-o", _LIB_PATH, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.oracle_dft1.argtypes = [i, p, i]
        lib.oracle_dft2.argtypes = [i, i, p, i]
        lib.oracle_propagator.argtypes = [i, i, d, d, d, d, d, p]
        lib.oracle_bpm.argtypes = [i, i, i, d, d, d, d, d, p, p, p, p]
        lib.oracle_bpm_adaptive.argtypes = [i, i, i, d, d, d, d, d, p, p, p, p]
        lib.oracle_bpm_absorbing.argtypes = [i, i, i, d, d, d, d, d, p, p, p, p, p]
        lib.oracle_multiplex_psf.argtypes = [i, i, d, d, d, d, i, p, p, p, p, d, p]
        lib.oracle_multiplex_annular.argtypes = [i, i, d, d, d, d, i, p, p, p, p, d, d, p]
        lib.oracle_light_sheet.argtypes = [i, i, d, d, d, d, d, d, p]
        for f in (lib.oracle_dft1, lib.oracle_dft2, lib.oracle_propagator, lib.oracle_bpm, lib.oracle_bpm_adaptive,
                  lib.oracle_bpm_absorbing,
                  lib.oracle_multiplex_psf, lib.oracle_multiplex_annular, lib.oracle_light_sheet):
            f.restype = i
        lib.oracle_num_threads.restype = i
        _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def num_threads() -> int:
    """OpenMP threads the oracle uses on this host."""
    return int(_load().oracle_num_threads())


def dft(x, sign: int = -1) -> np.ndarray:
    """Unnormalised 1D DFT, sum_j x[j] exp(sign 2 pi i j k / n)."""
    a = _c128(x).copy()
    _check(_load().oracle_dft1(a.size, _ptr(a), int(sign)), "dft")
    return a


def dft2(x, sign: int = -1) -> np.ndarray:
    """Unnormalised 2D DFT of a row-major [ny][nx] array."""
    a = _c128(x).copy()
    ny, nx = a.shape
    _check(_load().oracle_dft2(nx, ny, _ptr(a), int(sign)), "dft2")
    return a


def propagator(nx, ny, dx, dy, dz, lam, n0) -> np.ndarray:
    """Exact one-slice propagator exp(i kz dz), zero where kz^2 <= 0 (full kz)."""
    H = np.zeros((ny, nx), np.complex128)
    _check(_load().oracle_propagator(nx, ny, dx, dy, dz, lam, n0, _ptr(H)), "propagator")
    return H


def bpm(dn, E0, dx, dy, dz, lam, n0, want_intensity: bool = True, adaptive: bool = False, kappa=None):
    """Split-step BPM through every slice of ``dn`` ([nz][ny][nx], n - n0).

    Returns ``(E_out, I)`` where ``I`` is the [nz][ny][nx] volume of |E|^2 after
    each slice's screen (``None`` when ``want_intensity`` is false).  With
    ``adaptive`` the locally adapted expansion of reading B (per-slice mean
    index as the reference, first-order corrected propagator) is used.  With
    ``kappa`` (same shape as ``dn``) the index is complex, n0 + dn + i kappa,
    and each screen also attenuates by exp(-k0 kappa dz).
    """
    dn = np.ascontiguousarray(dn, dtype=np.float64)
    nz, ny, nx = dn.shape
    E0 = _c128(E0)
    assert E0.shape == (ny, nx)
    Eout = np.zeros((ny, nx), np.complex128)
    I = np.zeros((nz, ny, nx), np.float64) if want_intensity else None
    if kappa is not None:
        assert not adaptive, "the oracle has no adapted expansion with absorption"
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        assert kappa.shape == dn.shape
        rc = _load().oracle_bpm_absorbing(nx, ny, nz, dx, dy, dz, lam, n0, _ptr(dn), _ptr(kappa), _ptr(E0),
                                          _ptr(Eout), _ptr(I) if I is not None else None)
    else:
        fn = _load().oracle_bpm_adaptive if adaptive else _load().oracle_bpm
        rc = fn(nx, ny, nz, dx, dy, dz, lam, n0, _ptr(dn), _ptr(E0), _ptr(Eout), _ptr(I) if I is not None else None)
    _check(rc, "bpm")
    return Eout, I


def multiplex_psf(nx, ny, dx, dy, lam, n0, ix, iy, phase, zf, NA) -> np.ndarray:
    """Sum of focused fields, one per emitter at grid point (ix, iy) with phase
    ``phase`` and focal depth ``zf`` (arrays of equal length)."""
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    phase = np.ascontiguousarray(phase, dtype=np.float64)
    zf = np.ascontiguousarray(np.broadcast_to(zf, ix.shape), dtype=np.float64)
    E = np.zeros((ny, nx), np.complex128)
    rc = _load().oracle_multiplex_psf(nx, ny, dx, dy, lam, n0, ix.size, _ptr(ix), _ptr(iy),
                                      _ptr(phase), _ptr(zf), NA, _ptr(E))
    _check(rc, "multiplex_psf")
    return E


def multiplex_annular(nx, ny, dx, dy, lam, n0, ix, iy, phase, zf, NA_in, NA_out) -> np.ndarray:
    """As multiplex_psf with the annular pupil NA_in <= |k_perp|/k0 <= NA_out
    (Bessel beams; several emitters give a Bessel lattice)."""
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    phase = np.ascontiguousarray(phase, dtype=np.float64)
    zf = np.ascontiguousarray(np.broadcast_to(zf, ix.shape), dtype=np.float64)
    E = np.zeros((ny, nx), np.complex128)
    rc = _load().oracle_multiplex_annular(nx, ny, dx, dy, lam, n0, ix.size, _ptr(ix), _ptr(iy),
                                          _ptr(phase), _ptr(zf), NA_in, NA_out, _ptr(E))
    _check(rc, "multiplex_annular")
    return E


def light_sheet(nx, ny, dx, dy, lam, n0, NA, zf) -> np.ndarray:
    """Gaussian cylindrical light sheet focused at depth ``zf``."""
    E = np.zeros((ny, nx), np.complex128)
    _check(_load().oracle_light_sheet(nx, ny, dx, dy, lam, n0, NA, zf, _ptr(E)), "light_sheet")
    return E
