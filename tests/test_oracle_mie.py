"""Physics report: the oracle's forward BPM behind a weakly scattering sphere
(n 1.38 in 1.33, r = 2 um, lambda 0.5 um, size parameter k a = 33) against the
exact scalar Mie series, both cut to propagating transverse waves.  BPM is
forward-only and splits the sphere into slices, so agreement is approximate;
the test reports the error and bounds it loosely."""
import numpy as np

import oracle
from oracle import mie

LAM, N0, N1, A = 0.5, 1.33, 1.38, 2.0


def test_bpm_behind_sphere_matches_mie_series():
    n, d = 256, 0.1
    nz = 60
    zc = 3.0                                  # sphere centre depth
    x = (np.arange(n) - n // 2) * d
    z = (np.arange(nz) + 1) * d - zc          # depth of each slice's exit plane relative to the centre
    X, Y = np.meshgrid(x, x)
    dn = np.zeros((nz, n, n))
    for k in range(nz):
        zz = (k + 0.5) * d - zc               # slice mid-plane
        dn[k] = np.where(X ** 2 + Y ** 2 + zz ** 2 <= A * A, N1 - N0, 0.0)
    E0 = np.ones((n, n), complex)
    E, _ = oracle.bpm(dn, E0, d, d, d, LAM, N0)
    EB, _ = oracle.bpm(dn, E0, d, d, d, LAM, N0, adaptive=True)      # locally adapted expansion, reading B
    zp = z[-1]                                # plane 3 um behind the centre
    K = 2 * np.pi / LAM * N0
    # the BPM input has phase 0 at its entrance plane z = -zc: shift the
    # series' incident wave exp(i K z) accordingly
    ref = mie.field_outside(2 * np.pi / LAM, N0, N1, A, X, Y, np.full(X.shape, zp)) * np.exp(1j * K * zc)
    # compare on the propagating band only (BPM drops evanescent waves)
    k = 2 * np.pi * np.fft.fftfreq(n, d)
    mask = (k[None, :] ** 2 + k[:, None] ** 2) < (2 * np.pi / LAM * N0) ** 2 * 0.8
    lp = lambda f: np.fft.ifft2(np.fft.fft2(f) * mask)
    centre = (np.abs(X) < 6) & (np.abs(Y) < 6)
    err = np.linalg.norm((lp(E) - lp(ref))[centre]) / np.linalg.norm(lp(ref)[centre])
    incident = np.exp(1j * K * (zp + zc))
    scat_err = np.linalg.norm((lp(E) - lp(ref))[centre]) / np.linalg.norm((lp(ref) - incident)[centre])
    scat_err_b = np.linalg.norm((lp(EB) - lp(ref))[centre]) / np.linalg.norm((lp(ref) - incident)[centre])
    print(f"BPM vs Mie 3 um behind the sphere: field rel err {err:.3e}, scattered-part rel err {scat_err:.3e} "
          f"(reading B {scat_err_b:.3e})")
    assert err < 0.03
    assert scat_err < 0.06
    assert scat_err_b < 0.06
