"""Pins for the oracle's DFT: brute force on tiny lengths, numpy's FFT, the
Parseval identity and forward-then-inverse.  Split-step BPM rests on the 2D DFT
(Biobeam, arXiv:1706.02261, method paragraph: beam-propagation model)."""
import numpy as np
import pytest

import oracle


def brute_dft(x, sign):
    n = x.size
    j = np.arange(n)
    # exact integer phase index reduced mod n before scaling
    W = np.exp(sign * 2j * np.pi * ((j[:, None] * j[None, :]) % n) / n)
    return W @ x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 18, 24, 27, 32, 48, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_dft_matches_brute_force(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle.dft(x, sign)
    ref = brute_dft(x, sign)
    assert np.linalg.norm(got - ref) <= 1e-13 * max(1.0, np.linalg.norm(ref))


@pytest.mark.parametrize("n", [128, 192, 256, 384, 1024])
def test_dft_matches_numpy(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(oracle.dft(x, -1), np.fft.fft(x), rtol=0, atol=1e-11 * np.sqrt(n))
    assert np.allclose(oracle.dft(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-11 * np.sqrt(n))


@pytest.mark.parametrize("shape", [(4, 4), (8, 12), (12, 8), (6, 9), (16, 16), (24, 32)])
def test_dft2_matches_brute_force_and_numpy(shape):
    ny, nx = shape
    rng = np.random.default_rng(nx * 100 + ny)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = oracle.dft2(x, -1)
    # brute force: rows then columns, each by the definition
    ref = np.stack([brute_dft(r, -1) for r in x])
    ref = np.stack([brute_dft(c, -1) for c in ref.T]).T
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.allclose(got, np.fft.fft2(x), atol=1e-12 * np.linalg.norm(x))


@pytest.mark.parametrize("n", [64, 192, 256])
def test_parseval_and_roundtrip(n):
    rng = np.random.default_rng(7 * n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = oracle.dft2(x, -1)
    assert abs(np.vdot(X, X).real / (n * n) - np.vdot(x, x).real) <= 1e-12 * np.vdot(x, x).real
    back = oracle.dft2(X, +1) / (n * n)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x)) * np.log2(n)


def test_dft_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.dft(np.zeros(0, complex))
