"""The precision study's cross-correlation coefficient (Eq. ccc), CPU only:
the r2c estimator with its plane weights equals the same sums over every
mode of a full complex FFT with shells taken from |n| directly; identical
fields correlate to 1, and |xi| <= 1."""
import numpy as np
import pytest

import precision_study as ps
from oracle import mesh


def _xi_full(pos_a, pos_b, n, mass, n_bins):
    """Eq. ccc over all N^3 modes of a complex FFT, shell i = floor(|n| + 1/2)
    (|n| is never a half-integer for integer n, so no tie arises)."""
    def modes(p):
        rho = mesh.cic_deposit(np.mod(np.asarray(p, np.float64), n), n, mass)
        return np.fft.fftn(rho / rho.mean() - 1.0)
    da, db = modes(pos_a), modes(pos_b)
    f = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    shell = np.floor(np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) + 0.5).astype(np.int64)
    out = np.zeros(n_bins)
    for i in range(1, n_bins + 1):
        m = shell == i
        ab = np.sum((da[m] * np.conj(db[m])).real)
        out[i - 1] = ab / np.sqrt(np.sum(np.abs(da[m]) ** 2) * np.sum(np.abs(db[m]) ** 2))
    return out


@pytest.mark.parametrize("n,noise", [(16, 0.3), (24, 1.0), (16, 4.0)])
def test_cross_correlation_equals_the_full_fft_sums(n, noise):
    rng = np.random.default_rng(n)
    npart = 3 * n ** 3 // 8
    pos_a = rng.uniform(0, n, (3, npart))
    pos_b = np.mod(pos_a + noise * rng.standard_normal((3, npart)), n)
    mass = n ** 3 / npart
    n_bins = n // 2
    xi = ps.cross_correlation(pos_a, pos_b, n, mass, n_bins)
    assert np.allclose(xi, _xi_full(pos_a, pos_b, n, mass, n_bins), rtol=0, atol=1e-12)
    assert np.all(np.abs(xi) <= 1 + 1e-12)
    assert np.allclose(ps.cross_correlation(pos_a, pos_a, n, mass, n_bins), 1.0, rtol=0, atol=1e-14)
