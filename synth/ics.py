"""Seeded synthetic initial conditions: Gaussian random field + Zel'dovich.

This is the separate initial-condition generator of the method (Section 2.3.2,
Fig. "fig.ic"): a linear density field delta_L(q) on the Lagrangian lattice
(white noise x transfer function in Fourier space), the displacement
potential from -lap(Phi) = delta_L, Psi = grad Phi, and particles displaced by
the Zel'dovich approximation.  It is not part of the PM step; it feeds both the
CUDA library and the FP64 oracle the same float32 (pos, vel) arrays.

Units (shared with the library and the oracle): length in fine mesh cells,
time in 1/H0, particle momentum p = a^2 dx/dt = a^3 E(a) dx/da in fine
cells x H0.  Positions are returned in [0, N_f).

White noise is drawn per integer wave-vector from Philox-4x32-10 keyed by the
seed (see philox.py), with Hermitian partners taken as complex conjugates of
a canonical half-space representative, so the large-scale modes of a run do
not depend on the grid resolution.  Nyquist planes are zeroed.
"""
import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate

from .philox import mode_gaussians


# --------------------------------------------------------------------------- cosmology
@dataclass(frozen=True)
class Cosmology:
    omega_m: float = 1.0
    omega_l: float = 0.0
    h: float = 0.7
    sigma8: float = 0.8
    n_s: float = 1.0
    spectrum: str = "powerlaw"      # "powerlaw" (P = A k^slope) or "bbks"
    slope: float = -2.0

    def E(self, a):
        """Dimensionless Hubble rate H(a)/H0 of a flat or curved FRW model."""
        ok = 1.0 - self.omega_m - self.omega_l
        return math.sqrt(self.omega_m / a ** 3 + ok / a ** 2 + self.omega_l)

    def _heath(self, a):
        return integrate.quad(lambda x: 1.0 / (x * self.E(x)) ** 3, 0.0, a,
                              epsabs=0.0, epsrel=1e-13, limit=200)[0]

    def growth_D(self, a):
        """Linear growth factor from the Heath (1977) integral, D(1) = 1."""
        if self.omega_m == 1.0 and self.omega_l == 0.0:
            return a
        d = lambda x: 2.5 * self.omega_m * self.E(x) * self._heath(x)
        return d(a) / d(1.0)

    def growth_f(self, a):
        """f = dlnD/dlna of the Heath solution."""
        if self.omega_m == 1.0 and self.omega_l == 0.0:
            return 1.0
        e = self.E(a)
        dlnE = (-1.5 * self.omega_m / a ** 3 - (1.0 - self.omega_m - self.omega_l) / a ** 2) / e ** 2
        return dlnE + 1.0 / (a ** 2 * e ** 3 * self._heath(a))

    def p_growth(self, a):
        """g(a) = a^2 E f D: linear growth of the momentum p = a^3 E dx/da."""
        return a * a * self.E(a) * self.growth_f(a) * self.growth_D(a)

    # power spectrum at a = 1 in (Mpc/h)^3, k in h/Mpc
    def _shape(self, k):
        k = np.asarray(k, dtype=np.float64)
        if self.spectrum == "powerlaw":
            with np.errstate(divide="ignore"):
                return np.where(k > 0, k ** self.slope, 0.0)
        if self.spectrum == "bbks":
            q = k / (self.omega_m * self.h)
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (np.log1p(2.34 * q) / (2.34 * q)) * (
                    1 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25
                return np.where(k > 0, k ** self.n_s * t * t, 0.0)
        raise ValueError(self.spectrum)

    def amplitude(self):
        """A with sigma(R = 8 Mpc/h, a = 1) = sigma8 for a top-hat window."""
        def integrand(lnk):
            k = math.exp(lnk)
            x = 8.0 * k
            w = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3 if x > 1e-4 else 1.0 - x * x / 10.0
            return k ** 3 * float(self._shape(k)) * w * w / (2.0 * math.pi ** 2)
        s2 = integrate.quad(integrand, math.log(1e-6), math.log(1e3), limit=400, epsrel=1e-10)[0]
        return self.sigma8 ** 2 / s2

    def power(self, k):
        return self.amplitude() * self._shape(k)


def einstein_de_sitter(sigma8=0.8):
    """C1 cosmology: EdS with P(k) = A k^-2."""
    return Cosmology(omega_m=1.0, omega_l=0.0, h=0.7, sigma8=sigma8, spectrum="powerlaw", slope=-2.0)


def lcdm_bbks(omega_m=0.3, h=0.7, sigma8=0.8, n_s=0.96):
    """C2/C3 cosmology: flat LCDM with the BBKS transfer function."""
    return Cosmology(omega_m=omega_m, omega_l=1.0 - omega_m, h=h, sigma8=sigma8, n_s=n_s, spectrum="bbks")


# --------------------------------------------------------------------------- Gaussian field
def _canonical(nx, ny, nz):
    """True where (nx, ny, nz) is the representative of the pair {n, -n}."""
    return (nx > 0) | ((nx == 0) & (ny > 0)) | ((nx == 0) & (ny == 0) & (nz > 0))


def white_noise_modes(n_grid, seed):
    """Unit-variance complex white noise on the rfftn layout [kz][ky][kx>=0].

    Returns the array xi with <|xi|^2> = 1 on every non-Nyquist, non-DC mode
    and Hermitian symmetry on the kx = 0 plane.
    """
    f = np.fft.fftfreq(n_grid, d=1.0 / n_grid).astype(np.int64)
    fx = np.arange(n_grid // 2 + 1, dtype=np.int64)
    nz, ny, nx = np.meshgrid(f, f, fx, indexing="ij")
    canon = _canonical(nx, ny, nz)
    sx = np.where(canon, nx, -nx)
    sy = np.where(canon, ny, -ny)
    sz = np.where(canon, nz, -nz)
    g1, g2 = mode_gaussians(sx, sy, sz, seed)
    xi = (g1 + 1j * np.where(canon, g2, -g2)) / math.sqrt(2.0)
    half = n_grid // 2
    nyq = (np.abs(nx) == half) | (np.abs(ny) == half) | (np.abs(nz) == half)
    xi[nyq] = 0.0
    xi[0, 0, 0] = 0.0
    return xi


def linear_delta_k(n_grid, box, cosmo, seed):
    """Fourier coefficients (numpy rfftn normalisation) of delta_L at a = 1."""
    xi = white_noise_modes(n_grid, seed)
    f = np.fft.fftfreq(n_grid, d=1.0 / n_grid)
    fx = np.arange(n_grid // 2 + 1)
    kf = 2.0 * math.pi / box
    kz, ky, kx = np.meshgrid(f * kf, f * kf, fx * kf, indexing="ij")
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    pk = cosmo.power(k)
    amp = n_grid ** 3 * np.sqrt(pk / box ** 3)
    return xi * amp, (kx, ky, kz, k)


@dataclass
class InitialConditions:
    pos: np.ndarray          # float32 [3][N] fine-cell units in [0, N_f)
    vel: np.ndarray          # float32 [3][N] momentum p in fine cells x H0
    ids: np.ndarray          # uint32 [N], Lagrangian lattice index
    a: float
    n_fine: int
    box: float
    cosmo: Cosmology
    sigma_1d: float          # per-dimension velocity-residual scale (Eq. vdelta / 3)


def zeldovich(n_part_side, n_fine, box, cosmo, a_init, seed, ratio=4):
    """Zel'dovich initial conditions on a lattice of n_part_side^3 particles.

    Lagrangian sites q = s*i + 1/2 (fine units, s = n_fine/n_part_side), which
    gives an exactly uniform CIC density for s = 2.  x = q + D Psi and
    p = a^2 E f D Psi.
    """
    ng = n_part_side
    s = n_fine / ng
    dk, (kx, ky, kz, k) = linear_delta_k(ng, box, cosmo, seed)
    k2 = k * k
    k2[0, 0, 0] = 1.0
    to_fine = n_fine / box
    psi = []
    for kc in (kx, ky, kz):
        pk = 1j * kc * dk / k2
        pk[0, 0, 0] = 0.0
        psi.append(np.fft.irfftn(pk, s=(ng, ng, ng), axes=(0, 1, 2)) * to_fine)
    D = cosmo.growth_D(a_init)
    g = cosmo.p_growth(a_init)
    idx = np.arange(ng, dtype=np.float64)
    qz, qy, qx = np.meshgrid(idx, idx, idx, indexing="ij")
    q = [qx * s + 0.5, qy * s + 0.5, qz * s + 0.5]
    pos = np.empty((3, ng ** 3), dtype=np.float32)
    vel = np.empty((3, ng ** 3), dtype=np.float32)
    for d in range(3):
        x = np.mod(q[d] + D * psi[d], float(n_fine)).ravel()
        x32 = x.astype(np.float32)
        x32[x32 >= np.float32(n_fine)] = 0.0       # float32 rounding up to N_f wraps to 0
        pos[d] = x32
        vel[d] = (g * psi[d]).ravel().astype(np.float32)
    ids = np.arange(ng ** 3, dtype=np.uint32)
    sig = sigma_delta_1d(ng, n_fine, box, cosmo, a_init, ratio)
    return InitialConditions(pos, vel, ids, a_init, n_fine, box, cosmo, sig)


def _tophat(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    m = x > 1e-4
    xm = x[m]
    out[m] = 3.0 * (np.sin(xm) - xm * np.cos(xm)) / xm ** 3
    out[~m] = 1.0 - x[~m] ** 2 / 10.0
    return out


def sigma_delta_1d(n_part_side, n_fine, box, cosmo, a, ratio=4):
    """Per-dimension codec scale from Eqs. vdisp/vdelta (Section 2.2).

    sigma_v^2(a, r) = (a^2 E f D)^2 (1/V) sum_k P(k)/k^2 W^2(k r) over the
    non-zero modes of the particle lattice, in momentum units (fine cells x
    H0).  The residual variance is sigma_v^2(r_p) - sigma_v^2(r_c) with r_c
    the coarse cell side and r_p the mean particle separation, and each
    dimension takes one third of it.
    """
    ng = n_part_side
    f = np.fft.fftfreq(ng, d=1.0 / ng)
    kf = 2.0 * math.pi / box
    kz, ky, kx = np.meshgrid(f * kf, f * kf, f * kf, indexing="ij")
    k = np.sqrt(kx * kx + ky * ky + kz * kz).ravel()
    k = k[k > 0]
    pk = cosmo.power(k)
    r_c = box / (n_fine / ratio)
    r_p = box / ng
    base = pk / (k * k) / box ** 3
    s_c = np.sum(base * _tophat(k * r_c) ** 2)
    s_p = np.sum(base * _tophat(k * r_p) ** 2)
    g = cosmo.p_growth(a) * (n_fine / box)
    var = g * g * abs(s_p - s_c)
    return math.sqrt(var / 3.0)
