"""Fine-mesh operations of the PM force and the power spectrum (FP64).

Mesh arrays are indexed [z][y][x] (x fastest); particle arrays are [3][N]
with row 0 = x.  Positions are in fine-cell units, periodic in [0, N_f).

Readings (the paper uses CUBEP3M's force kernels without printing them,
Section 3): Poisson lap Phi = (3/2) Omega_m (rho - 1) solved with the
continuous Green's function -1/k^2, k_i = 2 pi n_i / N_f, divided by the CIC
window W(k) = prod_i sinc^2(k_i / 2) raised to `deconv_power` (2 compensates
deposit and gather); the k = 0 mode is zero.  The force is minus the
fourth-order central difference of Phi; CIC nodes sit at integer fine
coordinates.
"""
import numpy as np


def _split(pos, n):
    pos = np.asarray(pos, dtype=np.float64)
    i = np.floor(pos)
    w = pos - i
    return np.mod(i.astype(np.int64), n), w


def _corners(pos, n):
    """Yield (flat node index, CIC weight) for the 8 nodes around each particle."""
    (ix, iy, iz), (wx, wy, wz) = _split(pos, n)
    for dz in (0, 1):
        fz = wz if dz else 1.0 - wz
        z = (iz + dz) % n
        for dy in (0, 1):
            fy = wy if dy else 1.0 - wy
            y = (iy + dy) % n
            for dx in (0, 1):
                fx = wx if dx else 1.0 - wx
                x = (ix + dx) % n
                yield (z * n + y) * n + x, fx * fy * fz


def cic_deposit(pos, n, mass):
    """Cloud-in-cell density (Section 3.2): each particle of mass `mass`
    spreads over the 8 surrounding nodes with weights prod (1-w) / w.
    The weights are summed first and scaled by the mass once."""
    acc = np.zeros(n ** 3, dtype=np.float64)
    for idx, wt in _corners(pos, n):
        acc += np.bincount(idx, weights=wt, minlength=n ** 3)
    return (acc * mass).reshape(n, n, n)


def cic_gather(field, pos):
    """Trilinear (CIC) interpolation of a mesh field at the particles."""
    n = field.shape[0]
    flat = field.reshape(-1)
    out = np.zeros(np.asarray(pos).shape[1], dtype=np.float64)
    for idx, wt in _corners(pos, n):
        out += wt * flat[idx]
    return out


def wavenumbers(n):
    """Integer wave-vector components on the rfftn layout [kz][ky][kx >= 0]."""
    f = np.fft.fftfreq(n, d=1.0 / n)
    fx = np.arange(n // 2 + 1, dtype=np.float64)
    return np.meshgrid(f, f, fx, indexing="ij")     # nz, ny, nx


def cic_window(n):
    """W(k) = prod_i sinc^2(pi n_i / N) on the rfftn layout."""
    nz, ny, nx = wavenumbers(n)
    return (np.sinc(nx / n) * np.sinc(ny / n) * np.sinc(nz / n)) ** 2


def green(n, omega_m, deconv_power):
    """-(3/2) Omega_m / k^2 / W(k)^p, zero at k = 0."""
    nz, ny, nx = wavenumbers(n)
    k2 = (2 * np.pi / n) ** 2 * (nx * nx + ny * ny + nz * nz)
    k2[0, 0, 0] = 1.0
    g = -1.5 * omega_m / k2
    if deconv_power:
        g = g / cic_window(n) ** deconv_power
    g[0, 0, 0] = 0.0
    return g


def potential(rho, omega_m, deconv_power=2):
    """Phi from lap Phi = (3/2) Omega_m (rho - 1) via numpy's FFT."""
    n = rho.shape[0]
    return np.fft.irfftn(np.fft.rfftn(rho) * green(n, omega_m, deconv_power), s=rho.shape, axes=(0, 1, 2))


def fd4_gradient(phi):
    """4th-order central difference (8(f[i+1]-f[i-1]) - (f[i+2]-f[i-2]))/12
    along x, y, z (array axes 2, 1, 0)."""
    out = []
    for ax in (2, 1, 0):
        d1 = np.roll(phi, -1, ax) - np.roll(phi, 1, ax)
        d2 = np.roll(phi, -2, ax) - np.roll(phi, 2, ax)
        out.append((8.0 * d1 - d2) / 12.0)
    return out


def force_at(pos, rho, omega_m, deconv_power=2):
    """PM force F = -grad Phi (FD4) interpolated to the particles by CIC."""
    phi = potential(rho, omega_m, deconv_power)
    return np.stack([-cic_gather(g, pos) for g in fd4_gradient(phi)])


def force_at_points(phi, pos):
    """-grad Phi (FD4) interpolated by CIC at the particles `pos`, with the
    difference evaluated only at the 8 nodes around each particle: the same
    sums as the gather of fd4_gradient's meshes, for a sample of particles on
    a mesh too large to difference whole."""
    n = phi.shape[0]
    flat = np.asarray(phi, dtype=np.float64).reshape(-1)
    (ix, iy, iz), (wx, wy, wz) = _split(pos, n)
    out = np.zeros((3, ix.size), dtype=np.float64)

    def at(x, y, z):
        return flat[((z % n) * n + (y % n)) * n + (x % n)]

    for dz in (0, 1):
        fz = wz if dz else 1.0 - wz
        for dy in (0, 1):
            fy = wy if dy else 1.0 - wy
            for dx in (0, 1):
                fx = wx if dx else 1.0 - wx
                x, y, z = ix + dx, iy + dy, iz + dz
                wt = fx * fy * fz
                for d, (ex, ey, ez) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    d1 = at(x + ex, y + ey, z + ez) - at(x - ex, y - ey, z - ez)
                    d2 = at(x + 2 * ex, y + 2 * ey, z + 2 * ez) - at(x - 2 * ex, y - 2 * ey, z - 2 * ez)
                    out[d] -= wt * (8.0 * d1 - d2) / 12.0
    return out


# ---------------------------------------------------------------- power spectrum
def shell_index(n2):
    """Shell i with i - 1/2 <= |n| < i + 1/2, decided in integers:
    i(i-1) < n^2 <= i(i+1)."""
    n2 = np.asarray(n2, dtype=np.int64)
    i = np.floor(np.sqrt(n2.astype(np.float64))).astype(np.int64)
    i = np.where(i * i > n2, i - 1, i)
    i = np.where((i + 1) * (i + 1) <= n2, i + 1, i)     # i = isqrt(n2)
    return np.where(n2 > i * (i + 1), i + 1, i)


def power_spectrum_mesh(rho, box, n_bins, deconvolve=True):
    """Auto power spectrum (Eq. cps, Section 3.2) of a density mesh.

    delta = rho / mean(rho) - 1, P(k) = L^3 / N_m^2 |delta_k|^2 / W(k)^2 (if
    `deconvolve`), averaged over shells i = 1..n_bins of the integer |n|, each
    rfftn mode counted twice except on the kx = 0 and kx = N/2 planes.
    Returns (k [h/Mpc], P [(Mpc/h)^3], weighted mode count) per shell.
    """
    n = rho.shape[0]
    nm = n ** 3
    dk = np.fft.rfftn(rho / (rho.sum() / nm))
    p = (box ** 3 / nm ** 2) * np.abs(dk) ** 2
    if deconvolve:
        p = p / cic_window(n) ** 2
    nz, ny, nx = wavenumbers(n)
    n2 = (nx * nx + ny * ny + nz * nz).astype(np.int64)
    wt = np.where((nx == 0) | (nx == n // 2), 1.0, 2.0)
    sh = shell_index(n2)
    kmag = 2 * np.pi / box * np.sqrt(n2.astype(np.float64))
    sel = (sh >= 1) & (sh <= n_bins)
    s = sh[sel]
    cnt = np.bincount(s, weights=wt[sel], minlength=n_bins + 1)[1:]
    ksum = np.bincount(s, weights=(wt * kmag)[sel], minlength=n_bins + 1)[1:]
    psum = np.bincount(s, weights=(wt * p)[sel], minlength=n_bins + 1)[1:]
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt


def power_spectrum(pos, n, mass, box, n_bins):
    """P(k) of a particle set: CIC onto the fine mesh, then power_spectrum_mesh."""
    return power_spectrum_mesh(cic_deposit(pos, n, mass), box, n_bins, deconvolve=True)
