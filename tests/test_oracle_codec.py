"""Pins of the oracle's codec and storage order (Sections 2.1, 2.2).

Each test ties the oracle to something other than itself: the worked example
printed in Section 2.1, exact bin arithmetic, thresholds evaluated with
50-digit arithmetic, the Gaussian density the velocity mapping must match at
zero, and brute-force checks of the sort.
"""
import os

import mpmath
from fractions import Fraction

import numpy as np
import pytest

from oracle import codec, layout, pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                out[k] = [float(x) for x in v]
    return out


def test_decode_worked_example():
    """Section 2.1's 1-D example: chi, rho_c -> x, exactly."""
    g = _read_golden("sec2_1_decode_example.txt")
    n_chi = int(g["n_chi"][0])
    cells = layout.particle_cells(np.array(g["rho_c"], dtype=np.int64))
    x = codec.pos_decode(cells, np.array(g["chi"]), n_chi)
    assert np.array_equal(x, np.array(g["x"]))


@pytest.mark.parametrize("n_chi", [1, 2])
def test_position_roundtrip_half_bin(n_chi):
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 32, 200000).astype(np.float32).astype(np.float64)
    cell, chi = codec.pos_encode(x, n_chi)
    half = 2.0 ** (-8 * n_chi - 1)
    xr = codec.pos_decode(cell, chi, n_chi)
    assert np.max(np.abs(xr - x)) <= half
    lim = 2 ** (8 * n_chi - 1)
    assert chi.min() >= -lim and chi.max() <= lim - 1


@pytest.mark.parametrize("n_chi", [1, 2])
def test_position_encode_of_decode_is_identity(n_chi):
    lim = 2 ** (8 * n_chi - 1)
    chi = np.arange(-lim, lim)
    for c in (0, 5, 31):
        cell, chi2 = codec.pos_encode(codec.pos_decode(np.full(chi.shape, c), chi, n_chi), n_chi)
        assert np.all(cell == c) and np.array_equal(chi2, chi)


def test_position_floor_at_bin_edges():
    """[ ] in Eq. chi is the integer part (floor): an exact bin edge k/256
    belongs to bin k, the FP32 value just below it to bin k-1."""
    k = np.arange(256)
    edge = (3 + k / 256.0).astype(np.float32)
    below = np.nextafter(edge, np.float32(0))
    c1, chi1 = codec.pos_encode(edge.astype(np.float64), 1)
    c0, chi0 = codec.pos_encode(below.astype(np.float64), 1)
    assert np.all(c1 == 3) and np.array_equal(chi1, k - 128)
    assert np.array_equal(chi0[1:], k[1:] - 129) and c0[0] == 2 and chi0[0] == 127


@pytest.mark.parametrize("n_nu", [1, 2])
def test_velocity_encode_of_decode_is_identity(n_nu):
    lim = codec.nu_max(n_nu)
    nu = np.arange(-lim, lim + 1)
    sigma = 0.37
    dv = codec.vel_decode_offset(nu, sigma, n_nu)
    assert np.array_equal(codec.vel_encode(dv, sigma, n_nu), nu)


@pytest.mark.parametrize("n_nu", [1, 2])
def test_velocity_roundtrip_within_bin(n_nu):
    """|atan(s dv) - pi nu / M| <= pi / (2M): the decoded value is the centre of
    the tan-space bin that contains dv."""
    rng = np.random.default_rng(2)
    sigma = 0.05
    dv = rng.standard_cauchy(100000) * sigma
    nu = codec.vel_encode(dv, sigma, n_nu)
    m = 2 ** (8 * n_nu) - 1
    ang = np.arctan(dv * codec.vel_scale(sigma))
    assert np.max(np.abs(ang - np.pi * nu / m)) <= np.pi / (2 * m) * (1 + 1e-9)


@pytest.mark.parametrize("n_nu", [1, 2])
def test_velocity_codes_at_exact_thresholds(n_nu):
    """Eq. nu decides nu >= k exactly when |dv| >= tan(pi (k - 1/2) / M) / s.
    The thresholds are computed with 50 digits; the FP32 values on both sides
    of each threshold must land in bins k - 1 and k."""
    mpmath.mp.dps = 50
    m = 2 ** (8 * n_nu) - 1
    sigma = 0.0123
    s = mpmath.sqrt(mpmath.pi / (2 * mpmath.mpf(sigma) ** 2))
    ks = list(range(1, 40)) + list(range(codec.nu_max(n_nu) - 30, codec.nu_max(n_nu) + 1))
    lo, hi, want_lo, want_hi = [], [], [], []
    for k in ks:
        t = mpmath.tan(mpmath.pi * (k - mpmath.mpf(1) / 2) / m) / s
        f = np.float32(float(t))
        # the FP32 neighbours that straddle the exact threshold
        a = f if mpmath.mpf(float(f)) < t else np.nextafter(f, np.float32(0))
        b = np.nextafter(a, np.float32(np.inf))
        assert mpmath.mpf(float(a)) < t <= mpmath.mpf(float(b))
        lo.append(a), hi.append(b), want_lo.append(k - 1), want_hi.append(k)
    lo, hi = np.array(lo, np.float32), np.array(hi, np.float32)
    assert np.array_equal(codec.vel_encode(lo, sigma, n_nu), want_lo)
    assert np.array_equal(codec.vel_encode(hi, sigma, n_nu), want_hi)
    assert np.array_equal(codec.vel_encode(-hi, sigma, n_nu), -np.array(want_hi))


def test_velocity_mapping_matches_gaussian_density_at_zero():
    """Section 2.2: the tangent mapping takes the same variance at nu = 0 as
    the Gaussian-CDF mapping, i.e. codes per unit velocity at dv = 0 equal
    M times the normal density at 0: M / (sigma sqrt(2 pi))."""
    m = 255
    for sigma in (0.01, 0.3, 7.0):
        h = sigma * 1e-7
        cont = lambda dv: (m / np.pi) * np.arctan(dv * codec.vel_scale(sigma))
        slope = (cont(h) - cont(-h)) / (2 * h)
        assert slope == pytest.approx(m / (sigma * np.sqrt(2 * np.pi)), rel=1e-9)


def test_velocity_codes_are_clamped_and_odd():
    for n_nu in (1, 2):
        lim = codec.nu_max(n_nu)
        big = np.array([1e30, -1e30, np.inf, -np.inf])
        assert list(codec.vel_encode(big, 1.0, n_nu)) == [lim, -lim, lim, -lim]
        x = np.linspace(-3, 3, 1001)
        assert np.array_equal(codec.vel_encode(-x, 0.5, n_nu), -codec.vel_encode(x, 0.5, n_nu))


def test_snap_sigma_is_a_sixteenth_octave():
    rng = np.random.default_rng(3)
    for s in np.exp(rng.uniform(-20, 5, 200)):
        t = codec.snap_sigma(s)
        m = 16 * np.log2(t)
        assert abs(m - round(m)) < 1e-9
        assert abs(np.log2(t / s)) <= 1 / 32 + 1e-12
        assert codec.snap_sigma(t) == t
    assert codec.snap_sigma(0.0) == 2.0 ** -30


# ---------------------------------------------------------------- storage order
@pytest.mark.parametrize("nc,b", [(12, 4), (8, 2), (6, 2), (5, 1), (16, 16)])
def test_storage_order_is_brick_major_bijection(nc, b):
    cz, cy, cx = np.meshgrid(np.arange(nc), np.arange(nc), np.arange(nc), indexing="ij")
    idx = layout.storage_index(cx.ravel(), cy.ravel(), cz.ravel(), nc, b)
    assert np.array_equal(np.sort(idx), np.arange(nc ** 3))
    x, y, z = layout.cell_coords(idx, nc, b)
    assert np.array_equal(x, cx.ravel()) and np.array_equal(y, cy.ravel()) and np.array_equal(z, cz.ravel())
    # walk the storage order: inside a brick x is fastest, bricks follow x-fastest
    x, y, z = layout.cell_coords(np.arange(nc ** 3), nc, b)
    assert np.array_equal(x[:b], np.arange(b)) and np.all(y[:b] == 0) and np.all(z[:b] == 0)
    if nc // b > 1:
        assert (x[b ** 3], y[b ** 3], z[b ** 3]) == (b, 0, 0)
    if b == nc:
        assert np.array_equal(np.arange(nc ** 3), x + nc * (y + nc * z))


def test_auto_brick():
    assert [layout.auto_brick(n) for n in (32, 128, 24, 8, 4, 3, 6)] == [4, 4, 4, 2, 1, 1, 2]


def test_stable_order_bruteforce():
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 37, 5000)
    order = layout.stable_order(keys)
    k = keys[order]
    assert np.all(np.diff(k) >= 0)
    same = np.diff(k) == 0
    assert np.all(np.diff(order)[same] > 0)
    counts = np.bincount(keys, minlength=37)
    off = layout.offsets_from_counts(counts)
    assert off[-1] == len(keys) and np.all(np.diff(off) >= 0)
    assert np.array_equal(layout.particle_cells(counts), k)


def test_cell_mean_velocity_is_mean_and_order_free():
    rng = np.random.default_rng(5)
    n, cells = 20000, 300
    key = rng.integers(0, cells, n)
    vel = (rng.standard_normal((3, n)) * rng.uniform(1e-4, 10, (3, 1))).astype(np.float32)
    vc = pm.cell_mean_velocity(key, vel, cells)
    for d in range(3):
        for c in range(0, cells, 17):
            sel = key == c
            if sel.any():
                exact = vel[d][sel].astype(np.float64).mean()
                tol = 2.0 ** -25 + abs(exact) * 2.0 ** -23
                assert abs(float(vc[d][c]) - exact) <= tol
    perm = rng.permutation(n)
    assert np.array_equal(pm.cell_mean_velocity(key[perm], vel[:, perm], cells), vc)
    assert np.all(vc[:, np.bincount(key, minlength=cells) == 0] == 0)


def _round_f32_exact(x):
    """x (a Fraction) rounded to the nearest float32, ties to even, by exact
    comparison with its two float32 neighbours."""
    f = np.float32(float(x))
    while Fraction(float(f)) > x:
        f = np.nextafter(f, np.float32(-np.inf))
    while Fraction(float(np.nextafter(f, np.float32(np.inf)))) <= x:
        f = np.nextafter(f, np.float32(np.inf))
    hi = np.nextafter(f, np.float32(np.inf))
    lo_gap, hi_gap = x - Fraction(float(f)), Fraction(float(hi)) - x
    if lo_gap < hi_gap:
        return f
    if hi_gap < lo_gap:
        return hi
    return f if int(f.view(np.uint32)) % 2 == 0 else hi


def test_cell_mean_velocity_is_the_correctly_rounded_fixed_point_mean():
    """v_c = the exact rational mean of the 2^-24 fixed-point velocities,
    rounded once to float32 (ties to even), for random cells and for sums
    built to land next to a float32 rounding midpoint, where rounding twice
    (or summing in floating point) would differ."""
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(300):                                    # random cells
        n = int(rng.integers(1, 400))
        q = rng.integers(-2 ** 24 + 1, 2 ** 24, n)          # |v| < 1: every 2^-24 multiple is a float32
        cases.append(q)
    for _ in range(300):                                    # next to a midpoint
        n = int(rng.integers(2, 2000))
        m = np.float32(rng.uniform(-0.9, 0.9))
        mid = (Fraction(float(m)) + Fraction(float(np.nextafter(m, np.float32(np.inf))))) / 2
        total = round(mid * n * 2 ** 24) + int(rng.integers(-1, 2))
        q = np.full(n, total // n, dtype=np.int64)
        q[: total - int(q.sum())] += 1
        cases.append(q)
    for q in cases:
        vel = (q.astype(np.float64) / 2 ** 24).astype(np.float32)
        assert np.array_equal(np.rint(vel.astype(np.float64) * 2 ** 24).astype(np.int64), q)   # representable
        key = np.zeros(len(q), np.int64)
        got = pm.cell_mean_velocity(key, np.stack([vel] * 3), 1)[0, 0]
        want = _round_f32_exact(Fraction(int(q.sum()), len(q) * 2 ** 24))
        assert got == want, (len(q), int(q.sum()))
