"""Pins of the oracle's compressed-store KD step (`pm.step`) as a whole.

Each case checks the composition decode -> force -> kick -> re-code ->
drift -> rebuild against something fixed outside it:
  * a uniformly moving lattice translates by v * int da/(a^3 E), written in
    closed form for EdS, with every velocity code zero and every v_c equal to
    the bulk momentum (Sections 2.1-2.2: the codes hold v - v_c);
  * the 1-D Zel'dovich plane wave is followed as closely as the uncompressed
    FP64 step follows it, plus the position codes' resolution;
  * one step agrees with the uncompressed FP64 step from the store's decoded
    particles to within the half-widths of the velocity bins it passes through
    (Eq. v, twice: the kick is re-coded against the old v_c, the new store
    codes it against the new v_c) and half a position bin (Eq. x);
  * the next store's codec scale is the measured dispersion times the EdS
    momentum growth (a_{n+1}/a_n)^{3/2}, snapped to 1/16 octave (Section 2.2).
"""
import numpy as np
import pytest

from oracle import codec, cosmo, pm


def _lattice(n):
    """Particles at 2i + 1/2 fine cells: 8 per coarse cell of 4 fine cells."""
    g = np.arange(n // 2) * 2 + 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()])


def _eds_drift(a0, a1):
    """int_{a0}^{a1} da / (a^3 E) with E = a^{-3/2}."""
    return 2.0 * (a0 ** -0.5 - a1 ** -0.5)


def _wrap(d, n):
    return (d + n / 2) % n - n / 2


@pytest.mark.parametrize("xb,vb,brick", [(1, 1, 0), (1, 1, 1), (2, 2, 2), (2, 1, 0), (1, 2, 4)])
def test_uniform_lattice_translates_with_zero_velocity_codes(xb, vb, brick):
    """A lattice of spacing 2 fine cells deposits a density whose Fourier modes
    sit at k = 0 or pi on each axis, where the FD4 symbol vanishes, so it feels
    no force at any translation.  With one bulk momentum v0 (a multiple of
    2^-24) every occupied cell has v_c = v0 and every code nu = 0, the momentum
    stays v0 exactly, and each particle moves by v0 times the drift integral.
    Positions are re-coded every step: each step adds at most half a
    position bin of error, the first encode another half.  The total move
    (4, -6, 8 fine cells) crosses coarse cells and the periodic edge."""
    n, steps = 32, 8
    q = _lattice(n)
    v0 = np.array([1.5, -2.25, 3.0])
    vel = np.repeat(v0[:, None], q.shape[1], axis=1)
    P = pm.Params(n_fine=n, n_particles=q.shape[1], x_bytes=xb, v_bytes=vb, box=50.0, brick=brick)
    sched = np.linspace(0.1, 0.3, steps + 1)
    st = pm.run(pm.encode(P, q, vel, a=sched[0]), sched)
    pos, v, ids = pm.decode(st)
    assert np.array_equal(np.sort(ids), np.arange(q.shape[1]))
    assert np.all(st.counts == 8)
    assert np.all(st.nu == 0)
    assert np.array_equal(st.vc, np.repeat(v0[:, None], len(st.counts), axis=1).astype(np.float32))
    assert np.array_equal(v, np.repeat(v0[:, None], q.shape[1], axis=1))
    want = q[:, ids] + v0[:, None] * _eds_drift(sched[0], sched[-1])
    bound = (steps + 1) * 0.5 * P.ratio / 2 ** (8 * xb) + 1e-5
    assert np.max(np.abs(_wrap(pos - want, n))) <= bound
    assert (st.a, st.a_p) == (sched[-1], pytest.approx(0.5 * (sched[-2] + sched[-1])))


@pytest.mark.parametrize("xb,vb", [(2, 2), (1, 1)])
def test_zeldovich_plane_wave_through_the_codes(xb, vb):
    """EdS plane wave x = q + D Psi(q), Psi = -sin(kq)/(A k), crossing at D = A,
    followed from D = 0.1 A to 0.5 A in 20 steps of the compressed store.  The
    uncompressed FP64 step stays within 1% of the displacement amplitude
    without deconvolution; the codes add at most half a position bin per
    re-code (21 of them).  The transverse coordinates never move: they stay
    in their first bin, half a bin from q."""
    n, ng, steps = 64, 32, 20
    k = 2 * np.pi / n
    amp = 1.0
    q = _lattice(n)
    psi = -np.sin(k * q[0]) / (amp * k)

    def za(a):
        pos = q.copy()
        pos[0] = np.mod(q[0] + a * psi, n)
        vel = np.zeros_like(q)
        vel[0] = a ** 1.5 * psi                      # p = a^2 E f D Psi in EdS
        return pos, vel
    a0, a1 = 0.1 * amp, 0.5 * amp
    P = pm.Params(n_fine=n, n_particles=ng ** 3, box=100.0, x_bytes=xb, v_bytes=vb, deconv_power=0)
    st = pm.run(pm.encode(P, *za(a0), a=a0), np.linspace(a0, a1, steps + 1))
    pos, _, ids = pm.decode(st)
    want, _ = za(a1)
    half_bin = 0.5 * P.ratio / 2 ** (8 * xb)
    disp = a1 / (amp * k)
    assert np.max(np.abs(_wrap(pos[0] - want[0, ids], n))) < 0.01 * disp + (steps + 1) * half_bin
    assert np.max(np.abs(pos[1:] - q[1:, ids])) <= half_bin + 1e-12


def _vel_half_bin(nu, sigma, n_nu):
    """Largest distance from the decoded offset of code nu (Eq. v) to the
    edges of its bin, the points whose Eq. nu value is nu +- 1/2; the codes
    next to nu are included so that a value on a bin edge is covered."""
    m = 2 ** (8 * n_nu) - 1
    s = np.sqrt(2.0 * sigma * sigma / np.pi)
    out = np.zeros(np.shape(nu))
    for c in (nu - 1, nu, nu + 1):
        t = np.tan(np.pi * c / m)
        up = np.abs(np.tan(np.pi * (c + 0.5) / m) - t)
        dn = np.abs(t - np.tan(np.pi * (c - 0.5) / m))
        out = np.maximum(out, s * np.maximum(up, dn))
    return out


def _clustered(seed, n, npart):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0, n, (3, 6))
    pos = np.mod(centers[:, rng.integers(0, 6, npart)] + rng.standard_normal((3, npart)) * 2.0, n)
    vel = rng.standard_normal((3, npart)) * 0.5
    return pos.astype(np.float32), vel.astype(np.float32)


@pytest.mark.parametrize("om,ol", [(1.0, 0.0), (0.3, 0.7)])
@pytest.mark.parametrize("xb,vb", [(1, 1), (2, 2), (1, 2), (2, 1)])
def test_one_step_matches_the_uncompressed_step_within_code_bins(xb, vb, om, ol):
    n, npart, a0, a1 = 32, 4096, 0.2, 0.22
    pos, vel = _clustered(3, n, npart)
    P = pm.Params(n_fine=n, n_particles=npart, x_bytes=xb, v_bytes=vb, box=50.0, omega_m=om, omega_l=ol)
    st0 = pm.encode(P, pos, vel, a=a0)
    x0, v0, ids0 = pm.decode(st0)
    ex = pm.exact_step(pm.exact_from(P, x0, v0, a0), a0, a1)
    st1 = pm.step(st0, a0, a1, keep_drifted=True)
    x1, v1, ids1 = pm.decode(st1)
    assert np.max(np.abs(st1.nu)) < codec.nu_max(vb)           # no clamped code: the bins bound the error
    assert np.array_equal(np.sort(ids1), np.arange(npart))
    assert st1.counts.sum() == npart and (st1.a, st1.a_p) == (a1, 0.5 * (a0 + a1))
    # the uncompressed result, in the new storage order
    inv = np.empty(npart, np.int64)
    inv[ids0] = np.arange(npart)
    j = inv[ids1]
    xe, ve = ex.pos[:, j], ex.vel[:, j]
    # first re-code: the kicked momentum against the old v_c with the old scale
    key0 = np.repeat(np.arange(len(st0.counts)), st0.counts)
    nu_k = np.stack([codec.vel_encode(ex.vel[d] - st0.vc[d][key0], st0.sigma, vb) for d in range(3)])
    hb1 = np.stack([_vel_half_bin(nu_k[d], st0.sigma, vb) for d in range(3)])[:, j]
    # second re-code: against the new v_c with the new scale
    hb2 = np.stack([_vel_half_bin(st1.nu[d], st1.sigma, vb) for d in range(3)])
    eps = 1e-6 * (np.abs(ve) + 1.0)                               # FP32 storage of momenta and v_c
    assert np.all(np.abs(v1 - ve) <= hb1 + hb2 + eps)
    drift = cosmo.drift_factor(a0, a1, om, ol)
    moved = np.abs(_wrap(xe - x0[:, j], n))
    assert moved.max() > 0.5                                      # the step really moves particles
    bound = (hb1 + eps) * drift + 0.5 * P.ratio / 2 ** (8 * xb) + 1e-5
    assert np.all(np.abs(_wrap(x1 - xe, n)) <= bound)
    if om == 1.0:
        p = st1.extra["p"].astype(np.float64)
        disp = np.sqrt(np.mean((p - st0.vc[:, key0].astype(np.float64)) ** 2))
        target = 16 * np.log2(disp * (a1 / a0) ** 1.5)
        m = np.round(16 * np.log2(st1.sigma))
        assert st1.sigma == pytest.approx(2.0 ** (m / 16), rel=1e-14) and abs(m - target) <= 0.5 + 1e-9


# ---------------------------------------------------------------- the drift's single rounding
def _round_f32(x):
    """Nearest FP32 to the rational x, ties to even (x normal in FP32)."""
    from fractions import Fraction
    if x == 0:
        return 0.0
    sgn = -1 if x < 0 else 1
    m = abs(Fraction(x))
    e = 0
    while m >= 2 ** 24:
        m /= 2
        e += 1
    while m < 2 ** 23:
        m *= 2
        e -= 1
    q, r = divmod(m.numerator, m.denominator)
    rem = Fraction(r, m.denominator)
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q % 2 == 1):
        q += 1
    return float(sgn * Fraction(q) * Fraction(2) ** e)


def test_drift_offset_is_rounded_once():
    """The drifted offset u + p dc (Fig. update_xp) is the FP32 value of the
    exact sum, rounded once, as a fused multiply-add forms it.  Random FP32
    triples against exact rational rounding, and a tie that an FP64 add
    followed by an FP32 conversion rounds the wrong way: u = 1/2, p dc =
    3 2^-25 - 12 2^-71 lies just below the midpoint 1/2 + 3 2^-25, so the
    answer is 1/2 + 2^-24, while FP64 first rounds to the midpoint and the
    tie then goes to 1/2 + 2^-23."""
    from fractions import Fraction
    rng = np.random.default_rng(1712)
    n = 4000
    u = (2.0 * rng.integers(0, 256, n) + 1) / 512.0 * rng.choice([1, -1], n)
    p = (rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 2, n)).astype(np.float32)
    dc = (rng.uniform(0.01, 2.0, n) * 10.0 ** rng.uniform(-4, 0, n)).astype(np.float32)
    got = pm.fma_f32(p, dc, u)
    want = np.array([_round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))
                     for a, b, c in zip(p, dc, u.astype(np.float32))], np.float32)
    assert np.array_equal(got, want)
    p1 = np.float32((3 * 2 ** 22 + 3) * 2.0 ** -22)
    d1 = np.float32((2 ** 24 - 4) * 2.0 ** -49)
    exact = Fraction(float(p1)) * Fraction(float(d1)) + Fraction(1, 2)
    assert exact == Fraction(1, 2) + 3 * Fraction(1, 2 ** 25) - 12 * Fraction(1, 2 ** 71)
    assert _round_f32(exact) == 0.5 + 2.0 ** -24
    assert pm.fma_f32(p1, d1, np.float32(0.5)) == np.float32(0.5 + 2.0 ** -24)
    assert np.float32(np.float64(p1) * np.float64(d1) + 0.5) == np.float32(0.5 + 2.0 ** -23)
    # the same tie mirrored below zero
    assert pm.fma_f32(-p1, d1, np.float32(-0.5)) == np.float32(-(0.5 + 2.0 ** -24))
