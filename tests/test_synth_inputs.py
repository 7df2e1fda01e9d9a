"""The seeded input generators (no PM arithmetic) behind the ensemble and
serving workloads: the serving request stream has the stated distribution,
and rescaling a Zel'dovich realisation's amplitude equals generating it with
the scaled sigma8 (displacements, momenta and the velocity scale are linear
in the amplitude), to FP32 rounding."""
import dataclasses

import numpy as np

import synth


def test_serving_stream_follows_its_recipe():
    reqs = synth.serving_c5(400, rate=20.0, seed=7)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 20.0) < 0.01                    # Poisson: mean gap 1/rate
    ws = [r.workload for r in reqs]
    assert {w.n_part_side for w in ws} == {64, 96, 128, 192, 256}
    for w in ws:
        assert w.n_fine == 2 * w.n_part_side and w.box == 300.0 * w.n_part_side / 256
        assert 10 <= w.n_steps <= 60 and 0.7 <= w.sigma8 <= 0.9
        assert w.a_final == min(1.0, 0.02 + 0.0196 * w.n_steps) and w.x_bytes == w.v_bytes == 1
    assert len({w.seed for w in ws}) == len(ws)
    assert synth.serving_c5(400, rate=20.0, seed=7) == reqs      # seeded


def test_rescaled_realisation_equals_the_regenerated_one():
    w = dataclasses.replace(synth.WORKLOADS["pm64"], n_part_side=16, n_fine=32)
    ic = synth.make_ics(w)
    same = synth.rescaled_ics(ic, 1.0)
    assert np.array_equal(same.pos, ic.pos) and np.array_equal(same.vel, ic.vel)
    for f in (0.75, 1.1):
        got = synth.rescaled_ics(ic, f)
        want = synth.make_ics(dataclasses.replace(w, sigma8=w.sigma8 * f))
        d = got.pos.astype(np.float64) - want.pos
        d -= 32 * np.round(d / 32)
        assert np.max(np.abs(d)) <= 1e-5
        assert np.max(np.abs(got.vel - want.vel)) <= 1e-6 * np.max(np.abs(want.vel))
        assert abs(got.sigma_1d / want.sigma_1d - 1) < 1e-12
        assert np.array_equal(got.ids, ic.ids)
        assert np.all((got.pos >= 0) & (got.pos < 32))


def test_ensemble_follows_its_recipe():
    ws = synth.ensemble_c4(64)
    assert len(ws) == 64 and [w.seed for w in ws] == list(range(64))
    assert {w.n_part_side for w in ws} == {32, 48, 64, 96, 128}
    for w in ws:
        assert w.n_fine == 2 * w.n_part_side and 50.0 <= w.box <= 400.0 and 0.7 <= w.sigma8 <= 0.9
        assert (w.a_init, w.a_final, w.n_steps, w.x_bytes, w.v_bytes, w.cosmo_kind) == (0.02, 1.0, 30, 1, 1, "lcdm")
    assert len({(w.box, w.sigma8) for w in ws}) == 64                # every realisation differs
    assert synth.ensemble_c4(64) == ws                                # seeded


def test_philox_known_answers():
    """The initial conditions' noise generator reproduces the published
    Philox-4x32-10 known-answer vectors (tests/golden/philox4x32_10_kat.txt)."""
    import os
    from synth.philox import philox4x32
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = [[int(x, 16) for x in line.split()] for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        got = philox4x32(*[np.array([x], np.uint32) for x in r[:4]], r[4], r[5])
        assert [int(g[0]) for g in got] == r[6:]


def test_white_noise_is_keyed_by_wave_vector():
    """A Fourier mode draws the same noise at every grid size (the counter is
    the integer wave-vector), the kx = 0 plane is Hermitian, and DC and the
    Nyquist planes are zero."""
    from synth.ics import white_noise_modes
    a, b = white_noise_modes(16, 1712002), white_noise_modes(32, 1712002)
    f16 = np.fft.fftfreq(16, 1.0 / 16).astype(int)
    for iz, nz in enumerate(f16):
        for iy, ny in enumerate(f16):
            for nx in range(8):
                if max(abs(nz), abs(ny), nx) < 8:
                    assert a[iz, iy, nx] == b[nz % 32, ny % 32, nx]
    for iz, nz in enumerate(f16):
        for iy, ny in enumerate(f16):
            assert a[(-nz) % 16, (-ny) % 16, 0] == np.conj(a[iz, iy, 0])
    assert a[0, 0, 0] == 0 and np.all(a[8] == 0) and np.all(a[:, 8] == 0) and np.all(a[:, :, 8] == 0)
    live = np.abs(b[b != 0]) ** 2
    assert abs(live.mean() - 1.0) < 0.05
