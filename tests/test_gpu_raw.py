"""The uncompressed FP32 store (x_bytes = v_bytes = 4) against the oracle's
uncompressed FP64 mode (oracle.pm.exact_step): the comparison arm of the
precision study of Section 3.

FP32 particles and a FP32 mesh against FP64 throughout: densities within
1e-5 of the mean, one step's positions within 1e-4 fine cells and momenta
within 1e-4 of their largest value; over the 10-step 64^3 run the RMS
displacement difference stays below 1e-3 fine cells and P(k) within 0.5%.
"""
import numpy as np
import pytest

import synth
from oracle import mesh, pm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cube():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_lib
    build_lib()
    import paper_1712_06121_gb300 as c
    torch.cuda.set_device(0)
    return c


def _setup(cube, nps, nf, name="pm64"):
    w = synth.WORKLOADS[name]
    ic = synth.make_ics(w, n_part_side=nps, n_fine=nf)
    om, ol, _ = w.omega()
    prm = cube.make_params(nf, nps ** 3, x_bytes=4, v_bytes=4, box=w.box, omega_m=om, omega_l=ol)
    ctx = cube.cube_create(prm, torch.cuda.current_stream())
    P = pm.Params(n_fine=nf, n_particles=nps ** 3, x_bytes=1, v_bytes=1, box=w.box, omega_m=om, omega_l=ol)
    return w, ic, prm, ctx, P


def _decode(cube, ctx, n):
    pos = np.empty((3, n), np.float32)
    vel = np.empty((3, n), np.float32)
    ids = np.empty(n, np.uint32)
    cube.cube_decode(ctx, pos, vel, ids)
    return pos, vel, ids


def _wrapped(d, n):
    return d - n * np.round(d / n)


def test_raw_store_round_trip_and_view(cube):
    w, ic, prm, ctx, P = _setup(cube, 16, 32)
    n = 16 ** 3
    try:
        pos_in = ic.pos.copy()
        pos_in[0, :5] += 32.0                    # periodic images
        pos_in[1, 5:9] -= 32.0
        cube.cube_encode(ctx, pos_in, ic.vel, ic.ids, w.a_init, 0.0)
        pos, vel, ids = _decode(cube, ctx, n)
        assert np.all((pos >= 0) & (pos < 32))
        assert np.max(np.abs(_wrapped(pos.astype(np.float64) - ic.pos, 32))) <= 4e-6
        assert np.array_equal(vel, ic.vel)
        assert np.array_equal(ids, ic.ids)
        st = cube.cube_state_view(ctx)
        assert st.x_bytes == 4 and st.v_bytes == 4 and st.sigma == 0.0
        assert not st.counts and not st.offsets and not st.vc
        with pytest.raises(cube.CubeError) as e:
            cube.cube_keep_drifted(ctx, True)
        assert e.value.status == cube.CUBE_E_STATE
        stats = cube.cube_stats_get(ctx)
        want = np.rint(ic.vel.astype(np.float64) * 2.0 ** 24).sum(axis=1) * 2.0 ** -24
        assert np.allclose(stats.momentum, want, rtol=0, atol=1e-9)
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("nps,nf", [(16, 32), (32, 64), (24, 48)])
def test_raw_density_matches_oracle(cube, nps, nf):
    w, ic, prm, ctx, P = _setup(cube, nps, nf)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, 0.0)
        rho = np.empty((nf, nf, nf), np.float32)
        cube.cube_density(ctx, rho)
        want = mesh.cic_deposit(np.mod(ic.pos.astype(np.float64), nf), nf, P.mass)
        assert np.max(np.abs(rho - want)) <= 1e-5
    finally:
        cube.cube_destroy(ctx)


def test_raw_step_matches_oracle_exact_step(cube):
    w, ic, prm, ctx, P = _setup(cube, 32, 64)
    n = 32 ** 3
    a0, a1 = w.a_init, w.a_init + 0.01
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, a0, 0.0)
        cube.cube_pm_step(ctx, a0, a1)
        pos, vel, _ = _decode(cube, ctx, n)
        st = cube.cube_stats_get(ctx)
        assert st.a == a1 and st.a_p == pytest.approx(0.5 * (a0 + a1))
    finally:
        cube.cube_destroy(ctx)
    ref = pm.exact_step(pm.exact_from(P, np.mod(ic.pos.astype(np.float64), 64), ic.vel, a0), a0, a1)
    assert np.max(np.abs(_wrapped(pos - ref.pos, 64))) <= 1e-4
    assert np.max(np.abs(vel - ref.vel)) <= 1e-4 * np.max(np.abs(ref.vel))


def test_raw_run_pm64_matches_oracle(cube):
    """The 64^3 / 128^3 EdS workload, 10 steps a = 0.02 -> 0.1."""
    w = synth.WORKLOADS["pm64"]
    w_, ic, prm, ctx, P = _setup(cube, w.n_part_side, w.n_fine)
    n = w.n_particles
    sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    nb = w.n_fine // 2
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, 0.0)
        for i in range(w.n_steps):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
        pos, vel, ids = _decode(cube, ctx, n)
        k, pk, nm = (np.empty(nb) for _ in range(3))
        cube.cube_power_spectrum(ctx, nb, k, pk, nm)
    finally:
        cube.cube_destroy(ctx)
    ref = pm.exact_run(pm.exact_from(P, np.mod(ic.pos.astype(np.float64), w.n_fine), ic.vel, w.a_init), sched)
    d = _wrapped(pos.astype(np.float64) - ref.pos, w.n_fine)
    assert np.sqrt(np.mean(np.sum(d * d, axis=0))) <= 1e-3
    rk, rp, rm = mesh.power_spectrum(ref.pos, w.n_fine, P.mass, w.box, nb)
    assert np.array_equal(nm, rm)
    sel = k < 0.5 * np.pi * w.n_fine / w.box
    assert np.max(np.abs(pk[sel] / rp[sel] - 1)) <= 5e-3
