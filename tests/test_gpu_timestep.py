"""Step-size control (cube_max_speed, cube_next_epoch, cube_next_epoch_limited).

cube_max_speed equals the largest |p| of the decoded momenta (the same FP32
values cube_decode returns); cube_next_epoch's epoch makes the fastest
particle's drift p_max * int da / (a^3 E) equal to the limit (checked with
the oracle's drift integral, an independent quadrature) unless a_max comes
first; and a run whose uniform steps make a particle jump more than a
coarse cell (the smallest-box realisation of the ensemble generator to
z = 0 with 1-byte codes) completes without a clamped migration when each
step is cut by cube_next_epoch.
"""
import numpy as np
import pytest

import synth
from oracle import cosmo

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


def _ctx(cube, w, xb, vb):
    om, ol, _ = w.omega()
    prm = cube.make_params(w.n_fine, w.n_particles, x_bytes=xb, v_bytes=vb, box=w.box, omega_m=om, omega_l=ol)
    return cube.cube_create(prm, torch.cuda.current_stream())


@pytest.mark.parametrize("xb,vb", [(1, 1), (2, 2), (4, 4)])
def test_max_speed_is_the_largest_decoded_momentum(cube, xb, vb):
    w = synth.WORKLOADS["pm64"]
    ic = synth.make_ics(w, n_part_side=32, n_fine=64)
    n = 32 ** 3
    ctx = _ctx(cube, dict_replace(w, n_part_side=32, n_fine=64), xb, vb)
    sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d if xb != 4 else 0.0)
        for i in range(3):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
        pos = np.empty((3, n), np.float32)
        vel = np.empty((3, n), np.float32)
        cube.cube_decode(ctx, pos, vel, None)
        assert cube.cube_max_speed(ctx) == float(np.max(np.abs(vel)))
    finally:
        cube.cube_destroy(ctx)


def dict_replace(w, **kw):
    import dataclasses
    return dataclasses.replace(w, **kw)


def test_next_epoch_limits_the_fastest_drift(cube):
    w = synth.WORKLOADS["pm256"]
    w = dict_replace(w, n_part_side=32, n_fine=64, box=60.0)
    ic = synth.make_ics(w)
    om, ol, _ = w.omega()
    ctx = _ctx(cube, w, 1, 1)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, 0.5, ic.sigma_1d)
        p = cube.cube_max_speed(ctx)
        for cells in (0.25, 0.5, 1.0):
            a_to = cube.cube_next_epoch(ctx, 1.0, cells)
            assert 0.5 < a_to <= 1.0
            drift = p * cosmo.drift_factor(0.5, a_to, om, ol)
            if a_to < 1.0:
                assert drift == pytest.approx(cells * 4, rel=1e-9)
            else:
                assert drift <= cells * 4 * (1 + 1e-12)
        assert cube.cube_next_epoch(ctx, 0.5000001, 0.5) == 0.5000001
        with pytest.raises(cube.CubeError):
            cube.cube_next_epoch(ctx, 0.4, 0.5)
        with pytest.raises(cube.CubeError):
            cube.cube_next_epoch(ctx, 1.0, 1.5)
    finally:
        cube.cube_destroy(ctx)


def test_adaptive_steps_keep_every_move_within_a_cell(cube):
    ens = synth.ensemble_c4(64)
    w = min(ens, key=lambda x: x.box / x.n_part_side)      # the finest fine cells
    w = dict_replace(w, n_part_side=32, n_fine=64, box=w.box * 32 / w.n_part_side)
    ic = synth.make_ics(w)
    ctx = _ctx(cube, w, 1, 1)
    targets = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        a, steps = w.a_init, 0
        for t in targets[1:]:
            while a < t:
                a_to = cube.cube_next_epoch(ctx, t, 0.5)
                cube.cube_pm_step(ctx, a, a_to)
                a, steps = a_to, steps + 1
                assert steps < 2000
        st = cube.cube_stats_get(ctx)                    # raises if a migration was clamped
        assert st.max_migration <= 1 and st.a == w.a_final
        assert steps >= w.n_steps
    finally:
        cube.cube_destroy(ctx)


def test_limited_epoch_accounts_for_force_and_expansion(cube):
    """cube_max_force and cube_next_epoch_limited (Section 2.3.3: velocity,
    acceleration and expansion limits).  The force bound equals the largest
    FD4 gradient component of the oracle's FP64 potential of the same store
    (1e-4) and bounds the oracle's particle forces; the returned epoch puts
    the kicked fastest particle's drift (p_max + F_max K(a_p, a_mid)) D(a, a_to)
    exactly at the limit when that binds (oracle integrals, 1e-9), is
    a * exp(max_dlna) when expansion binds, and equals cube_next_epoch before
    any step (no potential yet: F_max = 0)."""
    from oracle import mesh, pm
    from gpu_util import oracle_params, read_store
    w = dict_replace(synth.WORKLOADS["pm256"], n_part_side=32, n_fine=64, box=60.0)
    ic = synth.make_ics(w)
    om, ol, _ = w.omega()
    ctx = _ctx(cube, w, 1, 1)
    try:
        # the ICs' momenta scaled to those of a later epoch, so that the limits bind
        cube.cube_encode(ctx, ic.pos, ic.vel * 200.0, ic.ids, 0.3, ic.sigma_1d * 200.0)
        cells = 0.05
        assert cube.cube_max_force(ctx) == 0.0
        a_v = cube.cube_next_epoch(ctx, 1.0, cells)
        a_l, why = cube.cube_next_epoch_limited(ctx, 1.0, cells, 0.0)
        assert a_l == a_v < 1.0 and why == 1
        g = read_store(cube, ctx)
        prm = cube.make_params(64, 32 ** 3, box=w.box, omega_m=om, omega_l=ol)
        st = pm.Store(oracle_params(pm, prm, g["brick"]), g["counts"], g["vc"], g["chi"], g["nu"], g["ids"],
                      g["sigma"], g["a"], g["a_p"])
        ref = pm.step(st, 0.3, 0.31, keep_drifted=True)
        cube.cube_pm_step(ctx, 0.3, 0.31)
        f = cube.cube_max_force(ctx)
        phi = mesh.potential(pm.density(st), om, prm.deconv_power)
        want = max(float(np.max(np.abs(gr))) for gr in mesh.fd4_gradient(phi))
        assert f == pytest.approx(want, rel=1e-4)
        assert f >= float(np.max(np.abs(ref.extra["force"]))) * (1 - 1e-4)
        s = cube.cube_stats_get(ctx)
        p = cube.cube_max_speed(ctx)
        a0, ap = s.a, s.a_p
        a_to, why = cube.cube_next_epoch_limited(ctx, 1.0, cells, 0.0)
        assert why == 1 and a0 < a_to < cube.cube_next_epoch(ctx, 1.0, cells)
        d = (p + f * cosmo.kick_factor(ap, 0.5 * (a0 + a_to), om, ol)) * cosmo.drift_factor(a0, a_to, om, ol)
        assert d == pytest.approx(cells * 4, rel=1e-9)
        # the host-only bound with the context's epochs and maxima is the same call
        assert cube.cube_epoch_bound(om, ol, 4, a0, ap, 1.0, p, f, cells, 0.0) == (a_to, why)
        # expansion limit
        a_to, why = cube.cube_next_epoch_limited(ctx, 1.0, 1.0, 1e-3)
        assert why == 2 and a_to == pytest.approx(a0 * np.exp(1e-3), rel=1e-15)
        # a_max itself
        a_to, why = cube.cube_next_epoch_limited(ctx, a0 + 1e-6, 1.0, 0.0)
        assert why == 0 and a_to == a0 + 1e-6
        with pytest.raises(cube.CubeError):
            cube.cube_next_epoch_limited(ctx, 1.0, 0.0, 0.0)
    finally:
        cube.cube_destroy(ctx)
