"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Integer work (counts, offsets, order, chi, nu, ids) must be bit-exact when
both sides start from identical inputs: the same float particles for encode,
the GPU's exported drifted particles for the re-sort.  The fixed-point cell
velocities v_c are bit-exact too.  Densities (exact integer CIC weights on
both sides) within 1e-5 of the mean; the potential (FP32 FFT) within 1e-4 of
its largest value; the power spectrum within 1e-4 relative.
"""
import numpy as np
import pytest

import synth
from oracle import cosmo, layout, mesh, pm

from gpu_util import assert_store_equal, oracle_params, read_store

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


def _ics(nps, nf, name="pm64", seed=None):
    w = synth.WORKLOADS[name]
    return w, synth.make_ics(w, n_part_side=nps, n_fine=nf, seed=seed)


def _ctx(cube, nf, n, xb, vb, w, brick=0, deconv=2):
    om, ol, _ = w.omega()
    prm = cube.make_params(nf, n, x_bytes=xb, v_bytes=vb, box=w.box, omega_m=om, omega_l=ol, brick=brick,
                           deconv_power=deconv)
    return prm, cube.cube_create(prm, torch.cuda.current_stream())


CODES = [(1, 1), (1, 2), (2, 1), (2, 2)]


# ---------------------------------------------------------------- encode / decode
@pytest.mark.parametrize("xb,vb", CODES)
@pytest.mark.parametrize("nps,nf", [(32, 64), (24, 48)])
def test_encode_matches_oracle(cube, xb, vb, nps, nf):
    w, ic = _ics(nps, nf)
    prm, ctx = _ctx(cube, nf, nps ** 3, xb, vb, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        g = read_store(cube, ctx)
        P = oracle_params(pm, prm, g["brick"])
        ref = pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, g["sigma"], snap=False)
        assert g["sigma"] == pytest.approx(pm.codec.snap_sigma(ic.sigma_1d), rel=1e-14)
        assert_store_equal(g, ref, f"encode x{xb}v{vb}")
    finally:
        cube.cube_destroy(ctx)


def test_encode_measured_sigma(cube):
    w, ic = _ics(32, 64)
    prm, ctx = _ctx(cube, 64, 32 ** 3, 1, 2, w)
    try:
        cube.cube_encode(ctx, torch.from_numpy(ic.pos).cuda(), torch.from_numpy(ic.vel).cuda(), None,
                         w.a_init, 0.0)
        g = read_store(cube, ctx)
        ref = pm.encode(oracle_params(pm, prm, g["brick"]), ic.pos, ic.vel, None, w.a_init, 0.0)
        assert g["sigma"] == pytest.approx(ref.sigma, rel=1e-12)
        assert np.array_equal(g["ids"], ref.ids)          # NULL ids -> input index
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("xb,vb", CODES)
def test_decode_matches_oracle(cube, xb, vb):
    w, ic = _ics(32, 64)
    n = 32 ** 3
    prm, ctx = _ctx(cube, 64, n, xb, vb, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        g = read_store(cube, ctx)
        ref = pm.encode(oracle_params(pm, prm, g["brick"]), ic.pos, ic.vel, ic.ids, w.a_init, g["sigma"],
                        snap=False)
        pos = torch.empty((3, n), dtype=torch.float32, device="cuda")
        vel = torch.empty((3, n), dtype=torch.float32, device="cuda")
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        cube.cube_decode(ctx, pos, vel, ids)
        rpos, rvel, rids = pm.decode(ref)
        assert np.array_equal(pos.cpu().numpy(), rpos.astype(np.float32))
        assert np.array_equal(ids.cpu().numpy().view(np.uint32), rids)
        err = np.abs(vel.cpu().numpy() - rvel)
        assert np.max(err) <= 4e-7 * np.max(np.abs(rvel))
        # host-pointer path returns the same bytes
        hp = np.empty((3, n), np.float32)
        hv = np.empty((3, n), np.float32)
        cube.cube_decode(ctx, hp, hv, None)
        assert np.array_equal(hp, pos.cpu().numpy()) and np.array_equal(hv, vel.cpu().numpy())
    finally:
        cube.cube_destroy(ctx)


def test_section_2_1_worked_example_on_gpu(cube):
    """Section 2.1's example along x (N_c = 4, 1-byte codes): chi = (-128, 127,
    0, 60), rho_c = (1, 0, 2, 1) decode to x = (0.001953125, 2.998046875,
    2.501953125, 3.736328125) coarse cells; y and z sit in bin 0 of cell 0."""
    x = np.array([0.001953125, 2.998046875, 2.501953125, 3.736328125])
    n = 4
    pos = np.zeros((3, n), np.float32)
    pos[0] = 4 * x                      # fine units, R = 4
    pos[1] = pos[2] = 4 * 0.001953125
    vel = np.zeros((3, n), np.float32)
    prm = cube.make_params(16, n, x_bytes=1, v_bytes=1, box=10.0)
    ctx = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        cube.cube_encode(ctx, pos, vel, None, 0.5, 1.0)
        g = read_store(cube, ctx)
        assert g["chi"][0].tolist() == [-128, 127, 0, 60]
        assert g["chi"][1].tolist() == [-128] * 4
        row = layout.storage_index(np.arange(4), 0, 0, 4, g["brick"])
        assert g["counts"][row].tolist() == [1, 0, 2, 1]
        out = np.empty((3, n), np.float32)
        cube.cube_decode(ctx, out, np.empty((3, n), np.float32), None)
        assert np.array_equal(out[0].astype(np.float64) / 4, x)
    finally:
        cube.cube_destroy(ctx)


# ---------------------------------------------------------------- mesh
@pytest.mark.parametrize("nps,nf,xb", [(32, 64, 1), (24, 48, 2), (8, 16, 1), (12, 24, 1), (48, 96, 1)])
def test_density_matches_oracle(cube, nps, nf, xb):
    w, ic = _ics(nps, nf)
    prm, ctx = _ctx(cube, nf, nps ** 3, xb, 1, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        g = read_store(cube, ctx)
        ref = pm.encode(oracle_params(pm, prm, g["brick"]), ic.pos, ic.vel, ic.ids, w.a_init, g["sigma"],
                        snap=False)
        rho = np.empty((nf, nf, nf), np.float32)
        cube.cube_density(ctx, rho)
        want = pm.density(ref)
        assert np.max(np.abs(rho - want)) <= 1e-5
        assert np.sum(rho, dtype=np.float64) == pytest.approx(nf ** 3, rel=1e-6)
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("nps,nf,deconv", [(8, 16, 2), (12, 24, 2), (16, 32, 0), (24, 48, 2), (32, 64, 1),
                                           (48, 96, 2), (64, 128, 2), (96, 192, 2), (128, 256, 2),
                                           (192, 384, 2)])
def test_potential_matches_oracle(cube, nps, nf, deconv):
    w, ic = _ics(nps, nf)
    prm, ctx = _ctx(cube, nf, nps ** 3, 1, 1, w, deconv=deconv)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        rho = np.empty((nf, nf, nf), np.float32)
        cube.cube_density(ctx, rho)
        phi = np.empty((nf, nf, nf), np.float32)
        cube.cube_potential(ctx, phi)
        want = mesh.potential(rho.astype(np.float64), prm.omega_m, deconv)
        err = np.max(np.abs(phi - want)) / np.max(np.abs(want))
        assert err <= 1e-4, err
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("nps,nf", [(32, 64), (48, 96)])
def test_power_spectrum_matches_oracle(cube, nps, nf):
    w, ic = _ics(nps, nf)
    prm, ctx = _ctx(cube, nf, nps ** 3, 1, 2, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        g = read_store(cube, ctx)
        ref = pm.encode(oracle_params(pm, prm, g["brick"]), ic.pos, ic.vel, ic.ids, w.a_init, g["sigma"],
                        snap=False)
        nb = nf // 2
        k, p, m = (np.empty(nb) for _ in range(3))
        cube.cube_power_spectrum(ctx, nb, k, p, m)
        rk, rp, rm = pm.power_spectrum(ref, nb)
        assert np.array_equal(m, rm)
        assert np.allclose(k, rk, rtol=1e-12)
        assert np.allclose(p, rp, rtol=1e-4)
    finally:
        cube.cube_destroy(ctx)


# ---------------------------------------------------------------- the step
def _drifted(cube, ctx, n):
    cell = np.empty((3, n), np.int32)
    u = np.empty((3, n), np.float32)
    p = np.empty((3, n), np.float32)
    sig = cube.cube_debug_drifted(ctx, cell, u, p)
    return cell, u, p, sig


@pytest.mark.parametrize("xb,vb", CODES)
@pytest.mark.parametrize("nps,nf,brick", [(32, 64, 0), (32, 64, 2), (24, 48, 0), (16, 32, 1)])
def test_step_resort_is_bit_exact(cube, xb, vb, nps, nf, brick):
    """Fig. update_xp: the GPU's re-sorted store equals the oracle's re-encode
    of the GPU's drifted particles (codes, counts, order, v_c), for 3 steps."""
    w, ic = _ics(nps, nf)
    n = nps ** 3
    prm, ctx = _ctx(cube, nf, n, xb, vb, w, brick=brick)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        cube.cube_keep_drifted(ctx, True)
        sched = synth.uniform_schedule(w.a_init, 0.05, 3)
        for i in range(3):
            before = read_store(cube, ctx)
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            cell, u, p, sig = _drifted(cube, ctx, n)
            g = read_store(cube, ctx)
            P = oracle_params(pm, prm, g["brick"])
            # the drifted cells are the old store's cells in old storage order
            old = pm.Store(P, before["counts"], before["vc"], before["chi"], before["nu"], before["ids"],
                           before["sigma"], before["a"], before["a_p"])
            assert np.array_equal(np.stack(old.cells()), cell)
            ref = pm.encode_drifted(P, cell, u, p, before["ids"], sig, g["a"], g["a_p"])
            assert_store_equal(g, ref, f"step {i} x{xb}v{vb}")
    finally:
        cube.cube_destroy(ctx)


def _crowded_ics(nps, nf, w, a0, a1, seed=1712101):
    """The pm64 generator's particles at a later epoch with two dense blobs:
    3000 particles (sigma 1.5 fine cells) inside one brick of side 8 or 16
    fine cells and 2000 (sigma 1.5) on a corner where eight bricks meet,
    their momenta normal with a drift of half a fine cell per step.  Bricks
    then hold far more than the mean (clustered late epochs)."""
    ic = synth.make_ics(w, n_part_side=nps, n_fine=nf)
    rng = np.random.default_rng(seed)
    pos = ic.pos.astype(np.float64).copy()
    vel = ic.vel.astype(np.float64).copy()
    om, ol, _ = w.omega()
    sp = 0.5 / cosmo.drift_factor(a0, a1, om, ol)
    for (lo, hi), c, s in (((0, 3000), (44.2, 43.8, 44.5), 1.5), ((3000, 5000), (31.9, 32.1, 31.95), 1.5)):
        pos[:, lo:hi] = np.asarray(c)[:, None] + s * rng.standard_normal((3, hi - lo))
        vel[:, lo:hi] = sp * rng.standard_normal((3, hi - lo))
    return np.mod(pos, nf).astype(np.float32), vel.astype(np.float32), ic.ids


@pytest.mark.parametrize("xb,vb", [(1, 1), (2, 2)])
def test_uniformly_moving_lattice_translates_exactly(cube, xb, vb):
    """Degenerate case: particles on the lattice q = 2i + 1/2 fine cells all
    moving with one velocity.  Their CIC density is exactly uniform, so the
    potential and the force are exactly zero on the GPU (FP32) as in the
    oracle (FP64); every velocity code is 0 with v_c = v, and the whole
    store after each step equals the oracle's full step (Figs. update_xp and
    update_vp) bit for bit, the lattice translated across cells and the
    periodic edge."""
    nps, nf = 16, 32
    n = nps ** 3
    w = synth.WORKLOADS["pm64"]
    g1 = (2.0 * np.arange(nps) + 0.5).astype(np.float32)
    z, y, x = np.meshgrid(g1, g1, g1, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()]).astype(np.float32)
    om, ol, _ = w.omega()
    a0 = w.a_init
    sched = [a0, a0 * 1.3, a0 * 1.7, a0 * 2.2]
    # a bulk flow of about 0.6 fine cells per step in x, less in y and z
    sp = 0.6 / cosmo.drift_factor(sched[0], sched[1], om, ol)
    vel = np.broadcast_to(np.array([[sp], [-0.45 * sp], [0.2 * sp]], np.float32), (3, n)).copy()
    ids = np.arange(n, dtype=np.uint32)
    prm, ctx = _ctx(cube, nf, n, xb, vb, w)
    try:
        cube.cube_encode(ctx, pos, vel, ids, a0, 1.0)
        cube.cube_keep_drifted(ctx, True)
        g = read_store(cube, ctx)
        ref = pm.Store(oracle_params(pm, prm, g["brick"]), g["counts"], g["vc"], g["chi"], g["nu"], g["ids"],
                       g["sigma"], g["a"], g["a_p"])
        assert np.all(g["nu"] == 0)
        for i in range(3):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            f = np.empty((3, n), np.float32)
            cube.cube_debug_force(ctx, f)
            assert np.all(f == 0.0)
            ref = pm.step(ref, sched[i], sched[i + 1])
            g = read_store(cube, ctx)
            assert_store_equal(g, ref, f"lattice step {i}")
            assert g["sigma"] == ref.sigma
        st = cube.cube_stats_get(ctx)
        assert st.max_migration <= 1
    finally:
        cube.cube_destroy(ctx)


def test_a_single_particle(cube):
    """The smallest store: one particle.  Encode against the oracle; its
    self-force vanishes in the oracle (the same CIC kernel deposits and
    interpolates and the FD4 difference is antisymmetric, so a particle
    exerts no net force on itself), and the GPU's is within 1e-4 of the
    largest FD4 gradient of the potential (FP32 rounding of a potential
    whose one source holds the whole box's mass); the re-sorted store of
    each step equals the oracle's re-encode of the GPU's drifted particle."""
    nf, n = 32, 1
    w = synth.WORKLOADS["pm64"]
    pos = np.array([[13.3], [0.7], [31.9]], np.float32)
    vel = np.array([[0.8], [-0.3], [0.05]], np.float32)
    ids = np.array([7], np.uint32)
    prm, ctx = _ctx(cube, nf, n, 1, 2, w)
    try:
        cube.cube_encode(ctx, pos, vel, ids, w.a_init, 0.5)
        P = oracle_params(pm, prm, read_store(cube, ctx)["brick"])
        want = pm.encode(P, pos, vel, ids, w.a_init, 0.5)
        assert_store_equal(read_store(cube, ctx), want, "single particle encode")
        cube.cube_keep_drifted(ctx, True)
        sched = synth.uniform_schedule(w.a_init, 0.05, 2)
        for i in range(2):
            before = read_store(cube, ctx)
            old = pm.Store(P, before["counts"], before["vc"], before["chi"], before["nu"], before["ids"],
                           before["sigma"], before["a"], before["a_p"])
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            f = np.empty((3, n), np.float32)
            cube.cube_debug_force(ctx, f)
            x, _, _ = pm.decode(old)
            rho = mesh.cic_deposit(x, nf, P.mass)
            fref = mesh.force_at(x, rho, prm.omega_m, prm.deconv_power)
            phi = mesh.potential(rho, prm.omega_m, prm.deconv_power)
            gscale = max(np.max(np.abs(gr)) for gr in mesh.fd4_gradient(phi))
            assert gscale > 0
            assert np.max(np.abs(fref)) <= 1e-9 * gscale
            assert np.max(np.abs(f - fref)) <= 1e-4 * gscale
            cell, u, p, sig = _drifted(cube, ctx, n)
            g = read_store(cube, ctx)
            ref = pm.encode_drifted(P, cell, u, p, before["ids"], sig, g["a"], g["a_p"])
            assert_store_equal(g, ref, f"single particle step {i}")
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("xb,vb,brick", [(1, 1, 4), (2, 2, 4), (1, 2, 2)])
def test_sparse_bricks_resort_is_bit_exact(cube, xb, vb, brick):
    """Bricks with about one particle per coarse cell and a third of the
    cells empty (4096 particles at uniform random positions, 16^3 coarse
    cells): with bricks of side 4 a round of 32 consecutive particles spans
    up to 49 cell starts, more than the re-sort's per-warp binary search
    covers, so it finishes those lanes' cells by a walk; bricks of side 2
    hold 17 or fewer particles, so every warp's only round is partial.  The
    re-sorted store equals the oracle's re-encode of the drifted particles
    (codes, counts, order, v_c) for 3 steps."""
    w = synth.WORKLOADS["pm64"]
    nf, n = 64, 4096
    rng = np.random.default_rng(1712202)
    pos = rng.uniform(0.0, nf, (3, n)).astype(np.float32)
    vel = (0.3 * rng.standard_normal((3, n))).astype(np.float32)
    ids = np.arange(n, dtype=np.uint32)
    sched = synth.uniform_schedule(0.5, 0.515, 3)
    prm, ctx = _ctx(cube, nf, n, xb, vb, w, brick=brick)
    try:
        cube.cube_encode(ctx, pos, vel, ids, sched[0], 0.3)
        cube.cube_keep_drifted(ctx, True)
        for i in range(3):
            before = read_store(cube, ctx)
            assert np.count_nonzero(before["counts"] == 0) > before["counts"].size // 4
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            cell, u, p, sig = _drifted(cube, ctx, n)
            g = read_store(cube, ctx)
            P = oracle_params(pm, prm, g["brick"])
            old = pm.Store(P, before["counts"], before["vc"], before["chi"], before["nu"], before["ids"],
                           before["sigma"], before["a"], before["a_p"])
            assert np.array_equal(np.stack(old.cells()), cell)
            ref = pm.encode_drifted(P, cell, u, p, before["ids"], sig, g["a"], g["a_p"])
            assert_store_equal(g, ref, f"sparse step {i} x{xb}v{vb} brick {brick}")
        assert cube.cube_stats_get(ctx).max_migration <= 1
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("xb,vb,brick", [(1, 1, 4), (2, 2, 4), (1, 2, 2)])
def test_crowded_bricks_resort_is_bit_exact(cube, xb, vb, brick):
    """Bricks with more particles than one warp's share (re-sorted by a whole
    CTA) give the same store as the oracle's re-encode of the drifted
    particles: codes, counts, order and v_c, for 3 steps."""
    w = synth.WORKLOADS["pm64"]
    nps, nf = 32, 64
    n = nps ** 3
    sched = synth.uniform_schedule(0.5, 0.515, 3)
    pos, vel, ids = _crowded_ics(nps, nf, w, sched[0], sched[1])
    prm, ctx = _ctx(cube, nf, n, xb, vb, w, brick=brick)
    try:
        cube.cube_encode(ctx, pos, vel, ids, sched[0], 0.0)
        cube.cube_keep_drifted(ctx, True)
        for i in range(3):
            before = read_store(cube, ctx)
            nbc = before["brick"] ** 3
            assert before["counts"].reshape(-1, nbc).sum(axis=1).max() > 2048
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            cell, u, p, sig = _drifted(cube, ctx, n)
            g = read_store(cube, ctx)
            P = oracle_params(pm, prm, g["brick"])
            old = pm.Store(P, before["counts"], before["vc"], before["chi"], before["nu"], before["ids"],
                           before["sigma"], before["a"], before["a_p"])
            assert np.array_equal(np.stack(old.cells()), cell)
            ref = pm.encode_drifted(P, cell, u, p, before["ids"], sig, g["a"], g["a_p"])
            assert_store_equal(g, ref, f"crowded step {i} x{xb}v{vb} brick {brick}")
        assert cube.cube_stats_get(ctx).max_migration <= 1
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("crowded,xb,brick", [(False, 1, 0), (True, 1, 4), (True, 2, 2)])
def test_density_after_steps_matches_oracle(cube, crowded, xb, brick):
    """The deposit of re-sorted stores (after each of 3 steps) equals the
    oracle's CIC deposit exactly once rounded to FP32: both sum exact integer
    weights (the oracle's FP64 sums of dyadic weights are exact, the mass is
    8), near the lattice and in dense blobs where node values reach the
    hundreds and FP32 rounding alone exceeds 1e-5 of the mean."""
    w = synth.WORKLOADS["pm64"]
    nps, nf = 32, 64
    n = nps ** 3
    if crowded:
        sched = synth.uniform_schedule(0.5, 0.515, 3)
        pos, vel, ids = _crowded_ics(nps, nf, w, sched[0], sched[1])
        sigma = 0.0
    else:
        sched = synth.uniform_schedule(w.a_init, 0.05, 3)
        ic = synth.make_ics(w, n_part_side=nps, n_fine=nf)
        pos, vel, ids, sigma = ic.pos, ic.vel, ic.ids, ic.sigma_1d
    prm, ctx = _ctx(cube, nf, n, xb, 1, w, brick=brick)
    try:
        cube.cube_encode(ctx, pos, vel, ids, sched[0], sigma)
        for i in range(3):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            g = read_store(cube, ctx)
            st = pm.Store(oracle_params(pm, prm, g["brick"]), g["counts"], g["vc"], g["chi"], g["nu"], g["ids"],
                          g["sigma"], g["a"], g["a_p"])
            rho = np.empty((nf, nf, nf), np.float32)
            cube.cube_density(ctx, rho)
            want = pm.density(st)
            assert np.array_equal(rho, want.astype(np.float32)), f"step {i}: max |diff| {np.max(np.abs(rho - want))}"
    finally:
        cube.cube_destroy(ctx)


def test_step_matches_oracle_step(cube):
    """One step from the same store: the GPU's drifted offsets and kicked
    momenta agree with the oracle's FP64 step (FP32 force differences flip a
    few velocity codes by one bin at most)."""
    w, ic = _ics(32, 64)
    n = 32 ** 3
    prm, ctx = _ctx(cube, 64, n, 2, 2, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        g0 = read_store(cube, ctx)
        P = oracle_params(pm, prm, g0["brick"])
        st = pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, g0["sigma"], snap=False)
        cube.cube_keep_drifted(ctx, True)
        cube.cube_pm_step(ctx, w.a_init, w.a_init + 0.008)
        cell, u, p, sig = _drifted(cube, ctx, n)
        ref = pm.step(st, w.a_init, w.a_init + 0.008, keep_drifted=True)
        assert np.array_equal(ref.extra["cell_old"], cell)
        dp = np.abs(p - ref.extra["p"]).astype(np.float64)
        # decoded momenta differ by rounding (FP32 table vs FP64 Eq. v) or, for a
        # code decided on the other side of a threshold, by that code's bin width
        sig0 = g0["sigma"]
        vco = st.vc[:, layout.particle_cells(st.counts)].astype(np.float64)
        nu_r = np.abs(np.stack([pm.codec.vel_encode((ref.extra["p"][d] - vco[d]).astype(np.float32), sig0, 2)
                                for d in range(3)]))
        bw = np.abs(pm.codec.vel_decode_offset(np.minimum(nu_r + 1, 32767), sig0, 2)
                    - pm.codec.vel_decode_offset(nu_r, sig0, 2))
        ulp = np.spacing(np.abs(ref.extra["p"]).astype(np.float32)).astype(np.float64)
        flips = dp > 4 * ulp
        assert np.mean(flips) < 0.05
        assert np.all(dp <= 1.01 * bw + 4 * ulp)
        assert np.max(np.abs(u - ref.extra["u_new"])) < 1e-5
        assert sig == pytest.approx(ref.sigma, rel=1e-12)
    finally:
        cube.cube_destroy(ctx)


@pytest.mark.parametrize("name,nps,nf,brick,deconv", [("pm64", 32, 64, 4, 2), ("pm64", 32, 64, 2, 2),
                                                      ("pm64", 32, 64, 1, 1), ("pm64", 24, 48, 0, 2),
                                                      ("pm256", 64, 128, 0, 2), ("pm256", 48, 96, 2, 0)])
def test_force_matches_oracle(cube, name, nps, nf, brick, deconv):
    """Pass A's gathered force (Section 2.3.3, update_vp: -grad Phi by FD4,
    CIC-interpolated) at every particle, element by element against the
    oracle's FP64 force_at from the same store's positions: within 1e-4 of
    the largest |F| (FP32 FFTs and differences), for brick sides 1, 2, 4, a
    3 * 2^a mesh and every deconvolution power."""
    w, ic = _ics(nps, nf, name)
    n = nps ** 3
    prm, ctx = _ctx(cube, nf, n, 1, 1, w, brick=brick, deconv=deconv)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        before = read_store(cube, ctx)
        cube.cube_keep_drifted(ctx, True)
        cube.cube_pm_step(ctx, w.a_init, w.a_init + 0.004)
        f = np.empty((3, n), np.float32)
        cube.cube_debug_force(ctx, f)
    finally:
        cube.cube_destroy(ctx)
    P = oracle_params(pm, prm, before["brick"])
    st = pm.Store(P, before["counts"], before["vc"], before["chi"], before["nu"], before["ids"], before["sigma"],
                  before["a"], before["a_p"])
    pos, _, _ = pm.decode(st)
    want = mesh.force_at(pos, mesh.cic_deposit(pos, nf, P.mass), prm.omega_m, deconv)
    scale = np.max(np.abs(want))
    assert scale > 0
    err = np.max(np.abs(f - want)) / scale
    assert err <= 1e-4, err


@pytest.mark.parametrize("xb", [1, 2])
@pytest.mark.parametrize("sigma", [0.05, 0.7, 3.0, 40.0])
def test_two_byte_velocity_tables_are_exact(cube, xb, sigma):
    """2-byte velocity codes (Section 2.2, Eqs. v and nu): the step kernels
    read the decode values and thresholds as a fixed FP32 approximation of
    tan plus a 4-bit correction; every entry they rebuild equals the full
    table's, for codec scales over three decades, after the encode and after
    each step (each step builds the next codec)."""
    w, ic = _ics(16, 32)
    n = 16 ** 3
    prm, ctx = _ctx(cube, 32, n, xb, 2, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, sigma)
        bad, whole = cube.cube_debug_velocity_tables(ctx)
        assert bad == 0 and whole == 0, (bad, whole)
        sched = synth.uniform_schedule(w.a_init, 0.05, 2)
        for i in range(2):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            bad, whole = cube.cube_debug_velocity_tables(ctx)
            assert bad == 0 and whole == 0, (i, bad, whole)
    finally:
        cube.cube_destroy(ctx)
    prm, ctx = _ctx(cube, 32, n, xb, 1, w)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, sigma)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_debug_velocity_tables(ctx)
        assert e.value.status == cube.CUBE_E_ARG
    finally:
        cube.cube_destroy(ctx)


def _decoded_momentum_bound(st):
    """(FP64 sum of the oracle-decoded momenta, bound on the GPU's sum): the
    GPU sums FP32 decodes (v_c + table offset, each within one FP32 rounding
    of its value and one of the offset) rounded to multiples of 2^-24."""
    key = layout.particle_cells(st.counts)
    p = st.params
    off = np.stack([pm.codec.vel_decode_offset(st.nu[d], st.sigma, p.v_bytes) for d in range(3)])
    v = st.vc[:, key].astype(np.float64) + off
    tot = v.sum(axis=1)
    ulp = np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)
    ulo = np.spacing(np.abs(off).astype(np.float32)).astype(np.float64)
    bound = 0.5 * (ulp + ulo).sum(axis=1) + v.shape[1] * 2.0 ** -25 + 1e-12 * np.abs(v).sum(axis=1)
    return tot, bound


@pytest.mark.parametrize("xb,vb", [(1, 1), (2, 2), (1, 2)])
def test_store_sums_match_oracle(cube, xb, vb):
    """cube_stats (Section 2.3.3 bookkeeping): the mass is the reduction of
    the cell counts times the particle mass, N_f^3 exactly; the momentum is
    the device reduction of the decoded momenta, against the FP64 sum of the
    oracle's decode of the same store within the FP32-decode and 2^-24
    fixed-point bounds, after the encode and after each of 3 steps."""
    w, ic = _ics(32, 64)
    n = 32 ** 3
    prm, ctx = _ctx(cube, 64, n, xb, vb, w)
    sched = synth.uniform_schedule(w.a_init, 0.05, 3)
    vel = (ic.vel + np.array([[0.3], [-0.2], [0.15]], np.float32)).astype(np.float32)  # a bulk flow
    try:
        cube.cube_encode(ctx, ic.pos, vel, ic.ids, w.a_init, ic.sigma_1d)
        for i in range(4):
            if i:
                cube.cube_pm_step(ctx, sched[i - 1], sched[i])
            stats = cube.cube_stats_get(ctx)
            g = read_store(cube, ctx)
            st = pm.Store(oracle_params(pm, prm, g["brick"]), g["counts"], g["vc"], g["chi"], g["nu"], g["ids"],
                          g["sigma"], g["a"], g["a_p"])
            assert stats.mass == 64.0 ** 3
            want, bound = _decoded_momentum_bound(st)
            got = np.array(stats.momentum)
            assert np.all(np.abs(got - want) <= bound), (i, got, want, bound)
            assert np.max(np.abs(want)) > 100 * np.max(bound)       # the sums are far from trivial
    finally:
        cube.cube_destroy(ctx)


def test_full_run_pm64_matches_oracle(cube):
    """The 64^3 / 128^3 EdS x1v2 workload, 10 steps a = 0.02 -> 0.1: RMS
    displacement difference (matched by id) <= 1e-3 fine cells and P(k)
    within 0.5% for k < k_Nyquist / 2."""
    w = synth.WORKLOADS["pm64"]
    ic = synth.make_ics(w)
    n = w.n_particles
    prm, ctx = _ctx(cube, w.n_fine, n, w.x_bytes, w.v_bytes, w)
    sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        for i in range(w.n_steps):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
        pos = np.empty((3, n), np.float32)
        vel = np.empty((3, n), np.float32)
        ids = np.empty(n, np.uint32)
        cube.cube_decode(ctx, pos, vel, ids)
        nb = w.n_fine // 2
        k, pk, nm = (np.empty(nb) for _ in range(3))
        cube.cube_power_spectrum(ctx, nb, k, pk, nm)
        g0 = None
    finally:
        cube.cube_destroy(ctx)
    P = pm.Params(n_fine=w.n_fine, n_particles=n, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box)
    st = pm.run(pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d), sched)
    rpos, rvel, rids = pm.decode(st)
    order_g = np.argsort(ids)
    order_r = np.argsort(rids)
    d = pos[:, order_g].astype(np.float64) - rpos[:, order_r]
    d -= w.n_fine * np.round(d / w.n_fine)
    rms = np.sqrt(np.mean(np.sum(d * d, axis=0)))
    assert rms <= 1e-3, rms
    rk, rp, rm = pm.power_spectrum(st, nb)
    sel = k < 0.5 * np.pi * w.n_fine / w.box
    assert np.max(np.abs(pk[sel] / rp[sel] - 1)) <= 5e-3
    del g0


# ---------------------------------------------------------------- errors, determinism
def test_call_order_and_argument_errors(cube):
    w, ic = _ics(16, 32)
    prm, ctx = _ctx(cube, 32, 16 ** 3, 1, 1, w)
    try:
        with pytest.raises(cube.CubeError) as e:
            cube.cube_pm_step(ctx, 0.02, 0.03)
        assert e.value.status == cube.CUBE_E_STATE
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, 0.02, ic.sigma_1d)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_pm_step(ctx, 0.03, 0.04)
        assert e.value.status == cube.CUBE_E_STATE
        with pytest.raises(cube.CubeError) as e:
            cube.cube_pm_step(ctx, 0.02, 0.02)
        assert e.value.status == cube.CUBE_E_ARG
        with pytest.raises(cube.CubeError) as e:
            cube.cube_debug_drifted(ctx, np.empty((3, 4096), np.int32), np.empty((3, 4096), np.float32),
                                    np.empty((3, 4096), np.float32))
        assert e.value.status == cube.CUBE_E_STATE
    finally:
        cube.cube_destroy(ctx)


def test_migration_beyond_one_cell_is_latched(cube):
    """A step far too long for the mesh moves particles more than one coarse
    cell: the kernels clamp the move, the flag is latched and the next
    synchronising call reports CUBE_E_MIGRATION."""
    n = 16 ** 3
    g = np.arange(16) * 2 + 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()]).astype(np.float32)
    vel = np.zeros((3, n), np.float32)
    vel[0] = 50.0                                    # 50 fine cells x H0
    prm = cube.make_params(32, n, x_bytes=1, v_bytes=2, box=50.0)
    ctx = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        cube.cube_encode(ctx, pos, vel, None, 0.5, 1.0)
        cube.cube_pm_step(ctx, 0.5, 0.6)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_stats_get(ctx)
        assert e.value.status == cube.CUBE_E_MIGRATION
    finally:
        cube.cube_destroy(ctx)


def test_nonfinite_input_is_reported(cube):
    w, ic = _ics(16, 32)
    pos = ic.pos.copy()
    pos[1, 7] = np.nan
    prm, ctx = _ctx(cube, 32, 16 ** 3, 1, 1, w)
    try:
        cube.cube_encode(ctx, pos, ic.vel, ic.ids, 0.02, ic.sigma_1d)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_stats_get(ctx)
        assert e.value.status == cube.CUBE_E_OVERFLOW
    finally:
        cube.cube_destroy(ctx)


def _run_decoded(cube, ic, w, nps, nf, brick, steps=3):
    n = nps ** 3
    prm, ctx = _ctx(cube, nf, n, 1, 2, w, brick=brick)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        sched = synth.uniform_schedule(w.a_init, 0.05, steps)
        for i in range(steps):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
        pos, vel, ids = np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32)
        cube.cube_decode(ctx, pos, vel, ids)
        o = np.argsort(ids)
        return pos[:, o], vel[:, o], read_store(cube, ctx)
    finally:
        cube.cube_destroy(ctx)


def test_runs_are_deterministic_and_brick_invariant(cube):
    """Section 3: different tilings give exactly the same results.  Two runs
    are bit-identical, and brick sides 1, 2, 4 give the same particles."""
    w, ic = _ics(32, 64)
    a = _run_decoded(cube, ic, w, 32, 64, 4)
    b = _run_decoded(cube, ic, w, 32, 64, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for k in ("counts", "chi", "nu", "ids", "vc"):
        assert np.array_equal(a[2][k], b[2][k])
    for brick in (1, 2):
        c = _run_decoded(cube, ic, w, 32, 64, brick)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])


@pytest.mark.parametrize("id_bytes", [1, 2])
def test_narrow_particle_ids_follow_their_particles(cube, id_bytes):
    """Section 2.1's PID array I_P with n_I = 1 or 2 bytes per particle (for
    instance particle types): the low n_I bytes of each ID travel with their
    particle through encode and three re-sorts exactly as the 4-byte IDs do,
    and the particles themselves are those of the 4-byte run."""
    w, ic = _ics(32, 64)
    n = 32 ** 3
    ids = np.random.default_rng(5).integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    out = {}
    for nb in (4, id_bytes):
        om, ol, _ = w.omega()
        prm = cube.make_params(64, n, x_bytes=1, v_bytes=2, id_bytes=nb, box=w.box, omega_m=om, omega_l=ol)
        ctx = cube.cube_create(prm, torch.cuda.current_stream())
        try:
            cube.cube_encode(ctx, ic.pos, ic.vel, ids, w.a_init, ic.sigma_1d)
            sched = synth.uniform_schedule(w.a_init, 0.05, 3)
            for i in range(3):
                cube.cube_pm_step(ctx, sched[i], sched[i + 1])
            g = read_store(cube, ctx)
            pos, vel, got = np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32)
            cube.cube_decode(ctx, pos, vel, got)
            out[nb] = (g, pos, vel, got)
        finally:
            cube.cube_destroy(ctx)
    mask = np.uint32((1 << (8 * id_bytes)) - 1)
    wide, narrow = out[4], out[id_bytes]
    for k in ("counts", "chi", "nu", "vc"):
        assert np.array_equal(wide[0][k], narrow[0][k])
    assert np.array_equal(wide[1], narrow[1]) and np.array_equal(wide[2], narrow[2])
    assert np.array_equal(wide[3] & mask, narrow[3])
    assert np.array_equal(narrow[0]["ids"], narrow[3])
