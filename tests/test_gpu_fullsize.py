"""Parity at the benchmark's full size: 256^3 particles, 512^3 mesh, x1v1,
LCDM, the launch configuration bench.py times.

The oracle handles this size in full (numpy, a few GB of host memory, about
a minute): the whole density and potential of the encoded store, and the
whole re-sorted store after one step, re-encoded by the oracle from the
GPU's drifted particles (bit-exact integers and v_c).
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


def test_full_size_mesh_and_resort_parity(cube):
    w = synth.WORKLOADS["pm256"]
    ic = synth.make_ics(w)
    n, nf = w.n_particles, w.n_fine
    om, ol, _ = w.omega()
    prm = cube.make_params(nf, n, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box, omega_m=om, omega_l=ol)
    ctx = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        cube.cube_encode(ctx, torch.from_numpy(ic.pos).cuda(), torch.from_numpy(ic.vel).cuda(),
                         torch.from_numpy(ic.ids.view(np.int32)).cuda(), w.a_init, ic.sigma_1d)
        g0 = read_store(cube, ctx)
        P = oracle_params(pm, prm, g0["brick"])
        ref0 = pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, g0["sigma"], snap=False)
        assert_store_equal(g0, ref0, "encode at full size")

        rho = torch.empty((nf, nf, nf), dtype=torch.float32, device="cuda")
        cube.cube_density(ctx, rho)
        want = pm.density(ref0)
        assert float(np.max(np.abs(rho.cpu().numpy() - want))) <= 1e-5
        phi = torch.empty((nf, nf, nf), dtype=torch.float32, device="cuda")
        cube.cube_potential(ctx, phi)
        want_phi = mesh.potential(want, om, prm.deconv_power)
        del want
        err = np.max(np.abs(phi.cpu().numpy() - want_phi)) / np.max(np.abs(want_phi))
        del phi
        assert err <= 1e-4, err

        cube.cube_keep_drifted(ctx, True)
        sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
        cube.cube_pm_step(ctx, sched[0], sched[1])
        cell = np.empty((3, n), np.int32)
        u = np.empty((3, n), np.float32)
        p = np.empty((3, n), np.float32)
        f = np.empty((3, n), np.float32)
        sig = cube.cube_debug_drifted(ctx, cell, u, p)
        cube.cube_debug_force(ctx, f)
        g1 = read_store(cube, ctx)
        assert np.array_equal(np.stack(ref0.cells()), cell)

        # force, kick and drift of a sample of particles against the oracle's
        # FP64 potential of the same store (Section 2.3.3 update_vp, Fig. update_xp)
        rng = np.random.default_rng(1712)
        idx = np.sort(rng.choice(n, 200_000, replace=False))
        pos0, _, _ = pm.decode(ref0)
        fref = mesh.force_at_points(want_phi, pos0[:, idx])
        del want_phi
        ferr = np.max(np.abs(f[:, idx] - fref)) / np.max(np.abs(fref))
        assert ferr <= 1e-4, ferr
        key = layout.particle_cells(ref0.counts)[idx]
        nb = 2 ** (8 * P.x_bytes)
        u0 = (ref0.chi[:, idx].astype(np.float64) + nb // 2 + 0.5) / nb
        a_mid = 0.5 * (sched[0] + sched[1])
        kf = cosmo.kick_factor(ref0.a_p, a_mid, om, ol)
        dc = np.float32(cosmo.drift_factor(sched[0], sched[1], om, ol) / P.ratio)
        vco = ref0.vc[:, key]
        p2, u2 = pm.kick_drift(P, u0, vco, ref0.nu[:, idx], ref0.sigma, fref, kf, dc)
        # the kicked momenta as decoded: equal up to the FP32 rounding of the
        # decode (table entry + v_c against FP64 Eq. v), except where the FP32
        # force decides a velocity code on the other side of a threshold,
        # which moves the momentum by at most that code's bin width
        dp = np.abs(p[:, idx] - p2).astype(np.float64)
        # the decode rounds v_c + offset in FP32: an ulp of the larger term
        mag = np.maximum(np.abs(p2), np.maximum(np.abs(vco), np.abs(p2 - vco)))
        ulp = np.spacing(mag.astype(np.float32)).astype(np.float64)
        flips = dp > 4 * ulp
        assert np.mean(flips) < 1e-3, np.mean(flips)
        nu_r = np.abs(np.stack([pm.codec.vel_encode((p2[d] - vco[d]).astype(np.float32), ref0.sigma, P.v_bytes)
                                for d in range(3)]))
        lim = pm.codec.nu_max(P.v_bytes)
        bw = np.abs(pm.codec.vel_decode_offset(np.minimum(nu_r + 1, lim), ref0.sigma, P.v_bytes)
                    - pm.codec.vel_decode_offset(nu_r, ref0.sigma, P.v_bytes))
        assert np.all(dp <= 1.01 * bw + 4 * ulp)
        # the drift from the GPU's own momenta: the offset rounded once, bit for bit
        assert np.array_equal(u[:, idx], pm.fma_f32(p[:, idx], np.broadcast_to(dc, u0.shape), u0))
        assert np.max(np.abs(u[:, idx] - u2)) <= np.max(1.01 * bw + 4 * ulp) * float(dc) + 1e-6
        ref1 = pm.encode_drifted(P, cell, u, p, g0["ids"], sig, g1["a"], g1["a_p"])
        assert_store_equal(g1, ref1, "one step at full size")
        st = cube.cube_stats_get(ctx)
        assert st.max_migration <= 1
    finally:
        cube.cube_destroy(ctx)
