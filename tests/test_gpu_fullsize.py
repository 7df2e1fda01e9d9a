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
from oracle import mesh, pm

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
        del want_phi
        assert err <= 1e-4, err

        cube.cube_keep_drifted(ctx, True)
        sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
        cube.cube_pm_step(ctx, sched[0], sched[1])
        cell = np.empty((3, n), np.int32)
        u = np.empty((3, n), np.float32)
        p = np.empty((3, n), np.float32)
        sig = cube.cube_debug_drifted(ctx, cell, u, p)
        g1 = read_store(cube, ctx)
        assert np.array_equal(np.stack(ref0.cells()), cell)
        ref1 = pm.encode_drifted(P, cell, u, p, g0["ids"], sig, g1["a"], g1["a_p"])
        assert_store_equal(g1, ref1, "one step at full size")
        st = cube.cube_stats_get(ctx)
        assert st.max_migration <= 1
    finally:
        cube.cube_destroy(ctx)
