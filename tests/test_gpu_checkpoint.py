"""Checkpoint of the compressed store (Section 2.3.1's {rho_c, v_c, chi_d,
nu_d, I_P}, plus sigma and the leapfrog epochs): save after steps, load
into a fresh context, and the store, its decode and every later step are
bit-identical to the context that never left the GPU; host and device
buffers give the same bytes; mismatched or corrupted checkpoints are
refused."""
import numpy as np
import pytest

import synth

from gpu_util import read_store

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


def _setup(cube, xb, vb, nps=32, id_bytes=4):
    w = synth.WORKLOADS["pm64"]
    ic = synth.make_ics(w, n_part_side=nps, n_fine=2 * nps)
    om, ol, _ = w.omega()
    prm = cube.make_params(2 * nps, nps ** 3, x_bytes=xb, v_bytes=vb, box=w.box, omega_m=om, omega_l=ol,
                           id_bytes=id_bytes)
    return w, ic, prm


def _decode(cube, ctx, n):
    out = (np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32))
    cube.cube_decode(ctx, *out)
    return out


@pytest.mark.parametrize("xb,vb,idb", [(1, 1, 4), (2, 2, 4), (1, 2, 4), (4, 4, 4), (1, 1, 1), (2, 1, 2)])
def test_checkpoint_round_trip_and_continuation(cube, xb, vb, idb):
    w, ic, prm = _setup(cube, xb, vb, id_bytes=idb)
    n = 32 ** 3
    sched = synth.uniform_schedule(w.a_init, 0.08, 6)
    a = cube.cube_create(prm, torch.cuda.current_stream())
    b = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        cube.cube_encode(a, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d if xb != 4 else 0.0)
        for i in range(3):
            cube.cube_pm_step(a, sched[i], sched[i + 1])
        size = cube.cube_checkpoint_size(prm)
        host = np.zeros(size, np.uint8)
        cube.cube_checkpoint_save(a, host)
        dev = torch.zeros(size, dtype=torch.uint8, device="cuda")
        cube.cube_checkpoint_save(a, dev)
        assert np.array_equal(dev.cpu().numpy(), host)
        cube.cube_checkpoint_load(b, host)
        for x, y in zip(_decode(cube, a, n), _decode(cube, b, n)):
            assert np.array_equal(x, y)
        for i in range(3, 6):
            cube.cube_pm_step(a, sched[i], sched[i + 1])
            cube.cube_pm_step(b, sched[i], sched[i + 1])
        if xb != 4:
            ga, gb = read_store(cube, a), read_store(cube, b)
            for k in ("counts", "offsets", "vc", "chi", "nu", "ids"):
                assert np.array_equal(ga[k], gb[k]), k
            assert ga["sigma"] == gb["sigma"] and ga["a"] == gb["a"] and ga["a_p"] == gb["a_p"]
        for x, y in zip(_decode(cube, a, n), _decode(cube, b, n)):
            assert np.array_equal(x, y)
        # the device copy loads the same way
        cube.cube_checkpoint_load(b, dev)
        sa = cube.cube_stats_get(b)
        assert sa.a == sched[3]
    finally:
        cube.cube_destroy(a)
        cube.cube_destroy(b)


def test_bad_checkpoints_are_refused(cube):
    w, ic, prm = _setup(cube, 1, 1)
    a = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        cube.cube_encode(a, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        size = cube.cube_checkpoint_size(prm)
        good = np.zeros(size, np.uint8)
        cube.cube_checkpoint_save(a, good)
        bad = good.copy()
        bad[0] ^= 1                                            # magic
        with pytest.raises(cube.CubeError) as e:
            cube.cube_checkpoint_load(a, bad)
        assert e.value.status == cube.CUBE_E_ARG
        bad = good.copy()
        bad[64] += 1                                           # counts no longer add up to N
        with pytest.raises(cube.CubeError) as e:
            cube.cube_checkpoint_load(a, bad)
        assert e.value.status == cube.CUBE_E_ARG
        bad = good.copy()
        cnt = bad[64:64 + 8].view(np.uint32)                   # the first two cells' counts
        cnt[0] = np.uint32(int(cnt[0]) + 2 ** 31)
        cnt[1] = np.uint32(int(cnt[1]) + 2 ** 31)              # + 2^32: the 32-bit sum still equals N
        assert int(good[64:].view(np.uint32)[:prm.n_fine ** 3 // 64].sum(dtype=np.uint32)) == \
            int(bad[64:].view(np.uint32)[:prm.n_fine ** 3 // 64].sum(dtype=np.uint32))
        with pytest.raises(cube.CubeError) as e:
            cube.cube_checkpoint_load(a, bad)
        assert e.value.status == cube.CUBE_E_ARG
        other = cube.make_params(64, 32 ** 3, x_bytes=1, v_bytes=2, box=prm.box, omega_m=prm.omega_m,
                                 omega_l=prm.omega_l)
        c2 = cube.cube_create(other, torch.cuda.current_stream())
        try:
            with pytest.raises(cube.CubeError) as e:
                cube.cube_checkpoint_load(c2, good)             # v_bytes differ
            assert e.value.status == cube.CUBE_E_ARG
        finally:
            cube.cube_destroy(c2)
        cube.cube_checkpoint_load(a, good)                     # the good one still loads
    finally:
        cube.cube_destroy(a)
