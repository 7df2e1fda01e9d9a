"""Many simulations at once: uneven realisations of the ensemble generator,
each in its own context, spread over several CUDA streams and stepped in
interleaved order, give stores bit-identical to the same runs made one after
another on one stream (every sum that decides the store is an integer, so
the overlap cannot change a result).  Each run's own parity with the oracle
is the subject of the step tests.  The brick autotuner returns the fastest
valid brick side (results are brick-invariant: test_gpu_parity).
"""
import dataclasses

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


def _ensemble():
    """Six realisations of the ensemble generator (their boxes, sigma8 and
    seeds) at 16^3 .. 32^3 particles, 10 steps to a = 0.1."""
    sides = [16, 24, 32, 16, 24, 32]
    return [dataclasses.replace(w, n_part_side=s, n_fine=2 * s, a_final=0.1, n_steps=10)
            for w, s in zip(synth.ensemble_c4(len(sides)), sides)]


def _run(cube, ens, streams):
    ctxs = []
    for i, w in enumerate(ens):
        om, ol, _ = w.omega()
        prm = cube.make_params(w.n_fine, w.n_particles, x_bytes=1, v_bytes=1, box=w.box, omega_m=om, omega_l=ol)
        ctxs.append(cube.cube_create(prm, streams[i % len(streams)]))
    ics = [synth.make_ics(w) for w in ens]
    scheds = [synth.uniform_schedule(w.a_init, w.a_final, w.n_steps) for w in ens]
    try:
        for c, w, ic in zip(ctxs, ens, ics):
            cube.cube_encode(c, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        for k in range(max(w.n_steps for w in ens)):
            for c, w, sch in zip(ctxs, ens, scheds):
                if k < w.n_steps:
                    cube.cube_pm_step(c, sch[k], sch[k + 1])
        torch.cuda.synchronize()
        return [read_store(cube, c) for c in ctxs]
    finally:
        for c in ctxs:
            cube.cube_destroy(c)


def test_concurrent_streams_match_sequential(cube):
    ens = _ensemble()
    seq = _run(cube, ens, [torch.cuda.current_stream()])
    con = _run(cube, ens, [torch.cuda.Stream() for _ in range(3)])
    for w, gs, gc in zip(ens, seq, con):
        for key in ("counts", "offsets", "vc", "chi", "nu", "ids"):
            assert np.array_equal(gs[key], gc[key]), (w.name, key)
        assert gs["sigma"] == gc["sigma"]
        assert int(gc["counts"].sum()) == w.n_particles
        assert np.array_equal(np.sort(gc["ids"]), np.arange(w.n_particles, dtype=np.uint32))


def test_autotuned_brick_is_the_fastest_valid_one(cube):
    """cube_autotune_brick times each valid brick side and returns the
    fastest; sides that do not fit the mesh report -1."""
    w = dataclasses.replace(synth.ensemble_c4(1)[0], n_part_side=16, n_fine=32)
    ic = synth.make_ics(w)
    om, ol, _ = w.omega()
    prm = cube.make_params(w.n_fine, w.n_particles, box=w.box, omega_m=om, omega_l=ol)
    best, ms = cube.cube_autotune_brick(prm, ic.pos, ic.vel, w.a_init, ic.sigma_1d, 3)
    assert ms[2] == -1.0                      # 8 coarse cells per side: 2 bricks of 4, fewer than 3
    valid = {b: t for b, t in zip((1, 2, 4), ms) if t >= 0}
    assert best in valid and valid[best] == min(valid.values()) and all(t > 0 for t in valid.values())
    # a mesh of 4 coarse cells per side admits brick 1 only
    w2 = dataclasses.replace(w, n_part_side=8, n_fine=16)
    ic2 = synth.make_ics(w2)
    prm2 = cube.make_params(16, 8 ** 3, box=w.box, omega_m=om, omega_l=ol)
    best2, ms2 = cube.cube_autotune_brick(prm2, ic2.pos, ic2.vel, w.a_init, ic2.sigma_1d, 2)
    assert best2 == 1 and ms2[1] == -1.0 and ms2[2] == -1.0 and ms2[0] > 0
