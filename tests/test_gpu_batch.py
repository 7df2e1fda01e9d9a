"""Batches: several simulations of the same geometry stepped with one launch
per kernel (cube_batch_*).

* Every member's store (counts, offsets, v_c, codes, ids, codec scale) after
  each batch step is bit-identical to the same simulation stepped alone on a
  plain context with the same epochs: the batch runs the same deterministic
  kernels with each member's own epochs, kick and drift factors (Section 3:
  the result does not depend on how the work is tiled).
* A member that sits a step out keeps its store; it then continues alone
  (cube_pm_step), and the batch refuses to step it with the others.
* cube_batch_next_epochs equals cube_next_epoch member by member, and its
  non-blocking form (enqueue, then poll) gives the same epochs.
* One batch step launches 16 kernels whatever the member count.
* The mesh half solved ahead (cube_batch_solve), for every member or for
  some, gives the same stores, and each potential is solved once.
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


def _members(nps, xb, vb, k=4):
    base = synth.WORKLOADS["pm256"]
    out = []
    for i in range(k):
        w = dataclasses.replace(base, name=f"m{i}", n_part_side=nps, n_fine=2 * nps, box=40.0 + 35.0 * i,
                                sigma8=0.7 + 0.05 * i, seed=1712300 + i, x_bytes=xb, v_bytes=vb)
        out.append((w, synth.make_ics(w)))
    return out


def _params(cube, w):
    om, ol, _ = w.omega()
    return cube.make_params(w.n_fine, w.n_particles, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                            omega_m=om, omega_l=ol)


STORE_KEYS = ("counts", "offsets", "vc", "chi", "nu", "ids")


@pytest.mark.parametrize("nps,xb,vb,ahead", [(32, 1, 1, "none"), (24, 2, 2, "none"), (16, 1, 2, "none"),
                                            (32, 1, 1, "all"), (24, 2, 2, "some")])
def test_batch_members_equal_their_runs_alone(cube, nps, xb, vb, ahead):
    mem = _members(nps, xb, vb)
    k = len(mem)
    nsteps = 5
    # each member its own epochs: a = 0.02 -> 0.06 + 0.02 i in uniform steps
    scheds = [synth.uniform_schedule(0.02, 0.06 + 0.02 * i, nsteps) for i in range(k)]
    stream = torch.cuda.current_stream()
    b = cube.cube_batch_create([_params(cube, w) for w, _ in mem], stream)
    try:
        ctxs = [cube.cube_batch_member(b, i) for i in range(k)]
        for c, (w, ic) in zip(ctxs, mem):
            cube.cube_encode(c, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        got = []
        l0 = cube.cube_batch_launches(b)
        for s in range(nsteps):
            if ahead != "none":
                flags = [1] * k if ahead == "all" else [i % 2 for i in range(k)]
                cube.cube_batch_solve(b, flags)
                cube.cube_batch_solve(b, flags)                  # already solved: no launches
            cube.cube_batch_step(b, [sc[s] for sc in scheds], [sc[s + 1] for sc in scheds])
            got.append([read_store(cube, c) for c in ctxs])
        # 10 launches of the particle half per step, 6 of the mesh half per solve
        assert cube.cube_batch_launches(b) - l0 == (16 if ahead != "some" else 22) * nsteps
        for c in ctxs:
            st = cube.cube_stats_get(c)                      # raises on a latched device error
            assert st.steps == nsteps and st.max_migration <= 1
    finally:
        cube.cube_batch_destroy(b)
    for i, (w, ic) in enumerate(mem):
        ctx = cube.cube_create(_params(cube, w), stream)
        try:
            cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
            for s in range(nsteps):
                cube.cube_pm_step(ctx, scheds[i][s], scheds[i][s + 1])
                want = read_store(cube, ctx)
                g = got[s][i]
                for key in STORE_KEYS:
                    assert np.array_equal(g[key], want[key]), (i, s, key)
                assert g["sigma"] == want["sigma"] and g["a"] == want["a"] and g["a_p"] == want["a_p"]
        finally:
            cube.cube_destroy(ctx)


def test_a_member_that_sits_out_keeps_its_store_and_continues_alone(cube):
    mem = _members(16, 1, 1, k=3)
    stream = torch.cuda.current_stream()
    b = cube.cube_batch_create([_params(cube, w) for w, _ in mem], stream)
    try:
        ctxs = [cube.cube_batch_member(b, i) for i in range(3)]
        for c, (w, ic) in zip(ctxs, mem):
            cube.cube_encode(c, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        cube.cube_batch_step(b, [0.02] * 3, [0.03] * 3)
        before = read_store(cube, ctxs[1])
        cube.cube_batch_step(b, [0.03] * 3, [0.04, 0.03, 0.04])     # member 1 sits out
        after = read_store(cube, ctxs[1])
        for key in STORE_KEYS:
            assert np.array_equal(before[key], after[key]), key
        assert after["a"] == 0.03
        with pytest.raises(cube.CubeError) as e:
            cube.cube_batch_step(b, [0.04, 0.03, 0.04], [0.05] * 3)
        assert e.value.status == cube.CUBE_E_STATE
        cube.cube_pm_step(ctxs[1], 0.03, 0.04)                       # alone, on the batch's stream
        cube.cube_batch_step(b, [0.04] * 3, [0.05] * 3)              # all caught up
        for c in ctxs:
            assert cube.cube_stats_get(c).a == 0.05
    finally:
        cube.cube_batch_destroy(b)


def test_batch_next_epochs_equal_cube_next_epoch(cube):
    mem = _members(24, 1, 1, k=3)
    stream = torch.cuda.current_stream()
    b = cube.cube_batch_create([_params(cube, w) for w, _ in mem], stream)
    try:
        ctxs = [cube.cube_batch_member(b, i) for i in range(3)]
        for c, (w, ic) in zip(ctxs, mem):
            cube.cube_encode(c, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        cube.cube_batch_step(b, [0.02] * 3, [0.05] * 3)
        a_max = np.array([0.5, 0.05, 0.9])                           # member 1: no room to step
        got = cube.cube_batch_next_epochs(b, a_max, 0.5)
        assert got[1] == 0.05
        for i in (0, 2):
            assert got[i] == cube.cube_next_epoch(ctxs[i], a_max[i], 0.5)
        cube.cube_batch_epochs_enqueue(b)                            # the same, without waiting
        polled = None
        for _ in range(1000000):
            polled = cube.cube_batch_epochs_poll(b, a_max, 0.5)
            if polled is not None:
                break
        assert np.array_equal(polled, got)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_batch_epochs_poll(b, a_max, 0.5)               # nothing in flight
        assert e.value.status == cube.CUBE_E_STATE
        with pytest.raises(cube.CubeError) as e:
            cube.cube_batch_create([_params(cube, mem[0][0]), cube.make_params(64, 32 ** 3)], stream)
        assert e.value.status == cube.CUBE_E_ARG                     # members must share the geometry
    finally:
        cube.cube_batch_destroy(b)
