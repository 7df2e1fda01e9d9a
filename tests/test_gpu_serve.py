"""Serving (continuous batching, the C5 row): many simulations through one
cube_server on several streams.

* Alone vs mix: each request's decoded particles (positions, momenta, ids)
  and P(k) mode counts are bit-identical to the same simulation run alone on
  a plain context (cube_create ... cube_power_spectrum): the step's kernels
  are deterministic and every work buffer a step reads it has first written,
  so sharing a stream's work area with other requests cannot change a
  result.  The P(k) bins' FP64 sums are accumulated with shared-memory
  atomics, so k and P(k) agree to rounding (1e-12 relative).
* Budget: the device bytes held (resident states + work areas) never exceed
  the budget while requests queue for memory; admission is in arrival order;
  releasing a request returns its state bytes.
* Arguments: bad epochs, step counts and bins are refused; a request larger
  than the whole budget is refused with CUBE_E_NOMEM.
* Velocity-limited steps: a request whose epochs are waypoints takes the
  same steps, and gives the same particles, as the cube_next_epoch loop.
"""
import dataclasses

import numpy as np
import pytest

import synth

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


def _mix():
    """Uneven realisations of the ensemble generator: 16^3 .. 48^3 particles,
    1- and 2-byte velocity codes, 3 .. 9 steps."""
    sides = [16, 32, 24, 48, 16, 32, 24]
    steps = [5, 3, 9, 4, 7, 6, 3]
    out = []
    for i, (w, s, n) in enumerate(zip(synth.ensemble_c4(len(sides)), sides, steps)):
        w = dataclasses.replace(w, n_part_side=s, n_fine=2 * s, a_final=0.1, n_steps=n,
                                v_bytes=1 + (i % 2))
        out.append(w)
    return out


def _params(cube, w):
    om, ol, _ = w.omega()
    return cube.make_params(w.n_fine, w.n_particles, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                            omega_m=om, omega_l=ol)


def _alone(cube, w, ic, nb):
    """The plain path: one context, one simulation."""
    ctx = cube.cube_create(_params(cube, w), torch.cuda.current_stream())
    n = w.n_particles
    try:
        sch = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        for i in range(w.n_steps):
            cube.cube_pm_step(ctx, sch[i], sch[i + 1])
        k, pk, nm = (np.empty(nb) for _ in range(3))
        cube.cube_power_spectrum(ctx, nb, k, pk, nm)
        pos, vel, ids = np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32)
        cube.cube_decode(ctx, pos, vel, ids)
        return k, pk, nm, pos, vel, ids
    finally:
        cube.cube_destroy(ctx)


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def test_requests_in_a_mix_equal_their_runs_alone(cube):
    mix = _mix()
    ics = [synth.make_ics(w) for w in mix]
    nb = 8
    srv = cube.cube_server_create(8 << 30, n_streams=3, max_running=16)
    try:
        keep, tickets = [], []
        for w, ic in zip(mix, ics):
            host = (_pinned(ic.pos), _pinned(ic.vel), _pinned(ic.ids.view(np.int32)))
            keep.append(host)
            sch = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
            tickets.append(cube.cube_server_submit(srv, _params(cube, w), *host, ic.sigma_1d, sch, nb))
        cube.cube_server_drain(srv)
        for w, ic, t in zip(mix, ics, tickets):
            info = cube.cube_server_info(srv, t)
            assert info.state == cube.CUBE_REQ_DONE, (w.name, info.error)
            assert info.steps_enqueued == info.n_steps == w.n_steps
            assert 0 <= info.t_submit <= info.t_admit <= info.t_done
            k, pk, nm = (np.empty(nb) for _ in range(3))
            cube.cube_server_result(srv, t, k, pk, nm)
            n = w.n_particles
            pos, vel, ids = np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32)
            cube.cube_server_decode(srv, t, pos, vel, ids)
            a = _alone(cube, w, ic, nb)
            for got, want in zip((nm, pos, vel, ids), a[2:]):
                assert np.array_equal(got, want), w.name
            assert np.allclose(k, a[0], rtol=1e-12, atol=0) and np.allclose(pk, a[1], rtol=1e-12, atol=0)
    finally:
        cube.cube_server_destroy(srv)


def test_budget_bounds_device_bytes_and_admission_is_fifo(cube):
    mix = _mix()[:5]
    ics = [synth.make_ics(w) for w in mix]
    sizes = [cube.cube_server_sizes(_params(cube, w)) for w in mix]
    # room for the largest work area per stream plus about two resident states
    budget = 2 * max(wb for _, wb in sizes) + 2 * max(sb for sb, _ in sizes)
    srv = cube.cube_server_create(budget, n_streams=2, max_running=8)
    try:
        keep, tickets = [], []
        for w, ic in zip(mix, ics):
            host = (_pinned(ic.pos), _pinned(ic.vel), _pinned(ic.ids.view(np.int32)))
            keep.append(host)
            sch = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
            tickets.append(cube.cube_server_submit(srv, _params(cube, w), *host, ic.sigma_1d, sch, 4))
        done = set()
        peak = 0
        for _ in range(1000000):
            cube.cube_server_pump(srv)
            peak = max(peak, cube.cube_server_bytes(srv))
            for t in tickets:
                if t in done:
                    continue
                info = cube.cube_server_info(srv, t)
                assert info.state != cube.CUBE_REQ_FAILED, info.error
                if info.state == cube.CUBE_REQ_DONE:
                    done.add(t)
                    held = cube.cube_server_bytes(srv)
                    cube.cube_server_release(srv, t)          # frees the state: queued requests fit
                    assert cube.cube_server_bytes(srv) == held - info.state_bytes
            if len(done) == len(tickets):
                break
        assert len(done) == len(tickets)
        assert peak <= budget
    finally:
        cube.cube_server_destroy(srv)


def test_admission_order_and_release(cube):
    mix = _mix()[:4]
    ics = [synth.make_ics(w) for w in mix]
    srv = cube.cube_server_create(8 << 30, n_streams=2, max_running=2)
    try:
        keep, tickets = [], []
        for w, ic in zip(mix, ics):
            host = (_pinned(ic.pos), _pinned(ic.vel), _pinned(ic.ids.view(np.int32)))
            keep.append(host)
            sch = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
            tickets.append(cube.cube_server_submit(srv, _params(cube, w), *host, ic.sigma_1d, sch, 4))
        cube.cube_server_drain(srv)
        infos = [cube.cube_server_info(srv, t) for t in tickets]
        admits = [i.t_admit for i in infos]
        assert admits == sorted(admits)                       # arrival order
        # at most max_running requests overlap: the third starts after the first finishes
        assert admits[2] >= min(infos[0].t_done, infos[1].t_done)
        before = cube.cube_server_bytes(srv)
        cube.cube_server_release(srv, tickets[0])
        assert cube.cube_server_bytes(srv) == before - infos[0].state_bytes
        with pytest.raises(cube.CubeError):
            cube.cube_server_info(srv, tickets[0])
    finally:
        cube.cube_server_destroy(srv)


def test_submit_rejects_bad_requests(cube):
    w = _mix()[0]
    ic = synth.make_ics(w)
    p = _params(cube, w)
    sb, wb = cube.cube_server_sizes(p)
    srv = cube.cube_server_create(sb + wb - 1, n_streams=1, max_running=1)
    try:
        sch = synth.uniform_schedule(w.a_init, w.a_final, 3)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_server_submit(srv, p, ic.pos, ic.vel, ic.ids, ic.sigma_1d, sch, 4)
        assert e.value.status == cube.CUBE_E_NOMEM
    finally:
        cube.cube_server_destroy(srv)
    srv = cube.cube_server_create(8 << 30, n_streams=1, max_running=1)
    try:
        for bad_sch, nb in ((sch[::-1], 4), (sch[:1], 4), (sch, 0), (sch, 4096)):
            with pytest.raises(cube.CubeError) as e:
                cube.cube_server_submit(srv, p, ic.pos, ic.vel, ic.ids, ic.sigma_1d, bad_sch, nb)
            assert e.value.status == cube.CUBE_E_ARG
        t = cube.cube_server_submit(srv, p, ic.pos, ic.vel, ic.ids, ic.sigma_1d, sch, 4)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_server_release(srv, t)                  # still queued
        assert e.value.status == cube.CUBE_E_STATE
        cube.cube_server_drain(srv)
        cube.cube_server_release(srv, t)
    finally:
        cube.cube_server_destroy(srv)


def test_adaptive_requests_equal_the_velocity_limited_run_alone(cube):
    """max_drift_cells > 0: the server cuts every step as cube_next_epoch
    does (fastest particle within half a coarse cell), reading the largest |p|
    back asynchronously.  The finest-cell ensemble realisation (whose uniform
    steps clamp a migration with 1-byte codes) completes, with the same steps
    and the same particles as the cube_next_epoch loop on a plain context."""
    ens = synth.ensemble_c4(64)
    w = min(ens, key=lambda x: x.box / x.n_part_side)
    w = dataclasses.replace(w, n_part_side=32, n_fine=64, box=w.box * 32 / w.n_part_side)
    ic = synth.make_ics(w)
    p = _params(cube, w)
    targets = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    n = w.n_particles
    # alone
    ctx = cube.cube_create(p, torch.cuda.current_stream())
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        a, steps = w.a_init, 0
        for t in targets[1:]:
            while a < t:
                a_to = cube.cube_next_epoch(ctx, t, 0.5)
                cube.cube_pm_step(ctx, a, a_to)
                a, steps = a_to, steps + 1
        want = (np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32))
        cube.cube_decode(ctx, *want)
    finally:
        cube.cube_destroy(ctx)
    srv = cube.cube_server_create(8 << 30, n_streams=2, max_running=4)
    try:
        host = (_pinned(ic.pos), _pinned(ic.vel), _pinned(ic.ids.view(np.int32)))
        t = cube.cube_server_submit(srv, p, *host, ic.sigma_1d, targets, 4, max_drift_cells=0.5)
        other = _mix()[1]                                   # a fixed-step request beside it
        oic = synth.make_ics(other)
        ohost = (_pinned(oic.pos), _pinned(oic.vel), _pinned(oic.ids.view(np.int32)))
        t2 = cube.cube_server_submit(srv, _params(cube, other), *ohost, oic.sigma_1d,
                                     synth.uniform_schedule(other.a_init, other.a_final, other.n_steps), 4)
        cube.cube_server_drain(srv)
        info = cube.cube_server_info(srv, t)
        assert info.state == cube.CUBE_REQ_DONE, info.error
        assert info.steps_enqueued == steps > w.n_steps and info.max_migration <= 1
        assert cube.cube_server_info(srv, t2).state == cube.CUBE_REQ_DONE
        got = (np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32))
        cube.cube_server_decode(srv, t, *got)
        for g, e in zip(got, want):
            assert np.array_equal(g, e)
        with pytest.raises(cube.CubeError) as e:
            cube.cube_server_submit(srv, p, *host, ic.sigma_1d, targets, 4, max_drift_cells=1.5)
        assert e.value.status == cube.CUBE_E_ARG
    finally:
        cube.cube_server_destroy(srv)


def test_a_work_area_that_cannot_grow_fails_only_the_new_request(cube):
    """Admission needs a larger work area for a bigger request on a stream
    whose area is in use.  When that allocation fails (made to fail on the
    host by the server's test hook), the stream keeps its old area, the
    running request finishes with the same result as alone, the new request
    ends FAILED with CUBE_E_NOMEM, the bytes held stay exact, and a later
    request of the same size is admitted and completes."""
    mix = _mix()
    small, big = mix[0], mix[3]                       # 16^3 and 48^3 particles
    ics = {w.n_part_side: synth.make_ics(w) for w in (small, big)}
    nb = 4
    s_sb, s_wb = cube.cube_server_sizes(_params(cube, small))
    b_sb, b_wb = cube.cube_server_sizes(_params(cube, big))
    assert b_wb > s_wb
    srv = cube.cube_server_create(8 << 30, n_streams=1, max_running=4)
    keep = []

    def submit(w):
        ic = ics[w.n_part_side]
        host = (_pinned(ic.pos), _pinned(ic.vel), _pinned(ic.ids.view(np.int32)))
        keep.append(host)
        sch = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
        return cube.cube_server_submit(srv, _params(cube, w), *host, ic.sigma_1d, sch, nb)
    try:
        ta = submit(small)
        cube.cube_server_pump(srv)
        assert cube.cube_server_info(srv, ta).state == cube.CUBE_REQ_RUNNING
        assert cube.cube_server_bytes(srv) == s_sb + s_wb
        cube.cube_server_inject_alloc_failures(srv, 1)
        tb = submit(big)
        cube.cube_server_pump(srv)
        ib = cube.cube_server_info(srv, tb)
        assert ib.state == cube.CUBE_REQ_FAILED and ib.error == cube.CUBE_E_NOMEM
        assert cube.cube_server_bytes(srv) == s_sb + s_wb        # the old area is kept, nothing leaked
        cube.cube_server_drain(srv)
        assert cube.cube_server_info(srv, ta).state == cube.CUBE_REQ_DONE
        n = small.n_particles
        got = (np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32))
        cube.cube_server_decode(srv, ta, *got)
        want = _alone(cube, small, ics[small.n_part_side], nb)
        for g, e in zip(got, want[3:]):
            assert np.array_equal(g, e)
        cube.cube_server_release(srv, tb)
        tc = submit(big)                                          # the allocation now succeeds
        cube.cube_server_drain(srv)
        assert cube.cube_server_info(srv, tc).state == cube.CUBE_REQ_DONE
        assert cube.cube_server_bytes(srv) == s_sb + b_sb + b_wb
        cube.cube_server_release(srv, ta)
        cube.cube_server_release(srv, tc)
        assert cube.cube_server_bytes(srv) == b_wb
    finally:
        cube.cube_server_destroy(srv)


def test_shortest_work_first_admission(cube):
    """CUBE_ADMIT_SHORTEST: with one request running at a time, queued
    requests are admitted in increasing particles x steps (ties in arrival
    order); CUBE_ADMIT_FIFO admits them in arrival order.  Results do not
    depend on the order."""
    mix = _mix()[:5]
    ics = [synth.make_ics(w) for w in mix]
    work = [w.n_particles * w.n_steps for w in mix]
    results = {}
    for policy in (cube.CUBE_ADMIT_FIFO, cube.CUBE_ADMIT_SHORTEST):
        srv = cube.cube_server_create(8 << 30, n_streams=1, max_running=1)
        try:
            cube.cube_server_set_policy(srv, policy)
            keep, tickets = [], []
            for w, ic in zip(mix, ics):
                host = (_pinned(ic.pos), _pinned(ic.vel), _pinned(ic.ids.view(np.int32)))
                keep.append(host)
                sch = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
                tickets.append(cube.cube_server_submit(srv, _params(cube, w), *host, ic.sigma_1d, sch, 4))
            cube.cube_server_drain(srv)
            infos = [cube.cube_server_info(srv, t) for t in tickets]
            assert all(i.state == cube.CUBE_REQ_DONE for i in infos)
            order = list(np.argsort([i.t_admit for i in infos], kind="stable"))
            outs = []
            for w, t in zip(mix, tickets):
                n = w.n_particles
                pos, vel, ids = np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32)
                cube.cube_server_decode(srv, t, pos, vel, ids)
                outs.append((pos, vel, ids))
            results[policy] = outs
        finally:
            cube.cube_server_destroy(srv)
        if policy == cube.CUBE_ADMIT_FIFO:
            assert order == list(range(len(mix)))
        else:
            assert order == sorted(range(len(mix)), key=lambda i: (work[i], i))
    for a, b in zip(results[cube.CUBE_ADMIT_FIFO], results[cube.CUBE_ADMIT_SHORTEST]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    with pytest.raises(cube.CubeError):
        srv = cube.cube_server_create(1 << 30, n_streams=1, max_running=1)
        try:
            cube.cube_server_set_policy(srv, 7)
        finally:
            cube.cube_server_destroy(srv)
