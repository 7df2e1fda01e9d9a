#!/usr/bin/env python
"""Throughput of CUBE's compressed-store PM step on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default pm256): 256^3 particles, 512^3 FP32 mesh, 300 Mpc/h flat
LCDM (Om 0.3, h 0.7, sigma8 0.8, BBKS), 1-byte positions and velocities,
Zel'dovich ICs at z = 49 from seeded synthetic Gaussian random fields, steps
uniform in a towards z = 0.  One "step" = one cube_pm_step (deposit, 3-D FFT
Poisson solve, force gather + kick + drift, two-pass re-sort) of the whole
store.  Prints one JSON line (rank 0).

Timing: W untimed steps, then exactly K steps between a barrier +
synchronize on both sides, CUDA events on the library's stream; max over
ranks.  Inputs exceed L2 (the 512^3 mesh alone is 537 MB), so no L2 flush.
N > 1 runs independent replicas (one simulation per GPU, seed + rank); the
path has no collective.  The K timed steps start at z = 49, where the store
is nearly uniform; `whole_run` times the workload's whole run to z = 0 step
by step beside them (late epochs are clustered and slower).

The CPU baseline and the reference arm (--impl reference) run the FP64
oracle as it stands at 128^3 particles / 256^3 mesh, one independent
replica per host core (processes started with spawn).
"""
import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pm256")
    ap.add_argument("--codes", default=None, choices=["x1v1", "x1v2", "x2v1", "x2v2", "fp32"],
                    help="override the workload's code widths; fp32 = the uncompressed FP32 store")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-whole-run", action="store_true",
                    help="skip the whole z_init -> z_final run timed step by step beside the K timed steps")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="run the C4 ensemble of this many uneven realisations (sims/s) instead of pm256")
    ap.add_argument("--streams", type=int, default=8, help="CUDA streams for --ensemble and --serve")
    ap.add_argument("--serve", type=int, default=0,
                    help="run the C5 serving stream of this many requests (latency, sims/s) instead of pm256")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="HBM budget of --serve")
    ap.add_argument("--nps", type=int, default=0,
                    help="particles per side (mesh = 2 x nps) instead of the workload's, for small profiling cases")
    return ap.parse_args()


def schedule(w, n):
    """First n steps of the workload's uniform-in-a schedule; a finer uniform
    schedule over the same range if n exceeds its step count."""
    import numpy as np
    total = max(w.n_steps, n)
    return np.linspace(w.a_init, w.a_final, total + 1)[: n + 1]


def phase_bytes(w, geo):
    """Algorithmic HBM bytes per launch of each traced kernel: the minimum
    the operation must move (each input read once, each output written
    once), from the particle count, mesh and coarse-grid sizes, code widths
    and brick geometry."""
    N = w.n_fine
    Np = w.n_particles
    Nm = N ** 3
    Ncc = (N // w.ratio) ** 3
    H3 = (geo["brick"] + 2) ** 3
    nbr = Ncc // geo["brick"] ** 3
    half = N * N * (N // 2 + 1) * 8          # half-complex mesh bytes
    s_x, s_v = 3 * w.x_bytes, 3 * w.v_bytes
    if w.x_bytes == 4:                       # uncompressed FP32 store: no codes, cells or re-sort
        return {"deposit": 12 * Np + 4 * Nm, "fft_x_r2c": 4 * Nm + half, "fft_y_fwd": 2 * half,
                "fft_z_green": 2 * half, "fft_y_inv": 2 * half, "fft_x_c2r": half + 4 * Nm,
                "pass_a": 48 * Np + 4 * Nm}
    return {
        "deposit": 4 * Nm + s_x * Np + 4 * Ncc,
        "fft_x_r2c": 4 * Nm + half,
        "fft_y_fwd": 2 * half,
        "fft_z_green": 2 * half,
        "fft_y_inv": 2 * half,
        "fft_x_c2r": half + 4 * Nm,
        "pass_a": (s_x + 2 * s_v) * Np + 4 * Nm + (4 + 12 + 28) * Ncc + 4 * H3 * nbr,
        "codec": 0,
        "scan": 12 * Ncc,
        "starts": (4 + 4 + 24 + 12) * Ncc + 8 * H3 * nbr,
        "pass_b": 2 * (s_x + s_v + 4) * Np + (4 + 12 + 12) * Ncc + 4 * H3 * nbr,
    }


def step_bytes(w):
    """Whole-step algorithmic bytes of the method's minimum model:
    (3s + 3n_nu) N_p + 32 N_coarse + 32 N_mesh, s = 3 n_chi + 3 n_nu; the
    uncompressed FP32 store: 60 N_p (read 24 + write 24 + deposit read 12)
    + 32 N_mesh."""
    if w.x_bytes == 4:
        return 60 * w.n_particles + 32 * w.n_fine ** 3
    s = 3 * w.x_bytes + 3 * w.v_bytes
    return (3 * s + 3 * w.v_bytes) * w.n_particles + 32 * (w.n_fine // w.ratio) ** 3 + 32 * w.n_fine ** 3


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x, dist):
    """The largest x over all ranks of the process group (x itself without
    one): the job's time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the device-code sources (the
    kernel files, their shared header and declarations; host-only files such
    as the C-ABI glue, the server and the tuner are left out)."""
    import hashlib
    src = os.path.join(ROOT, "paper_1712_06121_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        if f.startswith("k_") or f in ("cube_common.cuh", "kernels.h"):
            with open(os.path.join(src, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    rec = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or "=" not in line:
                continue
            k, v = line.strip().split("=", 1)
            rec[k.strip()] = v.strip()
    if rec.get("source_sha") != cur:
        return None
    v = rec.get(f"{kernel}.bytes_per_launch")
    return float(v) if v else None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        load = [s for s in sm if mx and s >= 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_state(w, ic, nps):
    """The oracle's state and step function for the workload's store: the
    compressed store (pm.encode / pm.step), or for the uncompressed FP32
    store the oracle's uncompressed FP64 mode (pm.exact_from / exact_step)."""
    import numpy as np
    from oracle import pm
    om, ol, _ = w.omega()
    if w.x_bytes == 4:
        P = pm.Params(n_fine=2 * nps, n_particles=nps ** 3, x_bytes=1, v_bytes=1, box=w.box, omega_m=om,
                      omega_l=ol)
        return pm.exact_from(P, np.mod(ic.pos.astype(np.float64), 2 * nps), ic.vel, w.a_init), pm.exact_step
    P = pm.Params(n_fine=2 * nps, n_particles=nps ** 3, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                  omega_m=om, omega_l=ol)
    return pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d), pm.step


ORACLE_NPS = 128            # the oracle's sample size: 128^3 particles, 256^3 mesh


def _oracle_replica(wname, nps, codes, sched, warm, barrier, out):
    """One oracle replica in its own process: the workload's ICs at nps^3
    particles, `warm` untimed steps, then (after every replica is ready)
    the remaining steps of `sched`, timed on the host clock."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    import dataclasses
    import synth
    w = synth.WORKLOADS[wname]
    if codes:
        w = dataclasses.replace(w, x_bytes=codes[0], v_bytes=codes[1])
    ic = synth.make_ics(w, n_part_side=nps, n_fine=2 * nps)
    st, step = oracle_state(w, ic, nps)
    for i in range(warm):
        st = step(st, float(sched[i]), float(sched[i + 1]))
    barrier.wait()
    t0 = time.perf_counter()
    for i in range(warm, len(sched) - 1):
        st = step(st, float(sched[i]), float(sched[i + 1]))
    out.put(time.perf_counter() - t0)


def oracle_replicas(w, sched, warm, workers=None):
    """The oracle as it stands, on the host's cores: `workers` independent
    replicas (one process each, started with spawn, numpy single-threaded),
    each stepping the workload at 128^3 particles / 256^3 mesh through
    `sched`.  Returns (particle-steps/s over all replicas, workers, wall s)."""
    import multiprocessing as mp
    if workers is None:
        cores = os.cpu_count() or 1
        try:                                              # each replica peaks near 2 GB
            mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES") / 2 ** 30
        except (ValueError, OSError):
            mem_gb = 16.0
        workers = max(1, min(cores, int(mem_gb // 3)))
    nps = min(ORACLE_NPS, w.n_part_side)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    out = ctx.Queue()
    codes = (w.x_bytes, w.v_bytes)
    procs = [ctx.Process(target=_oracle_replica, args=(w.name.split("@")[0], nps, codes, list(sched), warm, barrier,
                                                     out)) for _ in range(workers)]
    for p in procs:
        p.start()
    times = [out.get() for _ in procs]
    for p in procs:
        p.join()
    dt = max(times)
    steps = len(sched) - 1 - warm
    return workers * nps ** 3 * steps / dt, workers, dt


def cpu_baseline(w):
    """The FP64 oracle on the host cores: one step of the same workload at
    128^3 particles / 256^3 mesh (same seed and cosmology) in every replica."""
    import numpy as np
    sch = np.linspace(w.a_init, w.a_final, w.n_steps + 1)[:2]
    value, workers, dt = oracle_replicas(w, sch, 0)
    nps = min(ORACLE_NPS, w.n_part_side)
    return {"value": value, "unit": "particle-steps/s", "cores": workers, "kind": "oracle",
            "sample": f"one oracle step of {w.name} at {nps}^3 particles / {2 * nps}^3 mesh in each of {workers} "
                      f"independent replicas (numpy FP64, one process and one thread per core), {dt:.1f} s"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import dataclasses
    nps = min(ORACLE_NPS, w.n_part_side)
    sch = schedule(w, args.warmup + args.steps)
    value, workers, dt = oracle_replicas(w, sch, args.warmup)
    ws = dataclasses.replace(w, n_part_side=nps, n_fine=2 * nps)
    sample = (f"{args.steps} oracle steps after {args.warmup} warm-up steps of {w.name} at {nps}^3 particles / "
              f"{2 * nps}^3 mesh in each of {workers} independent replicas (numpy FP64, one process and one "
              f"thread per core)")
    print(json.dumps({
        "impl": "reference", "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(ws, mesh="FP64 (oracle)"),
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def e2e_overlapped(cube, prm, ic, w, sch, n_iter, dist, world):
    """The e2e loop (pinned host pos/vel/ids -> cube_encode -> cube_pm_step ->
    cube_decode -> pinned host) on two contexts with their own streams and
    host buffers, each driven by its own host thread: one iteration's copies
    overlap the other's kernels.  Every iteration still uploads its inputs
    and downloads its result inside the timed region."""
    import threading
    import numpy as np
    import torch
    lanes = []
    for _ in range(2):
        st = torch.cuda.Stream()
        c = cube.cube_create(prm, st)
        bufs = (torch.from_numpy(ic.pos).pin_memory(), torch.from_numpy(ic.vel).pin_memory(),
                torch.from_numpy(ic.ids.view(np.int32)).pin_memory())
        outs = tuple(torch.empty_like(b).pin_memory() for b in bufs)
        lanes.append((c, bufs, outs))

    def lane(c, bufs, outs, n, err):
        try:
            for _ in range(n):
                cube.cube_encode(c, *bufs, w.a_init, ic.sigma_1d)
                cube.cube_pm_step(c, sch[0], sch[1])
                cube.cube_decode(c, *outs)
        except Exception as e:                           # reported after the join
            err.append(e)

    def run(n):
        err = []
        th = [threading.Thread(target=lane, args=(c, b, o, n, err)) for c, b, o in lanes]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if err:
            raise err[0]

    try:
        run(1)                                          # warm the staging buffers
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(n_iter)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for c, _, _ in lanes:
            cube.cube_stats_get(c)                      # raises on a latched device error
    finally:
        for c, _, _ in lanes:
            cube.cube_destroy(c)
    nbytes = 28 * w.n_particles
    return {"value": world * w.n_particles * 2 * n_iter / max_over_ranks(dt, dist), "unit": "particle-steps/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "what": "the e2e loop on two contexts (own streams and pinned buffers), one host thread each, "
                    f"{n_iter} iterations per context: one iteration's copies overlap the other's kernels"}


def whole_run(cube, ctx, ic, w, stream):
    """The workload's whole run, z_init -> z_final, timed step by step with
    CUDA events on the library's stream (no host synchronisation inside).
    The schedule is the workload's uniform one unless it moves a particle
    more than one coarse cell in a step (the library clamps the move and
    reports CUBE_E_MIGRATION); then every step is cut by the velocity and
    acceleration limit of cube_next_epoch_limited (the fastest particle
    drifts at most half a coarse cell), with the uniform epochs as
    waypoints.  An untimed pass over the schedule comes first (it also
    fixes the limited schedule's epochs, which the timed pass replays)."""
    import numpy as np
    import torch
    uniform = list(np.linspace(w.a_init, w.a_final, w.n_steps + 1))

    def replay(sch, events=None):
        cube.cube_encode(ctx, torch.from_numpy(ic.pos).cuda(), torch.from_numpy(ic.vel).cuda(),
                         torch.from_numpy(ic.ids.view(np.int32)).cuda(), w.a_init, ic.sigma_1d)
        torch.cuda.synchronize()
        if events:
            events[0].record(stream)
        for i in range(len(sch) - 1):
            cube.cube_pm_step(ctx, sch[i], sch[i + 1])
            if events:
                events[i + 1].record(stream)
        torch.cuda.synchronize()
        return cube.cube_stats_get(ctx)              # raises on a latched device error

    kind = "uniform"
    try:
        replay(uniform)
        sch = uniform
    except cube.CubeError as e:
        if e.status != cube.CUBE_E_MIGRATION:
            raise
        kind = "velocity-limited"
        cube.cube_encode(ctx, torch.from_numpy(ic.pos).cuda(), torch.from_numpy(ic.vel).cuda(),
                         torch.from_numpy(ic.ids.view(np.int32)).cuda(), w.a_init, ic.sigma_1d)
        sch, a = [w.a_init], w.a_init
        for t in uniform[1:]:
            while a < t:
                a_to, _ = cube.cube_next_epoch_limited(ctx, t, 0.5)
                cube.cube_pm_step(ctx, a, a_to)
                sch.append(a_to)
                a = a_to
        cube.cube_stats_get(ctx)
    ev = [torch.cuda.Event(enable_timing=True) for _ in sch]
    st = replay(sch, ev)
    ms = np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(len(sch) - 1)])
    k = len(ms) // 3
    return {"schedule": f"{kind}, {len(ms)} steps z={1 / w.a_init - 1:g} -> {1 / w.a_final - 1:g}",
            "steps": len(ms), "ms_per_step": float(ms.mean()),
            "early_third_ms_per_step": float(ms[:k].mean()), "middle_third_ms_per_step": float(ms[k:-k].mean()),
            "late_third_ms_per_step": float(ms[-k:].mean()), "max_ms": float(ms.max()),
            "value": w.n_particles * len(ms) / (ms.sum() / 1e3), "unit": "particle-steps/s",
            "max_migration": int(st.max_migration)}


def codes_of(w):
    return "uncompressed FP32" if w.x_bytes == 4 else f"x{w.x_bytes}v{w.v_bytes}"


def step_model(w):
    return "60 N_p + 32 N_mesh" if w.x_bytes == 4 else "(3s+3n_nu)N_p + 32 N_coarse + 32 N_mesh"


def config_of(w, mesh="FP32"):
    return {"workload": f"{w.name}: {w.n_part_side}^3 particles, {w.n_fine}^3 {mesh} mesh, {w.box:g} Mpc/h, "
                        f"{'EdS' if w.cosmo_kind == 'eds' else 'LCDM BBKS'}, {codes_of(w)}, "
                        f"R={w.ratio}, steps uniform in a from z={1 / w.a_init - 1:g}",
            "l2": ("inputs larger than L2 (no flush)" if 4 * w.n_fine ** 3 > 129e6
                   else "L2-resident small workload"), "parallelism": "replicas"}


def run_ensemble(args):
    """The C4 ensemble (synth.ensemble_c4): every realisation in its own
    context, contexts spread over `--streams` CUDA streams and stepped in
    interleaved order so that small meshes overlap on the GPU, against the
    same realisations run one after another.  ICs are on the device before
    the timed region; each realisation's encode and all its steps are timed."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1712_06121_gb300 as cube
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ens = synth.ensemble_c4(args.ensemble)
    ics = [synth.make_ics(w) for w in ens]
    streams = [torch.cuda.Stream() for _ in range(args.streams)]
    dev = [(torch.from_numpy(ic.pos).cuda(), torch.from_numpy(ic.vel).cuda(),
            torch.from_numpy(ic.ids.view(np.int32)).cuda()) for ic in ics]

    def params(w, brick=0):
        om, ol, _ = w.omega()
        return cube.make_params(w.n_fine, w.n_particles, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                                omega_m=om, omega_l=ol, brick=brick)

    # the autotuner's brick per particle count (first realisation of each size)
    tuned, tune_ms = {}, {}
    for w, ic, d in zip(ens, ics, dev):
        if w.n_part_side not in tuned:
            tuned[w.n_part_side], tune_ms[w.n_part_side] = cube.cube_autotune_brick(
                params(w), d[0], d[1], w.a_init, ic.sigma_1d, 5, torch.cuda.current_stream())
    ctxs = []

    def make_ctxs(use_tuned):
        for c in ctxs:
            cube.cube_stats_get(c)                          # raises on a latched device error
            cube.cube_destroy(c)
        ctxs[:] = [cube.cube_create(params(w, tuned[w.n_part_side] if use_tuned else 0),
                                    streams[i % len(streams)]) for i, w in enumerate(ens)]
    scheds = [synth.uniform_schedule(w.a_init, w.a_final, w.n_steps) for w in ens]

    nsteps = [0] * len(ens)

    def advance(i):
        """One step of realisation i toward its next scheduled epoch, cut by
        cube_next_epoch so the fastest particle drifts at most half a
        coarse cell; False once the realisation has reached a_final."""
        c, sch = ctxs[i], scheds[i]
        a = state[i]["a"]
        if a >= sch[-1]:
            return False
        target = sch[np.searchsorted(sch, a, side="right")]
        a_to = cube.cube_next_epoch(c, target, 0.5)
        cube.cube_pm_step(c, a, a_to)
        state[i]["a"] = a_to
        nsteps[i] += 1
        return True

    def run(concurrent):
        for i in range(len(ens)):
            nsteps[i] = 0
        for i, (c, w, ic, d) in enumerate(zip(ctxs, ens, ics, dev)):
            state[i] = {"a": w.a_init}
            cube.cube_encode(c, *d, w.a_init, ic.sigma_1d)
            if not concurrent:
                while advance(i):
                    pass
                torch.cuda.synchronize()
        if concurrent:
            live = list(range(len(ens)))
            while live:
                live = [i for i in live if advance(i)]
        torch.cuda.synchronize()

    state = [None] * len(ens)

    times = {}
    for mode, use_tuned in ((False, False), (True, False), (True, True)):
        make_ctxs(use_tuned)
        run(mode)                                           # warm-up pass
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps // 10)):
            run(mode)
        times[(mode, use_tuned)] = (time.perf_counter() - t0) / max(1, args.steps // 10)
    make_ctxs(False)
    for c in ctxs:
        cube.cube_destroy(c)
    ctxs[:] = []

    # batched: the realisations of one size share their geometry (only the box
    # and sigma8 differ), so each size is one cube_batch stepped with one launch
    # per kernel; every member keeps its own velocity-limited epochs
    classes = {}
    for i, w in enumerate(ens):
        classes.setdefault(w.n_part_side, []).append(i)
    batches = []
    for j, (nps_, idx) in enumerate(sorted(classes.items())):
        b = cube.cube_batch_create([params(ens[i], tuned[nps_]) for i in idx], streams[j % len(streams)])
        batches.append((b, idx, [cube.cube_batch_member(b, k) for k in range(len(idx))]))
    bsteps = [0]

    def run_batched():
        """Every batch steps as soon as its members' largest momenta are back
        on the host (read back asynchronously behind its previous step), so
        the host never waits on one batch while the others have work; the
        mesh half of each batch's next step is enqueued behind that
        read-back, so its GPU works while the host waits."""
        bsteps[0] = 0
        cur = {}

        def solve_next(b, idx):
            cube.cube_batch_solve(b, [1 if cur[i] < scheds[i][-1] else 0 for i in idx])

        for b, idx, members in batches:
            for c, i in zip(members, idx):
                cube.cube_encode(c, *dev[i], ens[i].a_init, ics[i].sigma_1d)
                cur[i] = ens[i].a_init
            cube.cube_batch_epochs_enqueue(b)
            solve_next(b, idx)
        live = list(batches)
        while live:
            nxt, moved_on = [], False
            for b, idx, members in live:
                a_from = np.array([cur[i] for i in idx])
                a_max = np.array([scheds[i][np.searchsorted(scheds[i], cur[i], side="right")]
                                  if cur[i] < scheds[i][-1] else cur[i] for i in idx])
                if not np.any(a_max > a_from):
                    continue                                # every member has reached z = 0
                nxt.append((b, idx, members))
                a_to = cube.cube_batch_epochs_poll(b, a_max, 0.5)
                if a_to is None:
                    continue
                cube.cube_batch_step(b, a_from, a_to)
                cube.cube_batch_epochs_enqueue(b)
                bsteps[0] += 1
                moved_on = True
                for i, a in zip(idx, a_to):
                    cur[i] = float(a)
                solve_next(b, idx)
            live = nxt
            if not moved_on:
                time.sleep(2e-5)
        torch.cuda.synchronize()

    run_batched()                                           # warm-up pass
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 10)):
        run_batched()
    times[("batched", True)] = (time.perf_counter() - t0) / max(1, args.steps // 10)
    launches_batched = sum(cube.cube_batch_launches(b) for b, _, _ in batches)
    for b, _, members in batches:
        for c in members:
            cube.cube_stats_get(c)                          # raises on a latched device error
        cube.cube_batch_destroy(b)

    # the same realisations through cube_server: velocity-limited steps with
    # the largest |p| read back asynchronously, so no host wait per step
    def served():
        srv = cube.cube_server_create(64 << 30, args.streams, len(ens))
        try:
            tickets = [cube.cube_server_submit(srv, params(w, tuned[w.n_part_side]), d[0], d[1], d[2], ic.sigma_1d,
                                               sch, 8, max_drift_cells=0.5)
                       for w, ic, d, sch in zip(ens, ics, dev, scheds)]
            cube.cube_server_drain(srv)
            infos = [cube.cube_server_info(srv, t) for t in tickets]
            for t in tickets:
                cube.cube_server_release(srv, t)
        finally:
            cube.cube_server_destroy(srv)
        assert all(i.state == cube.CUBE_REQ_DONE for i in infos)
        return infos
    served()                                                # warm-up pass
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = served()
    t_srv = time.perf_counter() - t0
    times[("served", True)] = t_srv
    sizes = sorted({w.n_part_side for w in ens})
    best = min(times[(True, True)], t_srv, times[("batched", True)])
    print(json.dumps({
        "metric": "sims/s", "value": len(ens) / best, "unit": "sims/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded GRF Zel'dovich ICs)",
        "config": {"workload": f"C4 ensemble: {len(ens)} realisations, {sizes[0]}^3..{sizes[-1]}^3 particles "
                               f"(mesh 2x), box 50-400 Mpc/h, sigma8 0.7-0.9, LCDM BBKS, x1v1, z=49->0",
                   "streams": len(streams), "timing": "host wall clock, ICs resident, encode + all steps"},
        "sequential": {"value": len(ens) / times[(False, False)], "unit": "sims/s",
                       "what": "the same contexts run one after another, default bricks"},
        "concurrent_default_bricks": {"value": len(ens) / times[(True, False)], "unit": "sims/s"},
        "concurrent_tuned_bricks": {"value": len(ens) / times[(True, True)], "unit": "sims/s"},
        "served": {"value": len(ens) / t_srv, "unit": "sims/s", "steps": int(sum(i.steps_enqueued for i in infos)),
                   "what": "cube_server, all realisations admitted at once, velocity-limited steps with "
                           "asynchronous max-|p| read-back (no host wait per step), tuned bricks"},
        "batched": {"value": len(ens) / times[("batched", True)], "unit": "sims/s",
                    "batch_steps": bsteps[0], "launches_per_batch_step": 16,
                    "mesh_half": "enqueued behind each step's max-|p| read-back (cube_batch_solve)",
                    "kernel_launches_all_passes": launches_batched,
                    "what": f"one cube_batch per particle count ({len(batches)} batches), each step of a batch one "
                            "launch per kernel for all its members, members' own velocity-limited epochs, "
                            "batches on separate streams"},
        "tuned_bricks": {str(k): v for k, v in sorted(tuned.items())},
        "tuner_ms_per_step_b1_b2_b4": {str(k): [round(x, 4) for x in v] for k, v in sorted(tune_ms.items())},
        "steps_total": int(sum(nsteps)),
        "time_stepping": "30 scheduled epochs, each step cut by cube_next_epoch (fastest drift <= 0.5 coarse cell)",
        "speedup_vs_sequential": times[(False, False)] / best,
    }), flush=True)


def _serve_ics(w, out_dir, i):
    """One request's own Zel'dovich ICs (its seed and sigma8), written to
    out_dir as .npy files (a worker process of run_serve)."""
    import numpy as np
    import synth
    ic = synth.make_ics(w)
    for k, a in (("pos", ic.pos), ("vel", ic.vel), ("ids", ic.ids)):
        np.save(os.path.join(out_dir, f"{i}_{k}.npy"), a)
    return i, float(ic.sigma_1d)


def run_serve(args):
    """C5: a Poisson stream of simulation requests (sizes 64^3 .. 256^3,
    10 .. 60 steps, own seed and sigma8) through cube_server under an HBM
    budget, continuous batching on several streams (first-come and
    shortest-work-first admission) against the plain method (one request at a
    time, same arrivals).  Every request's ICs are generated before the GPU
    work (processes started with spawn, one per host core) and held in pinned
    host memory.  Latency = completion - arrival on the server's clock;
    throughput = requests / (last completion - first arrival)."""
    import multiprocessing as mp
    import shutil
    import numpy as np
    import synth
    reqs = synth.serving_c5(args.serve)
    tmp = tempfile.mkdtemp(dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
    try:
        with mp.get_context("spawn").Pool(max(1, min(len(reqs), os.cpu_count() or 1))) as pool:
            sig = dict(pool.starmap(_serve_ics, [(r.workload, tmp, i) for i, r in enumerate(reqs)]))
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_1712_06121_gb300 as cube
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        data = []
        for i, r in enumerate(reqs):
            w = r.workload
            om, ol, _ = w.omega()
            prm = cube.make_params(w.n_fine, w.n_particles, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                                   omega_m=om, omega_l=ol)
            arr = [np.load(os.path.join(tmp, f"{i}_{k}.npy")) for k in ("pos", "vel", "ids")]
            host = tuple(torch.from_numpy(np.ascontiguousarray(a if k < 2 else a.view(np.int32))).pin_memory()
                         for k, a in enumerate(arr))
            data.append((prm, host, sig[i], synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)))
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    budget = int(args.budget_gb * (1 << 30))

    def serve(n_streams, max_running, at_once=False, policy=0):
        srv = cube.cube_server_create(budget, n_streams, max_running)
        try:
            cube.cube_server_set_policy(srv, policy)
            seen = set()                                    # warm-up: one short run per size
            warm = []
            for r, (prm, host, sig, sch) in zip(reqs, data):
                if r.workload.n_part_side not in seen:
                    seen.add(r.workload.n_part_side)
                    warm.append(cube.cube_server_submit(srv, prm, *host, sig, sch[:3], 8))
            cube.cube_server_drain(srv)
            for t in warm:
                cube.cube_server_release(srv, t)
            torch.cuda.synchronize()
            tickets, nxt, peak = [], 0, 0
            t0 = time.perf_counter()
            while True:
                now = time.perf_counter() - t0
                while nxt < len(reqs) and (at_once or reqs[nxt].arrival <= now):
                    prm, host, sig, sch = data[nxt]
                    tickets.append(cube.cube_server_submit(srv, prm, *host, sig, sch, 8, max_drift_cells=0.5))
                    nxt += 1
                nr, nq = cube.cube_server_pump(srv)
                peak = max(peak, cube.cube_server_bytes(srv))
                if nxt == len(reqs) and nr + nq == 0:
                    break
                time.sleep(5e-5)
            infos = [cube.cube_server_info(srv, t) for t in tickets]
            for t in tickets:
                cube.cube_server_release(srv, t)
        finally:
            cube.cube_server_destroy(srv)
        ok = [i for i in infos if i.state == cube.CUBE_REQ_DONE]
        lat = np.array([i.t_done - i.t_submit for i in ok])
        span = max(i.t_done for i in ok) - min(i.t_submit for i in infos)
        steps = sum(i.steps_enqueued for i in ok)
        parts = sum(reqs[k].workload.n_particles * infos[k].steps_enqueued for k in range(len(infos))
                    if infos[k].state == cube.CUBE_REQ_DONE)
        failed = [f"{reqs[k].workload.name}: {cube.STATUS_NAMES[infos[k].error]}" for k in range(len(infos))
                  if infos[k].state != cube.CUBE_REQ_DONE]
        return {"sims_per_s": len(ok) / span, "latency_p50_s": float(np.percentile(lat, 50)),
                "latency_p99_s": float(np.percentile(lat, 99)), "makespan_s": span, "failed": failed,
                "steps": int(steps), "particle_steps_per_s": parts / span, "peak_device_gb": peak / (1 << 30),
                "streams": n_streams, "max_running": max_running}

    batched = serve(args.streams, 64)
    shortest = serve(args.streams, 64, policy=cube.CUBE_ADMIT_SHORTEST)
    sequential = serve(1, 1)
    cap_b = serve(args.streams, 64, at_once=True)          # capacity: every request queued at t = 0
    cap_s = serve(1, 1, at_once=True)
    sizes = sorted({r.workload.n_part_side for r in reqs})
    print(json.dumps({
        "metric": "sims/s (served, all requests queued at once)", "value": cap_b["sims_per_s"], "unit": "sims/s",
        "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded GRF Zel'dovich ICs)",
        "config": {"workload": f"C5 serving: {len(reqs)} requests, Poisson arrivals at 20/s, "
                               f"{sizes[0]}^3..{sizes[-1]}^3 particles (mesh 2x, 300 Mpc/h per 256 particles), "
                               "10-60 scheduled steps of Delta a 0.0196 from z=49, each cut so the fastest "
                               "particle drifts <= 0.5 coarse cell, sigma8 0.7-0.9, LCDM BBKS, x1v1",
                   "budget_gb": args.budget_gb,
                   "ics": "each request's own seeded Zel'dovich realisation at its sigma8, generated before the "
                          "timed region, pinned host memory, uploaded at admission"},
        "latency_p50_s": batched["latency_p50_s"], "latency_p99_s": batched["latency_p99_s"],
        "arrivals": {"rate_per_s": 20.0, "batched": batched, "batched_shortest_first": shortest,
                     "sequential": sequential},
        "capacity": {"batched": cap_b, "sequential": cap_s,
                     "speedup_vs_sequential": cap_b["sims_per_s"] / cap_s["sims_per_s"]},
    }), flush=True)


def main():
    args = parse()
    if args.ensemble:
        run_ensemble(args)
        return
    if args.serve:
        run_serve(args)
        return
    import dataclasses
    import synth
    w = synth.WORKLOADS[args.workload]
    if args.nps:
        w = dataclasses.replace(w, name=f"{w.name}@{args.nps}", n_part_side=args.nps, n_fine=2 * args.nps)
    if args.codes:
        xb, vb = (4, 4) if args.codes == "fp32" else (int(args.codes[1]), int(args.codes[3]))
        w = dataclasses.replace(w, x_bytes=xb, v_bytes=vb)
    if args.impl == "reference":
        run_reference(args, w)
        return
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1712_06121_gb300 as cube

    ic = synth.make_ics(w, seed=w.seed + rank)
    om, ol, _ = w.omega()
    prm = cube.make_params(w.n_fine, w.n_particles, ratio=w.ratio, x_bytes=w.x_bytes, v_bytes=w.v_bytes,
                           box=w.box, omega_m=om, omega_l=ol)
    stream = torch.cuda.Stream()
    ctx = cube.cube_create(prm, stream)
    pos_d = torch.from_numpy(ic.pos).cuda()
    vel_d = torch.from_numpy(ic.vel).cuda()
    ids_d = torch.from_numpy(ic.ids.view(np.int32)).cuda()
    torch.cuda.synchronize()
    cube.cube_encode(ctx, pos_d, vel_d, ids_d, w.a_init, ic.sigma_1d)
    sch = schedule(w, args.warmup + args.steps)
    for i in range(args.warmup):
        cube.cube_pm_step(ctx, sch[i], sch[i + 1])
    geo = {"brick": cube.cube_state_view(ctx).brick}
    launches0 = cube.cube_stats_get(ctx).kernel_launches
    cube.cube_profile(ctx, args.steps)
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.warmup, args.warmup + args.steps):
        cube.cube_pm_step(ctx, sch[i], sch[i + 1])
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    ms = ev0.elapsed_time(ev1)
    stats = cube.cube_stats_get(ctx)                      # raises on a latched device error
    launches = stats.kernel_launches - launches0
    phase_ms, phase_kernels, nst = cube.cube_profile_read(ctx)
    cube.cube_profile(ctx, 0)
    ms_max = max_over_ranks(ms, dist)
    value = world * w.n_particles * args.steps / (ms_max / 1e3)
    run = None if args.no_whole_run else whole_run(cube, ctx, ic, w, stream)

    # end to end through the C ABI with pinned host buffers: H2D of the
    # particles, encode, one step, decode, D2H, every iteration
    e2e = None
    e2e_ck = None
    e2e_ov = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(ic.pos).pin_memory()
        vel_h = torch.from_numpy(ic.vel).pin_memory()
        ids_h = torch.from_numpy(ic.ids.view(np.int32)).pin_memory()
        out_p = torch.empty_like(pos_h).pin_memory()
        out_v = torch.empty_like(vel_h).pin_memory()
        out_i = torch.empty_like(ids_h).pin_memory()
        n_e2e = max(3, min(args.steps, 10))
        for it in range(2):                                 # warm the staging buffers
            cube.cube_encode(ctx, pos_h, vel_h, ids_h, w.a_init, ic.sigma_1d)
            cube.cube_pm_step(ctx, sch[0], sch[1])
            cube.cube_decode(ctx, out_p, out_v, out_i)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(n_e2e):
            cube.cube_encode(ctx, pos_h, vel_h, ids_h, w.a_init, ic.sigma_1d)
            cube.cube_pm_step(ctx, sch[0], sch[1])
            cube.cube_decode(ctx, out_p, out_v, out_i)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nbytes = 28 * w.n_particles
        e2e = {"value": world * w.n_particles * n_e2e / max_over_ranks(dt, dist), "unit": "particle-steps/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "what": "per iteration: pinned host pos/vel/ids -> cube_encode -> cube_pm_step -> "
                       "cube_decode -> pinned host"}
        # the same loop on the compressed store's checkpoint (Section 2.3.1) instead of float particles
        ck = cube.cube_checkpoint_size(prm)
        ck_in = torch.empty(ck, dtype=torch.uint8).pin_memory()
        ck_out = torch.empty(ck, dtype=torch.uint8).pin_memory()
        cube.cube_encode(ctx, pos_h, vel_h, ids_h, w.a_init, ic.sigma_1d)
        cube.cube_pm_step(ctx, sch[0], sch[1])
        cube.cube_checkpoint_save(ctx, ck_in)
        for it in range(2):
            cube.cube_checkpoint_load(ctx, ck_in)
            cube.cube_pm_step(ctx, sch[1], sch[2])
            cube.cube_checkpoint_save(ctx, ck_out)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(n_e2e):
            cube.cube_checkpoint_load(ctx, ck_in)
            cube.cube_pm_step(ctx, sch[1], sch[2])
            cube.cube_checkpoint_save(ctx, ck_out)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_ck = {"value": world * w.n_particles * n_e2e / max_over_ranks(dt, dist), "unit": "particle-steps/s",
                  "h2d_bytes_per_step": ck, "d2h_bytes_per_step": ck,
                  "what": "per iteration: pinned host checkpoint of the compressed store -> cube_checkpoint_load "
                          "-> cube_pm_step -> cube_checkpoint_save -> pinned host"}
        e2e_ov = e2e_overlapped(cube, prm, ic, w, sch, n_e2e, dist, world)
    cube.cube_destroy(ctx)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_kind = peaks()
    pb = phase_bytes(w, geo)
    top = max((k for k in phase_ms if phase_kernels.get(k)), key=lambda k: phase_ms[k])
    per_launch_ms = phase_ms[top] / max(1, nst) / max(1, phase_kernels[top])
    achieved = pb[top] / (per_launch_ms / 1e3) / 1e9
    traffic = measured_traffic(top, w.name)
    step_frac = step_bytes(w) / (peak * 1e9) / (ms_max / args.steps / 1e3)
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded GRF Zel'dovich ICs)", "config": config_of(w),
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind},
        "step_roofline": {"bytes": step_bytes(w), "frac": step_frac, "model": step_model(w)},
        "phases_ms_per_step": {k: v / max(1, nst) for k, v in phase_ms.items()},
        "gpu_launches": int(launches),
        "tile_load": "tma" if stats.features & 1 else "cp.async",
        "clocks": clk,
        "e2e": e2e,
        "e2e_checkpoint": e2e_ck,
        "e2e_overlapped": e2e_ov,
        "whole_run": run,
    }
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
