"""The 256^3-particle LCDM workload as stated: 256^3 particles on a 512^3
FP32 mesh in a 300 Mpc/h box, Zel'dovich ICs at z = 49, 1-byte positions and
velocities, 50 steps uniform in a to z = 0 on the GPU; its final power
spectrum, and the error against the FP64 oracle's run of the same seed at
128^3 particles on a 256^3 mesh (the same mode-keyed white noise, so both
runs share their large-scale modes) with the same 50 steps.

If a uniform step moves a particle more than one coarse cell, the library
clamps the move and reports CUBE_E_MIGRATION; the run then repeats with
every step cut by cube_next_epoch_limited (the fastest particle drifts at
most half a coarse cell) and says so.

Test code: it runs the oracle.  `python tests/c2_run.py [out.json]` (needs
a GPU) prints one JSON object: the schedule used, the largest migration,
k, P_gpu(k), P_oracle(k), and max |P_gpu / P_oracle - 1| below several k.
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
from oracle import pm  # noqa: E402


def gpu_run(w, ic):
    import torch
    import paper_1712_06121_gb300 as cube
    om, ol, _ = w.omega()
    prm = cube.make_params(w.n_fine, w.n_particles, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                           omega_m=om, omega_l=ol)
    uniform = list(synth.uniform_schedule(w.a_init, w.a_final, w.n_steps))
    nb = w.n_fine // 2

    def run(limited):
        ctx = cube.cube_create(prm, torch.cuda.current_stream())
        try:
            cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
            sch, a = [w.a_init], w.a_init
            for t in uniform[1:]:
                while a < t:
                    a_to = cube.cube_next_epoch_limited(ctx, t, 0.5)[0] if limited else t
                    cube.cube_pm_step(ctx, a, a_to)
                    sch.append(a_to)
                    a = a_to
            st = cube.cube_stats_get(ctx)                    # raises CUBE_E_MIGRATION on a clamped move
            k, pk, nm = (np.empty(nb) for _ in range(3))
            cube.cube_power_spectrum(ctx, nb, k, pk, nm)
            return sch, st.max_migration, k, pk, nm
        finally:
            cube.cube_destroy(ctx)

    try:
        return "uniform", run(False)
    except cube.CubeError as e:
        if e.status != cube.CUBE_E_MIGRATION:
            raise
        return "velocity-limited", run(True)


def main(out=None):
    w = synth.WORKLOADS["pm256"]
    ic = synth.make_ics(w)
    t0 = time.time()
    kind, (sch, mig, k, pk, nm) = gpu_run(w, ic)
    t_gpu = time.time() - t0
    # the oracle at 128^3 particles / 256^3 mesh, same seed and epochs
    nps = 128
    ico = synth.make_ics(w, n_part_side=nps, n_fine=2 * nps)
    om, ol, _ = w.omega()
    P = pm.Params(n_fine=2 * nps, n_particles=nps ** 3, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box,
                  omega_m=om, omega_l=ol)
    t0 = time.time()
    st = pm.run(pm.encode(P, ico.pos, ico.vel, ico.ids, w.a_init, ico.sigma_1d), sch)
    t_or = time.time() - t0
    nbo = nps
    ko, po, mo = pm.power_spectrum(st, nbo)
    # the same shells (same box, same fundamental mode): bins 1 .. nbo
    r = pk[:nbo] / po - 1
    kny_o = np.pi * 2 * nps / w.box
    res = {"schedule": f"{kind}, {len(sch) - 1} steps z={1 / w.a_init - 1:g} -> {1 / sch[-1] - 1:g}",
           "max_migration": int(mig), "gpu_s": t_gpu, "oracle_s": t_or,
           "k": [float(x) for x in k[:nbo]], "P_gpu": [float(x) for x in pk[:nbo]],
           "P_oracle": [float(x) for x in po],
           "max_rel_err": {f"k<{kc:g}": float(np.max(np.abs(r[ko < kc]))) for kc in (0.1, 0.2, 0.5, kny_o / 2)},
           "k_nyquist_oracle": kny_o}
    s = json.dumps(res)
    if out:
        with open(out, "w") as f:
            f.write(s + "\n")
    print(json.dumps({kk: v for kk, v in res.items() if kk not in ("k", "P_gpu", "P_oracle")}))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
