"""Precision study of the compressed store (the experiment of Section 3):
every code width x1v1 ... x2v2 and the uncompressed FP32 store, run on the
GPU from the same initial conditions, against the oracle's uncompressed FP64
PM run (oracle.pm.exact_run) with the same force and time steps.

Per configuration, at the final epoch:
  dx      |x - x_ref| of each particle (matched by ID, periodic), fine cells:
          median, 99th percentile and maximum (the displacement offsets of
          Eq. offset);
  dP      largest |P(k) / P_ref(k) - 1| for k below half the mesh Nyquist;
  1 - r   largest 1 - xi(k) there, xi = P_ab / sqrt(P_aa P_bb) the
          cross-correlation coefficient of Eq. ccc between the two density
          fields.

Test code: it runs the oracle.  `python tests/precision_study.py` prints the
table (needs a GPU); `--c3` runs the study at 512^3 particles (run_c3).
"""
import dataclasses
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
from oracle import mesh, pm  # noqa: E402

CONFIGS = [("x1v1", 1, 1), ("x1v2", 1, 2), ("x2v1", 2, 1), ("x2v2", 2, 2), ("fp32", 4, 4)]


def study_workload():
    """64^3 particles on a 128^3 mesh in an 80 Mpc/h LCDM box (the paper's
    S256 box and cosmology class at 1/64 of its particles), a = 0.02 -> 1 in
    50 steps uniform in a."""
    w = synth.WORKLOADS["pm256"]
    return dataclasses.replace(w, name="study64", n_part_side=64, n_fine=128, box=80.0)


def _density_modes(pos, n, mass):
    rho = mesh.cic_deposit(np.mod(np.asarray(pos, np.float64), n), n, mass)
    return np.fft.rfftn(rho / rho.mean() - 1.0)


def cross_correlation(pos_a, pos_b, n, mass, n_bins):
    """xi(k) = P_ab / sqrt(P_aa P_bb) over shells i - 1/2 <= |n| < i + 1/2
    (Eq. ccc), r2c modes weighted 2 except on the kx = 0, N/2 planes."""
    da, db = _density_modes(pos_a, n, mass), _density_modes(pos_b, n, mass)
    f = np.fft.fftfreq(n, 1.0 / n).astype(np.int64)
    fx = np.arange(n // 2 + 1, dtype=np.int64)
    shell = mesh.shell_index(f[:, None, None] ** 2 + f[None, :, None] ** 2 + fx[None, None, :] ** 2)
    wgt = np.full(da.shape, 2.0)
    wgt[:, :, 0] = 1.0
    wgt[:, :, n // 2] = 1.0
    ok = (shell >= 1) & (shell <= n_bins)
    idx = shell[ok] - 1
    pab = np.bincount(idx, (wgt * (da * np.conj(db)).real)[ok], n_bins)
    paa = np.bincount(idx, (wgt * np.abs(da) ** 2)[ok], n_bins)
    pbb = np.bincount(idx, (wgt * np.abs(db) ** 2)[ok], n_bins)
    return pab / np.sqrt(paa * pbb)


def run_gpu(cube, torch, w, ic, xb, vb, sched, n_bins):
    """One GPU run; run_gpu.note says whether the one-cell migration limit
    had to clamp a particle (the run then continues with the clamped move)."""
    om, ol, _ = w.omega()
    n = w.n_particles
    prm = cube.make_params(w.n_fine, n, x_bytes=xb, v_bytes=vb, box=w.box, omega_m=om, omega_l=ol)
    ctx = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        sigma = ic.sigma_1d if xb != 4 else 0.0
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, sched[0], sigma)
        for i in range(len(sched) - 1):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
        pos = np.empty((3, n), np.float32)
        vel = np.empty((3, n), np.float32)
        ids = np.empty(n, np.uint32)
        note = ""
        try:
            cube.cube_decode(ctx, pos, vel, ids)
        except cube.CubeError as e:          # the particles are copied out before a latched error is reported
            if e.status != cube.CUBE_E_MIGRATION:
                raise
            note = "migration clamped"
        k, pk, nm = (np.empty(n_bins) for _ in range(3))
        try:
            cube.cube_power_spectrum(ctx, n_bins, k, pk, nm)
        except cube.CubeError as e:
            if e.status != cube.CUBE_E_MIGRATION:
                raise
    finally:
        cube.cube_destroy(ctx)
    order = np.argsort(ids, kind="stable")
    run_gpu.note = note
    return pos[:, order], k, pk


def run_study(cube, torch, configs=CONFIGS):
    w = study_workload()
    ic = synth.make_ics(w)
    n, nf = w.n_particles, w.n_fine
    sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    om, ol, _ = w.omega()
    P = pm.Params(n_fine=nf, n_particles=n, x_bytes=1, v_bytes=1, box=w.box, omega_m=om, omega_l=ol)
    ref = pm.exact_run(pm.exact_from(P, np.mod(ic.pos.astype(np.float64), nf), ic.vel, w.a_init), sched)
    n_bins = nf // 2
    rk, rp, _ = mesh.power_spectrum(ref.pos, nf, P.mass, w.box, n_bins)
    sel = rk < 0.5 * np.pi * nf / w.box
    out = {}
    for name, xb, vb in configs:
        pos, k, pk = run_gpu(cube, torch, w, ic, xb, vb, sched, n_bins)
        d = pos.astype(np.float64) - ref.pos          # ICs are in ID order
        d -= nf * np.round(d / nf)
        dx = np.sqrt(np.sum(d * d, axis=0))
        xi = cross_correlation(pos, ref.pos, nf, P.mass, n_bins)
        out[name] = {"dx_median": float(np.median(dx)), "dx_p99": float(np.percentile(dx, 99)),
                     "dx_max": float(dx.max()), "dP": float(np.max(np.abs(pk[sel] / rp[sel] - 1))),
                     "one_minus_r": float(np.max(1.0 - xi[sel])),
                     "bytes_per_particle": (3 * xb + 3 * vb) if xb != 4 else 24}
    return out


def run_c3(cube, torch, configs=(("fp32", 4, 4), ("x1v1", 1, 1), ("x1v2", 1, 2), ("x2v1", 2, 1), ("x2v2", 2, 2)),
           oracle_nps=128):
    """The study at the C3 size: 512^3 particles, 1024^3 mesh, 600 Mpc/h,
    z = 49 -> 0 in 50 steps.  Each code width against the uncompressed FP32
    run at the same resolution (the compression error alone), and every
    run's large-scale P(k) against the oracle's uncompressed FP64 run of the
    same seed at 128^3 particles / 256^3 mesh (mode-keyed noise: the same
    realisation on those scales), for k below half that mesh's Nyquist."""
    w = synth.WORKLOADS["pm512"]
    ic = synth.make_ics(w)
    n, nf = w.n_particles, w.n_fine
    sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    n_bins = nf // 2
    runs, notes = {}, {}
    for name, xb, vb in configs:
        runs[name] = run_gpu(cube, torch, w, ic, xb, vb, sched, n_bins)
        notes[name] = run_gpu.note
    del ic
    # oracle at 128^3 / 256^3, same seed and box
    wo = dataclasses.replace(w, n_part_side=oracle_nps, n_fine=2 * oracle_nps)
    ico = synth.make_ics(wo)
    om, ol, _ = w.omega()
    P = pm.Params(n_fine=wo.n_fine, n_particles=wo.n_particles, x_bytes=1, v_bytes=1, box=w.box, omega_m=om,
                  omega_l=ol)
    ref = pm.exact_run(pm.exact_from(P, np.mod(ico.pos.astype(np.float64), wo.n_fine), ico.vel, w.a_init), sched)
    ok_, op_, _ = mesh.power_spectrum(ref.pos, wo.n_fine, P.mass, w.box, wo.n_fine // 2)
    base_pos, base_k, base_pk = runs["fp32"]
    kmax_o = 0.5 * np.pi * wo.n_fine / w.box
    out = {}
    for name, xb, vb in configs:
        pos, k, pk = runs[name]
        d = pos.astype(np.float64) - base_pos
        d -= nf * np.round(d / nf)
        dx = np.sqrt(np.sum(d * d, axis=0))
        sel = k < 0.5 * np.pi * nf / w.box
        # P(k) of the shells both meshes resolve (shell i has the same |n| on both: same k)
        m = min(len(op_), len(pk))
        lo = (ok_[:m] < kmax_o)
        out[name] = {"dx_median": float(np.median(dx)), "dx_p99": float(np.percentile(dx, 99)),
                     "dx_max": float(dx.max()), "dP_vs_fp32": float(np.max(np.abs(pk[sel] / base_pk[sel] - 1))),
                     "dP_vs_oracle128_lowk": float(np.max(np.abs(pk[:m][lo] / op_[:m][lo] - 1))),
                     "bytes_per_particle": (3 * xb + 3 * vb) if xb != 4 else 24, "note": notes[name]}
    return out


def table_c3(res):
    lines = ["| store | bytes/particle | dx vs FP32 median | p99 | max | max dP vs FP32 (k < k_Ny/2) | "
             "max dP vs oracle 128^3 (k < k_Ny(256)/2) | note |", "|---|---:|---:|---:|---:|---:|---:|---|"]
    for name, r in res.items():
        lines.append(f"| {name} | {r['bytes_per_particle']} | {r['dx_median']:.2e} | {r['dx_p99']:.2e} | "
                     f"{r['dx_max']:.2e} | {r['dP_vs_fp32']:.2e} | {r['dP_vs_oracle128_lowk']:.2e} | {r['note']} |")
    return "\n".join(lines)


def table(res):
    lines = ["| store | bytes/particle (codes) | dx median | dx p99 | dx max | max dP (k < k_Ny/2) | max 1 - r |",
             "|---|---:|---:|---:|---:|---:|---:|"]
    for name, r in res.items():
        lines.append(f"| {name} | {r['bytes_per_particle']} | {r['dx_median']:.2e} | {r['dx_p99']:.2e} | "
                     f"{r['dx_max']:.2e} | {r['dP']:.2e} | {r['one_minus_r']:.2e} |")
    return "\n".join(lines)


if __name__ == "__main__":
    import torch

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from conftest import build_lib

    build_lib()
    import paper_1712_06121_gb300 as cube

    if "--c3" in sys.argv:
        print(table_c3(run_c3(cube, torch)))
    else:
        print(table(run_study(cube, torch)))
