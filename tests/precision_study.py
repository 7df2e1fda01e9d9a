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
table (needs a GPU).
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
        cube.cube_decode(ctx, pos, vel, ids)
        k, pk, nm = (np.empty(n_bins) for _ in range(3))
        cube.cube_power_spectrum(ctx, n_bins, k, pk, nm)
    finally:
        cube.cube_destroy(ctx)
    order = np.argsort(ids, kind="stable")
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

    print(table(run_study(cube, torch)))
