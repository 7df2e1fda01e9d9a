"""A matched-resolution nonlinear run to z = 0: 64^3 particles on a 128^3
mesh in a 75 Mpc/h box (the 256^3 workload's resolution), flat LCDM with the
BBKS spectrum, z = 49 -> 0 in 50 uniform steps, on the GPU and in the FP64
oracle with the same steps and the same code widths.

* P(k): within 0.5% of the oracle's at k < k_Nyquist / 2 (the stated
  tolerance), for 1- and 2-byte codes.
* Displacements (particles matched by id): in the nonlinear regime the FP32
  force differs from the oracle's FP64 force by about 1e-5 of its largest
  value, which decides some velocity codes on the other side of a threshold;
  a flipped code moves a particle by a bin width, and orbits in collapsed
  structures separate the two runs further.  The 1e-3 fine-cell RMS gate
  holds for the linear 10-step run (test_full_run_pm64_matches_oracle) but
  not here, so this test gates the GPU-oracle separation against the
  method's own error at the same resolution: the RMS and the median
  displacement between the GPU and the oracle must not exceed those between
  the oracle's compressed run and its uncompressed FP64 run (the error the
  paper's compression itself makes, Section 3).  Measured on GB300, GPU vs
  oracle against compressed vs uncompressed (RMS / median, fine cells):
  x1v1 0.31 / 0.035 against 0.62 / 0.25, x1v2 0.026 / 0 against 0.50 /
  0.23, x2v2 0.0018 / 0.0003 against 0.0035 / 0.0010; P(k) within 3.6e-3,
  6.3e-4 and 2.0e-5.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import pm

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


def _matched(ids_a, pa, ids_b, pb, n):
    d = pa[:, np.argsort(ids_a)].astype(np.float64) - pb[:, np.argsort(ids_b)].astype(np.float64)
    d -= n * np.round(d / n)
    return np.sqrt(np.sum(d * d, axis=0))


@pytest.mark.parametrize("xb,vb", [(1, 1), (1, 2), (2, 2)])
def test_lcdm_run_to_z0_matches_oracle(cube, xb, vb):
    base = synth.WORKLOADS["pm256"]
    w = dataclasses.replace(base, n_part_side=64, n_fine=128, box=base.box * 64 / 256, x_bytes=xb, v_bytes=vb)
    ic = synth.make_ics(w)
    om, ol, _ = w.omega()
    n = w.n_particles
    sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
    nb = w.n_fine // 2
    prm = cube.make_params(w.n_fine, n, x_bytes=xb, v_bytes=vb, box=w.box, omega_m=om, omega_l=ol)
    ctx = cube.cube_create(prm, torch.cuda.current_stream())
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        for i in range(w.n_steps):
            cube.cube_pm_step(ctx, sched[i], sched[i + 1])
        assert cube.cube_stats_get(ctx).max_migration <= 1
        pos, vel, ids = np.empty((3, n), np.float32), np.empty((3, n), np.float32), np.empty(n, np.uint32)
        cube.cube_decode(ctx, pos, vel, ids)
        k, pk, nm = (np.empty(nb) for _ in range(3))
        cube.cube_power_spectrum(ctx, nb, k, pk, nm)
    finally:
        cube.cube_destroy(ctx)
    P = pm.Params(n_fine=w.n_fine, n_particles=n, x_bytes=xb, v_bytes=vb, box=w.box, omega_m=om, omega_l=ol)
    st = pm.run(pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d), sched)
    rpos, _, rids = pm.decode(st)
    ex = pm.exact_run(pm.exact_from(P, np.mod(ic.pos.astype(np.float64), w.n_fine), ic.vel, w.a_init), sched)
    rk, rp, rm = pm.power_spectrum(st, nb)
    assert np.array_equal(nm, rm)
    sel = k < 0.5 * np.pi * w.n_fine / w.box
    dP = np.max(np.abs(pk[sel] / rp[sel] - 1))
    assert dP <= 5e-3, dP
    d_gpu = _matched(ids, pos, rids, rpos, w.n_fine)
    d_codec = _matched(rids, rpos, ic.ids, ex.pos, w.n_fine)
    rms_gpu, rms_codec = np.sqrt(np.mean(d_gpu ** 2)), np.sqrt(np.mean(d_codec ** 2))
    print(f"x{xb}v{vb}: dP {dP:.2e}, RMS gpu-oracle {rms_gpu:.3g}, compressed-exact {rms_codec:.3g}, "
          f"median {np.median(d_gpu):.3g} / {np.median(d_codec):.3g}")
    assert rms_gpu <= rms_codec, (rms_gpu, rms_codec)
    assert np.median(d_gpu) <= np.median(d_codec), (np.median(d_gpu), np.median(d_codec))
