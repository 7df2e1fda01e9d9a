"""The bench's algorithmic-byte model, CPU only: the whole-step minimum
B_step = (3s + 3 n_nu) N_p + 32 N_c^3 + 32 N_f^3 (s = 3 n_chi + 3 n_nu:
pass A reads the codes and writes the kicked nu, pass B reads and writes
the codes; 32 bytes per coarse cell of offsets, v_c, counts and new v_c;
per mesh cell the density write, the r2c sweeps' read and write, the z
sweep's read and write, the c2r sweeps' read and write and the gather's
read, 4 bytes each) at each workload's sizes, the per-kernel bytes the
roofline divides by, and the traffic record's key on the kernel sources."""
import dataclasses

import pytest

import bench
import synth


@pytest.mark.parametrize("name,xb,vb,want", [
    ("pm64", 1, 2, 64 ** 3 * (3 * 9 + 6) + 32 * 32 ** 3 + 32 * 128 ** 3),
    ("pm256", 1, 1, 256 ** 3 * (3 * 6 + 3) + 32 * 128 ** 3 + 32 * 512 ** 3),
    ("pm512", 1, 1, 512 ** 3 * (3 * 6 + 3) + 32 * 256 ** 3 + 32 * 1024 ** 3),
    ("pm512", 2, 2, 512 ** 3 * (3 * 12 + 6) + 32 * 256 ** 3 + 32 * 1024 ** 3),
    ("pm512", 4, 4, 512 ** 3 * 60 + 32 * 1024 ** 3),
])
def test_step_bytes(name, xb, vb, want):
    w = dataclasses.replace(synth.WORKLOADS[name], x_bytes=xb, v_bytes=vb)
    assert bench.step_bytes(w) == want


def test_step_bytes_at_the_published_sizes():
    """4.71 GB per step at 256^3 / 512^3 x1v1, 37.7 / 40.5 / 42.4 GB at
    512^3 / 1024^3 for x1v1, x2v2 and FP32, 77 MB at 64^3 / 128^3 x1v2."""
    pm512 = synth.WORKLOADS["pm512"]
    got = [bench.step_bytes(synth.WORKLOADS["pm256"]) / 1e9,
           bench.step_bytes(pm512) / 1e9,
           bench.step_bytes(dataclasses.replace(pm512, x_bytes=2, v_bytes=2)) / 1e9,
           bench.step_bytes(dataclasses.replace(pm512, x_bytes=4, v_bytes=4)) / 1e9,
           bench.step_bytes(synth.WORKLOADS["pm64"]) / 1e6]
    assert [round(g, 2 if i == 0 else 1) if i < 4 else round(g) for i, g in enumerate(got)] == [4.71, 37.7, 40.5,
                                                                                                 42.4, 77]


def test_phase_bytes_cover_the_minimum():
    """The kernels move at least B_step: five FFT sweeps of the half-complex
    mesh (read + write each) instead of the fused minimum, separate deposit
    and gather passes."""
    w = synth.WORKLOADS["pm256"]
    pb = bench.phase_bytes(w, {"brick": 4})
    half = 512 * 512 * 257 * 8
    assert pb["fft_y_fwd"] == pb["fft_z_green"] == pb["fft_y_inv"] == 2 * half
    assert pb["fft_x_r2c"] == pb["fft_x_c2r"] == 4 * 512 ** 3 + half
    assert pb["pass_a"] > (3 + 6) * w.n_particles + 4 * 512 ** 3
    assert sum(pb.values()) >= bench.step_bytes(w)


def test_traffic_record_is_keyed_on_the_kernel_sources():
    """The committed DRAM traffic applies only to the kernel sources it was
    captured on; the key ignores host-only files."""
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    t = bench.measured_traffic("pass_a", "pm256")
    assert t is None or t > 0
    assert bench.measured_traffic("pass_a", "no_such_workload") is None
