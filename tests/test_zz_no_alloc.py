"""The allocation-free entry point cube_counts_to_offsets_noalloc.

Some callers cannot call cudaMalloc (code inside a CUDA-graph capture, a
pooled allocator that must own every allocation, a fixed-budget embedded
runtime).  This entry point gives them the cell-ordered store's offsets from
per-cell counts using only the library's fixed device scratch.  Its output
must equal the offsets that cube_encode and cube_pm_step build for the same
counts, on consecutive calls (the scratch keeps the previous call's
contents).  The file is named to be collected last.
"""
import numpy as np
import pytest

import synth

from gpu_util import device_view

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


def test_noalloc_offsets_match_the_store_on_consecutive_calls(cube):
    w = synth.WORKLOADS["pm64"]
    ic = synth.make_ics(w)                               # 64^3 particles, 32^3 coarse cells
    prm = cube.make_params(w.n_fine, w.n_particles, x_bytes=w.x_bytes, v_bytes=w.v_bytes, box=w.box)
    stream = torch.cuda.current_stream()
    ctx = cube.cube_create(prm, stream)
    try:
        cube.cube_encode(ctx, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
        sched = synth.uniform_schedule(w.a_init, w.a_final, w.n_steps)
        for call in range(2):
            st = cube.cube_state_view(ctx)
            ncc = st.n_coarse ** 3
            counts = device_view(st.counts, (ncc,), "<u4").clone()
            want = device_view(st.offsets, (ncc + 1,), "<u4").cpu().numpy()
            out = torch.full((ncc + 1,), -1, dtype=torch.int32, device="cuda")
            cube.cube_counts_to_offsets_noalloc(counts, ncc, out, stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), f"call {call}"
            assert got[-1] == w.n_particles
            cube.cube_pm_step(ctx, sched[call], sched[call + 1])    # a new store for the next call
    finally:
        cube.cube_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch(cube):
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(cube.CubeError) as e:
        cube.cube_counts_to_offsets_noalloc(dummy, (1 << 28) + 1, dummy)
    assert e.value.status == cube.CUBE_E_ARG
    assert "268435456" in cube.cube_last_error()
