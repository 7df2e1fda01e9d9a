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
            c = counts.cpu().numpy().view(np.uint32).astype(np.int64)
            assert np.array_equal(got, np.concatenate([[0], np.cumsum(c)])), f"call {call}"
            assert got[-1] == w.n_particles
            cube.cube_pm_step(ctx, sched[call], sched[call + 1])    # a new store for the next call
    finally:
        cube.cube_destroy(ctx)


def _offsets(counts):
    return np.concatenate([[0], np.cumsum(counts.astype(np.int64))]).astype(np.uint32)


def test_noalloc_many_blocks_on_consecutive_calls(cube):
    """5,000,003 cells (1,221 scan blocks, more than one pass of the block-sum
    scan, and a ragged last block) with random counts, twice in a row with
    different counts, against numpy's cumulative sum (totals below 2^32)."""
    rng = np.random.default_rng(1712)
    n = 5_000_003
    stream = torch.cuda.current_stream()
    for call in range(2):
        c = rng.integers(0, 600 if call == 0 else 17, n).astype(np.uint32)
        counts = torch.from_numpy(c.view(np.int32)).cuda()
        out = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
        cube.cube_counts_to_offsets_noalloc(counts, n, out, stream)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), _offsets(c)), f"call {call}"


@pytest.mark.parametrize("n", [1, 3, 4097, 12345])
def test_noalloc_unaligned_arrays(cube, n):
    """Arrays that do not start on a 16-byte boundary and sizes that are not
    a multiple of 4 take the scalar loads and stores; one cell is the
    smallest case."""
    rng = np.random.default_rng(n)
    stream = torch.cuda.current_stream()
    for call in range(2):
        c = rng.integers(0, 1000, n).astype(np.uint32)
        base = torch.zeros(n + 3, dtype=torch.int32, device="cuda")
        base[1:n + 1] = torch.from_numpy(c.view(np.int32)).cuda()
        counts = base[1:n + 1]                             # 4 bytes past a 256-byte boundary
        outb = torch.full((n + 4,), -1, dtype=torch.int32, device="cuda")
        out = outb[3:n + 4]                                # 12 bytes past it
        assert counts.data_ptr() % 16 and out.data_ptr() % 16
        cube.cube_counts_to_offsets_noalloc(counts, n, out, stream)
        torch.cuda.synchronize()
        got = outb.cpu().numpy().view(np.uint32)
        assert np.array_equal(got[3:], _offsets(c)), f"call {call}"
        assert np.all(got[:3] == np.uint32(0xffffffff))    # nothing written before the array


def test_noalloc_rejects_sizes_beyond_its_scratch(cube):
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(cube.CubeError) as e:
        cube.cube_counts_to_offsets_noalloc(dummy, (1 << 28) + 1, dummy)
    assert e.value.status == cube.CUBE_E_ARG
    assert "268435456" in cube.cube_last_error()
