"""Section 2.1's 1-byte coarse density field (cube_counts_pack / _unpack,
host code): a byte per cell, the count itself below 255, 255 for a cell of
255 or more particles whose count follows in a 4-byte list in cell order.
Checked against that definition on the oracle's counts of a near-uniform
store (no overflow) and of a clustered one, and on the edge values 254,
255 and 2^32 - 1; malformed inputs are refused."""
import numpy as np
import pytest

import synth
from oracle import pm


@pytest.fixture(scope="module")
def cube():
    from conftest import build_lib
    build_lib()
    import paper_1712_06121_gb300 as c
    return c


def _check(cube, counts):
    b, ov = cube.cube_counts_pack(counts)
    assert np.array_equal(b, np.minimum(counts, 255).astype(np.uint8))
    assert np.array_equal(ov, counts[counts >= 255])
    assert np.array_equal(cube.cube_counts_unpack(b, ov), counts)
    return b, ov


def test_store_counts_round_trip(cube):
    w = synth.WORKLOADS["pm64"]
    ic = synth.make_ics(w, n_part_side=32, n_fine=64)
    P = pm.Params(n_fine=64, n_particles=32 ** 3)
    st = pm.encode(P, ic.pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
    b, ov = _check(cube, st.counts.astype(np.uint32))
    assert ov.size == 0 and int(b.sum()) == 32 ** 3            # 8 per coarse cell, none above 254
    # a clustered store: 5000 particles in one fine cell's neighbourhood
    pos = ic.pos.copy()
    pos[:, :5000] = np.float32(20.3)
    st = pm.encode(P, pos, ic.vel, ic.ids, w.a_init, ic.sigma_1d)
    counts = st.counts.astype(np.uint32)
    b, ov = _check(cube, counts)
    assert ov.size >= 1 and int(counts.sum()) == 32 ** 3
    assert np.array_equal(np.flatnonzero(b == 255), np.flatnonzero(counts >= 255))


def test_edge_values_and_errors(cube):
    counts = np.array([0, 254, 255, 256, 2 ** 32 - 1, 1], np.uint32)
    _check(cube, counts)
    _check(cube, np.zeros(0, np.uint32))
    with pytest.raises(cube.CubeError):
        cube.cube_counts_unpack(np.array([255, 1], np.uint8), np.zeros(0, np.uint32))      # missing entry
    with pytest.raises(cube.CubeError):
        cube.cube_counts_unpack(np.array([3, 1], np.uint8), np.array([300], np.uint32))      # extra entry
    with pytest.raises(cube.CubeError):
        cube.cube_counts_unpack(np.array([255], np.uint8), np.array([7], np.uint32))         # entry below 255
