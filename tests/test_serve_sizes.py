"""Serving, host side (no GPU): the device footprint the server admits by.

A resident request holds its state: two copies of the compressed store (the
step writes the re-sorted store beside the old one), so per particle
2 (3 n_chi + 3 n_nu + 4 id) bytes, per coarse cell 2 x 20 bytes (count,
offset, v_c), plus codec tables (up to 1.3 MB for 2-byte velocities); the
uncompressed FP32 store is updated in place (24 + 4 bytes per particle,
once).  The work area a stream shares holds the padded mesh 4 N^2 (N + 4),
the ghosted potential 4 (N + 8)(N + 5)^2, the encode scratch (keys,
permutation, radix sort buffers) and host staging (about 44 bytes per
particle) and the step histograms.  These bounds are the paper's memory
argument (Section 2.3, Table t.memory) in this layout.
"""
import pytest


@pytest.fixture(scope="module")
def cube():
    from conftest import build_lib
    build_lib()
    import paper_1712_06121_gb300 as c
    return c


@pytest.mark.parametrize("nps,xb,vb", [(256, 1, 1), (128, 1, 2), (64, 2, 2), (96, 2, 1), (48, 4, 4)])
def test_state_and_work_bytes_follow_the_layout(cube, nps, xb, vb):
    nf = 2 * nps
    n, ncc = nps ** 3, (nf // 4) ** 3
    sb, wb = cube.cube_server_sizes(cube.make_params(nf, n, x_bytes=xb, v_bytes=vb))
    if xb == 4:
        lo = 28 * n + 2 * 20 * ncc
    else:
        lo = 2 * (3 * xb + 3 * vb + 4) * n + 2 * 20 * ncc
    assert lo <= sb <= 1.01 * lo + (2 << 20)
    mesh = 4 * nf * nf * (nf + 4) + 4 * (nf + 8) * (nf + 5) ** 2
    assert mesh + 28 * n <= wb <= 1.01 * (mesh + 48 * n + 40 * ncc) + (1 << 20)


def test_compressed_state_is_a_small_part_of_a_request(cube):
    """x1v1 at 256^3 particles: the resident state is about a fifth of the
    work area; a stream's work area serves all its requests."""
    sb, wb = cube.cube_server_sizes(cube.make_params(512, 256 ** 3))
    assert sb < 0.25 * wb
    assert sb / 256 ** 3 < 26                     # bytes per particle, both stores and ids


def test_sizes_grow_with_the_request(cube):
    last = (0, 0)
    for nps in (32, 48, 64, 96, 128):
        sb, wb = cube.cube_server_sizes(cube.make_params(2 * nps, nps ** 3))
        assert sb > last[0] and wb > last[1]
        last = (sb, wb)


@pytest.mark.parametrize("field,value", [("n_fine", 100), ("x_bytes", 3), ("ratio", 3), ("n_particles", 0)])
def test_invalid_params_are_rejected(cube, field, value):
    prm = cube.make_params(64, 32 ** 3)
    setattr(prm, field, value)
    with pytest.raises(cube.CubeError) as e:
        cube.cube_server_sizes(prm)
    assert e.value.status == cube.CUBE_E_ARG


def test_server_argument_checks(cube):
    import ctypes
    for args in ((0, 1, 1), (1 << 30, 0, 1), (1 << 30, 65, 1), (1 << 30, 2, 0)):
        with pytest.raises(cube.CubeError) as e:
            cube.cube_server_create(*args)
        assert e.value.status == cube.CUBE_E_ARG
    assert cube._lib.cube_server_destroy(None) == cube.CUBE_OK
    nr = ctypes.c_int32()
    assert cube._lib.cube_server_pump(None, ctypes.byref(nr), ctypes.byref(nr)) == cube.CUBE_E_ARG
    assert cube._lib.cube_server_release(None, 1) == cube.CUBE_E_ARG


@pytest.mark.parametrize("nps,xb,vb,ids", [(256, 1, 1, 4), (64, 2, 2, 0), (48, 4, 4, 4), (64, 1, 1, 1), (32, 1, 2, 2)])
def test_checkpoint_size_follows_the_documented_layout(cube, nps, xb, vb, ids):
    """64-byte header, then counts, v_c, chi, nu, ids, each 16-byte aligned
    (uncompressed: positions and momenta as floats)."""
    nf = 2 * nps
    n, ncc = nps ** 3, (nf // 4) ** 3
    a16 = lambda x: (x + 15) // 16 * 16
    if xb == 4:
        want = 64 + a16(12 * n) + a16(12 * n) + a16(4 * n if ids else 0)
    else:
        want = 64 + a16(4 * ncc) + a16(12 * ncc) + a16(3 * n * xb) + a16(3 * n * vb) + a16(ids * n)
    got = cube.cube_checkpoint_size(cube.make_params(nf, n, x_bytes=xb, v_bytes=vb, id_bytes=ids))
    assert got == want
