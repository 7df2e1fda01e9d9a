"""The C-ABI library builds, loads and exports every entry point that
include/cube.h declares; argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cube.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cube_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from conftest import build_lib
    return ctypes.CDLL(build_lib())


def test_header_declares_the_api():
    names = _declared()
    for need in ("cube_create", "cube_destroy", "cube_encode", "cube_pm_step", "cube_decode",
                 "cube_power_spectrum", "cube_last_error"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_has_the_same_names(lib):
    import paper_1712_06121_gb300 as cube
    for name in _declared():
        assert callable(getattr(cube, name)), name


@pytest.mark.parametrize("field,value", [("n_fine", 100), ("n_fine", 2048), ("ratio", 3), ("x_bytes", 3),
                                         ("x_bytes", 4),
                                         ("v_bytes", 0), ("id_bytes", 3), ("deconv_power", 5), ("brick", 3),
                                         ("n_particles", 0), ("gradient", 7)])
def test_invalid_params_are_rejected_before_any_device_call(lib, field, value):
    import paper_1712_06121_gb300 as cube
    prm = cube.make_params(64, 32 ** 3)
    setattr(prm, field, value)
    with pytest.raises(cube.CubeError) as e:
        cube.cube_create(prm)
    assert e.value.status == cube.CUBE_E_ARG
    assert cube.cube_last_error()


def test_null_context_is_an_argument_error(lib):
    import paper_1712_06121_gb300 as cube
    assert lib.cube_destroy(None) == cube.CUBE_OK
    for fn, args in (("cube_pm_step", (ctypes.c_double(0.1), ctypes.c_double(0.2))),
                     ("cube_decode", (None, None, None)),
                     ("cube_keep_drifted", (ctypes.c_int32(1),))):
        assert getattr(lib, fn)(None, *args) == cube.CUBE_E_ARG
