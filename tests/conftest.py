import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libcube.so")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def build_lib():
    """Build libcube.so (loading build.py by path: the package refuses to
    import until the library exists) and return its path."""
    import importlib.util
    path = os.path.join(ROOT, "paper_1712_06121_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_cube_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
