import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: takes more than ~20 s on the CPU")


def pytest_collection_modifyitems(config, items):
    # keep collection order by file name; nothing else to reorder
    return None


def build_library():
    """Compile libbempol.so if needed (the build script is loaded by path: importing the
    package itself requires the compiled library)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_1810_03698_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("bempol_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


@pytest.fixture(scope="session")
def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
