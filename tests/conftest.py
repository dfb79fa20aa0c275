import ast
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests of the CUDA path)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def read_golden(name: str) -> dict:
    """key = value lines of a golden text file (comments start with #)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


def parse_configs(text: str):
    return [[int(x) for x in tok.split("-")] for tok in text.split()]


def parse_literal(text: str):
    return ast.literal_eval(text)


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def built_library():
    from paper_1104_1824_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def gpu(built_library):
    if not cuda_available():
        pytest.fail("the gpu-marked tests need a CUDA device")
    import paper_1104_1824_gb300 as snp
    return snp
