import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="session")
def hsc(torch_cuda):
    """The CUDA binding with libhsc.so built in-tree (fails when it cannot be)."""
    import paper_2404_10631_gb300 as pkg
    from paper_2404_10631_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.fixture(scope="session")
def ctx(hsc):
    """A context launching on torch's current stream: torch's fills, copies
    and edits of the test tensors and the library's kernels are then ordered
    on one stream (a context with a stream of its own does not wait for them)."""
    import torch
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    c = hsc.Context(0, stream=s)
    yield c
    c.close()
