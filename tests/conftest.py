import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libgmc.so")
    config.addinivalue_line("markers", "slow: long-running statistical test")


@pytest.fixture(scope="session")
def tmpdir_session(tmp_path_factory):
    return tmp_path_factory.mktemp("gmc")


@pytest.fixture(scope="session")
def gpu_ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    yield ctx
    ctx.close()


@pytest.fixture(scope="session")
def kaiming_file(tmp_path_factory):
    import synth
    p = tmp_path_factory.mktemp("w") / "kaiming_seed1.bin"
    synth.write_weights(str(p), synth.kaiming_weights(1))
    return str(p)
