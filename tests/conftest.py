import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def oracle_theta(orc):
    """v_theta fitted by the ORACLE's own FP64 gradient and Adam step (600
    full-batch steps on 1024 seeded points) to the manufactured solution
    u = sin(pi x) cos(pi y) + x y of the config-2 and config-5 PDE; returned as
    the float32 values both sides then use (the GPU stages them, the oracle
    reads them back in FP64).  Nothing in it comes from the CUDA library."""
    import numpy as np
    from paper_2301_05780_gb300 import workloads as W
    rng = np.random.default_rng(7)
    xy = rng.uniform(0, 1, size=(1024, 2))
    tgt = np.sin(np.pi * xy[:, 0]) * np.cos(np.pi * xy[:, 1]) + xy[:, 0] * xy[:, 1]
    th = W.mlp_init().astype(np.float64)
    m, v = np.zeros_like(th), np.zeros_like(th)
    for t in range(1, 601):
        _, g = orc.mlp_loss_grad(th, xy, tgt)
        orc.adam_step(th, g, m, v, t, lr=3e-3)
    return th.astype(np.float32)
