import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def oracle_system(w):
    """oracle.System from an ftlm_workloads dict."""
    import oracle
    return oracle.System(**{k: v for k, v in w.items() if k != "name"})


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)


def random_system(rng, two_s, dipolar=True, ion=True, field=True, scale=3.0):
    """A random anisotropic system with every term of Eq. (3) switched on."""
    n = len(two_s)
    w = {
        "name": "random",
        "two_s": np.asarray(two_s, dtype=np.int32),
        "J": rng.normal(size=(n, n)),
        "d_ion": rng.normal(size=n) * 2 if ion else None,
        "e_axes": rng.normal(size=(n, 3)) if ion else None,
        "g": 2.0 + 0.1 * rng.normal(),
        "B": rng.normal(size=3) if field else np.zeros(3),
        "pos": rng.normal(size=(n, 3)) * scale if dipolar else None,
    }
    return w
