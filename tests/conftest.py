import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical or trajectory check")


@pytest.fixture(scope="session")
def params():
    from paper_2606_14073_gb300 import nep_params
    return nep_params.load()


@pytest.fixture(scope="session")
def model(params):
    from oracle import oracle as O
    return O.Model(params)


def variant(params, **scale):
    """Copy of the parameter dict with coefficient groups scaled: scale keys are
    group names R, A, EX, DMI, ANI, SIA; 'net' scales w1."""
    groups = dict(R=0, A=1, EX=2, DMI=3, ANI=4, SIA=5)
    p = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in params.items()}
    for g, s in scale.items():
        if g == "net":
            p["w1"] = p["w1"] * s
        else:
            p["coeffs"][:, :, groups[g]] *= s
    return p
