"""Shared test setup: the ``gpu`` marker and oracle/workload helpers."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def oracle_params(w, **overrides):
    """oracle.Params for a workload; integer decisions in the workload's precision."""
    import oracle
    q = w.params
    d = dict(dim=q["dim"], lo=q["lo"], hi=q["hi"], periodic=q["periodic"], h=q["h"],
             cell_size=q["cell_size"], m_gas=q["m_gas"], m_dust=q["m_dust"], eos=q["eos"],
             cs=q["cs"], gamma=q["gamma"], av_alpha=q["av_alpha"], av_beta=q["av_beta"],
             tstar_mode=q["tstar_mode"], decide_fp32=1 if int(q["precision"]) == 0 else 0)
    d.update(overrides)
    return oracle.Params(**d)


def oracle_state(w):
    import oracle
    p = oracle_params(w)
    return oracle.make_state(p, w.gx, w.gv, w.dx, w.du, w.tstop, ge=w.ge, frozen=w.frozen)


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
