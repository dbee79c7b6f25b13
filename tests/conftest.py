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
             tstar_mode=q["tstar_mode"], path_fp32=1 if int(q["precision"]) == 0 else 0)
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


# ---------------------------------------------------------------------------
# GPU-side helpers (only used by tests marked gpu)
# ---------------------------------------------------------------------------
def gpu_lib():
    from paper_1908_01682_gb300 import build
    build.build()
    from paper_1908_01682_gb300 import binding
    binding.load()
    return binding


def gpu_context(w, **overrides):
    """Context on the workload's inputs (host arrays of the path's dtype)."""
    b = gpu_lib()
    p = b.params_from_dict(w.params, **overrides)
    dt = np.float64 if p.precision == 1 else np.float32
    ge = None if w.ge is None else w.ge.astype(dt)
    return b.Context(p, w.gx.astype(dt), w.gv.astype(dt), w.dx.astype(dt), w.du.astype(dt),
                     w.tstop.astype(dt), ge=ge, frozen=w.frozen)


def gpu_one_step(w, tau=None, g=None, **overrides):
    """Bins the input on the GPU, exports the binning, takes one step and exports
    the new state. Arrays in id order unless stated."""
    b = gpu_lib()
    out = {}
    with gpu_context(w, **overrides) as c:
        out["keys_g"] = c.debug(b.TFSPH_DEBUG_KEYS_G)
        out["keys_d"] = c.debug(b.TFSPH_DEBUG_KEYS_D)
        out["perm_g"] = c.debug(b.TFSPH_DEBUG_PERM_G)
        out["perm_d"] = c.debug(b.TFSPH_DEBUG_PERM_D)
        out["cstart_g"] = c.debug(b.TFSPH_DEBUG_CSTART_G)
        out["cstart_d"] = c.debug(b.TFSPH_DEBUG_CSTART_D)
        out["nb_count"] = c.debug(b.TFSPH_DEBUG_NEIGH_COUNT)
        out["nb_fprint"] = c.debug(b.TFSPH_DEBUG_NEIGH_FPRINT)
        out["rho_g"] = c.field(b.TFSPH_FIELD_RHO_G).astype(np.float64)
        out["rho_d"] = c.field(b.TFSPH_FIELD_RHO_D).astype(np.float64)
        c.step(w.tau if tau is None else tau, w.g if g is None else g)
        c.sync()
        out["acc_g"] = c.debug(b.TFSPH_DEBUG_ACC_G).astype(np.float64)
        out["gx"] = c.field(b.TFSPH_FIELD_POS_G).astype(np.float64)
        out["gv"] = c.field(b.TFSPH_FIELD_VEL_G).astype(np.float64)
        out["dx"] = c.field(b.TFSPH_FIELD_POS_D).astype(np.float64)
        out["du"] = c.field(b.TFSPH_FIELD_VEL_D).astype(np.float64)
        if w.params["eos"] == 1:
            out["ge"] = c.field(b.TFSPH_FIELD_ENERGY_G).astype(np.float64)
        out["info"] = c.info()
    return out


def normwise(a, ref, floor=0.0):
    """||a - ref||_2 / max(||ref||_2, floor)."""
    a = np.asarray(a, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    den = max(float(np.linalg.norm(ref)), floor)
    if den == 0.0:
        return float(np.linalg.norm(a - ref))
    return float(np.linalg.norm(a - ref)) / den
