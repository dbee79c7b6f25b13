"""The C ABI library: it builds, loads, exports every declared entry point,
and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tfsph.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1908_01682_gb300 import build, binding
    build.build()
    return binding.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tfsph_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tfsph_init", "tfsph_step", "tfsph_fields", "tfsph_destroy", "tfsph_max_dt",
                     "tfsph_set_stream", "tfsph_debug", "tfsph_sync", "tfsph_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    from paper_1908_01682_gb300 import binding as b
    assert b.tfsph_version() >= 10000
    assert b.tfsph_status_string(b.TFSPH_E_INVALID_ARG) == "TFSPH_E_INVALID_ARG"


def test_params_struct_layout_matches_header():
    """Field offsets of the ctypes mirror follow the C declaration order."""
    from paper_1908_01682_gb300 import binding as b
    P = b.tfsph_params
    assert P.periodic.offset == 16 and P.lo.offset == 40 and P.hi.offset == 64
    assert P.h.offset == 88 and P.av_beta.offset == 88 + 7 * 8
    assert C.sizeof(P) == 88 + 8 * 8


def _init(params, n=4):
    from paper_1908_01682_gb300 import binding as b
    x = np.linspace(0.1, 0.9, n).astype(np.float32)
    arrs = [x, x.copy(), x.copy()]
    ptrs = [a.ctypes.data for a in arrs[:2]]
    dptrs = [a.ctypes.data for a in arrs]
    return b.tfsph_init(params, ptrs, n, dptrs, n, None, b.TFSPH_MEM_HOST)


@pytest.mark.parametrize("field,value,code", [
    ("dim", 4, 1), ("dim", 0, 1), ("h", -1.0, 1), ("cell_size", 0.0, 1), ("m_gas", 0.0, 1),
    ("precision", 7, 1), ("eos", 5, 1), ("h", float("nan"), 2), ("drag", 7, 1),
])
def test_init_rejects_bad_parameters_on_the_host(lib, field, value, code):
    from paper_1908_01682_gb300 import binding as b
    p = b.make_params(1, (0.0,), (1.0,), (1,), 0.05, 0.1, 1.0, 1.0)
    setattr(p, field, value)
    rc, ctx = _init(p)
    assert rc == code and not ctx.value
    assert b.tfsph_last_error(None)


def test_init_rejects_short_periodic_box(lib):
    from paper_1908_01682_gb300 import binding as b
    p = b.make_params(1, (0.0,), (1.0,), (1,), 0.3, 0.6, 1.0, 1.0)  # L < 4h
    rc, ctx = _init(p)
    assert rc == b.TFSPH_E_INVALID_ARG and "4h" in b.tfsph_last_error(None)


def test_null_context_is_an_error_not_a_crash(lib):
    from paper_1908_01682_gb300 import binding as b
    assert b.tfsph_step(None, 0.1, None, 0, (0, 0, 0)) == b.TFSPH_E_INVALID_ARG
    assert b.tfsph_sync(None) == b.TFSPH_E_INVALID_ARG
    b.tfsph_destroy(None)


def _batch_args(b, dims=(1, 1), precision=0, n=4):
    params = [b.make_params(d, (0.0,) * d, (1.0,) * d, (1,) * d, 0.05, 0.1, 0.1, 0.1, precision=precision)
              for d in dims]
    x = np.linspace(0.1, 0.9, n * len(dims)).astype(np.float32)
    arrs = [x, x.copy(), x.copy()]
    return params, [n] * len(dims), [n] * len(dims), [a.ctypes.data for a in arrs[:2]], \
        [a.ctypes.data for a in arrs], arrs


def test_batch_init_rejects_bad_arguments_on_the_host(lib):
    """Mixed dimensions, FP64 state, an empty list and negative counts are
    refused before any device work (this runs without a GPU)."""
    from paper_1908_01682_gb300 import binding as b
    params, ng, nd, gp, dp, keep = _batch_args(b, dims=(1, 2))
    rc, h = b.tfsph_batch_init(params, ng, nd, gp, dp, None, b.TFSPH_MEM_HOST)
    assert rc == b.TFSPH_E_INVALID_ARG and "same dim" in b.tfsph_batch_last_error(None)
    params, ng, nd, gp, dp, keep = _batch_args(b, precision=1)
    rc, h = b.tfsph_batch_init(params, ng, nd, gp, dp, None, b.TFSPH_MEM_HOST)
    assert rc == b.TFSPH_E_INVALID_ARG and "FP32" in b.tfsph_batch_last_error(None)
    rc, h = b.tfsph_batch_init([], [], [], gp, dp, None, b.TFSPH_MEM_HOST)
    assert rc == b.TFSPH_E_INVALID_ARG
    params, ng, nd, gp, dp, keep = _batch_args(b)
    rc, h = b.tfsph_batch_init(params, [4, -1], nd, gp, dp, None, b.TFSPH_MEM_HOST)
    assert rc == b.TFSPH_E_INVALID_ARG and "instance 1" in b.tfsph_batch_last_error(None)


def test_batch_info_struct_layout():
    from paper_1908_01682_gb300 import binding as b
    I = b.tfsph_batch_info_t
    assert I.n_gas.offset == 8 and I.n_cells.offset == 24 and I.mode.offset == 32
    assert I.steps.offset == 48 and I.device_bytes.offset == 64 and C.sizeof(I) == 72
