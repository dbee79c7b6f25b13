"""Thin ctypes binding of libtfsph (the C ABI declared in include/tfsph.h).

The module-level functions carry the C names and only marshal arguments:
every step of the method runs in the library's CUDA kernels. The ``Context``
class is a convenience wrapper over the same calls that accepts numpy arrays
(host memory) or torch CUDA tensors (device memory).

Loading fails loudly when libtfsph.so has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtfsph.so")

# constants mirrored from include/tfsph.h
TFSPH_OK, TFSPH_E_INVALID_ARG, TFSPH_E_NONFINITE, TFSPH_E_OUT_OF_DOMAIN = 0, 1, 2, 3
TFSPH_E_CUDA, TFSPH_E_OOM, TFSPH_E_INTERNAL, TFSPH_E_TIMEOUT = 4, 5, 6, 7
TFSPH_BATCH_KERNELS, TFSPH_BATCH_PERSISTENT, TFSPH_BATCH_TILED = 0, 1, 2
TFSPH_MEM_HOST, TFSPH_MEM_DEVICE = 0, 1
TFSPH_FP32, TFSPH_FP64 = 0, 1
TFSPH_EOS_ISOTHERMAL, TFSPH_EOS_ADIABATIC = 0, 1
TFSPH_KERNEL_CUBIC = 0
TFSPH_TSTAR_ARITHMETIC, TFSPH_TSTAR_HARMONIC = 0, 1
TFSPH_CELL_ACC_FP32, TFSPH_CELL_ACC_FP64 = 0, 1
TFSPH_DRAG_IDIC, TFSPH_DRAG_ISPH, TFSPH_DRAG_MK = 0, 1, 2
(TFSPH_FIELD_POS_G, TFSPH_FIELD_VEL_G, TFSPH_FIELD_ENERGY_G, TFSPH_FIELD_RHO_G, TFSPH_FIELD_POS_D,
 TFSPH_FIELD_VEL_D, TFSPH_FIELD_TSTOP_D, TFSPH_FIELD_RHO_D) = range(8)
TFSPH_ORDER_ORIGINAL, TFSPH_ORDER_CELL = 0, 1
PROF_PHASES = ("count", "scan", "scatter", "gather", "density", "force", "drag")
TFSPH_PROF_NPHASE = len(PROF_PHASES)
(TFSPH_DEBUG_KEYS_G, TFSPH_DEBUG_KEYS_D, TFSPH_DEBUG_PERM_G, TFSPH_DEBUG_PERM_D, TFSPH_DEBUG_CSTART_G,
 TFSPH_DEBUG_CSTART_D, TFSPH_DEBUG_NEIGH_COUNT, TFSPH_DEBUG_NEIGH_FPRINT, TFSPH_DEBUG_ACC_G) = range(9)


class tfsph_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("precision", C.c_int32), ("kernel", C.c_int32), ("eos", C.c_int32),
        ("periodic", C.c_int32 * 3), ("tstar_mode", C.c_int32), ("cell_acc", C.c_int32),
        ("drag", C.c_int32),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("h", C.c_double), ("cell_size", C.c_double), ("m_gas", C.c_double), ("m_dust", C.c_double),
        ("cs", C.c_double), ("gamma", C.c_double), ("av_alpha", C.c_double), ("av_beta", C.c_double),
    ]


class tfsph_info_t(C.Structure):
    _fields_ = [
        ("n_gas", C.c_int64), ("n_dust", C.c_int64), ("n_cells", C.c_int32 * 3), ("reach", C.c_int32 * 3),
        ("n_cells_total", C.c_int64), ("steps", C.c_int64), ("device_bytes", C.c_int64),
        ("launches", C.c_int64),
    ]


class tfsph_batch_info_t(C.Structure):
    _fields_ = [
        ("n_inst", C.c_int32), ("dim", C.c_int32), ("n_gas", C.c_int64), ("n_dust", C.c_int64),
        ("n_cells", C.c_int64), ("mode", C.c_int32), ("block", C.c_int32), ("grid", C.c_int32),
        ("graph", C.c_int32), ("steps", C.c_int64), ("launches", C.c_int64), ("device_bytes", C.c_int64),
    ]


class tfsph_grid_spec(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic", C.c_int32 * 3),
        ("nbins", C.c_int32 * 3), ("mass", C.c_double), ("precision", C.c_int32),
    ]


def grid_spec(dim, lo, hi, periodic, nbins, mass, precision) -> tfsph_grid_spec:
    g = tfsph_grid_spec()
    g.dim, g.mass, g.precision = int(dim), float(mass), int(precision)
    for k in range(3):
        g.lo[k] = float(lo[k]) if k < len(lo) else 0.0
        g.hi[k] = float(hi[k]) if k < len(hi) else 1.0
        g.periodic[k] = int(periodic[k]) if k < len(periodic) else 0
        g.nbins[k] = int(nbins[k]) if k < len(nbins) else 1
    return g


class TfsphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_status_name(code)}: {msg}")
        self.code = code


_lib = None


def _status_name(code: int) -> str:
    try:
        return load().tfsph_status_string(code).decode()
    except OSError:
        return f"status {code}"


def load() -> C.CDLL:
    """Load libtfsph.so (built by ``paper_1908_01682_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtfsph.so is not built ({LIB_PATH}); run paper_1908_01682_gb300.build.build() "
                          "- there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
    ctxp = C.c_void_p
    lib.tfsph_init.argtypes = [C.POINTER(ctxp), C.POINTER(tfsph_params), vp, i64, vp, i64, vp, i32]
    lib.tfsph_set_state.argtypes = [ctxp, vp, vp, vp, i32]
    lib.tfsph_set_stream.argtypes = [ctxp, vp]
    lib.tfsph_step.argtypes = [ctxp, d, vp, i32, C.POINTER(d)]
    lib.tfsph_max_dt.argtypes = [ctxp, d, C.POINTER(d)]
    lib.tfsph_step_adjoint.argtypes = [ctxp, d, C.POINTER(d), vp, vp, vp, vp, vp, i32]
    lib.tfsph_state_bytes.argtypes = [ctxp, C.POINTER(i64)]
    lib.tfsph_save_state.argtypes = [ctxp, vp, i32]
    lib.tfsph_load_state.argtypes = [ctxp, vp, i32]
    lib.tfsph_fields.argtypes = [ctxp, i32, vp, i32, i32]
    lib.tfsph_debug.argtypes = [ctxp, i32, vp, i32]
    lib.tfsph_info.argtypes = [ctxp, C.POINTER(tfsph_info_t)]
    lib.tfsph_sync.argtypes = [ctxp]
    lib.tfsph_profile.argtypes = [ctxp, i32]
    lib.tfsph_cell_ranges_noalloc.argtypes = [vp, i64, C.c_uint32, vp, vp]
    lib.tfsph_profile_read.argtypes = [ctxp, vp, vp, vp]
    lib.tfsph_dust_profile.argtypes = [C.POINTER(tfsph_grid_spec), vp, i64, vp, vp, vp, vp, vp]
    lib.tfsph_last_error.argtypes = [ctxp]
    lib.tfsph_last_error.restype = C.c_char_p
    lib.tfsph_status_string.argtypes = [i32]
    lib.tfsph_status_string.restype = C.c_char_p
    lib.tfsph_destroy.argtypes = [ctxp]
    lib.tfsph_destroy.restype = None
    lib.tfsph_version.argtypes = []
    bp = C.c_void_p
    lib.tfsph_batch_init.argtypes = [C.POINTER(bp), vp, vp, vp, C.c_int32, vp, vp, vp, i32]
    lib.tfsph_batch_set_stream.argtypes = [bp, vp]
    lib.tfsph_batch_step.argtypes = [bp, vp, vp, C.c_int32]
    lib.tfsph_batch_config.argtypes = [bp, C.c_int32, C.c_int32, C.c_int32, d]
    lib.tfsph_batch_autotune.argtypes = [bp, C.c_int32, vp, vp, vp, vp]
    lib.tfsph_batch_fields.argtypes = [bp, i32, vp, i32]
    lib.tfsph_batch_info.argtypes = [bp, C.POINTER(tfsph_batch_info_t)]
    lib.tfsph_batch_sync.argtypes = [bp]
    lib.tfsph_batch_last_error.argtypes = [bp]
    lib.tfsph_batch_last_error.restype = C.c_char_p
    lib.tfsph_batch_destroy.argtypes = [bp]
    lib.tfsph_batch_destroy.restype = None
    for name in ("tfsph_batch_init", "tfsph_batch_set_stream", "tfsph_batch_step", "tfsph_batch_config",
                 "tfsph_batch_autotune", "tfsph_batch_fields", "tfsph_batch_info", "tfsph_batch_sync"):
        getattr(lib, name).restype = C.c_int
    for name in ("tfsph_init", "tfsph_set_state", "tfsph_set_stream", "tfsph_step", "tfsph_step_adjoint", "tfsph_max_dt",
                 "tfsph_fields", "tfsph_debug", "tfsph_info", "tfsph_sync", "tfsph_version",
                 "tfsph_profile", "tfsph_profile_read", "tfsph_cell_ranges_noalloc", "tfsph_state_bytes",
                 "tfsph_save_state", "tfsph_load_state", "tfsph_dust_profile"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# C-named entry points (argument marshalling only)
# ---------------------------------------------------------------------------
def tfsph_init(params: tfsph_params, gas_ptrs, n_gas: int, dust_ptrs, n_dust: int, frozen_ptr, mem_kind: int):
    """Returns (status, ctx handle)."""
    lib = load()
    ctx = C.c_void_p()
    ga = (C.c_void_p * max(1, len(gas_ptrs)))(*gas_ptrs)
    da = (C.c_void_p * max(1, len(dust_ptrs)))(*dust_ptrs)
    rc = lib.tfsph_init(C.byref(ctx), C.byref(params), C.cast(ga, C.c_void_p), int(n_gas),
                        C.cast(da, C.c_void_p), int(n_dust), frozen_ptr, int(mem_kind))
    return rc, ctx


def tfsph_set_state(ctx, gas_ptrs, dust_ptrs, frozen_ptr, mem_kind: int) -> int:
    ga = (C.c_void_p * max(1, len(gas_ptrs)))(*gas_ptrs)
    da = (C.c_void_p * max(1, len(dust_ptrs)))(*dust_ptrs)
    return load().tfsph_set_state(ctx, C.cast(ga, C.c_void_p), C.cast(da, C.c_void_p), frozen_ptr, int(mem_kind))


def tfsph_set_stream(ctx, stream_ptr) -> int:
    return load().tfsph_set_stream(ctx, stream_ptr)


def tfsph_step(ctx, tau: float, tstop_ptr, mem_kind: int, g) -> int:
    g3 = (C.c_double * 3)(*[float(g[k]) if k < len(g) else 0.0 for k in range(3)])
    return load().tfsph_step(ctx, float(tau), tstop_ptr, int(mem_kind), g3)


def tfsph_step_adjoint(ctx, tau: float, g, lam_gx, lam_gv, lam_dx, lam_du, lam_ts, mem_kind: int) -> int:
    g3 = (C.c_double * 3)(*[float(g[k]) if k < len(g) else 0.0 for k in range(3)])
    return load().tfsph_step_adjoint(ctx, float(tau), g3, lam_gx, lam_gv, lam_dx, lam_du, lam_ts, int(mem_kind))


def tfsph_state_bytes(ctx):
    n = C.c_int64(0)
    rc = load().tfsph_state_bytes(ctx, C.byref(n))
    return rc, n.value


def tfsph_save_state(ctx, buf_ptr, mem_kind: int) -> int:
    return load().tfsph_save_state(ctx, buf_ptr, int(mem_kind))


def tfsph_load_state(ctx, buf_ptr, mem_kind: int) -> int:
    return load().tfsph_load_state(ctx, buf_ptr, int(mem_kind))


def tfsph_dust_profile(grid: tfsph_grid_spec, x_ptr, n: int, target_ptr, rho_ptr, loss_ptr, lam_x_ptr,
                       stream_ptr) -> int:
    return load().tfsph_dust_profile(C.byref(grid), x_ptr, int(n), target_ptr, rho_ptr, loss_ptr, lam_x_ptr,
                                     stream_ptr)


def tfsph_max_dt(ctx, cfl: float):
    out = C.c_double(0.0)
    rc = load().tfsph_max_dt(ctx, float(cfl), C.byref(out))
    return rc, out.value


def tfsph_fields(ctx, field: int, out_ptr, mem_kind: int, order: int) -> int:
    return load().tfsph_fields(ctx, int(field), out_ptr, int(mem_kind), int(order))


def tfsph_debug(ctx, what: int, out_ptr, mem_kind: int) -> int:
    return load().tfsph_debug(ctx, int(what), out_ptr, int(mem_kind))


def tfsph_info(ctx):
    info = tfsph_info_t()
    rc = load().tfsph_info(ctx, C.byref(info))
    return rc, info


def tfsph_sync(ctx) -> int:
    return load().tfsph_sync(ctx)


def tfsph_profile(ctx, enable: int) -> int:
    return load().tfsph_profile(ctx, int(enable))


def tfsph_profile_read(ctx):
    """Returns (status, per-phase ms array, timed steps, kernel launches)."""
    ms = (C.c_double * TFSPH_PROF_NPHASE)()
    steps = C.c_int64(0)
    launches = C.c_int64(0)
    rc = load().tfsph_profile_read(ctx, C.cast(ms, C.c_void_p), C.cast(C.pointer(steps), C.c_void_p),
                                   C.cast(C.pointer(launches), C.c_void_p))
    return rc, np.array(ms[:], dtype=np.float64), steps.value, launches.value


def tfsph_cell_ranges_noalloc(keys_ptr, n: int, n_cells: int, starts_ptr, stream_ptr=None) -> int:
    """Cell ranges of device keys into device starts, using only static scratch."""
    return load().tfsph_cell_ranges_noalloc(keys_ptr, int(n), int(n_cells), starts_ptr, stream_ptr)


def tfsph_last_error(ctx) -> str:
    s = load().tfsph_last_error(ctx)
    return s.decode() if s else ""


def tfsph_status_string(code: int) -> str:
    return load().tfsph_status_string(int(code)).decode()


def tfsph_destroy(ctx) -> None:
    load().tfsph_destroy(ctx)


def tfsph_version() -> int:
    return load().tfsph_version()


def tfsph_batch_init(params_list, n_gas, n_dust, gas_ptrs, dust_ptrs, frozen_ptr, mem_kind: int):
    """Returns (status, batch handle)."""
    lib = load()
    b = C.c_void_p()
    n = len(params_list)
    pa = (tfsph_params * n)(*params_list)
    ng = (C.c_int64 * n)(*[int(x) for x in n_gas])
    nd = (C.c_int64 * n)(*[int(x) for x in n_dust])
    ga = (C.c_void_p * max(1, len(gas_ptrs)))(*gas_ptrs)
    da = (C.c_void_p * max(1, len(dust_ptrs)))(*dust_ptrs)
    rc = lib.tfsph_batch_init(C.byref(b), C.cast(pa, C.c_void_p), C.cast(ng, C.c_void_p), C.cast(nd, C.c_void_p),
                              n, C.cast(ga, C.c_void_p), C.cast(da, C.c_void_p), frozen_ptr, int(mem_kind))
    return rc, b


def tfsph_batch_set_stream(b, stream_ptr) -> int:
    return load().tfsph_batch_set_stream(b, stream_ptr)


def tfsph_batch_step(b, tau, g, nsteps: int) -> int:
    ta = None if tau is None else (C.c_double * len(tau))(*[float(x) for x in tau])
    ga = None if g is None else (C.c_double * len(g))(*[float(x) for x in g])
    return load().tfsph_batch_step(b, None if ta is None else C.cast(ta, C.c_void_p),
                                   None if ga is None else C.cast(ga, C.c_void_p), int(nsteps))


def tfsph_batch_config(b, mode: int, block: int, blocks_per_sm: int, barrier_timeout_ms: float) -> int:
    return load().tfsph_batch_config(b, int(mode), int(block), int(blocks_per_sm), float(barrier_timeout_ms))


def tfsph_batch_autotune(b, steps: int):
    """Returns (status, mode, block, blocks_per_sm, ms per step)."""
    m, blk, bps, ms = C.c_int32(0), C.c_int32(0), C.c_int32(0), C.c_float(0)
    rc = load().tfsph_batch_autotune(b, int(steps), C.cast(C.pointer(m), C.c_void_p), C.cast(C.pointer(blk), C.c_void_p),
                                     C.cast(C.pointer(bps), C.c_void_p), C.cast(C.pointer(ms), C.c_void_p))
    return rc, m.value, blk.value, bps.value, ms.value


def tfsph_batch_fields(b, field: int, out_ptr, mem_kind: int) -> int:
    return load().tfsph_batch_fields(b, int(field), out_ptr, int(mem_kind))


def tfsph_batch_info(b):
    info = tfsph_batch_info_t()
    rc = load().tfsph_batch_info(b, C.byref(info))
    return rc, info


def tfsph_batch_sync(b) -> int:
    return load().tfsph_batch_sync(b)


def tfsph_batch_last_error(b) -> str:
    s = load().tfsph_batch_last_error(b)
    return s.decode() if s else ""


def tfsph_batch_destroy(b) -> None:
    load().tfsph_batch_destroy(b)


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
def make_params(dim, lo, hi, periodic, h, cell_size, m_gas, m_dust, precision=TFSPH_FP32,
                eos=TFSPH_EOS_ISOTHERMAL, cs=1.0, gamma=1.4, av_alpha=0.0, av_beta=0.0,
                tstar_mode=TFSPH_TSTAR_ARITHMETIC, cell_acc=TFSPH_CELL_ACC_FP64, drag=TFSPH_DRAG_IDIC) -> tfsph_params:
    p = tfsph_params()
    p.dim, p.precision, p.kernel, p.eos = int(dim), int(precision), TFSPH_KERNEL_CUBIC, int(eos)
    p.tstar_mode, p.cell_acc, p.drag = int(tstar_mode), int(cell_acc), int(drag)
    for k in range(3):
        p.periodic[k] = int(periodic[k]) if k < len(periodic) else 0
        p.lo[k] = float(lo[k]) if k < len(lo) else 0.0
        p.hi[k] = float(hi[k]) if k < len(hi) else 1.0
    p.h, p.cell_size, p.m_gas, p.m_dust = float(h), float(cell_size), float(m_gas), float(m_dust)
    p.cs, p.gamma, p.av_alpha, p.av_beta = float(cs), float(gamma), float(av_alpha), float(av_beta)
    return p


def params_from_dict(d: dict, **overrides) -> tfsph_params:
    q = dict(d)
    q.update(overrides)
    return make_params(q["dim"], q["lo"], q["hi"], q["periodic"], q["h"], q["cell_size"], q["m_gas"],
                       q["m_dust"], precision=q.get("precision", 0), eos=q.get("eos", 0), cs=q.get("cs", 1.0),
                       gamma=q.get("gamma", 1.4), av_alpha=q.get("av_alpha", 0.0), av_beta=q.get("av_beta", 0.0),
                       tstar_mode=q.get("tstar_mode", 0), cell_acc=q.get("cell_acc", TFSPH_CELL_ACC_FP64),
                       drag=q.get("drag", TFSPH_DRAG_IDIC))


def _check(rc: int, ctx=None):
    if rc != TFSPH_OK:
        raise TfsphError(rc, tfsph_last_error(ctx))


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


class Context:
    """Owns one tfsph context. Inputs are either all numpy arrays (host) or all
    torch CUDA tensors (device), in the context's precision, component-major."""

    def __init__(self, params: tfsph_params, gx, gv, dx, du, tstop, ge=None, frozen=None, stream=None):
        self.params = params
        self.dim = params.dim
        self.dtype = np.float64 if params.precision == TFSPH_FP64 else np.float32
        self._keep = []
        gas, dust, fz, mem = self._arrays(gx, gv, dx, du, tstop, ge, frozen)
        self.n_gas = int(gx.shape[-1])
        self.n_dust = int(dx.shape[-1])
        rc, self.ctx = tfsph_init(params, gas, self.n_gas, dust, self.n_dust, fz, mem)
        self._keep = []
        if rc != TFSPH_OK:
            raise TfsphError(rc, tfsph_last_error(None))
        if stream is not None:
            self.set_stream(stream)

    def _arrays(self, gx, gv, dx, du, tstop, ge, frozen):
        d = self.dim
        if _is_torch(gx):
            mem = TFSPH_MEM_DEVICE
            conv = lambda a: a.contiguous()
            ptr = lambda a: a.data_ptr()
        else:
            mem = TFSPH_MEM_HOST
            conv = lambda a: np.ascontiguousarray(a, dtype=self.dtype)
            ptr = lambda a: a.ctypes.data
        comps = [conv(gx[k]) for k in range(d)] + [conv(gv[k]) for k in range(d)]
        if self.params.eos == TFSPH_EOS_ADIABATIC:
            comps.append(conv(ge))
        dcomps = [conv(dx[k]) for k in range(d)] + [conv(du[k]) for k in range(d)] + [conv(tstop)]
        fz = None
        if frozen is not None:
            fz = frozen.contiguous() if mem == TFSPH_MEM_DEVICE else np.ascontiguousarray(frozen, dtype=np.uint8)
        self._keep = comps + dcomps + ([fz] if fz is not None else [])
        return ([ptr(a) for a in comps], [ptr(a) for a in dcomps], None if fz is None else ptr(fz), mem)

    def set_state(self, gx, gv, dx, du, tstop, ge=None, frozen=None):
        gas, dust, fz, mem = self._arrays(gx, gv, dx, du, tstop, ge, frozen)
        _check(tfsph_set_state(self.ctx, gas, dust, fz, mem), self.ctx)
        self._keep = []

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        _check(tfsph_set_stream(self.ctx, C.c_void_p(int(handle) if handle else 0)), self.ctx)

    def step(self, tau: float, g=(0.0, 0.0, 0.0), tstop=None):
        tp, mem = None, TFSPH_MEM_HOST
        if tstop is not None:
            if _is_torch(tstop):
                tstop = tstop.contiguous()
                tp, mem = tstop.data_ptr(), TFSPH_MEM_DEVICE
            else:
                tstop = np.ascontiguousarray(tstop, dtype=self.dtype)
                tp = tstop.ctypes.data
        _check(tfsph_step(self.ctx, tau, tp, mem, g), self.ctx)

    def step_adjoint(self, tau: float, g, lam_gx, lam_gv, lam_dx, lam_du, lam_ts):
        """Reverse-mode derivative of one step from the current state, in place
        on the lambda arrays (numpy host arrays or torch CUDA tensors)."""
        arrs = (lam_gx, lam_gv, lam_dx, lam_du, lam_ts)
        if _is_torch(lam_gx):
            ptrs = [a.data_ptr() for a in arrs]
            mem = TFSPH_MEM_DEVICE
        else:
            for a in arrs:
                assert a.dtype == self.dtype and a.flags.c_contiguous
            ptrs = [a.ctypes.data for a in arrs]
            mem = TFSPH_MEM_HOST
        _check(tfsph_step_adjoint(self.ctx, tau, g, *ptrs, mem), self.ctx)

    def state_bytes(self) -> int:
        rc, n = tfsph_state_bytes(self.ctx)
        _check(rc, self.ctx)
        return n

    def save_state(self, buf=None):
        """Snapshot into ``buf`` (torch CUDA uint8 tensor or numpy uint8 array;
        a new device tensor when None)."""
        if buf is None:
            import torch
            buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device="cuda")
        if _is_torch(buf):
            _check(tfsph_save_state(self.ctx, buf.data_ptr(), TFSPH_MEM_DEVICE), self.ctx)
        else:
            _check(tfsph_save_state(self.ctx, buf.ctypes.data, TFSPH_MEM_HOST), self.ctx)
        return buf

    def load_state(self, buf):
        if _is_torch(buf):
            _check(tfsph_load_state(self.ctx, buf.data_ptr(), TFSPH_MEM_DEVICE), self.ctx)
        else:
            _check(tfsph_load_state(self.ctx, np.ascontiguousarray(buf).ctypes.data, TFSPH_MEM_HOST), self.ctx)

    def max_dt(self, cfl: float) -> float:
        rc, tau = tfsph_max_dt(self.ctx, cfl)
        _check(rc, self.ctx)
        return tau

    def field(self, field: int, order: int = TFSPH_ORDER_ORIGINAL, out=None):
        vec = field in (TFSPH_FIELD_POS_G, TFSPH_FIELD_VEL_G, TFSPH_FIELD_POS_D, TFSPH_FIELD_VEL_D)
        gas = field in (TFSPH_FIELD_POS_G, TFSPH_FIELD_VEL_G, TFSPH_FIELD_ENERGY_G, TFSPH_FIELD_RHO_G)
        n = self.n_gas if gas else self.n_dust
        shape = (self.dim, n) if vec else (n,)
        if out is None:
            out = np.zeros(shape, dtype=self.dtype)
        if _is_torch(out):
            _check(tfsph_fields(self.ctx, field, out.data_ptr(), TFSPH_MEM_DEVICE, order), self.ctx)
        else:
            _check(tfsph_fields(self.ctx, field, out.ctypes.data, TFSPH_MEM_HOST, order), self.ctx)
        return out

    def debug(self, what: int):
        n_c = self.info().n_cells_total
        spec = {
            TFSPH_DEBUG_KEYS_G: (self.n_gas, np.uint32), TFSPH_DEBUG_KEYS_D: (self.n_dust, np.uint32),
            TFSPH_DEBUG_PERM_G: (self.n_gas, np.uint32), TFSPH_DEBUG_PERM_D: (self.n_dust, np.uint32),
            TFSPH_DEBUG_CSTART_G: (n_c + 1, np.uint32), TFSPH_DEBUG_CSTART_D: (n_c + 1, np.uint32),
            TFSPH_DEBUG_NEIGH_COUNT: (self.n_gas, np.int32), TFSPH_DEBUG_NEIGH_FPRINT: (self.n_gas, np.uint64),
            TFSPH_DEBUG_ACC_G: ((self.dim, self.n_gas), self.dtype),
        }[what]
        out = np.zeros(spec[0], dtype=spec[1])
        _check(tfsph_debug(self.ctx, what, out.ctypes.data, TFSPH_MEM_HOST), self.ctx)
        return out

    def info(self) -> tfsph_info_t:
        rc, info = tfsph_info(self.ctx)
        _check(rc, self.ctx)
        return info

    def sync(self):
        _check(tfsph_sync(self.ctx), self.ctx)

    def profile(self, enable: bool = True):
        _check(tfsph_profile(self.ctx, 1 if enable else 0), self.ctx)

    def profile_read(self):
        """(dict phase -> total ms, timed steps, kernel launches)."""
        rc, ms, steps, launches = tfsph_profile_read(self.ctx)
        _check(rc, self.ctx)
        return dict(zip(PROF_PHASES, ms.tolist())), steps, launches

    def close(self):
        if getattr(self, "ctx", None):
            tfsph_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(rc: int, b=None):
    if rc != TFSPH_OK:
        raise TfsphError(rc, tfsph_batch_last_error(b))


class Batch:
    """A batch of independent instances (FP32 state). ``instances`` is a list
    of (params, gx, gv, dx, du, tstop[, frozen]) with numpy arrays of shape
    (dim, n) (tstop, frozen: (n,)); they are concatenated in list order."""

    def __init__(self, instances, stream=None):
        import numpy as _np
        params = [it[0] for it in instances]
        self.dim = int(params[0].dim)
        d = self.dim
        self.n_gas = [int(it[1].shape[-1]) for it in instances]
        self.n_dust = [int(it[3].shape[-1]) for it in instances]
        cat = lambda idx, k: _np.ascontiguousarray(
            _np.concatenate([_np.asarray(it[idx], dtype=_np.float32)[k] for it in instances]))
        gas = [cat(1, k) for k in range(d)] + [cat(2, k) for k in range(d)]
        dust = [cat(3, k) for k in range(d)] + [cat(4, k) for k in range(d)]
        dust.append(_np.ascontiguousarray(_np.concatenate([_np.asarray(it[5], dtype=_np.float32)
                                                           for it in instances])))
        has_fz = any(len(it) > 6 and it[6] is not None for it in instances)
        fz = None
        if has_fz:
            fz = _np.ascontiguousarray(_np.concatenate([
                _np.asarray(it[6], dtype=_np.uint8) if len(it) > 6 and it[6] is not None
                else _np.zeros(int(it[1].shape[-1]), _np.uint8) for it in instances]))
        keep = gas + dust + ([fz] if fz is not None else [])
        rc, self.b = tfsph_batch_init(params, self.n_gas, self.n_dust, [a.ctypes.data for a in gas],
                                      [a.ctypes.data for a in dust], None if fz is None else fz.ctypes.data,
                                      TFSPH_MEM_HOST)
        del keep
        if rc != TFSPH_OK:
            self.b = None
            raise TfsphError(rc, tfsph_batch_last_error(None))
        self.n_inst = len(instances)
        self.goff = _np.concatenate([[0], _np.cumsum(self.n_gas)]).astype(_np.int64)
        self.doff = _np.concatenate([[0], _np.cumsum(self.n_dust)]).astype(_np.int64)
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        _bcheck(tfsph_batch_set_stream(self.b, C.c_void_p(int(handle) if handle else 0)), self.b)

    def step(self, tau=None, g=None, nsteps: int = 1):
        gflat = None
        if g is not None:
            gflat = np.zeros(3 * self.n_inst)
            ga = np.asarray(g, dtype=np.float64).reshape(self.n_inst, -1)
            gflat.reshape(self.n_inst, 3)[:, :ga.shape[1]] = ga
        _bcheck(tfsph_batch_step(self.b, None if tau is None else list(np.broadcast_to(
            np.asarray(tau, dtype=np.float64), (self.n_inst,))), gflat, nsteps), self.b)

    def config(self, mode: int, block: int = 256, blocks_per_sm: int = 1, barrier_timeout_ms: float = 2000.0):
        _bcheck(tfsph_batch_config(self.b, mode, block, blocks_per_sm, barrier_timeout_ms), self.b)

    def autotune(self, steps: int = 5):
        rc, mode, block, bps, ms = tfsph_batch_autotune(self.b, steps)
        _bcheck(rc, self.b)
        return {"mode": mode, "block": block, "blocks_per_sm": bps, "ms_per_step": ms}

    def field(self, field: int):
        vec = field in (TFSPH_FIELD_POS_G, TFSPH_FIELD_VEL_G, TFSPH_FIELD_POS_D, TFSPH_FIELD_VEL_D)
        gas = field in (TFSPH_FIELD_POS_G, TFSPH_FIELD_VEL_G, TFSPH_FIELD_ENERGY_G, TFSPH_FIELD_RHO_G)
        n = int(self.goff[-1] if gas else self.doff[-1])
        out = np.zeros((self.dim, n) if vec else (n,), dtype=np.float32)
        _bcheck(tfsph_batch_fields(self.b, field, out.ctypes.data, TFSPH_MEM_HOST), self.b)
        return out

    def instance_field(self, field: int, i: int):
        """The field of instance i (a view of one export)."""
        a = self.field(field)
        gas = field in (TFSPH_FIELD_POS_G, TFSPH_FIELD_VEL_G, TFSPH_FIELD_ENERGY_G, TFSPH_FIELD_RHO_G)
        off = self.goff if gas else self.doff
        return a[..., off[i]:off[i + 1]]

    def info(self) -> tfsph_batch_info_t:
        rc, info = tfsph_batch_info(self.b)
        _bcheck(rc, self.b)
        return info

    def sync(self):
        _bcheck(tfsph_batch_sync(self.b), self.b)

    def close(self):
        if getattr(self, "b", None):
            tfsph_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
