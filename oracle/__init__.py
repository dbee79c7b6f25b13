"""FP64 CPU oracle of the SPH-IDIC two-fluid step (arXiv:1908.01682, Sec. 2.3).

TEST INFRASTRUCTURE ONLY. The oracle is the independent checker of the GPU
library: only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it. It shares no code with the CUDA path.

The arithmetic lives in ``tfsph_oracle.c`` (plain double-precision loops);
this module compiles it with gcc and marshals numpy arrays through ctypes.
Arrays are component-major: a position array of n particles in d dimensions
has shape (d, n). The closed forms that pin the oracle live in
``oracle.analytic``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfsph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("path_fp32", C.c_int32), ("eos", C.c_int32),
        ("tstar_mode", C.c_int32), ("periodic", C.c_int32 * 3), ("brute", C.c_int32),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("h", C.c_double), ("cell_size", C.c_double),
        ("m_gas", C.c_double), ("m_dust", C.c_double),
        ("cs", C.c_double), ("gamma", C.c_double),
        ("av_alpha", C.c_double), ("av_beta", C.c_double),
    ]


class _StepOut(C.Structure):
    _fields_ = [
        ("rho_g", C.c_void_p), ("acc_g", C.c_void_p), ("dedt_g", C.c_void_p), ("acc_scale_g", C.c_void_p),
        ("nb_count", C.c_void_p), ("nb_fprint", C.c_void_p), ("nb_band", C.c_void_p), ("nb_band_ids", C.c_void_p),
        ("keys_g", C.c_void_p), ("keys_d", C.c_void_p),
        ("perm_g", C.c_void_p), ("perm_d", C.c_void_p),
        ("cstart_g", C.c_void_p), ("cstart_d", C.c_void_p),
        ("n_drag_cells", C.c_int64),
    ]


class _XStepOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "rho_g", "rho_d", "acc_g", "acc_scale_g", "drag_g", "drag_d", "scale_g", "scale_d",
        "isph_acc_d", "isph_acc_scale_d", "isph_rho_dg", "isph_K_g", "isph_rho_gd")]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        vp, i64, d = C.c_void_p, C.c_int64, C.c_double
        _lib.orc_W.restype = d
        _lib.orc_W.argtypes = [C.c_int, d, d]
        _lib.orc_dWdr.restype = d
        _lib.orc_dWdr.argtypes = [C.c_int, d, d]
        _lib.orc_ncell.argtypes = [vp, vp]
        _lib.orc_bin.argtypes = [vp, i64, vp, vp, vp, vp]
        _lib.orc_density.argtypes = [vp, i64, vp, d, vp, vp, vp, vp, vp]
        _lib.orc_accel.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
        _lib.orc_neighbour.restype = C.c_int
        _lib.orc_neighbour.argtypes = [vp, vp, vp, vp]
        _lib.orc_cell_index.restype = i64
        _lib.orc_cell_index.argtypes = [vp, C.c_int, d]
        _lib.orc_dust_profile.argtypes = [vp, vp, i64, vp, d, vp]
        _lib.orc_set_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_max_dt.restype = d
        _lib.orc_max_dt.argtypes = [vp, i64, vp, vp, vp, d]
        _lib.orc_step.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, d, vp, vp, vp]
        _lib.orc_step_x.argtypes = [vp, C.c_int, i64, i64, vp, vp, vp, vp, vp, vp, vp, d, vp, vp]
    return _lib


@dataclass
class Params:
    """Problem parameters (mirrors the ``tfsph_params`` fields the oracle needs)."""
    dim: int
    lo: tuple
    hi: tuple
    periodic: tuple
    h: float
    cell_size: float
    m_gas: float
    m_dust: float
    eos: int = 0            # 0 isothermal, 1 adiabatic
    cs: float = 1.0
    gamma: float = 1.4
    av_alpha: float = 0.0
    av_beta: float = 0.0
    tstar_mode: int = 0     # 0 arithmetic mean, 1 harmonic mean
    path_fp32: int = 0      # the path under test computes in binary32: width of the reported pair band
    brute: int = 0          # all-pairs neighbour search

    def c(self) -> _Params:
        p = _Params()
        p.dim, p.path_fp32, p.eos, p.tstar_mode = self.dim, self.path_fp32, self.eos, self.tstar_mode
        p.brute = self.brute
        for k in range(3):
            p.periodic[k] = int(self.periodic[k]) if k < len(self.periodic) else 0
            p.lo[k] = float(self.lo[k]) if k < len(self.lo) else 0.0
            p.hi[k] = float(self.hi[k]) if k < len(self.hi) else 1.0
        p.h, p.cell_size, p.m_gas, p.m_dust = self.h, self.cell_size, self.m_gas, self.m_dust
        p.cs, p.gamma, p.av_alpha, p.av_beta = self.cs, self.gamma, self.av_alpha, self.av_beta
        return p


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def W(dim: int, h: float, r: float) -> float:
    return _load().orc_W(dim, h, r)


def dWdr(dim: int, h: float, r: float) -> float:
    return _load().orc_dWdr(dim, h, r)


def ncell(p: Params):
    out = (C.c_int32 * 3)()
    _load().orc_ncell(C.byref(p.c()), out)
    return tuple(out)


def bin_particles(p: Params, x):
    """Cell keys (per particle), sorted order (ids) and cell starts."""
    x = _f64(x, (p.dim, -1))
    n = x.shape[1]
    nc = ncell(p)
    keys = np.zeros(n, np.int64)
    perm = np.zeros(n, np.int64)
    cstart = np.zeros(int(np.prod(nc)) + 1, np.int64)
    pc = p.c()
    _load().orc_bin(C.byref(pc), n, _ptr(x), _ptr(keys), _ptr(perm), _ptr(cstart))
    return keys, perm, cstart


def neighbour(p: Params, xa, xb):
    """(inside, band) for one pair: inside = r^2 < 4h^2 over the reals; band =
    the pair lies within 8 ulp of 4h^2 in the path's precision (or its
    decision could not be certified)."""
    a = _f64(list(xa) + [0.0] * (3 - len(xa)))
    b = _f64(list(xb) + [0.0] * (3 - len(xb)))
    band = C.c_int32(0)
    pc = p.c()
    inside = _load().orc_neighbour(C.byref(pc), _ptr(a), _ptr(b), C.byref(band))
    return bool(inside), bool(band.value)


def cell_index(p: Params, axis: int, x: float) -> int:
    """floor((x - lo) n / L) along one axis, exact, clamped to [0, n-1]."""
    pc = p.c()
    return int(_load().orc_cell_index(C.byref(pc), int(axis), float(x)))


NBAND = 4  # band partner ids reported per particle (ORC_NBAND)


def density(p: Params, x, m: float, with_band: bool = False):
    """Summation density, neighbour counts and neighbour-set fingerprints.

    Membership is exact (r^2 < 4h^2 over the reals). Counts and fingerprints
    cover the neighbours outside the reported band (pairs within 8 ulp of 4h^2
    in the path's precision); with_band also returns the number of band pairs
    per particle and the ids of the first NBAND of them (-1 beyond)."""
    x = _f64(x, (p.dim, -1))
    n = x.shape[1]
    rho = np.zeros(n)
    cnt = np.zeros(n, np.int64)
    fp = np.zeros(n, np.uint64)
    nb = np.zeros(n, np.int64)
    ids = np.full((n, NBAND), -1, np.int64)
    pc = p.c()
    _load().orc_density(C.byref(pc), n, _ptr(x), m, _ptr(rho), _ptr(cnt), _ptr(fp), _ptr(nb), _ptr(ids))
    return (rho, cnt, fp, nb, ids) if with_band else (rho, cnt, fp)


def accel(p: Params, x, v, e, rho, with_scale: bool = False):
    """Pressure (+ viscous) acceleration and energy rate; with_scale also
    returns the per-particle magnitude sum of the pair terms."""
    x = _f64(x, (p.dim, -1))
    n = x.shape[1]
    v = _f64(v, (p.dim, n))
    e = None if e is None else _f64(e, (n,))
    rho = _f64(rho, (n,))
    acc = np.zeros((p.dim, n))
    dedt = np.zeros(n)
    scale = np.zeros(n)
    pc = p.c()
    _load().orc_accel(C.byref(pc), n, _ptr(x), _ptr(v), _ptr(e), _ptr(rho), _ptr(acc), _ptr(dedt),
                      _ptr(scale))
    return (acc, dedt, scale) if with_scale else (acc, dedt)


def max_dt(p: Params, v, e=None, frozen=None, cfl: float = 0.3) -> float:
    v = _f64(v, (p.dim, -1))
    n = v.shape[1]
    e = None if e is None else _f64(e, (n,))
    fr = None if frozen is None else np.ascontiguousarray(np.asarray(frozen, np.uint8))
    pc = p.c()
    return _load().orc_max_dt(C.byref(pc), n, _ptr(v), _ptr(e), _ptr(fr), cfl)


@dataclass
class State:
    """Particle state in user (id) order; arrays are float64, component-major."""
    gx: np.ndarray
    gv: np.ndarray
    dx: np.ndarray
    du: np.ndarray
    tstop: np.ndarray
    ge: np.ndarray | None = None
    frozen: np.ndarray | None = None

    def copy(self) -> "State":
        cp = lambda a: None if a is None else np.array(a, copy=True)
        return State(cp(self.gx), cp(self.gv), cp(self.dx), cp(self.du), cp(self.tstop),
                     cp(self.ge), cp(self.frozen))


@dataclass
class StepResult:
    rho_g: np.ndarray
    acc_g: np.ndarray
    dedt_g: np.ndarray
    acc_scale_g: np.ndarray
    nb_count: np.ndarray
    nb_fprint: np.ndarray
    nb_band: np.ndarray
    nb_band_ids: np.ndarray
    keys_g: np.ndarray
    keys_d: np.ndarray
    perm_g: np.ndarray
    perm_d: np.ndarray
    cstart_g: np.ndarray
    cstart_d: np.ndarray
    n_drag_cells: int


def make_state(p: Params, gx, gv, dx, du, tstop, ge=None, frozen=None) -> State:
    ng = np.asarray(gx).reshape(p.dim, -1).shape[1]
    nd = np.asarray(dx).reshape(p.dim, -1).shape[1]
    ts = np.asarray(tstop, dtype=np.float64)
    if ts.ndim == 0:
        ts = np.full(nd, float(ts))
    return State(_f64(gx, (p.dim, ng)).copy(), _f64(gv, (p.dim, ng)).copy(),
                 _f64(dx, (p.dim, nd)).copy(), _f64(du, (p.dim, nd)).copy(),
                 _f64(ts, (nd,)).copy(),
                 None if ge is None else _f64(ge, (ng,)).copy(),
                 None if frozen is None else np.ascontiguousarray(np.asarray(frozen, np.uint8)).copy())


def step(p: Params, s: State, tau: float, g=(0.0, 0.0, 0.0), acc_override=None) -> StepResult:
    """One SPH-IDIC step in place on ``s``; returns the step's diagnostics."""
    ng = s.gx.shape[1]
    nd = s.dx.shape[1]
    nc = ncell(p)
    ncells = int(np.prod(nc))
    r = StepResult(np.zeros(ng), np.zeros((p.dim, ng)), np.zeros(ng), np.zeros(ng), np.zeros(ng, np.int64),
                   np.zeros(ng, np.uint64), np.zeros(ng, np.int64), np.full((ng, NBAND), -1, np.int64),
                   np.zeros(ng, np.int64), np.zeros(nd, np.int64),
                   np.zeros(ng, np.int64), np.zeros(nd, np.int64),
                   np.zeros(ncells + 1, np.int64), np.zeros(ncells + 1, np.int64), 0)
    out = _StepOut(_ptr(r.rho_g), _ptr(r.acc_g), _ptr(r.dedt_g), _ptr(r.acc_scale_g), _ptr(r.nb_count),
                   _ptr(r.nb_fprint), _ptr(r.nb_band), _ptr(r.nb_band_ids),
                   _ptr(r.keys_g), _ptr(r.keys_d), _ptr(r.perm_g), _ptr(r.perm_d),
                   _ptr(r.cstart_g), _ptr(r.cstart_d), 0)
    g3 = (C.c_double * 3)(*[float(g[k]) if k < len(g) else 0.0 for k in range(3)])
    ao = None if acc_override is None else _f64(acc_override, (p.dim, ng))
    pc = p.c()
    rc = _load().orc_step(C.byref(pc), ng, nd, _ptr(s.gx), _ptr(s.gv), _ptr(s.ge), _ptr(s.frozen),
                          _ptr(s.dx), _ptr(s.du), _ptr(s.tstop), float(tau), g3, _ptr(ao),
                          C.byref(out))
    if rc != 0:
        raise RuntimeError(f"orc_step failed with code {rc}")
    r.n_drag_cells = int(out.n_drag_cells)
    return r


ISPH, MK = 1, 2


@dataclass
class XStepResult:
    """Diagnostics of one ISPH or MK step (id order). drag_g / drag_d: MK
    drag accelerations D_a, D_j (Eqs. 8-9); ISPH interpolated velocities u_a
    (dust at gas particles) and v_j (gas at dust particles) (Eq. 11)."""
    rho_g: np.ndarray
    rho_d: np.ndarray
    acc_g: np.ndarray
    acc_scale_g: np.ndarray
    drag_g: np.ndarray
    drag_d: np.ndarray
    scale_g: np.ndarray
    scale_d: np.ndarray
    isph_acc_d: np.ndarray
    isph_acc_scale_d: np.ndarray
    isph_rho_dg: np.ndarray
    isph_K_g: np.ndarray
    isph_rho_gd: np.ndarray


def step_x(p: Params, s: State, tau: float, g=(0.0, 0.0, 0.0), scheme: int = ISPH) -> XStepResult:
    """One step with the ISPH (Eqs. 11-16) or MK (Eqs. 8-10) drag, in place on ``s``."""
    ng = s.gx.shape[1]
    nd = s.dx.shape[1]
    dim = p.dim
    r = XStepResult(np.zeros(ng), np.zeros(nd), np.zeros((dim, ng)), np.zeros(ng), np.zeros((dim, ng)),
                    np.zeros((dim, nd)), np.zeros(ng), np.zeros(nd), np.zeros((dim, nd)), np.zeros(nd),
                    np.zeros(ng), np.zeros(ng), np.zeros(nd))
    out = _XStepOut(*[_ptr(getattr(r, f[0])) for f in _XStepOut._fields_])
    g3 = (C.c_double * 3)(*[float(g[k]) if k < len(g) else 0.0 for k in range(3)])
    pc = p.c()
    rc = _load().orc_step_x(C.byref(pc), int(scheme), ng, nd, _ptr(s.gx), _ptr(s.gv), _ptr(s.ge),
                            _ptr(s.frozen), _ptr(s.dx), _ptr(s.du), _ptr(s.tstop), float(tau), g3,
                            C.byref(out))
    if rc != 0:
        raise RuntimeError(f"orc_step_x failed with code {rc}")
    return r


def run(p: Params, s: State, tau: float, nsteps: int, g=(0.0, 0.0, 0.0), scheme: int = 0) -> State:
    """nsteps steps; scheme 0 = IDIC, ISPH or MK."""
    for _ in range(nsteps):
        if scheme == 0:
            step(p, s, tau, g)
        else:
            step_x(p, s, tau, g, scheme)
    return s


def dust_profile(p: Params, x, m: float, nbins):
    """Cloud-in-cell binned density of particles of mass m at x (dim, n) on
    nbins bins per axis over the box; array of shape nbins[::-1] flattened
    with axis 0 fastest (bin b = i0 + nb0 (i1 + nb1 i2))."""
    x = _f64(x, (p.dim, -1))
    n = x.shape[1]
    nb = (C.c_int32 * 3)(*[int(nbins[k]) if k < p.dim else 1 for k in range(3)])
    total = int(np.prod([nb[k] for k in range(p.dim)]))
    rho = np.zeros(total)
    pc = p.c()
    rc = _load().orc_dust_profile(C.byref(pc), nb, n, _ptr(x), float(m), _ptr(rho))
    if rc != 0:
        raise ValueError("orc_dust_profile: bad bin counts")
    return rho


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops from now on; returns the count in use."""
    return int(_load().orc_set_threads(int(n)))


def omp_threads() -> int:
    """Threads the oracle's OpenMP loops use (OMP_NUM_THREADS, else all cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    if v:
        try:
            return max(1, int(v))
        except ValueError:
            pass
    return os.cpu_count() or 1
