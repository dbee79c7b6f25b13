"""Seeded synthetic inputs shaped like the paper's test problems.

This module only builds inputs: particle lattices, seeded random fields and
parameter sets. It holds none of the method's arithmetic, imports neither the
oracle nor the GPU package, and serves both of them with identical bits.

Each generator returns a ``Workload``: a parameter dictionary (the fields of
``tfsph_params``), component-major particle arrays (float64 holding values
already rounded to the path's precision), the time step and gravity.

Workloads (sizes are the defaults; every generator can be scaled down):
- ``dustywave``: 1D periodic dusty sound wave (Sec. 3, Dustywave), 100 + 100
  particles on a lattice, cs = 1, rho_g = rho_d = 1, h = 1.2 dx, cell = 2h,
  amplitude 1e-4, t_stop = 1e-3, tau = CFL h / cs with CFL = 0.3, FP64.
- ``dustyshock``: 1D Sod-type dusty shock tube with walls (Sec. 3,
  Dustyshock), 2e5 gas + 2e5 dust, rho 1 / 0.125, p 1 / 0.1, gamma = 1.4,
  dust-to-gas ratio 1, per-particle t_stop log-uniform in [1e-5, 1],
  cell = 2h, frozen gas particles beyond both walls, FP32.
- ``box3d``: 3D periodic box, 128^3 gas + 128^3 dust on offset lattices,
  seeded Gaussian random velocity fields with a k^-2 power spectrum and rms
  0.1 cs, h = 1.2 dx (about 58 neighbours), 128^3 cells, t_stop = 1e-4, FP32.
- ``column2d``: 2D dust settling column, 512^2 gas in an exponential
  atmosphere + 512^2 dust, walls in y, g = (0, -1), per-particle t_stop
  log-uniform in [1e-3, 1e-1].
- ``ensemble1d``: many independent 1D dusty-wave instances of uneven sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    params: dict
    gx: np.ndarray          # (dim, n_gas)
    gv: np.ndarray          # (dim, n_gas)
    dx: np.ndarray          # (dim, n_dust)
    du: np.ndarray          # (dim, n_dust)
    tstop: np.ndarray       # (n_dust,)
    tau: float
    g: tuple = (0.0, 0.0, 0.0)
    ge: np.ndarray | None = None        # (n_gas,) specific internal energy
    frozen: np.ndarray | None = None    # (n_gas,) uint8, 1 = wall particle
    nsteps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return int(self.params["dim"])

    @property
    def n_gas(self) -> int:
        return int(self.gx.shape[1])

    @property
    def n_dust(self) -> int:
        return int(self.dx.shape[1])

    @property
    def fp32(self) -> bool:
        return int(self.params["precision"]) == 0


def _round(a, fp32: bool):
    a = np.asarray(a, dtype=np.float64)
    return a.astype(np.float32).astype(np.float64) if fp32 else a


def _finish(w: Workload) -> Workload:
    """Round every float input to the path's precision (both sides see these bits)."""
    f = w.fp32
    w.gx, w.gv, w.dx, w.du = (_round(a, f) for a in (w.gx, w.gv, w.dx, w.du))
    w.tstop = _round(w.tstop, f)
    if w.ge is not None:
        w.ge = _round(w.ge, f)
    w.gx = np.ascontiguousarray(w.gx)
    w.dx = np.ascontiguousarray(w.dx)
    return w


def base_params(dim: int, lo, hi, periodic, h: float, cell_size: float, m_gas: float,
                m_dust: float, precision: int, eos: int = 0, cs: float = 1.0,
                gamma: float = 1.4, av_alpha: float = 0.0, av_beta: float = 0.0,
                tstar_mode: int = 0) -> dict:
    pad = lambda t, v: tuple(float(t[k]) if k < len(t) else v for k in range(3))
    return dict(dim=dim, precision=precision, eos=eos, tstar_mode=tstar_mode,
                lo=pad(lo, 0.0), hi=pad(hi, 1.0),
                periodic=tuple(int(periodic[k]) if k < len(periodic) else 0 for k in range(3)),
                h=float(h), cell_size=float(cell_size), m_gas=float(m_gas), m_dust=float(m_dust),
                cs=float(cs), gamma=float(gamma), av_alpha=float(av_alpha), av_beta=float(av_beta))


# --------------------------------------------------------------------------
# 1D periodic dusty sound wave
# --------------------------------------------------------------------------
def dustywave(n: int = 100, amp: float = 1e-4, tstop: float = 1e-3, cfl: float = 0.3,
              h_factor: float = 1.2, cell_factor: float = 2.0, cs: float = 1.0,
              rho_g: float = 1.0, rho_d: float = 1.0, precision: int = 1, nsteps: int = 200,
              length: float = 1.0, dust_shift: float = 0.0, tau: float | None = None) -> Workload:
    """Lattice of n gas and n dust particles on [0, length) displaced so that
    rho/rho0 - 1 = amp sin(kx) and v = u = amp sin(kx), k = 2 pi / length."""
    dxl = length / n
    x0 = (np.arange(n) + 0.5) * dxl
    k = 2.0 * math.pi / length
    # displacement d(x0) with -d'(x0) = amp sin(k x0)
    xg = x0 + amp / k * np.cos(k * x0)
    xd = (x0 + dust_shift * dxl) + amp / k * np.cos(k * (x0 + dust_shift * dxl))
    xg = np.mod(xg, length)
    xd = np.mod(xd, length)
    vg = amp * np.sin(k * x0)
    ud = amp * np.sin(k * (x0 + dust_shift * dxl))
    h = h_factor * dxl
    p = base_params(1, (0.0,), (length,), (1,), h, cell_factor * h, rho_g * dxl, rho_d * dxl,
                    precision, cs=cs)
    t = tau if tau is not None else cfl * h / max(cs, float(np.max(np.abs(vg))))
    w = Workload("dustywave", p, xg[None, :], vg[None, :], xd[None, :], ud[None, :],
                 np.full(n, tstop), t, nsteps=nsteps,
                 meta=dict(k=k, amp=amp, rho_g=rho_g, rho_d=rho_d, cs=cs, tstop_scalar=tstop))
    return _finish(w)


# --------------------------------------------------------------------------
# 1D dusty shock tube with walls
# --------------------------------------------------------------------------
def dustyshock(n_left: int = 177778, n_right: int = 22222, rho_l: float = 1.0,
               rho_r: float = 0.125, p_l: float = 1.0, p_r: float = 0.1, gamma: float = 1.4,
               eps: float = 1.0, tstop=None, tstop_range=(1e-5, 1.0), seed: int = 2,
               h_factor: float = 1.2, cell_factor: float = 2.0, cfl: float = 0.3,
               precision: int = 0, eos: int = 1, cs: float = 1.0, av_alpha: float = 1.0,
               av_beta: float = 2.0, with_dust: bool = True, nsteps: int = 1) -> Workload:
    """Sod shock tube on [0, 1) split at 0.5, equal-mass gas particles on two
    lattices, dust on the same lattices with m_d = eps m_g, and frozen gas
    particles continuing each lattice beyond the walls at 0 and 1."""
    dxl = 0.5 / n_left
    dxr = 0.5 / n_right
    h = h_factor * max(dxl, dxr)
    xl = (np.arange(n_left) + 0.5) * dxl
    xr = 0.5 + (np.arange(n_right) + 0.5) * dxr
    m = rho_l * dxl  # equal particle mass on both sides (n_left/n_right = rho_l/rho_r)
    nwl = int(math.ceil(2.0 * h / dxl)) + 2
    nwr = int(math.ceil(2.0 * h / dxr)) + 2
    wl = -(np.arange(nwl) + 0.5) * dxl
    wr = 1.0 + (np.arange(nwr) + 0.5) * dxr
    gx = np.concatenate([xl, xr, wl[::-1], wr])
    nfl = n_left + n_right
    frozen = np.zeros(gx.size, np.uint8)
    frozen[nfl:] = 1
    rho0 = np.concatenate([np.full(n_left, rho_l), np.full(n_right, rho_r), np.full(nwl, rho_l),
                           np.full(nwr, rho_r)])
    pre0 = np.concatenate([np.full(n_left, p_l), np.full(n_right, p_r), np.full(nwl, p_l),
                           np.full(nwr, p_r)])
    ge = pre0 / ((gamma - 1.0) * rho0) if eos == 1 else None
    gv = np.zeros_like(gx)
    if with_dust:
        dxp = np.concatenate([xl, xr])
    else:
        dxp = np.zeros(0)
    du = np.zeros_like(dxp)
    nd = dxp.size
    rng = np.random.default_rng(seed)
    if tstop is None:
        lo, hi = math.log(tstop_range[0]), math.log(tstop_range[1])
        ts = np.exp(rng.uniform(lo, hi, size=nd))
    else:
        ts = np.full(nd, float(tstop))
    p = base_params(1, (0.0,), (1.0,), (0,), h, cell_factor * h, m, eps * m, precision, eos=eos,
                    cs=cs, gamma=gamma, av_alpha=av_alpha, av_beta=av_beta)
    cmax = math.sqrt(gamma * p_l / rho_l) if eos == 1 else cs
    w = Workload("dustyshock", p, gx[None, :], gv[None, :], dxp[None, :], du[None, :], ts,
                 cfl * h / cmax, ge=ge, frozen=frozen, nsteps=nsteps,
                 meta=dict(n_fluid=nfl, rho_l=rho_l, rho_r=rho_r, p_l=p_l, p_r=p_r, eps=eps))
    return _finish(w)


# --------------------------------------------------------------------------
# 3D periodic box with random velocity fields
# --------------------------------------------------------------------------
def random_velocity_field(nside: int, seed: int, rms: float, dim: int = 3) -> np.ndarray:
    """Gaussian random field on an nside^dim periodic grid, |v_k|^2 ~ k^-2 per
    component (no solenoidal projection), scaled to the given rms speed."""
    rng = np.random.default_rng(seed)
    freqs = np.fft.fftfreq(nside) * nside
    grids = np.meshgrid(*([freqs] * dim), indexing="ij")
    kk = np.sqrt(sum(g * g for g in grids))
    amp = np.zeros_like(kk)
    amp[kk > 0] = 1.0 / kk[kk > 0]  # amplitude ~ k^-1, power ~ k^-2
    comps = []
    for _ in range(dim):
        noise = rng.standard_normal((nside,) * dim)
        comps.append(np.real(np.fft.ifftn(np.fft.fftn(noise) * amp)))
    v = np.stack(comps)
    cur = math.sqrt(float(np.mean(np.sum(v * v, axis=0))))
    return v * (rms / cur)


def _trilinear(field: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """Periodic multilinear interpolation of a (dim, n^dim) grid field (nodes at i/n) at pos (dim, m)."""
    dim = pos.shape[0]
    n = field.shape[1]
    t = pos * n
    i0 = np.floor(t).astype(np.int64)
    f = t - i0
    out = np.zeros((field.shape[0], pos.shape[1]))
    for corner in range(1 << dim):
        wgt = np.ones(pos.shape[1])
        idx = []
        for d in range(dim):
            b = (corner >> d) & 1
            wgt = wgt * (f[d] if b else 1.0 - f[d])
            idx.append((i0[d] + b) % n)
        out += wgt * field[(slice(None),) + tuple(idx)]
    return out


def box3d(nside: int = 128, seed_gas: int = 3, seed_dust: int = 4, seed_jitter: int = 9,
          rms: float = 0.1, tstop: float = 1e-4, h_factor: float = 1.2, cell_factor: float = 1.0,
          jitter: float = 0.05, cfl: float = 0.3, precision: int = 0, cs: float = 1.0,
          nsteps: int = 100) -> Workload:
    """Gas at lattice points (i + 1/4) dx, dust at (i + 3/4) dx per axis, both
    jittered by a seeded uniform +-jitter dx; velocities from two independent
    random fields; unit densities."""
    n = nside
    dxl = 1.0 / n
    ax = np.arange(n, dtype=np.float64)
    gz, gy, gx_ = np.meshgrid(ax, ax, ax, indexing="ij")
    lat = np.stack([gx_.ravel(), gy.ravel(), gz.ravel()])
    rng = np.random.default_rng(seed_jitter)
    gpos = (lat + 0.25 + rng.uniform(-jitter, jitter, size=lat.shape)) * dxl
    dpos = (lat + 0.75 + rng.uniform(-jitter, jitter, size=lat.shape)) * dxl
    vg_field = random_velocity_field(n, seed_gas, rms * cs)
    vd_field = random_velocity_field(n, seed_dust, rms * cs)
    # field index order is (x, y, z) on axes (0, 1, 2)
    gv = _trilinear(vg_field, gpos)
    dv = _trilinear(vd_field, dpos)
    h = h_factor * dxl
    m = 1.0 / (n ** 3)
    p = base_params(3, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (1, 1, 1), h, cell_factor * dxl, m, m,
                    precision, cs=cs)
    vmax = float(np.max(np.sqrt(np.sum(gv * gv, axis=0))))
    tau = cfl * h / (cs + vmax)
    w = Workload("box3d", p, gpos, gv, dpos, dv, np.full(n ** 3, tstop), tau, nsteps=nsteps,
                 meta=dict(nside=n, rms=rms))
    return _finish(w)


# --------------------------------------------------------------------------
# 2D dust settling column
# --------------------------------------------------------------------------
def column2d(nside: int = 512, eps: float = 0.01, tstop_range=(1e-3, 1e-1), seed_tstop: int = 6,
             seed_noise: int = 7, noise: float = 1e-6, h_factor: float = 1.2,
             cell_factor: float = 2.0, cfl: float = 0.3, precision: int = 0, cs: float = 1.0,
             nsteps: int = 500) -> Workload:
    """Isothermal gas with rho ~ exp(-y) (scale height cs^2/g = 1) placed by
    the inverse CDF on nside columns, uniform dust, walls at y = 0 and 1 with
    frozen gas rows continuing the lattice, periodic in x, g = (0, -1)."""
    n = nside
    dxl = 1.0 / n
    xs = (np.arange(n) + 0.5) * dxl
    z = 1.0 - math.exp(-1.0)
    ys = -np.log(1.0 - (np.arange(n) + 0.5) / n * z)
    h = h_factor * dxl
    # frozen rows continuing the first and last row spacing
    dy0 = ys[1] - ys[0]
    dy1 = ys[-1] - ys[-2]
    nw0 = int(math.ceil(2.0 * h / dy0)) + 2
    nw1 = int(math.ceil(2.0 * h / dy1)) + 2
    y_below = ys[0] - (np.arange(nw0) + 1) * dy0
    y_above = ys[-1] + (np.arange(nw1) + 1) * dy1
    yall = np.concatenate([ys, y_below[::-1], y_above])
    X, Y = np.meshgrid(xs, yall, indexing="xy")
    gx = np.stack([X.ravel(), Y.ravel()])
    frozen = ((Y.ravel() < 0.0) | (Y.ravel() >= 1.0)).astype(np.uint8)
    m_gas = z / (n * n)  # total gas mass = integral of exp(-y) over [0,1]
    dX, dY = np.meshgrid(xs, (np.arange(n) + 0.5) * dxl, indexing="xy")
    dpos = np.stack([dX.ravel(), dY.ravel()])
    m_dust = eps * z / (n * n)
    rng = np.random.default_rng(seed_tstop)
    ts = np.exp(rng.uniform(math.log(tstop_range[0]), math.log(tstop_range[1]), size=n * n))
    rng2 = np.random.default_rng(seed_noise)
    gv = noise * rng2.standard_normal(gx.shape)
    gv[:, frozen == 1] = 0.0
    du = noise * rng2.standard_normal(dpos.shape)
    p = base_params(2, (0.0, 0.0), (1.0, 1.0), (1, 0), h, cell_factor * h, m_gas, m_dust,
                    precision, cs=cs)
    w = Workload("column2d", p, gx, gv, dpos, du, ts, cfl * h / cs, g=(0.0, -1.0, 0.0),
                 frozen=frozen, nsteps=nsteps, meta=dict(nside=n, eps=eps))
    return _finish(w)


# --------------------------------------------------------------------------
# Ensemble of independent 1D dusty waves (batched form)
# --------------------------------------------------------------------------
def ensemble1d(n_inst: int = 256, nmin: int = 1024, nmax: int = 65536, seed: int = 5,
               tstop_range=(1e-5, 1.0), amp_range=(1e-5, 1e-3), precision: int = 0):
    """List of ``dustywave`` workloads with log-uniform total particle counts
    (half gas, half dust), t_stop and amplitudes."""
    rng = np.random.default_rng(seed)
    ntot = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n_inst)).astype(np.int64)
    ts = np.exp(rng.uniform(math.log(tstop_range[0]), math.log(tstop_range[1]), size=n_inst))
    amps = np.exp(rng.uniform(math.log(amp_range[0]), math.log(amp_range[1]), size=n_inst))
    out = []
    for i in range(n_inst):
        nph = max(8, int(ntot[i]) // 2)
        out.append(dustywave(n=nph, amp=float(amps[i]), tstop=float(ts[i]), precision=precision,
                             nsteps=1))
    return out
