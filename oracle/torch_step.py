"""Differentiable FP64 re-expression of the oracle step (test infrastructure only).

The same SPH-IDIC step as ``tfsph_oracle.c`` (Sec. 2.3, Eqs. 17-21, isothermal
gas without artificial viscosity), written with plain PyTorch CPU tensor
operations in float64 so that autograd gives the exact derivative of the
discrete step: the oracle's own adjoint, against which the GPU's hand-written
adjoint is checked. All pairs are formed by brute force (small inputs only);
cell membership comes from the C oracle's binning and is held fixed, as
piecewise-constant cell membership has no derivative.

Pinned in ``tests/test_oracle_adjoint.py``: its forward equals the C oracle's
step, and its gradients equal central finite differences of the C oracle.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle


def _sigma(dim: int) -> float:
    return {1: 2.0 / 3.0, 2: 10.0 / (7.0 * math.pi), 3: 1.0 / math.pi}[dim]


def _W(q, dim, h):
    """M4 cubic spline W(r, h) as a function of q = r/h."""
    inner = 1.0 - 1.5 * q ** 2 + 0.75 * q ** 3
    outer = 0.25 * torch.clamp(2.0 - q, min=0.0) ** 3
    return _sigma(dim) / h ** dim * torch.where(q < 1.0, inner, outer)


def _dWdr(q, dim, h):
    inner = -3.0 * q + 2.25 * q ** 2
    outer = -0.75 * torch.clamp(2.0 - q, min=0.0) ** 2
    return _sigma(dim) / h ** (dim + 1) * torch.where(q < 1.0, inner, outer)


def _min_image(d, p: oracle.Params):
    out = []
    for k in range(p.dim):
        dk = d[..., k]
        if p.periodic[k]:
            L = p.hi[k] - p.lo[k]
            dk = dk - L * torch.round(dk / L).detach()
        out.append(dk)
    return torch.stack(out, dim=-1)


def step(p: oracle.Params, gx, gv, dx, du, tstop, tau: float, g=(0.0, 0.0, 0.0), frozen=None):
    """One step. Tensors are float64, shape (dim, n); returns (gx', gv', dx', du')."""
    assert p.eos == 0 and p.av_alpha == 0 and p.av_beta == 0
    dim = p.dim
    ng, nd = gx.shape[1], dx.shape[1]
    keys_g, _, _ = oracle.bin_particles(p, gx.detach().numpy())
    keys_d, _, _ = oracle.bin_particles(p, dx.detach().numpy())
    nc = int(np.prod(oracle.ncell(p)))
    kg = torch.as_tensor(keys_g)
    kd = torch.as_tensor(keys_d)
    moving = torch.ones(ng, dtype=torch.bool) if frozen is None else torch.as_tensor(np.asarray(frozen) == 0)

    # pair geometry (all pairs), membership r^2 < 4 h^2 held fixed
    xg = gx.T
    d = _min_image(xg[:, None, :] - xg[None, :, :], p)           # d_ab = x_a - x_b
    r2 = (d * d).sum(-1)
    member = (r2 < 4.0 * p.h * p.h).detach()
    nonself = member & (r2.detach() > 0.0)
    r = torch.sqrt(torch.where(nonself, r2, torch.ones_like(r2)))
    q = r / p.h
    # summation density (self term W(0))
    W = torch.where(nonself, _W(q, dim, p.h), torch.zeros_like(r2))
    rho = p.m_gas * (W.sum(1) + _sigma(dim) / p.h ** dim)
    pr = p.cs ** 2 / rho                                          # p / rho^2, isothermal
    # pressure acceleration (first term of Eq. 19)
    Fr = torch.where(nonself, _dWdr(q, dim, p.h) / r, torch.zeros_like(r2))
    coef = (pr[:, None] + pr[None, :]) * Fr
    A = -p.m_gas * (coef[:, :, None] * d).sum(1)                  # (ng, dim)

    gvec = torch.tensor([float(g[k]) if k < len(g) else 0.0 for k in range(dim)], dtype=torch.float64)
    # cell aggregates (Eqs. 17, 21)
    N = torch.zeros(nc, dtype=torch.float64).index_add(0, kg[moving], torch.ones(int(moving.sum()), dtype=torch.float64))
    L = torch.zeros(nc, dtype=torch.float64).index_add(0, kd, torch.ones(nd, dtype=torch.float64))
    sv = torch.zeros(nc, dim, dtype=torch.float64).index_add(0, kg[moving], gv.T[moving])
    sA = torch.zeros(nc, dim, dtype=torch.float64).index_add(0, kg[moving], A[moving])
    su = torch.zeros(nc, dim, dtype=torch.float64).index_add(0, kd, du.T)
    harmonic = p.tstar_mode == 1
    st = torch.zeros(nc, dtype=torch.float64).index_add(0, kd, 1.0 / tstop if harmonic else tstop)
    drag = ((N > 0) & (L > 0)).detach()
    Ns = torch.where(drag, N, torch.ones_like(N))
    Ls = torch.where(drag, L, torch.ones_like(L))
    sts = torch.where(drag, st, torch.ones_like(st))
    eps = p.m_dust * Ls / (p.m_gas * Ns)                          # Eq. 17
    tst = Ls / sts if harmonic else sts / Ls                       # t*_stop
    vs, us, Ab = sv / Ns[:, None], su / Ls[:, None], sA / Ns[:, None]
    w = vs - us
    wn = (w + tau * Ab) / (1.0 + tau * (1.0 + eps) / tst)[:, None]
    un = us + tau * gvec + (tau / tst)[:, None] * wn
    vn = un + wn
    # particle updates (Eqs. 19-20)
    kgc, kdc = kg, kd
    rhs_g = gv.T + tau * (A + gvec)
    kgas = (eps / tst)[kgc][:, None]
    v_drag = (rhs_g + tau * kgas * un[kgc]) / (1.0 + tau * kgas)
    dg = drag[kgc][:, None]
    v_new = torch.where(dg, v_drag, rhs_g)
    v_new = torch.where(moving[:, None], v_new, gv.T)
    rhs_d = du.T + tau * gvec
    kdust = (1.0 / tst)[kdc][:, None]
    u_drag = (rhs_d + tau * kdust * vn[kdc]) / (1.0 + tau * kdust)
    u_new = torch.where(drag[kdc][:, None], u_drag, rhs_d)
    x_new = torch.where(moving[:, None], xg + tau * v_new, xg)
    xd_new = dx.T + tau * u_new
    # periodic wrap (no derivative through the shift)
    def wrap(x):
        cols = []
        for k in range(dim):
            xk = x[:, k]
            if p.periodic[k]:
                Lk = p.hi[k] - p.lo[k]
                xk = xk - Lk * torch.floor((xk - p.lo[k]) / Lk).detach()
            cols.append(xk)
        return torch.stack(cols, 1)
    return wrap(x_new).T, v_new.T, wrap(xd_new).T, u_new.T
