"""Closed-form solutions that pin the oracle (test infrastructure only).

None of this is the method itself: these are exact solutions of the continuum
two-fluid equations (Sec. 1, Eqs. 1-3, in the K form of Eq. 7) for the two
test problems of Sec. 3 (Dustywave, Dustyshock), derived here because the
paper does not print them.

- ``dusty_wave``: linearised isothermal two-fluid equations for one Fourier
  mode, solved exactly with a matrix exponential; its eigenvalues are the
  roots of the dispersion cubic
  s^3 + (1+eps)/t_s s^2 + cs^2 k^2 s + cs^2 k^2 / t_s = 0.
- ``sod_exact``: exact Riemann solution of the ideal-gas Euler equations
  (pressure-function iteration, the textbook method of Godunov as set out in
  Toro's book), used for a dust-free adiabatic shock tube.
- ``isothermal_riemann``: exact Riemann solution of the isothermal Euler
  equations, which is the strongly coupled (t_stop -> 0) limit of an
  isothermal dusty gas with sound speed cs / sqrt(1 + eps) and density
  (1 + eps) rho_g.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm
from scipy.optimize import brentq


# --------------------------------------------------------------------------
# Dusty sound wave
# --------------------------------------------------------------------------
def dispersion_roots(k: float, cs: float, tstop: float, eps: float) -> np.ndarray:
    """Roots s of s^3 + (1+eps)/t s^2 + cs^2 k^2 s + cs^2 k^2 / t = 0."""
    return np.roots([1.0, (1.0 + eps) / tstop, cs * cs * k * k, cs * cs * k * k / tstop])


def wave_matrix(k: float, cs: float, rho_g: float, rho_d: float, tstop: float) -> np.ndarray:
    """Linear operator M of d/dt (drho_g, dv, du) = M (drho_g, dv, du) for e^{ikx}.

    From Eq. 7 with K = rho_d / t_stop, isothermal p = cs^2 rho_g, and the
    gas continuity equation of Eq. 1.
    """
    K = rho_d / tstop
    return np.array([
        [0.0, -1j * k * rho_g, 0.0],
        [-1j * k * cs * cs / rho_g, -K / rho_g, K / rho_g],
        [0.0, K / rho_d, -K / rho_d],
    ], dtype=complex)


def dusty_wave(x, t: float, k: float, cs: float, rho_g: float, rho_d: float, tstop: float,
               amp_rho: float, amp_v: float, amp_u: float):
    """Gas density, gas velocity and dust velocity at positions x and time t.

    Initial state: rho_g (1 + amp_rho sin kx), v = amp_v sin kx, u = amp_u sin kx.
    """
    y0 = np.array([amp_rho * rho_g, amp_v, amp_u], dtype=complex)
    y = expm(wave_matrix(k, cs, rho_g, rho_d, tstop) * t) @ y0
    ph = np.exp(1j * k * np.asarray(x, dtype=float))
    rho = rho_g + np.imag(y[0] * ph)
    v = np.imag(y[1] * ph)
    u = np.imag(y[2] * ph)
    return rho, v, u


# --------------------------------------------------------------------------
# Ideal-gas Riemann problem
# --------------------------------------------------------------------------
def _pfun(p, rho, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def sod_star(rl, ul, pl, rr, ur, pr, g):
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    f = lambda p: _pfun(p, rl, pl, cl, g) + _pfun(p, rr, pr, cr, g) + ur - ul
    ps = brentq(f, 1e-12, 10.0 * max(pl, pr), xtol=1e-15, rtol=1e-14, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_pfun(ps, rr, pr, cr, g) - _pfun(ps, rl, pl, cl, g))
    return ps, us


def sod_exact(x, t: float, x0: float, rl, ul, pl, rr, ur, pr, g: float):
    """Density, velocity and pressure of the exact ideal-gas Riemann solution."""
    x = np.asarray(x, dtype=float)
    ps, us = sod_star(rl, ul, pl, rr, ur, pr, g)
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    g6 = (g - 1.0) / (g + 1.0)
    rho = np.empty_like(x)
    vel = np.empty_like(x)
    pre = np.empty_like(x)
    for i, xi in enumerate(x):
        S = (xi - x0) / t
        if S <= us:
            if ps > pl:  # left shock
                SL = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if S < SL:
                    r, u, p = rl, ul, pl
                else:
                    r, u, p = rl * (ps / pl + g6) / (g6 * ps / pl + 1.0), us, ps
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if S < ul - cl:
                    r, u, p = rl, ul, pl
                elif S > us - csl:
                    r, u, p = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    u = 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * ul + S)
                    c = 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * (ul - S))
                    r = rl * (c / cl) ** (2.0 / (g - 1))
                    p = pl * (c / cl) ** (2.0 * g / (g - 1))
        else:
            if ps > pr:  # right shock
                SR = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if S > SR:
                    r, u, p = rr, ur, pr
                else:
                    r, u, p = rr * (ps / pr + g6) / (g6 * ps / pr + 1.0), us, ps
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if S > ur + cr:
                    r, u, p = rr, ur, pr
                elif S < us + csr:
                    r, u, p = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    u = 2.0 / (g + 1) * (-cr + 0.5 * (g - 1) * ur + S)
                    c = 2.0 / (g + 1) * (cr - 0.5 * (g - 1) * (ur - S))
                    r = rr * (c / cr) ** (2.0 / (g - 1))
                    p = pr * (c / cr) ** (2.0 * g / (g - 1))
        rho[i], vel[i], pre[i] = r, u, p
    return rho, vel, pre


# --------------------------------------------------------------------------
# Isothermal Riemann problem
# --------------------------------------------------------------------------
def _ifun(rs, rk, a):
    if rs > rk:  # shock
        z = rs / rk
        return a * (z - 1.0) / np.sqrt(z)
    return a * np.log(rs / rk)  # rarefaction


def isothermal_riemann(x, t: float, x0: float, rl, ul, rr, ur, a: float):
    """Density and velocity of the exact isothermal Riemann solution (sound speed a)."""
    x = np.asarray(x, dtype=float)
    f = lambda r: _ifun(r, rl, a) + _ifun(r, rr, a) + ur - ul
    rs = brentq(f, 1e-12 * min(rl, rr), 100.0 * max(rl, rr), xtol=1e-15, rtol=1e-14, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_ifun(rs, rr, a) - _ifun(rs, rl, a))
    rho = np.empty_like(x)
    vel = np.empty_like(x)
    for i, xi in enumerate(x):
        S = (xi - x0) / t
        if S <= us:
            if rs > rl:
                SL = ul - a * np.sqrt(rs / rl)
                r, u = (rl, ul) if S < SL else (rs, us)
            else:
                if S < ul - a:
                    r, u = rl, ul
                elif S > us - a:
                    r, u = rs, us
                else:
                    u = S + a
                    r = rl * np.exp((ul - u) / a)
        else:
            if rs > rr:
                SR = ur + a * np.sqrt(rs / rr)
                r, u = (rr, ur) if S > SR else (rs, us)
            else:
                if S > ur + a:
                    r, u = rr, ur
                elif S < us + a:
                    r, u = rs, us
                else:
                    u = S - a
                    r = rr * np.exp((u - ur) / a)
        rho[i], vel[i] = r, u
    return rho, vel
