"""The ISPH (Sec. 2.2) and MK (Sec. 2.1) drag schemes on the GPU against the
FP64 oracle (oracle.step_x), element by element after one step, and over
several steps on the dusty wave.

Bounds (tol = 1e-5 FP32, 1e-12 FP64; u the path's unit roundoff, K = 128):
- positions: normwise (minimum-image differences) <= tol;
- MK velocities: |v' - v'_ref| <= tol (|v'_ref| + |v|) + K u tau (S_a + S_D), with S_a
  the magnitude sum of the pressure pair terms and S_D that of the drag pair terms;
- ISPH velocities: |v' - v'_ref| <= tol (|v'_ref| + |v| + |u~|) + K u (S_u + tau S_A),
  with u~ the interpolated velocity of the other phase, S_u the magnitude sum
  of its interpolation terms and S_A that of the particle's pressure terms.
"""
import numpy as np
import pytest

import workloads
from conftest import gpu_context, gpu_lib, oracle_params
from parity import KAPPA, TOL, UNIT, _pos_err

pytestmark = pytest.mark.gpu


def _run(w, scheme, nsteps=1, g=None):
    b = gpu_lib()
    g = w.g if g is None else g
    with gpu_context(w, drag=scheme) as c:
        for _ in range(nsteps):
            c.step(w.tau, g)
        c.sync()
        return [c.field(f).astype(np.float64) for f in (b.TFSPH_FIELD_POS_G, b.TFSPH_FIELD_VEL_G,
                                                         b.TFSPH_FIELD_POS_D, b.TFSPH_FIELD_VEL_D)]


def _check(orc, w, scheme, prec):
    tol, ku = TOL[prec], KAPPA * UNIT[prec]
    gx, gv, dx, du = _run(w, scheme)
    p = oracle_params(w)
    s = orc.make_state(p, w.gx, w.gv, w.dx, w.du, w.tstop, ge=w.ge, frozen=w.frozen)
    r = orc.step_x(p, s, w.tau, w.g, scheme=scheme)
    assert _pos_err(gx, s.gx, w) <= tol and _pos_err(dx, s.dx, w) <= tol
    moving = np.ones(w.n_gas, bool) if w.frozen is None else w.frozen == 0
    tau = w.tau
    if scheme == orc.MK:
        bg = tol * (np.abs(s.gv) + np.abs(w.gv)) + ku * tau * (r.acc_scale_g + r.scale_g)
        bd = tol * (np.abs(s.du) + np.abs(w.du)) + ku * tau * r.scale_d
    else:
        bg = tol * (np.abs(s.gv) + np.abs(w.gv) + np.abs(r.drag_g)) + ku * (r.scale_g + tau * r.acc_scale_g)
        bd = tol * (np.abs(s.du) + np.abs(w.du) + np.abs(r.drag_d)) + ku * (r.scale_d + tau * r.isph_acc_scale_d)
    eg = np.abs(gv - s.gv)[:, moving] / np.maximum(bg[:, moving], 1e-300)
    ed = np.abs(du - s.du) / np.maximum(bd, 1e-300)
    assert (eg.size == 0 or eg.max() <= 1.0) and (ed.size == 0 or ed.max() <= 1.0), (
        eg.max() if eg.size else 0, ed.max() if ed.size else 0)
    return r


def _cases():
    w1 = workloads.dustywave(n=200, precision=1, tstop=2e-3)
    w2 = workloads.dustywave(n=300, precision=0, tstop=1e-3)
    w3 = workloads.column2d(nside=20, precision=0, nsteps=1)
    w4 = workloads.box3d(nside=10, precision=0)
    w5 = workloads.dustyshock(n_left=400, n_right=50, precision=0)
    return {"wave_fp64": (w1, 1), "wave_fp32": (w2, 0), "column2d": (w3, 0), "box3d": (w4, 0), "shock": (w5, 0)}


@pytest.mark.parametrize("case", ["wave_fp64", "wave_fp32", "column2d", "box3d", "shock"])
@pytest.mark.parametrize("scheme", [1, 2], ids=["isph", "mk"])
def test_xdrag_one_step_matches_oracle(orc, case, scheme):
    w, prec = _cases()[case]
    if scheme == orc.MK:
        # the explicit scheme is run within its stability limit, tau < t_stop
        w.tau = min(w.tau, 0.5 * float(np.min(w.tstop)))
    _check(orc, w, scheme, prec)


@pytest.mark.parametrize("scheme", [1, 2], ids=["isph", "mk"])
def test_xdrag_dusty_wave_ten_steps_fp64(orc, scheme):
    w = workloads.dustywave(n=120, precision=1, tstop=2e-3)
    w.tau = 5e-4
    gx, gv, dx, du = _run(w, scheme, nsteps=10)
    p = oracle_params(w)
    s = orc.make_state(p, w.gx, w.gv, w.dx, w.du, w.tstop)
    orc.run(p, s, w.tau, 10, scheme=scheme)
    scale = np.max(np.abs(s.gv)) + np.max(np.abs(s.du))
    assert np.max(np.abs(gv - s.gv)) <= 1e-11 * scale and np.max(np.abs(du - s.du)) <= 1e-11 * scale
    assert _pos_err(gx, s.gx, w) <= 1e-12 and _pos_err(dx, s.dx, w) <= 1e-12


def test_mk_conserves_momentum_on_the_gpu(orc):
    """FP64, 2D periodic random state, g = 0: total momentum after an MK step
    equals the momentum before to roundoff."""
    rng = np.random.default_rng(4)
    w = workloads.column2d(nside=16, precision=1, nsteps=1)
    ng, nd = 400, 300
    w.params.update(periodic=(1, 1))
    w.gx = rng.uniform(0, 1, (2, ng))
    w.gv = rng.normal(0, 0.1, (2, ng))
    w.dx = rng.uniform(0, 1, (2, nd))
    w.du = rng.normal(0, 0.1, (2, nd))
    w.tstop = np.exp(rng.uniform(np.log(1e-2), np.log(1e-1), nd))
    w.frozen = None
    w.params.update(h=0.05, cell_size=0.1, m_gas=1.0 / ng, m_dust=0.5 / nd)
    w.tau = 1e-3
    w.g = (0.0, 0.0, 0.0)
    gx, gv, dx, du = _run(w, 2)
    m_g, m_d = w.params["m_gas"], w.params["m_dust"]
    before = m_g * w.gv.sum(1) + m_d * w.du.sum(1)
    after = m_g * gv.sum(1) + m_d * du.sum(1)
    scale = m_g * np.abs(w.gv).sum() + m_d * np.abs(w.du).sum()
    assert np.max(np.abs(after - before)) <= 1e-13 * scale


def test_adjoint_and_batch_refuse_other_schemes(orc):
    b = gpu_lib()
    w = workloads.dustywave(n=50, precision=1)
    with gpu_context(w, drag=b.TFSPH_DRAG_ISPH) as c:
        z = np.zeros((1, 50))
        with pytest.raises(b.TfsphError):
            c.step_adjoint(w.tau, w.g, z, z.copy(), z.copy(), z.copy(), np.zeros(50))
    items = [(b.params_from_dict(w.params, precision=0, drag=b.TFSPH_DRAG_MK), w.gx, w.gv, w.dx, w.du, w.tstop)]
    with pytest.raises(b.TfsphError):
        b.Batch(items)
