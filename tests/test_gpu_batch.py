"""Batched ensembles (tfsph_batch_*) on the GPU.

- every instance of a batch against the FP64 oracle run on that instance
  alone, with the bounds of the single-context parity tests;
- the launch forms (one launch per phase, persistent cooperative launch;
  CTA sizes) against each other, bit for bit, over several steps;
- graph replay of n steps against n separate calls, bit for bit;
- the batch against single contexts holding one instance each (rounding of
  the neighbour sums only);
- the autotuner leaves the state as it found it;
- a persistent grid barrier whose wait limit is zero reports
  TFSPH_E_TIMEOUT instead of waiting.
"""
import numpy as np
import pytest

import workloads
from conftest import gpu_lib
from parity import KAPPA, TOL, UNIT, check_one_step, oracle_step

pytestmark = pytest.mark.gpu


def _waves():
    """Dusty waves of uneven sizes, t_stop and amplitudes (one on a longer
    box, one without dust)."""
    spec = [(8, 1e-3, 1e-5), (37, 5e-4, 1e-3), (100, 1e-4, 0.1), (513, 1e-5, 1.0), (2048, 1e-3, 3e-4)]
    ws = [workloads.dustywave(n=n, amp=a, tstop=t, precision=0, nsteps=1) for n, a, t in spec]
    ws.append(workloads.dustywave(n=300, amp=2e-4, tstop=2e-2, precision=0, nsteps=1, length=2.0))
    nod = workloads.dustywave(n=64, amp=3e-4, tstop=1e-2, precision=0, nsteps=1)
    nod.dx, nod.du, nod.tstop = nod.dx[:, :0], nod.du[:, :0], nod.tstop[:0]
    ws.append(nod)
    return ws


def _columns():
    """2D settling columns (walls of frozen gas, periodic x) of three sizes."""
    return [workloads.column2d(nside=n, precision=0, nsteps=1, seed_tstop=s) for n, s in ((12, 1), (16, 2), (24, 3))]


def _batch(b, ws, **over):
    items = [(b.params_from_dict(w.params, **over), w.gx, w.gv, w.dx, w.du, w.tstop, w.frozen) for w in ws]
    return b.Batch(items)


def _state(bt, b):
    return [bt.field(f) for f in (b.TFSPH_FIELD_POS_G, b.TFSPH_FIELD_VEL_G, b.TFSPH_FIELD_POS_D,
                                  b.TFSPH_FIELD_VEL_D)]


def _instance_out(bt, b, i, fields):
    gx, gv, dx, du = fields
    g0, g1 = bt.goff[i], bt.goff[i + 1]
    d0, d1 = bt.doff[i], bt.doff[i + 1]
    f64 = lambda a: np.asarray(a, np.float64)
    return {"gx": f64(gx[:, g0:g1]), "gv": f64(gv[:, g0:g1]), "dx": f64(dx[:, d0:d1]), "du": f64(du[:, d0:d1])}


@pytest.mark.parametrize("mode", ["kernels", "persistent", "tiled"])
def test_batch_1d_matches_oracle_per_instance(orc, mode):
    b = gpu_lib()
    ws = _waves()
    with _batch(b, ws) as bt:
        if mode == "persistent":
            bt.config(b.TFSPH_BATCH_PERSISTENT, 256, 2)
        elif mode == "tiled":
            bt.config(b.TFSPH_BATCH_TILED, 128, 1)
        rho = bt.field(b.TFSPH_FIELD_RHO_G)
        bt.step([w.tau for w in ws])
        bt.sync()
        out = _state(bt, b)
        for i, w in enumerate(ws):
            gpu = _instance_out(bt, b, i, out)
            gpu["rho_g"] = rho[bt.goff[i]:bt.goff[i + 1]].astype(np.float64)
            check_one_step(orc, w, gpu, 0)


@pytest.mark.parametrize("cell_acc", [0, 1])
def test_batch_ensemble_full_size_matches_oracle(orc, cell_acc):
    """The benchmarked ensemble, 256 dusty waves of 1k-64k particles (3.9M in
    total), with FP32 cell sums (cell_acc 0, the benchmarked form) and FP64
    cell sums, in the launch form the autotuner picks: every instance after
    one step against the oracle run on that instance alone."""
    b = gpu_lib()
    ws = workloads.ensemble1d(precision=0)
    with _batch(b, ws, cell_acc=cell_acc) as bt:
        bt.step([w.tau for w in ws], nsteps=0)
        pick = bt.autotune(steps=3)
        rho = bt.field(b.TFSPH_FIELD_RHO_G)
        bt.step(nsteps=1)
        bt.sync()
        assert bt.info().steps == 1
        out = _state(bt, b)
        worst = {}
        for i, w in enumerate(ws):
            gpu = _instance_out(bt, b, i, out)
            gpu["rho_g"] = rho[bt.goff[i]:bt.goff[i + 1]].astype(np.float64)
            _, errs = check_one_step(orc, w, gpu, 0)
            for k, e in errs.items():
                worst[k] = max(worst.get(k, 0.0), e)
    print(f"ensemble, cell_acc={cell_acc}, form {pick}: worst errors {worst}")


def test_batch_2d_walls_and_gravity_match_oracle(orc):
    b = gpu_lib()
    ws = _columns()
    gs = [(0.0, -1.0), (0.3, -0.5), (0.0, -2.0)]
    with _batch(b, ws) as bt:
        bt.step([w.tau for w in ws], g=gs)
        bt.sync()
        out = _state(bt, b)
        for i, w in enumerate(ws):
            check_one_step(orc, w, _instance_out(bt, b, i, out), 0, g=(gs[i][0], gs[i][1], 0.0))


@pytest.mark.parametrize("form", [("kernels", 128, 1), ("kernels", 512, 1), ("persistent", 128, 4),
                                  ("persistent", 512, 1), ("tiled", 128, 1), ("tiled", 256, 1), ("tiled", 512, 1)])
def test_batch_launch_forms_agree_bit_for_bit(form):
    b = gpu_lib()
    ws = _waves()
    taus = [w.tau for w in ws]
    with _batch(b, ws) as ref:
        ref.step(taus, nsteps=7)
        want = _state(ref, b)
    with _batch(b, ws) as bt:
        mode = {"persistent": b.TFSPH_BATCH_PERSISTENT, "kernels": b.TFSPH_BATCH_KERNELS,
                "tiled": b.TFSPH_BATCH_TILED}[form[0]]
        bt.config(mode, form[1], form[2])
        bt.step(taus, nsteps=7)
        bt.sync()
        got = _state(bt, b)
        info = bt.info()
        assert info.mode == mode and info.block == form[1] and info.steps == 7
    for a, r in zip(got, want):
        assert np.array_equal(a, r)


def test_batch_graph_replay_equals_separate_steps():
    b = gpu_lib()
    ws = _columns()
    taus = [w.tau for w in ws]
    g = [(0.0, -1.0)] * len(ws)
    with _batch(b, ws) as a:
        a.step(taus, g=g, nsteps=6)
        a.sync()
        ia = a.info()
        sa = _state(a, b)
    with _batch(b, ws) as c:
        c.step(taus, g=g, nsteps=0)
        for _ in range(6):
            c.step(nsteps=1)
        sc = _state(c, b)
    assert ia.graph == 1 and ia.steps == 6 and ia.launches == 6 * 10
    for x, y in zip(sa, sc):
        assert np.array_equal(x, y)


def test_batch_matches_single_contexts(orc):
    """Five steps of the batch against a single context per instance: the
    same method, only the summation order of neighbour terms differs, so the
    velocities may differ by the rounding of the pair sums, K u tau S_a per
    step and side (S_a: the oracle's magnitude sum of the pair terms)."""
    b = gpu_lib()
    ws = _waves()[:6]
    nsteps = 5
    with _batch(b, ws) as bt:
        bt.step([w.tau for w in ws], nsteps=nsteps)
        out = _state(bt, b)
    for i, w in enumerate(ws):
        p = b.params_from_dict(w.params)
        f32 = lambda a: np.ascontiguousarray(a, np.float32)
        with b.Context(p, f32(w.gx), f32(w.gv), f32(w.dx), f32(w.du), f32(w.tstop)) as c:
            for _ in range(nsteps):
                c.step(w.tau, w.g)
            single = [c.field(f) for f in (b.TFSPH_FIELD_POS_G, b.TFSPH_FIELD_VEL_G, b.TFSPH_FIELD_POS_D,
                                           b.TFSPH_FIELD_VEL_D)]
        _, _, r, _ = oracle_step(orc, w)
        S = float(np.max(r.acc_scale_g))
        vmax = float(np.max(np.abs(w.gv))) + float(np.max(np.abs(w.du)))
        vbound = nsteps * 2 * KAPPA * UNIT[0] * w.tau * 2 * S + TOL[0] * vmax
        xbound = 8 * UNIT[0] * (w.params["hi"][0] - w.params["lo"][0]) + nsteps * w.tau * vbound
        mine = _instance_out(bt, b, i, out)
        for key, sv in zip(("gx", "gv", "dx", "du"), single):
            d = np.abs(mine[key] - sv.astype(np.float64))
            bound = xbound if key in ("gx", "dx") else vbound
            assert d.max() <= bound, (i, key, d.max(), bound)


def test_batch_autotune_restores_state_and_picks_a_form():
    b = gpu_lib()
    ws = _waves()
    taus = [w.tau for w in ws]
    with _batch(b, ws) as ref:
        ref.step(taus, nsteps=3)
        want = _state(ref, b)
    with _batch(b, ws) as bt:
        bt.step(taus, nsteps=0)
        before = _state(bt, b)
        pick = bt.autotune(steps=3)
        after = _state(bt, b)
        assert pick["mode"] in (b.TFSPH_BATCH_KERNELS, b.TFSPH_BATCH_PERSISTENT)
        assert pick["block"] in (128, 256, 512) and pick["ms_per_step"] > 0
        assert bt.info().steps == 0
        bt.step(nsteps=3)
        got = _state(bt, b)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_batch_barrier_timeout_is_reported():
    """A persistent step whose barrier may not wait at all: every CTA but the
    last to arrive gives up at once, records the timeout and returns; the
    host sees TFSPH_E_TIMEOUT from the next sync and the GPU stays usable."""
    b = gpu_lib()
    ws = _waves()[:3]
    with _batch(b, ws) as bt:
        bt.config(b.TFSPH_BATCH_PERSISTENT, 128, 2, barrier_timeout_ms=0.0)
        bt.step([w.tau for w in ws])
        with pytest.raises(b.TfsphError) as ei:
            bt.sync()
        assert ei.value.code == b.TFSPH_E_TIMEOUT
    # a fresh batch on the same device runs normally
    with _batch(b, ws) as bt:
        bt.step([w.tau for w in ws])
        bt.sync()


def test_batch_tiled_form_refused_for_2d():
    """The tiled form stages windows of consecutive cells: 1D batches only."""
    b = gpu_lib()
    with _batch(b, _columns()) as bt:
        with pytest.raises(b.TfsphError) as ei:
            bt.config(b.TFSPH_BATCH_TILED, 256, 1)
        assert ei.value.code == b.TFSPH_E_INVALID_ARG
        bt.step([w.tau for w in _columns()], g=[(0.0, -1.0)] * 3)  # the batch stays usable
        bt.sync()
