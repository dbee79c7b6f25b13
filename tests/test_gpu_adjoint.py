"""The hand-written adjoint of the step against the oracle's own adjoint
(autograd through oracle.torch_step) and against central finite differences
of the C oracle over a checkpointed multi-step rollout.

Tolerances: FP64 path 1e-9 relative per component (both sides exact up to
rounding); FP32 path 1e-3 relative normwise; finite differences 1e-4
relative (the agreement asked of the differentiable rollout).
"""
import numpy as np
import pytest

import workloads
from conftest import gpu_lib, oracle_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _cases():
    rng = np.random.default_rng(12)
    n, m = 60, 45
    w1 = workloads.dustywave(n=n, precision=1)
    w1.gx = np.sort(rng.uniform(0, 1, n))[None]
    w1.dx = np.sort(rng.uniform(0, 1, m))[None]
    w1.gv = rng.normal(size=(1, n)) * 0.1
    w1.du = rng.normal(size=(1, m)) * 0.1
    w1.tstop = rng.uniform(1e-3, 1e-1, m)
    w1.params.update(h=0.03, cell_size=0.07, m_dust=0.8 / m, m_gas=1.0 / n)
    w1.tau = 2e-3
    w2 = workloads.column2d(nside=12, precision=1)
    w2.gv = w2.gv + 0.05 * rng.normal(size=w2.gv.shape) * (w2.frozen == 0)
    w2.du = 0.05 * rng.normal(size=w2.du.shape)
    w3 = workloads.box3d(nside=10, precision=1)
    return [w1, w2, w3]


def _gpu_adjoint(w, lam, precision=1):
    b = gpu_lib()
    dt = np.float64 if precision == 1 else np.float32
    p = b.params_from_dict(w.params, precision=precision)
    with b.Context(p, w.gx.astype(dt), w.gv.astype(dt), w.dx.astype(dt), w.du.astype(dt), w.tstop.astype(dt),
                   frozen=w.frozen) as c:
        arrs = [np.ascontiguousarray(a.astype(dt)) for a in lam] + [np.zeros(w.n_dust, dt)]
        c.step_adjoint(w.tau, w.g, *arrs)
        return [a.astype(np.float64) for a in arrs]


def _torch_adjoint(orc, w, lam):
    from oracle import torch_step
    p = oracle_params(w)
    T = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    ins = [T(w.gx), T(w.gv), T(w.dx), T(w.du), T(w.tstop)]
    out = torch_step.step(p, *ins, w.tau, w.g, frozen=w.frozen)
    loss = sum((o * torch.tensor(l)).sum() for o, l in zip(out, lam))
    loss.backward()
    g = [t.grad.numpy() if t.grad is not None else np.zeros(t.shape) for t in ins]
    # dust positions enter only through membership: their lambda passes through
    return [g[0], g[1], lam[2], g[3], g[4]]


@pytest.mark.parametrize("case", [0, 1, 2])
def test_step_adjoint_equals_oracle_autograd_fp64(orc, case):
    w = _cases()[case]
    rng = np.random.default_rng(7 + case)
    lam = [rng.normal(size=w.gx.shape), rng.normal(size=w.gv.shape), rng.normal(size=w.dx.shape),
           rng.normal(size=w.du.shape)]
    got = _gpu_adjoint(w, lam)
    ref = _torch_adjoint(orc, w, lam)
    moving = np.ones(w.n_gas, bool) if w.frozen is None else w.frozen == 0
    for name, a, r in zip(("gx", "gv", "dx", "du", "ts"), got, ref):
        if name in ("gx", "gv"):
            a, r = a[:, moving], r[:, moving]
        err = np.max(np.abs(a - r)) / max(np.max(np.abs(r)), 1e-300)
        assert err < 1e-9, (name, err)


def test_step_adjoint_fp32_close_to_oracle(orc):
    w = _cases()[1]
    rng = np.random.default_rng(21)
    lam = [rng.normal(size=w.gx.shape), rng.normal(size=w.gv.shape), rng.normal(size=w.dx.shape),
           rng.normal(size=w.du.shape)]
    w32 = workloads.column2d(nside=12, precision=0)
    w32.gv = w.gv.astype(np.float32).astype(np.float64)
    w32.du = w.du.astype(np.float32).astype(np.float64)
    got = _gpu_adjoint(w32, lam, precision=0)
    ref = _torch_adjoint(orc, w32, lam)
    moving = w32.frozen == 0
    for name, a, r in zip(("gx", "gv", "dx", "du", "ts"), got, ref):
        if name in ("gx", "gv"):
            a, r = a[:, moving], r[:, moving]
        err = np.linalg.norm(a - r) / np.linalg.norm(r)
        assert err < 1e-3, (name, err)


def test_checkpointed_rollout_matches_finite_differences(orc):
    """Column, 20 steps, checkpoint every 7: d(loss)/d(t_stop) and
    d(loss)/d(initial velocities) against central differences of the C oracle."""
    from paper_1908_01682_gb300 import adjoint
    b = gpu_lib()
    w = workloads.column2d(nside=12, precision=1)
    rng = np.random.default_rng(5)
    w.gv = w.gv + 0.02 * rng.normal(size=w.gv.shape) * (w.frozen == 0)
    w.du = 0.02 * rng.normal(size=w.du.shape)
    nsteps = 20
    wd = rng.normal(size=w.dx.shape)   # loss = sum wd * x_dust(final) + sum wv * v_gas(final)
    wv = rng.normal(size=w.gv.shape) * (w.frozen == 0)
    p = b.params_from_dict(w.params)
    dev = lambda a: torch.tensor(np.asarray(a, np.float64), device="cuda")
    with b.Context(p, w.gx, w.gv, w.dx, w.du, w.tstop, frozen=w.frozen) as c:
        roll = adjoint.Rollout(c, w.tau, w.g, nsteps, checkpoint_every=7, frozen=w.frozen)
        ts = dev(w.tstop).requires_grad_()
        gv0 = dev(w.gv).requires_grad_()
        du0 = dev(w.du).requires_grad_()
        gx, gvf, dx, du = adjoint.TFSPHRollout.apply(ts, gv0, du0, roll, dev(w.gx), dev(w.dx))
        loss = (dx * dev(wd)).sum() + (gvf * dev(wv)).sum()
        loss.backward()
        g_ts, g_gv, g_du = ts.grad.cpu().numpy(), gv0.grad.cpu().numpy(), du0.grad.cpu().numpy()
        # the rollout without intermediate checkpoints gives the same gradients
        roll1 = adjoint.Rollout(c, w.tau, w.g, nsteps, checkpoint_every=nsteps, frozen=w.frozen)
        ts1 = dev(w.tstop).requires_grad_()
        out1 = adjoint.TFSPHRollout.apply(ts1, dev(w.gv), dev(w.du), roll1, dev(w.gx), dev(w.dx))
        ((out1[2] * dev(wd)).sum() + (out1[1] * dev(wv)).sum()).backward()
        assert np.array_equal(ts1.grad.cpu().numpy(), g_ts)

    po = oracle_params(w)

    def L(ts_, gv_, du_):
        s = orc.make_state(po, w.gx, gv_, w.dx, du_, ts_, frozen=w.frozen)
        keys = []
        for _ in range(nsteps):
            r = orc.step(po, s, w.tau, w.g)
            keys.append((r.keys_g.copy(), r.keys_d.copy(), r.nb_count.copy()))
        return float(np.sum(wd * s.dx) + np.sum(wv * s.gv)), keys

    _, k0 = L(w.tstop, w.gv, w.du)
    checks = [("ts", j) for j in rng.choice(w.n_dust, 4, replace=False)]
    checks += [("du", j) for j in rng.choice(w.du.size, 3, replace=False)]
    moving_idx = np.where(np.tile(w.frozen == 0, 2))[0]
    checks += [("gv", j) for j in rng.choice(moving_idx, 3, replace=False)]
    for name, j in checks:
        base = {"ts": w.tstop.copy(), "gv": w.gv.copy(), "du": w.du.copy()}
        arr = base[name].reshape(-1)
        eps = 1e-5 * arr[j] if name == "ts" else 1e-6
        vals = []
        for sgn in (+1, -1):
            bb = {k: v.copy() for k, v in base.items()}
            bb[name].reshape(-1)[j] += sgn * eps
            lv, kk = L(bb["ts"], bb["gv"], bb["du"])
            assert all(np.array_equal(a[0], b0[0]) and np.array_equal(a[1], b0[1]) and np.array_equal(a[2], b0[2])
                       for a, b0 in zip(kk, k0)), "membership changed under the perturbation"
            vals.append(lv)
        fd = (vals[0] - vals[1]) / (2 * eps)
        ad = {"ts": g_ts, "gv": g_gv, "du": g_du}[name].reshape(-1)[j]
        assert abs(ad - fd) <= 1e-4 * abs(fd) + 1e-7, (name, j, ad, fd)


# ---------------------------------------------------------------------------
# The loss on the final dust-density profile
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_dust_profile_matches_oracle(orc, prec):
    """tfsph_dust_profile against the oracle's cloud-in-cell profile on the
    settling column's dust (and on positions beyond the walls), 64 x 64 bins:
    1e-12 (FP64 positions) or 1e-5 (FP32 positions) normwise; its gradient of
    the squared-error loss against central differences of the oracle's loss
    at a sample of particles."""
    from paper_1908_01682_gb300 import adjoint
    b = gpu_lib()
    w = workloads.column2d(nside=64, precision=prec)
    rng = np.random.default_rng(3)
    # the dust lattice sits on the bin centres, where the weights have kinks: jitter it off them
    x = w.dx + rng.uniform(-0.3, 0.3, w.dx.shape) / 64
    x[1, :50] = rng.uniform(-0.05, 0.0, 50)          # sunk below the bottom wall
    x[0, 50:100] = rng.uniform(0.99, 1.0, 50)        # next to the periodic seam
    dt = torch.float64 if prec == 1 else torch.float32
    p = b.params_from_dict(w.params)
    grid = b.grid_spec(2, (0.0, 0.0), (1.0, 1.0), (1, 0), (64, 64), w.params["m_dust"], prec)
    xd = torch.tensor(x, dtype=dt, device="cuda")
    rho = adjoint.dust_profile(grid, xd).cpu().numpy()
    po = oracle_params(w)
    ref = orc.dust_profile(po, xd.cpu().numpy().astype(np.float64), w.params["m_dust"], (64, 64))
    err = np.linalg.norm(rho - ref) / np.linalg.norm(ref)
    assert err < (1e-12 if prec == 1 else 1e-5), err
    target = torch.tensor(ref * (1 + 0.1 * rng.normal(size=ref.shape)), dtype=torch.float64, device="cuda")
    xg = xd.clone().requires_grad_()
    loss = adjoint.DustProfileLoss.apply(xg, target, grid)
    loss.backward()
    g = xg.grad.cpu().numpy().astype(np.float64)
    tgt = target.cpu().numpy()
    x64 = xd.cpu().numpy().astype(np.float64)
    L = lambda xx: float(np.sum((orc.dust_profile(po, xx, w.params["m_dust"], (64, 64)) - tgt) ** 2))
    assert abs(float(loss) - L(x64)) <= (1e-10 if prec == 1 else 1e-4) * L(x64)
    if prec == 1:
        for j in rng.choice(x.shape[1], 12, replace=False):
            for k in range(2):
                e = 1e-7
                xp, xm = x64.copy(), x64.copy()
                xp[k, j] += e
                xm[k, j] -= e
                fd = (L(xp) - L(xm)) / (2 * e)
                assert abs(g[k, j] - fd) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max(), (j, k, g[k, j], fd)


def test_profile_loss_rollout_matches_finite_differences(orc):
    """The rollout's gradient on a small settling column (FP64): the squared
    error of the final binned dust density (8 x 8 bins) against a seeded
    target after 20 steps checkpointed every 7, with respect to per-particle
    t_stop and the initial gas and dust velocities, against central
    differences of the C oracle's rollout and profile, 1e-4 relative."""
    from paper_1908_01682_gb300 import adjoint
    b = gpu_lib()
    w = workloads.column2d(nside=12, precision=1)
    rng = np.random.default_rng(8)
    w.gv = w.gv + 0.02 * rng.normal(size=w.gv.shape) * (w.frozen == 0)
    w.du = 0.02 * rng.normal(size=w.du.shape)
    nsteps, nb = 20, (8, 8)
    p = b.params_from_dict(w.params)
    dev = lambda a: torch.tensor(np.asarray(a, np.float64), device="cuda")
    po = oracle_params(w)
    ref0 = orc.dust_profile(po, w.dx, w.params["m_dust"], nb)
    target = ref0 * (1 + 0.2 * rng.normal(size=ref0.shape))
    with b.Context(p, w.gx, w.gv, w.dx, w.du, w.tstop, frozen=w.frozen) as c:
        roll = adjoint.Rollout(c, w.tau, w.g, nsteps, checkpoint_every=7, frozen=w.frozen)
        grid = adjoint.profile_grid(c, nb)
        ts = dev(w.tstop).requires_grad_()
        gv0 = dev(w.gv).requires_grad_()
        du0 = dev(w.du).requires_grad_()
        _, _, dxf, _ = adjoint.TFSPHRollout.apply(ts, gv0, du0, roll, dev(w.gx), dev(w.dx))
        loss = adjoint.DustProfileLoss.apply(dxf, dev(target), grid)
        loss.backward()
        g = {"ts": ts.grad.cpu().numpy(), "gv": gv0.grad.cpu().numpy(), "du": du0.grad.cpu().numpy()}
        gpu_loss = float(loss)

    def L(ts_, gv_, du_):
        s = orc.make_state(po, w.gx, gv_, w.dx, du_, ts_, frozen=w.frozen)
        keys = []
        for _ in range(nsteps):
            r = orc.step(po, s, w.tau, w.g)
            keys.append((r.keys_g.copy(), r.keys_d.copy(), r.nb_count.copy()))
        rho = orc.dust_profile(po, s.dx, w.params["m_dust"], nb)
        # the bins a particle's weights go to (the linear piece it is on)
        piece = np.floor((s.dx - 0.0) / (1.0 / np.array(nb)[:, None]) - 0.5)
        return float(np.sum((rho - target) ** 2)), keys, piece

    l0, k0, piece0 = L(w.tstop, w.gv, w.du)
    assert abs(gpu_loss - l0) <= 1e-9 * l0
    checks = [("ts", j) for j in rng.choice(w.n_dust, 4, replace=False)]
    checks += [("du", j) for j in rng.choice(w.du.size, 3, replace=False)]
    moving_idx = np.where(np.tile(w.frozen == 0, 2))[0]
    checks += [("gv", j) for j in rng.choice(moving_idx, 3, replace=False)]
    for name, j in checks:
        base = {"ts": w.tstop.copy(), "gv": w.gv.copy(), "du": w.du.copy()}
        arr = base[name].reshape(-1)
        eps = 1e-5 * arr[j] if name == "ts" else 1e-6
        vals = []
        for sgn in (+1, -1):
            bb = {k: v.copy() for k, v in base.items()}
            bb[name].reshape(-1)[j] += sgn * eps
            lv, kk, pc = L(bb["ts"], bb["gv"], bb["du"])
            assert all(np.array_equal(a[0], b0[0]) and np.array_equal(a[1], b0[1]) and np.array_equal(a[2], b0[2])
                       for a, b0 in zip(kk, k0)), "membership changed under the perturbation"
            assert np.array_equal(pc, piece0), "a particle crossed a bin centre under the perturbation"
            vals.append(lv)
        fd = (vals[0] - vals[1]) / (2 * eps)
        ad = g[name].reshape(-1)[j]
        assert abs(ad - fd) <= 1e-4 * abs(fd) + 1e-7 * abs(l0), (name, j, ad, fd)
