"""Pins of the oracle's own adjoint (autograd through oracle.torch_step).

Its forward must equal the C oracle's step, and its gradients must equal
central finite differences of the C oracle, with perturbations small enough
that no cell or neighbour membership changes (checked).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from conftest import oracle_params  # noqa: E402


def _small_cases(orc):
    rng = np.random.default_rng(12)
    n, m = 40, 30
    p1 = orc.Params(dim=1, lo=(0.0,), hi=(1.0,), periodic=(1,), h=0.04, cell_size=0.1, m_gas=1.0 / n,
                    m_dust=0.7 / m)
    c1 = dict(p=p1, gx=np.sort(rng.uniform(0, 1, n))[None], gv=rng.normal(size=(1, n)) * 0.1,
              dx=np.sort(rng.uniform(0, 1, m))[None], du=rng.normal(size=(1, m)) * 0.1,
              ts=rng.uniform(1e-3, 1e-1, m), frozen=None, tau=2e-3, g=(0.0,))
    w = workloads.column2d(nside=8, precision=1)
    p2 = oracle_params(w)
    c2 = dict(p=p2, gx=w.gx, gv=w.gv + 0.05 * rng.normal(size=w.gv.shape) * (w.frozen == 0),
              dx=w.dx, du=0.05 * rng.normal(size=w.du.shape), ts=w.tstop, frozen=w.frozen, tau=w.tau,
              g=(0.0, -1.0))
    return [c1, c2]


def _c_step(orc, c, gx, gv, dx, du, ts):
    s = orc.make_state(c["p"], gx, gv, dx, du, ts, frozen=c["frozen"])
    r = orc.step(c["p"], s, c["tau"], c["g"])
    return s, r


def test_torch_step_forward_equals_c_oracle(orc):
    from oracle import torch_step
    for c in _small_cases(orc):
        s, _ = _c_step(orc, c, c["gx"], c["gv"], c["dx"], c["du"], c["ts"])
        T = lambda a: torch.tensor(np.asarray(a, np.float64))
        out = torch_step.step(c["p"], T(c["gx"]), T(c["gv"]), T(c["dx"]), T(c["du"]), T(c["ts"]), c["tau"], c["g"],
                              frozen=c["frozen"])
        for a, b in zip(out, (s.gx, s.gv, s.dx, s.du)):
            assert np.max(np.abs(a.detach().numpy() - b)) < 1e-12 * (1.0 + np.max(np.abs(b)))


def test_torch_step_gradients_equal_finite_differences(orc):
    from oracle import torch_step
    rng = np.random.default_rng(3)
    for c in _small_cases(orc):
        T = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
        ins = [T(c[k]) for k in ("gx", "gv", "dx", "du", "ts")]
        out = torch_step.step(c["p"], *ins, c["tau"], c["g"], frozen=c["frozen"])
        weights = [rng.normal(size=o.shape) for o in out]
        loss = sum((o * torch.tensor(wt)).sum() for o, wt in zip(out, weights))
        loss.backward()
        base = {k: np.array(c[k], dtype=np.float64) for k in ("gx", "gv", "dx", "du", "ts")}

        def L(vals):
            s, r = _c_step(orc, c, vals["gx"], vals["gv"], vals["dx"], vals["du"], vals["ts"])
            return sum(float(np.sum(a * wt)) for a, wt in zip((s.gx, s.gv, s.dx, s.du), weights)), r

        _, r0 = L(base)
        for name, grad in zip(("gx", "gv", "du", "ts"), (ins[0].grad, ins[1].grad, ins[3].grad, ins[4].grad)):
            flat = base[name].reshape(-1)
            idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
            for i in idx:
                if name == "gx" and c["frozen"] is not None and c["frozen"][i % c["frozen"].size]:
                    continue
                eps = 1e-6 * max(1.0, abs(flat[i])) if name != "ts" else 1e-6 * flat[i]
                vp = {k: v.copy() for k, v in base.items()}
                vm = {k: v.copy() for k, v in base.items()}
                vp[name].reshape(-1)[i] += eps
                vm[name].reshape(-1)[i] -= eps
                lp, rp = L(vp)
                lm, rm = L(vm)
                # no membership change under the perturbation
                assert np.array_equal(rp.keys_g, r0.keys_g) and np.array_equal(rm.keys_g, r0.keys_g)
                assert np.array_equal(rp.nb_count, r0.nb_count) and np.array_equal(rm.nb_count, r0.nb_count)
                fd = (lp - lm) / (2 * eps)
                ad = float(grad.numpy().reshape(-1)[i])
                assert abs(fd - ad) <= 1e-6 * (1.0 + abs(fd)), (name, i, fd, ad)


# --------------------------------------------------------------------------
# Binned dust density (cloud in cell): the profile the rollout's loss is on
# --------------------------------------------------------------------------
def test_dust_profile_weights_by_hand(orc):
    """One particle at a bin centre puts its whole mass in that bin; one a
    quarter of the way between two centres splits it 3/4 : 1/4 along that
    axis (the product of per-axis splits in 2D); walled axes keep the mass in
    the end bins, periodic axes wrap it to the far end."""
    p = orc.Params(dim=2, lo=(0.0, 0.0), hi=(1.0, 2.0), periodic=(1, 0), h=0.1, cell_size=0.1, m_gas=1.0,
                   m_dust=1.0)
    nb = (4, 8)            # bins 0.25 x 0.25
    vol = 0.25 * 0.25
    rho = orc.dust_profile(p, np.array([[0.375], [1.125]]), 2.0, nb).reshape(8, 4)
    want = np.zeros((8, 4))
    want[4, 1] = 2.0 / vol
    assert np.array_equal(rho, want)
    # x at 0.375 + 0.0625 (a quarter of the way to the next centre), y at 0.125 - 0.0625 below the first centre
    rho = orc.dust_profile(p, np.array([[0.4375], [0.0625]]), 1.0, nb).reshape(8, 4)
    want = np.zeros((8, 4))
    want[0, 1] = 0.75 / vol
    want[0, 2] = 0.25 / vol
    np.testing.assert_allclose(rho, want, rtol=1e-15, atol=0)
    # across the periodic seam in x: 0.0625 lies between the centre of the last bin (0.875, wrapped) and the first
    rho = orc.dust_profile(p, np.array([[0.0625], [1.125]]), 1.0, nb).reshape(8, 4)
    want = np.zeros((8, 4))
    want[4, 0] = 0.75 / vol
    want[4, 3] = 0.25 / vol
    np.testing.assert_allclose(rho, want, rtol=1e-15, atol=0)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_dust_profile_conserves_mass(orc, dim):
    """sum_b rho_b V = n m for any positions, inside or beyond walled edges."""
    rng = np.random.default_rng(40 + dim)
    lo, hi = (0.0, -1.0, 0.5)[:dim], (1.0, 0.5, 2.0)[:dim]
    p = orc.Params(dim=dim, lo=lo, hi=hi, periodic=(1, 0, 1)[:dim], h=0.1, cell_size=0.1, m_gas=1.0, m_dust=1.0)
    nb = (7, 5, 6)[:dim]
    x = np.stack([rng.uniform(lo[k] - 0.2, hi[k] + 0.2, 3000) for k in range(dim)])
    rho = orc.dust_profile(p, x, 0.37, nb)
    vol = np.prod([(hi[k] - lo[k]) / nb[k] for k in range(dim)])
    assert abs(rho.sum() * vol - 3000 * 0.37) < 1e-10
    assert rho.size == int(np.prod(nb)) and np.all(rho >= 0)
