"""GPU path against the FP64 oracle, element by element, on seeded inputs.

Bit-exact: cell keys, the (cell key, id) sort order and cell ranges (both
sides take the exact floor of (x - lo) n / L), and the neighbour sets (count
and fingerprint per particle) outside a band of 8 ulp of 4h^2 around the
support radius, where the oracle's exact membership and the path's rounded
one may differ (reported).

Within tolerance after one step, tol = 1e-5 (FP32 path) or 1e-12 (FP64 path):
- densities, positions and energies: normwise ||x - x_ref|| / ||x_ref|| <= tol
  (the density sums have positive terms only);
- pressure acceleration and velocities, element by element:
      |A - A_ref|  <= tol |A_ref| + K u S_a
      |v' - v'_ref| <= tol (|v'_ref| + |v|) + K u tau (S_a + S_cell)
  where S_a is the magnitude sum of particle a's pair terms (reported by the
  oracle), S_cell its mean over the cell's gas, u the unit roundoff of the
  path (2^-24 or 2^-53) and K = 48 (parity.KAPPA_STEP; the conditioning test
  below keeps K = 128). The pressure force of a nearly uniform
  state is a small residual of large pair terms; rounding each term in the
  path's precision bounds its accuracy by u S_a, whatever the order of the sum.
"""
import math

import numpy as np
import pytest

import workloads
from conftest import gpu_context, gpu_lib, gpu_one_step, normwise, oracle_params
from parity import KAPPA, TOL, UNIT, check_neighbour_sets, check_one_step, oracle_step

pytestmark = pytest.mark.gpu


def _compare(orc, w, tol=None, normwise_v=None, **over):
    prec = int(over.get("precision", w.params["precision"]))
    gpu = gpu_one_step(w, **over)
    r = orc.step(oracle_params(w), orc.make_state(oracle_params(w), w.gx, w.gv, w.dx, w.du, w.tstop, ge=w.ge,
                                                  frozen=w.frozen), w.tau, w.g)
    # --- bit-exact integer results ---
    assert np.array_equal(gpu["perm_g"], r.perm_g), "gas sort order"
    assert np.array_equal(gpu["perm_d"], r.perm_d), "dust sort order"
    assert np.array_equal(gpu["keys_g"], r.keys_g[r.perm_g]), "gas cell keys"
    assert np.array_equal(gpu["keys_d"], r.keys_d[r.perm_d]), "dust cell keys"
    assert np.array_equal(gpu["cstart_g"], r.cstart_g), "gas cell ranges"
    assert np.array_equal(gpu["cstart_d"], r.cstart_d), "dust cell ranges"
    inv = np.empty_like(r.perm_g)
    inv[r.perm_g] = np.arange(len(r.perm_g))
    band = check_neighbour_sets(gpu["nb_count"][inv], gpu["nb_fprint"][inv], r)
    # --- floating point after one step ---
    r, errs = check_one_step(orc, w, gpu, prec, tol=tol, normwise_v=normwise_v)
    errs.update(band)
    print(f"{w.name}: {errs}")
    return gpu, r, errs


# ---------------------------------------------------------------------------
# Workloads at sizes the oracle finishes in seconds (several tiles, ragged tails)
# ---------------------------------------------------------------------------
def test_dustywave_fp64_one_step(orc):
    _compare(orc, workloads.dustywave(precision=1))


def test_dustywave_fp32_one_step(orc):
    _compare(orc, workloads.dustywave(n=1000, precision=0))


@pytest.mark.parametrize("cell_acc", [0, 1])
def test_dustyshock_fp32_one_step(orc, cell_acc):
    w = workloads.dustyshock(n_left=4000, n_right=500, precision=0)
    _compare(orc, w, cell_acc=cell_acc)


def test_dustyshock_fp64_one_step(orc):
    w = workloads.dustyshock(n_left=1600, n_right=200, precision=1)
    _compare(orc, w)


@pytest.mark.parametrize("nside", [12, 23])
def test_box3d_fp32_one_step(orc, nside):
    _compare(orc, workloads.box3d(nside=nside, precision=0))


def test_box3d_fp64_one_step(orc):
    _compare(orc, workloads.box3d(nside=10, precision=1))


def test_column2d_fp32_one_step(orc):
    _compare(orc, workloads.column2d(nside=64, precision=0))


def test_column2d_fp64_one_step(orc):
    _compare(orc, workloads.column2d(nside=32, precision=1))


def test_harmonic_tstar_fp64(orc):
    w = workloads.dustyshock(n_left=800, n_right=100, precision=1)
    w.params["tstar_mode"] = 1
    _compare(orc, w)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_no_dust(orc):
    w = workloads.dustyshock(n_left=800, n_right=100, with_dust=False, precision=1)
    _compare(orc, w)


def test_no_gas(orc):
    w = workloads.dustywave(n=50, precision=1)
    w.gx, w.gv = w.gx[:, :0], w.gv[:, :0]
    gpu = gpu_one_step(w)
    p, s, r, _ = oracle_step(orc, w)
    np.testing.assert_allclose(gpu["du"], s.du, rtol=1e-14, atol=1e-300)
    assert np.array_equal(gpu["cstart_d"], r.cstart_d)


def test_single_particles(orc):
    w = workloads.dustywave(n=1, precision=1)
    w.params["h"] = 0.2
    w.params["cell_size"] = 0.3
    _compare(orc, w)


def test_all_particles_in_one_cell(orc):
    """A cluster far denser than the rest: large segments in the rank sort."""
    rng = np.random.default_rng(17)
    w = workloads.box3d(nside=8, precision=0)
    w.gx[:, :300] = 0.5 + rng.uniform(0, 0.01, (3, 300))
    w.dx[:, :200] = 0.5 + rng.uniform(0, 0.01, (3, 200))
    w.gx = w.gx.astype(np.float32).astype(np.float64)
    w.dx = w.dx.astype(np.float32).astype(np.float64)
    _compare(orc, w)


def test_tile_overflowing_shared_memory(orc):
    """A cluster of 3000 gas particles in one cell of a 16^3 box: the tiles
    whose halo holds it do not fit shared memory and take the global-memory
    walk (density, force and the neighbour statistics)."""
    rng = np.random.default_rng(23)
    w = workloads.box3d(nside=16, precision=0)
    w.gx[:, :3000] = 0.5 + rng.uniform(0, 0.01, (3, 3000))
    w.gx = w.gx.astype(np.float32).astype(np.float64)
    _compare(orc, w)


def test_particles_on_cell_faces(orc):
    """Positions exactly on cell faces and on the periodic boundary."""
    w = workloads.box3d(nside=8, precision=0)
    w.gx[:, ::7] = np.round(w.gx[:, ::7] * 8) / 8
    w.dx[:, ::5] = np.round(w.dx[:, ::5] * 8) / 8 % 1.0
    _compare(orc, w)


def test_full_periodic_window(orc):
    """Fewer cells than the search window along every periodic axis."""
    w = workloads.box3d(nside=6, precision=1, h_factor=1.2, cell_factor=1.0)
    _compare(orc, w)


@pytest.mark.parametrize("tau_over_t", [1e-3, 1.0, 1e3, 1e6])
def test_stiff_drag_limits(orc, tau_over_t):
    """FP64 dusty wave from weak to stiff drag, every output against the
    oracle, velocities normwise at 1e-12. Amplitude 1e-3: the pressure force
    is then resolved by binary64 (see the low-amplitude test below)."""
    w = workloads.dustywave(n=200, amp=1e-3, precision=1)
    w.tstop[:] = w.tau / tau_over_t
    _compare(orc, w)


def test_dustywave_fp64_pressure_force_at_its_conditioning(orc):
    """At amplitude 1e-4 and weak drag the velocity change of a step is the
    pressure force, a residual about 1e-7 of its own pair terms: two binary64
    evaluations of it that round the terms in different orders differ by
    about u S_a (S_a the magnitude sum of the terms), and the oracle's own
    error is of the same size. Normwise, the velocities then agree to
    tol + K u tau ||S|| / ||v'|| (K = 128), the normwise form of the
    element-wise bound, and not to 1e-12 alone (measured: 2.9e-12)."""
    w = workloads.dustywave(n=200, precision=1)
    w.tstop[:] = w.tau / 1e-3
    gpu = gpu_one_step(w)
    p, s, r, _ = oracle_step(orc, w)
    err = normwise(gpu["gv"], s.gv)
    bound = TOL[1] + KAPPA * UNIT[1] * w.tau * np.linalg.norm(r.acc_scale_g) / np.linalg.norm(s.gv)
    print(f"dusty wave 1e-4, weak drag: normwise gas velocity error {err:.3e}, bound {bound:.3e}")
    assert err <= bound


@pytest.mark.parametrize("cell_acc", [1, 0])
def test_fp32_path_terminal_slip_at_tau_over_tstop_1e6(orc, cell_acc):
    """FP32 path, t_stop = tau / 1e6, on the settling column (gas held by its
    pressure against gravity, dust sinking through it; Sec. 2.3's
    asymptotic-preserving limit): one step against the oracle, and per drag
    cell the new slip u*' - v*' along g, read from the GPU's FP32 particle
    velocities, against the implicit cell solve evaluated in binary64 from the
    step's inputs and the GPU's own pressure force,
    -(w + tau Abar) / (1 + tau (1 + eps*)/t*), and against the oracle's own
    slip. The slip (~6e-9) is read from velocities up to ~1e-2, so each cell
    is allowed 1e-2 of its slip plus the FP32 resolution of its two mean
    velocities. The limit of the solve, t* (-Abar)/(1 + eps*), is g t* up
    to the column's force balance (the SPH pressure force exceeds gravity by
    8 % at this resolution). The new slip is solved first and the means
    follow from it, so FP32 cell sums keep the limit too; the FP64 cell sums
    change the common mixture velocity, not the slip."""
    w = workloads.column2d(nside=64, precision=0, nsteps=1)
    w.tstop[:] = np.float32(w.tau / 1e6)
    gpu, r, errs = _compare(orc, w, cell_acc=cell_acc)
    p = oracle_params(w)
    _, s_or, r_or, _ = oracle_step(orc, w)
    ncells = len(r.cstart_g) - 1
    moving = w.frozen == 0
    kg, kd = r.keys_g[moving], r.keys_d
    N = np.bincount(kg, minlength=ncells).astype(np.float64)
    L = np.bincount(kd, minlength=ncells).astype(np.float64)
    drag = (N > 0) & (L > 0)
    mean = lambda v, k, cnt: np.bincount(k, weights=v, minlength=ncells) / np.maximum(cnt, 1)
    eps = p.m_dust * L / (p.m_gas * np.maximum(N, 1))
    tst = mean(w.tstop, kd, L)
    ax = 1
    w0 = mean(w.gv[ax, moving], kg, N) - mean(w.du[ax], kd, L)
    abar = mean(gpu["acc_g"][ax, moving], kg, N)
    ref = -(w0 + w.tau * abar) / (1.0 + w.tau * (1.0 + eps) / np.maximum(tst, 1e-300))
    vbar = mean(gpu["gv"][ax, moving], kg, N)
    ubar = mean(gpu["du"][ax], kd, L)
    slip = ubar - vbar
    oslip = mean(s_or.du[ax], kd, L) - mean(s_or.gv[ax, moving], kg, N)
    res = np.spacing(np.abs(vbar).astype(np.float32)).astype(np.float64) + \
        np.spacing(np.abs(ubar).astype(np.float32)).astype(np.float64)
    for name, want in (("cell solve", ref), ("oracle", oslip)):
        excess = (np.abs(slip - want) / (1e-2 * np.abs(want) + 4.0 * res))[drag]
        print(f"terminal slip, cell_acc={cell_acc}, vs {name}: median relative error "
              f"{np.median(np.abs(slip - want)[drag] / np.abs(want[drag])):.3e}, max error / bound {excess.max():.3f}")
        assert excess.max() <= 1.0
    lim = tst * (-abar) / (1.0 + eps)
    assert np.median(np.abs(ref - lim)[drag] / np.abs(lim[drag])) < 1e-2
    ratio = float(np.median(ref[drag] / (w.g[1] * tst[drag])))
    print(f"terminal slip / (g t*): {ratio:.4f}")
    assert ratio == pytest.approx(1.0, rel=0.15)


# ---------------------------------------------------------------------------
# Other entry points
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_max_dt_matches_oracle(orc, prec):
    w = workloads.dustyshock(n_left=800, n_right=100, precision=prec)
    p = oracle_params(w)
    ref = orc.max_dt(p, w.gv, w.ge, w.frozen, cfl=0.3)
    with gpu_context(w) as c:
        got = c.max_dt(0.3)
    assert abs(got - ref) <= (1e-6 if prec == 0 else 1e-14) * ref


def test_tstop_argument_replaces_resident_values(orc):
    b = gpu_lib()
    w = workloads.dustyshock(n_left=800, n_right=100, precision=1)
    new_t = np.random.default_rng(3).uniform(1e-4, 1e-2, w.n_dust)
    w2 = workloads.dustyshock(n_left=800, n_right=100, precision=1)
    w2.tstop = new_t.copy()
    with gpu_context(w) as c:
        c.step(w.tau, w.g, tstop=new_t)
        gv = c.field(b.TFSPH_FIELD_VEL_G)
        ts = c.field(b.TFSPH_FIELD_TSTOP_D)
    _, s, _, _ = oracle_step(orc, w2)
    assert np.array_equal(ts, new_t)
    assert normwise(gv, s.gv) < 1e-12


def test_bad_tstop_is_reported(orc):
    b = gpu_lib()
    w = workloads.dustywave(n=50, precision=1)
    with gpu_context(w) as c:
        bad = np.full(w.n_dust, 1e-3)
        bad[7] = np.nan
        with pytest.raises(b.TfsphError) as ei:
            c.step(w.tau, w.g, tstop=bad)
        assert ei.value.code == b.TFSPH_E_NONFINITE
        c.step(w.tau, w.g)  # the context stays usable
        c.sync()


def test_device_inputs_match_host_inputs(orc):
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    w = workloads.box3d(nside=10, precision=0)
    ref = gpu_one_step(w)
    p = b.params_from_dict(w.params)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    with b.Context(p, t(w.gx), t(w.gv), t(w.dx), t(w.du), t(w.tstop)) as c:
        c.set_stream(torch.cuda.current_stream())
        c.step(w.tau, w.g)
        out = torch.zeros((3, w.n_gas), dtype=torch.float32, device="cuda")
        c.field(b.TFSPH_FIELD_VEL_G, out=out)
        torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.float64), ref["gv"])


def test_steps_are_deterministic():
    w = workloads.box3d(nside=12, precision=0)
    b = gpu_lib()
    res = []
    for _ in range(2):
        with gpu_context(w) as c:
            for _ in range(3):
                c.step(w.tau, w.g)
            res.append((c.field(b.TFSPH_FIELD_VEL_G), c.field(b.TFSPH_FIELD_POS_D)))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_set_state_restarts_the_run(orc):
    b = gpu_lib()
    w = workloads.dustywave(n=100, precision=1)
    with gpu_context(w) as c:
        c.step(w.tau, w.g)
        c.step(w.tau, w.g)
        c.set_state(w.gx, w.gv, w.dx, w.du, w.tstop)
        assert c.info().steps == 0
        c.step(w.tau, w.g)
        gv = c.field(b.TFSPH_FIELD_VEL_G)
    _, s, _, _ = oracle_step(orc, w)
    assert normwise(gv, s.gv) < 1e-12


def test_dustywave_fp64_200_steps(orc):
    """The full Dustywave run (100 + 100 particles, 200 steps, FP64) stays on
    the oracle's trajectory."""
    b = gpu_lib()
    w = workloads.dustywave(precision=1)
    p = oracle_params(w)
    s = orc.make_state(p, w.gx, w.gv, w.dx, w.du, w.tstop)
    with gpu_context(w) as c:
        for _ in range(w.nsteps):
            c.step(w.tau, w.g)
            orc.step(p, s, w.tau, w.g)
        gv = c.field(b.TFSPH_FIELD_VEL_G)
        du = c.field(b.TFSPH_FIELD_VEL_D)
    assert normwise(gv, s.gv) < 1e-9 and normwise(du, s.du) < 1e-9


# ---------------------------------------------------------------------------
# Full-size workloads, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cell_acc", [0, 1])
def test_box3d_full_size_one_step(orc, cell_acc):
    """3D box, 128^3 gas + 128^3 dust, with FP32 cell sums (cell_acc 0: the
    benchmarked form) and FP64 cell sums: every output against the oracle,
    velocities also normwise at 1e-5."""
    _compare(orc, workloads.box3d(nside=128, precision=0), normwise_v=True, cell_acc=cell_acc)


def test_box3d_192_one_step(orc):
    """3D box at 3.4x the benchmark's size, 192^3 gas + 192^3 dust (14.2M
    particles, 7.1M cells, 32,768 tiles), FP32 cell sums: every output against
    the oracle, so the index and offset arithmetic is checked beyond the
    benchmark's range."""
    _compare(orc, workloads.box3d(nside=192, precision=0), normwise_v=True, cell_acc=0)


@pytest.mark.parametrize("cell_acc", [0, 1])
def test_dustyshock_full_size_one_step(orc, cell_acc):
    _compare(orc, workloads.dustyshock(precision=0), cell_acc=cell_acc)


@pytest.mark.parametrize("cell_acc", [0, 1])
def test_column2d_full_size_one_step(orc, cell_acc):
    _compare(orc, workloads.column2d(nside=512, precision=0), cell_acc=cell_acc)


def test_save_and_load_state_resume_bit_for_bit(orc):
    """A snapshot taken mid-run and loaded back resumes the run exactly."""
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    w = workloads.column2d(nside=24, precision=0)
    with gpu_context(w) as c:
        for _ in range(3):
            c.step(w.tau, w.g)
        snap = c.save_state()
        host = c.save_state(np.zeros(c.state_bytes(), np.uint8))
        for _ in range(4):
            c.step(w.tau, w.g)
        ref = c.field(b.TFSPH_FIELD_VEL_D)
        c.load_state(snap)
        assert c.info().steps == 7          # a device load keeps the step count
        for _ in range(4):
            c.step(w.tau, w.g)
        again = c.field(b.TFSPH_FIELD_VEL_D)
        c.load_state(host)
        assert c.info().steps == 3          # a host load restores it
        for _ in range(4):
            c.step(w.tau, w.g)
        again_host = c.field(b.TFSPH_FIELD_VEL_D)
    assert np.array_equal(ref, again) and np.array_equal(ref, again_host)
    # a snapshot of another shape is refused (host: at once; device: at the next sync)
    w2 = workloads.column2d(nside=16, precision=0)
    with gpu_context(w2) as c2:
        with pytest.raises(b.TfsphError):
            c2.load_state(host)
        c2.sync()
        c2.load_state(snap[: c2.state_bytes()])
        with pytest.raises(b.TfsphError):
            c2.sync()


def test_step_adjoint_after_load_reuses_forward_quantities(orc):
    """The adjoint of a step started from a loaded snapshot (which carries the
    state's binning, density and pressure acceleration) equals the adjoint
    computed from the plain state, bit for bit."""
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    w = workloads.column2d(nside=24, precision=0)
    with gpu_context(w) as c:
        for _ in range(2):
            c.step(w.tau, w.g)
        snap = c.save_state()
        gen = torch.Generator(device="cpu").manual_seed(5)
        lam0 = [torch.randn(c.dim, c.n_gas, generator=gen), torch.randn(c.dim, c.n_gas, generator=gen),
                torch.randn(c.dim, c.n_dust, generator=gen), torch.randn(c.dim, c.n_dust, generator=gen)]
        outs = []
        for use_snapshot in (False, True):
            if use_snapshot:
                c.load_state(snap)
            else:
                # the same state without its forward quantities
                st = (c.field(b.TFSPH_FIELD_POS_G), c.field(b.TFSPH_FIELD_VEL_G), c.field(b.TFSPH_FIELD_POS_D),
                      c.field(b.TFSPH_FIELD_VEL_D), c.field(b.TFSPH_FIELD_TSTOP_D))
                c.set_state(*st, frozen=w.frozen)
            lam = [t.clone().cuda() for t in lam0]
            lts = torch.zeros(c.n_dust, dtype=torch.float32, device="cuda")
            c.step_adjoint(w.tau, w.g, lam[0], lam[1], lam[2], lam[3], lts)
            outs.append([t.cpu().numpy() for t in lam + [lts]])
    for a, r in zip(outs[1], outs[0]):
        assert np.array_equal(a, r)


def test_page_locked_host_buffers_match_pageable(orc):
    """set_state and fields with page-locked host buffers (read by the kernels
    in place; cell-order fields written in place, id-order fields through the
    staging buffer) give exactly what pageable buffers (staged) give."""
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    w = workloads.column2d(nside=20, precision=0)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = a
        return t

    fz = torch.empty(w.frozen.shape, dtype=torch.uint8, pin_memory=True)
    fz.numpy()[...] = w.frozen
    keep = [pinned(a) for a in (w.gx, w.gv, w.dx, w.du, w.tstop)]
    outs = {}
    for mode in ("pageable", "pinned"):
        with gpu_context(w) as c:
            if mode == "pinned":
                c.set_state(*[t.numpy() for t in keep], frozen=fz.numpy())
            else:
                c.set_state(*[np.ascontiguousarray(a, np.float32) for a in (w.gx, w.gv, w.dx, w.du, w.tstop)],
                            frozen=w.frozen)
            c.step(w.tau, w.g)
            res = []
            for f in (b.TFSPH_FIELD_POS_G, b.TFSPH_FIELD_VEL_G, b.TFSPH_FIELD_POS_D, b.TFSPH_FIELD_VEL_D,
                      b.TFSPH_FIELD_RHO_G):
                n = w.n_gas if f in (b.TFSPH_FIELD_POS_G, b.TFSPH_FIELD_VEL_G, b.TFSPH_FIELD_RHO_G) else w.n_dust
                shape = (n,) if f == b.TFSPH_FIELD_RHO_G else (w.dim, n)
                for order in (b.TFSPH_ORDER_ORIGINAL, b.TFSPH_ORDER_CELL):
                    if mode == "pinned":
                        t = torch.empty(shape, dtype=torch.float32, pin_memory=True)
                        c.field(f, order=order, out=t.numpy())
                        res.append(t.numpy().copy())
                    else:
                        res.append(c.field(f, order=order))
            outs[mode] = res
    for a, r in zip(outs["pinned"], outs["pageable"]):
        assert np.array_equal(a, r)
