"""Reverse-mode rollouts of the SPH-IDIC step with step checkpointing.

``Rollout`` runs ``nsteps`` steps on a context, keeping the state every
``checkpoint_every`` steps. Its backward recomputes one segment at a time
from its checkpoint (keeping the segment's per-step states) and applies the
library's hand-written step adjoint (``tfsph_step_adjoint``) in reverse,
so memory grows with the checkpoint interval, not with the rollout length.
A snapshot carries its state's binning, density and pressure acceleration,
so each step's force is evaluated once in the recompute and reused by the
adjoint after the snapshot is loaded.

``TFSPHRollout`` wraps it in a ``torch.autograd.Function``: gradients of any
loss on the final state with respect to the per-particle stopping times and
the initial gas and dust velocities. ``DustProfileLoss`` is such a loss: the
squared error of the binned (cloud-in-cell) dust density against a target
profile, evaluated with its gradient by ``tfsph_dust_profile``. All work is
done by the CUDA library; torch provides device tensors.
"""
from __future__ import annotations

import torch

from . import binding as b


class Rollout:
    def __init__(self, ctx: "b.Context", tau: float, g=(0.0, 0.0, 0.0), nsteps: int = 1,
                 checkpoint_every: int = 50, frozen=None):
        self.ctx = ctx
        self.tau = float(tau)
        self.g = tuple(g)
        self.nsteps = int(nsteps)
        self.every = max(1, int(checkpoint_every))
        self.dim = ctx.dim
        self.dtype = torch.float64 if ctx.params.precision == b.TFSPH_FP64 else torch.float32
        self.frozen = None if frozen is None else torch.as_tensor(frozen, dtype=torch.uint8, device="cuda")
        self.checkpoints = []   # device snapshots (tfsph_save_state) every `every` steps
        self.inputs = None      # the initial state as given
        self._segment = []      # snapshot buffers reused by the backward's recompute

    # state = (gx, gv, dx, du, tstop), device tensors in id order
    def export(self):
        c, d = self.ctx, self.dim
        z = lambda *s: torch.empty(s, dtype=self.dtype, device="cuda")
        gx, gv = z(d, c.n_gas), z(d, c.n_gas)
        dx, du, ts = z(d, c.n_dust), z(d, c.n_dust), z(c.n_dust)
        c.field(b.TFSPH_FIELD_POS_G, out=gx)
        c.field(b.TFSPH_FIELD_VEL_G, out=gv)
        c.field(b.TFSPH_FIELD_POS_D, out=dx)
        c.field(b.TFSPH_FIELD_VEL_D, out=du)
        c.field(b.TFSPH_FIELD_TSTOP_D, out=ts)
        return gx, gv, dx, du, ts

    def restore(self, st):
        gx, gv, dx, du, ts = st
        self.ctx.set_state(gx, gv, dx, du, ts, frozen=self.frozen)

    def forward(self, state0):
        self.inputs = tuple(t.detach().clone() for t in state0)
        self.restore(self.inputs)
        self.checkpoints = [self.ctx.save_state()]
        for i in range(self.nsteps):
            self.ctx.step(self.tau, self.g)
            if (i + 1) % self.every == 0 and i + 1 < self.nsteps:
                self.checkpoints.append(self.ctx.save_state())
        return self.export()

    def backward(self, lam_gx, lam_gv, lam_dx, lam_du):
        """Adjoints of the final state -> adjoints of the initial state and of t_stop."""
        lam = [t.detach().clone().contiguous() for t in (lam_gx, lam_gv, lam_dx, lam_du)]
        lam_ts = torch.zeros(self.ctx.n_dust, dtype=self.dtype, device="cuda")
        while len(self._segment) < self.every:
            self._segment.append(self.ctx.save_state())
        nseg = (self.nsteps + self.every - 1) // self.every
        for seg in reversed(range(nseg)):
            start = seg * self.every
            end = min(self.nsteps, start + self.every)
            self.ctx.load_state(self.checkpoints[seg])
            # recompute the segment's step-start states; the last step's
            # output is not needed, so the context ends at the last start state
            for i in range(end - start - 1):
                self.ctx.save_state(self._segment[i])
                self.ctx.step(self.tau, self.g)
            for i in reversed(range(end - start)):
                if i < end - start - 1:
                    self.ctx.load_state(self._segment[i])
                self.ctx.step_adjoint(self.tau, self.g, lam[0], lam[1], lam[2], lam[3], lam_ts)
        return lam[0], lam[1], lam[2], lam[3], lam_ts


class TFSPHRollout(torch.autograd.Function):
    """Differentiable rollout: (t_stop, gas velocities, dust velocities) ->
    final (gas x, gas v, dust x, dust u). Positions at t = 0 are constants."""

    @staticmethod
    def forward(fctx, tstop, gv0, du0, rollout: Rollout, gx0, dx0):
        out = rollout.forward((gx0, gv0, dx0, du0, tstop))
        fctx.rollout = rollout
        return out[0], out[1], out[2], out[3]

    @staticmethod
    def backward(fctx, lgx, lgv, ldx, ldu):
        r = fctx.rollout
        z = lambda like, t: torch.zeros_like(like) if t is None else t
        ref = r.inputs
        lgx, lgv, ldx, ldu = z(ref[0], lgx), z(ref[1], lgv), z(ref[2], ldx), z(ref[3], ldu)
        l0 = r.backward(lgx, lgv, ldx, ldu)
        return l0[4], l0[1], l0[3], None, None, None


def profile_grid(ctx: "b.Context", nbins) -> "b.tfsph_grid_spec":
    """Grid spec of a context's box for the dust profile (nbins per axis)."""
    p = ctx.params
    return b.grid_spec(p.dim, list(p.lo), list(p.hi), list(p.periodic), nbins, p.m_dust, p.precision)


def dust_profile(grid: "b.tfsph_grid_spec", dx: torch.Tensor) -> torch.Tensor:
    """Binned dust density (float64, bins with axis 0 fastest) of positions dx (dim, n)."""
    nb = 1
    for k in range(grid.dim):
        nb *= grid.nbins[k]
    rho = torch.empty(nb, dtype=torch.float64, device=dx.device)
    x = dx.detach().contiguous()
    rc = b.tfsph_dust_profile(grid, x.data_ptr(), x.shape[1], None, rho.data_ptr(), None, None,
                              torch.cuda.current_stream().cuda_stream)
    if rc != b.TFSPH_OK:
        raise b.TfsphError(rc, b.tfsph_last_error(None))
    return rho


class DustProfileLoss(torch.autograd.Function):
    """loss = sum_b (rho_b(dx) - target_b)^2 for the binned dust density of
    positions dx (dim, n); the library returns d loss / d dx with the loss."""

    @staticmethod
    def forward(fctx, dx, target, grid):
        x = dx.detach().contiguous()
        t = target.detach().to(torch.float64).contiguous()
        rho = torch.empty_like(t)
        loss = torch.empty(1, dtype=torch.float64, device=x.device)
        lam = torch.empty_like(x)
        rc = b.tfsph_dust_profile(grid, x.data_ptr(), x.shape[1], t.data_ptr(), rho.data_ptr(), loss.data_ptr(),
                                  lam.data_ptr(), torch.cuda.current_stream().cuda_stream)
        if rc != b.TFSPH_OK:
            raise b.TfsphError(rc, b.tfsph_last_error(None))
        fctx.save_for_backward(lam)
        return loss[0]

    @staticmethod
    def backward(fctx, gl):
        (lam,) = fctx.saved_tensors
        return lam * gl.to(lam.dtype), None, None
