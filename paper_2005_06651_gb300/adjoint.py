"""Differentiable rollout of many VL2 cycles behind torch.autograd.Function.

The forward pass advances the mesh through the C ABI and keeps the conserved state every k cycles
(k ~ sqrt(N) by default) plus the time steps it used.  The backward pass walks the segments in reverse:
it restores a segment's checkpoint (vl2_set_cons) and replays the segment's cycles with vl2_step_record,
which keeps in one tape per cycle what that cycle's adjoint reads; vl2_step_vjp_recorded then applies the
hand-written adjoint of each cycle from its tape, last cycle first.  The forward pass records the last
segment itself, so the backward pass starts without a replay.  Each cycle is thus computed once more
in the backward pass, not twice.  (With record=False the replay keeps only the states, and vl2_step_vjp
recomputes each cycle's intermediates from its state.)  The adjoint of the initial conserved state is
then taken back to the initial velocity (vl2_prims_vjp).  Time steps are those of the forward pass, held fixed (no derivative through the
CFL condition).  All arithmetic runs in the CUDA library; this module only moves tensors between calls.
"""
from __future__ import annotations

import math

import torch

from . import vl2 as _vl2


class Rollout:
    """N cycles of one mesh from an initial velocity field, with the density, pressure and face field of
    `prob` held fixed; differentiable in the velocity."""

    def __init__(self, prob, nsteps, checkpoint_every=None, device=None, riemann=_vl2.HLLD, record=True):
        self.prob = prob
        self.nsteps = int(nsteps)
        self.k = int(checkpoint_every or max(1, int(round(math.sqrt(self.nsteps)))))
        self.mesh = _vl2.Mesh(prob.nx, prob.mb, prob.xmin, prob.xmax, prob.gamma, bc=prob.bc, riemann=riemann,
                              device=device, adjoint=True)
        dev = self.mesh.device
        self.rho = torch.from_numpy(prob.w[0]).to(dev)
        self.p = torch.from_numpy(prob.w[4]).to(dev)
        self.b = tuple(torch.from_numpy(x).to(dev) for x in (prob.b1, prob.b2, prob.b3))
        self.fixed_dts = None  # set to a list to replay the same steps (finite-difference checks)
        self.dts = []
        self.checkpoints = {}
        self.w0 = None
        self.timing = {}
        self.record = bool(record)
        self.tail_recorded = False
        self.tapes = [self.mesh.new_tape() for _ in range(self.k)] if self.record else []

    def _state(self):
        m = self.mesh
        out = (torch.empty((5,) + m.shape, dtype=torch.float64, device=m.device),
               *[torch.empty(s, dtype=torch.float64, device=m.device) for s in m.face_shapes()])
        m.get_cons(out)
        return out

    def run_forward(self, v):
        m = self.mesh
        w = torch.stack([self.rho, v[0], v[1], v[2], self.p]).contiguous()
        self.w0 = w
        m.set_prims(w, *self.b)
        self.dts, self.checkpoints = [], {}
        # the last segment is recorded on the way (its tapes are the first the backward pass needs)
        last = ((self.nsteps - 1) // self.k) * self.k
        for s in range(self.nsteps):
            if s % self.k == 0:
                self.checkpoints[s] = self._state()
            dt = self.fixed_dts[s] if self.fixed_dts is not None else m.new_dt()
            self.dts.append(dt)
            if self.record and s >= last:
                m.step_record(dt, self.tapes[s - last])
            else:
                m.step(dt)
        self.tail_recorded = self.record
        return self._state()[0]

    def run_backward(self, grad_u):
        m = self.mesh
        lam = (grad_u.contiguous(), *[torch.zeros_like(x) for x in self.b])
        out = tuple(torch.empty_like(x) for x in lam)
        starts = sorted(self.checkpoints)
        for s0 in reversed(starts):
            s1 = min(s0 + self.k, self.nsteps)
            if self.record:
                if s1 == self.nsteps and self.tail_recorded:
                    self.tail_recorded = False  # the forward pass recorded this segment
                else:
                    m.set_cons(*self.checkpoints[s0])
                    for s in range(s0, s1):
                        m.step_record(self.dts[s], self.tapes[s - s0])
                for s in reversed(range(s0, s1)):
                    m.step_vjp_recorded(self.dts[s], self.tapes[s - s0], lam, out)
                    lam, out = out, lam
                continue
            m.set_cons(*self.checkpoints[s0])
            states = []
            for s in range(s0, s1):  # recompute the states before each cycle of the segment
                states.append(self.checkpoints[s0] if s == s0 else self._state())
                if s + 1 < s1:
                    m.step(self.dts[s])
            for s in reversed(range(s0, s1)):
                m.set_cons(*states[s - s0])
                m.step_vjp(self.dts[s], lam, out)
                lam, out = out, lam
        lam_w = m.prims_vjp(self.w0, lam[0])
        return lam_w[1:4].contiguous()


class _RolloutFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, runner):
        ctx.runner = runner
        return runner.run_forward(v.detach())

    @staticmethod
    def backward(ctx, grad_u):
        return ctx.runner.run_backward(grad_u), None


def rollout(v, runner):
    """Final conserved state [5][NZ][NY][NX] after runner.nsteps cycles from initial velocity v [3][NZ][NY][NX]."""
    return _RolloutFn.apply(v, runner)
