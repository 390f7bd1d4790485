"""Gradients of a receiver misfit through the leapfrog: torch.autograd on top of smx_step_adjoint.

The forward map is nsteps leapfrog steps (smx_step) from a fixed initial
state (d0, b0) with the current J = s_n jhat; the recorded quantities are the
receiver traces R e_n, n = 1..nsteps (smx_receivers_eval).  The reverse sweep
runs smx_step_adjoint step by step; the forward states it needs (d_n and
d_{n+1}) are recomputed segment by segment from sqrt(N) checkpoints of
(d, b, e), so memory holds about 2 sqrt(N) field vectors instead of N.

Only argument marshalling and bookkeeping live here; every operation on the
fields runs in the library's kernels.
"""
import math

import numpy as np
import torch

from . import smx


class LeapfrogProblem:
    """One context with block permittivity and receivers, plus the fixed parts of the run.

    precision "fp64" (default) or "mixed_refined": the forward steps and the reverse steps both in
    that arithmetic (the refined mixed form's reverse step uses its FP32 operators with one FP64
    residual refinement of each transposed Kronecker solve)."""

    def __init__(self, p, nel, eps_blocks, receivers_xhat, d0, b0, jhat, dt, nsteps, geometry="identity",
                 amplitude=0.05, mu=1.0, device="cuda", precision="fp64"):
        eps_blocks = np.asarray(eps_blocks, dtype=np.float64)
        self.ctx = smx.Context(p, nel, geometry=geometry, amplitude=amplitude, eps=("blocks", eps_blocks), mu=mu,
                               precision=precision)
        self.ctx.receivers_set(receivers_xhat)
        self.ctx.bind(device)
        self.eps_shape = eps_blocks.shape
        self.eps_current = eps_blocks.copy()
        self.device = torch.device(device)
        as_dev = lambda v: torch.as_tensor(np.asarray(v, dtype=np.float64)).to(self.device)
        self.d0, self.b0, self.jhat = as_dev(d0), as_dev(b0), as_dev(jhat)
        self.dt, self.nsteps = float(dt), int(nsteps)
        self.nrec = 3 * self.ctx.n_receivers
        self.N_e, self.N_h = self.ctx.N_e, self.ctx.N_h
        self.k = max(1, int(math.ceil(math.sqrt(self.nsteps))))  # checkpoint spacing

    def set_eps(self, eps_blocks):
        eps = np.asarray(eps_blocks, dtype=np.float64).reshape(self.eps_shape)
        if not np.array_equal(eps, self.eps_current):
            self.ctx.set_material_blocks(eps)
            self.eps_current = eps.copy()

    def _zeros(self, n):
        return torch.zeros(n, dtype=torch.float64, device=self.device)

    def _initial(self):
        d, b = self.d0.clone(), self.b0.clone()
        e = self._zeros(self.N_e)
        self.ctx.hodge_star(smx.FIELD_D, d, e)
        return d, b, e, self._zeros(self.N_h)

    def forward(self, amps, checkpoints=None):
        """Receiver traces (nsteps x 3 nr); optionally fills checkpoints {n: (d, b, e)} every k steps."""
        d, b, e, h = self._initial()
        traces = torch.empty(self.nsteps, self.nrec, dtype=torch.float64, device=self.device)
        for n in range(self.nsteps):
            if checkpoints is not None and n % self.k == 0:
                checkpoints[n] = (d.clone(), b.clone(), e.clone())
            self.ctx.step(d, b, e, h, self.dt, 1, jhat=self.jhat, amp=amps[n:n + 1])
            self.ctx.receivers_eval(e, traces[n])
        return traces

    def backward(self, amps, checkpoints, gtraces):
        """(dL/deps_blocks, dL/damps) for dL/dtraces = gtraces (nsteps x 3 nr)."""
        N, k = self.nsteps, self.k
        geps = self._zeros(int(np.prod(self.eps_shape)))
        gamp = self._zeros(N)
        ebar = self._zeros(self.N_e)
        # terminal step: dbar_N = S_E^T R^T g_N
        seg = self._segment(amps, checkpoints, (N - 1) // k * k, N)
        self.ctx.receivers_adjoint(gtraces[N - 1], 1.0, ebar)
        dbar = self._zeros(self.N_e)
        self.ctx.adjoint_terminal(seg[N], ebar, dbar, eps_bar=geps)
        bbar = self._zeros(self.N_h)
        for n in range(N - 1, -1, -1):
            if n not in seg:
                s0 = n // k * k
                seg = self._segment(amps, checkpoints, s0, min(s0 + k, N))
            ebar.zero_()
            if n >= 1:
                self.ctx.receivers_adjoint(gtraces[n - 1], 1.0, ebar)
            self.ctx.step_adjoint(seg[n], seg[n + 1], dbar, bbar, self.dt, ebar=ebar if n >= 1 else None,
                                  jhat=self.jhat, amp_bar=gamp[n:n + 1], eps_bar=geps)
        return geps.reshape(self.eps_shape), gamp

    def _segment(self, amps, checkpoints, s0, s1):
        """d_n for n = s0 .. s1, recomputed from the checkpoint at s0."""
        d, b, e = (t.clone() for t in checkpoints[s0])
        h = self._zeros(self.N_h)
        seg = {s0: d.clone()}
        for n in range(s0, s1):
            self.ctx.step(d, b, e, h, self.dt, 1, jhat=self.jhat, amp=amps[n:n + 1])
            seg[n + 1] = d.clone()
        return seg


class LeapfrogTraces(torch.autograd.Function):
    """traces = LeapfrogTraces.apply(eps_blocks, amps, problem): receiver traces of the leapfrog run,
    differentiable in the block permittivity and the source amplitudes (float64 tensors)."""

    @staticmethod
    def forward(ctx, eps_blocks, amps, problem):
        problem.set_eps(eps_blocks.detach().cpu().numpy())
        amps_dev = amps.detach().to(problem.device, torch.float64).contiguous()
        checkpoints = {}
        traces = problem.forward(amps_dev, checkpoints)
        ctx.problem, ctx.amps, ctx.checkpoints = problem, amps_dev, checkpoints
        ctx.eps = eps_blocks.detach().cpu().numpy().copy()
        ctx.eps_device, ctx.amps_device = eps_blocks.device, amps.device
        return traces

    @staticmethod
    def backward(ctx, gtraces):
        problem = ctx.problem
        problem.set_eps(ctx.eps)
        geps, gamp = problem.backward(ctx.amps, ctx.checkpoints, gtraces.contiguous())
        return geps.to(ctx.eps_device), gamp.to(ctx.amps_device), None


def misfit(traces, observed, dt):
    """L = 1/2 dt sum_n |traces_n - observed_n|^2."""
    return 0.5 * dt * torch.sum((traces - observed) ** 2)
