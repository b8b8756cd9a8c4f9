"""Gradients of run observables through the hand-written adjoint of the
lattice step (immobile particles), with sqrt(N) checkpointing.

Observables of a run of T steps from f(0) = f^eq(rho^k(0), 0):
  J_drag = (1/T) sum_t (1/n) sum_p sqrt(|F_liq,p(t+1/2)|^2 + eps^2)   (Eq. 22)
  A      = sum_x (1 - phi^2), phi = (rho_A - rho_B)/(rho_A + rho_B) at t = T
Parameters: tau_A, tau_B, G, zeta_A, zeta_B and the initial densities.

Every step of the forward and adjoint runs in the library's kernels (through
the C ABI); this module only schedules them: it stores the populations every
K = ceil(sqrt(T)) steps during the forward run, and for each segment in
reverse re-runs the forward steps with the library recording f(t) and the
link forces of every step on the device (lb_record), then applies
lb_adjoint_step_async backwards with dJ/dF_liq formed on the device
(lb_drag_gradient); the parameter gradients accumulate on the device and are
read once at the end.  ``LBObjective`` wraps this as a
torch.autograd.Function.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbgb


class AdjointRunner:
    """Forward run with checkpoints and its reverse sweep on one LBLattice."""

    def __init__(self, lattice: "lbgb.LBLattice", steps: int, checkpoint_every: int | None = None,
                 eps: float = 1e-12):
        import torch

        self.lat = lattice
        self.steps = int(steps)
        self.K = int(checkpoint_every or max(1, math.ceil(math.sqrt(self.steps))))
        self.eps = eps
        self.torch = torch
        dev = lattice.device
        self.state_bytes = lbgb.lb_state_bytes(lattice.h)
        fb, sb = lbgb.lb_adjoint_bytes(lattice.h)
        self.adj = [torch.empty(fb, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
        self.stack = torch.empty((self.K, self.state_bytes), dtype=torch.uint8, device=dev)
        self.checkpoints = {}
        self.generation = 0  # number of forward runs so far

    def _state(self):
        t = self.torch.empty(self.state_bytes, dtype=self.torch.uint8, device=self.lat.device)
        lbgb.lb_get_state(self.lat.h, t.data_ptr())
        return t

    def forward(self, params: dict, rhoA0, rhoB0, colloids: dict | None):
        """Run T steps; returns (J_drag, A).  ``colloids``: pos, radius (the
        particles are added immobile)."""
        lat, torch = self.lat, self.torch
        self.generation += 1
        lat.set_params(**params)
        lat.init_fields(rhoA0, rhoB0)
        self.n = 0
        if colloids is not None and len(colloids["pos"]):
            pos = np.asarray(colloids["pos"], dtype=np.float64).reshape(-1, 3)
            self.n = pos.shape[0]
            lat.add_colloids(pos, colloids["radius"], np.full(self.n, np.inf))
        n = max(self.n, 1)
        forces = torch.zeros((self.steps, n, 3), dtype=torch.float64, device=lat.device)
        self.fseg = torch.zeros((self.K, n, 3), dtype=torch.float64, device=lat.device)
        self.dJdF = torch.zeros((n, 3), dtype=torch.float64, device=lat.device)
        self.checkpoints = {}
        for start in range(0, self.steps, self.K):
            self.checkpoints[start] = self._state()
            m = min(self.K, self.steps - start)
            if self.n:
                lbgb.lb_record(lat.h, None, forces[start].data_ptr(), m)
            lat.step(m)
        self.checkpoints[self.steps] = self._state()
        J = 0.0
        if self.n:
            F = forces.cpu().numpy()
            J = float(np.mean(np.sqrt(np.sum(F * F, axis=2) + self.eps ** 2)))
        A = lbgb.lb_adjoint_seed(lat.h, 0.0, self.adj[0].data_ptr(), self.scratch.data_ptr())
        return J, A

    def backward(self, gJ: float, gA: float):
        """Gradients of gJ * J_drag + gA * A: (array of 5 parameter gradients
        [tau_A, tau_B, G, zeta_A, zeta_B], array [2, N] for rho^k(0))."""
        lat, torch = self.lat, self.torch
        lbgb.lb_set_state(lat.h, self.checkpoints[self.steps].data_ptr())
        cur, nxt = self.adj
        lbgb.lb_adjoint_seed(lat.h, gA, cur.data_ptr(), self.scratch.data_ptr())
        grads = np.zeros(5)
        T = self.steps
        weight = gJ / (T * self.n) if self.n else 0.0
        for start in reversed(range(0, T, self.K)):
            end = min(start + self.K, T)
            lbgb.lb_set_state(lat.h, self.checkpoints[start].data_ptr())
            lbgb.lb_record(lat.h, self.stack.data_ptr(), self.fseg.data_ptr() if self.n else None, end - start)
            lat.step(end - start)
            for t in reversed(range(start, end)):
                d_dJdF = None
                if self.n and gJ != 0.0:
                    lbgb.lb_drag_gradient(lat.h, self.fseg[t - start].data_ptr(), weight, self.eps,
                                          self.dJdF.data_ptr())
                    d_dJdF = self.dJdF.data_ptr()
                last = start == 0 and t == 0
                lbgb.lb_adjoint_step_async(lat.h, self.stack[t - start].data_ptr(), cur.data_ptr(), nxt.data_ptr(),
                                           self.scratch.data_ptr(), d_dJdF, grads if last else None)
                cur, nxt = nxt, cur
        g = torch.empty((2, lat.N), dtype=torch.float64, device=lat.device)
        lbgb.lb_adjoint_initial(lat.h, cur.data_ptr(), g.data_ptr())
        # leave the lattice in its final state
        lbgb.lb_set_state(lat.h, self.checkpoints[self.steps].data_ptr())
        return grads, g.cpu().numpy()


def _objective_function():
    import torch

    class LBObjective(torch.autograd.Function):
        """(theta, rhoA0, rhoB0) -> [J_drag, A]; theta = (tau_A, tau_B, G,
        zeta_A, zeta_B) as a float64 tensor.  Non-tensor inputs: the
        AdjointRunner, the remaining parameters and the particles."""

        @staticmethod
        def forward(ctx, theta, rhoA0, rhoB0, runner, base_params, colloids):
            t = [float(v) for v in theta.detach().cpu().tolist()]
            params = dict(base_params, tau=(t[0], t[1]), G=t[2], zeta=(t[3], t[4]))
            J, A = runner.forward(params, rhoA0.detach().cpu().numpy(), rhoB0.detach().cpu().numpy(), colloids)
            # the runner holds one forward's checkpoints: remember which one
            ctx.runner, ctx.generation = runner, runner.generation
            ctx.like = [(x.device, x.dtype) for x in (theta, rhoA0, rhoB0)]
            return torch.tensor([J, A], dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            if ctx.runner.generation != ctx.generation:
                raise RuntimeError("LBObjective: the AdjointRunner ran another forward since this graph was "
                                   "built, so its checkpoints belong to other inputs; use one runner per "
                                   "graph or call backward before the next forward")
            g = grad_out.detach().cpu()
            grads, grho = ctx.runner.backward(float(g[0]), float(g[1]))
            out = [torch.from_numpy(np.ascontiguousarray(x)) for x in (grads, grho[0], grho[1])]
            out = [x.to(device=d, dtype=t) for x, (d, t) in zip(out, ctx.like)]
            return (*out, None, None, None)

    return LBObjective


def LBObjective():
    """The torch.autograd.Function class (created on first use)."""
    global _CLS
    try:
        return _CLS
    except NameError:
        _CLS = _objective_function()
        return _CLS
