"""Differentiable atomic-transport stage: the gradient of a loss of the final state with respect to
the pair-potential parameters D and r0 (Eq. (3)'s well depth and equilibrium distance; r0 also sets
Eq. (1)'s r0/dx and the density unit n0 = r0^-3), as a torch.autograd.Function.

Loss: L = sum_nodes w(node) n(node)/n0 at the final step + kin * (total kinetic energy, J).
With w = -dx/nx on the rows above the initial surface, the first term is the smooth crater depth
of the transport simulation (the depth measure of the paper's transport section, made
differentiable by using the node density instead of a threshold).

Memory: forward keeps one device checkpoint every `every` steps; backward replays each segment
once, keeping its per-step states, and runs the adjoint kernels over them in reverse order
(two-level checkpoint-recompute: nsteps/every + every states on the device at most).
All arithmetic runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import (Simulation, pic_adjoint_seed, pic_adjoint_step, pic_checkpoint_restore, pic_checkpoint_save,
               pic_checkpoint_size, pic_node_functional)

QE = 1.602176634e-19


def crater_weights(nx: int, nz: int, slab_k: int, dx: float, device="cuda") -> torch.Tensor:
    """Node weights of the smooth crater depth: -dx/nx on the node rows below the initial surface."""
    w = torch.zeros((nz + 1, nx), dtype=torch.float64, device=device)
    w[:slab_k] = -dx / nx
    return w


class TransportRun:
    """A transport simulation with checkpoints for the reverse pass (sort_every must be 0: the
    particle order is the adjoint buffers' index)."""

    def __init__(self, phys: dict, D: float, r0: float, every: int = 20):
        over = dict(D_eV=D / QE, r0=r0, sort_every=0)
        self.sim = Simulation(phys, **over)
        self.every = max(1, int(every))
        self.ck_bytes = pic_checkpoint_size(self.sim.h)
        self.checkpoints = []

    def _buf(self):
        return torch.empty(self.ck_bytes, dtype=torch.uint8, device="cuda")

    def forward(self, nsteps: int, w: torch.Tensor, kin: float) -> float:
        self.nsteps = int(nsteps)
        self.checkpoints = []
        for t0 in range(0, self.nsteps, self.every):
            b = self._buf()
            pic_checkpoint_save(self.sim.h, b.data_ptr())
            self.checkpoints.append(b)
            self.sim.step(min(self.every, self.nsteps - t0))
        return self.loss(w, kin)

    def loss(self, w: torch.Tensor, kin: float) -> float:
        L = pic_node_functional(self.sim.h, w.data_ptr())
        if kin:
            L += kin * self.sim.energy()["kinetic_ion"]
        return L

    def backward(self, w: torch.Tensor, kin: float):
        """dL/dD (1/J) and dL/dr0 (1/m); leaves the context at the initial state."""
        n = self.sim.info()["num_particles"][0]
        lam_pos = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        lam_u = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        lam_nodes = torch.empty(w.numel(), dtype=torch.float64, device="cuda")
        grads = torch.zeros(2, dtype=torch.float64, device="cuda")
        g_r0 = pic_adjoint_seed(self.sim.h, kin, w.data_ptr(), lam_pos.data_ptr(), lam_u.data_ptr(),
                                lam_nodes.data_ptr())
        seg_states = [self._buf() for _ in range(min(self.every, self.nsteps))]
        for si in range(len(self.checkpoints) - 1, -1, -1):
            t0 = si * self.every
            m = min(self.every, self.nsteps - t0)
            pic_checkpoint_restore(self.sim.h, self.checkpoints[si].data_ptr())
            for j in range(m):
                pic_checkpoint_save(self.sim.h, seg_states[j].data_ptr())
                if j + 1 < m:
                    self.sim.step(1)
            for j in range(m - 1, -1, -1):
                pic_checkpoint_restore(self.sim.h, seg_states[j].data_ptr())
                pic_adjoint_step(self.sim.h, lam_pos.data_ptr(), lam_u.data_ptr(), lam_nodes.data_ptr(),
                                 grads.data_ptr())
        torch.cuda.current_stream().synchronize()
        gD, gR = grads.tolist()
        return gD, gR + g_r0

    def close(self):
        self.sim.close()
        self.checkpoints = []


class TransportLoss(torch.autograd.Function):
    """L(D, r0) of a transport run; D (J) and r0 (m) are 0-d float64 tensors."""

    @staticmethod
    def forward(ctx, D, r0, phys, nsteps, w, kin, every):
        run = TransportRun(phys, float(D), float(r0), every)
        L = run.forward(nsteps, w, kin)
        ctx.run, ctx.w, ctx.kin = run, w, kin
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        gD, gR = ctx.run.backward(ctx.w, ctx.kin)
        ctx.run.close()
        g = float(gL)
        return (torch.tensor(g * gD, dtype=torch.float64), torch.tensor(g * gR, dtype=torch.float64),
                None, None, None, None, None)


def transport_loss(D, r0, phys, nsteps, w, kin=0.0, every=20):
    return TransportLoss.apply(D, r0, phys, nsteps, w, kin, every)
