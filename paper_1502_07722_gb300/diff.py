"""Differentiable PIC run: gradients of a loss of the final state with respect to the pair-potential
parameters D and r0 (Eq. (3)'s well depth and equilibrium distance; r0 also sets Eq. (1)'s r0/dx
and the density unit n0 = r0^-3) and the laser peak intensity I0, as a torch.autograd.Function.

Loss: L = sum_nodes w(node) n(node)/n0 of the final ion (atom) density
          + kin * (total kinetic energy of all species, J per metre of y).
With w = -dx * omega_i on the rows below the initial surface (omega normalised over x) the first
term is the smooth crater depth (the paper measures the crater from density maps; the node density
replaces a threshold so that the depth is differentiable). The kinetic term is the energy the
particles absorbed.

Both the plain cycle (ions, electrons, fields, laser) and the atomic-transport stage (neutral
atoms, pair force only) are differentiable; I0 acts only in the plain cycle.

Memory: forward keeps one device checkpoint every `every` steps; backward replays each segment
once, keeping its per-step states, and runs the adjoint kernels over them in reverse order
(two-level checkpoint-recompute: nsteps/every + every states on the device at most).
All arithmetic runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import (PIC_MODE_FULL, Simulation, pic_adjoint_buffers, pic_adjoint_seed, pic_adjoint_step,
               pic_checkpoint_restore, pic_checkpoint_save, pic_checkpoint_size, pic_node_functional)

QE = 1.602176634e-19


def crater_weights(nx: int, nz: int, slab_k: int, dx: float, w0: float = 0.0, device="cuda") -> torch.Tensor:
    """Node weights of the smooth crater depth: -dx * omega_i on the node rows below the initial
    surface; omega is uniform (w0 = 0) or a Gaussian of width w0/2 about the beam axis, normalised."""
    i = torch.arange(nx, dtype=torch.float64)
    if w0 > 0:
        xr = (i + 0.5 - 0.5 * nx) * dx
        om = torch.exp(-2.0 * xr * xr / (0.5 * w0) ** 2)
    else:
        om = torch.ones(nx, dtype=torch.float64)
    om = om / om.sum()
    w = torch.zeros((nz + 1, nx), dtype=torch.float64)
    w[:slab_k] = -dx * om
    return w.to(device)


class DiffRun:
    """A simulation run with checkpoints for the reverse pass. The cell sort is off (the particle
    order is the adjoint buffers' index)."""

    def __init__(self, phys: dict, D: float, r0: float, I0: float | None = None, every: int = 20):
        over = dict(D_eV=D / QE, r0=r0, sort_every=0)
        if I0 is not None:
            over["I0"] = I0
        self.sim = Simulation(phys, **over)
        self.full = self.sim.cfg.mode == PIC_MODE_FULL
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
            e = self.sim.energy()
            L += kin * (e["kinetic_ion"] + e["kinetic_electron"])
        return L

    def _buffers(self, nn):
        info = self.sim.info()
        dev = dict(dtype=torch.float64, device="cuda")
        dev32 = dict(dtype=torch.float32, device="cuda")
        self._keep = []
        b = pic_adjoint_buffers()
        for s in range(self.sim.nspecies):
            n = info["num_particles"][s]
            lp, lu = torch.empty(2 * max(n, 1), **dev32), torch.empty(3 * max(n, 1), **dev32)
            self._keep += [lp, lu]
            b.lam_pos[s], b.lam_u[s] = lp.data_ptr(), lu.data_ptr()
        lam_nodes = torch.empty(nn, **dev32)
        grads = torch.zeros(3, **dev)
        self._keep += [lam_nodes, grads]
        b.lam_nodes, b.grads = lam_nodes.data_ptr(), grads.data_ptr()
        if self.full:
            lF, lj = torch.empty(9 * nn, **dev), torch.empty(3 * nn, **dev32)
            self._keep += [lF, lj]
            b.lam_F, b.lam_j = lF.data_ptr(), lj.data_ptr()
        return b, grads

    def backward(self, w: torch.Tensor, kin: float):
        """(dL/dD (1/J), dL/dr0 (1/m), dL/dI0 (m^2/W)); leaves the context at the initial state."""
        bufs, grads = self._buffers(w.numel())
        g_r0 = pic_adjoint_seed(self.sim.h, kin, w.data_ptr(), bufs)
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
                pic_adjoint_step(self.sim.h, bufs)
        torch.cuda.current_stream().synchronize()
        gD, gR, gI = grads.tolist()
        self._keep = []
        return gD, gR + g_r0, gI

    def close(self):
        self.sim.close()
        self.checkpoints = []


# the transport stage is the same run without fields
TransportRun = DiffRun


class PicLoss(torch.autograd.Function):
    """L(D, r0, I0) of a run; D (J), r0 (m), I0 (W/m^2) are 0-d float64 tensors."""

    @staticmethod
    def forward(ctx, D, r0, I0, phys, nsteps, w, kin, every):
        run = DiffRun(phys, float(D), float(r0), float(I0), every)
        L = run.forward(nsteps, w, kin)
        ctx.run, ctx.w, ctx.kin = run, w, kin
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        gD, gR, gI = ctx.run.backward(ctx.w, ctx.kin)
        ctx.run.close()
        g = float(gL)
        t = lambda v: torch.tensor(g * v, dtype=torch.float64)
        return t(gD), t(gR), t(gI), None, None, None, None, None


def pic_loss(D, r0, I0, phys, nsteps, w, kin=0.0, every=20):
    return PicLoss.apply(D, r0, I0, phys, nsteps, w, kin, every)


def transport_loss(D, r0, phys, nsteps, w, kin=0.0, every=20):
    return PicLoss.apply(D, r0, torch.tensor(float(phys.get("I0", 0.0)), dtype=torch.float64), phys, nsteps, w,
                         kin, every)

