"""torch.autograd.Function for running-DFT losses of a batch of 2D designs.

The forward pass runs the sm_103a leapfrog kernels on a batch context (one scene
per design) in segments; by default it keeps E^{n+1} - E^n over every design
cell in device memory, so the backward pass (fdtd_adjoint_grad) runs only the
transposed layers backwards in time (store=False keeps field checkpoints
instead and recomputes each segment first).  A CUDA design tensor stays on the
device: its coefficients are formed by a kernel.  PyTorch only carries the
tensors: every step runs in libgemfdtd.so.
"""
from __future__ import annotations

import numpy as np

from . import fdtd


class DesignBatch:
    """Scenes that share geometry and differ in their design-region eps_r.

    Each scene needs a source, DFT monitor cells + frequencies and a design
    rectangle (paper_2405_00814_gb300.scenes.adjoint_scenes builds such scenes)."""

    def __init__(self, scenes, *, ckpt_every=100, stream=None, tblock=4, segment=24, warps=8, store=True,
                 edges=False):
        """store: keep the forward pass's design-region history in device memory
        (no recompute in the gradient); False keeps field checkpoints only.
        edges: record the forward for edge_gradient (dL/dw of the 11 weights each
        design cell owns) instead of gradient."""
        self.scenes = scenes
        self.nsteps = scenes[0].nsteps
        self.sim = fdtd.Simulation.batch(scenes, stream=stream)
        self.mon_ids = []
        for k, sc in enumerate(scenes):
            self.sim.select(k)
            self.sim.set_scene_source(sc.source)
            i0, j0, w, h = sc.design
            self.sim.set_design(i0, j0, sc.design_eps)
            self.mon_ids.append(self.sim.add_dft_monitor(sc.monitors, sc.freqs))
        self.sim.set_option("tblock", tblock)
        self.sim.set_option("segment", segment)
        self.sim.set_option("warps", warps)
        self.sim.set_option("adj_store", 2 if edges else int(bool(store)))
        self.sim.set_checkpointing(ckpt_every)
        self.design_shape = (len(scenes), scenes[0].design[3], scenes[0].design[2])

    def forward(self, eps):
        """Run the forward solve for eps [B, h, w] (numpy array or torch tensor; a
        CUDA tensor is read on the device); returns F [B, n_cells, n_freq]."""
        if hasattr(eps, "is_cuda") and eps.is_cuda:
            import torch
            torch.cuda.current_stream(eps.device).synchronize()   # eps is complete before the library reads it
        elif hasattr(eps, "detach"):
            eps = eps.detach().cpu().numpy().astype(np.float64)
        else:
            eps = np.asarray(eps, np.float64)
        for k, sc in enumerate(self.scenes):
            i0, j0, _, _ = sc.design
            self.sim.select(k)
            self.sim.set_design(i0, j0, eps[k])
        self.sim.reset()
        self.sim.step(self.nsteps)
        return np.stack([self.sim.read_dft(m) for m in self.mon_ids])

    def gradient(self, dLdF, out=None):
        """dL/deps_r [B, h, w] for dL/dF (complex, same shape as forward's F)."""
        return self.sim.adjoint_grad([dLdF[k] for k in range(len(self.scenes))], self.design_shape, out=out)

    def edge_gradient(self, dLdF):
        """dL/dw [B, 11, h, w] of the edge classes of fdtd_edge_grad (needs edges=True)."""
        shapes = [(sc.design[3], sc.design[2]) for sc in self.scenes]
        return np.stack(self.sim.edge_grad([dLdF[k] for k in range(len(self.scenes))], shapes))

    def close(self):
        self.sim.close()


def dft_intensity_loss():
    """Returns a torch.autograd.Function computing L = sum |F|^2 per batch."""
    import torch

    class DFTIntensityLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, eps, batch):
            F = batch.forward(eps.detach())   # a CUDA tensor stays on the device
            ctx.batch = batch
            ctx.F = F
            ctx.device = eps.device
            return torch.tensor(float(np.sum(np.abs(F) ** 2)), dtype=torch.float64, device=eps.device)

        @staticmethod
        def backward(ctx, grad_out):
            dLdF = 2.0 * ctx.F * float(grad_out)
            g = torch.empty(ctx.batch.design_shape, dtype=torch.float32, device=ctx.device)
            if g.is_cuda:
                ctx.batch.gradient(dLdF, out=g)
            else:
                g.copy_(torch.from_numpy(ctx.batch.gradient(dLdF)))
            return g.to(torch.float64), None

    return DFTIntensityLoss
