"""Learned initial guess: data generation by the solver itself, training, application.

Workflow (the growth direction in which a network proposes u0 and red-black
Gauss-Seidel finishes to the same tolerance):
  1. `make_dataset`: Gaussian-random-field right-hand sides and random linear Dirichlet
     data (synth.learned_guess_sample), solved to a tight tolerance by
     rbgs_solve_batched (one persistent launch); inputs (f, ring mask, ring values) and
     targets (the converged grids) stay on the GPU.
  2. `train`: minibatch Adam steps, each one rbgs_unet_train_step (forward, backward and
     update in the library's kernels).
  3. `initial_guess`: a transfinite interpolation of the boundary data plus the
     network's predicted correction, with the Dirichlet ring restored; for a
     grid finer than the training grid, `initial_guess_coarse` predicts on the training
     resolution (f block-averaged, ring sampled) and interpolates bilinearly.
The solver then runs from that u0 to the requested tolerance, exactly as from u0 = 0.
"""
from __future__ import annotations

import numpy as np
import torch

from . import default_opts, rbgs_solve_batched, RBGS_FP64, RBGS_FP32_REFINE
from .unet import UNet, guess_assemble, guess_coarsen, guess_refine, guess_target, network_input


def grid_size(n: int) -> int:
    return (n + 2 + 7) // 8 * 8


def make_dataset(n: int, streams, tol: float = 1e-12, device="cuda", batch: int = 512, refine: bool = False):
    """(x, target, mask) on the device for problems drawn from `streams` at size n,
    targets solved by rbgs_solve_batched (FP64 sweeps, or FP32 sweeps with FP64
    refinement when `refine`)."""
    import synth
    size = grid_size(n)
    xs, ys = [], []
    streams = list(streams)
    h2 = synth.h_squared(n)
    opts = default_opts(precision=RBGS_FP32_REFINE if refine else RBGS_FP64, check_every=200,
                        inner_sweeps=400)
    for start in range(0, len(streams), batch):
        chunk = streams[start:start + batch]
        probs, outs, rings = [], [], []
        for s in chunk:
            f, u = synth.learned_guess_sample(n, s)
            fd, ud = torch.from_numpy(f).to(device), torch.from_numpy(u).to(device)
            probs.append((n, h2, fd, ud))
            outs.append(torch.empty_like(ud))
            rings.append(ud)
        res = rbgs_solve_batched(probs, tol, outs, opts)
        for (nn, _, fd, ud), sol in zip(probs, outs):
            xs.append(network_input(fd, ud, size))
            # the network learns the correction to the boundary interpolation
            ys.append(guess_target(sol, ud, size))
    x = torch.stack(xs)
    y = torch.stack(ys)
    mask = torch.zeros((size, size), dtype=torch.float32, device=device)
    mask[1:n + 1, 1:n + 1] = 1.0
    return x, y, mask.expand(x.shape[0], size, size).contiguous()


def train(net: UNet, x, y, mask, steps: int, batch: int = 16, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam minibatch training; returns the list of losses."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    nsamp = x.shape[0]
    for it in range(steps):
        idx = torch.randint(0, nsamp, (batch,), generator=g).to(x.device)
        step_lr = lr * (0.5 * (1 + np.cos(np.pi * it / max(steps, 1))))  # cosine decay
        losses.append(net.train_step(x[idx].contiguous(), y[idx].contiguous(), mask[idx].contiguous(), step_lr))
        if log_every and it % log_every == 0:
            print(f"step {it} loss {losses[-1]:.4e}", flush=True)
    return losses


def initial_guess(net: UNet, f: torch.Tensor, u_ring: torch.Tensor) -> torch.Tensor:
    """u0 on the (n+2)^2 grid: boundary interpolation plus the network's correction in the
    interior, the given Dirichlet ring."""
    n = f.shape[0]
    x = network_input(f, u_ring, grid_size(n)).unsqueeze(0)
    return guess_assemble(u_ring, net.forward(x)[0])


def initial_guess_coarse(net: UNet, f: torch.Tensor, u_ring: torch.Tensor, n_coarse: int) -> torch.Tensor:
    """Predict on an n_coarse grid (f averaged, ring sampled) and interpolate bilinearly to
    the fine grid; the fine Dirichlet ring is kept.  (n + 1) must be a multiple of
    (n_coarse + 1) so that coarse nodes coincide with fine nodes."""
    n = f.shape[0]
    if (n + 1) % (n_coarse + 1):
        raise ValueError("(n + 1) must be a multiple of (n_coarse + 1)")
    fc, uc_ring = guess_coarsen(f, u_ring, n_coarse)
    return guess_refine(initial_guess(net, fc, uc_ring), u_ring)
