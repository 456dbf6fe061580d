"""Warm-started fitting: the encoder (efunc_encoder_*) is trained on pairs of
(SDF sampled on the 32^3 cell centres, parameter grid fitted from scratch)
and then predicts the starting grid of a new shape's fit, in place of the
N(0, 1e-3) initialisation of the plain fit (Sec. 3.4 fits from scratch and
needs ~20 minutes per shape, Sec. 5).  Both starts are compared by the steps
and seconds the batched fit needs to reach a held-out MAE.

Every step of the computation (sampling aside) runs in the library's
kernels: the batched fit, the encoder's forward and backward, Adam.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import api, synth

R = api.ENC_R   # the encoder's grid


def random_shapes(seed0: int, n: int, prims=(4, 16)):
    """n unions of 4..16 random primitives (seeds seed0 .. seed0 + n - 1)."""
    g = synth.rng(seed0)
    counts = g.integers(prims[0], prims[1] + 1, size=n)
    return [synth.random_union(seed0 + i, n_prims=int(c)) for i, c in enumerate(counts)]


def sdf_grids(shapes, device) -> torch.Tensor:
    """(n, 32^3) SDF samples at the cell centres (the encoder's input)."""
    return torch.stack([synth.sdf_grid_torch(s, R, device).reshape(-1) for s in shapes])


def query_batches(shapes, J: int, seed: int, device, n_batches: int = 2) -> torch.Tensor:
    """n_batches batches of J rows per shape in the batched fit's layout."""
    return torch.cat([synth.sample_batch_torch(s, J, seed=seed + 7919 * b + i, device=device)
                      for b in range(n_batches) for i, s in enumerate(shapes)])


def heldout_rows(shapes, J: int, seed: int, device) -> torch.Tensor:
    """J held-out rows per shape (half uniform, half near the surface)."""
    return query_batches(shapes, J, seed, device, n_batches=1)


def fit_plain(shapes, J: int, steps: int, seed: int, device, lr: float = 1e-3, chunk_shapes: int = 128,
              params0: torch.Tensor | None = None):
    """Plain batched fits of the shapes (R = 32): (n, 32^3 x 13) fitted grids
    and the seconds the fits took (CUDA events)."""
    out, secs = [], 0.0
    for c0 in range(0, len(shapes), chunk_shapes):
        part = shapes[c0:c0 + chunk_shapes]
        b = api.Batch([R] * len(part), [J] * len(part), device=device)
        qo = query_batches(part, J, seed + c0, device)
        if params0 is None:
            p = torch.cat([torch.from_numpy(synth.init_params(R, seed=seed + c0 + i).reshape(-1))
                           for i in range(len(part))]).to(device)
        else:
            p = params0[c0:c0 + len(part)].reshape(-1).clone()
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.fit(p, m, v, qo, steps=steps, n_batches=2, lr=lr, graph=True)
        e1.record()
        torch.cuda.synchronize(device)
        secs += e0.elapsed_time(e1) * 1e-3
        out.append(p.view(len(part), -1))
    return torch.cat(out), secs


def slot_weights(params: torch.Tensor) -> torch.Tensor:
    """1 / variance of every slot over the training grids (so that the
    offsets, scales and values weigh alike in the encoder's loss)."""
    v = params.reshape(-1, 13).var(dim=0)
    return (1.0 / torch.clamp(v, min=1e-8)).to(torch.float32)


def train_encoder(sdf: torch.Tensor, params: torch.Tensor, epochs: int, batch: int, lr: float = 1e-3,
                  seed: int = 0, weights: torch.Tensor | None = None, per_slot: bool = False):
    """Adam on the encoder's MSE over the (sdf, params) pairs, starting from
    `weights` (or a He initialisation); per_slot weighs every slot by 1 / its
    variance (else all slots alike, so the values and slopes, which carry the
    function, dominate).  Returns (weights, per-epoch mean losses, seconds)."""
    device = sdf.device
    n = sdf.shape[0]
    w = (weights if weights is not None else api.encoder_init(seed)).to(device).contiguous()
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    sw = slot_weights(params).to(device) if per_slot else None
    enc = api.Encoder(batch, device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses, step = [], 0
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for _ in range(epochs):
        order = torch.randperm(n, generator=g)
        acc = torch.zeros(1, device=device)
        nb = 0
        for i in range(0, n - batch + 1, batch):
            idx = order[i:i + batch].to(device)
            grad, loss = enc.train_step(w, sdf[idx].contiguous(), params[idx].contiguous(), sw)
            step += 1
            api.efunc_adam_step(w, grad, m, v, step, lr=lr)
            acc += loss
            nb += 1
        losses.append(float(acc.item()) / max(1, nb))
    torch.cuda.synchronize(device)
    enc.status()
    return w, losses, time.perf_counter() - t0


def predict(weights: torch.Tensor, sdf: torch.Tensor, batch: int):
    """Encoder predictions (n, 32^3 x 13) and their seconds (CUDA events)."""
    device = sdf.device
    n = sdf.shape[0]
    enc = api.Encoder(batch, device)
    outs = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(0, n, batch):
        x = sdf[i:i + batch]
        if x.shape[0] < batch:   # the last partial batch, padded
            x = torch.cat([x, x[-1:].expand(batch - x.shape[0], -1)])
        outs.append(enc.forward(weights, x.contiguous())[:min(batch, n - i)])
    e1.record()
    torch.cuda.synchronize(device)
    return torch.cat(outs), e0.elapsed_time(e1) * 1e-3


def fit_curves(shapes, params0: torch.Tensor, J: int, max_steps: int, every: int, seed: int, held: torch.Tensor,
               lr: float = 1e-3):
    """Batched fits of all shapes from params0 (n, 32^3 x 13), the held-out
    MAE of every shape after every `every` steps.  Returns (steps list,
    (points, n) MAE array, seconds per step list)."""
    device = params0.device
    n = len(shapes)
    b = api.Batch([R] * n, [J] * n, device=device)
    bh = api.Batch([R] * n, [held.shape[0] // n] * n, device=device)
    qo = query_batches(shapes, J, seed, device)
    p = params0.reshape(-1).clone()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    steps, maes, secs = [0], [bh.eval(p, held)[:, 1].cpu().numpy()], [0.0]
    done = 0
    while done < max_steps:
        k = min(every, max_steps - done)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.fit(p, m, v, qo, steps=k, n_batches=2, step0=done, lr=lr, graph=True)
        e1.record()
        torch.cuda.synchronize(device)
        done += k
        steps.append(done)
        secs.append(secs[-1] + e0.elapsed_time(e1) * 1e-3)
        maes.append(bh.eval(p, held)[:, 1].cpu().numpy())
    return np.array(steps), np.stack(maes), np.array(secs)


def steps_to(curve_steps, maes, target):
    """First step at which each shape's MAE is <= its target (inf if never)."""
    hit = maes <= target[None, :]
    first = np.where(hit.any(0), hit.argmax(0), -1)
    return np.where(first >= 0, curve_steps[np.maximum(first, 0)], np.inf)
