"""Training data and training loop for the learned warm start (OTM_WS_LEARNED).

Pairs are (filtered density, zero-mean solutions of the three load cases)
snapshots taken after design iterations, held in a rolling device buffer; the
network learns y = chi / scale with the library's Adam step.  Everything
numeric runs in libotm's kernels; this module only schedules calls and owns
the buffers (torch device tensors).

  buf = PairBuffer(n=128, capacity=256)
  collect(params, rho0, iters=40, buf=buf)          # one design history
  u = otm.otm_unet_create(128, (16, 32, 64, 128), seed=0)
  scale = target_scale(buf)
  train(u, buf, steps=500, lr=1e-3, scale=scale)
  otm.otm_set_predictor(ctx, u, scale)
"""
from __future__ import annotations

import numpy as np

from . import otm


class PairBuffer:
    """Rolling device buffer of (rho_f [n^3], chi [3 n^3]) FP32 pairs."""

    def __init__(self, n: int, capacity: int, device: str = "cuda"):
        import torch
        self.n, self.N, self.capacity = n, n ** 3, capacity
        self.x = torch.empty((capacity, self.N), dtype=torch.float32, device=device)
        self.t = torch.empty((capacity, 3 * self.N), dtype=torch.float32, device=device)
        self.count = 0
        self.head = 0

    def add_from(self, ctx) -> int:
        """Store the context's current filtered density and solutions."""
        i = self.head
        otm.otm_get_field(ctx, otm.OTM_FIELD_RHO_FILT, self.x[i].data_ptr(), self.N, 1)
        otm.otm_get_field(ctx, otm.OTM_FIELD_CHI, self.t[i].data_ptr(), 3 * self.N, 1)
        self.head = (self.head + 1) % self.capacity
        self.count = min(self.count + 1, self.capacity)
        return i


def collect(params, rho0: np.ndarray, iters: int, buf: PairBuffer, every: int = 1):
    """Run `iters` design iterations from rho0 (host FP32, n^3) and store a
    pair after every `every`-th one.  Returns the per-iteration reports."""
    ctx = otm.otm_create_ex(params)
    infos = []
    try:
        r0 = np.ascontiguousarray(rho0, dtype=np.float32)
        otm.otm_set_density(ctx, r0.ctypes.data, 0)
        for it in range(iters):
            info, _ = otm.otm_step(ctx)
            infos.append(info.as_dict())
            if (it + 1) % every == 0:
                buf.add_from(ctx)
    finally:
        otm.otm_destroy(ctx)
    return infos


def target_scale(buf: PairBuffer, sample: int = 8) -> float:
    """Root mean square of the stored solutions over up to `sample` pairs
    (host copies): the scale that gives the network unit-variance targets."""
    idx = np.linspace(0, buf.count - 1, min(sample, buf.count)).astype(int)
    ms = [float(np.mean(buf.t[i].cpu().numpy().astype(np.float64) ** 2)) for i in idx]
    return float(np.sqrt(np.mean(ms))) if ms and np.mean(ms) > 0 else 1.0


def train(u, buf: PairBuffer, steps: int, lr: float, scale: float, seed: int = 0, stream=None):
    """`steps` Adam steps on pairs drawn uniformly from the buffer; returns
    the per-step losses."""
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(steps):
        i = int(rng.integers(buf.count))
        losses.append(otm.otm_unet_train_step(u, buf.x[i].data_ptr(), buf.t[i].data_ptr(), lr, scale, stream))
    return losses


def evaluate(u, buf: PairBuffer, scale: float, stream=None) -> float:
    """Mean loss over the buffer's pairs."""
    tot = 0.0
    for i in range(buf.count):
        tot += otm.otm_unet_eval(u, buf.x[i].data_ptr(), buf.t[i].data_ptr(), scale, stream)
    return tot / max(buf.count, 1)
