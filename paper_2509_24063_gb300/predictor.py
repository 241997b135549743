"""Learned predictor of the residual codec mode: sample collection, GPU
training and evaluation against the plain difference codec.

The network (8 -> 64 -> 64 -> 3, float32) predicts an agent's next
displacement from its last two displacements, its diameter and the number of
reference records in its cell (see include/tera.h).  Samples are written by
the encoder itself (the same feature code the codec uses), training runs in
the library's own kernels (tera_mlp_train), and the gain is measured as wire
bytes per record against plain XOR differences on the same iterations.
"""
from __future__ import annotations

import math

import torch

from ._lib import MLP_PARAMS, SAMPLE_FLOATS
from .api import Context
from .exchange import AuraExchange

LAYERS = ((0, 8, 64), (512 + 64, 64, 64), (512 + 64 + 4096 + 64, 64, 3))  # (offset, in, out)


def init_params(seed: int = 1, device="cuda") -> torch.Tensor:
    """He-uniform weights, zero biases (random numbers drawn by the caller)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    p = torch.zeros(MLP_PARAMS, dtype=torch.float32)
    for off, fan_in, fan_out in LAYERS:
        bound = math.sqrt(6.0 / fan_in)
        w = (torch.rand(fan_out * fan_in, generator=g, dtype=torch.float32) * 2 - 1) * bound
        if fan_out == 3:
            w *= 0.1  # small output layer: start near the zero prediction
        p[off:off + fan_out * fan_in] = w
    return p.to(device)


def collect(ctx: Context, states, max_agents: int, max_records: int, every: int = 1,
            path: str = "all_pairs") -> torch.Tensor:
    """Run the exchange (histories kept, no residual mode) over `states` and
    return the encoder's training samples of every `every`-th iteration
    (12 floats per reference slot; invalid rows have a zero flag)."""
    ex = AuraExchange(ctx, max_agents, max_records, path=path, predictor=True)
    picks = [t for t in range(2, len(states)) if (t - 2) % every == 0]
    buf = torch.zeros(len(picks) * max_records * SAMPLE_FLOATS, dtype=torch.float32,
                      device=ex.rec.device)
    k = 0
    for t, st in enumerate(states):
        if k < len(picks) and t == picks[k]:
            ex.samples = buf[k * max_records * SAMPLE_FLOATS:(k + 1) * max_records * SAMPLE_FLOATS]
            k += 1
        else:
            ex.samples = None
        ex.step(st)
    ctx.status()
    return buf


def train(ctx: Context, samples: torch.Tensor, params: torch.Tensor, steps: int = 4000,
          batch: int = 8192, lr: float = 0.02, clip: float = 1.0) -> int:
    """SGD with global-norm clipping on the GPU; returns the valid sample count."""
    return ctx.mlp_train(samples, params, steps, batch, lr, clip)


def wire_bytes(ctx: Context, states, max_agents, max_records, params=None, skip: int = 3,
               path: str = "all_pairs"):
    """(wire bytes, records) over states[skip:], with or without the predictor."""
    ex = AuraExchange(ctx, max_agents, max_records, path=path, predictor=params is not None,
                      params=params)
    total = recs = 0
    for t, st in enumerate(states):
        if t == skip:
            ctx.stats(reset=True)
        ex.step(st)
    s = ctx.stats(reset=True)
    ctx.status()
    return s["wire_bytes"], s["records"]
