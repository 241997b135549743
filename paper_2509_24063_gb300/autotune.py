"""Autotuner of the batched codec's schedule (tile/block size and resident
blocks per SM; each block's shared-memory match table takes what its share of
the SM's shared memory allows).

The schedule never changes the bytes produced, only the time.  Candidates are
timed on the real data of one iteration: after partition + pack, the batched
codec is re-run with each candidate (it is idempotent: it reads the packed
messages and both previous references and overwrites only its outputs), with
CUDA events on the launching stream; the fastest is kept and cached on disk
per (GPU, pair count, record count bucket).
"""
from __future__ import annotations

import json
import math
import os

import torch

# (threads per block, blocks per SM, table records (0: what fits), team blocks (0: by load))
CANDIDATES = [(b, c, 0, 0) for b in (128, 256, 512, 1024) for c in (1, 2, 4, 8, 16)
              if b * c <= 2048]


def cache_path() -> str:
    base = os.environ.get("TERA_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "tera_gb300", "autotune.json")
    return base


def _key(ctx, records: int) -> str:
    name = torch.cuda.get_device_name(ctx.device)
    bucket = 0 if records <= 0 else int(round(math.log2(records)))
    return f"{name}|P={ctx.n_pairs}|E~2^{bucket}"


def load_cached(ctx, records: int):
    try:
        with open(cache_path()) as f:
            v = json.load(f).get(_key(ctx, records))
        return tuple(v["tune"]) if v else None
    except Exception:
        return None


def store(ctx, records: int, tune, ms: float, table):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        try:
            with open(path) as f:
                data = json.load(f)
        except Exception:
            data = {}
        data[_key(ctx, records)] = {"tune": list(tune), "ms": ms,
                                    "candidates": {",".join(map(str, k)): v for k, v in table}}
        with open(path + ".tmp", "w") as f:
            json.dump(data, f, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass


def tune_batched(ex, state: dict, reps: int = 2, candidates=None, use_cache: bool = True):
    """Pick the batched-codec schedule for exchange `ex` on this state.

    Runs one eager iteration of `ex` on `state` (advancing it), then times
    every candidate by re-running the codec of that iteration.  Returns
    (tune, {candidate: ms})."""
    ctx = ex.ctx
    stream = torch.cuda.current_stream()
    t = ex.t
    ex.step(state)
    torch.cuda.synchronize()
    records = int(ex.pair_off[ex.slot_of(t)][-1].item())
    if use_cache:
        cached = load_cached(ctx, records)
        if cached is not None:
            ex.tune = cached
            return cached, {}
    args, kw = ex.codec_args(t)
    results = []
    for cand in (candidates or CANDIDATES):
        ctx.codec_batched(*args, **kw, mode=ex.mode, tune=cand, stream=stream)  # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.codec_batched(*args, **kw, mode=ex.mode, tune=cand, stream=stream)
        e1.record(stream)
        e1.synchronize()
        results.append((cand, e0.elapsed_time(e1) / reps))
    ctx.status()
    ctx.stats(reset=True)
    best, ms = min(results, key=lambda kv: kv[1])
    ex.tune = best
    store(ctx, records, best, ms, results)
    return best, dict(results)
