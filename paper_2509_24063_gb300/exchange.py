"""One aura-exchange iteration over every pair, with the per-pair references
kept on both sides between iterations (paper Sec. 2.3: each sender/receiver
pair stores the same reference and updates it every iteration here).

Paths (all produce the same bytes):
  "per_subdomain"  pack / encode / decode launched once per sending box
  "all_pairs"      pack / encode / decode launched once for all pairs
  "batched"        pack, then encode + decode of all pairs in one persistent
                   launch (tera_codec_batched); capturable in a CUDA graph

Buffers are allocated once for a maximum agent count and record count; the
sender and receiver references are double-buffered (previous / next).

Reference interval K (paper Sec. 2.3: the reference is updated at regular
intervals): the message of iteration 0 and of every K-th iteration after it
becomes the reference of the next K iterations; in between, messages are
encoded (and decoded) against that older reference, and their outputs go to
the other buffer.  K = 1 updates the reference every iteration.
"""
from __future__ import annotations

import torch

from ._lib import MODE_XOR
from .api import Context, PartitionBuffers, ref_schedule

PATHS = ("per_subdomain", "all_pairs", "batched")


class AuraExchange:
    def __init__(self, ctx: Context, max_agents: int, max_records: int, mode: int = MODE_XOR,
                 per_subdomain: bool = False, path: str | None = None, tune=None,
                 predictor: bool = False, params=None, allow_residual: bool = True,
                 ref_interval: int = 1, id_columns: bool = True):
        self.ctx = ctx
        self.mode = mode
        if ref_interval < 1:
            raise ValueError("ref_interval must be >= 1")
        self.K = int(ref_interval)
        self.path = path or ("per_subdomain" if per_subdomain else "all_pairs")
        if self.path not in PATHS:
            raise ValueError(f"path must be one of {PATHS}")
        self.tune = tune
        P = ctx.n_pairs
        dev = torch.device("cuda", ctx.device)
        self.P = P
        self.max_agents = max_agents
        self.max_records = max_records
        ctx.reserve(max_agents, max_records)
        units = max_records + P
        u8 = dict(dtype=torch.uint8, device=dev)
        i64 = dict(dtype=torch.int64, device=dev)
        self.part = PartitionBuffers.allocate(max_agents, P, max_records, dev)
        self.pair_off = [torch.zeros(P + 1, **i64), torch.zeros(P + 1, **i64)]
        self.rec = torch.empty(units * 64, **u8)
        self.ref = [torch.empty(units * 64, **u8), torch.empty(units * 64, **u8)]
        self.recv = [torch.empty(units * 64, **u8), torch.empty(units * 64, **u8)]
        self.recv_off = [torch.zeros(P + 1, **i64), torch.zeros(P + 1, **i64)]
        # id columns of the packed records and of both sender references (the
        # batched codec matches ids from them instead of re-reading records)
        self.id_columns = bool(id_columns) and self.path == "batched" and not (
            predictor or params is not None)
        if self.id_columns:
            self.rec_ids = torch.empty(units, dtype=torch.int64, device=dev)
            self.ref_ids = [torch.empty(units, dtype=torch.int64, device=dev),
                            torch.empty(units, dtype=torch.int64, device=dev)]
        self.wire_cap = 80 * P + 72 * max_records + 64
        self.wire = torch.empty(self.wire_cap, **u8)
        self.wire_off = torch.zeros(P + 1, **i64)
        self.wire_len = torch.zeros(P, **i64)
        self.t = 0
        # learned predictor: per-slot histories on both sides, the network's
        # weights, and (optionally) a buffer receiving training samples
        self.predictor = predictor or params is not None
        self.params = params
        self.allow_residual = allow_residual
        self.samples = None
        if self.predictor:
            hb = max(max_records, 1) * 48
            self.hist = [torch.zeros(hb, **u8), torch.zeros(hb, **u8)]
            self.rhist = [torch.zeros(hb, **u8), torch.zeros(hb, **u8)]

    def reset(self):
        """Forget both references: the next iteration is sent without a reference."""
        self.t = 0

    def ranges(self):
        if self.path != "per_subdomain":
            return [(0, self.P)]
        return [(27 * s, 27 * s + 27) for s in range(self.P // 27)]

    def schedule(self, t: int):
        """(output buffer, reference buffer or -1, reference iteration) of
        iteration t under the reference interval K (tera_ref_schedule)."""
        return ref_schedule(t, self.K)

    def slot_of(self, t: int) -> int:
        """Buffer of iteration t's outputs."""
        return self.schedule(t)[0]

    def _launch(self, state: dict, t: int, stream=None):
        """Enqueue iteration t on the stream (outputs and references in the
        buffers tera_ref_schedule names)."""
        ctx = self.ctx
        first = t == 0
        cur, prv, _ = self.schedule(t)
        if first:
            prv = 1 - cur
        part = self.part
        pair_off = self.pair_off[cur]
        part.pair_off = pair_off  # this iteration's offsets become the next one's reference layout
        ctx.partition(state, part, stream)
        ref_prev = None if first else self.ref[prv]
        ref_off_prev = None if first else self.pair_off[prv]
        recv_prev = None if first else self.recv[prv]
        recv_off_prev = None if first else self.recv_off[prv]
        if self.id_columns:
            ctx.pack_ids(state, part, self.rec, self.rec_ids, stream)
        else:
            for (a, b) in self.ranges():
                ctx.pack(state, part, self.rec, a, b, stream)
        if self.predictor:
            enc = dict(params=self.params, hist_prev=None if first else self.hist[prv],
                       hist_next=self.hist[cur], samples=self.samples,
                       allow_residual=self.allow_residual)
            dec = dict(params=self.params, hist_prev=None if first else self.rhist[prv],
                       hist_next=self.rhist[cur])
            if self.path == "batched":
                ctx.codec_batched_pred(self.rec, pair_off, ref_prev, ref_off_prev, self.ref[cur],
                                       self.wire, self.wire_off, self.wire_len, recv_prev,
                                       recv_off_prev, self.recv[cur], self.recv_off[cur], enc,
                                       dec, self.mode, self.tune, stream)
                return
            for (a, b) in self.ranges():
                ctx.delta_encode_pred(self.rec, pair_off, ref_prev, ref_off_prev, self.ref[cur],
                                      self.wire, self.wire_off, self.wire_len, enc, self.mode, a,
                                      b, stream)
            for (a, b) in self.ranges():
                ctx.delta_decode_pred(self.wire, self.wire_off, recv_prev, recv_off_prev,
                                      self.recv[cur], self.recv_off[cur], dec, a, b, stream)
            return
        if self.path == "batched":
            args, kw = self.codec_args(t)
            ctx.codec_batched(*args, **kw, mode=self.mode, tune=self.tune, stream=stream)
            return
        for (a, b) in self.ranges():
            ctx.delta_encode(self.rec, pair_off, ref_prev, ref_off_prev, self.ref[cur],
                             self.wire, self.wire_off, self.wire_len, self.mode, a, b, stream)
        for (a, b) in self.ranges():
            ctx.delta_decode(self.wire, self.wire_off, recv_prev, recv_off_prev, self.recv[cur],
                             self.recv_off[cur], a, b, stream)

    def codec_args(self, t: int):
        """Positional and keyword arguments of the batched codec of iteration t
        (buffers from the reference schedule), without mode, tune and stream."""
        cur, prv, _ = self.schedule(t)
        first = t == 0
        args = (self.rec, self.pair_off[cur], None if first else self.ref[prv],
                None if first else self.pair_off[prv], self.ref[cur], self.wire, self.wire_off,
                self.wire_len, None if first else self.recv[prv],
                None if first else self.recv_off[prv], self.recv[cur], self.recv_off[cur])
        kw = {}
        if self.id_columns:
            kw["ids"] = dict(msg=self.rec_ids, ref_prev=None if first else self.ref_ids[prv],
                             ref_next=self.ref_ids[cur])
        return args, kw

    def step(self, state: dict, stream=None):
        """Classify, pack, encode and decode every pair for one iteration."""
        self._launch(state, self.t, stream)
        self.t += 1
        return self.last

    def capture(self, state: dict, t: int | None = None) -> torch.cuda.CUDAGraph:
        """A CUDA graph of iteration t (default: the next one) on this state's buffers.

        Replaying it is equivalent to step(state) at that iteration; call
        advance() after each replay.  Scratch must already be reserved (one
        eager step beforehand does it)."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._launch(state, self.t if t is None else t, torch.cuda.current_stream())
        return g

    def advance(self):
        self.t += 1

    # --- checkpoint / resume ---
    def _spec(self) -> dict:
        g = self.ctx.grid
        return {"lo": tuple(g.lo), "hi": tuple(g.hi), "n": tuple(g.n), "w": g.w,
                "periodic": int(g.periodic), "class_id": self.ctx.class_id, "P": self.P,
                "mode": self.mode, "K": self.K, "id_columns": self.id_columns,
                "predictor": self.predictor}

    def checkpoint(self) -> dict:
        """The state the next iterations read, copied to host memory: the
        iteration counter and, once an iteration has run, the reference buffer
        the next iteration reads (tera_ref_schedule) on both sides: the sender
        reference with its offsets (and id column), the receive buffer with its
        offsets (and both sides' predictor histories).  Only the used bytes are
        copied.  Pairs marked with reset_reference are not part of it.  A new
        exchange on an equal grid resumes the chain with restore(); without a
        checkpoint the chain can only restart from a raw iteration (reset())."""
        torch.cuda.synchronize(self.ctx.device)
        state = {"version": 1, "t": self.t, "spec": self._spec()}
        if self.t == 0:
            return state
        _, prv, _ = self.schedule(self.t)
        off = self.pair_off[prv].cpu()
        roff = self.recv_off[prv].cpu()
        E, R = int(off[-1]), int(roff[-1])
        state["ref_off"] = off
        state["ref"] = self.ref[prv][:(E + self.P) * 64].cpu()
        state["recv_off"] = roff
        state["recv"] = self.recv[prv][:(R + self.P) * 64].cpu()
        if self.id_columns:
            state["ref_ids"] = self.ref_ids[prv][:E].cpu()
        if self.predictor:
            state["hist"] = self.hist[prv][:E * 48].cpu()
            state["rhist"] = self.rhist[prv][:R * 48].cpu()
        return state

    def restore(self, state: dict):
        """Resume from checkpoint(): the next step() runs the checkpoint's next
        iteration against its references, producing the bytes the original
        chain would have produced.  The exchange must have the same grid,
        class id, mode, reference interval, id columns and predictor setting,
        and room for the references (ValueError otherwise)."""
        if state.get("version") != 1:
            raise ValueError("unknown checkpoint version")
        spec = self._spec()
        if state["spec"] != spec:
            diff = sorted(k for k in spec if state["spec"].get(k) != spec[k])
            raise ValueError(f"checkpoint taken with another configuration: {diff}")
        t = int(state["t"])
        if t > 0:
            _, prv, _ = self.schedule(t)
            units = self.max_records + self.P
            ref, recv = state["ref"], state["recv"]
            if ref.numel() > units * 64 or recv.numel() > units * 64:
                raise ValueError("checkpoint references exceed this exchange's max_records")
            self.pair_off[prv].copy_(state["ref_off"])
            self.ref[prv][:ref.numel()].copy_(ref)
            self.recv_off[prv].copy_(state["recv_off"])
            self.recv[prv][:recv.numel()].copy_(recv)
            if self.id_columns:
                ids = state["ref_ids"]
                self.ref_ids[prv][:ids.numel()].copy_(ids)
            if self.predictor:
                self.hist[prv][:state["hist"].numel()].copy_(state["hist"])
                self.rhist[prv][:state["rhist"].numel()].copy_(state["rhist"])
            torch.cuda.synchronize(self.ctx.device)
        self.t = t

    # --- views of the last iteration's outputs ---
    @property
    def last(self) -> int:
        return self.slot_of(self.t - 1) if self.t > 0 else 0

    def sender_ref(self):
        return self.ref[self.last], self.pair_off[self.last]

    def sender_hist(self):
        return self.hist[self.last]

    def receiver_hist(self):
        return self.rhist[self.last]

    def receiver_ref(self):
        return self.recv[self.last], self.recv_off[self.last]
