"""One aura-exchange iteration over every pair, with the per-pair references
kept on both sides between iterations (paper Sec. 2.3: each sender/receiver
pair stores the same reference and updates it every iteration here).

Buffers are allocated once for a maximum agent count and record count; the
sender and receiver references are double-buffered (previous / next).
"""
from __future__ import annotations

import torch

from ._lib import MODE_XOR
from .api import Context, PartitionBuffers


class AuraExchange:
    def __init__(self, ctx: Context, max_agents: int, max_records: int, mode: int = MODE_XOR,
                 per_subdomain: bool = False):
        self.ctx = ctx
        self.mode = mode
        self.per_subdomain = per_subdomain
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
        self.wire_cap = 80 * P + 72 * max_records + 64
        self.wire = torch.empty(self.wire_cap, **u8)
        self.wire_off = torch.zeros(P + 1, **i64)
        self.wire_len = torch.zeros(P, **i64)
        self.t = 0

    def reset(self):
        """Forget both references: the next iteration is sent without a reference."""
        self.t = 0

    def ranges(self):
        if not self.per_subdomain:
            return [(0, self.P)]
        return [(27 * s, 27 * s + 27) for s in range(self.P // 27)]

    def step(self, state: dict, stream=None):
        """Classify, pack, encode and decode every pair for one iteration."""
        ctx = self.ctx
        cur, prv = self.t % 2, (self.t + 1) % 2
        first = self.t == 0
        part = self.part
        pair_off = self.pair_off[cur]
        part.pair_off = pair_off  # this iteration's offsets become the next one's reference layout
        ctx.partition(state, part, stream)
        ref_prev = None if first else self.ref[prv]
        ref_off_prev = None if first else self.pair_off[prv]
        recv_prev = None if first else self.recv[prv]
        recv_off_prev = None if first else self.recv_off[prv]
        for (a, b) in self.ranges():
            ctx.pack(state, part, self.rec, a, b, stream)
        for (a, b) in self.ranges():
            ctx.delta_encode(self.rec, pair_off, ref_prev, ref_off_prev, self.ref[cur],
                             self.wire, self.wire_off, self.wire_len, self.mode, a, b, stream)
        for (a, b) in self.ranges():
            ctx.delta_decode(self.wire, self.wire_off, recv_prev, recv_off_prev, self.recv[cur],
                             self.recv_off[cur], a, b, stream)
        self.t += 1
        return cur

    # --- views of the last iteration's outputs ---
    @property
    def last(self) -> int:
        return (self.t + 1) % 2

    def sender_ref(self):
        return self.ref[self.last], self.pair_off[self.last]

    def receiver_ref(self):
        return self.recv[self.last], self.recv_off[self.last]
