"""Agent migration between the boxes of one grid (paper Sec. 2.1, "Agent
Migration"), through ``tera_migrate_send`` / ``tera_migrate_recv``.

The state is box-major: box s holds agents ``[box_off[s], box_off[s+1])``.
After the agents moved, a step sends every agent whose position now lies in
another box to that box as a raw TeraAgent IO record (one inbox per receiver
box and arrival side), keeps the stayers in order, and receives the inboxes
after each box's stayers.  Box offsets are int64 tensors holding u64 values.
"""
from __future__ import annotations

import ctypes as C

import torch

from ._lib import Soa, check
from .api import FIELDS, _ptr, _stream, soa_from_state


def _soa(st: dict) -> Soa:
    return soa_from_state(st)


class Migration:
    """Inbox arena and offsets of one context; the caller owns the states."""

    def __init__(self, ctx, max_agents: int, max_leavers: int | None = None):
        self.ctx = ctx
        self.lib = ctx.lib
        self.Q = int(ctx.n_pairs)
        self.B = self.Q // 27
        if max_leavers is None:
            max_leavers = max(4096, int(max_agents) // 8)
        self.arena_units = self.Q + int(max_leavers)
        dev = torch.device("cuda", ctx.device)
        self.arena = torch.zeros(self.arena_units * 64, dtype=torch.uint8, device=dev)
        self.inbox_off = torch.zeros(self.Q + 1, dtype=torch.int64, device=dev)

    def empty_like(self, st: dict) -> dict:
        return {f: torch.empty_like(st[f]) for f in FIELDS}

    def send(self, prev: dict, box_off_prev, nxt: dict, box_off_next, stream=None):
        """Classify, serialize the leavers into the inboxes, place the stayers."""
        sp, sn = _soa(prev), _soa(nxt)
        check(self.lib.tera_migrate_send(self.ctx.h, C.byref(sp), _ptr(box_off_prev),
                                         _ptr(self.arena), self.arena_units,
                                         _ptr(self.inbox_off), C.byref(sn), _ptr(box_off_next),
                                         _stream(stream)), "tera_migrate_send")

    def recv(self, nxt: dict, box_off_next, stream=None, arena=None, inbox_off=None):
        """Deserialize every inbox into the next state after its box's stayers
        (from this object's arena, or from another inbox arena and offsets)."""
        sn = _soa(nxt)
        a = self.arena if arena is None else arena
        o = self.inbox_off if inbox_off is None else inbox_off
        check(self.lib.tera_migrate_recv(self.ctx.h, _ptr(a), a.numel() // 64, _ptr(o),
                                         _ptr(box_off_next), C.byref(sn), _stream(stream)),
              "tera_migrate_recv")

    def step(self, prev: dict, box_off_prev, nxt: dict | None = None, box_off_next=None,
             stream=None):
        """One migration step; returns (next state, next box offsets)."""
        if nxt is None:
            nxt = self.empty_like(prev)
        if box_off_next is None:
            box_off_next = torch.empty_like(box_off_prev)
        self.send(prev, box_off_prev, nxt, box_off_next, stream)
        self.recv(nxt, box_off_next, stream)
        return nxt, box_off_next

    def regroup(self, st: dict, stream=None):
        """Box-major copy of a state in any order: a step in which every agent
        starts in box 0, so every box receives its agents in index order.
        Every agent outside box 0 is a leaver: max_leavers must be >= n."""
        n = int(st["x"].shape[0])
        if self.arena_units - self.Q < n:
            raise ValueError(f"regroup of {n} agents needs max_leavers >= {n} "
                             f"(this arena holds {self.arena_units - self.Q})")
        off = torch.full((self.B + 1,), n, dtype=torch.int64, device=st["x"].device)
        off[0] = 0
        return self.step({f: st[f] for f in FIELDS}, off, stream=stream)
