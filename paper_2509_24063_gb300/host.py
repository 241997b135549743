"""Exchange iterations on host-resident agent state.

Each step copies the eight state columns from pinned host memory to the
device (on a copy stream), runs the exchange (partition, pack, encode and
decode of every pair) and writes the iteration's wire messages back into a
pinned host buffer with tera_wire_to_host, whose length is known only on the
device: nothing inside a step waits for the host.  Device inputs are
double-buffered, so the copy of the next step's inputs runs while this step
computes, as a data loader would.
"""
from __future__ import annotations

import torch

from .api import Context
from .exchange import AuraExchange

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


class Pending:
    """A step in flight: its event and the pinned word receiving its wire length."""

    def __init__(self, event: torch.cuda.Event, count: torch.Tensor, out: torch.Tensor):
        self.event = event
        self.count = count
        self.out = out

    def wait(self) -> int:
        """Block until the step's wire bytes are in host memory; return their count."""
        self.event.synchronize()
        return int(self.count[0])


class HostExchange:
    def __init__(self, ctx: Context, max_agents: int, max_records: int, path: str = "batched",
                 tune=None, depth: int = 2, ref_interval: int = 1):
        self.ctx = ctx
        self.ex = AuraExchange(ctx, max_agents, max_records, path=path, tune=tune,
                               ref_interval=ref_interval)
        dev = torch.device("cuda", ctx.device)
        self.depth = depth
        self.inputs = [{f: torch.empty(max_agents, dtype=torch.int64 if f == "id" else torch.float64,
                                       device=dev) for f in FIELDS} for _ in range(depth)]
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.free = [None] * depth  # event: the step that last read buffer k is done
        self.k = 0

    @property
    def wire_capacity(self) -> int:
        return self.ex.wire_cap

    def step(self, host_state: dict, host_out: torch.Tensor, stream=None) -> Pending:
        """Enqueue one iteration: host_state holds the eight columns as pinned
        host tensors (id int64, the rest float64); host_out is a pinned uint8
        buffer of at least wire_capacity bytes.  Returns at once."""
        compute = stream or torch.cuda.current_stream()
        slot = self.k % self.depth
        buf = self.inputs[slot]
        n = int(host_state["x"].shape[0])
        if n > buf["x"].shape[0]:
            raise ValueError("more agents than max_agents")
        if self.free[slot] is not None:
            self.copy_stream.wait_event(self.free[slot])
        with torch.cuda.stream(self.copy_stream):
            for f in FIELDS:
                buf[f][:n].copy_(host_state[f], non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(self.copy_stream)
        compute.wait_event(copied)
        view = {f: buf[f][:n] for f in FIELDS}
        self.ex.step(view, compute)
        count = torch.zeros(1, dtype=torch.int64).pin_memory()  # held by the Pending
        self.ctx.wire_to_host(self.ex.wire, self.ex.wire_off, host_out, count, compute)
        done = torch.cuda.Event()
        done.record(compute)
        self.free[slot] = done
        self.k += 1
        return Pending(done, count, host_out)
