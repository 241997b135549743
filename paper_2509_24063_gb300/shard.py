"""Boxes of one grid sharded over several ranks (paper Sec. 2.1: the
partitioning boxes are distributed over the ranks, aura agents are copied and
migrating agents moved between them; Sec. 2.4 "Load Balancing": the diffusive
method moves boxes between neighbouring ranks).

One process per GPU.  Every rank holds the agents of the boxes it owns and runs
the library's kernels on them over the whole grid's pair (or inbox) index
space: a pair whose sender box lives on another rank is simply empty there.
Only the wire messages of pairs whose receiver box lives on another rank, and
the migration inboxes of boxes on another rank, move between ranks: point to
point, into the receiving rank's own memory (torch.distributed send/recv:
NCCL between GPUs, gloo between hosts), where they are decoded.

This module is host logic only: which rank owns which box, which message goes
where, the arenas each rank decodes, and the diffusive rebalancing.  Encoding,
decoding and migration run in the library's kernels (tera_delta_encode,
tera_delta_decode, tera_migrate_send / tera_migrate_recv); ShardedExchange and
ShardedMigration put them together with a transport.

Byte formats are those of include/tera.h: a wire message is 16-byte padded, an
empty raw message is its 64-byte header alone, an inbox arena holds one
64-byte TAIO header per inbox followed by its records.
"""
from __future__ import annotations

import numpy as np
import torch

WIRE_MAGIC = 0x41524554  # "TERA"
TAIO_MAGIC = 0x4F494154  # "TAIO"
FORMAT_VERSION = 1
REC = 64


# ---------------- geometry of the box grid ----------------

def n_boxes(n) -> int:
    return int(n[0]) * int(n[1]) * int(n[2])


def neighbour(n, periodic: int, s, b):
    """Box at neighbour bit b of box s (b = (ox+1) + 3 (oy+1) + 9 (oz+1)), or -1
    when there is none (beyond a closed axis, or b = 13, the box itself).  On a
    periodic axis the index wraps modulo n.  Works on arrays."""
    s = np.asarray(s, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    n0, n1, n2 = (int(v) for v in n)
    c = [s % n0, (s // n0) % n1, s // (n0 * n1)]
    o = [b % 3 - 1, (b // 3) % 3 - 1, b // 9 - 1]
    ok = b != 13
    j = []
    for a, na in enumerate((n0, n1, n2)):
        v = c[a] + o[a]
        if (periodic >> a) & 1:
            v = np.mod(v, na)
        else:
            ok = ok & (v >= 0) & (v < na)
        j.append(v)
    d = j[0] + n0 * (j[1] + n1 * j[2])
    return np.where(ok, d, -1)


def pair_receivers(n, periodic: int = 0) -> np.ndarray:
    """Receiver box of every pair p = s*27 + b (-1: the pair never carries a record)."""
    P = n_boxes(n) * 27
    p = np.arange(P, dtype=np.int64)
    return neighbour(n, periodic, p // 27, p % 27)


def adjacent_boxes(n, periodic: int, s: int) -> np.ndarray:
    """The (up to 26) boxes adjacent to box s, ascending."""
    d = neighbour(n, periodic, np.full(27, s), np.arange(27))
    return np.unique(d[d >= 0])


# ---------------- which rank owns which box ----------------

def slab_owners(B: int, world: int, weight=None) -> np.ndarray:
    """Contiguous ranges of box indices, one per rank in rank order, each close
    to 1/world of the total weight (uniform weights when none are given)."""
    w = np.ones(B, dtype=np.float64) if weight is None else np.asarray(weight, np.float64)
    total = float(w.sum())
    if total <= 0.0:
        w = np.ones(B, dtype=np.float64)
        total = float(B)
    mid = np.cumsum(w) - 0.5 * w  # weight before each box's middle
    owner = np.floor(world * mid / total).astype(np.int64)
    return np.clip(owner, 0, world - 1).astype(np.int32)


def rank_adjacency(box_owner, n, periodic: int = 0) -> dict:
    """rank -> sorted list of the other ranks owning a box adjacent to one of its boxes."""
    owner = np.asarray(box_owner)
    B = owner.shape[0]
    d = neighbour(n, periodic, np.repeat(np.arange(B), 27), np.tile(np.arange(27), B))
    s = np.repeat(np.arange(B), 27)
    keep = d >= 0
    a, b = owner[s[keep]], owner[d[keep]]
    out = {int(r): set() for r in np.unique(owner)}
    for r, q in zip(a.tolist(), b.tolist()):
        if r != q:
            out[r].add(q)
    return {r: sorted(v) for r, v in out.items()}


def diffusive_rebalance(box_owner, box_cost, rank_time, n, periodic: int = 0) -> np.ndarray:
    """One round of diffusive load balancing (Sec. 2.4): a rank whose runtime
    exceeds the average over itself and its neighbour ranks gives boxes to the
    neighbours whose runtime is below that average.

    A box's time is its share of its rank's runtime, in proportion to
    box_cost (e.g. its agents).  Rank r gives neighbour q the boxes of r that
    touch a box of q (ascending index), each while its time fits in both what
    r has above the average and what q has below it; r keeps at least one box.
    Ranks are visited in ascending order on the map as it stood at the start of
    the round, and a box moves at most once per round.  Returns the new map."""
    owner0 = np.asarray(box_owner, dtype=np.int32)
    cost = np.asarray(box_cost, dtype=np.float64)
    t = np.asarray(rank_time, dtype=np.float64)
    owner = owner0.copy()
    adj = rank_adjacency(owner0, n, periodic)
    moved = np.zeros(owner.shape[0], dtype=bool)
    gained = np.zeros(t.shape[0], dtype=np.float64)  # time given to each rank this round
    for r in sorted(adj):
        nbrs = adj[r]
        if not nbrs:
            continue
        avg = float(np.mean(t[[r] + nbrs]))
        excess = t[r] - avg
        if excess <= 0.0:
            continue
        mine = np.nonzero(owner0 == r)[0]
        c_r = float(cost[mine].sum())
        if c_r <= 0.0:
            continue
        sec = t[r] / c_r  # seconds per unit of cost on rank r
        for q in nbrs:
            room = avg - (t[q] + gained[q])
            if room <= 0.0 or excess <= 0.0:
                continue
            give = min(excess, room)
            for k in mine:
                if moved[k] or owner[k] != r:
                    continue
                if int(np.count_nonzero(owner == r)) <= 1:
                    break
                if not np.any(owner[adjacent_boxes(n, periodic, int(k))] == q):
                    continue
                tk = float(cost[k]) * sec
                if tk > give:
                    continue
                owner[k] = q
                moved[k] = True
                give -= tk
                excess -= tk
                gained[q] += tk
    return owner


def pairs_to_reset(old_owner, new_owner, n, periodic: int = 0) -> np.ndarray:
    """Pairs whose sender or receiver box changed rank: their references are no
    longer held by the same two ranks, so the new sender must send them raw
    once (tera_reset_reference)."""
    old = np.asarray(old_owner)
    new = np.asarray(new_owner)
    d = pair_receivers(n, periodic)
    P = d.shape[0]
    s = np.arange(P) // 27
    has = d >= 0
    dd = np.where(has, d, 0)
    changed = (old[s] != new[s]) | (has & (old[dd] != new[dd]))
    return np.nonzero(changed & has)[0]


# ---------------- the aura exchange's wire messages ----------------

class WirePlan:
    """Which pairs rank `rank` sends to / receives from every other rank.

    mine: pairs whose receiver box this rank owns (decoded here), ascending;
    send[q] / recv[q]: pairs this rank sends to / receives from rank q, ascending;
    local: pairs with both boxes on this rank."""

    def __init__(self, box_owner, n, periodic: int, rank: int, world: int):
        owner = np.asarray(box_owner, dtype=np.int64)
        d = pair_receivers(n, periodic)
        P = d.shape[0]
        s_rank = owner[np.arange(P) // 27]
        r_rank = np.where(d >= 0, owner[np.where(d >= 0, d, 0)], -1)
        self.rank = rank
        self.P = P
        ranks = [q for q in range(world) if q != rank]
        self.mine = np.nonzero(r_rank == rank)[0]
        self.local = np.nonzero((r_rank == rank) & (s_rank == rank))[0]
        self.send = {q: np.nonzero((s_rank == rank) & (r_rank == q))[0] for q in ranks}
        self.recv = {q: np.nonzero((s_rank == q) & (r_rank == rank))[0] for q in ranks}


def _byte_index(starts: torch.Tensor, lengths: torch.Tensor) -> torch.Tensor:
    """Indices of the bytes [starts[i], starts[i] + lengths[i]) for every i, in order."""
    total = int(lengths.sum().item()) if lengths.numel() else 0
    if total == 0:
        return torch.zeros(0, dtype=torch.int64, device=starts.device)
    first = torch.cumsum(lengths, 0) - lengths
    seg = torch.repeat_interleave(torch.arange(lengths.numel(), device=starts.device), lengths)
    return starts[seg] + (torch.arange(total, device=starts.device) - first[seg])


def gather_messages(wire, wire_off, wire_len, pairs):
    """The messages of `pairs` (ascending), concatenated: (lengths, bytes).
    wire_off / wire_len are int64 tensors holding the library's u64 values."""
    dev = wire.device
    idx = torch.as_tensor(np.asarray(pairs, dtype=np.int64), device=dev)
    lens = wire_len.to(torch.int64)[idx]
    starts = wire_off.to(torch.int64)[idx]
    return lens, wire[_byte_index(starts, lens)]


def empty_messages(pairs, class_id: int) -> np.ndarray:
    """64-byte headers of empty raw messages (no slots, no records) for pairs."""
    pairs = np.asarray(pairs, dtype=np.uint64)
    h = np.zeros((pairs.shape[0], 8), dtype=np.uint64)
    h[:, 0] = WIRE_MAGIC | (FORMAT_VERSION << 32) | (REC << 48)
    h[:, 1] = np.uint64(class_id)  # mode 0 (raw) in the high half
    h[:, 6] = pairs                # pair p, then a zero word
    h[:, 7] = 64                   # message bytes
    return h.view(np.uint8).reshape(-1)


def decode_arena(plan: WirePlan, class_id: int, local, received: dict, device):
    """The wire arena this rank decodes: for every pair, its message if the
    receiver box is here (local ones from this rank's own wire, the others as
    received), else an empty raw message.  local = (wire, wire_off, wire_len);
    received[q] = (lengths, bytes) of the pairs plan.recv[q].
    Returns (wire_in uint8, wire_off_in int64[P+1])."""
    P = plan.P
    lens = torch.full((P,), 64, dtype=torch.int64, device=device)
    parts = []  # (pairs, lengths, bytes)
    if plan.local.size:
        ll, lb = gather_messages(*local, plan.local)
        parts.append((plan.local, ll.to(device), lb.to(device)))
    for q, pq in plan.recv.items():
        if pq.size:
            rl, rb = received[q]
            parts.append((pq, rl.to(device), rb.to(device)))
    for pq, pl, _ in parts:
        lens[torch.as_tensor(pq, device=device)] = pl
    off = torch.zeros(P + 1, dtype=torch.int64, device=device)
    off[1:] = torch.cumsum(lens, 0)
    wire_in = torch.empty(int(off[-1].item()), dtype=torch.uint8, device=device)
    others = np.setdiff1d(np.arange(P), plan.mine)
    if others.size:
        hdr = torch.from_numpy(empty_messages(others, class_id)).to(device)
        wire_in[_byte_index(off[torch.as_tensor(others, device=device)],
                            torch.full((others.size,), 64, dtype=torch.int64,
                                       device=device))] = hdr
    for pq, pl, pb in parts:
        wire_in[_byte_index(off[torch.as_tensor(pq, device=device)], pl)] = pb
    return wire_in, off


# ---------------- migration inboxes ----------------

class InboxPlan:
    """Inbox q = d*27 + b belongs to the rank owning box d.  send[r] lists the
    inboxes this rank fills for rank r (every inbox of r's boxes), ascending."""

    def __init__(self, box_owner, rank: int, world: int):
        owner = np.asarray(box_owner, dtype=np.int64)
        Q = owner.shape[0] * 27
        dest = owner[np.arange(Q) // 27]
        self.rank = rank
        self.Q = Q
        self.mine = np.nonzero(dest == rank)[0]
        self.ranks = list(range(world))
        self.send = {r: np.nonzero(dest == r)[0] for r in self.ranks if r != rank}


def gather_inboxes(arena, inbox_off, inboxes):
    """Record counts and records (without headers) of `inboxes` (ascending) of
    an inbox arena: (counts int64, bytes)."""
    dev = arena.device
    off = inbox_off.to(torch.int64)
    q = torch.as_tensor(np.asarray(inboxes, dtype=np.int64), device=dev)
    counts = off[q + 1] - off[q]
    starts = (off[q] + q + 1) * REC
    return counts, arena[_byte_index(starts, counts * REC)]


def taio_headers(inboxes, counts: np.ndarray, class_id: int) -> np.ndarray:
    """64-byte TAIO headers of inboxes with these record counts."""
    q = np.asarray(inboxes, dtype=np.uint64)
    h = np.zeros((q.shape[0], 8), dtype=np.uint64)
    h[:, 0] = TAIO_MAGIC | (FORMAT_VERSION << 32) | (REC << 48)
    h[:, 1] = np.uint64(class_id) | (q << np.uint64(32))
    h[:, 2] = np.asarray(counts, dtype=np.uint64)
    return h.view(np.uint8).reshape(-1)


def merge_inboxes(plan: InboxPlan, class_id: int, own, received: dict, device):
    """The inbox arena of this rank's boxes: inbox q's records from every rank
    in rank order (this rank's own at its place), so that an inbox holds its
    agents as the single-rank step would (ascending global index, the ranks'
    states being the box-major state's consecutive parts).  own = (arena,
    inbox_off) of this rank's tera_migrate_send; received[r] = (counts,
    bytes) of plan.send-ordered inboxes from rank r (the inboxes of this
    rank's boxes).  Inboxes of other ranks' boxes are empty.
    Returns (arena uint8, inbox_off int64[Q+1])."""
    Q = plan.Q
    mine = plan.mine
    srcs = []
    for r in plan.ranks:
        if r == plan.rank:
            c, b = gather_inboxes(*own, mine)
        else:
            c, b = received[r]
        srcs.append((c.to(device), b.to(device)))
    counts = torch.zeros(Q, dtype=torch.int64, device=device)
    mine_t = torch.as_tensor(mine, device=device)
    for c, _ in srcs:
        counts[mine_t] += c
    off = torch.zeros(Q + 1, dtype=torch.int64, device=device)
    off[1:] = torch.cumsum(counts, 0)
    arena = torch.empty(int((off[-1] + Q).item()) * REC, dtype=torch.uint8, device=device)
    hdr = torch.from_numpy(taio_headers(np.arange(Q), counts.cpu().numpy(), class_id)).to(device)
    arena[_byte_index((off[:-1] + torch.arange(Q, device=device)) * REC,
                      torch.full((Q,), REC, dtype=torch.int64, device=device))] = hdr
    # each source's records go after the earlier sources' records of the same inbox
    done = torch.zeros(mine.size, dtype=torch.int64, device=device)
    for c, b in srcs:
        starts = (off[mine_t] + mine_t + 1 + done) * REC
        arena[_byte_index(starts, c * REC)] = b
        done += c
    return arena, off


def box_offsets(counts_per_box: torch.Tensor) -> torch.Tensor:
    off = torch.zeros(counts_per_box.numel() + 1, dtype=torch.int64,
                      device=counts_per_box.device)
    off[1:] = torch.cumsum(counts_per_box.to(torch.int64), 0)
    return off


# ---------------- transport ----------------

class DistTransport:
    """Byte buffers exchanged point to point with every other rank of a
    torch.distributed process group: the sizes first, then the bytes, each
    direction one send/recv pair batched together (NCCL for device tensors,
    gloo for host tensors).  A buffer arrives in the receiving rank's memory."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, sends: dict, device) -> dict:
        """sends[q] = tensor (any dtype, contiguous, 1-D) for rank q (every other
        rank must appear, possibly empty).  Returns {q: tensor received from q}
        of the same dtype."""
        dist = self.dist
        peers = [q for q in range(self.world) if q != self.rank]
        if not peers:
            return {}
        dtype = next(iter(sends.values())).dtype
        size_out = {q: torch.tensor([sends[q].numel()], dtype=torch.int64, device=device)
                    for q in peers}
        size_in = {q: torch.zeros(1, dtype=torch.int64, device=device) for q in peers}
        ops = []
        for q in peers:
            ops.append(dist.P2POp(dist.isend, size_out[q], q, self.group))
            ops.append(dist.P2POp(dist.irecv, size_in[q], q, self.group))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        out = {q: torch.empty(int(size_in[q].item()), dtype=dtype, device=device) for q in peers}
        ops = []
        for q in peers:
            if sends[q].numel():
                ops.append(dist.P2POp(dist.isend, sends[q].contiguous(), q, self.group))
            if out[q].numel():
                ops.append(dist.P2POp(dist.irecv, out[q], q, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return out


def outgoing_wire(plan: WirePlan, local) -> dict:
    """{q: (lengths, bytes)} of this rank's messages for rank q's boxes."""
    return {q: gather_messages(*local, pq) for q, pq in plan.send.items()}


def outgoing_inboxes(plan: InboxPlan, own) -> dict:
    """{r: (counts, bytes)} of this rank's inboxes for rank r's boxes."""
    return {r: gather_inboxes(*own, qs) for r, qs in plan.send.items()}


def _exchange_pairs(transport, out: dict, device) -> dict:
    a = transport.exchange({q: v[0].to(device) for q, v in out.items()}, device)
    b = transport.exchange({q: v[1].to(device) for q, v in out.items()}, device)
    return {q: (a[q], b[q]) for q in out}


def route_wire(plan: WirePlan, transport, local, class_id: int, device):
    """Send this rank's messages for other ranks' boxes, receive theirs for this
    rank's boxes, and return this rank's decode arena (decode_arena)."""
    received = _exchange_pairs(transport, outgoing_wire(plan, local), device)
    return decode_arena(plan, class_id, local, received, device)


def route_inboxes(plan: InboxPlan, transport, own, class_id: int, device):
    """Send the inboxes of other ranks' boxes to their owners, receive this
    rank's from every rank, and return the merged arena (merge_inboxes)."""
    received = _exchange_pairs(transport, outgoing_inboxes(plan, own), device)
    return merge_inboxes(plan, class_id, own, received, device)


def stayer_layout(box_off_sent, own_inbox_off, merged_inbox_off):
    """Where the stayers go once other ranks' immigrants are known.

    tera_migrate_send placed box d's stayers at the start of box d of its own
    layout box_off_sent (stayers + this rank's own immigrants).  With the
    merged inboxes, box d holds its stayers, then every rank's immigrants.
    Returns (final box offsets [B+1], source positions, destination positions)
    of the stayers: next_final[dst] = next_sent[src]."""
    off = box_off_sent.to(torch.int64)
    B = off.numel() - 1
    dev = off.device
    own = own_inbox_off.to(torch.int64)
    mrg = merged_inbox_off.to(dev).to(torch.int64)
    own_in = (own[1:] - own[:-1]).reshape(B, 27).sum(1)
    mrg_in = (mrg[1:] - mrg[:-1]).reshape(B, 27).sum(1)
    stay = (off[1:] - off[:-1]) - own_in
    final = box_offsets(stay + mrg_in)
    src = _byte_index(off[:-1], stay)
    dst = _byte_index(final[:-1], stay)
    return final, src, dst


def transfer_boxes(state: dict, box_off, old_owner, new_owner, rank: int, transport, device):
    """Move the agents of boxes that changed rank (after a rebalance): each
    rank sends the agents of the boxes it gave away to their new owners and
    receives those of the boxes it gained; every box keeps its agents' order.
    state: this rank's box-major state (dict of 1-D tensors), box_off [B+1].
    Returns the new (state, box_off)."""
    old = np.asarray(old_owner)
    new = np.asarray(new_owner)
    off = box_off.to(torch.int64).to(device)
    B = old.shape[0]
    world = transport.world if transport is not None else 1
    keys = list(state)
    counts = off[1:] - off[:-1]
    sends, counts_out = {}, {}
    for q in range(world):
        if q == rank:
            continue
        boxes = np.nonzero((old == rank) & (new == q))[0]
        bt = torch.as_tensor(boxes, device=device)
        idx = _byte_index(off[bt], counts[bt])
        counts_out[q] = counts[bt]
        sends[q] = {k: state[k][idx] for k in keys}
    got_counts = transport.exchange(counts_out, device) if world > 1 else {}
    got = {}
    for k in keys:
        r = transport.exchange({q: sends[q][k] for q in sends}, device) if world > 1 else {}
        for q, v in r.items():
            got.setdefault(q, {})[k] = v
    # the new layout: every box this rank owns now, in box order
    new_counts = torch.zeros(B, dtype=torch.int64, device=device)
    kept = np.nonzero((old == rank) & (new == rank))[0]
    kt = torch.as_tensor(kept, device=device)
    new_counts[kt] = counts[kt]
    for q in got_counts:
        boxes = torch.as_tensor(np.nonzero((old == q) & (new == rank))[0], device=device)
        new_counts[boxes] = got_counts[q]
    new_off = box_offsets(new_counts)
    n_new = int(new_off[-1].item())
    out = {k: torch.empty(n_new, dtype=state[k].dtype, device=device) for k in keys}
    src = _byte_index(off[kt], counts[kt])
    dst = _byte_index(new_off[kt], counts[kt])
    for k in keys:
        out[k][dst] = state[k][src]
    for q in got:
        boxes = torch.as_tensor(np.nonzero((old == q) & (new == rank))[0], device=device)
        dst = _byte_index(new_off[boxes], got_counts[q])
        for k in keys:
            out[k][dst] = got[q][k]
    return out, new_off


class ShardedExchange:
    """The aura exchange of one rank's boxes (paper Sec. 2.1 "Aura Update",
    Sec. 2.3), with the boxes of the grid sharded over ranks by box_owner.

    Each iteration: send_phase (tera_partition, tera_pack, tera_delta_encode of
    every pair from this rank's agents; pairs of other ranks' boxes are empty),
    the messages for other ranks' boxes move point to point (route_wire), and
    recv_phase decodes every pair with tera_delta_decode on the arena of the
    messages for this rank's boxes (decode_arena).  References stay on the
    rank that holds each side of a pair.  The reference is updated every
    iteration (interval 1).  rebalance() changes the box map and resets the
    references of every pair whose sender or receiver changed rank."""

    def __init__(self, ctx, box_owner, rank: int, world: int, max_agents: int,
                 max_records: int, mode: int = 1):
        from .api import PartitionBuffers
        self.ctx = ctx
        self.rank, self.world = rank, world
        self.mode = mode
        self.n = tuple(int(v) for v in ctx.grid.n)
        self.periodic = int(ctx.grid.periodic)
        self.owner = np.asarray(box_owner, dtype=np.int32)
        self.plan = WirePlan(self.owner, self.n, self.periodic, rank, world)
        P = ctx.n_pairs
        self.P = P
        dev = torch.device("cuda", ctx.device)
        self.dev = dev
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
        self.wire = torch.empty(80 * P + 72 * max_records + 64, **u8)
        self.wire_off = torch.zeros(P + 1, **i64)
        self.wire_len = torch.zeros(P, **i64)
        self.t = 0

    @property
    def cur(self) -> int:
        return self.t % 2

    def send_phase(self, state: dict, stream=None):
        ctx, cur, prv = self.ctx, self.cur, 1 - self.cur
        first = self.t == 0
        self.part.pair_off = self.pair_off[cur]
        ctx.partition(state, self.part, stream)
        ctx.pack(state, self.part, self.rec, stream=stream)
        ctx.delta_encode(self.rec, self.pair_off[cur], None if first else self.ref[prv],
                         None if first else self.pair_off[prv], self.ref[cur], self.wire,
                         self.wire_off, self.wire_len, self.mode, stream=stream)

    def outgoing(self) -> dict:
        return outgoing_wire(self.plan, (self.wire, self.wire_off, self.wire_len))

    def recv_phase(self, received: dict, stream=None):
        ctx, cur, prv = self.ctx, self.cur, 1 - self.cur
        first = self.t == 0
        wire_in, off_in = decode_arena(self.plan, ctx.class_id,
                                       (self.wire, self.wire_off, self.wire_len), received,
                                       self.dev)
        ctx.delta_decode(wire_in, off_in, None if first else self.recv[prv],
                         None if first else self.recv_off[prv], self.recv[cur],
                         self.recv_off[cur], stream=stream)
        self.t += 1

    def step(self, state: dict, transport, stream=None):
        """One iteration of this rank (collective over the transport's ranks)."""
        self.send_phase(state, stream)
        received = _exchange_pairs(transport, self.outgoing(), self.dev) if self.world > 1 else {}
        self.recv_phase(received, stream)

    def rebalance(self, new_owner):
        """Adopt a new box map; pairs this rank now sends whose sender or
        receiver moved are sent raw once."""
        new = np.asarray(new_owner, dtype=np.int32)
        for p in pairs_to_reset(self.owner, new, self.n, self.periodic):
            if new[p // 27] == self.rank:
                self.ctx.reset_reference(int(p))
        self.owner = new
        self.plan = WirePlan(new, self.n, self.periodic, self.rank, self.world)

    def sender_ref(self):
        """New sender reference arena and offsets of the last iteration."""
        last = (self.t - 1) % 2
        return self.ref[last], self.pair_off[last]

    def receiver_ref(self):
        last = (self.t - 1) % 2
        return self.recv[last], self.recv_off[last]


class ShardedMigration:
    """Agent migration of one rank's box-major state (paper Sec. 2.1 "Agent
    Migration") with the boxes sharded over ranks: tera_migrate_send, the
    inboxes of other ranks' boxes move to their owners (route_inboxes), the
    stayers make room for every rank's immigrants (stayer_layout), and
    tera_migrate_recv unpacks the merged inboxes."""

    def __init__(self, ctx, box_owner, rank: int, world: int, max_agents: int,
                 max_leavers: int | None = None):
        from .migrate import Migration
        self.ctx = ctx
        self.rank, self.world = rank, world
        self.mig = Migration(ctx, max_agents, max_leavers)
        self.plan = InboxPlan(box_owner, rank, world)
        self.dev = torch.device("cuda", ctx.device)

    def send_phase(self, prev: dict, box_off_prev, stream=None):
        nxt = self.mig.empty_like(prev)
        off = torch.empty_like(box_off_prev)
        self.mig.send(prev, box_off_prev, nxt, off, stream)
        return nxt, off

    def outgoing(self) -> dict:
        return outgoing_inboxes(self.plan, (self.mig.arena, self.mig.inbox_off))

    def recv_phase(self, sent: dict, sent_off, received: dict, stream=None):
        own = (self.mig.arena, self.mig.inbox_off)
        arena, inbox_off = merge_inboxes(self.plan, self.ctx.class_id, own, received, self.dev)
        final, src, dst = stayer_layout(sent_off, self.mig.inbox_off, inbox_off)
        n = int(final[-1].item())
        out = {k: torch.empty(n, dtype=v.dtype, device=self.dev) for k, v in sent.items()}
        for k in out:
            out[k][dst] = sent[k][src]
        self.mig.recv(out, final, stream, arena=arena, inbox_off=inbox_off)
        return out, final

    def step(self, prev: dict, box_off_prev, transport, stream=None):
        sent, sent_off = self.send_phase(prev, box_off_prev, stream)
        received = _exchange_pairs(transport, self.outgoing(), self.dev) if self.world > 1 else {}
        return self.recv_phase(sent, sent_off, received, stream)
