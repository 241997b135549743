"""Thin wrappers of the C ABI taking torch CUDA tensors (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import _lib
from ._lib import Grid, PartitionOut, Soa, check

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("libtera takes CUDA tensors only (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _host_ptr(t):
    """Address of a pinned host tensor (the device writes it directly)."""
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu" or not t.is_pinned():
        raise TypeError("expected a pinned host tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def soa_from_state(st: dict) -> Soa:
    """Struct-of-arrays view of a state dict (id int64, fields float64, on CUDA)."""
    n = int(st["x"].shape[0])
    s = Soa()
    for f in FIELDS:
        t = st[f]
        if t.shape[0] != n:
            raise ValueError(f"field {f} has {t.shape[0]} agents, expected {n}")
        want = torch.int64 if f == "id" else torch.float64
        if t.dtype != want:
            raise TypeError(f"field {f} must be {want}")
        setattr(s, f, _ptr(t).value if n else None)
    s.n = n
    return s


@dataclasses.dataclass
class PartitionBuffers:
    """Caller-owned outputs of tera_partition (u64 arrays stored as int64)."""
    owner: torch.Tensor       # int32 [n]
    mask: torch.Tensor        # int32 [n] (uint32 bits)
    pair_count: torch.Tensor  # int64 [P]
    pair_off: torch.Tensor    # int64 [P+1]
    pair_idx: torch.Tensor    # int32 [capacity]

    @staticmethod
    def allocate(n_agents: int, n_pairs: int, capacity: int, device) -> "PartitionBuffers":
        z = dict(device=device)
        return PartitionBuffers(
            owner=torch.empty(max(n_agents, 1), dtype=torch.int32, **z),
            mask=torch.empty(max(n_agents, 1), dtype=torch.int32, **z),
            pair_count=torch.empty(n_pairs, dtype=torch.int64, **z),
            pair_off=torch.empty(n_pairs + 1, dtype=torch.int64, **z),
            pair_idx=torch.empty(max(capacity, 1), dtype=torch.int32, **z))

    def c_struct(self) -> PartitionOut:
        o = PartitionOut()
        o.owner = self.owner.data_ptr()
        o.mask = self.mask.data_ptr()
        o.pair_count = self.pair_count.data_ptr()
        o.pair_off = self.pair_off.data_ptr()
        o.pair_idx = self.pair_idx.data_ptr()
        o.idx_capacity = int(self.pair_idx.numel())
        return o


def _tune(tune):
    """tera_tune from (block, ctas_per_sm[, table_records[, team_blocks[, wait_limit_us]]])."""
    if tune is None:
        return None
    v = [int(x) for x in tune] + [0] * (5 - len(tune))
    return _lib.Tune(v[0], v[1], v[2], v[3], v[4], 0)


def ref_schedule(t: int, ref_interval: int):
    """tera_ref_schedule: (output buffer, reference buffer (-1 at t = 0),
    reference iteration) of iteration t with reference interval K."""
    lib = _lib.load()
    ob, rb, ri = C.c_int32(), C.c_int32(), C.c_uint64()
    check(lib.tera_ref_schedule(int(t), int(ref_interval), C.byref(ob), C.byref(rb),
                                C.byref(ri)), "tera_ref_schedule")
    return int(ob.value), int(rb.value), int(ri.value)


def cell_thresholds(lo: float, hi: float, w: float):
    """tera_cell_thresholds: the n + 1 keys of one axis of the predictor's cell
    grid (n = floor((hi - lo) / w) + 1), as a numpy uint64 array."""
    import math
    import numpy as np
    n = int(math.floor((hi - lo) / w)) + 1
    out = np.zeros(n + 1, dtype=np.uint64)
    check(_lib.load().tera_cell_thresholds(float(lo), float(hi), float(w), n,
                                           out.ctypes.data_as(C.c_void_p)),
          "tera_cell_thresholds")
    return out


AXIS_BUCKETS = 8192  # TERA_AXIS_BUCKETS


def axis_buckets(lo, hi, n, w, periodic: int = 0):
    """tera_axis_buckets: (tab, flo, fs) of the grid's classification tables
    (tab: uint8 array of shape (3, AXIS_BUCKETS); flo, fs: float32 arrays of 3),
    or None when the grid gets no tables."""
    import numpy as np
    g = Grid()
    for a in range(3):
        g.lo[a], g.hi[a], g.n[a] = float(lo[a]), float(hi[a]), int(n[a])
    g.w = float(w)
    g.periodic = int(periodic)
    tab = np.zeros((3, AXIS_BUCKETS), dtype=np.uint8)
    flo = np.zeros(3, dtype=np.float32)
    fs = np.zeros(3, dtype=np.float32)
    on = C.c_int(0)
    check(_lib.load().tera_axis_buckets(C.byref(g), tab.ctypes.data_as(C.c_void_p),
                                        flo.ctypes.data_as(C.c_void_p),
                                        fs.ctypes.data_as(C.c_void_p), C.byref(on)),
          "tera_axis_buckets")
    return (tab, flo, fs) if on.value else None


class Context:
    """One partitioning grid on one GPU (owns scratch, hash table, status word)."""

    def __init__(self, lo, hi, n, w, device: int = 0, class_id: int = 1, periodic: int = 0):
        """``periodic``: bit a makes axis a toroidal (box n-1 next to box 0)."""
        self.lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("libtera needs a CUDA device (there is no CPU path)")
        g = Grid()
        for a in range(3):
            g.lo[a], g.hi[a], g.n[a] = float(lo[a]), float(hi[a]), int(n[a])
        g.w = float(w)
        g.periodic = int(periodic)
        self.grid = g
        self.device = int(device)
        self.class_id = int(class_id)
        h = C.c_void_p()
        check(self.lib.tera_ctx_create(C.byref(h), C.byref(g), self.device, self.class_id),
              "tera_ctx_create")
        self.h = h
        self.n_pairs = int(self.lib.tera_n_pairs(h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tera_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(self.lib.tera_ctx_launches(self.h))

    def profile(self, enable: bool = True):
        """Bracket every kernel launch with CUDA events (per-kernel timing)."""
        check(self.lib.tera_ctx_profile(self.h, 1 if enable else 0), "tera_ctx_profile")

    def profile_table(self, reset: bool = False) -> dict:
        """{kernel name: (launches, total ms)} of the launches recorded so far."""
        check(self.lib.tera_ctx_profile_collect(self.h), "tera_ctx_profile_collect")
        out = {}
        for i in range(self.lib.tera_ctx_profile_entries(self.h)):
            name = C.c_char_p()
            n = C.c_uint64()
            ms = C.c_double()
            check(self.lib.tera_ctx_profile_entry(self.h, i, C.byref(name), C.byref(n),
                                                  C.byref(ms)), "tera_ctx_profile_entry")
            out[name.value.decode()] = (int(n.value), float(ms.value))
        if reset:
            check(self.lib.tera_ctx_profile_reset(self.h), "tera_ctx_profile_reset")
        return out

    def stats(self, reset: bool = False, stream=None) -> dict:
        """Device-side totals since the last reset (see tera_stats)."""
        s = _lib.Stats()
        check(self.lib.tera_ctx_stats(self.h, C.byref(s), 1 if reset else 0, _stream(stream)),
              "tera_ctx_stats")
        return {k: int(getattr(s, k)) for k, _ in s._fields_}

    def reserve(self, max_agents: int, max_records: int):
        check(self.lib.tera_ctx_reserve(self.h, int(max_agents), int(max_records)),
              "tera_ctx_reserve")

    def status(self, stream=None, raise_on_error=True):
        req = C.c_uint64(0)
        st = self.lib.tera_ctx_status(self.h, C.byref(req), _stream(stream))
        if st != _lib.OK and raise_on_error:
            raise _lib.TeraError(st, "device status", int(req.value))
        return st, int(req.value)

    def partition(self, state: dict, out: PartitionBuffers, stream=None):
        soa = soa_from_state(state)
        o = out.c_struct()
        check(self.lib.tera_partition(self.h, C.byref(soa), C.byref(o), _stream(stream)),
              "tera_partition")

    def pack(self, state: dict, part: PartitionBuffers, arena: torch.Tensor, pair_begin=0,
             pair_end=None, stream=None):
        soa = soa_from_state(state)
        o = part.c_struct()
        pe = self.n_pairs if pair_end is None else pair_end
        check(self.lib.tera_pack(self.h, C.byref(soa), C.byref(o), pair_begin, pe, _ptr(arena),
                                 arena.numel() // 64, _stream(stream)), "tera_pack")

    def pack_ids(self, state: dict, part: PartitionBuffers, arena: torch.Tensor,
                 rec_ids: torch.Tensor, stream=None):
        """tera_pack of every pair plus the records' id column (tera_pack_ids)."""
        soa = soa_from_state(state)
        o = part.c_struct()
        check(self.lib.tera_pack_ids(self.h, C.byref(soa), C.byref(o), _ptr(arena),
                                     arena.numel() // 64, _ptr(rec_ids), _stream(stream)),
              "tera_pack_ids")

    def delta_encode(self, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire, wire_off,
                     wire_len, mode=_lib.MODE_XOR, pair_begin=0, pair_end=None, stream=None):
        pe = self.n_pairs if pair_end is None else pair_end
        check(self.lib.tera_delta_encode(
            self.h, _ptr(rec_arena), _ptr(pair_off), _ptr(ref_prev), _ptr(ref_off_prev),
            pair_begin, pe, _ptr(ref_next), _ptr(wire), wire.numel(), _ptr(wire_off),
            _ptr(wire_len), int(mode), _stream(stream)), "tera_delta_encode")

    def delta_decode(self, wire, wire_off, ref_prev, ref_off_prev, recv, recv_off, pair_begin=0,
                     pair_end=None, stream=None):
        pe = self.n_pairs if pair_end is None else pair_end
        check(self.lib.tera_delta_decode(
            self.h, _ptr(wire), _ptr(wire_off), _ptr(ref_prev), _ptr(ref_off_prev), pair_begin,
            pe, _ptr(recv), recv.numel() // 64, _ptr(recv_off), _stream(stream)),
            "tera_delta_decode")

    def codec_batched(self, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire, wire_off,
                      wire_len, recv_prev, recv_off_prev, recv, recv_off, mode=_lib.MODE_XOR,
                      tune=None, stream=None, ids=None):
        """Encode + decode of every pair in one persistent launch (tera_codec_batched;
        with ids = dict(msg, ref_prev, ref_next) of id columns, tera_codec_batched_ids)."""
        t = _tune(tune)
        if ids is not None:
            c = _lib.Ids(_ptr(ids["msg"]).value,
                         None if ids.get("ref_prev") is None else _ptr(ids["ref_prev"]).value,
                         _ptr(ids["ref_next"]).value)
            check(self.lib.tera_codec_batched_ids(
                self.h, _ptr(rec_arena), _ptr(pair_off), _ptr(ref_prev), _ptr(ref_off_prev),
                _ptr(ref_next), _ptr(wire), wire.numel(), _ptr(wire_off), _ptr(wire_len),
                _ptr(recv_prev), _ptr(recv_off_prev), _ptr(recv), recv.numel() // 64,
                _ptr(recv_off), int(mode), C.byref(t) if t is not None else None, C.byref(c),
                _stream(stream)), "tera_codec_batched_ids")
            return
        check(self.lib.tera_codec_batched(
            self.h, _ptr(rec_arena), _ptr(pair_off), _ptr(ref_prev), _ptr(ref_off_prev),
            _ptr(ref_next), _ptr(wire), wire.numel(), _ptr(wire_off), _ptr(wire_len),
            _ptr(recv_prev), _ptr(recv_off_prev), _ptr(recv), recv.numel() // 64, _ptr(recv_off),
            int(mode), C.byref(t) if t is not None else None, _stream(stream)),
            "tera_codec_batched")

    @staticmethod
    def _pred(pred):
        """tera_predictor from a dict(params, hist_prev, hist_next, samples, allow_residual)."""
        if pred is None:
            return None
        p = _lib.Predictor()
        for k in ("params", "hist_prev", "hist_next", "samples"):
            t = pred.get(k)
            setattr(p, k, None if t is None else _ptr(t).value)
        p.allow_residual = 1 if pred.get("allow_residual") else 0
        return p

    def delta_encode_pred(self, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                          wire_off, wire_len, pred: dict, mode=_lib.MODE_XOR, pair_begin=0,
                          pair_end=None, stream=None):
        pe = self.n_pairs if pair_end is None else pair_end
        p = self._pred(pred)
        check(self.lib.tera_delta_encode_pred(
            self.h, _ptr(rec_arena), _ptr(pair_off), _ptr(ref_prev), _ptr(ref_off_prev),
            pair_begin, pe, _ptr(ref_next), _ptr(wire), wire.numel(), _ptr(wire_off),
            _ptr(wire_len), int(mode), C.byref(p), _stream(stream)), "tera_delta_encode_pred")

    def delta_decode_pred(self, wire, wire_off, ref_prev, ref_off_prev, recv, recv_off,
                          pred: dict, pair_begin=0, pair_end=None, stream=None):
        pe = self.n_pairs if pair_end is None else pair_end
        p = self._pred(pred)
        check(self.lib.tera_delta_decode_pred(
            self.h, _ptr(wire), _ptr(wire_off), _ptr(ref_prev), _ptr(ref_off_prev), pair_begin,
            pe, _ptr(recv), recv.numel() // 64, _ptr(recv_off), C.byref(p), _stream(stream)),
            "tera_delta_decode_pred")

    def codec_batched_pred(self, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                           wire_off, wire_len, recv_prev, recv_off_prev, recv, recv_off,
                           enc_pred: dict, dec_pred: dict, mode=_lib.MODE_XOR, tune=None,
                           stream=None):
        t = _tune(tune)
        pe, pd = self._pred(enc_pred), self._pred(dec_pred)
        check(self.lib.tera_codec_batched_pred(
            self.h, _ptr(rec_arena), _ptr(pair_off), _ptr(ref_prev), _ptr(ref_off_prev),
            _ptr(ref_next), _ptr(wire), wire.numel(), _ptr(wire_off), _ptr(wire_len),
            _ptr(recv_prev), _ptr(recv_off_prev), _ptr(recv), recv.numel() // 64, _ptr(recv_off),
            int(mode), C.byref(t) if t is not None else None,
            C.byref(pe) if pe is not None else None, C.byref(pd) if pd is not None else None,
            _stream(stream)), "tera_codec_batched_pred")

    def mlp_grad(self, samples, params, grad, stream=None) -> int:
        nv = C.c_uint64()
        check(self.lib.tera_mlp_grad(self.h, _ptr(samples), samples.numel() // 12, _ptr(params),
                                     _ptr(grad), C.byref(nv), _stream(stream)), "tera_mlp_grad")
        return int(nv.value)

    def mlp_train(self, samples, params, steps, batch, lr, clip=1.0, stream=None) -> int:
        nv = C.c_uint64()
        check(self.lib.tera_mlp_train(self.h, _ptr(samples), samples.numel() // 12, _ptr(params),
                                      int(steps), int(batch), float(lr), float(clip), C.byref(nv),
                                      _stream(stream)), "tera_mlp_train")
        return int(nv.value)

    def unpack_inplace(self, arena: torch.Tensor, byte_offset: int, length: int, stream=None):
        """Header check of one TAIO buffer; returns (device address of record 0, count)."""
        view = C.c_void_p()
        cnt = C.c_uint64()
        check(self.lib.tera_unpack_inplace(C.c_void_p(arena.data_ptr() + byte_offset), length,
                                           self.class_id, C.byref(view), C.byref(cnt),
                                           _stream(stream)), "tera_unpack_inplace")
        return int(view.value or 0), int(cnt.value)

    def unpack_validate(self, arena, off, stream=None):
        check(self.lib.tera_unpack_validate(self.h, _ptr(arena), _ptr(off), _stream(stream)),
              "tera_unpack_validate")

    def wire_to_host(self, wire, wire_off, host_out, host_count, stream=None):
        """Wire messages wire[0, wire_off[-1]) into pinned host memory host_out
        (uint8) and the byte count into host_count (pinned int64, 1 element),
        with the length read on the device (tera_wire_to_host)."""
        check(self.lib.tera_wire_to_host(self.h, _ptr(wire), _ptr(wire_off), _host_ptr(host_out),
                                         host_out.numel(), _host_ptr(host_count),
                                         _stream(stream)),
              "tera_wire_to_host")

    def reset_reference(self, pair: int):
        check(self.lib.tera_reset_reference(self.h, int(pair)), "tera_reset_reference")
