"""Oracle for the aura-exchange codec (TeraAgent, Sec. 2.1, 2.2.1, 2.3).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path
(``paper_2509_24063_gb300``) never does.  It is a thin ctypes wrapper over the
plain single-threaded C code in ``tera_oracle.c`` (built with gcc, no CUDA).

Every array here is a host numpy array.  Record arenas are ``uint8`` arrays of
64-byte units; pair ``p`` occupies units ``[off[p] + p, off[p+1] + p + 1)``:
one 64-byte buffer header, then its records.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "tera_oracle.c"), os.path.join(HERE, "tera_oracle_mt.c"),
           os.path.join(HERE, "mlp_oracle.c")]

OK, EINVAL, ENOMEM, ECAPACITY, ECORRUPT, EDOMAIN, EREFMISMATCH = range(7)
MODE_RAW, MODE_XOR, MODE_RESIDUAL = 0, 1, 2
NPARAM = 8 * 64 + 64 + 64 * 64 + 64 + 3 * 64 + 3
HIST = 48
REC = 64
HDR = 64

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction, no fast-math)."""
    newest = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "tera_oracle.h")])
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", "-o", tmp] + SOURCES + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Grid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int32 * 3),
                ("w", C.c_double), ("periodic", C.c_uint32), ("reserved", C.c_uint32)]


def make_grid(lo, hi, n, w, periodic: int = 0) -> Grid:
    """Grid of Sec. 2.1; bit a of ``periodic`` makes axis a toroidal (Sec. 2.5)."""
    g = Grid()
    for a in range(3):
        g.lo[a], g.hi[a], g.n[a] = float(lo[a]), float(hi[a]), int(n[a])
    g.w = float(w)
    g.periodic = int(periodic)
    return g


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            P = C.c_void_p
            u64, i64, u32, i32 = C.c_uint64, C.c_int64, C.c_uint32, C.c_int32
            G = C.POINTER(Grid)
            L.or_grid_check.argtypes = [G]
            L.or_axis_edges.argtypes = [G, C.c_int, P]
            L.or_axis_edges.restype = None
            L.or_classify.argtypes = [G, P, P, P, i64, P, P]
            L.or_pair_lists.argtypes = [G, P, P, i64, P, P, P, u64]
            L.or_pack.argtypes = [P, P, u64, P, P, u32, P]
            L.or_pack.restype = None
            L.or_encode_pair.argtypes = [P, u64, P, u64, u32, u32, u32, P, u64, P, P]
            L.or_decode_pair.argtypes = [P, u64, P, u64, u32, u32, P, u64, P]
            L.or_wire_slabs.argtypes = [u64, P, P, P]
            L.or_wire_slabs.restype = None
            L.or_encode_all.argtypes = [u64, u32, u32, P, P, P, P, P, P, P, P, P]
            L.or_decode_all.argtypes = [u64, u32, P, P, P, P, P, u64, P]
            L.or_exchange_iteration.argtypes = [G, P, P, i64, u32, u32, P, P, P, P, P, P, P,
                                                P, P, u64, P, P, P, P, P, P, u64, P, P]
            L.or_exchange_iteration_mt.argtypes = [G, P, P, i64, u32, u32, P, P, P, P, P, P, P,
                                                   P, P, u64, P, P, P, P, P, P, u64, P, P,
                                                   C.c_int]
            L.or_delta_records.argtypes = [P, u64, P, u64, P, C.POINTER(C.c_uint64)]
            L.or_migrate_inbox_bit.argtypes = [G, i32, i32]
            L.or_migrate_send.argtypes = [G, P, P, i64, P, u32, P, P, u64, P, P, P]
            L.or_migrate_recv.argtypes = [G, P, P, u32, P, P, P]
            D3 = C.POINTER(C.c_double)
            L.or_mlp_nparam.argtypes = []
            L.or_mlp_infer_f32.argtypes = [P, P, P]
            L.or_mlp_infer_f32.restype = None
            L.or_mlp_loss_grad_f64.argtypes = [P, P, P, i64, P]
            L.or_mlp_loss_grad_f64.restype = C.c_double
            L.or_mlp_sgd_f64.argtypes = [P, P, C.c_double]
            L.or_mlp_sgd_f64.restype = None
            L.or_mlp_sgd_clip_f64.argtypes = [P, P, C.c_double, C.c_double]
            L.or_mlp_sgd_clip_f64.restype = None
            L.or_zigzag.argtypes = [u64]
            L.or_zigzag.restype = u64
            L.or_unzigzag.argtypes = [u64]
            L.or_unzigzag.restype = u64
            L.or_cell_counts.argtypes = [P, u64, D3, C.c_double, P]
            L.or_cell_counts.restype = None
            L.or_features.argtypes = [P, P, u32, P]
            L.or_predict.argtypes = [P, P, P, u32, P]
            L.or_hist_next.argtypes = [P, P, P]
            L.or_hist_next.restype = None
            L.or_sample.argtypes = [P, P, P, u32, P, P]
            L.or_encode_pair_pred.argtypes = [P, u64, P, u64, P, P, D3, C.c_double, C.c_int, u32,
                                              u32, P, u64, P, P, P]
            L.or_decode_pair_pred.argtypes = [P, u64, P, u64, P, P, D3, C.c_double, u32, u32, P,
                                              u64, P, P]
            L.or_encode_all_pred.argtypes = [u64, u32, C.c_int, P, P, P, P, P, P, D3, C.c_double,
                                             P, P, P, P, P]
            L.or_decode_all_pred.argtypes = [u64, u32, P, P, P, P, P, P, D3, C.c_double, P, u64,
                                             P, P]
            for f in ("or_grid_check", "or_classify", "or_pair_lists", "or_encode_pair",
                      "or_decode_pair", "or_encode_all", "or_decode_all",
                      "or_exchange_iteration", "or_exchange_iteration_mt", "or_mlp_nparam", "or_features", "or_predict",
                      "or_sample", "or_encode_pair_pred", "or_decode_pair_pred",
                      "or_encode_all_pred", "or_decode_all_pred", "or_migrate_inbox_bit",
                      "or_delta_records",
                      "or_migrate_send", "or_migrate_recv"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def n_pairs(grid: Grid) -> int:
    return int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2]) * 27


def grid_check(grid: Grid) -> int:
    return lib().or_grid_check(C.byref(grid))


def axis_edges(grid: Grid, axis: int) -> np.ndarray:
    e = np.zeros(int(grid.n[axis]) + 1, dtype=np.float64)
    lib().or_axis_edges(C.byref(grid), axis, _p(e))
    return e


def classify(grid: Grid, x, y, z, threads: int = 1):
    """or_classify; threads > 1 classifies contiguous agent ranges on host
    threads (every agent independently, so the outputs are the same)."""
    x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
    n = x.shape[0]
    owner = np.zeros(n, dtype=np.int32)
    mask = np.zeros(n, dtype=np.uint32)
    if threads <= 1 or n < 65536:
        st = lib().or_classify(C.byref(grid), _p(x), _p(y), _p(z), n, _p(owner), _p(mask))
        return st, owner, mask
    import concurrent.futures as cf
    step = -(-n // threads)
    L = lib()

    def part(a):
        b = min(n, a + step)
        return L.or_classify(C.byref(grid), _p(x[a:b]), _p(y[a:b]), _p(z[a:b]), b - a,
                             _p(owner[a:b]), _p(mask[a:b]))
    with cf.ThreadPoolExecutor(threads) as ex:
        sts = list(ex.map(part, range(0, n, step)))
    st = next((s for s in sts if s != OK), OK)
    return st, owner, mask


def _popcount(words) -> int:
    """Set bits of a uint32 array (how many records the masks give)."""
    if hasattr(np, "bitwise_count"):
        return int(np.bitwise_count(words).sum(dtype=np.uint64))
    return int(np.unpackbits(words.view(np.uint8)).sum())


def pair_lists(grid: Grid, owner, mask, idx_capacity=None):
    P = n_pairs(grid)
    n = owner.shape[0]
    cnt = np.zeros(P, dtype=np.uint64)
    off = np.zeros(P + 1, dtype=np.uint64)
    total = int(sum(bin(int(m)).count("1") for m in mask[owner >= 0])) if n < 4096 else \
        _popcount(mask[owner >= 0])
    cap = total if idx_capacity is None else idx_capacity
    idx = np.zeros(max(cap, 1), dtype=np.uint32)
    st = lib().or_pair_lists(C.byref(grid), _p(np.ascontiguousarray(owner)),
                             _p(np.ascontiguousarray(mask)), n, _p(cnt), _p(off), _p(idx), cap)
    return st, cnt, off, idx[:int(off[-1])] if st == OK else idx


def soa_cols(soa: dict):
    """The seven float64 columns in record word order w1..w7."""
    return [np.ascontiguousarray(soa[k], dtype=np.float64)
            for k in ("x", "y", "z", "diameter", "volume", "adherence", "density")]


def pack(soa: dict, pair_off, pair_idx, class_id: int = 1) -> np.ndarray:
    P = pair_off.shape[0] - 1
    units = int(pair_off[-1]) + P
    arena = np.zeros(units * REC, dtype=np.uint8)
    ids = np.ascontiguousarray(soa["id"], dtype=np.uint64)
    cols = soa_cols(soa)
    arr = (C.c_void_p * 7)(*[c.ctypes.data for c in cols])
    idx = np.ascontiguousarray(pair_idx, dtype=np.uint32)
    if idx.size == 0:
        idx = np.zeros(1, dtype=np.uint32)
    lib().or_pack(_p(ids), arr, P, _p(np.ascontiguousarray(pair_off)), _p(idx), class_id,
                  _p(arena))
    return arena


def encode_pair(msg: np.ndarray, ref: np.ndarray, class_id=1, mode=MODE_XOR, pair=0):
    """msg, ref: (m, 8) / (r, 8) uint64 records.  Returns (status, wire bytes, ref_next)."""
    msg = np.ascontiguousarray(msg, dtype=np.uint64).reshape(-1, 8)
    ref = np.ascontiguousarray(ref, dtype=np.uint64).reshape(-1, 8)
    m, r = msg.shape[0], ref.shape[0]
    cap = 64 + 4 * (r + m) + 64 * m + 16
    wire = np.zeros(cap, dtype=np.uint8)
    wl = np.zeros(1, dtype=np.uint64)
    nxt = np.zeros((max(m, 1), 8), dtype=np.uint64)
    st = lib().or_encode_pair(_p(msg), m, _p(ref), r, class_id, mode, pair, _p(wire), cap,
                              _p(wl), _p(nxt))
    return st, wire[:int(wl[0])].copy(), nxt[:m].copy()


def decode_pair(wire: np.ndarray, ref: np.ndarray, class_id=1, pair=0, out_cap=None):
    wire = np.ascontiguousarray(wire, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint64).reshape(-1, 8)
    cap = out_cap if out_cap is not None else max(1, wire.size // 4 + ref.shape[0])
    out = np.zeros((max(cap, 1), 8), dtype=np.uint64)
    m = np.zeros(1, dtype=np.uint64)
    buf = wire if wire.size else np.zeros(1, dtype=np.uint8)
    st = lib().or_decode_pair(_p(buf), wire.size, _p(ref), ref.shape[0], class_id, pair,
                              _p(out), cap, _p(m))
    return st, out[:int(m[0])].copy()


def delta_records(msg: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Difference-serialized message before compression (Sec. 2.3 B and C):
    (r + a, 8) uint64 words, XOR for matched slots, zeros for placeholders,
    then the records absent from the reference."""
    msg = np.ascontiguousarray(msg, dtype=np.uint64).reshape(-1, 8)
    ref = np.ascontiguousarray(ref, dtype=np.uint64).reshape(-1, 8)
    out = np.zeros((len(msg) + len(ref), 8), dtype=np.uint64)
    ne = C.c_uint64(0)
    st = lib().or_delta_records(_p(msg), len(msg), _p(ref), len(ref), _p(out), C.byref(ne))
    assert st == OK, st
    return out[:ne.value]


def wire_slabs(pair_off, ref_off=None) -> np.ndarray:
    P = pair_off.shape[0] - 1
    wo = np.zeros(P + 1, dtype=np.uint64)
    lib().or_wire_slabs(P, _p(np.ascontiguousarray(pair_off, dtype=np.uint64)),
                        None if ref_off is None else _p(np.ascontiguousarray(ref_off,
                                                                             dtype=np.uint64)),
                        _p(wo))
    return wo


def encode_all(rec_arena, pair_off, ref_arena=None, ref_off=None, class_id=1, mode=MODE_XOR,
               reset=None):
    """Returns (status, wire, wire_off, wire_len, ref_next arena)."""
    P = pair_off.shape[0] - 1
    wo = wire_slabs(pair_off, ref_off)
    wire = np.zeros(max(int(wo[-1]), 1), dtype=np.uint8)
    wl = np.zeros(P, dtype=np.uint64)
    nxt = np.zeros((int(pair_off[-1]) + P) * REC, dtype=np.uint8)
    rs = None if reset is None else np.ascontiguousarray(reset, dtype=np.uint8)
    st = lib().or_encode_all(P, class_id, mode, _p(rec_arena), _p(pair_off),
                             _p(ref_arena), _p(ref_off), _p(rs), _p(wire), _p(wo), _p(wl),
                             _p(nxt))
    return st, wire, wo, wl, nxt


def decode_all(wire, wire_off, ref_arena=None, ref_off=None, class_id=1, cap_units=None):
    """Returns (status, recv arena, recv_off)."""
    P = wire_off.shape[0] - 1
    if cap_units is None:
        cap_units = P + int(wire.size // 4 + (0 if ref_off is None else int(ref_off[-1])) + 1)
    recv = np.zeros(cap_units * REC, dtype=np.uint8)
    ro = np.zeros(P + 1, dtype=np.uint64)
    st = lib().or_decode_all(P, class_id, _p(wire), _p(wire_off), _p(ref_arena), _p(ref_off),
                             _p(recv), cap_units, _p(ro))
    used = (int(ro[-1]) + P) * REC
    return st, recv[:used].copy(), ro


def arena_pair(arena: np.ndarray, off: np.ndarray, p: int) -> np.ndarray:
    """Records of pair p (excluding its header) as an (n, 8) uint64 view."""
    a, b = int(off[p]) + p + 1, int(off[p + 1]) + p + 1
    return arena[a * REC:b * REC].view(np.uint64).reshape(-1, 8)


def exchange_iteration(grid: Grid, soa: dict, ref=None, recv_ref=None, class_id=1,
                       mode=MODE_XOR, threads: int = 1):
    """One whole iteration (classify, lists, pack, encode, decode) in one C call.

    ref / recv_ref: (arena, off) of the sender / receiver reference or None.
    threads > 1 spreads agents and pairs over that many host threads
    (or_exchange_iteration_mt; same outputs).
    Returns a dict of every output plus per-step seconds."""
    n = int(soa["x"].shape[0])
    P = n_pairs(grid)
    ids = np.ascontiguousarray(soa["id"], dtype=np.uint64)
    cols = soa_cols(soa)
    arr = (C.c_void_p * 7)(*[c.ctypes.data for c in cols])
    st, owner, mask = classify(grid, cols[0], cols[1], cols[2])
    total = _popcount(mask[owner >= 0]) if n else 0
    cap = max(total, 1)
    r_tot = 0 if ref is None else int(ref[1][-1])
    owner = np.zeros(n, dtype=np.int32)
    mask = np.zeros(n, dtype=np.uint32)
    cnt = np.zeros(P, dtype=np.uint64)
    off = np.zeros(P + 1, dtype=np.uint64)
    idx = np.zeros(cap, dtype=np.uint32)
    rec = np.zeros((total + P) * REC, dtype=np.uint8)
    wo = np.zeros(P + 1, dtype=np.uint64)
    wire = np.zeros(64 * P + 4 * (r_tot + total) + 64 * total + 16 * P + 16, dtype=np.uint8)
    wl = np.zeros(P, dtype=np.uint64)
    nxt = np.zeros((total + P) * REC, dtype=np.uint8)
    recv = np.zeros((total + P) * REC, dtype=np.uint8)
    ro = np.zeros(P + 1, dtype=np.uint64)
    ts = np.zeros(4, dtype=np.float64)
    ra, rof = (None, None) if ref is None else ref
    va, vof = (None, None) if recv_ref is None else recv_ref
    args = (C.byref(grid), _p(ids), arr, n, class_id, mode, _p(ra), _p(rof), _p(va), _p(vof),
            _p(owner), _p(mask), _p(cnt), _p(off), _p(idx), cap, _p(rec), _p(wire), _p(wo),
            _p(wl), _p(nxt), _p(recv), total + P, _p(ro), _p(ts))
    if threads > 1:
        st = lib().or_exchange_iteration_mt(*args, int(threads))
    else:
        st = lib().or_exchange_iteration(*args)
    return dict(status=st, owner=owner, mask=mask, pair_count=cnt, pair_off=off,
                pair_idx=idx[:total], rec=rec, wire=wire, wire_off=wo, wire_len=wl,
                ref_next=nxt, recv=recv, recv_off=ro, t_steps=ts)


# ---------------- agent migration (Sec. 2.1 "Agent Migration") ----------------

COLS = ("x", "y", "z", "diameter", "volume", "adherence", "density")


def inbox_bit(grid: Grid, s: int, d: int) -> int:
    """Side b of box d that an agent from box s arrives from (13: not a neighbour)."""
    return int(lib().or_migrate_inbox_bit(C.byref(grid), int(s), int(d)))


def migrate(grid: Grid, soa: dict, box_off_prev, class_id=1, arena_units=None):
    """Send and receive of one migration step of a box-major state.

    Returns dict(status, inbox_off, arena, box_off_next, next) where next is
    the box-major state after migration (same keys as soa), arena the raw
    TAIO inboxes (pair field = inbox index q = d*27 + b)."""
    n = int(soa["x"].shape[0])
    nb = int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2])
    Q = nb * 27
    ids = np.ascontiguousarray(soa["id"], dtype=np.uint64)
    cols = soa_cols(soa)
    arr = (C.c_void_p * 7)(*[c.ctypes.data for c in cols])
    bo = np.ascontiguousarray(box_off_prev, dtype=np.uint64)
    assert bo.shape[0] == nb + 1
    units = n + Q if arena_units is None else int(arena_units)
    arena = np.zeros(max(units, 1) * REC, dtype=np.uint8)
    inbox_off = np.zeros(Q + 1, dtype=np.uint64)
    box_next = np.zeros(nb + 1, dtype=np.uint64)
    id_next = np.zeros(n, dtype=np.uint64)
    cn = [np.zeros(n, dtype=np.float64) for _ in range(7)]
    arr_n = (C.c_void_p * 7)(*[c.ctypes.data for c in cn])
    st = lib().or_migrate_send(C.byref(grid), _p(ids), arr, n, _p(bo), class_id, _p(inbox_off),
                               _p(arena), units, _p(box_next), _p(id_next), arr_n)
    if st == OK:
        st = lib().or_migrate_recv(C.byref(grid), _p(arena), _p(inbox_off), class_id,
                                   _p(box_next), _p(id_next), arr_n)
    nxt = {"id": id_next}
    nxt.update({k: c for k, c in zip(COLS, cn)})
    return dict(status=st, inbox_off=inbox_off, arena=arena, box_off_next=box_next, next=nxt)


def migrate_recv(grid: Grid, arena, inbox_off, box_off_next, next_soa: dict, class_id=1) -> int:
    """Deserialize the inboxes into next_soa (modified in place); returns the status."""
    ids = next_soa["id"]
    cn = [next_soa[k] for k in COLS]
    for c in [ids] + cn:
        assert c.flags["C_CONTIGUOUS"]
    arr_n = (C.c_void_p * 7)(*[c.ctypes.data for c in cn])
    return int(lib().or_migrate_recv(C.byref(grid), _p(np.ascontiguousarray(arena)),
                                     _p(np.ascontiguousarray(inbox_off, dtype=np.uint64)),
                                     class_id,
                                     _p(np.ascontiguousarray(box_off_next, dtype=np.uint64)),
                                     _p(ids), arr_n))


# ---------------- learned predictor and residual mode ----------------

def _d3(v):
    return (C.c_double * 3)(*[float(t) for t in v])


def mlp_infer(params, x):
    """float32 inference (fixed fmaf order) of one feature vector."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(3, dtype=np.float32)
    lib().or_mlp_infer_f32(_p(p), _p(x), _p(out))
    return out


def mlp_loss_grad(params64, X, Y, with_grad=True):
    p = np.ascontiguousarray(params64, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    g = np.zeros(NPARAM, dtype=np.float64) if with_grad else None
    loss = lib().or_mlp_loss_grad_f64(_p(p), _p(X), _p(Y), X.shape[0], _p(g))
    return loss, g


def mlp_sgd_clip(params64, grad64, lr, clip):
    """One float64 SGD step with global-norm clipping (a new array)."""
    p = np.ascontiguousarray(params64, dtype=np.float64).copy()
    g = np.ascontiguousarray(grad64, dtype=np.float64)
    lib().or_mlp_sgd_clip_f64(_p(p), _p(g), float(lr), float(clip))
    return p


def zigzag(d):
    return int(lib().or_zigzag(d & (2**64 - 1)))


def unzigzag(z):
    return int(lib().or_unzigzag(z & (2**64 - 1)))


def cell_counts(ref_recs, lo, w):
    ref = np.ascontiguousarray(ref_recs, dtype=np.uint64).reshape(-1, 8)
    cnt = np.zeros(max(ref.shape[0], 1), dtype=np.uint32)
    lib().or_cell_counts(_p(ref), ref.shape[0], _d3(lo), float(w), _p(cnt))
    return cnt[:ref.shape[0]]


def features(rec, hist, ncount):
    rec = np.ascontiguousarray(rec, dtype=np.uint64)
    hist = np.ascontiguousarray(hist, dtype=np.uint8)
    f = np.zeros(8, dtype=np.float32)
    ok = lib().or_features(_p(rec), _p(hist), int(ncount), _p(f))
    return ok, f


def hist_next(rec=None, hist=None):
    out = np.zeros(HIST, dtype=np.uint8)
    lib().or_hist_next(None if rec is None else _p(np.ascontiguousarray(rec, dtype=np.uint64)),
                       None if hist is None else _p(np.ascontiguousarray(hist, dtype=np.uint8)),
                       _p(out))
    return out


def encode_pair_pred(msg, ref, hist, params, lo, w, allow_residual=True, class_id=1, pair=0):
    msg = np.ascontiguousarray(msg, dtype=np.uint64).reshape(-1, 8)
    ref = np.ascontiguousarray(ref, dtype=np.uint64).reshape(-1, 8)
    m, r = msg.shape[0], ref.shape[0]
    cap = 64 + 4 * (r + m) + 64 * m + 16
    wire = np.zeros(cap, dtype=np.uint8)
    wl = np.zeros(1, dtype=np.uint64)
    nxt = np.zeros((max(m, 1), 8), dtype=np.uint64)
    hn = np.zeros((max(m, 1), HIST), dtype=np.uint8)
    h = None if hist is None else np.ascontiguousarray(hist, dtype=np.uint8)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    st = lib().or_encode_pair_pred(_p(msg), m, _p(ref), r, _p(h), _p(pr), _d3(lo), float(w),
                                   1 if allow_residual else 0, class_id, pair, _p(wire), cap,
                                   _p(wl), _p(nxt), _p(hn))
    return st, wire[:int(wl[0])].copy(), nxt[:m].copy(), hn[:m].copy()


def decode_pair_pred(wire, ref, hist, params, lo, w, class_id=1, pair=0, out_cap=None):
    wire = np.ascontiguousarray(wire, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint64).reshape(-1, 8)
    cap = out_cap if out_cap is not None else max(1, wire.size // 4 + ref.shape[0])
    out = np.zeros((max(cap, 1), 8), dtype=np.uint64)
    hn = np.zeros((max(cap, 1), HIST), dtype=np.uint8)
    m = np.zeros(1, dtype=np.uint64)
    h = None if hist is None else np.ascontiguousarray(hist, dtype=np.uint8)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    buf = wire if wire.size else np.zeros(1, dtype=np.uint8)
    st = lib().or_decode_pair_pred(_p(buf), wire.size, _p(ref), ref.shape[0], _p(h), _p(pr),
                                   _d3(lo), float(w), class_id, pair, _p(out), cap, _p(m), _p(hn))
    k = int(m[0])
    return st, out[:k].copy(), hn[:k].copy()


def encode_all_pred(rec_arena, pair_off, ref_arena, ref_off, hist, params, lo, w,
                    allow_residual=True, class_id=1):
    """Returns (status, wire, wire_off, wire_len, ref_next, hist_next)."""
    P = pair_off.shape[0] - 1
    wo = wire_slabs(pair_off, ref_off)
    wire = np.zeros(max(int(wo[-1]), 1), dtype=np.uint8)
    wl = np.zeros(P, dtype=np.uint64)
    E = int(pair_off[-1])
    nxt = np.zeros((E + P) * REC, dtype=np.uint8)
    hn = np.zeros(max(E, 1) * HIST, dtype=np.uint8)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    st = lib().or_encode_all_pred(P, class_id, 1 if allow_residual else 0, _p(rec_arena),
                                  _p(pair_off), _p(ref_arena), _p(ref_off), _p(hist), _p(pr),
                                  _d3(lo), float(w), _p(wire), _p(wo), _p(wl), _p(nxt), _p(hn))
    return st, wire, wo, wl, nxt, hn[:E * HIST]


def decode_all_pred(wire, wire_off, ref_arena, ref_off, hist, params, lo, w, class_id=1,
                    cap_units=None):
    """Returns (status, recv arena, recv_off, hist_next)."""
    P = wire_off.shape[0] - 1
    if cap_units is None:
        cap_units = P + int(wire.size // 4 + (0 if ref_off is None else int(ref_off[-1])) + 1)
    recv = np.zeros(cap_units * REC, dtype=np.uint8)
    ro = np.zeros(P + 1, dtype=np.uint64)
    hn = np.zeros(max(cap_units, 1) * HIST, dtype=np.uint8)
    pr = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    st = lib().or_decode_all_pred(P, class_id, _p(wire), _p(wire_off), _p(ref_arena), _p(ref_off),
                                  _p(hist), _p(pr), _d3(lo), float(w), _p(recv), cap_units,
                                  _p(ro), _p(hn))
    E = int(ro[-1])
    return st, recv[:(E + P) * REC].copy(), ro, hn[:E * HIST].copy()
