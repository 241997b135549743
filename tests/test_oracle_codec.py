"""Pins for the oracle's difference codec (paper Sec. 2.3, steps B, C, D) and
its significant-byte packer (the stand-in for the paper's LZ4, Sec. 3.11).

Pinned against: two hand-derived wire messages (tests/golden/), hand vectors
of the byte-length rule, the round trip decode(encode(M, R), R), the
unchanged-state property (all codes zero, empty payload), the count identity
r - holes + new = m, an independent Python restatement of the slot order, and
rejection of every malformed-message class the format defines.
"""
import os
import struct

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


def f2u(v: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def parse_records(text):
    recs = []
    for item in text.split(";"):
        words = [0] * 8
        for kv in item.split():
            k, v = kv.split("=")
            i = FIELDS.index(k)
            words[i] = int(v) if k == "id" else f2u(float(v))
        recs.append(words)
    return np.array(recs, dtype=np.uint64).reshape(-1, 8)


def load_golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or ":" not in line:
                continue
            k, v = line.split(":", 1)
            d[k.strip()] = v.strip()
    return d


@pytest.mark.parametrize("name", ["wire_xor_example.txt", "wire_raw_example.txt"])
def test_golden_wire_message(oracle, name):
    d = load_golden(name)
    ref, msg = parse_records(d["ref"]), parse_records(d["msg"])
    expect = bytes.fromhex("".join((d["header"] + d["codes"] + d["payload"] +
                                    d["padding"]).split()))
    st, wire, nxt = oracle.encode_pair(msg, ref, class_id=int(d["class_id"]),
                                       mode=int(d["mode"]), pair=int(d["pair"]))
    assert st == oracle.OK
    assert bytes(wire) == expect
    assert [int(v) for v in nxt[:, 0]] == [int(t) for t in d["ref_next_ids"].split()]
    # decode restores exactly the sender's new reference
    st, out = oracle.decode_pair(np.frombuffer(expect, dtype=np.uint8), ref,
                                 class_id=int(d["class_id"]), pair=int(d["pair"]))
    assert st == oracle.OK
    np.testing.assert_array_equal(out, nxt)


@pytest.mark.parametrize("value,L", [(0, 0), (1, 1), (0xFF, 1), (0x100, 2),
                                     (0x0000000000010000, 3), (0x00FFFFFFFFFFFFFF, 7),
                                     (0x0100000000000000, 8), (0x8000000000000000, 8),
                                     (0xFFFFFFFFFFFFFFFF, 8)])
def test_byte_length_hand_vectors(oracle, value, L):
    # one new record (no reference): every word is sent raw with its own length
    rec = np.array([[7, value, 0, value, 0, 0, 0, value]], dtype=np.uint64)
    st, wire, _ = oracle.encode_pair(rec, np.zeros((0, 8), np.uint64), mode=oracle.MODE_XOR)
    assert st == oracle.OK
    code = int(wire[64:68].view(np.uint32)[0])
    nib = [(code >> (4 * w)) & 0xF for w in range(8)]
    assert nib == [1, L, 0, L, 0, 0, 0, L]
    payload = int(wire[40:48].view(np.uint64)[0])
    assert payload == 1 + 3 * L
    # payload bytes are the low L bytes, least significant first
    pay = bytes(wire[68:68 + payload])
    lo = value.to_bytes(8, "little")[:L]
    assert pay == bytes([7]) + lo + lo + lo


def rand_records(rng, ids):
    n = len(ids)
    r = np.zeros((n, 8), dtype=np.uint64)
    r[:, 0] = np.array(ids, dtype=np.uint64)
    r[:, 1:] = rng.integers(0, 2**63, (n, 7), dtype=np.uint64) ^ \
        rng.integers(0, 2, (n, 7), dtype=np.uint64) << np.uint64(63)
    return r


def expected_order(msg, ref):
    """Independent restatement of step B's output order."""
    mids = {int(i): k for k, i in enumerate(msg[:, 0])}
    slots = [mids.get(int(i)) for i in ref[:, 0]]
    used = {k for k in slots if k is not None}
    new = [k for k in range(msg.shape[0]) if k not in used]
    return slots, new


@pytest.mark.parametrize("seed", range(25))
def test_round_trip_and_counts(oracle, seed):
    rng = np.random.default_rng(seed)
    pool = rng.choice(10_000, 400, replace=False)
    r = int(rng.integers(0, 150)); m = int(rng.integers(0, 150))
    ref_ids = rng.choice(pool, r, replace=False)
    msg_ids = rng.choice(pool, m, replace=False)
    ref = rand_records(rng, ref_ids)
    msg = rand_records(rng, msg_ids)
    # make matched records close to their reference (a few low bits differ)
    slots, new = expected_order(msg, ref)
    for j, k in enumerate(slots):
        if k is not None and rng.random() < 0.7:
            msg[k, 1:] = ref[j, 1:] ^ rng.integers(0, 1 << int(rng.integers(0, 40)), 7,
                                                   dtype=np.uint64)
    st, wire, nxt = oracle.encode_pair(msg, ref, pair=3)
    assert st == oracle.OK
    n_slots, n_new, n_holes, payload = (int(v) for v in wire[16:48].view(np.uint64))
    holes = sum(1 for k in slots if k is None)
    assert (n_slots, n_new, n_holes) == (r, len(new), holes)
    assert r - holes + len(new) == m
    assert len(wire) % 16 == 0 and int(wire[56:64].view(np.uint64)[0]) == len(wire)
    # new reference = matched records (current values) in slot order, then new ones
    want = [msg[k] for k in slots if k is not None] + [msg[k] for k in new]
    np.testing.assert_array_equal(nxt, np.array(want, dtype=np.uint64).reshape(-1, 8))
    st, out = oracle.decode_pair(wire, ref, pair=3)
    assert st == oracle.OK
    np.testing.assert_array_equal(out, nxt)
    # codes: placeholders exactly at the unmatched slots; matched w0 code 0
    codes = wire[64:64 + 4 * (r + len(new))].view(np.uint32)
    for j, k in enumerate(slots):
        assert (int(codes[j]) == 0xF) == (k is None)
        if k is not None:
            assert int(codes[j]) & 0xF == 0
    assert sum(sum((int(c) >> (4 * w)) & 0xF for w in range(8)) for c in codes
               if int(c) != 0xF) == payload


@pytest.mark.parametrize("shuffle", [False, True])
def test_unchanged_state_sends_nothing(oracle, shuffle):
    rng = np.random.default_rng(5)
    ref = rand_records(rng, rng.choice(1000, 64, replace=False))
    msg = ref[rng.permutation(64)] if shuffle else ref.copy()
    st, wire, nxt = oracle.encode_pair(msg, ref)
    assert st == oracle.OK
    assert int(wire[40:48].view(np.uint64)[0]) == 0  # empty payload
    assert not wire[64:64 + 4 * 64].any()  # every code 0
    np.testing.assert_array_equal(nxt, ref)  # reference order is kept
    assert len(wire) == 64 + 4 * 64


def test_special_float_values_round_trip_bitwise(oracle):
    specials = [0x7FF8000000000001, 0xFFF0000000000000, 0x7FF0000000000000,
                0x8000000000000000, 0x0000000000000001, 0x000FFFFFFFFFFFFF,
                0x7FF7FFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF]
    ref = np.array([[i] + specials[i:] + specials[:i] for i in range(1, 8)],
                   dtype=np.uint64)[:, :8]
    msg = ref[::-1].copy()
    msg[:, 1:] = np.roll(msg[:, 1:], 1, axis=0)
    st, wire, nxt = oracle.encode_pair(msg, ref)
    assert st == oracle.OK
    st, out = oracle.decode_pair(wire, ref)
    assert st == oracle.OK
    np.testing.assert_array_equal(out, nxt)
    assert sorted(map(tuple, out.tolist())) == sorted(map(tuple, msg.tolist()))


def test_duplicate_ids_rejected(oracle):
    rng = np.random.default_rng(1)
    msg = rand_records(rng, [1, 2, 1])
    st, _, _ = oracle.encode_pair(msg, np.zeros((0, 8), np.uint64))
    assert st == oracle.EINVAL
    ref = rand_records(rng, [4, 4])
    st, _, _ = oracle.encode_pair(rand_records(rng, [4]), ref)
    assert st == oracle.EINVAL


def golden_case(oracle):
    d = load_golden("wire_xor_example.txt")
    ref, msg = parse_records(d["ref"]), parse_records(d["msg"])
    st, wire, nxt = oracle.encode_pair(msg, ref, pair=42)
    return ref, wire.copy()


def put(buf, off, fmt, v):
    buf[off:off + struct.calcsize(fmt)] = np.frombuffer(struct.pack(fmt, v), dtype=np.uint8)


@pytest.mark.parametrize("mutate,status", [
    (lambda w: put(w, 0, "<I", 0x41524555), "ECORRUPT"),      # magic
    (lambda w: put(w, 4, "<H", 2), "ECORRUPT"),               # version
    (lambda w: put(w, 6, "<H", 32), "ECORRUPT"),              # record size
    (lambda w: put(w, 8, "<I", 2), "ECORRUPT"),               # class id
    (lambda w: put(w, 48, "<I", 41), "ECORRUPT"),             # pair id
    (lambda w: put(w, 12, "<I", 7), "ECORRUPT"),              # unknown mode
    (lambda w: put(w, 16, "<Q", 2), "EREFMISMATCH"),          # n_slots != receiver r
    (lambda w: put(w, 32, "<Q", 0), "ECORRUPT"),              # hole count
    (lambda w: put(w, 40, "<Q", 17), "ECORRUPT"),             # payload length
    (lambda w: put(w, 56, "<Q", 112), "ECORRUPT"),            # message length
    (lambda w: put(w, 64 + 8, "<I", 0x79), "ECORRUPT"),       # nibble 9 (w1)
    (lambda w: put(w, 64 + 8, "<I", 0xE0), "ECORRUPT"),       # nibble 14 (w1)
    (lambda w: put(w, 64 + 4, "<I", 0xFF), "ECORRUPT"),       # placeholder + other nibble
    (lambda w: put(w, 64 + 8, "<I", 0xF0), "ECORRUPT"),       # 0xF on w1
    (lambda w: put(w, 64 + 12, "<I", 0x0F), "ECORRUPT"),      # placeholder among new
    (lambda w: put(w, 64 + 0, "<I", 0x1), "ECORRUPT"),        # match with id delta
    (lambda w: put(w, 64 + 12, "<I", 0x82), "ECORRUPT"),      # payload overrun
])
def test_malformed_messages_rejected(oracle, mutate, status):
    ref, wire = golden_case(oracle)
    w = wire.copy()
    mutate(w)
    st, _ = oracle.decode_pair(w, ref, pair=42)
    assert st == getattr(oracle, status)


def test_truncated_message_rejected(oracle):
    ref, wire = golden_case(oracle)
    for cut in (0, 10, 63, 64, 80, 95):
        st, _ = oracle.decode_pair(wire[:cut], ref, pair=42)
        assert st == oracle.ECORRUPT


def test_wrong_reference_length(oracle):
    ref, wire = golden_case(oracle)
    st, _ = oracle.decode_pair(wire, ref[:2], pair=42)
    assert st == oracle.EREFMISMATCH


def test_output_capacity(oracle):
    ref, wire = golden_case(oracle)
    st, _ = oracle.decode_pair(wire, ref, pair=42, out_cap=2)
    assert st == oracle.ECAPACITY
