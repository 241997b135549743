"""Pins for the oracle's difference-serialized message before compression
(paper Sec. 2.3, steps B and C; the input of the paper's LZ4 stage, Sec. 3.11).

  * expanding the wire message (4-bit length codes and little-endian payload
    bytes, read here straight from the documented format) gives exactly these
    records, so the two outputs describe one message;
  * each matched slot XOR its reference record is the message record with the
    slot's id, each new entry is a message record absent from the reference;
  * an unchanged state gives all-zero slots and no new entries.
"""
import numpy as np
import pytest


def expand_wire(wire):
    w = wire.view(np.uint8)
    hdr = w[:64]
    n_slots = int(hdr[16:24].view(np.uint64)[0])
    n_new = int(hdr[24:32].view(np.uint64)[0])
    n = n_slots + n_new
    codes = w[64:64 + 4 * n].view(np.uint32)
    pos = 64 + 4 * n
    out = np.zeros((n, 8), dtype=np.uint64)
    for e in range(n):
        c = int(codes[e])
        if c & 0xF == 0xF:
            continue  # placeholder
        for word in range(8):
            L = (c >> (4 * word)) & 0xF
            v = 0
            for b in range(L):
                v |= int(w[pos + b]) << (8 * b)
            pos += L
            out[e, word] = v
    return out, n_slots


def records(rng, ids):
    r = rng.integers(0, 2**63, size=(len(ids), 8), dtype=np.uint64)
    r[:, 0] = ids
    return r


@pytest.mark.parametrize("seed", range(8))
def test_delta_records_match_the_wire(oracle, seed):
    rng = np.random.default_rng(900 + seed)
    ref_ids = rng.choice(10_000, size=int(rng.integers(0, 300)), replace=False).astype(np.uint64)
    ref = records(rng, ref_ids)
    keep = ref_ids[rng.random(len(ref_ids)) < 0.8]
    new_ids = np.setdiff1d(rng.choice(20_000, size=int(rng.integers(0, 100)), replace=False),
                           ref_ids).astype(np.uint64)
    msg_ids = rng.permutation(np.concatenate([keep, new_ids]))
    msg = records(rng, msg_ids)
    # some matched records change only in a few low bytes
    small = rng.random(len(msg)) < 0.5
    for i in np.nonzero(small)[0]:
        j = np.nonzero(ref_ids == msg_ids[i])[0]
        if len(j):
            msg[i] = ref[j[0]] ^ rng.integers(0, 256, 8, dtype=np.uint64)
            msg[i, 0] = msg_ids[i]
    st, wire, _ = oracle.encode_pair(msg, ref)
    assert st == oracle.OK
    delta = oracle.delta_records(msg, ref)
    expanded, r = expand_wire(wire)
    np.testing.assert_array_equal(delta, expanded)
    assert r == len(ref)
    by_id = {int(m[0]): m for m in msg}
    for j in range(r):
        if ref_ids[j] in by_id:
            np.testing.assert_array_equal(delta[j] ^ ref[j], by_id[int(ref_ids[j])])
        else:
            assert not delta[j].any()
    new = delta[r:]
    assert sorted(int(v) for v in new[:, 0]) == sorted(int(v) for v in new_ids)


def test_unchanged_state_is_all_zero(oracle):
    rng = np.random.default_rng(5)
    ref = records(rng, np.arange(50, dtype=np.uint64))
    d = oracle.delta_records(ref[rng.permutation(50)], ref)
    assert d.shape == (50, 8) and not d.any()
