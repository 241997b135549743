"""Pins for the oracle's per-pair lists and serialization (Sec. 2.1, Sec. 2.2.1).

Message p = (sender box s, neighbour bit b) holds the agents owned by s whose
aura mask has bit b, in ascending agent index, serialized as 64-byte records
whose words are the raw bits of the agent's fields, after one buffer header.
"""
import numpy as np
import pytest

from synth import Generator, Workload


def small_state(seed, n=3000, grid=(3, 2, 2), side=60.0, w=9.0):
    wl = Workload("t", n, (0.0, 0.0, 0.0), (side * grid[0], side * grid[1], side * grid[2]),
                  grid, w, 3, seed=seed)
    gen = Generator(wl)
    from synth import to_numpy
    return wl, to_numpy(gen.initial())


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pair_lists_equal_filter_definition(oracle, seed):
    wl, s = small_state(seed)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    st, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
    assert st == oracle.OK
    st, cnt, off, idx = oracle.pair_lists(g, owner, mask)
    assert st == oracle.OK
    P = wl.n_pairs
    # sum of message sizes = total number of set mask bits
    assert int(off[-1]) == int(sum(bin(int(m)).count("1") for m in mask))
    assert np.all(off[1:] - off[:-1] == cnt)
    for p in range(P):
        sbox, b = divmod(p, 27)
        want = np.nonzero((owner == sbox) & (((mask >> b) & 1) == 1))[0]
        got = idx[int(off[p]):int(off[p + 1])]
        np.testing.assert_array_equal(got, want)
        if b == 13:
            assert cnt[p] == 0


def test_pack_records_are_raw_field_bits(oracle):
    wl, s = small_state(7)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    _, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
    _, cnt, off, idx = oracle.pair_lists(g, owner, mask)
    arena = oracle.pack(s, off, idx, class_id=77)
    P = wl.n_pairs
    assert arena.size == (int(off[-1]) + P) * 64
    fields = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")
    for p in range(P):
        h = arena[(int(off[p]) + p) * 64:(int(off[p]) + p + 1) * 64]
        assert bytes(h[:4]) == b"TAIO"
        assert int(h[4:6].view(np.uint16)[0]) == 1
        assert int(h[6:8].view(np.uint16)[0]) == 64
        assert int(h[8:12].view(np.uint32)[0]) == 77
        assert int(h[12:16].view(np.uint32)[0]) == p
        assert int(h[16:24].view(np.uint64)[0]) == cnt[p]
        assert not h[24:].any()
        recs = oracle.arena_pair(arena, off, p)
        ii = idx[int(off[p]):int(off[p + 1])]
        for w, f in enumerate(fields):
            col = s[f] if f == "id" else s[f].view(np.uint64)
            np.testing.assert_array_equal(recs[:, w], col[ii])


def test_empty_population(oracle):
    g = oracle.make_grid((0, 0, 0), (10, 10, 10), (2, 1, 1), 1.0)
    e = np.zeros(0)
    st, owner, mask = oracle.classify(g, e, e, e)
    assert st == oracle.OK and owner.size == 0
    st, cnt, off, idx = oracle.pair_lists(g, owner, mask)
    assert st == oracle.OK and int(off[-1]) == 0 and off.size == 2 * 27 + 1


def test_capacity_error(oracle):
    g = oracle.make_grid((0, 0, 0), (10, 10, 10), (2, 1, 1), 2.0)
    x = np.array([4.0, 5.5, 1.0]); y = np.ones(3); z = np.ones(3)
    st, owner, mask = oracle.classify(g, x, y, z)
    st, cnt, off, idx = oracle.pair_lists(g, owner, mask, idx_capacity=1)
    assert st == oracle.ECAPACITY
