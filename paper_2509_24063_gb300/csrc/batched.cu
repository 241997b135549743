// Batched codec: steps a3-a5 (paper Sec. 2.3, steps B, C and D) for every
// pair of one iteration in ONE persistent launch (on the plain path the small
// pairs run in a second launch of one-warp blocks beside it), after a setup
// of two short launches that lays out the wire slabs and the work list.
//
// Each block takes whole pairs (an atomic ticket over the work list, claimed
// whenever the block is free) and carries a pair through every step on its
// own, so no block ever waits for another (pairs far above the average load
// go to a team of blocks instead):
//
//   match   index the message ids, look every reference slot's id up, mark
//           the message records the slots take.  A pair with at most
//           table_records (<= 8191) records does this in a shared-memory hash
//           table (u16 entries: (record + 1) << 3 | 3-bit fingerprint, ids
//           compared against word 0 of the message's records), or, when the
//           message's ids ascend, by a windowed bisection over them with no
//           table; larger pairs use the pair's global hash segment.
//   slots   difference, code, payload and new-reference record of every slot
//           (tiles of T slots; payload positions from a running prefix kept
//           on chip; the wire puts the slot payload after all r + n_new codes,
//           and n_new = m - matched is known once the match is done)
//   new     records no slot took, in message order; the last tile writes the
//           header, the padding and the iteration totals
//   decode  the receiver's side from the wire and its own reference: codes,
//           payload and receive buffer, again with an on-chip running prefix
//           (a tile's prefix is scanned while the previous tile's bytes and
//           reference records arrive)
//
// Tile size T (block size) and blocks per SM come from the caller (tera_tune,
// picked by the autotuner); the bytes produced do not depend on them.  The
// receive layout is the pair layout of the iteration (every header's record
// count is checked against it).
#include "codec.cuh"

using namespace tera;

namespace {

enum { PT_MATCHED = 0, PT_XOR = 1, PT_RES = 2, PT_COUNT = 4 };
// message entries per thread of a new-record tile (XOR mode: few are new)
constexpr u32 kNewPerThread = 8;
// hash phases take kIlp entries per thread (entry i*T + thread of the tile),
// so several independent probes / atomics are in flight per thread
constexpr u32 kIlp = 4;

struct BatchArgs {
  u64 n_pairs;
  u64* ticket;
  u64* ptot;          // [P * PT_COUNT] per-pair totals of the match step
  u32* abort;
  const u64* items;   // work items: pair << 32 | member << 16 | team size
  const u64* n_items;
  u32* team;          // [P * 8] barrier counters of the teams
  U64x2* tsum;        // per-tile totals of team pairs (slot tiles, then decode tiles)
  const u64* tbase;   // [P] first tile total of a team pair
  u64 wait_ns;        // time limit of one team barrier (global timer)
  // the work list is split in two: items [0, *n_first) (teams, then the other
  // pairs) and [*n_first, *n_items) (the small pairs, carried by a launch of
  // one-warp blocks); part selects the range and its ticket
  u64* n_first;
  u64* ticket_small;
  u32 part;
};

__device__ __forceinline__ u64 make_item(u64 p, u32 member, u32 g) {
  return (p << 32) | ((u64)member << 16) | (u64)g;
}

__device__ __forceinline__ u64 ceil_div(u64 a, u64 b) { return (a + b - 1) / b; }

// Entries per thread of pair p's new-record tiles.
__device__ __forceinline__ u32 new_per_thread(u64 mode) {
  return mode == TERA_MODE_RAW ? 1u : kNewPerThread;
}

// Shared-memory matching state of the block's current pair.
struct SmemTable {
  unsigned short* tbl;  // hash table, or nullptr: the pair uses its global hash segment
  u32 mask;             // table entries - 1
  u32* bits;            // bit k: message record k was taken by a slot
};

constexpr u32 kFpBits = 3, kFpMask = (1u << kFpBits) - 1u;
constexpr u32 kTableMax = (1u << (16 - kFpBits)) - 1u;  // records of a u16 entry
__device__ __forceinline__ u32 fp_of(u64 h) { return (u32)h & kFpMask; }
__device__ __forceinline__ u32 tbl_start(u64 h, u32 mask) { return (u32)(h >> 32) & mask; }

// Block scan of two per-thread counts packed in one word (payload bytes in
// the low half, records in the high half; a tile's totals fit in 32 bits).
__device__ __forceinline__ U64x2 tile_scan(u32 bytes, u32 recs, U64x2* sm, U64x2* total) {
  u64 tot;
  const u64 ex = block_excl_scan<u64>((u64)bytes | ((u64)recs << 32), reinterpret_cast<u64*>(sm),
                                      &tot);
  *total = U64x2{tot & 0xFFFFFFFFull, tot >> 32};
  return U64x2{ex & 0xFFFFFFFFull, ex >> 32};
}

// Exclusive block scan of packed counts (low / high 32 bits) with one
// barrier: each warp publishes its total, and after the barrier every warp
// scans the warps' totals itself.  The caller alternates `buf` (33 words)
// between consecutive scans: a buffer is written again only after the next
// scan's barrier, which every warp passes after its reads of this one.  After
// the last scan of a run, one __syncthreads() must precede other uses of buf.
__device__ __forceinline__ u64 scan_packed(u64 v, u64* buf, u64* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  const u64 incl = warp_incl_scan<u64>(v);
  if (lane == 31) buf[warp] = incl;
  __syncthreads();
  const u64 x = lane < nwarps ? buf[lane] : 0ull;
  const u64 xi = warp_incl_scan<u64>(x);
  *total = __shfl_sync(0xFFFFFFFFu, xi, nwarps - 1);
  return __shfl_sync(0xFFFFFFFFu, xi - x, warp) + incl - v;
}

// Each warp stages its own contiguous byte range in a private region and
// stores it with 16-byte stores inside and byte stores on the edges it shares
// with the neighbouring warps.  32 records + 16 bytes: the decode stages from
// the 16-byte boundary below its first byte, and the encode's flush reads one
// word past its last.
constexpr u32 kWarpStage = 32 * kRecBytes + 16;

// Per-thread record stash in shared memory: 16-byte part k of thread i's
// record at stash[k T + i], so each part of a warp's records is one
// contiguous 512-byte row.  It holds the record a slot or decode tile needs
// after its block scan, which would otherwise stay in registers across the
// barrier (and spill).  Only the owning thread reads its entries, so no
// barrier guards them.
template <int T>
__device__ __forceinline__ void stash_put(ulonglong2* st, const Rec& r) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    st[k * T + threadIdx.x] = make_ulonglong2(r.w[2 * k], r.w[2 * k + 1]);
}

template <int T>
__device__ __forceinline__ Rec stash_get(const ulonglong2* st) {
  Rec r;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const ulonglong2 v = st[k * T + threadIdx.x];
    r.w[2 * k] = v.x;
    r.w[2 * k + 1] = v.y;
  }
  return r;
}

// The record at g (16-byte aligned) into the stash by asynchronous
// copies; stash_wait() before reading it.
template <int T>
__device__ __forceinline__ void stash_async(ulonglong2* st, const uint8_t* g) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const u32 dst = (u32)__cvta_generic_to_shared(st + k * T + threadIdx.x);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" : : "r"(dst), "l"(g + 16 * k)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" : : : "memory");
}

__device__ __forceinline__ void stash_wait() { asm volatile("cp.async.wait_all;" : : : "memory"); }

// The L significant bytes of v (its higher bytes are zero) at byte offset o of
// a zeroed, 4-byte-aligned stage: ORed into the at most three 32-bit words
// they touch, so neighbouring lanes' bytes in a shared word are kept.
__device__ __forceinline__ void stage_or(uint8_t* st, u32 o, u64 v, u32 L) {
  if (L == 0) return;
  u32* w = reinterpret_cast<u32*>(st + (o & ~3u));
  const u32 sh = (o & 3u) * 8u;
  const u64 lo = v << sh;
  const u32 nb = (o & 3u) + L;  // bytes from the first word's start, at most 11
  atomicOr(&w[0], (u32)lo);
  if (nb > 4) atomicOr(&w[1], (u32)(lo >> 32));
  if (nb > 8) atomicOr(&w[2], (u32)(v >> (64u - sh)));
}

// Zero the first n bytes of a 16-byte-aligned warp stage (rounded up to 16).
__device__ __forceinline__ void warp_zero(uint8_t* wst, u32 n) {
  for (u32 c = threadIdx.x & 31; c < ((n + 15u) >> 4); c += 32)
    *reinterpret_cast<uint4*>(wst + (c << 4)) = make_uint4(0u, 0u, 0u, 0u);
}

// Store the n bytes at the start of a warp stage to gW, whatever its
// alignment: each whole 16-byte chunk of the destination is assembled from
// five 32-bit stage words by funnel shifts and stored at once; the edge
// chunks, shared with the neighbouring warps' bytes, are stored byte by byte.
// The stage has at least 16 bytes beyond n, so the fifth word stays inside it.
__device__ __forceinline__ void warp_flush(const uint8_t* wst, uint8_t* gW, u32 n) {
  const u32 s0 = (u32)((uintptr_t)gW & 15u);
  uint8_t* g16 = gW - s0;
  const u32 end = s0 + n;
  const u32 nchunks = (end + 15u) >> 4;
  const u32* w32 = reinterpret_cast<const u32*>(wst);
  for (u32 c = threadIdx.x & 31; c < nchunks; c += 32) {
    const u32 lo = c << 4, hi = lo + 16u;
    if (lo >= s0 && hi <= end) {
      const u32 o = lo - s0;  // stage offset of the chunk's first byte
      const u32 i = o >> 2, sh = (o & 3u) * 8u;
      u32 v[4];
      if (sh == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = w32[i + k];
      } else {
        u32 a = w32[i];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const u32 b = w32[i + k + 1];
          v[k] = __funnelshift_r(a, b, sh);
          a = b;
        }
      }
      *reinterpret_cast<uint4*>(g16 + lo) = make_uint4(v[0], v[1], v[2], v[3]);
    } else {
      for (u32 x = (lo > s0 ? lo : s0); x < (hi < end ? hi : end); ++x) g16[x] = wst[x - s0];
    }
  }
}

// Blocks that carry a pair of `size` entries (reference slots + message
// records + receiver slots): 1, or a team when the pair exceeds the average
// load of a block (so no single block holds up the end of the launch).
// forced > 0 (the schedule's team_blocks) gives every such pair exactly that
// many blocks.
__device__ __forceinline__ u32 team_size(u64 size, u64 thresh, u32 gmax, int pred, u32 forced) {
  (void)pred;
  if (size <= thresh) return 1u;
  if (forced) return forced;
  const u64 g = ceil_div(size, thresh);
  return (u32)(g < gmax ? g : gmax);
}

// Tile totals a team pair keeps: slot tiles, new-record tiles (at most one per
// T records), decode tiles (a valid message has at most rr + m entries).
__device__ __forceinline__ u64 team_tiles(u64 r, u64 m, u64 rr, u32 T) {
  return ceil_div(r, T) + ceil_div(m, T) + ceil_div(rr + m, T);
}

// ---------------- setup: per-pair facts, layouts, capacity checks ----------------

// Per-pair facts of the setup (raw or XOR mode, slots, records, slab, team).
struct PairFacts {
  u64 r, r_full, m, rr, slab;
  u32 g;
  bool raw;
};

// The work-list count word of a pair carried by one block: 1 (low half) for an
// ordinary pair, 1 << 32 (high half) for a small one.
__device__ __forceinline__ u64 single_word(const PairFacts& f, u64 small_max) {
  const bool small = small_max > 0 && f.r <= small_max && f.m <= small_max && f.rr <= small_max;
  return small ? (1ull << 32) : 1ull;
}

__device__ __forceinline__ PairFacts pair_facts(const EncArgs& E, const DecArgs& D, u64 p, int mode,
                                                u64 thresh, u32 gmax, int pred, u32 forced) {
  PairFacts f;
  f.m = E.pair_off[p + 1] - E.pair_off[p];
  f.r_full = E.ref_off ? E.ref_off[p + 1] - E.ref_off[p] : 0;
  f.raw = mode == TERA_MODE_RAW || E.reset[p];
  f.r = (f.raw || E.ref_off == nullptr) ? 0 : f.r_full;
  f.rr = D.ref_off ? D.ref_off[p + 1] - D.ref_off[p] : 0;
  f.slab = round16((u64)kHdrBytes + 4 * (f.r_full + f.m) + (u64)kRecBytes * f.m);
  f.g = team_size(f.r + f.m + f.rr, thresh, gmax, pred, forced);
  return f;
}

// A pair becomes a team when its entries exceed the average per block of the
// launch (and min_team).
__device__ __forceinline__ u64 setup_thresh(const EncArgs& E, const DecArgs& D, u64 P, u32 blocks,
                                            u64 min_team) {
  const u64 total = E.pair_off[P] + (E.ref_off ? E.ref_off[P] : 0) + (D.ref_off ? D.ref_off[P] : 0);
  const u64 avg = ceil_div(total, blocks);
  return avg > min_team ? avg : min_team;
}

// The setup's two scanned values of a pair: (slab bytes, team tiles) and
// (team items, work-list count word).
__device__ __forceinline__ void setup_values(const PairFacts& f, u32 T, u64 small_max, U64x2* va,
                                             U64x2* vb) {
  const bool team = f.g > 1;
  *va = U64x2{f.slab, team ? team_tiles(f.r, f.m, f.rr, T) : 0};
  *vb = U64x2{team ? f.g : 0u, team ? 0u : single_word(f, small_max)};
}

constexpr int kSetupThreads = 1024;

// Setup, first launch: one pair per thread, kSetupThreads pairs per block.
// Writes the per-pair facts (slots, records, mode, receive offsets) and the
// block's sums of the two scanned values (part[2b], part[2b + 1]).
__global__ void __launch_bounds__(kSetupThreads)
    bat_setup_sums_kernel(EncArgs E, DecArgs D, u64 P, int mode, u32 T, u32 blocks, u32 gmax,
                          u32 forced, u64 min_team, int pred, u64 small_max,
                          U64x2* __restrict__ part) {
  __shared__ U64x2 sm2[33];
  __shared__ u64 s_thresh;
  if (threadIdx.x == 0) s_thresh = setup_thresh(E, D, P, blocks, min_team);
  __syncthreads();
  const u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  U64x2 va{0, 0}, vb{0, 0};
  if (p < P) {
    const PairFacts f = pair_facts(E, D, p, mode, s_thresh, gmax, pred, forced);
    u64* pi = E.info + p * 8;
    pi[PI_R] = f.r;
    pi[PI_M] = f.m;
    pi[PI_MODE] = f.raw ? TERA_MODE_RAW : TERA_MODE_XOR;
    D.recv_off[p] = E.pair_off[p];  // receive buffers sized by the record counts
    setup_values(f, T, small_max, &va, &vb);
  }
  U64x2 ta, tb;
  block_excl_scan2(va, sm2, &ta);
  block_excl_scan2(vb, sm2, &tb);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ta;
    part[2 * blockIdx.x + 1] = tb;
  }
}

// Setup, second launch (the same blocks): each block adds up the first
// launch's block sums before it (its carry) and over all blocks (the totals),
// then scans its pairs into the wire slab offsets, the work list (team items
// first, so the large pairs start early, then one item per other pair, then,
// when small_max > 0, one item per small pair: at most small_max slots,
// records and receiver slots; each group in pair order) and the teams' first
// tile totals.  The counts of the other and the small pairs travel packed in
// one word (low and high 32 bits) through the scans.  The last block's thread
// 0 writes the totals, checks the capacities and resets the claim tickets.
__global__ void __launch_bounds__(kSetupThreads)
    bat_setup_place_kernel(EncArgs E, DecArgs D, BatchArgs B, u64 P, int mode,
                           u64* __restrict__ wire_off, u64 wire_cap, u64 rec_cap, u64 recv_cap,
                           u32* epoch, u32 T, u32 blocks, u32 gmax, u32 forced, u64 min_team,
                           int pred, u64* __restrict__ items, u64 items_cap,
                           u64* __restrict__ tbase, u64 tsum_cap, u64* __restrict__ n_items,
                           u64 small_max, const U64x2* __restrict__ part) {
  __shared__ U64x2 sm2[33];
  __shared__ u64 s_thresh;
  if (threadIdx.x == 0) s_thresh = setup_thresh(E, D, P, blocks, min_team);
  U64x2 ca{0, 0}, cb{0, 0}, qa{0, 0}, qb{0, 0};  // (before this block), (all blocks)
  for (u32 i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
    const U64x2 a = part[2 * i], b = part[2 * i + 1];
    if (i < blockIdx.x) {
      ca += a;
      cb += b;
    }
    qa += a;
    qb += b;
  }
  U64x2 carry_a, carry_b, tot_a, tot_b;
  block_excl_scan2(ca, sm2, &carry_a);
  block_excl_scan2(cb, sm2, &carry_b);
  block_excl_scan2(qa, sm2, &tot_a);
  block_excl_scan2(qb, sm2, &tot_b);
  const u64 tw = tot_a.a, ttiles = tot_a.b, tbig = tot_b.a;
  const u64 n_other = tot_b.b & 0xFFFFFFFFull, n_small = tot_b.b >> 32;
  const u64 tsmall = n_other + n_small;
  const bool fits = tbig + tsmall <= items_cap && ttiles <= tsum_cap;
  const u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  PairFacts f{};
  U64x2 va{0, 0}, vb{0, 0};
  if (p < P) {
    f = pair_facts(E, D, p, mode, s_thresh, gmax, pred, forced);
    setup_values(f, T, small_max, &va, &vb);
  }
  U64x2 ta, tb;
  const U64x2 ea = carry_a + block_excl_scan2(va, sm2, &ta);
  const U64x2 eb = carry_b + block_excl_scan2(vb, sm2, &tb);
  if (p < P) {
    wire_off[p] = ea.a;
    if (fits) {
      if (f.g > 1) {
        for (u32 i = 0; i < f.g; ++i) items[eb.a + i] = make_item(p, i, f.g);
        tbase[p] = ea.b;
      } else if (vb.b == 1u) {
        items[tbig + (eb.b & 0xFFFFFFFFull)] = make_item(p, 0, 1);
      } else {
        items[tbig + n_other + (eb.b >> 32)] = make_item(p, 0, 1);
      }
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const u32 ep = *epoch + 1u;
    *epoch = ep == 0u ? 1u : ep;
    wire_off[P] = tw;
    D.recv_off[P] = E.pair_off[P];
    bool abort = false;
    if (tw > wire_cap) {
      latch(E.st, TERA_ECAPACITY);
      need(E.st, tw);
      abort = true;
    }
    // record scratch is sized for rec_cap records per side
    const u64 rmax = E.ref_off ? E.ref_off[P] : 0, dmax = D.ref_off ? D.ref_off[P] : 0;
    const u64 big = E.pair_off[P] > rmax ? (E.pair_off[P] > dmax ? E.pair_off[P] : dmax)
                                          : (rmax > dmax ? rmax : dmax);
    if (big > rec_cap) {
      latch(E.st, TERA_ECAPACITY);
      need(E.st, big);
      abort = true;
    }
    if (E.pair_off[P] + P > recv_cap) {
      latch(E.st, TERA_ECAPACITY);
      need(E.st, E.pair_off[P] + P);
      abort = true;
    }
    if (!fits) {  // cannot happen: the work list is sized for it
      latch(E.st, TERA_ECAPACITY);
      abort = true;
    }
    *n_items = abort ? 0 : tbig + tsmall;
    *B.n_first = abort ? 0 : tbig + n_other;
    *B.abort = abort ? 1u : 0u;
    *B.ticket = 0;
    *B.ticket_small = 0;
  }
}

// ---------------- match in shared memory ----------------

// Index message records [0, m) of pair p.  A second record with an id already
// present is an invalid message (TERA_EINVAL) and is not indexed.
template <int T>
__device__ __forceinline__ void smem_build(const EncArgs& A, u32 p, u64 m, const SmemTable& tb) {
  const u64 g_lo = A.pair_off[p];
  for (u32 i = threadIdx.x; i <= tb.mask; i += T) tb.tbl[i] = 0;
  for (u32 i = threadIdx.x; i < (u32)((m + 31) / 32); i += T) tb.bits[i] = 0u;
  // message ids are read one batch ahead, so they arrive while a batch inserts
  u64 id_next[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    const u64 k = (u64)i * T + threadIdx.x;
    id_next[i] = k < m ? msg_id(A, p, g_lo + k) : 0;
  }
  __syncthreads();
  for (u64 k0 = 0; k0 < m; k0 += (u64)T * kIlp) {
    u64 id[kIlp];
#pragma unroll
    for (u32 i = 0; i < kIlp; ++i) {
      id[i] = id_next[i];
      const u64 k = k0 + (u64)(kIlp + i) * T + threadIdx.x;
      id_next[i] = k < m ? msg_id(A, p, g_lo + k) : 0;
    }
#pragma unroll
    for (u32 i = 0; i < kIlp; ++i) {
      const u64 k = k0 + (u64)i * T + threadIdx.x;
      if (k >= m) continue;
      const u64 h = mix64(id[i]);
      const u32 fp = fp_of(h);
      const unsigned short e = (unsigned short)(((u32)(k + 1) << kFpBits) | fp);
      u32 at = tbl_start(h, tb.mask);
      for (u32 probe = 0; probe <= tb.mask; ++probe) {
        const u32 old = atomicCAS(&tb.tbl[at], (unsigned short)0, e);
        if (old == 0u) break;
        if ((old & kFpMask) == fp && msg_id(A, p, g_lo + (old >> kFpBits) - 1) == id[i]) {
          latch(A.st, TERA_EINVAL);  // ids must be unique within a message
          break;
        }
        at = (at + 1) & tb.mask;
      }
    }
  }
}

// Message record (index in the pair) with this id, probing from `at`; kNoMatch if none.
__device__ __forceinline__ u32 smem_find(const EncArgs& A, u32 p, const SmemTable& tb, u64 g_lo,
                                         u64 id, u32 fp, u32 at) {
  for (u32 probe = 0; probe <= tb.mask; ++probe) {
    const u32 e = tb.tbl[at];
    if (e == 0u) return kNoMatch;
    if ((e & kFpMask) == fp && msg_id(A, p, g_lo + (e >> kFpBits) - 1) == id)
      return (e >> kFpBits) - 1;
    at = (at + 1) & tb.mask;
  }
  return kNoMatch;
}

// Look every slot of pair p up; slot_src[slot] = global record index or
// kNoMatch; bits mark the taken records.  Returns this thread's match count.
template <int T>
__device__ __forceinline__ u32 smem_match(const EncArgs& A, u32 p, u64 r, const SmemTable& tb) {
  // no reference (r = 0): ref_off is null and no slot is read
  const u64 ro = A.ref_off ? A.ref_off[p] : 0, g_lo = A.pair_off[p];
  u32 found = 0;
  // slot ids are read one batch ahead, so they arrive while a batch probes
  u64 id_next[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    const u64 j = (u64)i * T + threadIdx.x;
    id_next[i] = j < r ? ref_id(A, p, ro, j) : 0;
  }
  for (u64 j0 = 0; j0 < r; j0 += (u64)T * kIlp) {
    u64 id[kIlp];
#pragma unroll
    for (u32 i = 0; i < kIlp; ++i) {
      id[i] = id_next[i];
      const u64 j = j0 + (u64)(kIlp + i) * T + threadIdx.x;
      id_next[i] = j < r ? ref_id(A, p, ro, j) : 0;
    }
    // first fingerprint hit of every slot (shared memory only), then the
    // id checks of all of them in flight together
    u32 cand[kIlp], at[kIlp], fp[kIlp];
#pragma unroll
    for (u32 i = 0; i < kIlp; ++i) {
      const u64 j = j0 + (u64)i * T + threadIdx.x;
      cand[i] = kNoMatch;
      const u64 h = mix64(id[i]);
      fp[i] = fp_of(h);
      at[i] = tbl_start(h, tb.mask);
      if (j >= r) continue;
      for (u32 probe = 0; probe <= tb.mask; ++probe) {
        const u32 e = tb.tbl[at[i]];
        if (e == 0u) break;
        if ((e & kFpMask) == fp[i]) {
          cand[i] = (e >> kFpBits) - 1;
          break;
        }
        at[i] = (at[i] + 1) & tb.mask;
      }
    }
    u64 cid[kIlp];
#pragma unroll
    for (u32 i = 0; i < kIlp; ++i) cid[i] = cand[i] != kNoMatch ? msg_id(A, p, g_lo + cand[i]) : 0;
#pragma unroll
    for (u32 i = 0; i < kIlp; ++i) {
      const u64 j = j0 + (u64)i * T + threadIdx.x;
      if (j >= r) continue;
      u32 k = cand[i];
      if (k != kNoMatch && cid[i] != id[i])  // fingerprint collision: keep probing
        k = smem_find(A, p, tb, g_lo, id[i], fp[i], (at[i] + 1) & tb.mask);
      if (k != kNoMatch) {
        const u32 bit = 1u << (k & 31u);
        if (atomicOr(&tb.bits[k >> 5], bit) & bit) {
          latch(A.st, TERA_EINVAL);  // a second slot with the same id: that slot is a hole
          k = kNoMatch;
        }
      }
      found += k != kNoMatch;
      A.slot_src[ro + j] = k != kNoMatch ? (u32)(g_lo + k) : kNoMatch;
    }
  }
  return found;
}

// ---------------- match of ascending id lists ----------------
//
// When the ids of a pair's message strictly ascend (agents kept in the order
// their ids were given, so that each list, in agent order, is in id order), a
// slot's match is found without an index: the round of reference slots from
// j0 (2 kIlp per thread) loads the message ids from kWinSlack before to
// kWinSlack after [j0 + d, j0 + d + 2 kIlp T) into shared memory, d = (message
// index - slot index) of the last match so far, and each slot searches that
// window by bisection (a slot whose id lies outside it searches all message
// ids).  Every slot is looked up by bisection, so the matches are the index's
// whatever the reference order; an ascending reference keeps the searches in
// the window.  Pairs whose message ids do not ascend take the index.

constexpr u32 kWinSlack = 64;

// The message ids of pair p strictly ascending (the same answer in every
// thread).  A reference slot whose id repeats finds a record already taken,
// which the search treats as the index does (an invalid reference; the slot
// is a hole).
template <int T>
__device__ __forceinline__ bool ids_ascending(const EncArgs& A, u32 p, u64 m) {
  const u64 g_lo = A.pair_off[p];
  int bad = 0;
  for (u64 k0 = threadIdx.x; k0 + 1 < m; k0 += 4 * (u64)T) {
    u64 a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const u64 k = k0 + (u64)i * T;
      a[i] = k + 1 < m ? msg_id(A, p, g_lo + k) : 0;
      b[i] = k + 1 < m ? msg_id(A, p, g_lo + k + 1) : 1;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) bad |= !(a[i] < b[i]);
  }
  return __syncthreads_or(bad) == 0;
}

// Every slot of pair p looked up (ascending message ids): slot_src[slot] =
// global record index or kNoMatch, and the taken bits; 2 kIlp slots per
// thread per round.  Returns this thread's match count.  win: shared memory
// for 2 kIlp T + 2 kWinSlack ids.
template <int T>
__device__ __forceinline__ u32 sorted_match(const EncArgs& A, u32 p, u64 m, u64 r,
                                            const SmemTable& tb, u64* win) {
  constexpr u32 kW = 2 * kIlp;  // slots per thread per round
  constexpr u64 kSpan = (u64)T * kW;
  __shared__ long long s_d;
  __shared__ unsigned long long s_jk;
  const u64 ro = A.ref_off ? A.ref_off[p] : 0, g_lo = A.pair_off[p];
  for (u32 i = threadIdx.x; i < (u32)((m + 31) / 32); i += T) tb.bits[i] = 0u;
  if (threadIdx.x == 0) {
    s_d = 0;
    s_jk = 0;
  }
  __syncthreads();
  u32 found = 0;
  for (u64 j0 = 0; j0 < r; j0 += kSpan) {  // block-uniform
    const long long ws = (long long)j0 + s_d - (long long)kWinSlack;
    const u64 wlo = ws < 0 ? 0 : ((u64)ws < m ? (u64)ws : m);
    const u64 whi = wlo + kSpan + 2 * kWinSlack < m ? wlo + kSpan + 2 * kWinSlack : m;
    u64 x[kW];
#pragma unroll
    for (u32 i = 0; i < kW; ++i) {
      const u64 j = j0 + (u64)i * T + threadIdx.x;
      x[i] = j < r ? ref_id(A, p, ro, j) : 0;
    }
    for (u64 k = wlo + threadIdx.x; k < whi; k += T) win[k - wlo] = msg_id(A, p, g_lo + k);
    __syncthreads();  // the window is loaded
    const u64 n = whi - wlo;
    u64 last = 0;  // (slot + 1) << 32 | record of this thread's last match
#pragma unroll
    for (u32 i = 0; i < kW; ++i) {
      const u64 j = j0 + (u64)i * T + threadIdx.x;
      if (j >= r) continue;
      u32 k = kNoMatch;
      if (n > 0 && x[i] >= win[0] && x[i] <= win[n - 1]) {
        u64 lo = 0, hi = n;
        while (lo < hi) {
          const u64 mid = (lo + hi) >> 1;
          if (win[mid] < x[i]) lo = mid + 1;
          else hi = mid;
        }
        if (win[lo] == x[i]) k = (u32)(wlo + lo);
      } else {
        u64 lo = 0, hi = m;
        while (lo < hi) {
          const u64 mid = (lo + hi) >> 1;
          if (msg_id(A, p, g_lo + mid) < x[i]) lo = mid + 1;
          else hi = mid;
        }
        if (lo < m && msg_id(A, p, g_lo + lo) == x[i]) k = (u32)lo;
      }
      if (k != kNoMatch) {
        const u32 bit = 1u << (k & 31u);
        if (atomicOr(&tb.bits[k >> 5], bit) & bit) {
          latch(A.st, TERA_EINVAL);  // a second slot with the same id: that slot is a hole
          k = kNoMatch;
        }
      }
      if (k != kNoMatch) {
        ++found;
        last = ((j + 1) << 32) | k;
      }
      A.slot_src[ro + j] = k != kNoMatch ? (u32)(g_lo + k) : kNoMatch;
    }
    // the round's last match: its offset carries to the next round
    u64 wl = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const u64 t = __shfl_xor_sync(0xFFFFFFFFu, wl, o);
      wl = t > wl ? t : wl;
    }
    if ((threadIdx.x & 31) == 0 && wl) atomicMax(&s_jk, wl);
    __syncthreads();  // the window is read, s_jk is final
    if (threadIdx.x == 0 && s_jk) {
      s_d = (long long)(s_jk & 0xFFFFFFFFull) - (long long)((s_jk >> 32) - 1);
      s_jk = 0;
    }
    __syncthreads();
  }
  return found;
}

// ---------------- match in the global hash segments ----------------

template <int T>
__device__ __forceinline__ void bat_build(const EncArgs& A, u32 p, u64 tile, u32 epoch) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 m = pi[PI_M];
  const u64 g_lo = A.pair_off[p];
  const u64 base = seg_base(g_lo, p), size = seg_size(m);
  u64 id[kIlp], at[kIlp], cur[kIlp];
  bool live[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    const u64 k = tile * T * kIlp + (u64)i * T + threadIdx.x;
    live[i] = k < m;
    id[i] = live[i] ? msg_id(A, p, g_lo + k) : 0;
  }
  // first probe of every entry: one load each, then one CAS each
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    at[i] = seg_start(id[i], size);
    cur[i] = live[i] ? __ldcg(&A.seg[base + at[i]].a) : 0;
  }
  // the CASes of all entries in flight together, then the stragglers
  u64 prev[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    const u64 k = tile * T * kIlp + (u64)i * T + threadIdx.x;
    const bool empty = live[i] && (u32)(cur[i] >> 32) != epoch;
    prev[i] = empty ? atomicCAS(&A.seg[base + at[i]].a, cur[i], ((u64)epoch << 32) | k) : ~0ull;
  }
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    if (!live[i]) continue;
    const u64 k = tile * T * kIlp + (u64)i * T + threadIdx.x;
    if ((u32)(cur[i] >> 32) != epoch && prev[i] == cur[i]) {
      A.seg[base + at[i]].b = id[i];
    } else {  // taken in this iteration: continue along the probe sequence
      seg_insert_from<true>(A.seg, base, size, id[i], ((u64)epoch << 32) | k, epoch,
                            at[i] + 1 == size ? 0 : at[i] + 1);
    }
  }
}

// Predictor work of a matched slot: the training sample, and the slot's
// residual payload size from the prediction the pre-pass made (predictions
// exist only with both a history and the network, and then the pre-pass has
// run).
template <bool PR>
__device__ __forceinline__ u64 pred_slot(const EncArgs& A, u32 p, u64 j, u64 r, u64 mode,
                                         const Rec& R, const Rec& M, u32 bxor) {
  u64 vres = bxor;
  if (!A.pr.hist || mode != TERA_MODE_XOR) return vres;
  if (A.pr.samples) {
    const Hist H = load_hist(A.pr.hist + kHistBytes * (A.ref_off[p] + j));
    const u32 nc = cell_count(A.pr.cseg, seg_base(A.ref_off[p], p), seg_size(r),
                              cell_key(R, A.pr));
    float f[kMlpIn];
    if (features(R, H, nc, f)) {
      float* smp = A.pr.samples + (u64)kSampleFloats * (A.ref_off[p] + j);
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) smp[i] = f[i];
#pragma unroll
      for (int a = 0; a < 3; ++a)
        smp[kMlpIn + a] = __double2float_rn(
            __dsub_rn(__longlong_as_double((long long)M.w[1 + a]),
                      __longlong_as_double((long long)R.w[1 + a])));
      smp[11] = 1.0f;
    }
  }
  if (A.pr.pre) {
    const u64* ps = A.pr.pscr + 4 * (A.ref_off[p] + j);
    if (__ldcg(ps + 3)) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        vres += sig_bytes(zigzag(M.w[1 + a] - __ldcg(ps + a)));
        vres -= sig_bytes(M.w[1 + a] ^ R.w[1 + a]);
      }
    }
  }
  return vres;
}

template <int T>
__device__ __forceinline__ void bat_match_ilp(const EncArgs& A, const BatchArgs& B, u32 p,
                                              u64 tile, u32 epoch) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 r = pi[PI_R], m = pi[PI_M];
  const u64 ro = A.ref_off[p], g_lo = A.pair_off[p];
  const u64 base = seg_base(g_lo, p), size = seg_size(m);
  u64 id[kIlp], at[kIlp];
  U64x2 e[kIlp];
  bool live[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    const u64 j = tile * T * kIlp + (u64)i * T + threadIdx.x;
    live[i] = j < r;
    id[i] = live[i] ? ref_id(A, p, ro, j) : 0;
  }
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    at[i] = seg_start(id[i], size);
    e[i] = live[i] ? ldx<true>(A.seg + base + at[i]) : U64x2{0, 0};
  }
  u32 g[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    g[i] = kNoMatch;
    if (!live[i] || (u32)(e[i].a >> 32) != epoch) continue;
    if (e[i].b == id[i]) g[i] = (u32)(g_lo + (u32)e[i].a);
    else g[i] = seg_lookup_from<true>(A.seg, epoch, base, size, g_lo, id[i],
                                      at[i] + 1 == size ? 0 : at[i] + 1);
  }
  u32 old[kIlp];
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) old[i] = g[i] != kNoMatch ? atomicExch(&A.matched[g[i]], epoch) : 0u;
  int found = 0;
#pragma unroll
  for (u32 i = 0; i < kIlp; ++i) {
    if (!live[i]) continue;
    // a second slot with the same id: invalid reference; that slot is a hole
    if (g[i] != kNoMatch && old[i] == epoch) {
      latch(A.st, TERA_EINVAL);
      g[i] = kNoMatch;
    }
    found += g[i] != kNoMatch;
    A.slot_src[ro + tile * T * kIlp + (u64)i * T + threadIdx.x] = g[i];
  }
  // block total of matches: warp sums, one atomic per warp
  int wsum = found;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xFFFFFFFFu, wsum, o);
  if ((threadIdx.x & 31) == 0 && wsum)
    atomicAdd(B.ptot + (u64)p * PT_COUNT + PT_MATCHED, (u64)wsum);
}

template <int T, bool PR>
__device__ __forceinline__ void bat_match(const EncArgs& A, const BatchArgs& B, u32 p, u64 tile,
                                          u32 epoch, U64x2* sm) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 r = pi[PI_R], m = pi[PI_M];
  const u64 j = tile * T + threadIdx.x;
  int found = 0;
  u64 bx = 0, br = 0;
  if (j < r) {
    const u64 ro = A.ref_off[p];
    const uint8_t* rp = A.ref + (ro + p + 1 + j) * kRecBytes;
    if constexpr (PR) {
      if (A.pr.samples) A.pr.samples[(u64)kSampleFloats * (ro + j) + 11] = 0.0f;
    }
    Rec R;
    u64 id;
    if constexpr (PR) {
      R = load_rec(rp);
      id = R.w[0];
    } else {
      id = *reinterpret_cast<const u64*>(rp);
    }
    u32 g = seg_lookup<true>(A.seg, epoch, p, A.pair_off[p], m, id);
    // a second slot with the same id: invalid reference; that slot is a hole
    if (g != kNoMatch && atomicExch(&A.matched[g], epoch) == epoch) {
      latch(A.st, TERA_EINVAL);
      g = kNoMatch;
    }
    if (g != kNoMatch) {
      found = 1;
      if constexpr (PR) {
        const Rec M = load_rec(A.rec + ((u64)g + p + 1) * kRecBytes);
        u32 b = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) b += sig_bytes(M.w[w] ^ R.w[w]);
        bx = b;
        br = pred_slot<PR>(A, p, j, r, pi[PI_MODE], R, M, b);
      }
    }
    A.slot_src[ro + j] = g;
  }
  if constexpr (PR) {
    U64x2 tot;
    block_excl_scan2(U64x2{bx, br}, sm, &tot);
    const int c = __syncthreads_count(found);
    if (threadIdx.x == 0) {
      u64* pt = B.ptot + (u64)p * PT_COUNT;
      if (c) atomicAdd(pt + PT_MATCHED, (u64)c);
      if (tot.a) atomicAdd(pt + PT_XOR, tot.a);
      if (tot.b) atomicAdd(pt + PT_RES, tot.b);
    }
  } else {
    const int c = __syncthreads_count(found);
    if (threadIdx.x == 0 && c) atomicAdd(B.ptot + (u64)p * PT_COUNT + PT_MATCHED, (u64)c);
  }
}

// The predictor's match totals of one slot tile of pair p after a match in
// shared memory (slot_src written by this block): the XOR and residual
// payload bytes of the matched slots (and their training samples), as
// bat_match makes them in the global path.
template <int T, bool PR>
__device__ __forceinline__ void bat_sizes(const EncArgs& A, const BatchArgs& B, u32 p, u64 tile,
                                          U64x2* sm) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 r = pi[PI_R];
  const u64 j = tile * T + threadIdx.x;
  u64 bx = 0, br = 0;
  if (j < r) {
    const u64 ro = A.ref_off[p];
    if (A.pr.samples) A.pr.samples[(u64)kSampleFloats * (ro + j) + 11] = 0.0f;
    const u32 g = A.slot_src[ro + j];
    if (g != kNoMatch) {
      const Rec R = load_rec(A.ref + (ro + p + 1 + j) * kRecBytes);
      const Rec M = load_rec(A.rec + ((u64)g + p + 1) * kRecBytes);
      u32 b = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) b += sig_bytes(M.w[w] ^ R.w[w]);
      bx = b;
      br = pred_slot<PR>(A, p, j, r, pi[PI_MODE], R, M, b);
    }
  }
  U64x2 tot;
  block_excl_scan2(U64x2{bx, br}, sm, &tot);
  if (threadIdx.x == 0) {
    u64* pt = B.ptot + (u64)p * PT_COUNT;
    if (tot.a) atomicAdd(pt + PT_XOR, tot.a);
    if (tot.b) atomicAdd(pt + PT_RES, tot.b);
  }
}

// Message mode of pair p once MATCH is complete.
template <bool PR>
__device__ __forceinline__ u64 pair_mode(const EncArgs& A, const BatchArgs& B, u32 p) {
  u64 mode = A.info[(u64)p * 8 + PI_MODE];
  if constexpr (PR) {
    const u64* pt = B.ptot + (u64)p * PT_COUNT;
    if (A.pr.params && A.pr.allow_residual && mode == TERA_MODE_XOR &&
        __ldcg(pt + PT_RES) < __ldcg(pt + PT_XOR))
      mode = kModeResidual;
  }
  return mode;
}

// Offsets of pair p that every tile of its encode steps uses, read once per
// pair: read inside each tile they put dependent global loads in front of
// the tile's record loads and stores.
struct SlotPair {
  u64 r, m;      // reference slots, message records
  u64 ro, g_lo;  // first slot in the reference, first record in the arena
  u64 n_new;     // records no slot takes (m - matched, known after the match)
  uint8_t* w8;   // the pair's message
};

__device__ __forceinline__ SlotPair slot_pair(const EncArgs& A, const BatchArgs& B, u32 p) {
  const u64* pi = A.info + (u64)p * 8;
  SlotPair q;
  q.r = pi[PI_R];
  q.m = pi[PI_M];
  q.ro = A.ref_off ? A.ref_off[p] : 0;
  q.g_lo = A.pair_off[p];
  q.n_new = q.m - __ldcg(B.ptot + (u64)p * PT_COUNT + PT_MATCHED);
  q.w8 = A.wire + A.wire_off[p];
  return q;
}

// One tile of slots; g = this thread's slot source (read one tile ahead).
// The difference d is formed in place of the reference record and its bytes
// are staged before the block scan, at offsets within the warp's range (a
// warp scan); the scan then only places the warp's range in the message.  So
// across the barrier a thread holds no record but the message record, and
// that one waits in the stash.
template <int T, bool PR>
__device__ __forceinline__ void bat_slot(const EncArgs& A, const BatchArgs& B, u32 p,
                                         const SlotPair& q, u64 tile, u32 g, u64* buf,
                                         uint8_t* stage, ulonglong2* stash, U64x2& run) {
  const u64 r = q.r, ro = q.ro;
  const u64 j = tile * T + threadIdx.x;
  Rec cur, d;
  u32 vb = 0, vn = 0;
  if (j < r) {
    // both records in flight at once
    d = load_rec(A.ref + (ro + p + 1 + j) * kRecBytes);
    u32 code = 0xFu;  // placeholder
    if (g != kNoMatch) {
      cur = load_rec(A.rec + ((u64)g + p + 1) * kRecBytes);
#pragma unroll
      for (int w = 0; w < 8; ++w) d.w[w] ^= cur.w[w];
      if constexpr (PR) {
        if (pair_mode<PR>(A, B, p) == kModeResidual) {
          const u64* ps = A.pr.pscr + 4 * (ro + j);
          if (__ldcg(ps + 3)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) d.w[1 + a] = zigzag(cur.w[1 + a] - __ldcg(ps + a));
          }
        }
      }
      u32 b = 0;
      code = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const u32 L = sig_bytes(d.w[w]);
        b += L;
        code |= L << (4 * w);
      }
      vb = b;
      vn = 1;
      stash_put<T>(stash, cur);  // the new reference's record, stored after the scan
    }
    if (in_bounds(A.st, j, 0, r + q.n_new)) reinterpret_cast<u32*>(q.w8 + kHdrBytes)[j] = code;
  }
  // this warp's payload bytes, staged from offset 0 of its stage
  const u32 wincl = warp_incl_scan<u32>(vb);
  const u32 wbytes = __shfl_sync(0xFFFFFFFFu, wincl, 31);
  uint8_t* wst = stage + (threadIdx.x >> 5) * kWarpStage;
  warp_zero(wst, wbytes);
  __syncwarp();
  if (vn) {
    u32 o = wincl - vb;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const u32 L = sig_bytes(d.w[w]);
      stage_or(wst, o, d.w[w], L);
      o += L;
    }
  }
  u64 tot64;
  const u64 ex64 = scan_packed((u64)vb | ((u64)vn << 32), buf, &tot64);
  const U64x2 ex{ex64 & 0xFFFFFFFFull, ex64 >> 32}, tot{tot64 & 0xFFFFFFFFull, tot64 >> 32};
  const U64x2 pre = run;
  run = pre + tot;
  // this warp's bytes start at wstart of the tile's payload
  const u32 wstart = __shfl_sync(0xFFFFFFFFu, (u32)ex.a, 0);
  uint8_t* gW = q.w8 + kHdrBytes + 4 * (r + q.n_new) + pre.a + wstart;
  if (vn) {
    const u64 pos = pre.b + ex.b;
    store_ref_next(A, p, q.g_lo + pos, stash_get<T>(stash));
    if constexpr (PR) {
      if (A.pr.hist_next) {
        const Rec R = load_rec(A.ref + (ro + p + 1 + j) * kRecBytes);
        uint8_t* hn = A.pr.hist_next + kHistBytes * (q.g_lo + pos);
        if (A.pr.hist) {
          const Hist H = load_hist(A.pr.hist + kHistBytes * (ro + j));
          store_hist_next(hn, &R, &H);
        } else {
          store_hist_next(hn, &R, nullptr);
        }
      }
    }
  }
  __syncwarp();
  warp_flush(wst, gW, wbytes);
  __syncwarp();
}

// Header, padding, iteration totals and the new reference's header of pair p
// once every slot and new record is written (warp 0).  slot_tot / new_tot:
// (payload bytes, records) of the slots and of the new records.
template <bool PR>
__device__ __forceinline__ void finish_pair(const EncArgs& A, const BatchArgs& B, u32 p, u64 r,
                                            u64 m, u64 matched, U64x2 slot_tot, U64x2 new_tot) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const u64 n_new = m - matched;
  const u64 payload = slot_tot.a + new_tot.a;
  const u64 body = (u64)kHdrBytes + 4 * (r + n_new) + payload;
  const u64 msg = round16(body);
  const u64 mode = pair_mode<PR>(A, B, p);
  uint8_t* w8 = A.wire + A.wire_off[p];
  // the message fits the slab reserved for it (checked after the fact)
  if (lane == 0) (void)in_bounds(A.st, msg, 0, A.wire_off[p + 1] - A.wire_off[p] + 1);
  if (lane == 0) {
    if (new_tot.b != n_new || slot_tot.b != matched) latch(A.st, TERA_EINVAL);
    ulonglong2* h = reinterpret_cast<ulonglong2*>(w8);
    h[0] = make_ulonglong2((u64)kWireMagic | ((u64)kVersion << 32) | ((u64)kRecBytes << 48),
                           (u64)A.class_id | (mode << 32));
    h[1] = make_ulonglong2(r, n_new);
    h[2] = make_ulonglong2(r - matched, payload);
    h[3] = make_ulonglong2((u64)p, msg);
    A.wire_len[p] = msg;
    atomicAdd(&A.stats->ref_slots, r);
    atomicAdd(&A.stats->holes, r - matched);
    atomicAdd(&A.stats->new_records, n_new);
    atomicAdd(&A.stats->payload_bytes, payload);
    atomicAdd(&A.stats->wire_bytes, msg);
    write_taio_header(A.ref_next + (A.pair_off[p] + p) * kRecBytes, A.class_id, p, m);
    A.reset[p] = 0;
  }
  if (body + lane < msg) w8[body + lane] = 0;  // zero padding (< 16 bytes)
}

// Payload bytes of one word: staged, or stored directly when the tile's
// payload does not fit the stage.
__device__ __forceinline__ void put_word(uint8_t* dst, u32& o, u64 v, u32 L) {
  for (u32 b = 0; b < L; ++b) dst[o++] = (uint8_t)(v >> (8 * b));
}

template <int T, bool PR>
__device__ __forceinline__ void bat_new(const EncArgs& A, const BatchArgs& B, u32 p, u64 tile,
                                        u32 epoch, U64x2* sm, uint8_t* stage, u32 stage_cap,
                                        U64x2& run, U64x2 slot_tot, const SmemTable& tb) {
  u64* pi = A.info + (u64)p * 8;
  const u64 r = pi[PI_R], m = pi[PI_M];
  const u64 matched = __ldcg(B.ptot + (u64)p * PT_COUNT + PT_MATCHED);
  const u64 n_new = m - matched;
  const u64 slot_pay = slot_tot.a;
  const u32 V = new_per_thread(pi[PI_MODE]);
  const u64 g_lo = A.pair_off[p];
  const u64 kb = tile * T * V + (u64)threadIdx.x * V;
  u32 nmask = 0;
  for (u32 i = 0; i < V; ++i) {
    const u64 k = kb + i;
    if (k >= m) continue;
    const bool taken = tb.tbl ? ((tb.bits[k >> 5] >> (k & 31u)) & 1u) != 0u
                              : __ldcg(A.matched + g_lo + k) == epoch;
    if (!taken) nmask |= 1u << i;
  }
  u64 bytes = 0, cnt = 0;
  for (u32 mm = nmask; mm; mm &= mm - 1) {
    const u64 g = g_lo + kb + (u64)(__ffs(mm) - 1);
    const Rec M = load_rec(A.rec + (g + p + 1) * kRecBytes);
    // a second record with the same id in this pair would be found instead of
    // this one (the shared-memory index rejected such records when it was built)
    if (!tb.tbl && seg_lookup<true>(A.seg, epoch, p, g_lo, m, M.w[0]) != (u32)g)
      latch(A.st, TERA_EINVAL);
#pragma unroll
    for (int w = 0; w < 8; ++w) bytes += sig_bytes(M.w[w]);
    ++cnt;
  }
  U64x2 tot;
  const U64x2 ex = tile_scan((u32)bytes, (u32)cnt, sm, &tot);
  const U64x2 pre = run;
  run = pre + tot;
  uint8_t* w8 = A.wire + A.wire_off[p];
  uint8_t* gA = w8 + kHdrBytes + 4 * (r + n_new) + slot_pay + pre.a;
  const u32 s0 = (u32)((uintptr_t)gA & 15u);
  const bool staged = s0 + tot.a <= stage_cap;  // block-uniform
  if (nmask) {
    u32 o = staged ? s0 + (u32)ex.a : 0u;
    uint8_t* dst = staged ? stage : gA + ex.a;
    u64 rank = pre.b + ex.b;
    for (u32 mm = nmask; mm; mm &= mm - 1) {
      const u64 g = g_lo + kb + (u64)(__ffs(mm) - 1);
      const Rec M = load_rec(A.rec + (g + p + 1) * kRecBytes);
      u32 code = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const u32 L = sig_bytes(M.w[w]);
        code |= L << (4 * w);
        put_word(dst, o, M.w[w], L);
      }
      if (in_bounds(A.st, rank, 0, n_new)) reinterpret_cast<u32*>(w8 + kHdrBytes)[r + rank] = code;
      store_ref_next(A, p, g_lo + matched + rank, M);
      if constexpr (PR) {
        if (A.pr.hist_next)
          store_hist_next(A.pr.hist_next + kHistBytes * (g_lo + matched + rank), nullptr, nullptr);
      }
      ++rank;
    }
  }
  __syncthreads();
  if (staged) flush_stage(stage, gA, tot.a);
  __syncthreads();
  // the last tile: header, padding and the iteration totals
  const u64 ntiles = ceil_div(m, (u64)T * V);
  if (tile + 1 < (ntiles ? ntiles : 1)) return;
  finish_pair<PR>(A, B, p, r, m, matched, slot_tot, run);
}

// Shared-memory path: the message records no slot took, in message order,
// into list[0, n) (the hash table's memory, free once matching is done).
// Returns n (block-uniform).
template <int T>
__device__ __forceinline__ u32 smem_new_list(const SmemTable& tb, u64 m, unsigned short* list,
                                             u32* sm32) {
  const u32 words = (u32)((m + 31) / 32);
  const u32 per = (words + T - 1) / T;
  const u32 w0 = threadIdx.x * per, w1 = w0 + per < words ? w0 + per : words;
  u32 cnt = 0;
  for (u32 w = w0; w < w1; ++w) {
    const u32 valid = (w + 1) * 32 <= m ? 0xFFFFFFFFu : ((1u << (m & 31u)) - 1u);
    cnt += __popc(~tb.bits[w] & valid);
  }
  u32 tot;
  u32 pos = block_excl_scan<u32>(cnt, sm32, &tot);
  for (u32 w = w0; w < w1; ++w) {
    const u32 valid = (w + 1) * 32 <= m ? 0xFFFFFFFFu : ((1u << (m & 31u)) - 1u);
    for (u32 x = ~tb.bits[w] & valid; x; x &= x - 1)
      list[pos++] = (unsigned short)(w * 32 + (u32)(__ffs(x) - 1));
  }
  __syncthreads();
  return tot;
}

// One tile of T new records (list entries tile*T + thread): codes, payload
// and new-reference records; the running prefix is carried in `run`.  Every
// list entry is a new record and the list is in message order, so entry i's
// rank among the new records is i: its code and new-reference record are
// written before the block scan, and its payload is staged within the warp's
// range as in the slot step, so no record is held across the barrier.
template <int T, bool PR>
__device__ __forceinline__ void bat_new_list(const EncArgs& A, u32 p, const SlotPair& q,
                                             u64 matched, U64x2 slot_tot,
                                             const unsigned short* list, u32 n_list, u64 tile,
                                             u64* buf, uint8_t* stage, U64x2& run) {
  const u64 r = q.r, n_new = q.m - matched;
  const u64 g_lo = q.g_lo;
  const u64 i = tile * T + threadIdx.x;
  const bool live = i < n_list;
  u32 vb = 0;
  Rec M;
  if (live) {
    M = load_rec(A.rec + (g_lo + list[i] + p + 1) * kRecBytes);
    u32 code = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const u32 L = sig_bytes(M.w[w]);
      vb += L;
      code |= L << (4 * w);
    }
    if (in_bounds(A.st, i, 0, n_new)) reinterpret_cast<u32*>(q.w8 + kHdrBytes)[r + i] = code;
    store_ref_next(A, p, g_lo + matched + i, M);
    if constexpr (PR) {
      if (A.pr.hist_next)
        store_hist_next(A.pr.hist_next + kHistBytes * (g_lo + matched + i), nullptr, nullptr);
    }
  }
  const u32 wincl = warp_incl_scan<u32>(vb);
  const u32 wbytes = __shfl_sync(0xFFFFFFFFu, wincl, 31);
  uint8_t* wst = stage + (threadIdx.x >> 5) * kWarpStage;
  warp_zero(wst, wbytes);
  __syncwarp();
  if (live) {
    u32 o = wincl - vb;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const u32 L = sig_bytes(M.w[w]);
      stage_or(wst, o, M.w[w], L);
      o += L;
    }
  }
  u64 tot;
  const u64 ex = scan_packed((u64)vb, buf, &tot);
  const u64 left = (u64)n_list - tile * T;
  const U64x2 pre = run;
  run = pre + U64x2{tot, left < (u64)T ? left : (u64)T};
  const u32 wstart = __shfl_sync(0xFFFFFFFFu, (u32)ex, 0);
  uint8_t* gW = q.w8 + kHdrBytes + 4 * (r + n_new) + slot_tot.a + pre.a + wstart;
  __syncwarp();
  warp_flush(wst, gW, wbytes);
  __syncwarp();
}

// ---------------- decode phase ----------------

// The L (0..8) bytes at byte offset o of an 8-byte-aligned stage, as a
// little-endian word: two aligned 8-byte loads and a funnel shift (the stage
// is followed by at least 16 bytes of shared memory, so the second load stays
// inside the allocation; bytes past the staged data are masked off).
__device__ __forceinline__ u64 stage_bytes_at(const uint8_t* st, u32 o, u32 L) {
  const u64* w = reinterpret_cast<const u64*>(st + (o & ~7u));
  const u32 sh = (o & 7u) * 8u;
  const u64 lo = w[0], hi = w[1];
  const u64 x = sh ? (lo >> sh) | (hi << (64u - sh)) : lo;
  return L >= 8u ? x : (x & ((1ull << (8u * L)) - 1ull));
}

struct DecShared {
  u64 ns, nn, pay, mode;
  int ok;
};

// Offsets of pair p that every decode tile uses, read once per pair.
struct DecPair {
  u64 ro;             // first slot of the receiver's reference
  u64 rv;             // first record of the receive buffer
  const uint8_t* w8;  // the pair's message
};

__device__ __forceinline__ DecPair dec_pair(const DecArgs& A, u32 p) {
  return DecPair{A.ref_off ? A.ref_off[p] : 0, A.recv_off[p], A.wire + A.wire_off[p]};
}

// One tile of entries; code = this thread's entry code (read one tile ahead).
template <int T, bool PR>
__device__ __forceinline__ void bat_dec_tile(const DecArgs& A, const BatchArgs& B, u32 p,
                                             const DecPair& q, u64 tile, u32 code,
                                             const DecShared& h, u64 m, u64* buf,
                                             uint8_t* stage, ulonglong2* stash, U64x2& run) {
  const u64 ns = h.ns, n = h.ns + h.nn;
  const uint8_t* w8 = q.w8;
  const u64 e = tile * T + threadIdx.x;
  u32 b = 0;
  bool hole = true;
  int bad = 0;
  if (e < n && !check_code(code, e, ns, &hole, &b)) {
    bad = 1;
    b = 0;  // a malformed nibble may claim more than a record: it takes no payload
    latch(A.st, TERA_ECORRUPT);  // malformed code: its entry is not decoded
  }
  // the slot's reference record is copied into the stash while the prefix
  // is found
  if (e < ns && !hole && !bad) stash_async<T>(stash, A.ref + (q.ro + p + 1 + e) * kRecBytes);
  const u32 vn = (e < n && !hole) ? 1u : 0u;
  u64 tot64;
  const u64 ex64 = scan_packed((u64)b | ((u64)vn << 32), buf, &tot64);
  const U64x2 ex{ex64 & 0xFFFFFFFFull, ex64 >> 32}, tot{tot64 & 0xFFFFFFFFull, tot64 >> 32};
  const U64x2 pre = run;
  run = pre + tot;
  // more payload / records than the header announces (block-uniform)
  const bool ok = pre.a + tot.a <= h.pay && pre.b + tot.b <= m;
  if (!ok && threadIdx.x == 0) latch(A.st, TERA_ECORRUPT);
  // this warp's payload bytes [wstart, wend) of the tile, staged with 16-byte
  // loads; the slab is 16-byte aligned and padded, and the range was checked,
  // so the loads stay inside the message
  const u32 wstart = __shfl_sync(0xFFFFFFFFu, (u32)ex.a, 0);
  const u32 wend = __shfl_sync(0xFFFFFFFFu, (u32)ex.a + b, 31);
  const uint8_t* gW = w8 + kHdrBytes + 4 * n + pre.a + wstart;
  const u32 s0 = (u32)((uintptr_t)gW & 15u);
  uint8_t* wst = stage + (threadIdx.x >> 5) * kWarpStage;
  if (ok) {
    const uint8_t* g16 = gW - s0;
    const u32 nchunks = (s0 + (wend - wstart) + 15u) >> 4;
    for (u32 c = threadIdx.x & 31; c < nchunks; c += 32)
      *reinterpret_cast<uint4*>(wst + (c << 4)) =
          __ldcg(reinterpret_cast<const uint4*>(g16 + (c << 4)));
  }
  stash_wait();
  __syncwarp();
  if (ok && vn && !bad) {
    u32 o = s0 + ((u32)ex.a - wstart);
    Rec rec;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const u32 L = (code >> (4 * w)) & 0xFu;
      rec.w[w] = stage_bytes_at(wst, o, L);
      o += L;
    }
    const u64 pos = pre.b + ex.b;
    if (e < ns) {
      const Rec R = stash_get<T>(stash);
      bool pred_ok = false;
      u64 pred[3];
      if constexpr (PR) {
        Hist H;
        if (A.pr.hist) H = load_hist(A.pr.hist + kHistBytes * (q.ro + e));
        // the receiver's own prediction, made by the pre-pass (a residual
        // message needs the network, so the header check has rejected one
        // that arrives without it)
        if (A.pr.pre && h.mode == kModeResidual) {
          const u64* ps = A.pr.pscr + 4 * (q.ro + e);
          pred_ok = __ldcg(ps + 3) != 0;
#pragma unroll
          for (int a = 0; a < 3; ++a) pred[a] = __ldcg(ps + a);
        }
        if (A.pr.hist_next)
          store_hist_next(A.pr.hist_next + kHistBytes * (q.rv + pos), &R,
                          A.pr.hist ? &H : nullptr);
      }
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        if (pred_ok && w >= 1 && w <= 3) rec.w[w] = pred[w - 1] + unzigzag(rec.w[w]);
        else rec.w[w] ^= R.w[w];
      }
    } else {
      if constexpr (PR) {
        if (A.pr.hist_next)
          store_hist_next(A.pr.hist_next + kHistBytes * (q.rv + pos), nullptr, nullptr);
      }
    }
    if (in_bounds(A.st, pos, 0, m)) store_rec(A.recv + (q.rv + p + 1 + pos) * kRecBytes, rec);
  }
  __syncwarp();
  // the last tile: every byte and record the header announced was decoded
  if (ok && threadIdx.x == 0 && tile + 1 == (n ? ceil_div(n, T) : 1) &&
      (pre.a + tot.a != h.pay || pre.b + tot.b != m))
    latch(A.st, TERA_ECORRUPT);
}

// Header of pair p's received message (thread 0 reads and checks it; the
// first caller of a pair also latches its error and writes the receive
// buffer's TAIO header).  Returns the facts to every thread.
template <bool PR>
__device__ __forceinline__ DecShared dec_header(const DecArgs& A, u32 p, u64 m, DecShared* hs,
                                                bool first) {
  if (threadIdx.x == 0) {
    DecHdr H;
    const u32 err = dec_read_header<true, PR>(A, p, m, &H);
    hs->ns = H.ns;
    hs->nn = H.nn;
    hs->pay = H.pay;
    hs->mode = H.mode;
    hs->ok = err ? 0 : 1;
    if (first) {
      if (err) latch(A.st, err);
      write_taio_header(A.recv + (A.recv_off[p] + p) * kRecBytes, A.class_id, p, m);
    }
  }
  __syncthreads();
  return *hs;
}

// Facts of one entry of a decode tile from its code.
struct DecEnt {
  u32 b, vn;  // payload bytes, record decoded (not a placeholder)
  bool hole;
  bool bad;   // malformed code: not decoded, no payload
};

__device__ __forceinline__ DecEnt dec_entry(DevStatus* st, u32 code, u64 e, u64 n, u64 ns) {
  DecEnt x{0u, 0u, true, false};
  if (e < n && !check_code(code, e, ns, &x.hole, &x.b)) {
    x.bad = true;
    x.b = 0;
    latch(st, TERA_ECORRUPT);
  }
  x.vn = (e < n && !x.hole) ? 1u : 0u;
  return x;
}

// The decode step of pair p (no predictor) as bat_dec_tile, software
// pipelined: a tile's byte counts come from its codes alone, so the block
// scan of tile t + 1 runs while tile t's payload and reference records are
// in flight (both copied into shared memory by cp.async), and tile t's
// payload is requested as soon as the tile starts.
template <int T>
__device__ __forceinline__ void dec_tiles_pipelined(const DecArgs& A, u32 p, const DecPair& q,
                                                    const DecShared& h, u64 m, u64* bufs,
                                                    uint8_t* stage, ulonglong2* stash) {
  const u64 ns = h.ns, n = h.ns + h.nn;
  const u64 ntiles = n ? ceil_div(n, T) : 1;
  const u32* codes = reinterpret_cast<const u32*>(q.w8 + kHdrBytes);
  const uint8_t* pay = q.w8 + kHdrBytes + 4 * n;
  uint8_t* wst = stage + (threadIdx.x >> 5) * kWarpStage;
  u64 e = threadIdx.x;
  u32 code = e < n ? __ldcg(codes + e) : 0u;
  u32 c_next = e + T < n ? __ldcg(codes + e + T) : 0u;
  DecEnt x = dec_entry(A.st, code, e, n, ns);
  u64 tot64;
  u64 ex64 = scan_packed((u64)x.b | ((u64)x.vn << 32), bufs, &tot64);
  U64x2 run{0, 0};
  for (u64 t = 0; t < ntiles; ++t, e += T) {
    const U64x2 ex{ex64 & 0xFFFFFFFFull, ex64 >> 32}, tot{tot64 & 0xFFFFFFFFull, tot64 >> 32};
    const U64x2 pre = run;
    run = pre + tot;
    // more payload / records than the header announces (block-uniform)
    const bool ok = pre.a + tot.a <= h.pay && pre.b + tot.b <= m;
    if (!ok && threadIdx.x == 0) latch(A.st, TERA_ECORRUPT);
    // this warp's payload bytes [wstart, wend) of the tile; the slab is
    // 16-byte aligned and padded, and the range was checked, so the copies
    // stay inside the message
    const u32 wstart = __shfl_sync(0xFFFFFFFFu, (u32)ex.a, 0);
    const u32 wend = __shfl_sync(0xFFFFFFFFu, (u32)ex.a + x.b, 31);
    const uint8_t* gW = pay + pre.a + wstart;
    const u32 s0 = (u32)((uintptr_t)gW & 15u);
    if (ok) {
      const uint8_t* g16 = gW - s0;
      const u32 n16 = (s0 + (wend - wstart) + 15u) >> 4;
      for (u32 k = threadIdx.x & 31; k < n16; k += 32) {
        const u32 dst = (u32)__cvta_generic_to_shared(wst + (k << 4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" : : "r"(dst), "l"(g16 + (k << 4))
                     : "memory");
      }
    }
    if (e < ns && !x.hole && !x.bad) stash_async<T>(stash, A.ref + (q.ro + p + 1 + e) * kRecBytes);
    asm volatile("cp.async.commit_group;" : : : "memory");
    // the next tile's facts and prefix while the copies are in flight
    const DecEnt xt = x;
    const u32 ct = code;
    code = c_next;
    const u64 e2 = e + 2 * (u64)T;
    c_next = e2 < n ? __ldcg(codes + e2) : 0u;
    if (t + 1 < ntiles) {  // block-uniform
      x = dec_entry(A.st, code, e + T, n, ns);
      ex64 = scan_packed((u64)x.b | ((u64)x.vn << 32), bufs + 33 * ((t + 1) & 1), &tot64);
    }
    stash_wait();
    __syncwarp();
    if (ok && xt.vn && !xt.bad) {
      u32 o = s0 + ((u32)ex.a - wstart);
      Rec rec;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const u32 L = (ct >> (4 * w)) & 0xFu;
        rec.w[w] = stage_bytes_at(wst, o, L);
        o += L;
      }
      if (e < ns) {
        const Rec R = stash_get<T>(stash);
#pragma unroll
        for (int w = 0; w < 8; ++w) rec.w[w] ^= R.w[w];
      }
      if (in_bounds(A.st, pre.b + ex.b, 0, m))
        store_rec(A.recv + (q.rv + p + 1 + pre.b + ex.b) * kRecBytes, rec);
    }
    __syncwarp();
    // the last tile: every byte and record the header announced was decoded
    if (ok && threadIdx.x == 0 && t + 1 == ntiles && (run.a != h.pay || run.b != m))
      latch(A.st, TERA_ECORRUPT);
  }
}

template <int T, bool PR>
__device__ __forceinline__ void bat_dec(const DecArgs& A, const BatchArgs& B, u32 p,
                                        DecShared* hs, u64* bufs, uint8_t* stage,
                                        ulonglong2* stash) {
  const u64 m = A.recv_off[p + 1] - A.recv_off[p];
  const DecShared h = dec_header<PR>(A, p, m, hs, true);
  if (!h.ok) return;  // block-uniform
  const u64 n = h.ns + h.nn;
  const DecPair q = dec_pair(A, p);
  if constexpr (!PR) {
    dec_tiles_pipelined<T>(A, p, q, h, m, bufs, stage, stash);
    __syncthreads();  // the scan buffers and the stage are reused next
    return;
  }
  const u64 ntiles = n ? ceil_div(n, T) : 1;
  U64x2 run{0, 0};
  const u32* codes = reinterpret_cast<const u32*>(q.w8 + kHdrBytes);
  u32 c_next = threadIdx.x < n ? __ldcg(codes + threadIdx.x) : 0u;
  for (u64 t = 0; t < ntiles; ++t) {
    const u32 c = c_next;
    const u64 en = (t + 1) * T + threadIdx.x;
    c_next = en < n ? __ldcg(codes + en) : 0u;
    bat_dec_tile<T, PR>(A, B, p, q, t, c, h, m, bufs + 33 * (t & 1), stage, stash, run);
  }
  __syncthreads();  // the scan buffers and the stage are reused next
}

// ---------------- pairs carried by a team of blocks ----------------

__device__ __forceinline__ u32 ld_acquire(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(u32* p, u32 v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u64 global_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Backstop on the number of polls of one wait, should the global timer not
// advance: a poll (an L2 round trip plus a 64 ns sleep) takes far longer than
// 16 ns, so the time limit always ends the wait first.
__device__ __forceinline__ u64 spin_cap(u64 limit_ns) { return limit_ns / 16 + 1024; }

// Every member of a team arrives, then waits for the others, for at most
// limit_ns nanoseconds of the global timer.  The members were claimed, in
// list order, by running blocks that wait for nothing else, so the wait ends
// when every member can be resident at once.  Returns false (block-uniform)
// when it gave up: TERA_ETIMEOUT is latched, and the caller abandons the pair
// without touching its outputs again.  A member that returns true has seen
// every member arrive, so everything the team wrote before the barrier is
// complete.
__device__ __forceinline__ bool team_barrier(u32* ctr, u32 g, DevStatus* st, u64 limit_ns) {
  __syncthreads();
  int late = 0;
  if (threadIdx.x == 0) {
    red_release_add(ctr, 1u);
    const u64 t0 = global_ns();
    const u64 cap = spin_cap(limit_ns);
    u64 spin = 0;
    while (ld_acquire(ctr) < g) {
      if (global_ns() - t0 > limit_ns || ++spin > cap) {
        latch(st, TERA_ETIMEOUT);
        late = 1;
        break;
      }
      __nanosleep(64);
    }
  }
  return __syncthreads_or(late) == 0;
}

// Block sum of two counts (red: 66 words of shared memory).
__device__ __forceinline__ U64x2 block_sum2(u64 a, u64 b, u64* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    red[warp] = a;
    red[32 + warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 sa = 0, sb = 0;
    for (int w = 0; w < nwarps; ++w) {
      sa += red[w];
      sb += red[32 + w];
    }
    red[64] = sa;
    red[65] = sb;
  }
  __syncthreads();
  const U64x2 r{red[64], red[65]};
  __syncthreads();
  return r;
}

// Sum of the first t tile totals.
template <int T>
__device__ __forceinline__ U64x2 tiles_prefix(const U64x2* ts, u64 t, u64* red) {
  u64 a = 0, b = 0;
  for (u64 x = threadIdx.x; x < t; x += T) {
    const U64x2 v = ldx<true>(ts + x);
    a += v.a;
    b += v.b;
  }
  return block_sum2(a, b, red);
}

// Totals (payload bytes, matched) of one slot tile: the bytes bat_slot
// writes (XOR difference, or with the predictor in residual mode the
// residual on the position words of each predictable slot).
template <int T, bool PR>
__device__ __forceinline__ void team_slot_sum(const EncArgs& A, const BatchArgs& B, u32 p, u64 r,
                                              u64 ro, u64 tile, U64x2* ts, u64* red) {
  const u64 j = tile * T + threadIdx.x;
  u64 b = 0, f = 0;
  if (j < r) {
    const u32 g = __ldcg(A.slot_src + ro + j);
    if (g != kNoMatch) {
      const Rec R = load_rec(A.ref + (ro + p + 1 + j) * kRecBytes);
      const Rec M = load_rec(A.rec + ((u64)g + p + 1) * kRecBytes);
      Rec d;
#pragma unroll
      for (int w = 0; w < 8; ++w) d.w[w] = R.w[w] ^ M.w[w];
      if constexpr (PR) {
        if (pair_mode<PR>(A, B, p) == kModeResidual) {
          const u64* ps = A.pr.pscr + 4 * (ro + j);
          if (__ldcg(ps + 3)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) d.w[1 + a] = zigzag(M.w[1 + a] - __ldcg(ps + a));
          }
        }
      }
#pragma unroll
      for (int w = 0; w < 8; ++w) b += sig_bytes(d.w[w]);
      f = 1;
    }
  }
  const U64x2 t = block_sum2(b, f, red);
  if (threadIdx.x == 0) ts[tile] = t;
}

// Totals (payload bytes, records) of the new records of one new-record tile
// (entries as in bat_new: V per thread).
template <int T>
__device__ __forceinline__ void team_new_sum(const EncArgs& A, u32 p, u64 m, u32 V, u64 tile,
                                             u32 epoch, U64x2* ns, u64* red) {
  const u64 g_lo = A.pair_off[p];
  const u64 kb = tile * T * V + (u64)threadIdx.x * V;
  u64 b = 0, c = 0;
  for (u32 i = 0; i < V; ++i) {
    const u64 k = kb + i;
    if (k >= m || __ldcg(A.matched + g_lo + k) == epoch) continue;
    const Rec M = load_rec(A.rec + (g_lo + k + p + 1) * kRecBytes);
#pragma unroll
    for (int w = 0; w < 8; ++w) b += sig_bytes(M.w[w]);
    ++c;
  }
  const U64x2 t = block_sum2(b, c, red);
  if (threadIdx.x == 0) ns[tile] = t;
}

// Totals (payload bytes, records) of one decode tile, from the codes.
template <int T>
__device__ __forceinline__ void team_dec_sum(const DecArgs& A, u32 p, const DecShared& h,
                                             u64 tile, U64x2* ds, u64* red) {
  const u64 ns = h.ns, n = h.ns + h.nn;
  const u64 e = tile * T + threadIdx.x;
  u64 b = 0, f = 0;
  if (e < n) {
    const u32 code = __ldcg(reinterpret_cast<const u32*>(A.wire + A.wire_off[p] + kHdrBytes) + e);
    bool hole;
    u32 bb;
    if (!check_code(code, e, ns, &hole, &bb)) {
      latch(A.st, TERA_ECORRUPT);
      bb = 0;  // as in bat_dec_tile: a malformed entry takes no payload
    }
    b = bb;
    f = hole ? 0 : 1;
  }
  const U64x2 t = block_sum2(b, f, red);
  if (threadIdx.x == 0) ds[tile] = t;
}

// Member i of a team of g blocks carries its share of pair p's tiles through
// every step (global hash segments).  Team barriers separate the steps; the
// payload positions of a member's tiles come from the sums of all tile totals
// before them (written in a first pass over the tiles).  With the predictor,
// both sides' cell counts are taken with the index (before the first
// barrier), the match makes the predictions and the residual sizes, and the
// message mode is read once the match is complete.
template <int T, bool PR>
__device__ __noinline__ void team_pair(const EncArgs& E, const DecArgs& D, const BatchArgs& B,
                                          u32 p, u32 i, u32 g, u32 epoch, U64x2* sm, u64* red,
                                          uint8_t* stage, ulonglong2* stash, DecShared* hs) {
  constexpr u32 kStageCap = (u32)T * kRecBytes + 48;
  const u64* pi = E.info + (u64)p * 8;
  const u64 r = pi[PI_R], m = pi[PI_M];
  const u64 ro = E.ref_off ? E.ref_off[p] : 0;
  u32* ctr = B.team + (u64)p * 8;
  u64* bufs = reinterpret_cast<u64*>(sm);
  const u64 nst = ceil_div(r, T);
  for (u64 t = i; t < ceil_div(m, (u64)T * kIlp); t += g) bat_build<T>(E, p, t, epoch);
  if constexpr (PR) {
    // cell counts for the training samples when no pre-pass has made them
    if (E.pr.hist && E.pr.samples && !E.pr.pre)
      for (u64 t = i; t < nst; t += g) cells_unit(E.pr, E.ref, E.ref_off, p, t, r, T);
  }
  if (!team_barrier(ctr + 0, g, E.st, B.wait_ns)) return;
  if constexpr (PR) {
    for (u64 t = i; t < nst; t += g) bat_match<T, PR>(E, B, p, t, epoch, sm);
  } else {
    for (u64 t = i; t < ceil_div(r, (u64)T * kIlp); t += g) bat_match_ilp<T>(E, B, p, t, epoch);
  }
  if (!team_barrier(ctr + 1, g, E.st, B.wait_ns)) return;
  const u32 V = new_per_thread(pi[PI_MODE]);
  const u64 ntn = ceil_div(m, (u64)T * V);
  U64x2* ts = B.tsum + B.tbase[p];
  U64x2* nts = ts + nst;
  for (u64 t = i; t < nst; t += g) team_slot_sum<T, PR>(E, B, p, r, ro, t, ts, red);
  for (u64 t = i; t < ntn; t += g) team_new_sum<T>(E, p, m, V, t, epoch, nts, red);
  if (!team_barrier(ctr + 2, g, E.st, B.wait_ns)) return;
  u32 k = 0;
  const SlotPair q = slot_pair(E, B, p);
  for (u64 t = i; t < nst; t += g, ++k) {
    U64x2 run = tiles_prefix<T>(ts, t, red);
    const u64 j = t * T + threadIdx.x;
    const u32 src = j < r ? __ldcg(E.slot_src + ro + j) : kNoMatch;
    bat_slot<T, PR>(E, B, p, q, t, src, bufs + 33 * (k & 1), stage, stash, run);
  }
  __syncthreads();
  // the new records (the member with the last new tile writes the header)
  const U64x2 slot_tot = tiles_prefix<T>(ts, nst, red);
  const SmemTable none{nullptr, 0u, nullptr};
  for (u64 t = i; t < (ntn ? ntn : 1); t += g) {
    U64x2 run = tiles_prefix<T>(nts, t, red);
    bat_new<T, PR>(E, B, p, t, epoch, sm, stage, kStageCap, run, slot_tot, none);
  }
  if (!team_barrier(ctr + 3, g, E.st, B.wait_ns)) return;
  const u64 mr = D.recv_off[p + 1] - D.recv_off[p];
  const DecShared h = dec_header<PR>(D, p, mr, hs, i == 0);
  const u64 n = h.ok ? h.ns + h.nn : 0;
  const u64 ndt = h.ok ? (n ? ceil_div(n, T) : 1) : 0;
  U64x2* ds = nts + ceil_div(m, T);
  for (u64 t = i; t < ndt; t += g) team_dec_sum<T>(D, p, h, t, ds, red);
  if (!team_barrier(ctr + 4, g, E.st, B.wait_ns)) return;
  const DecPair dq = dec_pair(D, p);
  const u32* codes = reinterpret_cast<const u32*>(dq.w8 + kHdrBytes);
  k = 0;
  for (u64 t = i; t < ndt; t += g, ++k) {
    U64x2 run = tiles_prefix<T>(ds, t, red);
    const u64 e = t * T + threadIdx.x;
    const u32 c = e < n ? __ldcg(codes + e) : 0u;
    bat_dec_tile<T, PR>(D, B, p, dq, t, c, h, mr, bufs + 33 * (k & 1), stage, stash, run);
  }
  __syncthreads();
}

// ---------------- the predictor's pre-pass ----------------
//
// A slot's prediction depends only on its reference record, its history and
// the cell counts of its pair's reference, not on the message: each side makes
// the predictions of its own reference before the codec runs, over every slot
// of every pair at once: the cell counts, the features (one thread per slot,
// few registers, so that many loads are in flight), then the network (two
// slots per thread, in a kernel with room for both slots' accumulators).  The
// codec then reads them.

// The pair of slot g of an arena laid out with off[0..P] (off[p] <= g < off[p+1]).
__device__ __forceinline__ u32 pair_of_slot(const u64* __restrict__ off, u32 P, u64 g) {
  u32 lo = 0, hi = P;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Slots the pre-pass covers: the reference's, or none when they exceed the
// cap slots its scratch holds (the codec's setup then reports the capacity
// error before any use of the predictions).
__device__ __forceinline__ u64 prepass_slots(const u64* __restrict__ off, u32 P, u64 cap) {
  const u64 n = off[P];
  return n <= cap ? n : 0;
}

// The slots [*g0, *g1) of the calling warp: the arena's slots split into
// equal runs of whole 32-slot steps, one run per warp of the grid, so that a
// warp finds the pair of its first slot once and then walks the pairs.
__device__ __forceinline__ void warp_run(u64 total, u64* g0, u64* g1) {
  const u64 wpb = blockDim.x / 32;
  const u64 nw = (u64)gridDim.x * wpb;
  const u64 w = (u64)blockIdx.x * wpb + threadIdx.x / 32;
  const u64 per = ceil_div(ceil_div(total, 32), nw) * 32;
  const u64 a = w * per, b = a + per;
  *g0 = a < total ? a : total;
  *g1 = b < total ? b : total;
}

// Every reference record counted in its cell (segments zeroed before).
__global__ void __launch_bounds__(256) pred_cells_kernel(PredArgs pr, const uint8_t* __restrict__ ref,
                                                         const u64* __restrict__ off, u32 P,
                                                         u64 cap) {
  u64 g0, g1;
  warp_run(prepass_slots(off, P, cap), &g0, &g1);
  if (g0 >= g1) return;
  u32 p = pair_of_slot(off, P, g0);
  for (u64 g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
    while (__ldg(off + p + 1) <= g) ++p;
    const u64 o = __ldg(off + p), r = __ldg(off + p + 1) - o;
    const Rec R = load_rec(ref + (g + p + 1) * kRecBytes);
    cell_insert(pr.cseg, seg_base(o, p), seg_size(r), cell_key(R, pr));
  }
}

// The network's weights in shared memory with layer 2 stored by columns: the
// weights of hidden input k for neurons 0 .. 63 at kMlpW2 + 64 k (the other
// arrays as in the parameter vector).
__device__ __forceinline__ void load_mlp_cols(float* sW, const float* __restrict__ params) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    int d = i;
    if (i >= kMlpW2 && i < kMlpW2 + kMlpH * kMlpH) {
      const int j = (i - kMlpW2) / kMlpH, k = (i - kMlpW2) % kMlpH;
      d = kMlpW2 + k * kMlpH + j;
    }
    sW[d] = __ldg(params + i);
  }
  __syncthreads();
}

// First-layer neuron k of one feature vector: its bias, then the inputs in
// ascending order, then ReLU (as mlp_infer).
__device__ __forceinline__ float hidden1(const float4 wa, const float4 wb, float bias,
                                         const float* f) {
  float h = bias;
  h = __fmaf_rn(wa.x, f[0], h);
  h = __fmaf_rn(wa.y, f[1], h);
  h = __fmaf_rn(wa.z, f[2], h);
  h = __fmaf_rn(wa.w, f[3], h);
  h = __fmaf_rn(wb.x, f[4], h);
  h = __fmaf_rn(wb.y, f[5], h);
  h = __fmaf_rn(wb.z, f[6], h);
  h = __fmaf_rn(wb.w, f[7], h);
  return h > 0.0f ? h : 0.0f;
}

// The network on two feature vectors A and B with the same fused
// multiply-adds, in the same order per neuron, as mlp_infer (so the same
// bits), each weight read from shared memory once for both vectors.  The
// second layer runs in two halves of 32 neurons (the first layer is made
// again for each half, one neuron k at a time, and its output enters the
// half's 32 accumulators of both vectors); each second-layer neuron adds its
// inputs k = 0 .. 63 in ascending order, and each output adds j = 0 .. 63 in
// ascending order across the halves.
__device__ __forceinline__ void mlp_infer_pair(const float* __restrict__ sW, const float* fA,
                                               const float* fB, float* oA, float* oB) {
  const float4* W4 = reinterpret_cast<const float4*>(sW);
#pragma unroll
  for (int a = 0; a < kMlpOut; ++a) oA[a] = oB[a] = sW[kMlpB3 + a];
#pragma unroll 1
  for (int hf = 0; hf < 2; ++hf) {
    float accA[32], accB[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) accA[j] = accB[j] = sW[kMlpB2 + 32 * hf + j];
#pragma unroll 1
    for (int k = 0; k < kMlpH; ++k) {
      const float4 wa = W4[(kMlpW1 + k * kMlpIn) / 4], wb = W4[(kMlpW1 + k * kMlpIn) / 4 + 1];
      const float bias = sW[kMlpB1 + k];
      const float hA = hidden1(wa, wb, bias, fA), hB = hidden1(wa, wb, bias, fB);
      const float4* col = W4 + (kMlpW2 + k * kMlpH + 32 * hf) / 4;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 w = col[q];
        accA[4 * q] = __fmaf_rn(w.x, hA, accA[4 * q]);
        accB[4 * q] = __fmaf_rn(w.x, hB, accB[4 * q]);
        accA[4 * q + 1] = __fmaf_rn(w.y, hA, accA[4 * q + 1]);
        accB[4 * q + 1] = __fmaf_rn(w.y, hB, accB[4 * q + 1]);
        accA[4 * q + 2] = __fmaf_rn(w.z, hA, accA[4 * q + 2]);
        accB[4 * q + 2] = __fmaf_rn(w.z, hB, accB[4 * q + 2]);
        accA[4 * q + 3] = __fmaf_rn(w.w, hA, accA[4 * q + 3]);
        accB[4 * q + 3] = __fmaf_rn(w.w, hB, accB[4 * q + 3]);
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float h2A = accA[j] > 0.0f ? accA[j] : 0.0f, h2B = accB[j] > 0.0f ? accB[j] : 0.0f;
#pragma unroll
      for (int a = 0; a < kMlpOut; ++a) {
        const float w = sW[kMlpW3 + a * kMlpH + 32 * hf + j];
        oA[a] = __fmaf_rn(w, h2A, oA[a]);
        oB[a] = __fmaf_rn(w, h2B, oB[a]);
      }
    }
  }
}

// Every reference slot's features into out[4 g .. 4 g + 3] (8 floats), the
// first one a NaN when the slot is not predictable (features() false; a
// predictable slot's features are all finite).
__global__ void __launch_bounds__(256) pred_features_kernel(PredArgs pr,
                                                            const uint8_t* __restrict__ ref,
                                                            const u64* __restrict__ off, u32 P,
                                                            u64 cap, u64* __restrict__ out) {
  u64 g0, g1;
  warp_run(prepass_slots(off, P, cap), &g0, &g1);
  if (g0 >= g1) return;
  u32 p = pair_of_slot(off, P, g0);
  for (u64 g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
    while (__ldg(off + p + 1) <= g) ++p;
    const u64 o0 = __ldg(off + p), r = __ldg(off + p + 1) - o0;
    const Rec R = load_rec(ref + (g + p + 1) * kRecBytes);
    const Hist H = load_hist(pr.hist + kHistBytes * g);
    const u32 nc = cell_count(pr.cseg, seg_base(o0, p), seg_size(r), cell_key(R, pr));
    float f[kMlpIn];
    if (!features(R, H, nc, f)) f[0] = __int_as_float(0x7FC00000);
    float4* o = reinterpret_cast<float4*>(out + 4 * g);
    o[0] = make_float4(f[0], f[1], f[2], f[3]);
    o[1] = make_float4(f[4], f[5], f[6], f[7]);
  }
}

// One slot's features from out (read before its prediction replaces them);
// false when the slot is not predictable.
__device__ __forceinline__ bool load_features(const u64* out, u64 g, float* f) {
  const float4* fi = reinterpret_cast<const float4*>(out + 4 * g);
  const float4 a = __ldcs(fi), b = __ldcs(fi + 1);
  const bool ok = !isnan(a.x);
  f[0] = ok ? a.x : 0.0f;
  f[1] = ok ? a.y : 0.0f;
  f[2] = ok ? a.z : 0.0f;
  f[3] = ok ? a.w : 0.0f;
  f[4] = ok ? b.x : 0.0f;
  f[5] = ok ? b.y : 0.0f;
  f[6] = ok ? b.z : 0.0f;
  f[7] = ok ? b.w : 0.0f;
  return ok;
}

// The prediction of slot g (pair p) from the network's output, into
// out[4 g .. 4 g + 3]: bits of the three predicted positions and whether it
// is usable.
__device__ __forceinline__ void store_pred(const uint8_t* __restrict__ ref, u32 p, u64* out,
                                           u64 g, const float* y, bool ok) {
  u64 pred[3] = {0, 0, 0};
  if (ok) {
    const u64* rp = reinterpret_cast<const u64*>(ref + (g + p + 1) * kRecBytes);
    Rec R;
    R.w[1] = __ldg(rp + 1);
    R.w[2] = __ldg(rp + 2);
    R.w[3] = __ldg(rp + 3);
    ok = predict_out(R, y, pred);
  }
  ulonglong2* o = reinterpret_cast<ulonglong2*>(out + 4 * g);
  o[0] = make_ulonglong2(pred[0], pred[1]);
  o[1] = make_ulonglong2(pred[2], ok ? 1ull : 0ull);
}

// Every reference slot's prediction from its features (in out[4 g .. 4 g +
// 3], replaced).  A thread takes two slots of its warp's run at a time (gA
// and gA + 32) and runs the network on both at once.
__global__ void __launch_bounds__(256, 2) pred_slots_kernel(PredArgs pr,
                                                            const uint8_t* __restrict__ ref,
                                                            const u64* __restrict__ off, u32 P,
                                                            u64 cap, u64* __restrict__ out) {
  __shared__ __align__(16) float sW[(kMlpParams + 3) & ~3];
  load_mlp_cols(sW, pr.params);
  u64 g0, g1;
  warp_run(prepass_slots(off, P, cap), &g0, &g1);
  if (g0 >= g1) return;
  u32 pA = pair_of_slot(off, P, g0), pB = pA;
  for (u64 gA = g0 + (threadIdx.x & 31); gA < g1; gA += 64) {
    const bool liveB = gA + 32 < g1;
    const u64 gB = liveB ? gA + 32 : gA;
    float fA[kMlpIn], fB[kMlpIn];
    const bool okA = load_features(out, gA, fA);
    const bool okB = liveB && load_features(out, gB, fB);
    if (!liveB)
      for (int i = 0; i < kMlpIn; ++i) fB[i] = 0.0f;
    float yA[kMlpOut] = {0.0f, 0.0f, 0.0f}, yB[kMlpOut] = {0.0f, 0.0f, 0.0f};
    if (__any_sync(__activemask(), okA || okB)) mlp_infer_pair(sW, fA, fB, yA, yB);
    while (__ldg(off + pA + 1) <= gA) ++pA;
    store_pred(ref, pA, out, gA, yA, okA);
    if (liveB) {
      if (pB < pA) pB = pA;
      while (__ldg(off + pB + 1) <= gB) ++pB;
      store_pred(ref, pB, out, gB, yB, okB);
    }
  }
}

// Zeroes the cell counts' segments of every pair of a reference laid out
// with off[0..P] (seg_base(off[P], P) entries of 16 bytes; the segments are
// contiguous), the part of the cell hash the codec and the pre-pass use, at
// most the cap entries allocated.
__global__ void __launch_bounds__(256) cells_clear_kernel(u64* __restrict__ cseg,
                                                          const u64* __restrict__ off, u32 P,
                                                          u64 cap) {
  const u64 used = seg_base(off[P], P);
  const u64 n = used < cap ? used : cap;
  ulonglong2* c = reinterpret_cast<ulonglong2*>(cseg);
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    c[i] = make_ulonglong2(0ull, 0ull);
}

static tera_status cells_clear(tera_ctx* ctx, u64* cseg, const u64* off, cudaStream_t s) {
  prof_begin(ctx, s);
  const u64 P = ctx->n_pairs;
  cells_clear_kernel<<<(unsigned)(ctx->num_sms * 4), 256, 0, s>>>(cseg, off, (u32)P,
                                                                  2 * ctx->pred_cap + 2 * P);
  return check_launch(ctx, "cells_clear_kernel", s);
}

static tera_status pred_prepass(tera_ctx* ctx, const PredArgs& pr, const uint8_t* ref,
                                const u64* off, u64* out, cudaStream_t s) {
  const unsigned grid = (unsigned)(ctx->num_sms * 2);
  prof_begin(ctx, s);
  const u64 cap = ctx->pred_cap;
  pred_cells_kernel<<<grid, 256, 0, s>>>(pr, ref, off, (u32)ctx->n_pairs, cap);
  tera_status st = check_launch(ctx, "pred_cells_kernel", s);
  if (st != TERA_OK) return st;
  prof_begin(ctx, s);
  pred_features_kernel<<<(unsigned)(ctx->num_sms * 8), 256, 0, s>>>(pr, ref, off,
                                                                   (u32)ctx->n_pairs, cap, out);
  if ((st = check_launch(ctx, "pred_features_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  pred_slots_kernel<<<grid, 256, 0, s>>>(pr, ref, off, (u32)ctx->n_pairs, cap, out);
  return check_launch(ctx, "pred_slots_kernel", s);
}

// ---------------- the persistent kernel ----------------

// Shared memory, for c = table_records: one region that holds the hash table
// (up to 2c u16 entries, match step), then the list of new records (c u16,
// new step) or the record stash (T records, slot and decode steps),
// followed by the stage (the block's T records + 48 bytes for the new step,
// or one region per warp for the slot and decode steps) | MLP weights
// (predictor) | taken bits (c / 8).
__host__ __device__ constexpr size_t stage_bytes(u32 T) {
  // the block stage (T records + 48 bytes) or the warps' stages, the larger
  return (size_t)(T / 32) * kWarpStage > (size_t)T * kRecBytes + 48 ? (size_t)(T / 32) * kWarpStage
                                                                      : (size_t)T * kRecBytes + 48;
}
__host__ __device__ constexpr size_t stash_bytes(u32 T) { return (size_t)T * kRecBytes; }
// where the stage starts: after the list and after the stash
__host__ __device__ constexpr size_t stage_off(u32 T, u32 c) {
  return 2 * (size_t)c > stash_bytes(T) ? 2 * (size_t)c : stash_bytes(T);
}
__host__ __device__ constexpr size_t region_bytes(u32 T, u32 c) {
  return (4 * (size_t)c > stage_off(T, c) + stage_bytes(T)) ? 4 * (size_t)c
                                                            : stage_off(T, c) + stage_bytes(T);
}

template <int T, bool PR>
__global__ void __launch_bounds__(T, (1024 / T) > 0 ? (1024 / T) : 1)
    codec_persistent_kernel(EncArgs E, DecArgs D, BatchArgs B, u32 table_records) {
  extern __shared__ __align__(16) uint8_t dyn[];
  constexpr u32 kStageCap = (u32)T * kRecBytes + 48;
  const size_t region = region_bytes(T, table_records);
  unsigned short* tbl = reinterpret_cast<unsigned short*>(dyn);
  unsigned short* list = tbl;
  uint8_t* stage = dyn + stage_off(T, table_records);
  ulonglong2* stash = reinterpret_cast<ulonglong2*>(dyn);
  u32* bits = reinterpret_cast<u32*>(dyn + region);
  __shared__ U64x2 sm[33];
  __shared__ u64 red[66];
  __shared__ u64 s_item;
  __shared__ u32 s_cnt;
  __shared__ DecShared hs;
  const u32 epoch = __ldcg(E.epoch);
  // this launch's range of the work list (see BatchArgs)
  const u64 first = B.part ? __ldcg(B.n_first) : 0;
  const u64 n_items = B.part ? __ldcg(B.n_items) : __ldcg(B.n_first);
  u64* ticket = B.part ? B.ticket_small : B.ticket;
  if (threadIdx.x == 0) s_cnt = 0;
  for (;;) {
    // claim the next item only when this block is free: a team member never
    // waits for an item that a busy block holds
    if (threadIdx.x == 0) {
      const u64 t = first + atomicAdd(ticket, 1ull);
      s_item = (t < n_items && !*(volatile u32*)B.abort) ? B.items[t] : ~0ull;
    }
    __syncthreads();
    const u64 it = s_item;
    if (it == ~0ull) break;
    const u32 p = (u32)(it >> 32);
    const u32 g = (u32)it & 0xFFFFu;
    if (g > 1) {
      team_pair<T, PR>(E, D, B, p, (u32)(it >> 16) & 0xFFFFu, g, epoch, sm, red, stage, stash,
                       &hs);
      continue;
    }
    const u64* pi = E.info + (u64)p * 8;
    const u64 r = pi[PI_R], m = pi[PI_M];
    SmemTable tb{nullptr, 0u, bits};
    if (table_records > 0 && m <= table_records && m <= kTableMax) {
      u32 size = 32;
      while (size < 2 * m) size <<= 1;
      tb.tbl = tbl;
      tb.mask = size - 1;
      u32 c;
      if (ids_ascending<T>(E, p, m)) {
        c = sorted_match<T>(E, p, m, r, tb, reinterpret_cast<u64*>(dyn));
      } else {
        smem_build<T>(E, p, m, tb);
        __syncthreads();
        c = smem_match<T>(E, p, r, tb);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
      if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
      __syncthreads();
      if (threadIdx.x == 0) {
        B.ptot[(u64)p * PT_COUNT + PT_MATCHED] = s_cnt;
        s_cnt = 0;
      }
      if constexpr (PR) {
        if (E.pr.hist && E.pr.samples && !E.pr.pre) {
          for (u64 t = 0; t < ceil_div(r, T); ++t) cells_unit(E.pr, E.ref, E.ref_off, p, t, r, T);
          __syncthreads();
        }
        for (u64 t = 0; t < ceil_div(r, T); ++t) bat_sizes<T, PR>(E, B, p, t, sm);
      }
    } else {
      const u64 ntb = ceil_div(m, (u64)T * kIlp);
      for (u64 t = 0; t < ntb; ++t) bat_build<T>(E, p, t, epoch);
      __syncthreads();
      if constexpr (PR) {
        const u64 nst = ceil_div(r, T);
        if (E.pr.hist && E.pr.samples && !E.pr.pre) {
          for (u64 t = 0; t < nst; ++t) cells_unit(E.pr, E.ref, E.ref_off, p, t, r, T);
          __syncthreads();
        }
        for (u64 t = 0; t < nst; ++t) bat_match<T, PR>(E, B, p, t, epoch, sm);
      } else {
        const u64 ntm = ceil_div(r, (u64)T * kIlp);
        for (u64 t = 0; t < ntm; ++t) bat_match_ilp<T>(E, B, p, t, epoch);
      }
    }
    __syncthreads();
    U64x2 run{0, 0};
    const u64 nst = ceil_div(r, T);
    const SlotPair q = slot_pair(E, B, p);
    {
      u32 g_next = threadIdx.x < r ? __ldcg(E.slot_src + q.ro + threadIdx.x) : kNoMatch;
      for (u64 t = 0; t < nst; ++t) {
        const u32 g = g_next;
        const u64 jn = (t + 1) * T + threadIdx.x;
        g_next = jn < r ? __ldcg(E.slot_src + q.ro + jn) : kNoMatch;
        bat_slot<T, PR>(E, B, p, q, t, g, reinterpret_cast<u64*>(sm) + 33 * (t & 1), stage,
                        stash, run);
      }
      __syncthreads();  // the scan buffers and the stage are reused next
    }
    const U64x2 slot_tot = run;
    run = U64x2{0, 0};
    if (tb.tbl) {
      const u64 matched = slot_tot.b;
      const u32 n_list = smem_new_list<T>(tb, m, list, reinterpret_cast<u32*>(sm));
      const u64 tl = ceil_div(n_list, T);
      for (u64 t = 0; t < tl; ++t)
        bat_new_list<T, PR>(E, p, q, matched, slot_tot, list, n_list, t,
                            reinterpret_cast<u64*>(sm) + 33 * (t & 1), stage, run);
      finish_pair<PR>(E, B, p, r, m, matched, slot_tot, run);
    } else {
      const u64 tn = ceil_div(m, (u64)T * new_per_thread(pi[PI_MODE]));
      for (u64 t = 0; t < (tn ? tn : 1); ++t)
        bat_new<T, PR>(E, B, p, t, epoch, sm, stage, kStageCap, run, slot_tot, tb);
    }
    __syncthreads();
    bat_dec<T, PR>(D, B, p, &hs, reinterpret_cast<u64*>(sm), stage, stash);
    __syncthreads();
  }
}

// Shared memory of one block for tile size T: (bytes, table_records).
inline void persistent_smem(u32 T, bool PR, int ctas_per_sm, u32 want_records, size_t* bytes,
                            u32* records) {
  // per-SM shared memory (228 KB) split over the blocks, minus the static
  // shared memory and the 1 KB the runtime reserves per block
  const size_t per_block = (size_t)228 * 1024 / (size_t)(ctas_per_sm > 0 ? ctas_per_sm : 1);
  size_t cap = per_block > 2048 ? per_block - 2048 : 0;
  if (cap > (size_t)227 * 1024) cap = (size_t)227 * 1024;
  u32 rec = 0;
  for (u32 c = 32; c <= 8192; c <<= 1)
    if (region_bytes(T, c) + c / 8 + 16 <= cap && (want_records == 0 || c <= want_records))
      rec = c;
  *records = rec;
  // + 16 bytes: the decode's 8-byte reads may pass the end of the stage
  *bytes = region_bytes(T, rec) + rec / 8 + 16;
}

// Small pairs (at most kSmallPair slots, records and receiver slots) of the
// plain codec are carried by a launch of their own: one-warp blocks,
// kSmallCtas per SM, so that thousands of them are in flight at once (each
// small pair is a chain of latency-bound steps that a 256-thread block would
// carry with most of its threads idle).
constexpr u64 kSmallPair = 512;
constexpr int kSmallCtas = 32;

template <int T, bool PR>
tera_status launch_persistent(tera_ctx* ctx, const EncArgs& E, const DecArgs& D,
                              const BatchArgs& B, int ctas_per_sm, u32 want_records,
                              cudaStream_t s, bool profiled = true) {
  size_t smem;
  u32 records;
  persistent_smem(T, PR, ctas_per_sm, want_records, &smem, &records);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(codec_persistent_kernel<T, PR>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return TERA_ECUDA;
  const unsigned grid = (unsigned)(ctx->num_sms * (ctas_per_sm > 0 ? ctas_per_sm : 1));
  if (profiled) prof_begin(ctx, s);
  codec_persistent_kernel<T, PR><<<grid, T, smem, s>>>(E, D, B, records);
  if (profiled) return check_launch(ctx, "codec_persistent_kernel", s);
  ctx->launches += 1;
  if (cudaGetLastError() != cudaSuccess) return TERA_ECUDA;
  return TERA_OK;
}

// The plain codec's two launches side by side: the other pairs on the
// caller's stream, the small pairs on the context's side stream (forked after
// the setup, joined before the call returns).  The first launch's blocks fill
// the SMs, so the small pairs' one-warp blocks run as its blocks retire, in
// its tail.  One profile entry covers both.
template <int T>
tera_status launch_plain_pair(tera_ctx* ctx, const EncArgs& E, const DecArgs& D,
                              const BatchArgs& B, int ctas_per_sm, u32 want_records,
                              cudaStream_t s) {
  BatchArgs Bs = B;
  Bs.part = 1;
  prof_begin(ctx, s);
  if (cudaEventRecord(ctx->b_fork, s) != cudaSuccess ||
      cudaStreamWaitEvent(ctx->b_side, ctx->b_fork, 0) != cudaSuccess)
    return TERA_ECUDA;
  tera_status st = launch_persistent<T, false>(ctx, E, D, B, ctas_per_sm, want_records, s, false);
  const tera_status st2 = launch_persistent<32, false>(ctx, E, D, Bs, kSmallCtas, 0, ctx->b_side,
                                                       false);
  if (cudaEventRecord(ctx->b_join, ctx->b_side) != cudaSuccess ||
      cudaStreamWaitEvent(s, ctx->b_join, 0) != cudaSuccess)
    return TERA_ECUDA;
  if (st != TERA_OK) return st;
  if (st2 != TERA_OK) return st2;
  ctx->launches -= 1;  // check_launch counts one of the two again
  return check_launch(ctx, "codec_persistent_kernel", s);
}

}  // namespace

static tera_status batched_impl(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, const tera_predictor* enc_pred,
    const tera_predictor* dec_pred, const tera_ids* ids, void* stream) {
  if (!ctx || !rec_arena || !pair_off || !ref_next || !wire || !wire_off || !wire_len || !recv ||
      !recv_off)
    return TERA_EINVAL;
  if (ids) {
    if (!ids->msg || !ids->ref_next || (ids->ref_prev == nullptr) != (ref_prev == nullptr))
      return TERA_EINVAL;
    if (((uintptr_t)ids->msg | (uintptr_t)ids->ref_next |
         (uintptr_t)(ids->ref_prev ? ids->ref_prev : ids->msg)) & 7u)
      return TERA_EINVAL;
  }
  if ((ref_prev == nullptr) != (ref_off_prev == nullptr)) return TERA_EINVAL;
  if ((recv_prev == nullptr) != (recv_off_prev == nullptr)) return TERA_EINVAL;
  if (mode != TERA_MODE_RAW && mode != TERA_MODE_XOR) return TERA_EINVAL;
  if (((uintptr_t)rec_arena | (uintptr_t)ref_next | (uintptr_t)wire | (uintptr_t)recv |
       (uintptr_t)(ref_prev ? ref_prev : wire) | (uintptr_t)(recv_prev ? recv_prev : wire)) & 15u)
    return TERA_EINVAL;
  tera_tune tn = tune ? *tune : tera_tune{256, 4, 0, 0, 0, 0};
  if (enc_pred && enc_pred->params && ((uintptr_t)enc_pred->params & 3u)) return TERA_EINVAL;
  if (tn.block != 128 && tn.block != 256 && tn.block != 512 && tn.block != 1024) return TERA_EINVAL;
  if (tn.ctas_per_sm < 1 || tn.ctas_per_sm > 16 || tn.block * tn.ctas_per_sm > 2048)
    return TERA_EINVAL;
  if (tn.table_records < 0 || (tn.table_records > 0 && (tn.table_records < 32 ||
                                                        (tn.table_records & (tn.table_records - 1)))))
    return TERA_EINVAL;
  if (tn.team_blocks != 0 && (tn.team_blocks < 2 || tn.team_blocks > 1024)) return TERA_EINVAL;
  if (tn.wait_limit_us < 0 || tn.wait_limit_us > 60000000) return TERA_EINVAL;
  if (tn.reserved != 0) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u64 P = ctx->n_pairs;
  const bool PR = enc_pred != nullptr || dec_pred != nullptr;
  if (PR && tn.block > 256) tn.block = 256;  // stash, stage and weights stay within 70 KB
  const u32 T = (u32)tn.block;
  tera_status st = ensure_records(ctx, ctx->cap_records, s);
  if (st != TERA_OK) return st;
  if ((st = ensure_batched(ctx)) != TERA_OK) return st;
  if (!ctx->pair_info) return TERA_EINVAL;  // allocated with the context

  EncArgs E;
  E.rec = rec_arena;
  E.pair_off = reinterpret_cast<const u64*>(pair_off);
  E.ref = ref_prev;
  E.ref_off = reinterpret_cast<const u64*>(ref_off_prev);
  E.ref_next = ref_next;
  E.wire = wire;
  E.wire_off = reinterpret_cast<const u64*>(wire_off);
  E.wire_len = reinterpret_cast<u64*>(wire_len);
  E.unit_off = nullptr;
  E.units_total = nullptr;
  E.unit_pair = nullptr;
  E.unit_sum = nullptr;
  E.unit_base = nullptr;
  E.info = ctx->pair_info;
  E.slot_src = ctx->slot_src;
  E.matched = ctx->matched;
  E.reset = ctx->d_reset;
  E.seg = ctx->seg;
  E.epoch = ctx->d_epoch;
  E.p0 = 0;
  E.p1 = (u32)P;
  E.class_id = ctx->class_id;
  E.st = ctx->d_status;
  E.stats = ctx->d_stats;
  if (ids) {
    E.msg_ids = reinterpret_cast<const u64*>(ids->msg);
    E.ref_ids = reinterpret_cast<const u64*>(ids->ref_prev);
    E.ref_ids_next = reinterpret_cast<u64*>(ids->ref_next);
  }

  DecArgs D;
  D.wire = wire;
  D.wire_off = reinterpret_cast<const u64*>(wire_off);
  D.ref = recv_prev;
  D.ref_off = reinterpret_cast<const u64*>(recv_off_prev);
  D.recv = recv;
  D.recv_off = reinterpret_cast<u64*>(recv_off);
  D.unit_off = nullptr;
  D.units_total = nullptr;
  D.unit_pair = nullptr;
  D.unit_sum = nullptr;
  D.unit_base = nullptr;
  D.info = ctx->pair_info + 8 * P;
  D.p0 = 0;
  D.p1 = (u32)P;
  D.class_id = ctx->class_id;
  D.st = ctx->d_status;

  BatchArgs B;
  B.n_pairs = P;
  B.ticket = ctx->b_scalars + 1;
  B.ptot = ctx->b_ptot;
  B.abort = reinterpret_cast<u32*>(ctx->b_scalars + 2);
  B.items = ctx->b_items;
  B.n_items = ctx->b_scalars + 0;
  B.team = ctx->b_team;
  B.tsum = ctx->b_tsum;
  B.tbase = ctx->b_tbase;
  B.wait_ns = 1000ull * (u64)(tn.wait_limit_us ? tn.wait_limit_us : 1000000);
  B.n_first = ctx->b_scalars + 3;
  B.ticket_small = ctx->b_scalars + 4;
  B.part = 0;

  if (PR) {
    if ((st = ensure_pred(ctx)) != TERA_OK) return st;
    if (enc_pred) {
      if ((enc_pred->hist_prev != nullptr) != (ref_prev != nullptr)) return TERA_EINVAL;
      fill_pred(ctx, &E.pr, enc_pred, ctx->cseg_enc);
      E.pr.samples = enc_pred->samples;
      E.pr.allow_residual = enc_pred->allow_residual;
      if (E.pr.hist && (st = cells_clear(ctx, ctx->cseg_enc, E.ref_off, s)) != TERA_OK) return st;
    }
    if (dec_pred) {
      if ((dec_pred->hist_prev != nullptr) != (recv_prev != nullptr)) return TERA_EINVAL;
      fill_pred(ctx, &D.pr, dec_pred, ctx->cseg_dec);
      if (D.pr.hist && D.pr.params &&
          (st = cells_clear(ctx, ctx->cseg_dec, D.ref_off, s)) != TERA_OK)
        return st;
    }
    // each side's predictions of its own reference, before the codec
    if (enc_pred && E.pr.hist && E.pr.params) {
      if ((st = pred_prepass(ctx, E.pr, ref_prev, E.ref_off, ctx->pscr, s)) != TERA_OK) return st;
      E.pr.pre = 1;
    }
    if (dec_pred && D.pr.hist && D.pr.params) {
      D.pr.pscr = ctx->pscr_dec;
      if ((st = pred_prepass(ctx, D.pr, recv_prev, D.ref_off, ctx->pscr_dec, s)) != TERA_OK)
        return st;
      D.pr.pre = 1;
    }
  }
  cudaMemsetAsync(ctx->b_ptot, 0, sizeof(u64) * P * PT_COUNT, s);
  cudaMemsetAsync(ctx->b_team, 0, sizeof(u32) * P * 8, s);
  const int c = tn.ctas_per_sm;
  const u32 want = (u32)tn.table_records;
  size_t smem_bytes;
  u32 table_records;
  persistent_smem(T, PR, c, want, &smem_bytes, &table_records);
  const u32 blocks = (u32)(ctx->num_sms * c);
  // teams of at most 64 blocks (never more than the blocks resident at once)
  const u32 gmax = blocks / 2 < 64 ? (blocks / 2 > 1 ? blocks / 2 : 1) : 64;
  // pairs smaller than this stay on one block (and in shared memory if they fit)
  const u64 min_team = (u64)16 * T > 2 * (u64)table_records ? (u64)16 * T : 2 * (u64)table_records;
  const u64 small_max = PR ? 0 : kSmallPair;
  const unsigned setup_blocks = (unsigned)(P == 0 ? 1 : (P + kSetupThreads - 1) / kSetupThreads);
  U64x2* part = reinterpret_cast<U64x2*>(ctx->b_part);
  prof_begin(ctx, s);
  bat_setup_sums_kernel<<<setup_blocks, kSetupThreads, 0, s>>>(
      E, D, P, mode, T, blocks, gmax, (u32)tn.team_blocks, min_team, PR ? 1 : 0, small_max, part);
  if ((st = check_launch(ctx, "bat_setup_sums_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  bat_setup_place_kernel<<<setup_blocks, kSetupThreads, 0, s>>>(
      E, D, B, P, mode, reinterpret_cast<u64*>(wire_off), wire_capacity, ctx->cap_records,
      recv_capacity_units, ctx->d_epoch, T, blocks, gmax, (u32)tn.team_blocks, min_team,
      PR ? 1 : 0, ctx->b_items, ctx->b_items_cap, ctx->b_tbase, ctx->b_tsum_cap,
      ctx->b_scalars + 0, small_max, part);
  if ((st = check_launch(ctx, "bat_setup_place_kernel", s)) != TERA_OK) return st;
  if (PR) {
    if (T == 128) return launch_persistent<128, true>(ctx, E, D, B, c, want, s);
    return launch_persistent<256, true>(ctx, E, D, B, c, want, s);
  }
  switch (T) {
    case 128: return launch_plain_pair<128>(ctx, E, D, B, c, want, s);
    case 256: return launch_plain_pair<256>(ctx, E, D, B, c, want, s);
    case 512: return launch_plain_pair<512>(ctx, E, D, B, c, want, s);
    default: return launch_plain_pair<1024>(ctx, E, D, B, c, want, s);
  }
}

extern "C" tera_status tera_codec_batched(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, void* stream) {
  TERA_CALL_RANGE("tera_codec_batched");
  return batched_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                      wire_capacity, wire_off, wire_len, recv_prev, recv_off_prev, recv,
                      recv_capacity_units, recv_off, mode, tune, nullptr, nullptr, nullptr,
                      stream);
}

extern "C" tera_status tera_codec_batched_ids(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, const tera_ids* ids, void* stream) {
  TERA_CALL_RANGE("tera_codec_batched_ids");
  if (!ids) return TERA_EINVAL;
  return batched_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                      wire_capacity, wire_off, wire_len, recv_prev, recv_off_prev, recv,
                      recv_capacity_units, recv_off, mode, tune, nullptr, nullptr, ids, stream);
}

extern "C" tera_status tera_codec_batched_pred(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, const tera_predictor* enc_pred,
    const tera_predictor* dec_pred, void* stream) {
  TERA_CALL_RANGE("tera_codec_batched_pred");
  return batched_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                      wire_capacity, wire_off, wire_len, recv_prev, recv_off_prev, recv,
                      recv_capacity_units, recv_off, mode, tune, enc_pred, dec_pred, nullptr,
                      stream);
}
