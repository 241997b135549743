// Agent migration (paper Sec. 2.1 "Agent Migration"): an agent whose new
// position lies in another box moves to that box.  It travels as a raw
// TeraAgent IO record (Sec. 2.2.1); the difference encoding of Sec. 2.3 is for
// the aura only.
//
// State layout: box-major, box s holds agents [box_off[s], box_off[s+1]).
// Inbox q = d*27 + b of receiver box d collects the leavers that arrive from
// side b (the neighbour bit of the offset from d to their previous box; 13
// when that box is not a neighbour, the paper's second case, whose lookup is
// the same classification here), in ascending agent index.  The inboxes form
// one TAIO arena: inbox q at units [off[q] + q, off[q+1] + q + 1), a header
// and its records.  The next state of box d is its stayers in their previous
// order, then its inboxes in ascending side.
//
// tera_migrate_send
//   mig_count_kernel   one pass over x, y, z: owner box of every agent; leavers
//                      per warp tile, per source box and per inbox
//   scan of the warp-tile counts (leavers before every warp tile)
//   mig_scan_kernel    one block: checks box_off_prev; inbox offsets, next box
//                      offsets, leavers of the boxes before each box, capacity
//   mig_move_kernel    one pass over the 8 columns: every stayer to its place in
//                      the next state, every leaver listed with its inbox
//   stable radix sort of the leaver list by inbox (agent order kept): each
//                      leaver's position in inbox order
//   mig_pack_kernel    inbox headers, then every leaver's record, read in
//                      agent order (serialization)
// tera_migrate_recv
//   mig_unpack_kernel  every inbox record into the next state after the
//                      receiver's stayers (deserialization), headers checked
#include "classify.cuh"
#include "tera_internal.cuh"

using namespace tera;

namespace {

struct Cols {
  const u64* c[8];  // id, x, y, z, diameter, volume, adherence, density
};
struct ColsOut {
  u64* c[8];
};

// Largest s in [lo, hi] with off[s] <= a; lo when there is none.  Any result
// lies in [lo, hi], whatever the array holds.
__device__ __forceinline__ u32 box_search(const u64* __restrict__ off, u32 lo, u32 hi, u64 a) {
  while (lo < hi) {
    const u32 mid = lo + ((hi - lo + 1) >> 1);
    if (off[mid] <= a) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Side of box d that an agent from box s arrives from: the neighbour bit of
// the offset s - d (per axis -1, 0 or +1; modulo n on a toroidal axis), 13
// when s is not one of d's neighbours.
__device__ __forceinline__ u32 inbox_side(u32 s, u32 d, const SmemGrid& g) {
  const u32 n0 = (u32)g.n[0], n1 = (u32)g.n[1];
  const int cs[3] = {(int)(s % n0), (int)((s / n0) % n1), (int)(s / (n0 * n1))};
  const int cd[3] = {(int)(d % n0), (int)((d / n0) % n1), (int)(d / (n0 * n1))};
  u32 bit = 0, mult = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int o = cs[a] - cd[a];
    if ((g.periodic >> a) & 1) {
      const int n = g.n[a];
      if (o == n - 1) o = -1;
      else if (o == -(n - 1)) o = 1;
    }
    if (o < -1 || o > 1) return 13u;
    bit += (u32)(o + 1) * mult;
    mult *= 3u;
  }
  return bit;
}

// Keys of the edges of one box on the three axes: a position is in the box
// when key_lo[a] <= key(v[a]) < key_hi[a] on every axis.
struct BoxBounds {
  u64 lo[3], hi[3];
};

__device__ __forceinline__ void box_bounds(u32 s, const SmemGrid& g, BoxBounds* b) {
  const u32 n0 = (u32)g.n[0], n1 = (u32)g.n[1];
  const u32 c[3] = {s % n0, (s / n0) % n1, s / (n0 * n1)};
  const BoxKeys* rows = grid_rows();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const BoxKeys& r = rows[g.koff[a] + (int)c[a]];
    b->lo[a] = r.e0;
    b->hi[a] = r.e1;
  }
}

__device__ __forceinline__ bool inside_box(u64 bx, u64 by, u64 bz, const BoxBounds& b) {
  const u64 kx = key_of(bx), ky = key_of(by), kz = key_of(bz);
  return kx >= b.lo[0] && kx < b.hi[0] && ky >= b.lo[1] && ky < b.hi[1] && kz >= b.lo[2] &&
         kz < b.hi[2];
}

// Owner box of an agent of box s: s itself when the position is still inside
// it (the common case, six key comparisons with the warp's cached bounds of
// box s_lo), else the full classification (-1 outside the domain).
__device__ __forceinline__ int new_owner(u64 bx, u64 by, u64 bz, u32 s, u32 s_lo,
                                         const BoxBounds& lo_bounds, const SmemGrid& g) {
  if (s == s_lo) {
    if (inside_box(bx, by, bz, lo_bounds)) return (int)s;
  } else {
    BoxBounds b;
    box_bounds(s, g, &b);
    if (inside_box(bx, by, bz, b)) return (int)s;
  }
  return locate_agent(bx, by, bz, g);
}

// atomicAdd(&ctr[key], 1) for every lane with `on`, one atomic per distinct
// key of the warp (all lanes of the warp take part).
__device__ __forceinline__ void warp_count(u64* ctr, u32 key, bool on) {
  const u32 k = on ? key : 0xFFFFFFFFu;
  const u32 peers = __match_any_sync(0xFFFFFFFFu, k);
  const u32 lane = threadIdx.x & 31;
  if (on && (__ffs(peers) - 1) == (int)lane) atomicAdd(&ctr[key], (u64)__popc(peers));
}

// Largest s in [lo, hi] with off[s] <= a, found by the whole warp: each step
// probes 32 evenly spaced boxes at once (two steps for 513 offsets); lo when
// there is none.  Every lane returns the same result, in [lo, hi].
__device__ __forceinline__ u32 warp_box_search(const u64* __restrict__ off, u32 lo, u32 hi, u64 a) {
  const u32 lane = threadIdx.x & 31;
  while (lo < hi) {
    const u32 step = (hi - lo + 32) / 32;  // ceil((hi - lo + 1) / 32)
    const u32 idx = lo + lane * step;
    const bool ok = idx <= hi && off[idx] <= a;
    const u32 bal = __ballot_sync(0xFFFFFFFFu, ok);
    if (bal == 0u) break;  // off[lo] > a
    const u32 last = 31u - (u32)__clz(bal);
    const u32 nlo = lo + last * step;
    const u32 nhi = nlo + step - 1u;
    lo = nlo;
    hi = nhi < hi ? nhi : hi;
    if (step == 1u) break;
  }
  return lo;
}

// Box range of the agents [w0, w_end) of one warp tile.
__device__ __forceinline__ void warp_boxes(const u64* __restrict__ box_off, u32 n_boxes, u64 w0,
                                           u64 w_end, u32* lo, u32* hi) {
  *lo = warp_box_search(box_off, 0, n_boxes - 1, w0);
  *hi = warp_box_search(box_off, *lo, n_boxes - 1, w_end - 1);
}

// Leavers are counted per warp tile (kWarpAgents agents), so their order
// (agent order) needs no block-wide step.

__global__ void __launch_bounds__(kClassifyThreads, 5)
    mig_count_kernel(const u64* __restrict__ x, const u64* __restrict__ y,
                     const u64* __restrict__ z, u64 n, const u64* __restrict__ box_off,
                     u32 n_boxes, const GridTables* __restrict__ g, u32* __restrict__ tile_cnt,
                     u64 n_wtiles, u64* __restrict__ from, u64* __restrict__ cnt, DevStatus* st) {
  __shared__ SmemGrid sg;
  load_grid(sg, g);
  const int lane = threadIdx.x & 31;
  const u64 w = (u64)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const u64 w0 = w * kWarpAgents;
  if (w0 >= n) {
    if (lane == 0 && w < n_wtiles) tile_cnt[w] = 0;
    return;
  }
  const u64 w_end = w0 + kWarpAgents < n ? w0 + kWarpAgents : n;
  u32 s_lo, s_hi;
  warp_boxes(box_off, n_boxes, w0, w_end, &s_lo, &s_hi);
  __shared__ BoxBounds wbounds[kWarpsPerBlock];
  BoxBounds& lo_bounds = wbounds[threadIdx.x >> 5];
  if (lane == 0) box_bounds(s_lo, sg, &lo_bounds);
  __syncwarp();
  u32 leavers = 0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kWarpRounds; ++k) {
    const u64 a0 = w0 + (u64)k * 64 + 2u * lane;
    u64 vx[2], vy[2], vz[2];
    if (a0 + 1 < n) {
      const ulonglong2 tx = *reinterpret_cast<const ulonglong2*>(x + a0);
      const ulonglong2 ty = *reinterpret_cast<const ulonglong2*>(y + a0);
      const ulonglong2 tz = *reinterpret_cast<const ulonglong2*>(z + a0);
      vx[0] = tx.x; vx[1] = tx.y; vy[0] = ty.x; vy[1] = ty.y; vz[0] = tz.x; vz[1] = tz.y;
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const bool in = a0 + q < n;
        vx[q] = in ? x[a0 + q] : 0ull;
        vy[q] = in ? y[a0 + q] : 0ull;
        vz[q] = in ? z[a0 + q] : 0ull;
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const u64 a = a0 + q;
      bool leave = false;
      u32 s = 0, key = 0;
      if (a < n) {
        s = box_search(box_off, s_lo, s_hi, a);
        const int d = new_owner(vx[q], vy[q], vz[q], s, s_lo, lo_bounds, sg);
        if (d < 0) {
          bad = true;  // stays in its box; TERA_EDOMAIN
        } else if ((u32)d != s) {
          leave = true;
          key = (u32)d * 27u + inbox_side(s, (u32)d, sg);
        }
      }
      if (__any_sync(0xFFFFFFFFu, leave)) {
        leavers += leave;
        warp_count(from, s, leave);
        warp_count(cnt, key, leave);
      }
    }
  }
  if (bad) latch(st, TERA_EDOMAIN);
  leavers = warp_sum(leavers);
  if (lane == 0) tile_cnt[w] = leavers;
}

// One block: checks box_off_prev (0 first, n last, non-decreasing), then
// inbox_off = exclusive scan of the inbox counts, before = exclusive scan of
// the leavers per source box, and box_off_next from the next box sizes
// (previous size - leavers + immigrants).
__global__ void __launch_bounds__(1024)
    mig_scan_kernel(const u64* __restrict__ box_off_prev, u64 n, u32 n_boxes,
                    const u64* __restrict__ from, const u64* __restrict__ cnt, u64 arena_units,
                    u64 lv_cap, u64* __restrict__ inbox_off, u64* __restrict__ box_off_next,
                    u64* __restrict__ before, DevStatus* st) {
  __shared__ u64 sm[33];
  __shared__ u32 bad;
  const u64 Q = (u64)n_boxes * 27u;
  if (threadIdx.x == 0) bad = (box_off_prev[0] != 0 || box_off_prev[n_boxes] != n) ? 1u : 0u;
  __syncthreads();
  for (u64 b = threadIdx.x; b < n_boxes; b += blockDim.x)
    if (box_off_prev[b + 1] < box_off_prev[b]) bad = 1u;
  u64 carry = 0;
  for (u64 base = 0; base < Q; base += blockDim.x) {
    const u64 i = base + threadIdx.x;
    u64 tot;
    const u64 ex = block_excl_scan<u64>(i < Q ? cnt[i] : 0ull, sm, &tot);
    if (i < Q) inbox_off[i] = carry + ex;
    carry += tot;
  }
  const u64 leavers = carry;
  if (threadIdx.x == 0) inbox_off[Q] = leavers;
  carry = 0;
  for (u64 base = 0; base < n_boxes; base += blockDim.x) {
    const u64 i = base + threadIdx.x;
    u64 tot;
    const u64 ex = block_excl_scan<u64>(i < n_boxes ? from[i] : 0ull, sm, &tot);
    if (i < n_boxes) before[i] = carry + ex;
    carry += tot;
  }
  __syncthreads();  // inbox_off complete
  carry = 0;
  for (u64 base = 0; base < n_boxes; base += blockDim.x) {
    const u64 i = base + threadIdx.x;
    u64 v = 0;
    if (i < n_boxes)
      v = (box_off_prev[i + 1] - box_off_prev[i]) - from[i] +
          (inbox_off[27 * i + 27] - inbox_off[27 * i]);
    u64 tot;
    const u64 ex = block_excl_scan<u64>(v, sm, &tot);
    if (i < n_boxes) box_off_next[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    box_off_next[n_boxes] = carry;
    if (bad) {
      latch(st, TERA_EINVAL);
      atomicExch(&st->abort, 1u);
    } else if (leavers + Q > arena_units || leavers > lv_cap) {
      latch(st, TERA_ECAPACITY);
      need(st, leavers + Q);
      atomicExch(&st->abort, 1u);
    }
  }
}

__device__ __forceinline__ bool aborted(const DevStatus* st) {
  return *reinterpret_cast<const volatile u32*>(&st->abort) != 0u;
}

// Stayer a of box s goes to box_off_next[s] + (a - box_off_prev[s]) minus the
// leavers of box s before it; leaver k (in agent order) is listed with its
// inbox.  Same warp tiles as mig_count_kernel; a leaver's rank is the count
// before its warp tile plus two ballots per round.
__global__ void __launch_bounds__(kClassifyThreads, 4)
    mig_move_kernel(Cols prev, u64 n, const u64* __restrict__ box_off_prev, u32 n_boxes,
                    const GridTables* __restrict__ g, const u64* __restrict__ tile_base,
                    const u64* __restrict__ box_off_next, const u64* __restrict__ before,
                    ColsOut next, u32* __restrict__ lv_key, u32* __restrict__ lv_agent, u64 lv_cap,
                    const DevStatus* st) {
  __shared__ SmemGrid sg;
  if (aborted(st)) return;
  load_grid(sg, g);
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  const u64 w = (u64)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const u64 w0 = w * kWarpAgents;
  if (w0 >= n) return;
  const u64 w_end = w0 + kWarpAgents < n ? w0 + kWarpAgents : n;
  u32 s_lo, s_hi;
  warp_boxes(box_off_prev, n_boxes, w0, w_end, &s_lo, &s_hi);
  __shared__ BoxBounds wbounds[kWarpsPerBlock];
  BoxBounds& lo_bounds = wbounds[threadIdx.x >> 5];
  if (lane == 0) box_bounds(s_lo, sg, &lo_bounds);
  __syncwarp();
  u64 run = tile_base[w];
  for (int k = 0; k < kWarpRounds; ++k) {
    const u64 a0 = w0 + (u64)k * 64 + 2u * lane;
    if (w0 + (u64)k * 64 >= n) break;  // warp-uniform
    u64 v[8][2];
    if (a0 + 1 < n) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(prev.c[c] + a0);
        v[c][0] = t.x;
        v[c][1] = t.y;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        v[c][0] = a0 < n ? prev.c[c][a0] : 0ull;
        v[c][1] = 0ull;
      }
    }
    bool leave[2] = {false, false};
    u32 key[2] = {0u, 0u}, box[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const u64 a = a0 + q;
      if (a >= n) continue;
      box[q] = box_search(box_off_prev, s_lo, s_hi, a);
      const int d = new_owner(v[1][q], v[2][q], v[3][q], box[q], s_lo, lo_bounds, sg);
      if (d >= 0 && (u32)d != box[q]) {
        leave[q] = true;
        key[q] = (u32)d * 27u + inbox_side(box[q], (u32)d, sg);
      }
    }
    const u32 b0 = __ballot_sync(0xFFFFFFFFu, leave[0]);
    const u32 b1 = __ballot_sync(0xFFFFFFFFu, leave[1]);
    const u64 k0 = run + __popc(b0 & lt) + __popc(b1 & lt);  // leavers before agent a0
    u64 dst[2] = {0ull, 0ull};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const u64 a = a0 + q;
      const u64 kq = k0 + (q == 1 && leave[0] ? 1u : 0u);
      if (a < n && !leave[q])
        dst[q] = box_off_next[box[q]] + (a - box_off_prev[box[q]]) - (kq - before[box[q]]);
    }
    const bool pair = a0 + 1 < n && !leave[0] && !leave[1] && box[0] == box[1] && !(dst[0] & 1ull);
    if (pair) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<ulonglong2*>(next.c[c] + dst[0]) = make_ulonglong2(v[c][0], v[c][1]);
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const u64 a = a0 + q;
        if (a >= n) continue;
        const u64 kq = k0 + (q == 1 && leave[0] ? 1u : 0u);
        if (leave[q]) {
          if (kq < lv_cap) {
            lv_key[kq] = key[q];
            lv_agent[kq] = (u32)a;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) next.c[c][dst[q]] = v[c][q];
        }
      }
    }
    run += __popc(b0) + __popc(b1);
  }
}

// Serialization: thread t < Q writes the header of inbox t; the 4 threads of
// leaver k (agent order, so the reads of each column are ascending) write the
// 16-byte quarters of its record, words 2c and 2c+1, at unit dest[k] + q + 1
// (dest[k] = its position in inbox order, from the sort).
__global__ void __launch_bounds__(256)
    mig_pack_kernel(Cols prev, const u64* __restrict__ inbox_off, u64 Q,
                    const u32* __restrict__ lv_key, const u32* __restrict__ lv_agent,
                    const u32* __restrict__ lv_dest, u32 class_id, uint8_t* __restrict__ arena,
                    const DevStatus* st) {
  if (aborted(st)) return;
  const u64 L = inbox_off[Q];
  const u64 total = Q + 4 * L;
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (u64)gridDim.x * blockDim.x) {
    if (t < Q) {
      const u64 off = inbox_off[t];
      ulonglong2* h = reinterpret_cast<ulonglong2*>(arena + (off + t) * kRecBytes);
      const u64 w0 = (u64)kTaioMagic | ((u64)kVersion << 32) | ((u64)kRecBytes << 48);
      const u64 w1 = (u64)class_id | (t << 32);
      h[0] = make_ulonglong2(w0, w1);
      h[1] = make_ulonglong2(inbox_off[t + 1] - off, 0ull);
      h[2] = make_ulonglong2(0ull, 0ull);
      h[3] = make_ulonglong2(0ull, 0ull);
    } else {
      const u64 r = t - Q;
      const u64 k = r >> 2;
      const u32 c = (u32)(r & 3u);
      const u32 a = lv_agent[k];
      const u64 unit = (u64)lv_dest[k] + lv_key[k] + 1;
      ulonglong2* dst = reinterpret_cast<ulonglong2*>(arena + unit * kRecBytes) + c;
      u64 w0v, w1v;
      switch (c) {  // constant column indexes keep the pointers in registers
        case 0: w0v = prev.c[0][a]; w1v = prev.c[1][a]; break;
        case 1: w0v = prev.c[2][a]; w1v = prev.c[3][a]; break;
        case 2: w0v = prev.c[4][a]; w1v = prev.c[5][a]; break;
        default: w0v = prev.c[6][a]; w1v = prev.c[7][a]; break;
      }
      *dst = make_ulonglong2(w0v, w1v);
    }
  }
}

// Deserialization: thread t < Q checks the header of inbox t; the 4 threads of
// record j find its inbox q by a binary search of inbox_off, and write words
// 2c and 2c+1 into the next state of box d = q / 27, after its stayers.
// Every index is checked against the arena and the state before use.
__global__ void __launch_bounds__(256)
    mig_unpack_kernel(const uint8_t* __restrict__ arena, u64 arena_units,
                      const u64* __restrict__ inbox_off, u64 Q, const u64* __restrict__ box_off_next,
                      u32 class_id, ColsOut next, u64 n_next, DevStatus* st) {
  if (aborted(st)) return;
  const u64 L = inbox_off[Q];
  if (L > arena_units || L + Q > arena_units) {  // more records than the arena holds
    if (blockIdx.x == 0 && threadIdx.x == 0) latch(st, TERA_ECORRUPT);
    return;
  }
  const u64 total = Q + 4 * L;
  bool bad = false;
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (u64)gridDim.x * blockDim.x) {
    if (t < Q) {
      const u64 off = inbox_off[t];
      if (off + t >= arena_units || inbox_off[t + 1] < off) {
        bad = true;
        continue;
      }
      const u64* h = reinterpret_cast<const u64*>(arena + (off + t) * kRecBytes);
      const u64 w0 = h[0], w1 = h[1], m = h[2];
      bad |= !((u32)w0 == kTaioMagic && (u32)((w0 >> 32) & 0xFFFFu) == kVersion &&
               (u32)(w0 >> 48) == kRecBytes && (u32)w1 == class_id && (w1 >> 32) == t &&
               m == inbox_off[t + 1] - off);
    } else {
      const u64 r = t - Q;
      const u64 j = r >> 2;
      const u32 c = (u32)(r & 3u);
      // largest q with inbox_off[q] <= j
      u64 lo = 0, hi = Q - 1;
      while (lo < hi) {
        const u64 mid = lo + ((hi - lo + 1) >> 1);
        if (inbox_off[mid] <= j) lo = mid;
        else hi = mid - 1;
      }
      const u64 q = lo, d = q / 27u;
      const u64 first = inbox_off[27 * d], imm = inbox_off[27 * d + 27] - first;
      const u64 size = box_off_next[d + 1] - box_off_next[d];
      const u64 unit = j + q + 1;
      if (imm > size || j < first || unit >= arena_units) {
        bad = true;
        continue;
      }
      const u64 dst = box_off_next[d] + (size - imm) + (j - first);
      if (dst >= n_next) {
        bad = true;
        continue;
      }
      const ulonglong2 w = *(reinterpret_cast<const ulonglong2*>(arena + unit * kRecBytes) + c);
      u64 *p0, *p1;
      switch (c) {  // constant column indexes keep the pointers in registers
        case 0: p0 = next.c[0]; p1 = next.c[1]; break;
        case 1: p0 = next.c[2]; p1 = next.c[3]; break;
        case 2: p0 = next.c[4]; p1 = next.c[5]; break;
        default: p0 = next.c[6]; p1 = next.c[7]; break;
      }
      p0[dst] = w.x;
      p1[dst] = w.y;
    }
  }
  if (bad) latch(st, TERA_ECORRUPT);
}

bool soa_cols(const tera_soa* s, Cols* c) {
  const void* p[8] = {s->id, s->x, s->y, s->z, s->diameter, s->volume, s->adherence, s->density};
  for (int k = 0; k < 8; ++k) {
    if (s->n > 0 && (!p[k] || ((uintptr_t)p[k] & 15u))) return false;
    c->c[k] = reinterpret_cast<const u64*>(p[k]);
  }
  return true;
}

bool soa_cols_out(const tera_soa_mut* s, ColsOut* c) {
  void* p[8] = {s->id, s->x, s->y, s->z, s->diameter, s->volume, s->adherence, s->density};
  for (int k = 0; k < 8; ++k) {
    if (s->n > 0 && (!p[k] || ((uintptr_t)p[k] & 15u))) return false;
    c->c[k] = reinterpret_cast<u64*>(p[k]);
  }
  return true;
}

}  // namespace

extern "C" tera_status tera_migrate_send(tera_ctx* ctx, const tera_soa* prev,
                                         const uint64_t* box_off_prev, uint8_t* arena,
                                         uint64_t arena_units, uint64_t* inbox_off,
                                         const tera_soa_mut* next, uint64_t* box_off_next,
                                         void* stream) {
  TERA_CALL_RANGE("tera_migrate_send");
  if (!ctx || !prev || !next || !box_off_prev || !inbox_off || !box_off_next) return TERA_EINVAL;
  if (prev->n < 0 || prev->n > (int64_t)0xFFFFFFFFll || next->n != prev->n) return TERA_EINVAL;
  if (arena_units > 0 && (!arena || ((uintptr_t)arena & 15u))) return TERA_EINVAL;
  Cols cp;
  ColsOut cn;
  if (!soa_cols(prev, &cp) || !soa_cols_out(next, &cn)) return TERA_EINVAL;
  for (int k = 0; k < 8; ++k)
    if (prev->n > 0 && (const void*)cp.c[k] == (const void*)cn.c[k]) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u64 n = (u64)prev->n;
  const u64* off_prev = reinterpret_cast<const u64*>(box_off_prev);
  u64* off_next = reinterpret_cast<u64*>(box_off_next);
  u64* inbox = reinterpret_cast<u64*>(inbox_off);
  const u64 B = ctx->n_boxes, Q = ctx->n_pairs;
  const u64 lv_cap = arena_units > Q ? (arena_units - Q < n ? arena_units - Q : n) : 0;
  tera_status st;
  if ((st = ensure_migrate(ctx, n, lv_cap)) != TERA_OK) return st;
  cudaMemsetAsync(&ctx->d_status->abort, 0, sizeof(u32), s);
  cudaMemsetAsync(ctx->m_from, 0, sizeof(u64) * B, s);
  cudaMemsetAsync(ctx->m_cnt, 0, sizeof(u64) * Q, s);
  const u64 blocks = n == 0 ? 1 : (n + kBlockAgents - 1) / kBlockAgents;
  const u64 wtiles = n == 0 ? 1 : (n + kWarpAgents - 1) / kWarpAgents;
  prof_begin(ctx, s);
  mig_count_kernel<<<(unsigned)blocks, kClassifyThreads, grid_smem_bytes(ctx->grid), s>>>(
      cp.c[1], cp.c[2], cp.c[3], n, off_prev, (u32)B, ctx->d_grid, ctx->m_tile_cnt, wtiles,
      ctx->m_from, ctx->m_cnt, ctx->d_status);
  if ((st = check_launch(ctx, "mig_count_kernel", s)) != TERA_OK) return st;
  if ((st = scan_u32(ctx, ctx->m_tile_cnt, ctx->m_tile_base, nullptr, wtiles, s)) != TERA_OK)
    return st;
  prof_begin(ctx, s);
  mig_scan_kernel<<<1, 1024, 0, s>>>(off_prev, n, (u32)B, ctx->m_from, ctx->m_cnt, arena_units,
                                     lv_cap, inbox, off_next, ctx->m_before, ctx->d_status);
  if ((st = check_launch(ctx, "mig_scan_kernel", s)) != TERA_OK) return st;
  if (n > 0) {
    prof_begin(ctx, s);
    mig_move_kernel<<<(unsigned)blocks, kClassifyThreads, grid_smem_bytes(ctx->grid), s>>>(
        cp, n, off_prev, (u32)B, ctx->d_grid, ctx->m_tile_base, off_next, ctx->m_before, cn,
        ctx->m_key, ctx->m_agent, lv_cap, ctx->d_status);
    if ((st = check_launch(ctx, "mig_move_kernel", s)) != TERA_OK) return st;
  }
  // the leaver count is read on the device from inbox[Q]; more than
  // lv_cap leavers (capacity error, latched above) sorts nothing
  const SortBufs bufs{ctx->m_keys_b,   ctx->m_keys_c,   ctx->m_vals_b, ctx->m_vals_c,
                      ctx->m_agents_b, ctx->m_agents_c, ctx->m_hist};
  const u32* sorted = ctx->m_key;
  if ((st = radix_sort_entries(ctx, bufs, ctx->m_key, ctx->m_agent, ctx->m_dest, ctx->m_sorted,
                               inbox + Q, lv_cap, Q, &sorted, s)) != TERA_OK)
    return st;
  prof_begin(ctx, s);
  mig_pack_kernel<<<(unsigned)grid_for(ctx, 4), 256, 0, s>>>(cp, inbox, Q, ctx->m_key,
                                                             ctx->m_agent, ctx->m_dest,
                                                             ctx->class_id, arena, ctx->d_status);
  return check_launch(ctx, "mig_pack_kernel", s);
}

extern "C" tera_status tera_migrate_recv(tera_ctx* ctx, const uint8_t* arena, uint64_t arena_units,
                                         const uint64_t* inbox_off, const uint64_t* box_off_next,
                                         const tera_soa_mut* next, void* stream) {
  TERA_CALL_RANGE("tera_migrate_recv");
  if (!ctx || !next || !inbox_off || !box_off_next) return TERA_EINVAL;
  if (!arena || ((uintptr_t)arena & 15u)) return TERA_EINVAL;
  if (next->n < 0 || next->n > (int64_t)0xFFFFFFFFll) return TERA_EINVAL;
  ColsOut cn;
  if (!soa_cols_out(next, &cn)) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(ctx, s);
  mig_unpack_kernel<<<(unsigned)grid_for(ctx, 4), 256, 0, s>>>(
      arena, arena_units, reinterpret_cast<const u64*>(inbox_off), ctx->n_pairs,
      reinterpret_cast<const u64*>(box_off_next), ctx->class_id, cn, (u64)next->n,
      ctx->d_status);
  return check_launch(ctx, "mig_unpack_kernel", s);
}
