// Step a1 — grid classification and per-pair message lists (paper Sec. 2.1,
// "Aura Update": agents within the interaction distance of a neighbouring
// box are sent to it every iteration; the aura is narrower than the box).
//
// Kernels:
//   classify_kernel  one pass over x,y,z (coalesced 16-byte loads): owner box,
//                    26-bit aura mask, count of (agent, pair) entries of every
//                    run of 64 consecutive agents; per axis a bucket table in
//                    shared memory answers most coordinates, the exact key
//                    comparisons the rest
//   emit_kernel      stable compaction of the entries in agent order (warp
//                    scans inside a run, run bases from a scan)
//   rs_hist_kernel / rs_scatter_kernel
//                    stable LSD radix sort of the entry indices by pair
//                    index, so each pair's list keeps ascending agent order
//                    (tiles staged into shared memory by cp.async); the last
//                    pass writes the agent of every record and the record
//                    index of every entry (pack reads in agent order)
//   pair_off_kernel  per-pair counts and offsets from the sorted keys
#include "classify.cuh"
#include "tera_internal.cuh"

using namespace tera;

namespace {

// One axis by the bucket table when the coordinate's bucket holds an answer,
// else by the exact key comparisons.  The estimate is taken only for
// magnitudes in the float normal range (2^-126 <= |v| < 2^128, which also
// sends NaN and infinities to the exact path).
__device__ __forceinline__ u32 classify_axis_table(u64 bits, int a, const SmemGrid& s,
                                                   const uint8_t* tab, float flo, float fs,
                                                   int* idx) {
  const u32 hi = (u32)(bits >> 32);
  const u32 ha = hi & 0x7FFFFFFFu;
  if (ha - 0x38100000u < 0x0FE00000u) {
    const float af = __uint_as_float((hi & 0x80000000u) | ((ha - 0x38000000u) << 3));
    const int j = __float2int_rz((af - flo) * fs);
    if ((u32)j < (u32)kAxisBuckets) {
      const u32 e = tab[j];
      if (!(e & kBucketExact)) {
        *idx = (int)(e >> 2);
        return 2u | (e & 1u) | ((e & 2u) << 1);
      }
    }
  }
  return classify_axis(bits, a, s, idx);
}

// classify_agent with the bucket tables in shared memory (tab: three axes of
// kAxisBuckets entries).
__device__ __forceinline__ void classify_agent_table(u64 bx, u64 by, u64 bz, const SmemGrid& s,
                                                     const uint8_t* tab, const float* flo,
                                                     const float* fs, int* owner, u32* mask,
                                                     bool* ok) {
  int ix, iy, iz;
  const u32 ox = classify_axis_table(bx, 0, s, tab, flo[0], fs[0], &ix);
  const u32 oy = classify_axis_table(by, 1, s, tab + kAxisBuckets, flo[1], fs[1], &iy);
  const u32 oz = classify_axis_table(bz, 2, s, tab + 2 * kAxisBuckets, flo[2], fs[2], &iz);
  *ok = ox && oy && oz;
  if (!*ok) {
    *owner = -1;
    *mask = 0;
    return;
  }
  *owner = ix + s.n[0] * (iy + s.n[1] * iz);
  const u32 m = ox * spread3(oy, 3) * spread3(oz, 9);
  *mask = m & ~(1u << 13);
}

// Each block classifies tiles of kClassifyTile agents (tile blockIdx.x, then
// every gridDim.x-th: the grid holds the blocks resident at once, so the grid
// rows and the bucket tables are copied into shared memory once per block).
// In round k of a tile, thread t holds agents 512k + 2t and 512k + 2t + 1 (one
// 16-byte load per coordinate), so every warp load is fully coalesced, and
// each warp covers a run of kRunAgents consecutive agents per round; the
// number of (agent, pair) entries of every run is written (runs are in agent
// order).  bk == nullptr: every agent takes the exact key comparisons.
__global__ void __launch_bounds__(kClassifyThreads, 6)
    classify_kernel(const u64* __restrict__ x, const u64* __restrict__ y,
                    const u64* __restrict__ z, u64 n, const GridTables* __restrict__ g,
                    const AxisBuckets* __restrict__ bk, u64 n_tiles, int* __restrict__ owner,
                    u32* __restrict__ mask, u32* __restrict__ run_cnt, u64 n_runs, DevStatus* st,
                    DevStats* stats) {
  __shared__ SmemGrid sg;
  __shared__ float s_flo[3], s_fs[3];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    stats->iterations += 1;
    stats->agents += n;
  }
  // the tables follow the grid rows (a multiple of 32 bytes) in dynamic shared memory
  uint8_t* tab = reinterpret_cast<uint8_t*>(grid_rows() + (g->n[0] + g->n[1] + g->n[2]));
  if (bk) {
    const uint4* src = reinterpret_cast<const uint4*>(bk->tab);
    uint4* dst = reinterpret_cast<uint4*>(tab);
    for (int i = threadIdx.x; i < 3 * kAxisBuckets / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x < 3) {
      s_flo[threadIdx.x] = bk->flo[threadIdx.x];
      s_fs[threadIdx.x] = bk->fs[threadIdx.x];
    }
  }
  load_grid(sg, g);  // ends with a block barrier
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (u64 tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const u64 tile0 = tile * kClassifyTile;
#pragma unroll
    for (int k = 0; k < kClassifyPerThread / 2; ++k) {
      const u64 a0 = tile0 + (u64)k * (2 * kClassifyThreads) + 2u * threadIdx.x;
      u64 vx[2], vy[2], vz[2];
      if (a0 + 1 < n) {
        ulonglong2 tx = *reinterpret_cast<const ulonglong2*>(x + a0);
        ulonglong2 ty = *reinterpret_cast<const ulonglong2*>(y + a0);
        ulonglong2 tz = *reinterpret_cast<const ulonglong2*>(z + a0);
        vx[0] = tx.x; vx[1] = tx.y; vy[0] = ty.x; vy[1] = ty.y; vz[0] = tz.x; vz[1] = tz.y;
      } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (a0 + q < n) {
            vx[q] = x[a0 + q]; vy[q] = y[a0 + q]; vz[q] = z[a0 + q];
          } else {
            vx[q] = vy[q] = vz[q] = 0ull;
          }
        }
      }
      int o[2];
      u32 m[2];
      u32 cnt = 0;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        bool ok;
        if (bk)
          classify_agent_table(vx[q], vy[q], vz[q], sg, tab, s_flo, s_fs, &o[q], &m[q], &ok);
        else
          classify_agent(vx[q], vy[q], vz[q], sg, &o[q], &m[q], &ok);
        if (a0 + q < n) {
          bad |= !ok;
          cnt += __popc(m[q]);
        }
      }
      if (a0 + 1 < n) {
        *reinterpret_cast<int2*>(owner + a0) = make_int2(o[0], o[1]);
        *reinterpret_cast<uint2*>(mask + a0) = make_uint2(m[0], m[1]);
      } else if (a0 < n) {
        owner[a0] = o[0];
        mask[a0] = m[0];
      }
      cnt = warp_sum(cnt);
      const u64 run = (a0 - 2u * lane) / kRunAgents;
      if (lane == 0 && run < n_runs) run_cnt[run] = cnt;
    }
  }
  if (bad) latch(st, TERA_EDOMAIN);
}

// Emit (pair, agent) entries in agent order, with the rounds and runs of
// classify_kernel: run r writes its entries from run_base[r]; within a run,
// lanes are ranked by a warp scan.
__global__ void __launch_bounds__(kClassifyThreads)
    emit_kernel(const int* __restrict__ owner, const u32* __restrict__ mask, u64 n,
                const u64* __restrict__ run_base, u64 n_runs, u32* __restrict__ keys,
                u32* __restrict__ vals, u64 cap, DevStatus* st) {
  const u64 total = run_base[n_runs];
  const u64 n_entries = total;  // (a warp's own count below is also called total)
  if (total > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      latch(st, TERA_ECAPACITY);
      need(st, total);
      atomicExch(&st->abort, 1u);
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const u64 tile0 = (u64)blockIdx.x * kClassifyTile;
  for (int k = 0; k < kClassifyPerThread / 2; ++k) {
    const u64 a0 = tile0 + (u64)k * (2 * kClassifyThreads) + 2u * threadIdx.x;
    const u64 first = a0 - 2u * lane;
    if (first >= n) break;  // warp-uniform
    u32 m[2] = {0u, 0u};
    int o[2] = {0, 0};
    if (a0 + 1 < n) {
      uint2 mm = *reinterpret_cast<const uint2*>(mask + a0);
      m[0] = mm.x; m[1] = mm.y;
      if (m[0] | m[1]) {
        int2 oo = *reinterpret_cast<const int2*>(owner + a0);
        o[0] = oo.x; o[1] = oo.y;
      }
    } else if (a0 < n) {
      m[0] = mask[a0];
      if (m[0]) o[0] = owner[a0];
    }
    const u32 c = __popc(m[0]) + __popc(m[1]);
    const u32 inc = warp_incl_scan<u32>(c);
    const u32 total = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const u64 base = run_base[first / kRunAgents];
    // the run's entries written by the whole warp, lane i taking entry i of
    // each 32: its source lane is the first whose inclusive count exceeds i
    for (u32 r0 = 0; r0 < total; r0 += 32) {  // warp-uniform
      const u32 idx = r0 + (u32)lane;
      u32 src = 0;
#pragma unroll
      for (u32 b = 16; b >= 1; b >>= 1)
        if (__shfl_sync(0xFFFFFFFFu, inc, (int)(src + b - 1)) <= idx) src += b;
      const u32 s_inc = __shfl_sync(0xFFFFFFFFu, inc, (int)src);
      const u32 s_c = __shfl_sync(0xFFFFFFFFu, c, (int)src);
      const u32 s_m0 = __shfl_sync(0xFFFFFFFFu, m[0], (int)src);
      const u32 s_m1 = __shfl_sync(0xFFFFFFFFu, m[1], (int)src);
      const int s_o0 = __shfl_sync(0xFFFFFFFFu, o[0], (int)src);
      const int s_o1 = __shfl_sync(0xFFFFFFFFu, o[1], (int)src);
      if (idx >= total) continue;
      u32 k = idx - (s_inc - s_c);  // entry k of the source lane's two agents
      const u32 n0 = __popc(s_m0);
      const bool second = k >= n0;
      u32 mm = second ? s_m1 : s_m0;
      k = second ? k - n0 : k;
      for (u32 t = 0; t < k; ++t) mm &= mm - 1;
      const u32 b = (u32)(__ffs(mm) - 1);
      if (!in_bounds(st, base + idx, 0, n_entries)) continue;
      keys[base + idx] = (u32)(second ? s_o1 : s_o0) * 27u + b;
      vals[base + idx] = (u32)(first + 2u * src + (second ? 1u : 0u));  // the entry's agent
    }
  }
}

__device__ __forceinline__ u64 live_entries(const u64* total_ptr, u64 cap) {
  u64 t = *total_ptr;
  return t > cap ? 0 : t;
}

// Digit histogram of one sort tile; hist is digit-major: hist[d * n_tiles + t].
__global__ void __launch_bounds__(kSortThreads)
    rs_hist_kernel(const u32* __restrict__ keys, const u64* __restrict__ total_ptr, u64 cap,
                   u32 shift, u32 radix, u32* __restrict__ hist, u32 n_tiles) {
  __shared__ u32 cnt[kRadix];
  const u64 E = live_entries(total_ptr, cap);
  for (u32 d = threadIdx.x; d < radix; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  const u64 t0 = (u64)blockIdx.x * kSortTile;
  if (t0 < E) {
#pragma unroll 4
    for (int k = 0; k < kSortPerThread; ++k) {
      u64 i = t0 + (u64)k * kSortThreads + threadIdx.x;
      if (i < E) atomicAdd(&cnt[(keys[i] >> shift) & (radix - 1)], 1u);
    }
  }
  __syncthreads();
  for (u32 d = threadIdx.x; d < radix; d += blockDim.x) hist[(u64)d * n_tiles + blockIdx.x] = cnt[d];
}

// Stable scatter of one sort tile of kSortTile entries.  The tile's input
// (keys, entry indices when given, agents) is first copied into shared memory
// in input order by cp.async in 16-byte pieces (a ragged end, or unaligned
// arrays, by plain loads), so the tile pays the latency of its global loads
// once.  The tile is then ranked in kSortPerThread / 4 rounds: in a round warp
// w takes 128 consecutive entries (4 sub-steps of 32, lane order), ranks equal
// digits with match_any against warp-private counters, and one prefix over the
// warps places them; the tile-local sorted position of every entry (digit
// start + rank) records the entry's place in the tile (inv).  The tile is
// written out in sorted order, so consecutive threads write consecutive
// addresses of a digit's run.  Each entry carries its index (vals_in ==
// nullptr on the first pass: entry i is at position i) and its agent
// (agents_in, read in input order: the entry list's agents on the first pass,
// the previous pass's output after it).  Every pass but the last writes both;
// the last writes the agent as the value (vals_out[pos] = agent) and, when
// dest is given, the entry's record index (dest[e] = pos).  kR bounds the
// radix (digit arrays in shared memory).
constexpr int kSortSub = 4;  // sub-steps of 32 entries per warp and round

// Dynamic shared memory of a scatter: raw keys and agents, the sorted-position
// index, and the raw entry indices when the pass reads them.
__host__ __device__ constexpr size_t sort_smem_bytes(bool with_vals) {
  return (with_vals ? 3 : 2) * sizeof(u32) * kSortTile + sizeof(unsigned short) * kSortTile;
}

__device__ __forceinline__ void cp_async16(u32* smem_dst, const u32* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" : : "r"(dst), "l"(gmem_src) : "memory");
}

template <u32 kR>
__global__ void __launch_bounds__(kSortThreads)
    rs_scatter_kernel(const u32* __restrict__ keys_in, const u32* __restrict__ vals_in,
                      const u32* __restrict__ agents_in, u32* __restrict__ keys_out,
                      u32* __restrict__ vals_out, u32* __restrict__ agents_out,
                      u32* __restrict__ dest, int last, const u64* __restrict__ total_ptr, u64 cap,
                      u32 shift, u32 radix, const u32* __restrict__ hist_scan, u32 n_tiles,
                      DevStatus* st) {
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kRoundEntries = kSortThreads * kSortSub;
  extern __shared__ __align__(16) u32 sort_stage[];
  u32* rkey = sort_stage;
  u32* ragt = sort_stage + kSortTile;
  unsigned short* inv = reinterpret_cast<unsigned short*>(sort_stage + 2 * kSortTile);
  u32* rval = sort_stage + 2 * kSortTile + kSortTile / 2;  // only when vals_in != nullptr
  __shared__ u32 base[kR];    // global start of each digit for this tile
  __shared__ u32 lstart[kR];  // tile-local start of each digit
  __shared__ u32 run[kR];     // entries of each digit placed in earlier rounds
  __shared__ u32 wcnt[kWarps][kR];
  __shared__ u32 sm[33];
  const u64 E = live_entries(total_ptr, cap);
  const u64 t0 = (u64)blockIdx.x * kSortTile;
  if (t0 >= E) return;
  const u32 tile_n = (u32)(E - t0 < (u64)kSortTile ? E - t0 : (u64)kSortTile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  {
    const uintptr_t al = reinterpret_cast<uintptr_t>(keys_in) |
                         reinterpret_cast<uintptr_t>(agents_in) |
                         reinterpret_cast<uintptr_t>(vals_in);
    const u32 n4 = (al & 15u) == 0 ? tile_n / 4 : 0;  // t0 is a multiple of 4 entries
    for (u32 c = threadIdx.x; c < n4; c += blockDim.x) {
      cp_async16(rkey + 4 * c, keys_in + t0 + 4 * c);
      cp_async16(ragt + 4 * c, agents_in + t0 + 4 * c);
      if (vals_in) cp_async16(rval + 4 * c, vals_in + t0 + 4 * c);
    }
    asm volatile("cp.async.commit_group;" : : : "memory");
    for (u32 li = 4 * n4 + threadIdx.x; li < tile_n; li += blockDim.x) {
      rkey[li] = keys_in[t0 + li];
      ragt[li] = agents_in[t0 + li];
      if (vals_in) rval[li] = vals_in[t0 + li];
    }
  }
  {
    const u32 d = threadIdx.x;
    u32 c = 0;
    if (d < radix) {
      const u64 at = (u64)d * n_tiles + blockIdx.x;
      base[d] = hist_scan[at];
      c = hist_scan[at + 1] - hist_scan[at];
      run[d] = 0;
    }
    u32 tot;
    const u32 ex = block_excl_scan<u32>(c, sm, &tot);
    if (d < radix) lstart[d] = ex;
  }
  asm volatile("cp.async.wait_all;" : : : "memory");
  __syncthreads();
  for (u32 r0 = 0; r0 < tile_n; r0 += kRoundEntries) {  // block-uniform
    for (u32 d = lane; d < radix; d += 32) wcnt[warp][d] = 0;
    __syncwarp();
    u32 dig[kSortSub], rank[kSortSub];
#pragma unroll
    for (int q = 0; q < kSortSub; ++q) {
      const u32 li = r0 + (u32)warp * (32 * kSortSub) + (u32)q * 32 + (u32)lane;
      const bool live = li < tile_n;
      dig[q] = live ? ((rkey[li] >> shift) & (radix - 1)) : kR;  // sentinel for padding
      const u32 peers = __match_any_sync(0xFFFFFFFFu, dig[q]);
      rank[q] = (live ? wcnt[warp][dig[q]] : 0u) + __popc(peers & lt);
      __syncwarp();
      if (live && (peers & lt) == 0u) wcnt[warp][dig[q]] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    for (u32 d = threadIdx.x; d < radix; d += blockDim.x) {
      u32 sacc = run[d];
      for (int w = 0; w < kWarps; ++w) {
        const u32 c = wcnt[w][d];
        wcnt[w][d] = sacc;
        sacc += c;
      }
      run[d] = sacc;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSortSub; ++q) {
      if (dig[q] < kR) {
        const u32 li = r0 + (u32)warp * (32 * kSortSub) + (u32)q * 32 + (u32)lane;
        inv[lstart[dig[q]] + wcnt[warp][dig[q]] + rank[q]] = (unsigned short)li;
      }
    }
    __syncthreads();
  }
  for (u32 lp = threadIdx.x; lp < tile_n; lp += blockDim.x) {
    const u32 src = inv[lp];
    const u32 key = rkey[src], a = ragt[src];
    const u32 v = vals_in ? rval[src] : (u32)(t0 + src);
    const u32 d = (key >> shift) & (radix - 1);
    const u32 pos = base[d] + (lp - lstart[d]);
    if (!in_bounds(st, pos, 0, E) || !in_bounds(st, v, 0, E)) continue;
    keys_out[pos] = key;
    if (last) {
      vals_out[pos] = a;
      if (dest) dest[v] = pos;
    } else {
      vals_out[pos] = v;
      agents_out[pos] = a;
    }
  }
}

__device__ __forceinline__ u64 lower_bound_u32(const u32* a, u64 n, u32 v) {
  u64 lo = 0, hi = n;
  while (lo < hi) {
    u64 mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void pair_off_kernel(const u32* __restrict__ sorted_keys,
                                const u64* __restrict__ total_ptr, u64 cap, u64 n_pairs,
                                u64* __restrict__ pair_off, u64* __restrict__ pair_count,
                                DevStats* stats) {
  const u64 E = live_entries(total_ptr, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) stats->records += E;
  for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p <= n_pairs;
       p += (u64)gridDim.x * blockDim.x) {
    u64 a = lower_bound_u32(sorted_keys, E, (u32)p);
    pair_off[p] = a;
    if (p < n_pairs) pair_count[p] = lower_bound_u32(sorted_keys, E, (u32)(p + 1)) - a;
  }
}

}  // namespace

namespace tera {

// Stable LSD radix sort of entries by a u32 key (every key < key_limit),
// ceil(bits / 8) digit passes.  The entry count is read on the device
// (*total_ptr; nothing is sorted when it exceeds cap).  Pass k reads (kin, vin,
// ain) and writes the b buffers (k even) or the c buffers; the last pass
// writes the sorted keys to the buffer it does not read, vals_final[pos] =
// agent[e] for the entry e sorted to pos, and dest[e] = pos (dest may be null).
// The agents travel with the entries (read in order on every pass).
tera_status radix_sort_entries(tera_ctx* ctx, const SortBufs& b, const u32* keys_in,
                               const u32* agent, u32* dest, u32* vals_final, const u64* total_ptr,
                               u64 cap, u64 key_limit, const u32** sorted_keys, cudaStream_t s) {
  int bits = 1;
  while ((1ull << bits) < key_limit) ++bits;
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  const int dbits = (bits + passes - 1) / passes;
  const u32 radix = 1u << dbits;
  const u64 sort_tiles = cap == 0 ? 1 : (cap + kSortTile - 1) / kSortTile;
  const u32* kin = keys_in;
  const u32* vin = nullptr;
  const u32* ain = agent;
  u32* kfinal = (passes & 1) ? b.keys_b : b.keys_c;
  tera_status st;
  static bool smem_set = false;
  if (!smem_set) {
    cudaFuncSetAttribute(rs_scatter_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem_bytes(true));
    cudaFuncSetAttribute(rs_scatter_kernel<kRadix>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem_bytes(true));
    smem_set = true;
  }
  for (int pass = 0; pass < passes && cap > 0; ++pass) {
    const u32 shift = (u32)(pass * dbits);
    const bool last = pass + 1 == passes;
    u32* kout = last ? kfinal : ((pass & 1) ? b.keys_c : b.keys_b);
    u32* vout = last ? vals_final : ((pass & 1) ? b.vals_c : b.vals_b);
    u32* aout = last ? nullptr : ((pass & 1) ? b.agents_c : b.agents_b);
    prof_begin(ctx, s);
    rs_hist_kernel<<<(unsigned)sort_tiles, kSortThreads, 0, s>>>(kin, total_ptr, cap, shift, radix,
                                                                 b.hist, (u32)sort_tiles);
    if ((st = check_launch(ctx, "rs_hist_kernel", s)) != TERA_OK) return st;
    if ((st = scan_u32(ctx, b.hist, nullptr, b.hist, (u64)radix * sort_tiles, s)) != TERA_OK)
      return st;
    prof_begin(ctx, s);
    const size_t smem = sort_smem_bytes(vin != nullptr);
    if (radix <= 128)
      rs_scatter_kernel<128><<<(unsigned)sort_tiles, kSortThreads, smem, s>>>(
          kin, vin, ain, kout, vout, aout, last ? dest : nullptr, last ? 1 : 0, total_ptr, cap,
          shift, radix, b.hist, (u32)sort_tiles, ctx->d_status);
    else
      rs_scatter_kernel<kRadix><<<(unsigned)sort_tiles, kSortThreads, smem, s>>>(
          kin, vin, ain, kout, vout, aout, last ? dest : nullptr, last ? 1 : 0, total_ptr, cap,
          shift, radix, b.hist, (u32)sort_tiles, ctx->d_status);
    if ((st = check_launch(ctx, "rs_scatter_kernel", s)) != TERA_OK) return st;
    kin = kout;
    vin = vout;
    ain = aout;
  }
  *sorted_keys = kin;
  return TERA_OK;
}

}  // namespace tera

extern "C" tera_status tera_partition(tera_ctx* ctx, const tera_soa* soa, tera_partition_out* out,
                                      void* stream) {
  TERA_CALL_RANGE("tera_partition");
  if (!ctx || !soa || !out) return TERA_EINVAL;
  if (soa->n < 0 || soa->n > (int64_t)0xFFFFFFFFll) return TERA_EINVAL;
  if (soa->n > 0 && (!soa->x || !soa->y || !soa->z)) return TERA_EINVAL;
  if (!out->owner || !out->mask || !out->pair_count || !out->pair_off ||
      (out->idx_capacity > 0 && !out->pair_idx))
    return TERA_EINVAL;
  if (out->idx_capacity > 0xFFFFFFFFull) return TERA_EINVAL;
  // 16-byte loads of x, y, z and 8-byte stores of owner / mask
  if (((uintptr_t)soa->x | (uintptr_t)soa->y | (uintptr_t)soa->z) & 15u) return TERA_EINVAL;
  if (((uintptr_t)out->owner | (uintptr_t)out->mask) & 7u) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u64 n = (u64)soa->n;
  tera_status st;
  if ((st = ensure_agents(ctx, soa->n, s)) != TERA_OK) return st;
  if (!ctx->tile_cnt || !ctx->tile_base) return TERA_ENOMEM;
  if ((st = ensure_records(ctx, out->idx_capacity, s)) != TERA_OK) return st;
  ctx->iterations += 1;
  cudaMemsetAsync(&ctx->d_status->abort, 0, sizeof(u32), s);
  const u64 blocks = n == 0 ? 1 : (n + kClassifyTile - 1) / kClassifyTile;
  const u64 runs = n == 0 ? 1 : (n + kRunAgents - 1) / kRunAgents;
  if (n == 0) cudaMemsetAsync(ctx->tile_cnt, 0, sizeof(u32), s);
  // resident blocks only (6 per SM): each copies the tables into shared memory once
  const size_t csmem =
      grid_smem_bytes(ctx->grid) + (ctx->d_buckets ? 3 * (size_t)kAxisBuckets : 0);
  static bool csmem_set = false;
  if (!csmem_set) {
    cudaFuncSetAttribute(classify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(BoxKeys) * 3 * kMaxAxis + 3 * (size_t)kAxisBuckets));
    csmem_set = true;
  }
  const u64 cgrid = blocks < (u64)ctx->num_sms * 6 ? blocks : (u64)ctx->num_sms * 6;
  prof_begin(ctx, s);
  classify_kernel<<<(unsigned)cgrid, kClassifyThreads, csmem, s>>>(
      reinterpret_cast<const u64*>(soa->x), reinterpret_cast<const u64*>(soa->y),
      reinterpret_cast<const u64*>(soa->z), n, ctx->d_grid, ctx->d_buckets, blocks, out->owner,
      out->mask, ctx->tile_cnt, runs, ctx->d_status, ctx->d_stats);
  if ((st = check_launch(ctx, "classify_kernel", s)) != TERA_OK) return st;
  if ((st = scan_u32(ctx, ctx->tile_cnt, ctx->tile_base, nullptr, runs, s)) != TERA_OK)
    return st;

  const u64 P = ctx->n_pairs;
  const u64 cap = out->idx_capacity;
  const u64* total_ptr = ctx->tile_base + runs;
  if (cap > 0 || n > 0) {
    prof_begin(ctx, s);
    emit_kernel<<<(unsigned)blocks, kClassifyThreads, 0, s>>>(
        out->owner, out->mask, n, ctx->tile_base, runs, ctx->keys_a, ctx->ent_agent, cap,
        ctx->d_status);
    if ((st = check_launch(ctx, "emit_kernel", s)) != TERA_OK) return st;
  }
  const SortBufs bufs{ctx->keys_b,   ctx->keys_c,   ctx->vals_b, ctx->vals_c,
                      ctx->agents_b, ctx->agents_c, ctx->rs_hist};
  const u32* sorted = nullptr;
  if ((st = radix_sort_entries(ctx, bufs, ctx->keys_a, ctx->ent_agent, ctx->ent_dest, out->pair_idx,
                               total_ptr, cap, P, &sorted, s)) != TERA_OK)
    return st;
  ctx->rec_pair = const_cast<u32*>(sorted);
  ctx->pack_n = soa->n;
  prof_begin(ctx, s);
  pair_off_kernel<<<(unsigned)((P + 256) / 256), 256, 0, s>>>(
      sorted, total_ptr, cap, P, reinterpret_cast<u64*>(out->pair_off),
      reinterpret_cast<u64*>(out->pair_count), ctx->d_stats);
  return check_launch(ctx, "pair_off_kernel", s);
}
