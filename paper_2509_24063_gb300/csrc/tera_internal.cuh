// Internal definitions shared by the CUDA translation units of libtera.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tera.h"

namespace tera {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u32 kTaioMagic = 0x4F494154u;  // "TAIO"
constexpr u32 kWireMagic = 0x41524554u;  // "TERA"
constexpr u32 kVersion = 1u;
constexpr u32 kRecBytes = 64u;
constexpr u32 kHdrBytes = 64u;
constexpr int kMaxAxis = 256;
constexpr u32 kNoMatch = 0xFFFFFFFFu;

// Agents per classification tile and records per codec tile.
constexpr int kClassifyThreads = 256;
constexpr int kClassifyPerThread = 8;
constexpr int kClassifyTile = kClassifyThreads * kClassifyPerThread;  // 2048
constexpr int kCodecTile = 256;
// Warp tiles of the agent passes (classification, emit, migration): warp w
// owns agents [w * kWarpAgents, (w+1) * kWarpAgents); in round r lane l holds
// agents 64 r + 2 l and 64 r + 2 l + 1 of it (16-byte loads, coalesced).
// Per-warp counts give every warp its output position with no block-wide
// step; a block of kClassifyThreads threads covers kBlockAgents agents.
constexpr int kWarpAgents = 256;
constexpr int kWarpRounds = kWarpAgents / 64;
constexpr int kWarpsPerBlock = kClassifyThreads / 32;
constexpr int kBlockAgents = kWarpAgents * kWarpsPerBlock;  // 2048
// Runs of the partition's classification: 64 consecutive agents (one warp,
// one round of a classification tile), counted one by one.
constexpr int kRunAgents = 64;

// Radix sort of (pair, agent) entries.
constexpr int kSortThreads = 256;
constexpr int kSortPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // 4096
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Generic scan chunking.
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanChunk = kScanThreads * kScanPerThread;

struct DevStatus {
  u32 code;
  u32 abort;  // set when a partition overflowed: later kernels of the iteration skip work
  u64 required;
  u64 detail;
};

// Grid tables in device memory.  Every binary64 boundary is stored as an
// order-preserving 64-bit key (see key_of), so classification compares
// integers: exact, and independent of the GPU's binary64 throughput.
struct GridTables {
  int n[3];
  int periodic;                   // bit a: axis a is toroidal (box n-1 next to box 0)
  float flo[3], fscale[3];        // float estimate of the box index: (x - lo) * n / (hi - lo)
  u64 klo[3], khi[3];             // domain [lo, hi)
  u64 ke[3][kMaxAxis + 1];        // box edges e[k]
  u64 ktl[3][kMaxAxis];           // e[k] + w   (aura towards box k-1)
  u64 kth[3][kMaxAxis];           // e[k+1] - w (aura towards box k+1)
};

// Order-preserving key of a binary64 bit pattern: for non-NaN a, b,
// a < b  <=>  key(a) < key(b) as unsigned integers (-0.0 is first mapped to
// +0.0, as IEEE-754 compares them equal).  Positive NaNs map above +inf and
// negative NaNs below -inf, so a NaN never lies inside a finite [lo, hi).
__host__ __device__ __forceinline__ u64 key_of(u64 b) {
  b = (b == 0x8000000000000000ull) ? 0ull : b;
  const u64 neg = (u64)((long long)b >> 63);
  return b ^ (neg | 0x8000000000000000ull);
}

// Device-side totals (layout of tera_stats).
struct DevStats {
  u64 iterations, agents, records, ref_slots, holes, new_records, payload_bytes, wire_bytes;
};


__device__ __forceinline__ void latch(DevStatus* s, u32 code) { atomicCAS(&s->code, 0u, code); }
__device__ __forceinline__ void need(DevStatus* s, u64 req) { atomicMax(&s->required, req); }

__device__ __forceinline__ u64 mix64(u64 z) {
  // splitmix64 finalizer (Steele, Lea, Flood 2014)
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// Per-pair hash segments: pair p owns 2 m_p + 2 entries starting at
// 2 pair_off[p] + 2 p; an entry is (epoch << 32) | record index within the
// pair, and entries of older epochs are empty, so nothing is ever cleared.
__device__ __forceinline__ u64 seg_base(u64 pair_off_p, u32 p) { return 2 * pair_off_p + 2 * (u64)p; }
__device__ __forceinline__ u64 seg_size(u64 m) { return 2 * m + 2; }
__device__ __forceinline__ u64 seg_start(u64 id, u64 size) {
  return ((mix64(id) >> 32) * size) >> 32;  // range reduction without division
}

// Significant low bytes of a word: 0 for zero, else 8 - (leading zero bits / 8).
__device__ __forceinline__ u32 sig_bytes(u64 v) { return v ? 8u - ((u32)__clzll(v) >> 3) : 0u; }

__device__ __forceinline__ u32 round16(u32 v) { return (v + 15u) & ~15u; }
__device__ __forceinline__ u64 round16(u64 v) { return (v + 15ull) & ~15ull; }

// ---- warp / block scans (shuffle based) ----
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Exclusive block scan; `smem` holds >= 32 T.  Returns the exclusive prefix,
// writes the block total to *total.  All threads of the block must call it.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* smem, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) smem[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T s = lane < nwarps ? smem[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < nwarps) smem[lane] = si - s;
    if (lane == nwarps - 1) smem[32] = si;
  }
  __syncthreads();
  T res = smem[warp] + incl - v;
  *total = smem[32];
  __syncthreads();
  return res;
}

// Pair scan of two counters at once.
struct U64x2 {
  u64 a, b;
  __device__ __forceinline__ U64x2 operator+(const U64x2& o) const { return {a + o.a, b + o.b}; }
  __device__ __forceinline__ U64x2& operator+=(const U64x2& o) {
    a += o.a;
    b += o.b;
    return *this;
  }
  __device__ __forceinline__ U64x2 operator-(const U64x2& o) const { return {a - o.a, b - o.b}; }
};

__device__ __forceinline__ U64x2 shfl_up(U64x2 v, int o) {
  return {__shfl_up_sync(0xFFFFFFFFu, v.a, o), __shfl_up_sync(0xFFFFFFFFu, v.b, o)};
}

__device__ __forceinline__ U64x2 block_excl_scan2(U64x2 v, U64x2* smem, U64x2* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  U64x2 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    U64x2 t = shfl_up(incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) smem[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    U64x2 s = lane < nwarps ? smem[lane] : U64x2{0, 0};
    U64x2 si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      U64x2 t = shfl_up(si, o);
      if (lane >= o) si += t;
    }
    if (lane < nwarps) smem[lane] = si - s;
    if (lane == nwarps - 1) smem[32] = si;
  }
  __syncthreads();
  U64x2 res = smem[warp] + incl - v;
  *total = smem[32];
  __syncthreads();
  return res;
}

// 64-byte record as four 16-byte vectors.
struct Rec {
  u64 w[8];
};

__device__ __forceinline__ Rec load_rec(const uint8_t* p) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
  Rec r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ulonglong2 v = q[i];
    r.w[2 * i] = v.x;
    r.w[2 * i + 1] = v.y;
  }
  return r;
}

__device__ __forceinline__ void store_rec(uint8_t* p, const Rec& r) {
  ulonglong2* q = reinterpret_cast<ulonglong2*>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = make_ulonglong2(r.w[2 * i], r.w[2 * i + 1]);
}

__device__ __forceinline__ void write_taio_header(uint8_t* h, u32 class_id, u32 pair, u64 n) {
  ulonglong2* q = reinterpret_cast<ulonglong2*>(h);
  u64 w0 = (u64)kTaioMagic | ((u64)kVersion << 32) | ((u64)kRecBytes << 48);
  u64 w1 = (u64)class_id | ((u64)pair << 32);
  q[0] = make_ulonglong2(w0, w1);
  q[1] = make_ulonglong2(n, 0ull);
  q[2] = make_ulonglong2(0ull, 0ull);
  q[3] = make_ulonglong2(0ull, 0ull);
}

// Binary search: largest p in [lo, hi) with off[p] <= v (off non-decreasing).
template <typename T>
__device__ __forceinline__ u32 upper_pair(const T* off, u32 lo, u32 hi, u64 v) {
  while (hi - lo > 1) {
    u32 mid = (lo + hi) >> 1;
    if ((u64)off[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace tera

// The context (host side).
struct tera_ctx {
  int device;
  uint32_t class_id;
  tera_grid grid;
  uint32_t n_boxes;
  uint64_t n_pairs;
  int num_sms;
  uint64_t launches;
  uint64_t iterations;

  tera::GridTables* d_grid;
  tera::DevStatus* d_status;
  tera::DevStatus* h_status;  // pinned
  uint32_t* d_epoch;
  uint8_t* d_reset;  // [P] pairs to send raw once

  // partition scratch
  int64_t cap_agents;
  uint64_t cap_records;
  uint32_t* tile_cnt;      // [runs + 1] entries per run of 64 agents
  tera::u64* tile_base;     // [runs + 1] entries before each run
  // entries (agent, pair) of the last partition in agent order, and where
  // each went in the pair-sorted order (pack reads them in agent order)
  uint32_t* keys_a;        // [cap_records] pair of entry e
  uint32_t* ent_agent;     // [cap_records] agent of entry e
  uint32_t* ent_dest;      // [cap_records] record index of entry e
  uint32_t* keys_b;        // sort passes
  uint32_t* keys_c;
  uint32_t* vals_b;
  uint32_t* vals_c;
  uint32_t* rec_pair;      // pair of each record of the last partition (sorted keys)
  uint32_t* rs_hist;       // [kRadix * sort tiles]
  tera::u64* scan_part;     // partials of the generic scan
  uint64_t scan_part_cap;
  tera::u64* d_total;       // [4] scalars: total records, ...

  // per-pair hash segments + codec scratch
  tera::U64x2* seg;      // [2 cap_records + 2 P] hash entries {tag, id}
  uint32_t* matched;     // [cap_records] epoch of the iteration in which a slot took the record
  uint32_t* slot_src;  // [cap_records]
  tera::u64* unit_off;  // [P + 1]
  uint64_t cap_units;
  tera::U64x2* unit_sum;   // [cap_units]
  uint32_t* unit_pair;     // [cap_units] pair of each codec unit
  tera::U64x2* unit_base;  // [cap_units]
  tera::u64* pair_info;     // [P * 8] per-pair codec facts
  tera::u64* d_units_total;
  void* prof;  // per-kernel CUDA-event timing (ctx.cu)
  tera::DevStats* d_stats;


  // learned predictor (cell counts of both sides, per-slot predictions)
  uint64_t ncell[3];
  uint64_t pred_cap;
  tera::u64* cseg_enc;
  tera::u64* cseg_dec;
  tera::u64* pscr;
  tera::u64* unit_res;
  uint64_t unit_res_cap;
  float* mlp_scratch;       // training: compacted samples + gradient partials
  uint64_t mlp_scratch_cap;
  // batched codec (batched.cu)
  tera::u64* b_scalars;  // [0] work items, [1] ticket, [2] abort flag
  tera::u64* b_ptot;     // [P * 4] per-pair totals of the match step
  tera::u64* b_items;    // work list (team items first)
  uint64_t b_items_cap;
  uint32_t* b_team;      // [P * 8] barrier counters of the teams
  tera::U64x2* b_tsum;   // per-tile totals of the team pairs
  uint64_t b_tsum_cap;
  tera::u64* b_tbase;    // [P] first tile total of each team pair
  // agent migration (migrate.cu)
  uint64_t m_cap_agents;   // agents the tile arrays cover
  uint64_t m_cap_leavers;  // leavers the list and sort buffers hold
  uint32_t* m_tile_cnt;    // [warp tiles + 1] leavers per warp tile of 256 agents
  tera::u64* m_tile_base;  // [warp tiles + 1] leavers before each warp tile (total last)
  tera::u64* m_from;       // [boxes] leavers per source box
  tera::u64* m_before;     // [boxes] leavers of the boxes before each box
  tera::u64* m_cnt;        // [boxes * 27] leavers per inbox
  uint32_t* m_key;         // [m_cap_leavers] inbox of leaver k (agent order)
  uint32_t* m_agent;       // [m_cap_leavers] agent of leaver k
  uint32_t* m_sorted;      // [m_cap_leavers] agent of inbox record j
  uint32_t* m_dest;        // [m_cap_leavers] inbox-order position of leaver k
  uint32_t* m_keys_b;
  uint32_t* m_keys_c;
  uint32_t* m_vals_b;
  uint32_t* m_vals_c;
  uint32_t* m_hist;
};

namespace tera {
// ctx.cu
void prof_begin(tera_ctx* ctx, cudaStream_t s);
tera_status check_launch(tera_ctx* ctx, const char* name, cudaStream_t s);
tera_status ensure_agents(tera_ctx* ctx, int64_t n, cudaStream_t s);
tera_status ensure_records(tera_ctx* ctx, uint64_t cap, cudaStream_t s);
tera_status ensure_units(tera_ctx* ctx, uint64_t cap, cudaStream_t s);
// Exclusive scan of n u32 values into n+1 outputs (total last), any n.
tera_status scan_u32(tera_ctx* ctx, const u32* in, u64* out64, u32* out32, u64 n, cudaStream_t s);
int grid_for(tera_ctx* ctx, int blocks_per_sm);
// unit_pair[u] = p0 + k for every unit u of range pair k (skipped when
// units_total[1] flags an aborted call).
tera_status launch_unit_map(tera_ctx* ctx, u32 p0, u64 npr, cudaStream_t s);
// Scratch of the learned predictor for the current record capacity.
tera_status ensure_pred(tera_ctx* ctx);
// Scratch of the batched codec.
tera_status ensure_batched(tera_ctx* ctx);
// Scratch of agent migration for n agents and up to `leavers` leavers.
tera_status ensure_migrate(tera_ctx* ctx, uint64_t n, uint64_t leavers);

// partition.cu: stable LSD radix sort of entries by u32 key.
struct SortBufs {
  u32* keys_b;
  u32* keys_c;
  u32* vals_b;
  u32* vals_c;
  u32* hist;  // [kRadix * sort tiles + 1]
};
tera_status radix_sort_entries(tera_ctx* ctx, const SortBufs& b, const u32* keys_in,
                               const u32* agent, u32* dest, u32* vals_final, const u64* total_ptr,
                               u64 cap, u64 key_limit, const u32** sorted_keys, cudaStream_t s);
}  // namespace tera
