// Device-side definitions shared by the CUDA translation units of libtera:
// constants, status and grid tables, keys, scans and hash-segment helpers.
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
constexpr int kSortPerThread = 12;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // 3072
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

// A float32 near a binary64 value from the high word of its bits, by integer
// operations only (exponent re-biased, mantissa cut to 20 bits; a binary64
// conversion instruction runs at the GPU's low binary64 rate).  Values
// outside the normal float range give a meaningless estimate: callers only
// use it as the start of an exact search.
__device__ __forceinline__ float approx_f32(u64 bits) {
  const u32 hi = (u32)(bits >> 32);
  return __uint_as_float((hi & 0x80000000u) | (((hi & 0x7FFFFFFFu) - 0x38000000u) << 3));
}

// Device-side totals (layout of tera_stats).
struct DevStats {
  u64 iterations, agents, records, ref_slots, holes, new_records, payload_bytes, wire_bytes;
};


__device__ __forceinline__ void latch(DevStatus* s, u32 code) { atomicCAS(&s->code, 0u, code); }
__device__ __forceinline__ void need(DevStatus* s, u64 req) { atomicMax(&s->required, req); }

// Bounds check of the debug build (compiled with TERA_DEBUG_BOUNDS): true
// when lo <= i < hi; otherwise TERA_EBOUNDS is latched and the caller skips
// its write.  Other builds check nothing (always true, no code).
__device__ __forceinline__ bool in_bounds(DevStatus* s, u64 i, u64 lo, u64 hi) {
#ifdef TERA_DEBUG_BOUNDS
  if (i >= lo && i < hi) return true;
  latch(s, TERA_EBOUNDS);
  return false;
#else
  (void)s;
  (void)i;
  (void)lo;
  (void)hi;
  return true;
#endif
}

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
