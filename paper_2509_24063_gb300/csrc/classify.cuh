// Grid classification of one agent (paper Sec. 2.1 "Aura Update"): owner box
// and 26-bit aura mask by exact comparisons of order-preserving 64-bit keys.
// Shared by the partition and migration kernels.
#pragma once

#include "tera_internal.cuh"

namespace tera {

// Keys of one box along one axis: its edges e[i], e[i+1] and the aura
// thresholds e[i] + w (towards box i-1), e[i+1] - w (towards box i+1).
struct __align__(16) BoxKeys {
  u64 e0, e1, tl, th;
};

// Per-block copy of the grid: the box rows of the three axes sit in dynamic
// shared memory (grid_smem_bytes), axis a from row koff[a].
struct SmemGrid {
  u64 klo[3], khi[3];
  float flo[3], fscale[3];
  int n[3];
  int koff[3];
  int periodic;
};

__device__ __forceinline__ BoxKeys* grid_rows() {
  extern __shared__ BoxKeys tera_grid_rows[];
  return tera_grid_rows;
}

// Dynamic shared memory a kernel that calls load_grid is launched with.
inline size_t grid_smem_bytes(const tera_grid& g) {
  return sizeof(BoxKeys) * (size_t)(g.n[0] + g.n[1] + g.n[2]);
}

__device__ __forceinline__ void load_grid(SmemGrid& s, const GridTables* __restrict__ g) {
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    s.n[a] = g->n[a];
    s.klo[a] = g->klo[a];
    s.khi[a] = g->khi[a];
    s.flo[a] = g->flo[a];
    s.fscale[a] = g->fscale[a];
    s.koff[a] = a == 0 ? 0 : (a == 1 ? g->n[0] : g->n[0] + g->n[1]);
  }
  if (threadIdx.x == 0) s.periodic = g->periodic;
  BoxKeys* rows = grid_rows();
  int off = 0;
  for (int a = 0; a < 3; ++a) {
    const int n = g->n[a];
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      rows[off + k] = BoxKeys{g->ke[a][k], g->ke[a][k + 1], g->ktl[a][k], g->kth[a][k]};
    off += n;
  }
  __syncthreads();
}

// Box index along one axis of a value inside [lo, hi) (k = key_of(bits)):
// i = #{k in 1..n-1 : v >= e[k]}, and the keys of that box in *r.  A float32
// estimate of i is corrected by exact comparisons of the 64-bit keys, so the
// result is exactly the rule's; the estimate only saves the binary search.
__device__ __forceinline__ int axis_index(u64 bits, u64 k, int a, const SmemGrid& s, BoxKeys* r) {
  const int n = s.n[a];
  const BoxKeys* rows = grid_rows() + s.koff[a];
  const float f = (approx_f32(bits) - s.flo[a]) * s.fscale[a];
  int i = f > 0.0f ? (int)f : 0;
  i = i < n - 1 ? i : n - 1;
  BoxKeys b = rows[i];
  while (i > 0 && k < b.e0) b = rows[--i];
  while (i < n - 1 && k >= b.e1) b = rows[++i];
  *r = b;
  return i;
}

// One axis: the box index and the neighbour offsets whose aura holds v.
// Returns opts: bit 0 offset -1 qualifies (i > 0 and v < e[i] + w), bit 1
// offset 0, bit 2 offset +1 (i < n-1 and v >= e[i+1] - w); on a periodic
// axis the neighbour always exists.  0 when v is not in [lo, hi).
__device__ __forceinline__ u32 classify_axis(u64 bits, int a, const SmemGrid& s, int* idx) {
  const u64 k = key_of(bits);
  if (!(k >= s.klo[a] && k < s.khi[a])) {
    *idx = 0;
    return 0u;
  }
  const int n = s.n[a];
  BoxKeys b;
  const int i = axis_index(bits, k, a, s, &b);
  *idx = i;
  const bool wrap = (s.periodic >> a) & 1;
  const u32 lowq = (i > 0 || wrap) && (k < b.tl);
  const u32 highq = (i < n - 1 || wrap) && (k >= b.th);
  return 2u | lowq | (highq << 2);
}

// Bits 0, 1, 2 of v moved to bits 0, d, 2d.
__device__ __forceinline__ u32 spread3(u32 v, u32 d) {
  return (v & 1u) | ((v & 2u) << (d - 1)) | ((v & 4u) << (2 * d - 2));
}

__device__ __forceinline__ void classify_agent(u64 bx, u64 by, u64 bz, const SmemGrid& s,
                                               int* owner, u32* mask, bool* ok) {
  int ix, iy, iz;
  const u32 ox = classify_axis(bx, 0, s, &ix);
  const u32 oy = classify_axis(by, 1, s, &iy);
  const u32 oz = classify_axis(bz, 2, s, &iz);
  *ok = ox && oy && oz;
  if (!*ok) {
    *owner = -1;
    *mask = 0;
    return;
  }
  *owner = ix + s.n[0] * (iy + s.n[1] * iz);
  // bit (dx + 3 dy + 9 dz) for every qualifying offset triple: the products
  // place copies of ox at 3 dy and of that row at 9 dz (no carries)
  const u32 m = ox * spread3(oy, 3) * spread3(oz, 9);
  *mask = m & ~(1u << 13);
}

// Owner box of a position (the same rule without the aura mask), -1 when it
// is not in [lo, hi) on every axis.
__device__ __forceinline__ int locate_agent(u64 bx, u64 by, u64 bz, const SmemGrid& s) {
  const u64 b[3] = {bx, by, bz};
  int i[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const u64 k = key_of(b[a]);
    if (!(k >= s.klo[a] && k < s.khi[a])) return -1;
    BoxKeys r;
    i[a] = axis_index(b[a], k, a, s, &r);
  }
  return i[0] + s.n[0] * (i[1] + s.n[1] * i[2]);
}

}  // namespace tera
