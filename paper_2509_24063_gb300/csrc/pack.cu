// Step a2 — TeraAgent IO serialization (paper Sec. 2.2.1): every message is one
// contiguous buffer; each agent is copied as one fixed 64-byte block; the
// class identity is written once in the buffer header.  The receiver can use
// the buffer in place.
//
// pack_entries_kernel (all pairs): one thread per (agent, pair) entry, in
// agent order, as tera_partition emitted them: consecutive threads read
// nearby agents, so the column reads sweep the state arrays instead of
// jumping, and each record leaves as one 64-byte store to its place
// (entry -> record index from the partition's sort).
//
// pack_kernel (a range of pairs): eight adjacent threads build one record
// (each gathers one of the eight struct-of-arrays columns and writes one
// word), so a record leaves as one 64-byte segment.

#include "tera_internal.cuh"

using namespace tera;

namespace {

struct SoaPtrs {
  const u64* col[8];  // id, x, y, z, diameter, volume, adherence, density (as raw 64-bit words)
};

__device__ __forceinline__ const u64* column(const SoaPtrs& s, u32 w) {
  // select, not an indexed load from the parameter block
  const u64* c = s.col[0];
  c = w == 1 ? s.col[1] : c;
  c = w == 2 ? s.col[2] : c;
  c = w == 3 ? s.col[3] : c;
  c = w == 4 ? s.col[4] : c;
  c = w == 5 ? s.col[5] : c;
  c = w == 6 ? s.col[6] : c;
  c = w == 7 ? s.col[7] : c;
  return c;
}

// Eight adjacent threads build one record: thread w gathers column w of the
// agent and writes word w, so the record leaves as one 64-byte segment and
// eight independent gathers per record are in flight.
__global__ void __launch_bounds__(256)
    pack_kernel(SoaPtrs soa, const u32* __restrict__ pair_idx, const u64* __restrict__ pair_off,
                const u32* __restrict__ rec_pair, u32 p0, u32 p1, uint8_t* __restrict__ arena,
                u64 arena_units, u32 class_id, DevStatus* st) {
  const u64 g_lo = pair_off[p0], g_hi = pair_off[p1];
  if (g_hi + p1 > arena_units) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      latch(st, TERA_ECAPACITY);
      need(st, g_hi + p1);
    }
    return;
  }
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  // headers of the pair range
  for (u64 p = p0 + tid; p < p1; p += stride) {
    u64 m = pair_off[p + 1] - pair_off[p];
    write_taio_header(arena + (pair_off[p] + p) * kRecBytes, class_id, (u32)p, m);
  }
  const u64 work = (g_hi - g_lo) * 8;
  const u32 w = (u32)(tid & 7);  // stride is a multiple of 8
  const u64* col = column(soa, w);
  for (u64 q = tid; q < work; q += stride) {
    const u64 g = g_lo + (q >> 3);
    const u32 p = rec_pair[g];
    const u32 i = pair_idx[g];
    const u64 v = col[i];
    reinterpret_cast<u64*>(arena + (g + p + 1) * kRecBytes)[w] = v;
  }
}


// One thread per entry e of the last partition (agent order).
__global__ void __launch_bounds__(256)
    pack_entries_kernel(SoaPtrs soa, const u32* __restrict__ ent_key,
                        const u32* __restrict__ ent_agent, const u32* __restrict__ ent_dest,
                        const u64* __restrict__ pair_off, u64 P, uint8_t* __restrict__ arena,
                        u64 arena_units, u32 class_id, DevStatus* st) {
  const u64 E = pair_off[P];
  if (E + P > arena_units) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      latch(st, TERA_ECAPACITY);
      need(st, E + P);
    }
    return;
  }
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  for (u64 p = tid; p < P; p += stride) {
    const u64 m = pair_off[p + 1] - pair_off[p];
    write_taio_header(arena + (pair_off[p] + p) * kRecBytes, class_id, (u32)p, m);
  }
  for (u64 e = tid; e < E; e += stride) {
    const u32 a = ent_agent[e];
    const u64 g = ent_dest[e];
    const u64 p = ent_key[e];
    Rec R;
#pragma unroll
    for (int w = 0; w < 8; ++w) R.w[w] = soa.col[w][a];
    store_rec(arena + (g + p + 1) * kRecBytes, R);
  }
}

}  // namespace

extern "C" tera_status tera_pack(tera_ctx* ctx, const tera_soa* soa, const tera_partition_out* part,
                                 uint32_t pair_begin, uint32_t pair_end, uint8_t* rec_arena,
                                 uint64_t arena_units, void* stream) {
  if (!ctx || !soa || !part || !rec_arena) return TERA_EINVAL;
  if (pair_begin > pair_end || pair_end > ctx->n_pairs) return TERA_EINVAL;
  if (!part->pair_off || (!part->pair_idx && part->idx_capacity > 0)) return TERA_EINVAL;
  if (((uintptr_t)rec_arena) & 15u) return TERA_EINVAL;
  if (soa->n > 0 && (!soa->id || !soa->x || !soa->y || !soa->z || !soa->diameter || !soa->volume ||
                     !soa->adherence || !soa->density))
    return TERA_EINVAL;
  if (pair_begin == pair_end) return TERA_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  tera_status st = ensure_records(ctx, part->idx_capacity, s);
  if (st != TERA_OK) return st;
  SoaPtrs p;
  p.col[0] = reinterpret_cast<const u64*>(soa->id);
  p.col[1] = reinterpret_cast<const u64*>(soa->x);
  p.col[2] = reinterpret_cast<const u64*>(soa->y);
  p.col[3] = reinterpret_cast<const u64*>(soa->z);
  p.col[4] = reinterpret_cast<const u64*>(soa->diameter);
  p.col[5] = reinterpret_cast<const u64*>(soa->volume);
  p.col[6] = reinterpret_cast<const u64*>(soa->adherence);
  p.col[7] = reinterpret_cast<const u64*>(soa->density);
  // enough threads to cover every record of the range once on a full GPU
  u64 est = part->idx_capacity * 8 / 256 + 1;
  u64 maxg = (u64)grid_for(ctx, 8);
  unsigned blocks = (unsigned)(est < maxg ? est : maxg);
  if (!ctx->rec_pair) return TERA_EINVAL;  // tera_partition has not run on this context
  if (pair_begin == 0 && pair_end == ctx->n_pairs) {
    prof_begin(ctx, s);
    pack_entries_kernel<<<(unsigned)grid_for(ctx, 8), 256, 0, s>>>(
        p, ctx->keys_a, ctx->ent_agent, ctx->ent_dest,
        reinterpret_cast<const u64*>(part->pair_off), ctx->n_pairs, rec_arena, arena_units,
        ctx->class_id, ctx->d_status);
    return check_launch(ctx, "pack_entries_kernel", s);
  }
  prof_begin(ctx, s);
  pack_kernel<<<blocks, 256, 0, s>>>(p, part->pair_idx, reinterpret_cast<const u64*>(part->pair_off),
                                     ctx->rec_pair, pair_begin, pair_end, rec_arena, arena_units,
                                     ctx->class_id, ctx->d_status);
  return check_launch(ctx, "pack_kernel", s);
}
