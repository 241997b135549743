// Step a2 — TeraAgent IO serialization (paper Sec. 2.2.1): every message is one
// contiguous buffer; each agent is copied as one fixed 64-byte block; the
// class identity is written once in the buffer header.  The receiver can use
// the buffer in place.
//
// pack_runs_kernel (all pairs, columns 16-byte aligned): one pass over the
// agents in the classification's runs of 64; a lane loads the columns of its
// two agents once (16-byte loads) and stores the record once per entry, at
// the record index the partition's sort gave the entry.
//
// pack_entries_kernel (all pairs, any alignment): one thread per (agent,
// pair) entry, in agent order, as tera_partition emitted them, each record
// one 64-byte store to its place.
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
                        u64 arena_units, u32 class_id, DevStatus* st, u64* __restrict__ rec_ids) {
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
    if (!in_bounds(st, g, pair_off[p], pair_off[p + 1])) continue;
    store_rec(arena + (g + p + 1) * kRecBytes, R);
    if (rec_ids) rec_ids[g] = R.w[0];
  }
}

// All pairs, after tera_partition of the same state: one pass over the agents
// in the classification's tiles and rounds, each warp a run of 64 consecutive
// agents, two per lane.  A lane whose agents have entries loads their eight
// columns with 16-byte loads (every warp request covers whole sectors) and
// stores each agent's record once per entry, at the record index the
// partition's sort gave the entry; the entries of a run are numbered from
// run_base[run] in agent order.
__global__ void __launch_bounds__(kClassifyThreads)
    pack_runs_kernel(SoaPtrs soa, u64 n, const int* __restrict__ owner,
                     const u32* __restrict__ mask, const u64* __restrict__ run_base, u64 n_runs,
                     const u32* __restrict__ ent_dest, const u64* __restrict__ pair_off, u64 P,
                     uint8_t* __restrict__ arena, u64 arena_units, u32 class_id, DevStatus* st,
                     u64* __restrict__ rec_ids) {
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
  // a partition that overflowed its capacity left no record indices
  if (run_base[n_runs] != E) return;
  const int lane = threadIdx.x & 31;
  const u64 tile0 = (u64)blockIdx.x * kClassifyTile;
  for (int k = 0; k < kClassifyPerThread / 2; ++k) {
    const u64 a0 = tile0 + (u64)k * (2 * kClassifyThreads) + 2u * threadIdx.x;
    const u64 first = a0 - 2u * lane;
    if (first >= n) break;  // warp-uniform
    u32 m[2] = {0u, 0u};
    if (a0 + 1 < n) {
      const uint2 mm = *reinterpret_cast<const uint2*>(mask + a0);
      m[0] = mm.x;
      m[1] = mm.y;
    } else if (a0 < n) {
      m[0] = mask[a0];
    }
    const u32 c = __popc(m[0]) + __popc(m[1]);
    const u32 inc = warp_incl_scan<u32>(c);
    u64 e = run_base[first / kRunAgents] + (inc - c);
    if (!(m[0] | m[1])) continue;
    u64 v[8][2];
    int o[2];
    if (a0 + 1 < n) {
      const int2 oo = *reinterpret_cast<const int2*>(owner + a0);
      o[0] = oo.x;
      o[1] = oo.y;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(soa.col[w] + a0);
        v[w][0] = t.x;
        v[w][1] = t.y;
      }
    } else {
      o[0] = owner[a0];
      o[1] = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        v[w][0] = soa.col[w][a0];
        v[w][1] = 0ull;
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      Rec R;
#pragma unroll
      for (int w = 0; w < 8; ++w) R.w[w] = v[w][q];
      for (u32 mm = m[q]; mm; mm &= mm - 1) {
        const u64 p = (u64)o[q] * 27u + (u64)(__ffs(mm) - 1);
        const u64 g = ent_dest[e];
        if (in_bounds(st, g, pair_off[p], pair_off[p + 1])) {
          store_rec(arena + (g + p + 1) * kRecBytes, R);
          if (rec_ids) rec_ids[g] = R.w[0];
        }
        ++e;
      }
    }
  }
}

}  // namespace

static tera_status pack_impl(tera_ctx* ctx, const tera_soa* soa, const tera_partition_out* part,
                             uint32_t pair_begin, uint32_t pair_end, uint8_t* rec_arena,
                             uint64_t arena_units, uint64_t* rec_ids, void* stream) {
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
  bool aligned = part->owner && part->mask && ((uintptr_t)part->owner & 7u) == 0 &&
                 ((uintptr_t)part->mask & 7u) == 0;
  for (int w = 0; w < 8; ++w) aligned = aligned && ((uintptr_t)p.col[w] & 15u) == 0;
  if (pair_begin == 0 && pair_end == ctx->n_pairs && aligned && ctx->pack_n == soa->n) {
    const u64 n = (u64)soa->n;
    const u64 blocks = n == 0 ? 1 : (n + kClassifyTile - 1) / kClassifyTile;
    const u64 runs = n == 0 ? 1 : (n + kRunAgents - 1) / kRunAgents;
    prof_begin(ctx, s);
    pack_runs_kernel<<<(unsigned)blocks, kClassifyThreads, 0, s>>>(
        p, n, part->owner, part->mask, ctx->tile_base, runs, ctx->ent_dest,
        reinterpret_cast<const u64*>(part->pair_off), ctx->n_pairs, rec_arena, arena_units,
        ctx->class_id, ctx->d_status, reinterpret_cast<u64*>(rec_ids));
    return check_launch(ctx, "pack_runs_kernel", s);
  }
  if (pair_begin == 0 && pair_end == ctx->n_pairs) {
    prof_begin(ctx, s);
    pack_entries_kernel<<<(unsigned)grid_for(ctx, 8), 256, 0, s>>>(
        p, ctx->keys_a, ctx->ent_agent, ctx->ent_dest,
        reinterpret_cast<const u64*>(part->pair_off), ctx->n_pairs, rec_arena, arena_units,
        ctx->class_id, ctx->d_status, reinterpret_cast<u64*>(rec_ids));
    return check_launch(ctx, "pack_entries_kernel", s);
  }
  if (rec_ids) return TERA_EINVAL;  // the id column is written for all pairs only
  prof_begin(ctx, s);
  pack_kernel<<<blocks, 256, 0, s>>>(p, part->pair_idx, reinterpret_cast<const u64*>(part->pair_off),
                                     ctx->rec_pair, pair_begin, pair_end, rec_arena, arena_units,
                                     ctx->class_id, ctx->d_status);
  return check_launch(ctx, "pack_kernel", s);
}

extern "C" tera_status tera_pack(tera_ctx* ctx, const tera_soa* soa, const tera_partition_out* part,
                                 uint32_t pair_begin, uint32_t pair_end, uint8_t* rec_arena,
                                 uint64_t arena_units, void* stream) {
  TERA_CALL_RANGE("tera_pack");
  return pack_impl(ctx, soa, part, pair_begin, pair_end, rec_arena, arena_units, nullptr, stream);
}

extern "C" tera_status tera_pack_ids(tera_ctx* ctx, const tera_soa* soa,
                                     const tera_partition_out* part, uint8_t* rec_arena,
                                     uint64_t arena_units, uint64_t* rec_ids, void* stream) {
  TERA_CALL_RANGE("tera_pack_ids");
  if (!ctx || !rec_ids || ((uintptr_t)rec_ids & 7u)) return TERA_EINVAL;
  return pack_impl(ctx, soa, part, 0, (uint32_t)ctx->n_pairs, rec_arena, arena_units, rec_ids,
                   stream);
}
