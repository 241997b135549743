// Steps a3 + a4 — difference encoding against the pair's reference and
// significant-byte packing (paper Sec. 2.3, steps B and C; the compression
// stage that follows the difference in Sec. 3.11).
//
// Work is cut into units of kCodecTile entries that never cross a pair: per
// pair, ceil(r/T) slot units (reference slots) followed by ceil(m/T) message
// units (records of the message).  Kernels, in stream order:
//   enc_setup_kernel  wire slab layout (all pairs) + unit layout (the range)
//   enc_match_kernel  slot units: find the message record with the slot's id
//                     (hash on (pair, id)), write the slot's code, sum bytes
//   enc_new_kernel    message units: records no slot matched are new; sum
//   enc_scan_kernel   one warp per pair: unit prefixes, header, padding
//   enc_emit_kernel   all units: payload bytes (staged in shared memory and
//                     stored 16 bytes at a time), codes of new records and
//                     the new sender reference
#include "tera_internal.cuh"

using namespace tera;

namespace {

enum { PI_R = 0, PI_M = 1, PI_NST = 2, PI_MODE = 3, PI_MATCHED = 4, PI_NEW = 5, PI_SLOTPAY = 6,
       PI_PAY = 7 };

// Record index (global) of the message record of pair p with this id, or
// kNoMatch; probes pair p's hash segment, comparing ids in record order.
__device__ __forceinline__ u32 seg_lookup(const u64* __restrict__ seg, const u64* __restrict__ msg_id,
                                          u32 epoch, u32 p, u64 g_lo, u64 m, u64 id) {
  const u64 base = seg_base(g_lo, p), size = seg_size(m);
  u64 i = seg_start(id, size);
  for (u64 probe = 0; probe < size; ++probe) {
    const u64 e = seg[base + i];
    if ((u32)(e >> 32) != epoch) return kNoMatch;
    const u64 g = g_lo + (u32)e;
    if (msg_id[g] == id) return (u32)g;
    i = (i + 1 == size) ? 0 : i + 1;
  }
  return kNoMatch;
}

__device__ __forceinline__ u32 rec_code(const Rec& d, u32* bytes) {
  u32 code = 0, b = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    u32 L = sig_bytes(d.w[w]);
    code |= L << (4 * w);
    b += L;
  }
  *bytes = b;
  return code;
}

__global__ void __launch_bounds__(1024)
    enc_setup_kernel(const u64* __restrict__ pair_off, const u64* __restrict__ ref_off, u64 P,
                     u32 p0, u32 p1, int mode, const uint8_t* __restrict__ reset,
                     u64* __restrict__ wire_off, u64 wire_cap, u64* __restrict__ unit_off,
                     u64* __restrict__ units_total, u64 units_cap, u64 rec_cap,
                     u64* __restrict__ info, DevStatus* st) {
  __shared__ u64 sm[33];
  u64 carry = 0;
  for (u64 b0 = 0; b0 < P; b0 += blockDim.x) {
    const u64 p = b0 + threadIdx.x;
    u64 v = 0;
    if (p < P) {
      u64 m = pair_off[p + 1] - pair_off[p];
      u64 r = ref_off ? ref_off[p + 1] - ref_off[p] : 0;
      v = round16((u64)kHdrBytes + 4 * (r + m) + (u64)kRecBytes * m);
    }
    u64 tot;
    u64 ex = block_excl_scan<u64>(v, sm, &tot);
    if (p < P) wire_off[p] = carry + ex;
    carry += tot;
  }
  bool abort = false;
  if (threadIdx.x == 0) {
    wire_off[P] = carry;
    if (carry > wire_cap) {
      latch(st, TERA_ECAPACITY);
      need(st, carry);
    }
    if (ref_off && ref_off[P] > rec_cap) {
      latch(st, TERA_ECAPACITY);
      need(st, ref_off[P]);
    }
  }
  abort = carry > wire_cap || (ref_off && ref_off[P] > rec_cap);
  const u64 npr = p1 - p0;
  carry = 0;
  for (u64 b0 = 0; b0 < npr; b0 += blockDim.x) {
    const u64 k = b0 + threadIdx.x;
    u64 v = 0;
    if (k < npr && !abort) {
      const u64 p = p0 + k;
      u64 m = pair_off[p + 1] - pair_off[p];
      // raw: the reference is ignored (mode or a reset); no reference at all
      // (first iteration) is a difference against an empty reference
      bool raw = mode == TERA_MODE_RAW || reset[p];
      u64 r = (raw || ref_off == nullptr) ? 0 : ref_off[p + 1] - ref_off[p];
      u64 nst = (r + kCodecTile - 1) / kCodecTile;
      u64* pi = info + p * 8;
      pi[PI_R] = r;
      pi[PI_M] = m;
      pi[PI_NST] = nst;
      pi[PI_MODE] = raw ? TERA_MODE_RAW : TERA_MODE_XOR;
      v = nst + (m + kCodecTile - 1) / kCodecTile;
    }
    u64 tot;
    u64 ex = block_excl_scan<u64>(v, sm, &tot);
    if (k < npr) unit_off[k] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    unit_off[npr] = carry;
    const bool over = carry > units_cap;  // cannot happen: scratch is sized for it
    if (over) latch(st, TERA_ECAPACITY);
    units_total[0] = (abort || over) ? 0 : carry;
    units_total[1] = (abort || over) ? 1 : 0;
  }
}

struct EncArgs {
  const uint8_t* rec;      // packed messages
  const u64* pair_off;
  const uint8_t* ref;      // sender reference (may be null)
  const u64* ref_off;
  uint8_t* ref_next;
  uint8_t* wire;
  const u64* wire_off;
  u64* wire_len;
  const u64* unit_off;
  const u64* units_total;
  const u32* unit_pair;
  U64x2* unit_sum;
  U64x2* unit_base;
  u64* info;
  u32* slot_src;
  u32* matched;
  uint8_t* reset;
  u64* seg;
  const u64* msg_id;
  const u32* epoch;
  u32 p0, p1;
  u32 class_id;
  DevStatus* st;
  DevStats* stats;
};

__device__ __forceinline__ void locate(const EncArgs& A, u64 U, u32* p, u64* local) {
  *p = A.unit_pair[U];
  *local = U - A.unit_off[*p - A.p0];
}

// Message units: index every record of the pair by id in the pair's segment.
__global__ void __launch_bounds__(kCodecTile) enc_build_kernel(EncArgs A) {
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    const u64* pi = A.info + (u64)p * 8;
    const u64 nst = pi[PI_NST];
    if (local < nst) continue;  // slot unit
    const u64 m = pi[PI_M];
    const u64 k = (local - nst) * kCodecTile + threadIdx.x;
    if (k >= m) continue;
    const u64 g_lo = A.pair_off[p];
    const u64 id = A.msg_id[g_lo + k];
    const u64 base = seg_base(g_lo, p), size = seg_size(m);
    const u64 mine = ((u64)epoch << 32) | k;
    u64 i = seg_start(id, size);
    for (u64 probe = 0; probe < size; ++probe) {
      u64 cur = A.seg[base + i];
      bool done = false;
      while ((u32)(cur >> 32) != epoch) {  // empty for this iteration: claim it
        const u64 prev = atomicCAS(&A.seg[base + i], cur, mine);
        if (prev == cur) {
          done = true;
          break;
        }
        cur = prev;
      }
      if (done) break;
      i = (i + 1 == size) ? 0 : i + 1;
    }
  }
}

__global__ void __launch_bounds__(kCodecTile) enc_match_kernel(EncArgs A) {
  __shared__ U64x2 sm[33];
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    const u64* pi = A.info + (u64)p * 8;
    if (local >= pi[PI_NST]) continue;  // message unit (block-uniform)
    const u64 r = pi[PI_R];
    const u64 j = local * kCodecTile + threadIdx.x;
    U64x2 v{0, 0};
    if (j < r) {
      const u64 g_lo = A.pair_off[p];
      const Rec R = load_rec(A.ref + (A.ref_off[p] + p + 1 + j) * kRecBytes);
      u32 g = seg_lookup(A.seg, A.msg_id, epoch, p, g_lo, pi[PI_M], R.w[0]);
      u32 code;
      if (g != kNoMatch) {
        if (atomicExch(&A.matched[g], epoch) == epoch) latch(A.st, TERA_EINVAL);  // duplicate id
        const Rec M = load_rec(A.rec + ((u64)g + p + 1) * kRecBytes);
        Rec d;
#pragma unroll
        for (int w = 0; w < 8; ++w) d.w[w] = M.w[w] ^ R.w[w];
        u32 b;
        code = rec_code(d, &b);
        v = U64x2{b, 1};
      } else {
        code = 0xFu;  // placeholder
      }
      A.slot_src[A.ref_off[p] + j] = g;
      reinterpret_cast<u32*>(A.wire + A.wire_off[p] + kHdrBytes)[j] = code;
    }
    U64x2 tot;
    block_excl_scan2(v, sm, &tot);
    if (threadIdx.x == 0) A.unit_sum[U] = tot;
  }
}

__global__ void __launch_bounds__(kCodecTile) enc_new_kernel(EncArgs A) {
  __shared__ U64x2 sm[33];
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    const u64* pi = A.info + (u64)p * 8;
    const u64 nst = pi[PI_NST];
    if (local < nst) continue;  // slot unit
    const u64 m = pi[PI_M];
    const u64 k = (local - nst) * kCodecTile + threadIdx.x;
    U64x2 v{0, 0};
    if (k < m) {
      const u64 g = A.pair_off[p] + k;
      if (A.matched[g] != epoch) {
        const Rec M = load_rec(A.rec + (g + p + 1) * kRecBytes);
        // a second record with the same id in this pair would be found instead of this one
        if (seg_lookup(A.seg, A.msg_id, epoch, p, A.pair_off[p], m, M.w[0]) != (u32)g)
          latch(A.st, TERA_EINVAL);
        u32 b;
        rec_code(M, &b);
        v = U64x2{b, 1};
      }
    }
    U64x2 tot;
    block_excl_scan2(v, sm, &tot);
    if (threadIdx.x == 0) A.unit_sum[U] = tot;
  }
}

// One warp per pair of the range.
__global__ void enc_scan_kernel(EncArgs A) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  if (A.units_total[1]) return;  // capacity exceeded: write nothing
  for (u64 k = warp; k < (u64)(A.p1 - A.p0); k += nwarps) {
    const u32 p = A.p0 + (u32)k;
    u64* pi = A.info + (u64)p * 8;
    const u64 u0 = A.unit_off[k], u1 = A.unit_off[k + 1];
    const u64 nst = pi[PI_NST];
    const u64 r = pi[PI_R], m = pi[PI_M];
    // slot units
    U64x2 run{0, 0};
    for (u64 b = 0; b < nst; b += 32) {
      u64 i = b + lane;
      U64x2 v = i < nst ? A.unit_sum[u0 + i] : U64x2{0, 0};
      U64x2 incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        U64x2 t = shfl_up(incl, o);
        if (lane >= o) incl += t;
      }
      if (i < nst) A.unit_base[u0 + i] = run + incl - v;
      run += U64x2{__shfl_sync(0xFFFFFFFFu, incl.a, 31), __shfl_sync(0xFFFFFFFFu, incl.b, 31)};
    }
    const u64 slot_pay = run.a, matched = run.b;
    U64x2 run2{0, 0};
    const u64 nmt = (u1 - u0) - nst;
    for (u64 b = 0; b < nmt; b += 32) {
      u64 i = b + lane;
      U64x2 v = i < nmt ? A.unit_sum[u0 + nst + i] : U64x2{0, 0};
      U64x2 incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        U64x2 t = shfl_up(incl, o);
        if (lane >= o) incl += t;
      }
      if (i < nmt) {
        U64x2 ex = run2 + incl - v;
        A.unit_base[u0 + nst + i] = U64x2{slot_pay + ex.a, ex.b};
      }
      run2 += U64x2{__shfl_sync(0xFFFFFFFFu, incl.a, 31), __shfl_sync(0xFFFFFFFFu, incl.b, 31)};
    }
    const u64 n_new = run2.b, payload = slot_pay + run2.a;
    const u64 body = (u64)kHdrBytes + 4 * (r + n_new) + payload;
    const u64 msg = round16(body);
    uint8_t* w = A.wire + A.wire_off[p];
    if (lane == 0) {
      if (matched + n_new != m) latch(A.st, TERA_EINVAL);
      pi[PI_MATCHED] = matched;
      pi[PI_NEW] = n_new;
      pi[PI_SLOTPAY] = slot_pay;
      pi[PI_PAY] = payload;
      ulonglong2* h = reinterpret_cast<ulonglong2*>(w);
      h[0] = make_ulonglong2((u64)kWireMagic | ((u64)kVersion << 32) | ((u64)kRecBytes << 48),
                             (u64)A.class_id | (pi[PI_MODE] << 32));
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
    if (body + lane < msg) w[body + lane] = 0;  // zero padding (< 16 bytes)
  }
}

__device__ __forceinline__ void stage_word(uint8_t* stage, u32& o, u64 v, u32 L) {
  for (u32 b = 0; b < L; ++b) stage[o++] = (uint8_t)(v >> (8 * b));
}

__device__ __forceinline__ void flush_stage(const uint8_t* stage, uint8_t* gA, u64 nbytes) {
  const u32 s0 = (u32)((uintptr_t)gA & 15u);
  uint8_t* g16 = gA - s0;
  const u32 end = s0 + (u32)nbytes;
  const u32 nchunks = (end + 15u) >> 4;
  for (u32 c = threadIdx.x; c < nchunks; c += blockDim.x) {
    const u32 lo = c << 4, hi = lo + 16u;
    if (lo >= s0 && hi <= end) {
      *reinterpret_cast<uint4*>(g16 + lo) = *reinterpret_cast<const uint4*>(stage + lo);
    } else {
      for (u32 x = (lo > s0 ? lo : s0); x < (hi < end ? hi : end); ++x) g16[x] = stage[x];
    }
  }
}

__global__ void __launch_bounds__(kCodecTile) enc_emit_kernel(EncArgs A) {
  __shared__ U64x2 sm[33];
  __shared__ __align__(16) uint8_t stage[kCodecTile * kRecBytes + 32];
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    const u64* pi = A.info + (u64)p * 8;
    const u64 nst = pi[PI_NST], r = pi[PI_R], n_new = pi[PI_NEW];
    const bool slot_unit = local < nst;
    const u64 e = slot_unit ? local * kCodecTile + threadIdx.x
                            : (local - nst) * kCodecTile + threadIdx.x;
    Rec d, cur;
    u32 L[8];
    U64x2 v{0, 0};
    u64 g = 0;
    if (slot_unit) {
      if (e < r) {
        u32 gg = A.slot_src[A.ref_off[p] + e];
        if (gg != kNoMatch) {
          g = gg;
          cur = load_rec(A.rec + (g + p + 1) * kRecBytes);
          const Rec R = load_rec(A.ref + (A.ref_off[p] + p + 1 + e) * kRecBytes);
          u32 b = 0;
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            d.w[w] = cur.w[w] ^ R.w[w];
            L[w] = sig_bytes(d.w[w]);
            b += L[w];
          }
          v = U64x2{b, 1};
        }
      }
    } else if (e < pi[PI_M]) {
      g = A.pair_off[p] + e;
      if (A.matched[g] != epoch) {
        cur = load_rec(A.rec + (g + p + 1) * kRecBytes);
        u32 b = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          d.w[w] = cur.w[w];
          L[w] = sig_bytes(d.w[w]);
          b += L[w];
        }
        v = U64x2{b, 1};
      }
    }
    U64x2 tot;
    U64x2 ex = block_excl_scan2(v, sm, &tot);
    const U64x2 base = A.unit_base[U];
    uint8_t* w8 = A.wire + A.wire_off[p];
    uint8_t* gA = w8 + kHdrBytes + 4 * (r + n_new) + base.a;
    const u32 s0 = (u32)((uintptr_t)gA & 15u);
    if (v.b) {
      u32 o = s0 + (u32)ex.a;
#pragma unroll
      for (int w = 0; w < 8; ++w) stage_word(stage, o, d.w[w], L[w]);
      u64 pos;
      if (slot_unit) {
        pos = base.b + ex.b;
      } else {
        const u64 rank = base.b + ex.b;
        u32 code = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) code |= L[w] << (4 * w);
        reinterpret_cast<u32*>(w8 + kHdrBytes)[r + rank] = code;
        pos = pi[PI_MATCHED] + rank;
      }
      store_rec(A.ref_next + (A.pair_off[p] + p + 1 + pos) * kRecBytes, cur);
    }
    __syncthreads();
    flush_stage(stage, gA, tot.a);
    __syncthreads();
  }
}

}  // namespace

extern "C" tera_status tera_delta_encode(tera_ctx* ctx, const uint8_t* rec_arena,
                                         const uint64_t* pair_off, const uint8_t* ref_prev,
                                         const uint64_t* ref_off_prev, uint32_t pair_begin,
                                         uint32_t pair_end, uint8_t* ref_next, uint8_t* wire,
                                         uint64_t wire_capacity, uint64_t* wire_off,
                                         uint64_t* wire_len, int mode, void* stream) {
  if (!ctx || !rec_arena || !pair_off || !ref_next || !wire || !wire_off || !wire_len)
    return TERA_EINVAL;
  if ((ref_prev == nullptr) != (ref_off_prev == nullptr)) return TERA_EINVAL;
  if (pair_begin > pair_end || pair_end > ctx->n_pairs) return TERA_EINVAL;
  if (mode != TERA_MODE_RAW && mode != TERA_MODE_XOR) return TERA_EINVAL;
  if (((uintptr_t)rec_arena | (uintptr_t)ref_next | (uintptr_t)wire |
       (uintptr_t)(ref_prev ? ref_prev : rec_arena)) & 15u)
    return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  tera_status st = ensure_records(ctx, ctx->cap_records, s);
  if (st != TERA_OK) return st;
  const u64 P = ctx->n_pairs;
  if ((st = ensure_units(ctx, 2 * (ctx->cap_records / kCodecTile) + 2 * P + 16, s)) != TERA_OK)
    return st;
  EncArgs A;
  A.rec = rec_arena;
  A.pair_off = reinterpret_cast<const u64*>(pair_off);
  A.ref = ref_prev;
  A.ref_off = reinterpret_cast<const u64*>(ref_off_prev);
  A.ref_next = ref_next;
  A.wire = wire;
  A.wire_off = reinterpret_cast<const u64*>(wire_off);
  A.wire_len = reinterpret_cast<u64*>(wire_len);
  A.unit_off = ctx->unit_off;
  A.units_total = ctx->d_units_total;
  A.unit_pair = ctx->unit_pair;
  A.unit_sum = ctx->unit_sum;
  A.unit_base = ctx->unit_base;
  A.info = ctx->pair_info;
  A.slot_src = ctx->slot_src;
  A.matched = ctx->matched;
  A.reset = ctx->d_reset;
  A.seg = ctx->seg;
  A.msg_id = ctx->msg_id;
  A.epoch = ctx->d_epoch;
  A.p0 = pair_begin;
  A.p1 = pair_end;
  A.class_id = ctx->class_id;
  A.st = ctx->d_status;
  A.stats = ctx->d_stats;
  prof_begin(ctx, s);
  enc_setup_kernel<<<1, 1024, 0, s>>>(A.pair_off, A.ref_off, P, pair_begin, pair_end, mode,
                                      ctx->d_reset, reinterpret_cast<u64*>(wire_off),
                                      wire_capacity, ctx->unit_off, ctx->d_units_total,
                                      ctx->cap_units, ctx->cap_records, ctx->pair_info,
                                      ctx->d_status);
  if ((st = check_launch(ctx, "enc_setup_kernel", s)) != TERA_OK) return st;
  if (pair_begin == pair_end) return TERA_OK;
  if ((st = launch_unit_map(ctx, pair_begin, pair_end - pair_begin, s)) != TERA_OK) return st;
  const u64 est_units = 2 * (ctx->cap_records / kCodecTile) + 2 * (u64)(pair_end - pair_begin) + 1;
  const u64 maxg = (u64)grid_for(ctx, 8);
  const unsigned g = (unsigned)(est_units < maxg ? est_units : maxg);
  prof_begin(ctx, s);
  enc_build_kernel<<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_build_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  enc_match_kernel<<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_match_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  enc_new_kernel<<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_new_kernel", s)) != TERA_OK) return st;
  const u64 npr = pair_end - pair_begin;
  prof_begin(ctx, s);
  enc_scan_kernel<<<(unsigned)((npr + 7) / 8), 256, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_scan_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  enc_emit_kernel<<<g, kCodecTile, 0, s>>>(A);
  return check_launch(ctx, "enc_emit_kernel", s);
}
