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
#include "codec.cuh"

using namespace tera;

namespace {

__global__ void __launch_bounds__(1024)
    enc_setup_kernel(const u64* __restrict__ pair_off, const u64* __restrict__ ref_off, u64 P,
                     u32 p0, u32 p1, int mode, const uint8_t* __restrict__ reset,
                     u64* __restrict__ wire_off, u64 wire_cap, u64* __restrict__ unit_off,
                     u64* __restrict__ units_total, u64 units_cap, u64 rec_cap,
                     u64* __restrict__ info, DevStatus* st, u32* epoch) {
  __shared__ u64 sm[33];
  if (threadIdx.x == 0) {
    // a new epoch for this call's hash segments and matched flags
    const u32 ep = *epoch + 1u;
    *epoch = ep == 0u ? 1u : ep;
  }
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

__device__ __forceinline__ void locate(const EncArgs& A, u64 U, u32* p, u64* local) {
  *p = A.unit_pair[U];
  *local = U - A.unit_off[*p - A.p0];
}

__global__ void __launch_bounds__(kCodecTile) enc_build_kernel(EncArgs A) {
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    if (local < A.info[(u64)p * 8 + PI_NST]) continue;  // slot unit
    enc_build_unit<kCodecTile, false>(A, p, local, epoch);
  }
}

// Slot units: count every reference record in its cell (predictor only).
__global__ void __launch_bounds__(kCodecTile) enc_cells_kernel(EncArgs A) {
  const u64 units = *A.units_total;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    const u64* pi = A.info + (u64)p * 8;
    if (local >= pi[PI_NST]) continue;  // message unit
    cells_unit(A.pr, A.ref, A.ref_off, p, local, pi[PI_R], kCodecTile);
  }
}

template <bool PR>
__global__ void __launch_bounds__(kCodecTile) enc_match_kernel(EncArgs A) {
  __shared__ U64x2 sm[33];
  __shared__ float sW[PR ? kMlpParams : 1];
  if (PR && A.pr.params) load_mlp(sW, A.pr.params);
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    if (local >= A.info[(u64)p * 8 + PI_NST]) continue;  // message unit (block-uniform)
    enc_match_unit<kCodecTile, false, PR>(A, p, local, U, epoch, sm, sW);
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
    if (local < A.info[(u64)p * 8 + PI_NST]) continue;  // slot unit
    enc_new_unit<kCodecTile, false>(A, p, local, U, epoch, sm);
  }
}

// One warp per pair of the range.
template <bool PR>
__global__ void enc_scan_kernel(EncArgs A) {
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  if (A.units_total[1]) return;  // capacity exceeded: write nothing
  for (u64 k = warp; k < (u64)(A.p1 - A.p0); k += nwarps)
    enc_scan_pair<false, PR>(A, A.p0 + (u32)k, A.unit_off[k], A.unit_off[k + 1] - A.unit_off[k]);
}

template <bool PR>
__global__ void __launch_bounds__(kCodecTile) enc_emit_kernel(EncArgs A) {
  __shared__ U64x2 sm[33];
  __shared__ __align__(16) uint8_t stage[kCodecTile * kRecBytes + 32];
  const u64 units = *A.units_total;
  const u32 epoch = *A.epoch;
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    enc_emit_unit<kCodecTile, false, PR>(A, p, local, U, epoch, sm, stage);
  }
}

}  // namespace

static tera_status encode_impl(tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off,
                               const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                               uint32_t pair_begin, uint32_t pair_end, uint8_t* ref_next,
                               uint8_t* wire, uint64_t wire_capacity, uint64_t* wire_off,
                               uint64_t* wire_len, int mode, const tera_predictor* pred,
                               void* stream) {
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
  A.epoch = ctx->d_epoch;
  A.p0 = pair_begin;
  A.p1 = pair_end;
  A.class_id = ctx->class_id;
  A.st = ctx->d_status;
  A.stats = ctx->d_stats;
  const bool PR = pred != nullptr;
  if (PR) {
    if ((st = ensure_pred(ctx)) != TERA_OK) return st;
    if (pred->params && ((uintptr_t)pred->params & 3u)) return TERA_EINVAL;
    if (((uintptr_t)pred->hist_prev | (uintptr_t)pred->hist_next) & 15u) return TERA_EINVAL;
    if (pred->hist_prev && !ref_prev) return TERA_EINVAL;
    fill_pred(ctx, &A.pr, pred, ctx->cseg_enc);
    A.pr.hist = ref_prev ? pred->hist_prev : nullptr;
    A.pr.samples = pred->samples;
    A.pr.allow_residual = pred->allow_residual;
    if (A.pr.hist) {
      const u64 cwords = 2 * (2 * ctx->cap_records + 2 * P);
      cudaMemsetAsync(ctx->cseg_enc, 0, sizeof(u64) * cwords, s);
    }
  }
  prof_begin(ctx, s);
  enc_setup_kernel<<<1, 1024, 0, s>>>(A.pair_off, A.ref_off, P, pair_begin, pair_end, mode,
                                      ctx->d_reset, reinterpret_cast<u64*>(wire_off),
                                      wire_capacity, ctx->unit_off, ctx->d_units_total,
                                      ctx->cap_units, ctx->cap_records, ctx->pair_info,
                                      ctx->d_status, ctx->d_epoch);
  if ((st = check_launch(ctx, "enc_setup_kernel", s)) != TERA_OK) return st;
  if (pair_begin == pair_end) return TERA_OK;
  if ((st = launch_unit_map(ctx, pair_begin, pair_end - pair_begin, s)) != TERA_OK) return st;
  const u64 est_units = 2 * (ctx->cap_records / kCodecTile) + 2 * (u64)(pair_end - pair_begin) + 1;
  const u64 maxg = (u64)grid_for(ctx, 8);
  const unsigned g = (unsigned)(est_units < maxg ? est_units : maxg);
  prof_begin(ctx, s);
  enc_build_kernel<<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_build_kernel", s)) != TERA_OK) return st;
  if (PR && A.pr.hist) {
    prof_begin(ctx, s);
    enc_cells_kernel<<<g, kCodecTile, 0, s>>>(A);
    if ((st = check_launch(ctx, "enc_cells_kernel", s)) != TERA_OK) return st;
  }
  prof_begin(ctx, s);
  if (PR) enc_match_kernel<true><<<g, kCodecTile, 0, s>>>(A);
  else enc_match_kernel<false><<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_match_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  enc_new_kernel<<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_new_kernel", s)) != TERA_OK) return st;
  const u64 npr = pair_end - pair_begin;
  prof_begin(ctx, s);
  if (PR) enc_scan_kernel<true><<<(unsigned)((npr + 7) / 8), 256, 0, s>>>(A);
  else enc_scan_kernel<false><<<(unsigned)((npr + 7) / 8), 256, 0, s>>>(A);
  if ((st = check_launch(ctx, "enc_scan_kernel", s)) != TERA_OK) return st;
  prof_begin(ctx, s);
  if (PR) enc_emit_kernel<true><<<g, kCodecTile, 0, s>>>(A);
  else enc_emit_kernel<false><<<g, kCodecTile, 0, s>>>(A);
  return check_launch(ctx, "enc_emit_kernel", s);
}

extern "C" tera_status tera_delta_encode(tera_ctx* ctx, const uint8_t* rec_arena,
                                         const uint64_t* pair_off, const uint8_t* ref_prev,
                                         const uint64_t* ref_off_prev, uint32_t pair_begin,
                                         uint32_t pair_end, uint8_t* ref_next, uint8_t* wire,
                                         uint64_t wire_capacity, uint64_t* wire_off,
                                         uint64_t* wire_len, int mode, void* stream) {
  TERA_CALL_RANGE("tera_delta_encode");
  return encode_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, pair_begin, pair_end,
                     ref_next, wire, wire_capacity, wire_off, wire_len, mode, nullptr, stream);
}

extern "C" tera_status tera_delta_encode_pred(tera_ctx* ctx, const uint8_t* rec_arena,
                                              const uint64_t* pair_off, const uint8_t* ref_prev,
                                              const uint64_t* ref_off_prev, uint32_t pair_begin,
                                              uint32_t pair_end, uint8_t* ref_next,
                                              uint8_t* wire, uint64_t wire_capacity,
                                              uint64_t* wire_off, uint64_t* wire_len, int mode,
                                              const tera_predictor* pred, void* stream) {
  TERA_CALL_RANGE("tera_delta_encode_pred");
  if (!pred) return TERA_EINVAL;
  return encode_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, pair_begin, pair_end,
                     ref_next, wire, wire_capacity, wire_off, wire_len, mode, pred, stream);
}
