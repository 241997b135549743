// Step a5 — restore and defragment (paper Sec. 2.3, step D): the receiver
// rebuilds every record from its reference and the received difference, drops
// the placeholders, and hands the defragmented buffer (which is also its next
// reference) to higher-level code; the original order is not restored.
//
// Kernels, in stream order:
//   dec_setup_kernel  receive layout from ALL headers (m_p = n_slots - n_holes
//                     + n_new), full header checks and unit layout for the range
//   dec_sum_kernel    units of kCodecTile codes: check nibbles, sum bytes and
//                     non-placeholders
//   dec_scan_kernel   one warp per pair: unit prefixes, totals checked against
//                     the header, receive-buffer header
//   dec_emit_kernel   payload tile staged in shared memory with 16-byte loads,
//                     words rebuilt, XOR with the reference slot, record written
#include "codec.cuh"

using namespace tera;

namespace {

__device__ __forceinline__ void locate(const DecArgs& A, u64 U, u32* p, u64* local) {
  *p = A.unit_pair[U];
  *local = U - A.unit_off[*p - A.p0];
}

template <bool PR>
__global__ void __launch_bounds__(1024) dec_setup_kernel(DecArgs A, u64 P, u64 recv_cap,
                                                         u64* __restrict__ units_total,
                                                         u64 units_cap) {
  __shared__ u64 sm[33];
  u64 carry = 0;
  for (u64 b0 = 0; b0 < P; b0 += blockDim.x) {
    const u64 p = b0 + threadIdx.x;
    u64 m = 0;
    if (p < P) {
      const u64 avail = A.wire_off[p + 1] - A.wire_off[p];
      const u64* h = reinterpret_cast<const u64*>(A.wire + A.wire_off[p]);
      if (avail >= kHdrBytes && (u32)h[0] == kWireMagic) {
        u64 ns = h[2], nn = h[3], nh = h[4];
        if (nh <= ns && ns <= avail && nn <= avail) m = ns - nh + nn;
      }
    }
    u64 tot;
    u64 ex = block_excl_scan<u64>(m, sm, &tot);
    if (p < P) A.recv_off[p] = carry + ex;
    carry += tot;
  }
  const bool abort = carry + P > recv_cap;
  if (threadIdx.x == 0) {
    A.recv_off[P] = carry;
    if (abort) {
      latch(A.st, TERA_ECAPACITY);
      need(A.st, carry + P);
    }
  }
  const u64 npr = A.p1 - A.p0;
  u64 ucarry = 0;
  for (u64 b0 = 0; b0 < npr; b0 += blockDim.x) {
    const u64 k = b0 + threadIdx.x;
    u64 v = 0;
    if (k < npr && !abort) {
      const u32 p = A.p0 + (u32)k;
      const u32 err = dec_check_header<false, PR>(A, p, ~0ull);
      if (err) latch(A.st, err);
      u64* pi = A.info + (u64)p * 8;
      const u64 nt = err ? 0 : (pi[DI_NS] + pi[DI_NN] + kCodecTile - 1) / kCodecTile;
      pi[DI_NT] = nt;
      v = nt;
    }
    u64 tot;
    u64 ex = block_excl_scan<u64>(v, sm, &tot);
    if (k < npr) const_cast<u64*>(A.unit_off)[k] = ucarry + ex;
    ucarry += tot;
  }
  if (threadIdx.x == 0) {
    const_cast<u64*>(A.unit_off)[npr] = ucarry;
    // a context's scratch is sized for every tile; the fixed scratch of
    // tera_delta_decode_noalloc can overflow: TERA_ECAPACITY with no required
    // capacity recorded (no receive capacity would help)
    const bool over = ucarry > units_cap;
    if (over) latch(A.st, TERA_ECAPACITY);
    units_total[0] = (abort || over) ? 0 : ucarry;
    units_total[1] = (abort || over) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kCodecTile) dec_sum_kernel(DecArgs A) {
  __shared__ U64x2 sm[33];
  const u64 units = A.units_total[0];
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    dec_sum_unit<kCodecTile, false>(A, p, local, U, sm);
  }
}

__global__ void dec_scan_kernel(DecArgs A) {
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  if (A.units_total[1]) return;
  for (u64 k = warp; k < (u64)(A.p1 - A.p0); k += nwarps)
    dec_scan_pair<false>(A, A.p0 + (u32)k, A.unit_off[k], A.unit_off[k + 1] - A.unit_off[k]);
}

template <bool PR>
__global__ void __launch_bounds__(kCodecTile) dec_emit_kernel(DecArgs A) {
  __shared__ U64x2 sm[33];
  __shared__ __align__(16) uint8_t stage[kCodecTile * kRecBytes + 48];
  __shared__ float sW[PR ? kMlpParams : 1];
  if (PR && A.pr.params) load_mlp(sW, A.pr.params);
  const u64 units = A.units_total[0];
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    dec_emit_unit<kCodecTile, false, PR>(A, p, local, U, sm, stage, sW);
  }
}

// Every record of the receiver's reference: count it in its cell (predictor).
__global__ void dec_cells_kernel(DecArgs A) {
  const u64 g0 = A.ref_off[A.p0], g1 = A.ref_off[A.p1];
  for (u64 g = g0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; g < g1;
       g += (u64)gridDim.x * blockDim.x) {
    const u32 p = upper_pair(A.ref_off, A.p0, A.p1, g);
    const u64 r = A.ref_off[p + 1] - A.ref_off[p];
    const Rec R = load_rec(A.ref + (g + p + 1) * kRecBytes);
    cell_insert(A.pr.cseg, seg_base(A.ref_off[p], p), seg_size(r), cell_key(R, A.pr));
  }
}

}  // namespace

#ifndef TERA_DECODE_KERNELS_ONLY
static tera_status decode_impl(tera_ctx* ctx, const uint8_t* wire, const uint64_t* wire_off,
                               const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                               uint32_t pair_begin, uint32_t pair_end, uint8_t* recv,
                               uint64_t recv_capacity_units, uint64_t* recv_off,
                               const tera_predictor* pred, void* stream) {
  if (!ctx || !wire || !wire_off || !recv || !recv_off) return TERA_EINVAL;
  if ((ref_prev == nullptr) != (ref_off_prev == nullptr)) return TERA_EINVAL;
  if (pair_begin > pair_end || pair_end > ctx->n_pairs) return TERA_EINVAL;
  if (((uintptr_t)wire | (uintptr_t)recv | (uintptr_t)(ref_prev ? ref_prev : recv)) & 15u)
    return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u64 P = ctx->n_pairs;
  tera_status st = ensure_records(ctx, ctx->cap_records, s);
  if (st != TERA_OK) return st;
  if ((st = ensure_units(ctx, 2 * (ctx->cap_records / kCodecTile) + 2 * P + 16, s)) != TERA_OK)
    return st;
  DecArgs A;
  A.wire = wire;
  A.wire_off = reinterpret_cast<const u64*>(wire_off);
  A.ref = ref_prev;
  A.ref_off = reinterpret_cast<const u64*>(ref_off_prev);
  A.recv = recv;
  A.recv_off = reinterpret_cast<u64*>(recv_off);
  A.unit_off = ctx->unit_off;
  A.units_total = ctx->d_units_total;
  A.unit_pair = ctx->unit_pair;
  A.unit_sum = ctx->unit_sum;
  A.unit_base = ctx->unit_base;
  A.info = ctx->pair_info;
  A.p0 = pair_begin;
  A.p1 = pair_end;
  A.class_id = ctx->class_id;
  A.st = ctx->d_status;
  const bool PR = pred != nullptr;
  if (PR) {
    if ((st = ensure_pred(ctx)) != TERA_OK) return st;
    if (pred->params && ((uintptr_t)pred->params & 3u)) return TERA_EINVAL;
    if (((uintptr_t)pred->hist_prev | (uintptr_t)pred->hist_next) & 15u) return TERA_EINVAL;
    if (pred->hist_prev && !ref_prev) return TERA_EINVAL;
    fill_pred(ctx, &A.pr, pred, ctx->cseg_dec);
    A.pr.hist = ref_prev ? pred->hist_prev : nullptr;
    if (A.pr.hist) {
      const u64 cwords = 2 * (2 * ctx->cap_records + 2 * P);
      cudaMemsetAsync(ctx->cseg_dec, 0, sizeof(u64) * cwords, s);
    }
  }
  prof_begin(ctx, s);
  if (PR)
    dec_setup_kernel<true><<<1, 1024, 0, s>>>(A, P, recv_capacity_units, ctx->d_units_total,
                                              ctx->cap_units);
  else
    dec_setup_kernel<false><<<1, 1024, 0, s>>>(A, P, recv_capacity_units, ctx->d_units_total,
                                               ctx->cap_units);
  if ((st = check_launch(ctx, "dec_setup_kernel", s)) != TERA_OK) return st;
  if (pair_begin == pair_end) return TERA_OK;
  if ((st = launch_unit_map(ctx, pair_begin, pair_end - pair_begin, s)) != TERA_OK) return st;
  const u64 est_units = 2 * (ctx->cap_records / kCodecTile) + 2 * (u64)(pair_end - pair_begin) + 1;
  const u64 maxg = (u64)grid_for(ctx, 8);
  const unsigned g = (unsigned)(est_units < maxg ? est_units : maxg);
  prof_begin(ctx, s);
  dec_sum_kernel<<<g, kCodecTile, 0, s>>>(A);
  if ((st = check_launch(ctx, "dec_sum_kernel", s)) != TERA_OK) return st;
  const u64 npr = pair_end - pair_begin;
  prof_begin(ctx, s);
  dec_scan_kernel<<<(unsigned)((npr + 7) / 8), 256, 0, s>>>(A);
  if ((st = check_launch(ctx, "dec_scan_kernel", s)) != TERA_OK) return st;
  if (PR && A.pr.hist) {
    prof_begin(ctx, s);
    dec_cells_kernel<<<g, 256, 0, s>>>(A);
    if ((st = check_launch(ctx, "dec_cells_kernel", s)) != TERA_OK) return st;
  }
  prof_begin(ctx, s);
  if (PR) dec_emit_kernel<true><<<g, kCodecTile, 0, s>>>(A);
  else dec_emit_kernel<false><<<g, kCodecTile, 0, s>>>(A);
  return check_launch(ctx, "dec_emit_kernel", s);
}

extern "C" tera_status tera_delta_decode(tera_ctx* ctx, const uint8_t* wire,
                                         const uint64_t* wire_off, const uint8_t* ref_prev,
                                         const uint64_t* ref_off_prev, uint32_t pair_begin,
                                         uint32_t pair_end, uint8_t* recv,
                                         uint64_t recv_capacity_units, uint64_t* recv_off,
                                         void* stream) {
  TERA_CALL_RANGE("tera_delta_decode");
  return decode_impl(ctx, wire, wire_off, ref_prev, ref_off_prev, pair_begin, pair_end, recv,
                     recv_capacity_units, recv_off, nullptr, stream);
}

extern "C" tera_status tera_delta_decode_pred(tera_ctx* ctx, const uint8_t* wire,
                                              const uint64_t* wire_off, const uint8_t* ref_prev,
                                              const uint64_t* ref_off_prev, uint32_t pair_begin,
                                              uint32_t pair_end, uint8_t* recv,
                                              uint64_t recv_capacity_units, uint64_t* recv_off,
                                              const tera_predictor* pred, void* stream) {
  TERA_CALL_RANGE("tera_delta_decode_pred");
  if (!pred) return TERA_EINVAL;
  return decode_impl(ctx, wire, wire_off, ref_prev, ref_off_prev, pair_begin, pair_end, recv,
                     recv_capacity_units, recv_off, pred, stream);
}
#endif  // TERA_DECODE_KERNELS_ONLY
