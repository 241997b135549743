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
#include "tera_internal.cuh"

using namespace tera;

namespace {

enum { DI_NS = 0, DI_NN = 1, DI_NH = 2, DI_PAY = 3, DI_OK = 4, DI_MODE = 5, DI_NT = 6 };

struct DecArgs {
  const uint8_t* wire;
  const u64* wire_off;
  const uint8_t* ref;
  const u64* ref_off;
  uint8_t* recv;
  u64* recv_off;
  const u64* unit_off;
  const u64* units_total;
  const u32* unit_pair;
  U64x2* unit_sum;
  U64x2* unit_base;
  u64* info;
  u32 p0, p1;
  u32 class_id;
  DevStatus* st;
};

__device__ __forceinline__ void locate(const DecArgs& A, u64 U, u32* p, u64* local) {
  *p = A.unit_pair[U];
  *local = U - A.unit_off[*p - A.p0];
}

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
      const u64 avail = A.wire_off[p + 1] - A.wire_off[p];
      const u64* h = reinterpret_cast<const u64*>(A.wire + A.wire_off[p]);
      u64* pi = A.info + (u64)p * 8;
      u32 err = 0;
      u64 ns = 0, nn = 0, nh = 0, pay = 0, mode = 0;
      if (avail < kHdrBytes) {
        err = TERA_ECORRUPT;
      } else {
        const u64 w0 = h[0], w1 = h[1];
        ns = h[2]; nn = h[3]; nh = h[4]; pay = h[5];
        const u64 w6 = h[6], msg = h[7];
        mode = w1 >> 32;
        const u64 r = A.ref ? A.ref_off[p + 1] - A.ref_off[p] : 0;
        if ((u32)w0 != kWireMagic || ((w0 >> 32) & 0xFFFF) != kVersion || (w0 >> 48) != kRecBytes ||
            (u32)w1 != A.class_id || w6 != (u64)p) {
          err = TERA_ECORRUPT;
        } else if (mode == TERA_MODE_XOR) {
          if (ns != r) err = TERA_EREFMISMATCH;
        } else if (mode == TERA_MODE_RAW) {
          if (ns != 0) err = TERA_ECORRUPT;
        } else {
          err = TERA_ECORRUPT;
        }
        if (!err) {
          if (ns > avail || nn > avail || pay > avail || nh > ns) err = TERA_ECORRUPT;
          else if (msg != round16((u64)kHdrBytes + 4 * (ns + nn) + pay) || msg > avail)
            err = TERA_ECORRUPT;
        }
        if (!err && mode == TERA_MODE_XOR && A.ref) {
          // the receiver's reference buffer must be the one this message refers to
          const u64* rh = reinterpret_cast<const u64*>(A.ref + (A.ref_off[p] + p) * kRecBytes);
          if ((u32)rh[0] != kTaioMagic || (u32)rh[1] != A.class_id || (u32)(rh[1] >> 32) != p ||
              rh[2] != r)
            err = TERA_ECORRUPT;
        }
      }
      if (err) latch(A.st, err);
      const u64 nt = err ? 0 : (ns + nn + kCodecTile - 1) / kCodecTile;
      pi[DI_NS] = ns;
      pi[DI_NN] = nn;
      pi[DI_NH] = nh;
      pi[DI_PAY] = pay;
      pi[DI_OK] = err ? 0 : 1;
      pi[DI_MODE] = mode;
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
    const bool over = ucarry > units_cap;  // cannot happen: scratch is sized for it
    if (over) latch(A.st, TERA_ECAPACITY);
    units_total[0] = (abort || over) ? 0 : ucarry;
    units_total[1] = (abort || over) ? 1 : 0;
  }
}

// Returns L_w nibbles checked: false when the code is malformed for entry e.
__device__ __forceinline__ bool check_code(u32 code, u64 e, u64 ns, bool* hole, u32* bytes) {
  *bytes = 0;
  *hole = (code & 0xFu) == 0xFu;
  if (*hole) return e < ns && (code >> 4) == 0u;
  u32 b = 0;
  bool ok = true;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    u32 L = (code >> (4 * w)) & 0xFu;
    ok &= L <= 8u;
    b += L;
  }
  if (e < ns) ok &= (code & 0xFu) == 0u;  // same id: the word-0 difference is zero
  *bytes = b;
  return ok;
}

__global__ void __launch_bounds__(kCodecTile) dec_sum_kernel(DecArgs A) {
  __shared__ U64x2 sm[33];
  const u64 units = A.units_total[0];
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    u64* pi = A.info + (u64)p * 8;
    const u64 ns = pi[DI_NS], n = ns + pi[DI_NN];
    const u64 e = local * kCodecTile + threadIdx.x;
    U64x2 v{0, 0};
    if (e < n) {
      const u32 code =
          reinterpret_cast<const u32*>(A.wire + A.wire_off[p] + kHdrBytes)[e];
      bool hole;
      u32 b;
      if (!check_code(code, e, ns, &hole, &b)) {
        latch(A.st, TERA_ECORRUPT);
        pi[DI_OK] = 0;
      }
      v = U64x2{b, hole ? 0ull : 1ull};
    }
    U64x2 tot;
    block_excl_scan2(v, sm, &tot);
    if (threadIdx.x == 0) A.unit_sum[U] = tot;
  }
}

__global__ void dec_scan_kernel(DecArgs A) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  if (A.units_total[1]) return;
  for (u64 k = warp; k < (u64)(A.p1 - A.p0); k += nwarps) {
    const u32 p = A.p0 + (u32)k;
    u64* pi = A.info + (u64)p * 8;
    const u64 u0 = A.unit_off[k], u1 = A.unit_off[k + 1];
    U64x2 run{0, 0};
    for (u64 b = 0; b < u1 - u0; b += 32) {
      u64 i = b + lane;
      U64x2 v = u0 + i < u1 ? A.unit_sum[u0 + i] : U64x2{0, 0};
      U64x2 incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        U64x2 t = shfl_up(incl, o);
        if (lane >= o) incl += t;
      }
      if (u0 + i < u1) A.unit_base[u0 + i] = run + incl - v;
      run += U64x2{__shfl_sync(0xFFFFFFFFu, incl.a, 31), __shfl_sync(0xFFFFFFFFu, incl.b, 31)};
    }
    const u64 m = A.recv_off[p + 1] - A.recv_off[p];
    if (lane == 0) {
      if (pi[DI_OK] && (run.a != pi[DI_PAY] || run.b != m)) {
        latch(A.st, TERA_ECORRUPT);
        pi[DI_OK] = 0;
      }
      write_taio_header(A.recv + (A.recv_off[p] + p) * kRecBytes, A.class_id, p, m);
    }
  }
}

__global__ void __launch_bounds__(kCodecTile) dec_emit_kernel(DecArgs A) {
  __shared__ U64x2 sm[33];
  __shared__ __align__(16) uint8_t stage[kCodecTile * kRecBytes + 48];
  const u64 units = A.units_total[0];
  for (u64 U = blockIdx.x; U < units; U += gridDim.x) {
    u32 p;
    u64 local;
    locate(A, U, &p, &local);
    const u64* pi = A.info + (u64)p * 8;
    if (!pi[DI_OK]) continue;  // block-uniform
    const u64 ns = pi[DI_NS], n = ns + pi[DI_NN];
    const u64 e = local * kCodecTile + threadIdx.x;
    const uint8_t* w8 = A.wire + A.wire_off[p];
    u32 code = 0;
    u32 b = 0;
    bool hole = true;
    if (e < n) {
      code = reinterpret_cast<const u32*>(w8 + kHdrBytes)[e];
      check_code(code, e, ns, &hole, &b);
    }
    U64x2 v{b, (e < n && !hole) ? 1ull : 0ull};
    U64x2 tot;
    U64x2 ex = block_excl_scan2(v, sm, &tot);
    const U64x2 base = A.unit_base[U];
    // stage [gA, gA + tot.a) with 16-byte loads; the slab is 16-byte aligned and
    // padded, so the rounded range stays inside this pair's slab
    const uint8_t* gA = w8 + kHdrBytes + 4 * n + base.a;
    const u32 s0 = (u32)((uintptr_t)gA & 15u);
    const uint8_t* g16 = gA - s0;
    const u32 nchunks = (u32)((s0 + tot.a + 15u) >> 4);
    for (u32 c = threadIdx.x; c < nchunks; c += blockDim.x)
      *reinterpret_cast<uint4*>(stage + (c << 4)) = *reinterpret_cast<const uint4*>(g16 + (c << 4));
    __syncthreads();
    if (v.b) {
      u32 o = s0 + (u32)ex.a;
      Rec rec;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const u32 L = (code >> (4 * w)) & 0xFu;
        u64 x = 0;
        for (u32 q = 0; q < L; ++q) x |= (u64)stage[o + q] << (8 * q);
        o += L;
        rec.w[w] = x;
      }
      if (e < ns) {
        const Rec R = load_rec(A.ref + (A.ref_off[p] + p + 1 + e) * kRecBytes);
#pragma unroll
        for (int w = 0; w < 8; ++w) rec.w[w] ^= R.w[w];
      }
      const u64 pos = base.b + ex.b;
      store_rec(A.recv + (A.recv_off[p] + p + 1 + pos) * kRecBytes, rec);
    }
    __syncthreads();
  }
}

}  // namespace

#ifndef TERA_DECODE_KERNELS_ONLY
extern "C" tera_status tera_delta_decode(tera_ctx* ctx, const uint8_t* wire,
                                         const uint64_t* wire_off, const uint8_t* ref_prev,
                                         const uint64_t* ref_off_prev, uint32_t pair_begin,
                                         uint32_t pair_end, uint8_t* recv,
                                         uint64_t recv_capacity_units, uint64_t* recv_off,
                                         void* stream) {
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
  prof_begin(ctx, s);
  dec_setup_kernel<<<1, 1024, 0, s>>>(A, P, recv_capacity_units, ctx->d_units_total,
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
  prof_begin(ctx, s);
  dec_emit_kernel<<<g, kCodecTile, 0, s>>>(A);
  return check_launch(ctx, "dec_emit_kernel", s);
}
#endif  // TERA_DECODE_KERNELS_ONLY
