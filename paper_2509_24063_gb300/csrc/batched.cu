// Batched codec: steps a3-a5 (paper Sec. 2.3, steps B, C and D) for every
// pair of one iteration in ONE persistent launch over a work list.
//
// The work list holds (phase, pair, tile) items.  Pairs are taken in windows
// of W pairs; inside a window the items are ordered phase by phase, so a
// window's pairs move through build -> match -> new -> scan -> emit ->
// decode-setup -> decode-sum -> decode-scan -> decode-emit while their data
// is still in L2.  Persistent blocks claim items in list order with one
// atomic ticket; an item first waits (bounded, with __nanosleep) until the
// items of the earlier phases of ITS pair are done.  Those items have lower
// tickets, so they were claimed by blocks that are running or finished: the
// waits always end, and a wait that exceeds its bound latches TERA_ETIMEOUT
// and stops every block instead of hanging.
//
// Tile size T (block size), blocks per SM and W come from the caller
// (tera_tune, picked by the autotuner); the bytes produced do not depend on
// them.  The receive layout is the pair layout of the iteration (every
// header's record count is checked against it).
#include "codec.cuh"

using namespace tera;

namespace {

enum { PH_BUILD = 0, PH_CELLS, PH_MATCH, PH_NEW, PH_SCAN, PH_EMIT, PH_DSETUP, PH_DSUM, PH_DSCAN,
       PH_DCELLS, PH_DEMIT, PH_COUNT };
static_assert(PH_COUNT == kBatchPhases, "phase count");

// phases an item of phase `ph` waits for (bit mask over phases of the same pair)
__device__ __forceinline__ u32 deps(int ph) {
  switch (ph) {
    case PH_MATCH: return (1u << PH_BUILD) | (1u << PH_CELLS);
    case PH_NEW: return (1u << PH_BUILD) | (1u << PH_MATCH);
    case PH_SCAN: return (1u << PH_MATCH) | (1u << PH_NEW);
    case PH_EMIT: return 1u << PH_SCAN;
    case PH_DSETUP: return (1u << PH_SCAN) | (1u << PH_EMIT);
    case PH_DSUM: return 1u << PH_DSETUP;
    case PH_DSCAN: return (1u << PH_DSETUP) | (1u << PH_DSUM);
    case PH_DEMIT: return (1u << PH_DSCAN) | (1u << PH_DCELLS);
    default: return 0u;
  }
}

struct BatchArgs {
  const u64* items;
  const u64* n_items;
  u64* ticket;
  u32* done;        // [P * PH_COUNT]
  const u32* need;  // [P * PH_COUNT]
  const u64* enc_uoff;
  const u64* dec_uoff;
  u32* abort;
};

constexpr u64 kSpinLimit = 1ull << 25;  // x ~100 ns sleeps: several seconds

__device__ __forceinline__ u32 ld_acquire(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(u32* p, u32 v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u64 make_item(u32 ph, u32 p, u32 t) {
  return ((u64)ph << 60) | ((u64)p << 32) | (u64)t;
}

// ---------------- setup: per-pair facts, layouts, capacity checks ----------------

__global__ void __launch_bounds__(1024)
    bat_setup_kernel(EncArgs E, DecArgs D, BatchArgs B, u64 P, int mode, u32 T, u32 K,
                     int enc_cells, int dec_cells,
                     u64* __restrict__ wire_off, u64 wire_cap, u64 rec_cap, u64 recv_cap,
                     u64 units_cap, u32* __restrict__ need_out, u64* __restrict__ enc_uoff,
                     u64* __restrict__ dec_uoff, u32* epoch) {
  __shared__ u64 sm[33];
  if (threadIdx.x == 0) {
    const u32 ep = *epoch + 1u;
    *epoch = ep == 0u ? 1u : ep;
  }
  u64 cw = 0, ce = 0, cd = 0;
  for (u64 b0 = 0; b0 < P; b0 += blockDim.x) {
    const u64 p = b0 + threadIdx.x;
    u64 vw = 0, ve = 0, vd = 0;
    if (p < P) {
      const u64 m = E.pair_off[p + 1] - E.pair_off[p];
      const u64 r_full = E.ref_off ? E.ref_off[p + 1] - E.ref_off[p] : 0;
      const bool raw = mode == TERA_MODE_RAW || E.reset[p];
      const u64 r = (raw || E.ref_off == nullptr) ? 0 : r_full;
      const u64 ts = (r + T - 1) / T, tm = (m + T - 1) / T, td = (r + m + T - 1) / T;
      u64* pi = E.info + p * 8;
      pi[PI_R] = r;
      pi[PI_M] = m;
      pi[PI_NST] = ts;
      pi[PI_MODE] = raw ? TERA_MODE_RAW : TERA_MODE_XOR;
      // items per phase: K tiles per item (one item for the per-pair phases)
      u32* nd = need_out + p * PH_COUNT;
      nd[PH_BUILD] = (u32)((tm + K - 1) / K);
      nd[PH_CELLS] = enc_cells ? (u32)((ts + K - 1) / K) : 0u;
      const u64 rr = D.ref_off ? D.ref_off[p + 1] - D.ref_off[p] : 0;
      nd[PH_DCELLS] = dec_cells ? (u32)(((rr + T - 1) / T + K - 1) / K) : 0u;
      nd[PH_MATCH] = (u32)((ts + K - 1) / K);
      nd[PH_NEW] = (u32)((tm + K - 1) / K);
      nd[PH_SCAN] = 1;
      nd[PH_EMIT] = (u32)((ts + tm + K - 1) / K);
      nd[PH_DSETUP] = 1;
      nd[PH_DSUM] = (u32)((td + K - 1) / K);
      nd[PH_DSCAN] = 1;
      nd[PH_DEMIT] = (u32)((td + K - 1) / K);
      vw = round16((u64)kHdrBytes + 4 * (r_full + m) + (u64)kRecBytes * m);
      ve = ts + tm;
      vd = td;
      D.recv_off[p] = E.pair_off[p];  // receive buffers sized by the record counts
    }
    u64 tw, te, td;
    const u64 xw = block_excl_scan<u64>(vw, sm, &tw);
    const u64 xe = block_excl_scan<u64>(ve, sm, &te);
    const u64 xd = block_excl_scan<u64>(vd, sm, &td);
    if (p < P) {
      wire_off[p] = cw + xw;
      enc_uoff[p] = ce + xe;
      dec_uoff[p] = cd + xd;
    }
    cw += tw;
    ce += te;
    cd += td;
  }
  if (threadIdx.x == 0) {
    wire_off[P] = cw;
    enc_uoff[P] = ce;
    dec_uoff[P] = cd;
    D.recv_off[P] = E.pair_off[P];
    bool abort = false;
    if (cw > wire_cap) {
      latch(E.st, TERA_ECAPACITY);
      need(E.st, cw);
      abort = true;
    }
    if (E.ref_off && E.ref_off[P] > rec_cap) {
      latch(E.st, TERA_ECAPACITY);
      need(E.st, E.ref_off[P]);
      abort = true;
    }
    if (E.pair_off[P] + P > recv_cap) {
      latch(E.st, TERA_ECAPACITY);
      need(E.st, E.pair_off[P] + P);
      abort = true;
    }
    if (ce > units_cap || cd > units_cap) {  // cannot happen: scratch is sized for it
      latch(E.st, TERA_ECAPACITY);
      abort = true;
    }
    *B.abort = abort ? 1u : 0u;
    *B.ticket = 0;
  }
}

// items of a window: total per window (one block of W threads per window)
__global__ void bat_window_count_kernel(const u32* __restrict__ need, u64 P, u32 W,
                                        u32* __restrict__ win_total) {
  __shared__ u64 sm[33];
  const u64 p = (u64)blockIdx.x * W + threadIdx.x;
  u64 c = 0;
  if (threadIdx.x < W && p < P)
    for (int ph = 0; ph < PH_COUNT; ++ph) c += need[p * PH_COUNT + ph];
  u64 tot;
  block_excl_scan<u64>(c, sm, &tot);
  if (threadIdx.x == 0) win_total[blockIdx.x] = (u32)tot;
}

// items of a window, phase by phase, pair by pair, tile by tile
__global__ void bat_window_fill_kernel(const u32* __restrict__ need, u64 P, u32 W,
                                       const u64* __restrict__ win_base, u64 n_windows,
                                       u64* __restrict__ items, u64* __restrict__ n_items,
                                       const u32* __restrict__ abort) {
  __shared__ u64 sm[33];
  if (*abort) {  // capacities exceeded: no work list (and no write past its end)
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_items = 0;
    return;
  }
  const u64 p = (u64)blockIdx.x * W + threadIdx.x;
  const bool live = threadIdx.x < W && p < P;
  u64 pos = win_base[blockIdx.x];
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    const u64 c = live ? need[p * PH_COUNT + ph] : 0;
    u64 tot;
    const u64 ex = block_excl_scan<u64>(c, sm, &tot);
    for (u64 t = 0; t < c; ++t) items[pos + ex + t] = make_item((u32)ph, (u32)p, (u32)t);
    pos += tot;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_items = win_base[n_windows];
}

// ---------------- the persistent kernel ----------------

__device__ __forceinline__ bool wait_deps(const BatchArgs& B, u32 p, int ph, DevStatus* st) {
  const u32 mask = deps(ph);
  for (int q = 0; q < PH_COUNT; ++q) {
    if (!((mask >> q) & 1u)) continue;
    const u32 want = B.need[(u64)p * PH_COUNT + q];
    const u32* ctr = B.done + (u64)p * PH_COUNT + q;
    u64 spin = 0;
    while (ld_acquire(ctr) < want) {
      if (*(volatile u32*)B.abort) return false;
      if (++spin > kSpinLimit) {
        latch(st, TERA_ETIMEOUT);
        atomicExch(B.abort, 1u);
        return false;
      }
      __nanosleep(100);
    }
  }
  return true;
}

// At least 1024 resident threads per SM: the codec is latency-bound.
template <int T, bool PR>
__global__ void __launch_bounds__(T, 1024 / T)
    codec_persistent_kernel(EncArgs E, DecArgs D, BatchArgs B, u32 K) {
  extern __shared__ __align__(16) uint8_t stage[];
  __shared__ U64x2 sm[33];
  __shared__ u64 s_item;
  __shared__ int s_go;
  float* sW = reinterpret_cast<float*>(stage + ((size_t)T * kRecBytes + 48));
  if (PR) {
    const float* params = E.pr.params ? E.pr.params : D.pr.params;
    if (params) load_mlp(sW, params);
  }
  const u64 n_items = __ldcg(B.n_items);
  const u32 epoch = __ldcg(E.epoch);
  for (;;) {
    if (threadIdx.x == 0) {
      s_go = 0;
      if (!*(volatile u32*)B.abort) {
        const u64 t = atomicAdd(B.ticket, 1ull);
        if (t < n_items) {
          const u64 it = B.items[t];
          s_item = it;
          s_go = wait_deps(B, (u32)(it >> 32) & 0x0FFFFFFFu, (int)(it >> 60), E.st) ? 1 : 0;
        }
      }
    }
    __syncthreads();
    if (!s_go) break;
    const u64 it = s_item;
    const int ph = (int)(it >> 60);
    const u32 p = (u32)(it >> 32) & 0x0FFFFFFFu;
    const u64 k0 = (u64)(u32)it * K;  // first tile of this item
    const u64* pi = E.info + (u64)p * 8;
    const u64 nst = pi[PI_NST];
    const u64 ntm = (pi[PI_M] + T - 1) / T;
    const u64 ntd = B.dec_uoff[p + 1] - B.dec_uoff[p];
    switch (ph) {
      case PH_BUILD:
        for (u64 t = k0; t < k0 + K && t < ntm; ++t) enc_build_unit<T, true>(E, p, nst + t, epoch);
        break;
      case PH_CELLS:
        if constexpr (PR)
          for (u64 t = k0; t < k0 + K && t < nst; ++t)
            cells_unit(E.pr, E.ref, E.ref_off, p, t, pi[PI_R], T);
        break;
      case PH_MATCH:
        for (u64 t = k0; t < k0 + K && t < nst; ++t)
          enc_match_unit<T, true, PR>(E, p, t, B.enc_uoff[p] + t, epoch, sm, sW);
        break;
      case PH_NEW:
        for (u64 t = k0; t < k0 + K && t < ntm; ++t)
          enc_new_unit<T, true>(E, p, nst + t, B.enc_uoff[p] + nst + t, epoch, sm);
        break;
      case PH_SCAN:
        if (threadIdx.x < 32)
          enc_scan_pair<true, PR>(E, p, B.enc_uoff[p], B.enc_uoff[p + 1] - B.enc_uoff[p]);
        break;
      case PH_EMIT:
        for (u64 t = k0; t < k0 + K && t < nst + ntm; ++t)
          enc_emit_unit<T, true, PR>(E, p, t, B.enc_uoff[p] + t, epoch, sm, stage);
        break;
      case PH_DSETUP:
        if (threadIdx.x == 0) {
          const u32 err = dec_check_header<true, PR>(D, p, E.pair_off[p + 1] - E.pair_off[p]);
          if (err) latch(D.st, err);
        }
        break;
      case PH_DSUM:
        for (u64 t = k0; t < k0 + K && t < ntd; ++t)
          dec_sum_unit<T, true>(D, p, t, B.dec_uoff[p] + t, sm);
        break;
      case PH_DSCAN:
        if (threadIdx.x < 32) dec_scan_pair<true>(D, p, B.dec_uoff[p], ntd);
        break;
      case PH_DCELLS:
        if constexpr (PR) {
          const u64 rr = D.ref_off[p + 1] - D.ref_off[p];
          const u64 ntr = (rr + T - 1) / T;
          for (u64 t = k0; t < k0 + K && t < ntr; ++t) cells_unit(D.pr, D.ref, D.ref_off, p, t, rr, T);
        }
        break;
      case PH_DEMIT:
        for (u64 t = k0; t < k0 + K && t < ntd; ++t)
          dec_emit_unit<T, true, PR>(D, p, t, B.dec_uoff[p] + t, sm, stage, sW);
        break;
      default: break;
    }
    // release: the barrier orders every thread's writes before thread 0's
    // release, which publishes them (with this item's count) at GPU scope
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(B.done + (u64)p * PH_COUNT + ph, 1u);
  }
}

template <int T, bool PR>
tera_status launch_persistent(tera_ctx* ctx, const EncArgs& E, const DecArgs& D,
                              const BatchArgs& B, int ctas_per_sm, u32 K, cudaStream_t s) {
  // stage (+ MLP weights): at most 36 KB, no opt-in needed
  const size_t smem = (size_t)T * kRecBytes + 48 + (PR ? sizeof(float) * kMlpParams : 0);
  const unsigned grid = (unsigned)(ctx->num_sms * (ctas_per_sm > 0 ? ctas_per_sm : 1));
  prof_begin(ctx, s);
  codec_persistent_kernel<T, PR><<<grid, T, smem, s>>>(E, D, B, K);
  return check_launch(ctx, "codec_persistent_kernel", s);
}

}  // namespace

static tera_status batched_impl(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, const tera_predictor* enc_pred,
    const tera_predictor* dec_pred, void* stream) {
  if (!ctx || !rec_arena || !pair_off || !ref_next || !wire || !wire_off || !wire_len || !recv ||
      !recv_off)
    return TERA_EINVAL;
  if ((ref_prev == nullptr) != (ref_off_prev == nullptr)) return TERA_EINVAL;
  if ((recv_prev == nullptr) != (recv_off_prev == nullptr)) return TERA_EINVAL;
  if (mode != TERA_MODE_RAW && mode != TERA_MODE_XOR) return TERA_EINVAL;
  if (((uintptr_t)rec_arena | (uintptr_t)ref_next | (uintptr_t)wire | (uintptr_t)recv |
       (uintptr_t)(ref_prev ? ref_prev : wire) | (uintptr_t)(recv_prev ? recv_prev : wire)) & 15u)
    return TERA_EINVAL;
  tera_tune tn = tune ? *tune : tera_tune{256, 4, 64, 4};
  if (enc_pred && enc_pred->params && ((uintptr_t)enc_pred->params & 3u)) return TERA_EINVAL;
  if (tn.block != 128 && tn.block != 256 && tn.block != 512) return TERA_EINVAL;
  if (tn.ctas_per_sm < 1 || tn.ctas_per_sm > 16) return TERA_EINVAL;
  if (tn.window < 1 || tn.window > 1024) return TERA_EINVAL;
  if (tn.tiles_per_item < 1 || tn.tiles_per_item > 64) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const u64 P = ctx->n_pairs;
  const bool PR = enc_pred != nullptr || dec_pred != nullptr;
  if (PR && tn.block > 256) tn.block = 256;  // stage + weights stay within 48 KB
  const u32 T = (u32)tn.block, W = (u32)tn.window, K = (u32)tn.tiles_per_item;
  tera_status st = ensure_records(ctx, ctx->cap_records, s);
  if (st != TERA_OK) return st;
  if ((st = ensure_batched(ctx, T, W)) != TERA_OK) return st;

  EncArgs E;
  E.rec = rec_arena;
  E.pair_off = reinterpret_cast<const u64*>(pair_off);
  E.ref = ref_prev;
  E.ref_off = reinterpret_cast<const u64*>(ref_off_prev);
  E.ref_next = ref_next;
  E.wire = wire;
  E.wire_off = reinterpret_cast<const u64*>(wire_off);
  E.wire_len = reinterpret_cast<u64*>(wire_len);
  E.unit_off = nullptr;
  E.units_total = nullptr;
  E.unit_pair = nullptr;
  E.unit_sum = ctx->unit_sum;
  E.unit_base = ctx->unit_base;
  E.info = ctx->pair_info;
  E.slot_src = ctx->slot_src;
  E.matched = ctx->matched;
  E.reset = ctx->d_reset;
  E.seg = ctx->seg;
  E.msg_id = ctx->msg_id;
  E.epoch = ctx->d_epoch;
  E.p0 = 0;
  E.p1 = (u32)P;
  E.class_id = ctx->class_id;
  E.st = ctx->d_status;
  E.stats = ctx->d_stats;

  DecArgs D;
  D.wire = wire;
  D.wire_off = reinterpret_cast<const u64*>(wire_off);
  D.ref = recv_prev;
  D.ref_off = reinterpret_cast<const u64*>(recv_off_prev);
  D.recv = recv;
  D.recv_off = reinterpret_cast<u64*>(recv_off);
  D.unit_off = nullptr;
  D.units_total = nullptr;
  D.unit_pair = nullptr;
  D.unit_sum = ctx->b_unit_sum;
  D.unit_base = ctx->b_unit_base;
  D.info = ctx->pair_info + 8 * P;
  D.p0 = 0;
  D.p1 = (u32)P;
  D.class_id = ctx->class_id;
  D.st = ctx->d_status;

  BatchArgs B;
  B.items = ctx->b_items;
  B.n_items = ctx->b_scalars + 0;
  B.ticket = ctx->b_scalars + 1;
  B.done = ctx->b_done;
  B.need = ctx->b_need;
  B.enc_uoff = ctx->b_enc_uoff;
  B.dec_uoff = ctx->b_dec_uoff;
  B.abort = reinterpret_cast<u32*>(ctx->b_scalars + 2);

  int enc_cells = 0, dec_cells = 0;
  if (PR) {
    if ((st = ensure_pred(ctx)) != TERA_OK) return st;
    E.pr.unit_res = ctx->unit_res;
    const u64 cwords = 2 * (2 * ctx->cap_records + 2 * P);
    if (enc_pred) {
      if ((enc_pred->hist_prev != nullptr) != (ref_prev != nullptr)) return TERA_EINVAL;
      fill_pred(ctx, &E.pr, enc_pred, ctx->cseg_enc);
      E.pr.samples = enc_pred->samples;
      E.pr.allow_residual = enc_pred->allow_residual;
      if (E.pr.hist) {
        enc_cells = 1;
        cudaMemsetAsync(ctx->cseg_enc, 0, sizeof(u64) * cwords, s);
      }
    }
    if (dec_pred) {
      if ((dec_pred->hist_prev != nullptr) != (recv_prev != nullptr)) return TERA_EINVAL;
      fill_pred(ctx, &D.pr, dec_pred, ctx->cseg_dec);
      if (D.pr.hist) {
        dec_cells = 1;
        cudaMemsetAsync(ctx->cseg_dec, 0, sizeof(u64) * cwords, s);
      }
    }
  }
  const u64 n_windows = (P + W - 1) / W;
  cudaMemsetAsync(ctx->b_done, 0, sizeof(u32) * P * PH_COUNT, s);
  prof_begin(ctx, s);
  bat_setup_kernel<<<1, 1024, 0, s>>>(E, D, B, P, mode, T, K, enc_cells, dec_cells,
                                      reinterpret_cast<u64*>(wire_off),
                                      wire_capacity, ctx->cap_records, recv_capacity_units,
                                      ctx->b_units_cap < ctx->cap_units ? ctx->b_units_cap
                                                                        : ctx->cap_units,
                                      ctx->b_need, ctx->b_enc_uoff,
                                      ctx->b_dec_uoff, ctx->d_epoch);
  if ((st = check_launch(ctx, "bat_setup_kernel", s)) != TERA_OK) return st;
  const unsigned wthreads = W < 32 ? 32u : ((W + 31) / 32) * 32;
  prof_begin(ctx, s);
  bat_window_count_kernel<<<(unsigned)n_windows, wthreads, 0, s>>>(ctx->b_need, P, W,
                                                                    ctx->b_win_total);
  if ((st = check_launch(ctx, "bat_window_count_kernel", s)) != TERA_OK) return st;
  if ((st = scan_u32(ctx, ctx->b_win_total, ctx->b_win_base, nullptr, n_windows, s)) != TERA_OK)
    return st;
  prof_begin(ctx, s);
  bat_window_fill_kernel<<<(unsigned)n_windows, wthreads, 0, s>>>(
      ctx->b_need, P, W, ctx->b_win_base, n_windows, ctx->b_items, ctx->b_scalars + 0,
      reinterpret_cast<const u32*>(ctx->b_scalars + 2));
  if ((st = check_launch(ctx, "bat_window_fill_kernel", s)) != TERA_OK) return st;
  if (PR) {
    if (T == 128) return launch_persistent<128, true>(ctx, E, D, B, tn.ctas_per_sm, K, s);
    return launch_persistent<256, true>(ctx, E, D, B, tn.ctas_per_sm, K, s);
  }
  switch (T) {
    case 128: return launch_persistent<128, false>(ctx, E, D, B, tn.ctas_per_sm, K, s);
    case 512: return launch_persistent<512, false>(ctx, E, D, B, tn.ctas_per_sm, K, s);
    default: return launch_persistent<256, false>(ctx, E, D, B, tn.ctas_per_sm, K, s);
  }
}

extern "C" tera_status tera_codec_batched(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, void* stream) {
  return batched_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                      wire_capacity, wire_off, wire_len, recv_prev, recv_off_prev, recv,
                      recv_capacity_units, recv_off, mode, tune, nullptr, nullptr, stream);
}

extern "C" tera_status tera_codec_batched_pred(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, const tera_predictor* enc_pred,
    const tera_predictor* dec_pred, void* stream) {
  return batched_impl(ctx, rec_arena, pair_off, ref_prev, ref_off_prev, ref_next, wire,
                      wire_capacity, wire_off, wire_len, recv_prev, recv_off_prev, recv,
                      recv_capacity_units, recv_off, mode, tune, enc_pred, dec_pred, stream);
}
