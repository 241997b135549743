// Context, scratch memory, status word, generic scan and the in-place
// deserialization check of libtera.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tera_internal.cuh"

using namespace tera;

namespace {

template <typename T>
void free_dev(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
tera_status alloc_dev(T*& p, size_t count) {
  free_dev(p);
  if (count == 0) count = 1;
  if (cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return TERA_ENOMEM;
  }
  return TERA_OK;
}

// ---- generic exclusive scan of u32 values (reduce, scan partials, down-sweep) ----

__global__ void scan_reduce_kernel(const u32* __restrict__ in, u64 n, u64* __restrict__ part) {
  __shared__ u64 sm[33];
  const u64 base = (u64)blockIdx.x * kScanChunk;
  u64 s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    u64 i = base + (u64)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    u64 t = threadIdx.x < (kScanThreads / 32) ? sm[threadIdx.x] : 0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of part[0..m) in place, total to part[m].
__global__ void scan_partials_kernel(u64* part, u64 m) {
  __shared__ u64 sm[33];
  u64 carry = 0;
  for (u64 base = 0; base < m; base += kScanThreads) {
    u64 i = base + threadIdx.x;
    u64 v = i < m ? part[i] : 0;
    u64 tot;
    u64 ex = block_excl_scan<u64>(v, sm, &tot);
    if (i < m) part[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) part[m] = carry;
}

__global__ void scan_down_kernel(const u32* __restrict__ in, u64 n, const u64* __restrict__ part,
                                 u64* __restrict__ out64, u32* __restrict__ out32) {
  __shared__ u64 sm[33];
  const u64 base = (u64)blockIdx.x * kScanChunk + (u64)threadIdx.x * kScanPerThread;
  u32 v[kScanPerThread];
  u64 s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    u64 i = base + k;
    v[k] = i < n ? in[i] : 0u;
    s += v[k];
  }
  u64 tot;
  u64 ex = block_excl_scan<u64>(s, sm, &tot);
  u64 run = part[blockIdx.x] + ex;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    u64 i = base + k;
    if (i < n) {
      if (out64) out64[i] = run;
      if (out32) out32[i] = (u32)run;
    }
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    u64 total = part[gridDim.x];
    if (out64) out64[n] = total;
    if (out32) out32[n] = (u32)total;
  }
}

__global__ void unit_map_kernel(const u64* __restrict__ unit_off, u64 npr, u32 p0,
                                u32* __restrict__ unit_pair, const u64* __restrict__ units_total) {
  if (units_total[1]) return;
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  for (u64 k = warp; k < npr; k += nwarps)
    for (u64 u = unit_off[k] + lane; u < unit_off[k + 1]; u += 32) unit_pair[u] = p0 + (u32)k;
}

__global__ void validate_arena_kernel(const uint8_t* __restrict__ arena,
                                      const u64* __restrict__ off, u64 n_pairs, u32 class_id,
                                      DevStatus* st) {
  for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
       p += (u64)gridDim.x * blockDim.x) {
    const u64* h = reinterpret_cast<const u64*>(arena + (off[p] + p) * kRecBytes);
    u64 w0 = h[0], w1 = h[1], n = h[2];
    bool ok = (u32)w0 == kTaioMagic && (u32)((w0 >> 32) & 0xFFFF) == kVersion &&
              (u32)(w0 >> 48) == kRecBytes && (u32)w1 == class_id && (u32)(w1 >> 32) == (u32)p &&
              n == off[p + 1] - off[p];
    if (!ok) latch(st, TERA_ECORRUPT);
  }
}

}  // namespace

namespace tera {

// Optional per-kernel timing: an event pair around every launch, resolved by
// tera_ctx_profile_collect.  Off by default.
struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Pending {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  cudaEvent_t open_a = nullptr;
  std::vector<std::string> names;
  std::vector<uint64_t> count;
  std::vector<double> ms;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

static ProfState* prof(tera_ctx* ctx) { return reinterpret_cast<ProfState*>(ctx->prof); }

// Inside a stream capture an event becomes a graph node only when recorded as
// "external"; outside a capture it is recorded directly.
static void record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

void prof_begin(tera_ctx* ctx, cudaStream_t s) {
  ProfState* p = prof(ctx);
  if (!p || !p->on) return;
  p->open_a = p->get();
  record_event(p->open_a, s);
}

tera_status check_launch(tera_ctx* ctx, const char* name, cudaStream_t s) {
  ctx->launches += 1;
  ProfState* p = prof(ctx);
  if (p && p->on && p->open_a) {
    cudaEvent_t b = p->get();
    record_event(b, s);
    p->pending.push_back({name, p->open_a, b});
    p->open_a = nullptr;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "libtera: launch of %s failed: %s\n", name, cudaGetErrorString(e));
    return TERA_ECUDA;
  }
  return TERA_OK;
}

int grid_for(tera_ctx* ctx, int blocks_per_sm) { return ctx->num_sms * blocks_per_sm; }

tera_status launch_unit_map(tera_ctx* ctx, u32 p0, u64 npr, cudaStream_t s) {
  if (npr == 0) return TERA_OK;
  prof_begin(ctx, s);
  unit_map_kernel<<<(unsigned)((npr + 7) / 8), 256, 0, s>>>(ctx->unit_off, npr, p0, ctx->unit_pair,
                                                            ctx->d_units_total);
  return check_launch(ctx, "unit_map_kernel", s);
}

static tera_status ensure_scan_part(tera_ctx* ctx, u64 n) {
  u64 need = (n + kScanChunk - 1) / kScanChunk + 2;
  if (need <= ctx->scan_part_cap) return TERA_OK;
  cudaDeviceSynchronize();
  u64 cap = need * 2;
  tera_status st = alloc_dev(ctx->scan_part, cap);
  if (st != TERA_OK) return st;
  ctx->scan_part_cap = cap;
  return TERA_OK;
}

tera_status scan_u32(tera_ctx* ctx, const u32* in, u64* out64, u32* out32, u64 n,
                     cudaStream_t s) {
  tera_status st = ensure_scan_part(ctx, n);
  if (st != TERA_OK) return st;
  u64 chunks = (n + kScanChunk - 1) / kScanChunk;
  if (chunks == 0) chunks = 1;
  if (chunks == 1) {
    cudaMemsetAsync(ctx->scan_part, 0, sizeof(u64), s);
    // part[1] = total is written by the down kernel through part[gridDim.x]; compute it
    prof_begin(ctx, s);
    scan_reduce_kernel<<<1, kScanThreads, 0, s>>>(in, n, ctx->scan_part + 1);
    if ((st = check_launch(ctx, "scan_reduce_kernel", s)) != TERA_OK) return st;
  } else {
    prof_begin(ctx, s);
    scan_reduce_kernel<<<(unsigned)chunks, kScanThreads, 0, s>>>(in, n, ctx->scan_part);
    if ((st = check_launch(ctx, "scan_reduce_kernel", s)) != TERA_OK) return st;
    prof_begin(ctx, s);
    scan_partials_kernel<<<1, kScanThreads, 0, s>>>(ctx->scan_part, chunks);
    if ((st = check_launch(ctx, "scan_partials_kernel", s)) != TERA_OK) return st;
  }
  prof_begin(ctx, s);
  scan_down_kernel<<<(unsigned)chunks, kScanThreads, 0, s>>>(in, n, ctx->scan_part, out64, out32);
  return check_launch(ctx, "scan_down_kernel", s);
}

tera_status ensure_agents(tera_ctx* ctx, int64_t n, cudaStream_t s) {
  (void)s;
  if (n <= ctx->cap_agents && ctx->tile_cnt && ctx->tile_base) return TERA_OK;
  cudaDeviceSynchronize();
  int64_t cap = n + n / 8 + kClassifyTile;
  u64 tiles = ((u64)cap + kRunAgents - 1) / kRunAgents;  // runs of the classification
  tera_status st;
  if ((st = alloc_dev(ctx->tile_cnt, tiles + 1)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->tile_base, tiles + 1)) != TERA_OK) return st;
  ctx->cap_agents = cap;
  return ensure_scan_part(ctx, tiles + 1);
}

tera_status ensure_records(tera_ctx* ctx, uint64_t cap, cudaStream_t s) {
  (void)s;
  if (cap <= ctx->cap_records && ctx->seg) return TERA_OK;
  cudaDeviceSynchronize();
  u64 c = cap < 1024 ? 1024 : cap;
  tera_status st;
  if ((st = alloc_dev(ctx->keys_a, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->ent_agent, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->ent_dest, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->keys_b, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->keys_c, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->vals_b, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->vals_c, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->agents_b, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->agents_c, c)) != TERA_OK) return st;
  u64 tiles = (c + kSortTile - 1) / kSortTile;
  if ((st = alloc_dev(ctx->rs_hist, (u64)kRadix * tiles + 1)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->matched, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->slot_src, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->seg, 2 * c + 2 * ctx->n_pairs)) != TERA_OK) return st;
  // epoch 0 is never current, so zeroed segments and flags are empty
  cudaMemset(ctx->seg, 0, sizeof(U64x2) * (2 * c + 2 * ctx->n_pairs));
  cudaMemset(ctx->matched, 0, sizeof(u32) * c);
  ctx->cap_records = c;
  return ensure_scan_part(ctx, (u64)kRadix * tiles + 1);
}

tera_status ensure_units(tera_ctx* ctx, uint64_t cap, cudaStream_t s) {
  (void)s;
  if (cap <= ctx->cap_units) return TERA_OK;
  cudaDeviceSynchronize();
  u64 c = cap + cap / 4 + 1024;
  tera_status st;
  if ((st = alloc_dev(ctx->unit_sum, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->unit_base, c)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->unit_pair, c)) != TERA_OK) return st;
  ctx->cap_units = c;
  return TERA_OK;
}

tera_status ensure_batched(tera_ctx* ctx) {
  const u64 P = ctx->n_pairs;
  // work items: one per pair, plus at most (blocks + pairs) for the teams
  const u64 items = 2 * P + (u64)ctx->num_sms * 16 + 64;
  // tile totals of team pairs: (slots + 2 records + receiver slots) / 128 + 3 per pair
  const u64 tsum = 4 * (ctx->cap_records / 128) + 3 * P + 64;
  if (ctx->b_ptot && ctx->b_items_cap >= items && ctx->b_tsum_cap >= tsum) return TERA_OK;
  cudaDeviceSynchronize();
  tera_status st;
  if (!ctx->b_ptot) {
    if ((st = alloc_dev(ctx->b_ptot, P * 4)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->b_scalars, 6)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->b_team, P * 8)) != TERA_OK) return st;
    if (!ctx->b_side &&
        (cudaStreamCreateWithFlags(&ctx->b_side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&ctx->b_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&ctx->b_join, cudaEventDisableTiming) != cudaSuccess))
      return TERA_ECUDA;
    if ((st = alloc_dev(ctx->b_tbase, P)) != TERA_OK) return st;
    // block sums of the setup's first launch: 4 words per block of 1024 pairs
    if ((st = alloc_dev(ctx->b_part, 4 * (P / 1024 + 1))) != TERA_OK) return st;
    cudaMemset(ctx->b_scalars, 0, 6 * sizeof(u64));
  }
  if ((st = alloc_dev(ctx->b_items, items)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->b_tsum, tsum)) != TERA_OK) return st;
  ctx->b_items_cap = items;
  ctx->b_tsum_cap = tsum;
  return TERA_OK;
}

tera_status ensure_migrate(tera_ctx* ctx, uint64_t n, uint64_t leavers) {
  tera_status st;
  if (!ctx->m_from) {
    cudaDeviceSynchronize();
    if ((st = alloc_dev(ctx->m_from, ctx->n_boxes)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_before, ctx->n_boxes)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_cnt, ctx->n_pairs)) != TERA_OK) return st;
  }
  if (n > ctx->m_cap_agents || !ctx->m_tile_cnt) {
    cudaDeviceSynchronize();
    u64 cap = n + n / 8 + kClassifyTile;
    u64 tiles = (cap + kWarpAgents - 1) / kWarpAgents;  // warp tiles
    if ((st = alloc_dev(ctx->m_tile_cnt, tiles + 1)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_tile_base, tiles + 1)) != TERA_OK) return st;
    if ((st = ensure_scan_part(ctx, tiles + 1)) != TERA_OK) return st;
    ctx->m_cap_agents = cap;
  }
  if (leavers > ctx->m_cap_leavers || !ctx->m_key) {
    cudaDeviceSynchronize();
    u64 c = leavers < 1024 ? 1024 : leavers;
    if ((st = alloc_dev(ctx->m_key, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_agent, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_sorted, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_dest, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_keys_b, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_keys_c, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_vals_b, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_vals_c, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_agents_b, c)) != TERA_OK) return st;
    if ((st = alloc_dev(ctx->m_agents_c, c)) != TERA_OK) return st;
    u64 tiles = (c + kSortTile - 1) / kSortTile;
    if ((st = alloc_dev(ctx->m_hist, (u64)kRadix * tiles + 1)) != TERA_OK) return st;
    if ((st = ensure_scan_part(ctx, (u64)kRadix * tiles + 1)) != TERA_OK) return st;
    ctx->m_cap_leavers = c;
  }
  return TERA_OK;
}

// Axes with more cells than this keep the binary64 formula on the device.
constexpr uint64_t kCellTableMax = 1ull << 16;

static double value_of_key(uint64_t k) {
  const uint64_t b = k >= 0x8000000000000000ull ? k ^ 0x8000000000000000ull : ~k;
  double d;
  memcpy(&d, &b, 8);
  return d;
}

static uint64_t key_of_value(double d) {
  uint64_t b;
  memcpy(&b, &d, 8);
  return key_of(b);
}

// Cell thresholds of one axis of the predictor's cell grid: T[0] = key(lo),
// T[n] = key(hi), and for 1 <= k < n, T[k] = the key of the smallest binary64
// x with floor((x - lo) / w) >= k, the quotient evaluated in binary64 exactly
// as the device's formula evaluates it (IEEE subtraction and division, round
// to nearest).  The cell is monotone in x, so each T[k] is found by bisection
// over the keys of [lo, hi], starting above T[k - 1].
void cell_thresholds(double lo, double hi, double w, uint64_t n, uint64_t* T) {
  auto cell = [&](uint64_t k) { return (int64_t)std::floor((value_of_key(k) - lo) / w); };
  const uint64_t klo = key_of_value(lo), khi = key_of_value(hi);
  T[0] = klo;
  T[n] = khi;
  uint64_t below = klo;  // cell(below) < k
  for (uint64_t k = 1; k < n; ++k) {
    uint64_t L = below, H = khi;  // cell(L) < k <= cell(H) = n - 1
    while (H - L > 1) {
      const uint64_t M = L + (H - L) / 2;
      if (cell(M) >= (int64_t)k) H = M;
      else L = M;
    }
    T[k] = H;
    below = H - 1;
  }
}

// The predictor's cell threshold tables (once per context).
static tera_status ensure_cell_tables(tera_ctx* ctx) {
  if (ctx->d_ckeys) return TERA_OK;
  uint64_t total = 0, off[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) {
    off[a] = total;
    if (ctx->ncell[a] <= kCellTableMax) total += ctx->ncell[a] + 1;
  }
  if (total == 0) return TERA_OK;
  std::vector<uint64_t> h(total);
  for (int a = 0; a < 3; ++a)
    if (ctx->ncell[a] <= kCellTableMax)
      cell_thresholds(ctx->grid.lo[a], ctx->grid.hi[a], ctx->grid.w, ctx->ncell[a], h.data() + off[a]);
  tera_status st = alloc_dev(ctx->d_ckeys, total);
  if (st != TERA_OK) return st;
  if (cudaMemcpy(ctx->d_ckeys, h.data(), 8 * total, cudaMemcpyHostToDevice) != cudaSuccess)
    return TERA_ECUDA;
  for (int a = 0; a < 3; ++a) {
    ctx->ck[a] = ctx->ncell[a] <= kCellTableMax ? ctx->d_ckeys + off[a] : nullptr;
    ctx->ck_flo[a] = (float)ctx->grid.lo[a];
    ctx->ck_fs[a] = (float)(1.0 / ctx->grid.w);
  }
  return TERA_OK;
}

tera_status ensure_pred(tera_ctx* ctx) {
  const u64 cap = ctx->cap_records, P = ctx->n_pairs;
  if (ctx->cseg_enc && ctx->pred_cap >= cap && ctx->unit_res && ctx->unit_res_cap >= ctx->cap_units)
    return TERA_OK;
  cudaDeviceSynchronize();
  tera_status st;
  if ((st = ensure_cell_tables(ctx)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->cseg_enc, 2 * (2 * cap + 2 * P))) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->cseg_dec, 2 * (2 * cap + 2 * P))) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->pscr, 4 * cap)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->pscr_dec, 4 * cap)) != TERA_OK) return st;
  if ((st = alloc_dev(ctx->unit_res, ctx->cap_units)) != TERA_OK) return st;
  ctx->pred_cap = cap;
  ctx->unit_res_cap = ctx->cap_units;
  return TERA_OK;
}

}  // namespace tera

namespace tera {

// The key tables of a grid (and its cell counts per axis); TERA_EINVAL for a
// grid tera_ctx_create rejects.
static tera_status grid_tables(const tera_grid* grid, GridTables* tp, uint64_t ncell[3]) {
  GridTables& t = *tp;
  if (grid->reserved != 0 || (grid->periodic & ~7u) != 0) return TERA_EINVAL;
  memset(&t, 0, sizeof(t));
  auto key = [](double d) {
    uint64_t b;
    memcpy(&b, &d, 8);
    return key_of(b);
  };
  for (int a = 0; a < 3; ++a) {
    int n = grid->n[a];
    if (n < 1 || n > kMaxAxis) return TERA_EINVAL;
    if ((grid->periodic >> a & 1u) && n < 3) return TERA_EINVAL;
    if (!(grid->lo[a] < grid->hi[a])) return TERA_EINVAL;
    if (!std::isfinite(grid->lo[a]) || !std::isfinite(grid->hi[a])) return TERA_EINVAL;
    double lo = grid->lo[a], hi = grid->hi[a];
    std::vector<double> e((size_t)n + 1);
    for (int k = 0; k < n; ++k) e[k] = lo + ((hi - lo) * (double)k) / (double)n;
    e[n] = hi;
    if (!(grid->w > 0.0)) return TERA_EINVAL;
    for (int k = 0; k <= n; ++k) t.ke[a][k] = key(e[k]);
    for (int k = 0; k < n; ++k) {
      if (!(grid->w < e[k + 1] - e[k])) return TERA_EINVAL;
      t.ktl[a][k] = key(e[k] + grid->w);
      t.kth[a][k] = key(e[k + 1] - grid->w);
    }
    t.klo[a] = key(lo);
    t.khi[a] = key(hi);
    t.n[a] = n;
    t.periodic = (int)grid->periodic;
    // only a starting guess: the index is fixed by exact key comparisons
    t.flo[a] = (float)lo;
    t.fscale[a] = (float)((double)n / (hi - lo));
    ncell[a] = (uint64_t)std::floor((hi - lo) / grid->w) + 1;
  }
  return TERA_OK;
}

// The classification table of the grid (see AxisBuckets); false when the grid
// gets none.  The device's bucket position of v differs from the true one,
// (v - lo) * kAxisBuckets / (hi - lo), by at most: the estimate's mantissa cut
// to 20 bits (2^-20 of |v|; only |v| <= 2 max(|lo|, |hi|) can land inside the
// table at all), lo and the scale rounded to float (2^-24 each) and the
// subtraction and product rounded (2^-24 of a position below kAxisBuckets);
// twice that sum is the margin kept around every threshold.
static bool build_axis_buckets(const tera_grid& g, const GridTables& t, AxisBuckets* b) {
  memset(b, 0, sizeof(*b));
  const double eps20 = std::ldexp(1.0, -20), eps24 = std::ldexp(1.0, -24);
  for (int a = 0; a < 3; ++a) {
    const int n = t.n[a];
    const double lo = g.lo[a], hi = g.hi[a];
    const double mag = std::fmax(std::fabs(lo), std::fabs(hi));
    if (n > 32 || !(mag < 1e37)) return false;
    const double s = (double)kAxisBuckets / (hi - lo);
    b->flo[a] = (float)lo;
    b->fs[a] = (float)s;
    if (!std::isfinite(s) || !std::isfinite(b->fs[a]) || !(b->fs[a] > 0.0f)) return false;
    const double err = 2.0 * (2.0 * mag * eps20 * s + std::fabs(lo) * eps24 * s +
                              4.0 * kAxisBuckets * eps24) + 1e-9;
    if (!(err < 0.25)) return false;
    // the values where the classification can change, ascending
    std::vector<double> th;
    th.push_back(lo);
    th.push_back(hi);
    for (int k = 0; k < n; ++k) {
      const double e0 = lo + ((hi - lo) * (double)k) / (double)n;
      const double e1 = k + 1 == n ? hi : lo + ((hi - lo) * (double)(k + 1)) / (double)n;
      if (k > 0) th.push_back(e0);
      th.push_back(e0 + g.w);
      th.push_back(e1 - g.w);
    }
    std::sort(th.begin(), th.end());
    const bool wrap = (t.periodic >> a) & 1;
    for (int j = 0; j < kAxisBuckets; ++j) {
      const double A = lo + ((double)j - err) / s, B = lo + ((double)j + 1.0 + err) / s;
      bool exact = !(A > lo) || !(B < hi);
      const auto it = std::lower_bound(th.begin(), th.end(), A);
      if (it != th.end() && *it <= B) exact = true;
      if (exact) {
        b->tab[a][j] = kBucketExact;
        continue;
      }
      // every value of [A, B] classifies as its midpoint: the rule on the keys
      const double v = 0.5 * (A + B);
      uint64_t bits;
      memcpy(&bits, &v, 8);
      const u64 k = key_of(bits);
      int i = 0;
      while (i < n - 1 && k >= t.ke[a][i + 1]) ++i;
      const u32 lowq = (i > 0 || wrap) && k < t.ktl[a][i];
      const u32 highq = (i < n - 1 || wrap) && k >= t.kth[a][i];
      b->tab[a][j] = (uint8_t)((u32)i << 2 | lowq | highq << 1);
    }
  }
  b->on = 1;
  return true;
}

}  // namespace tera

extern "C" {

const char* tera_version(void) { return "tera-gb300 1.0 (sm_103a)"; }

tera_status tera_cell_thresholds(double lo, double hi, double w, uint64_t n, uint64_t* T) {
  if (!T || !std::isfinite(lo) || !std::isfinite(hi) || !std::isfinite(w) || !(lo < hi) ||
      !(w > 0.0))
    return TERA_EINVAL;
  const double c = std::floor((hi - lo) / w);
  if (!(c >= 0.0 && c < 1.8e19) || n != (uint64_t)c + 1) return TERA_EINVAL;
  tera::cell_thresholds(lo, hi, w, n, T);
  return TERA_OK;
}

tera_status tera_axis_buckets(const tera_grid* grid, uint8_t* tab, float* flo, float* fs,
                              int* on) {
  if (!grid || !tab || !flo || !fs || !on) return TERA_EINVAL;
  GridTables* t = new (std::nothrow) GridTables;
  AxisBuckets* b = new (std::nothrow) AxisBuckets;
  tera_status st = (t && b) ? TERA_OK : TERA_ENOMEM;
  uint64_t ncell[3];
  if (st == TERA_OK) st = grid_tables(grid, t, ncell);
  if (st == TERA_OK) {
    *on = build_axis_buckets(*grid, *t, b) ? 1 : 0;
    if (*on) {
      memcpy(tab, b->tab, sizeof(b->tab));
      for (int a = 0; a < 3; ++a) {
        flo[a] = b->flo[a];
        fs[a] = b->fs[a];
      }
    }
  }
  delete t;
  delete b;
  return st;
}

tera_status tera_ref_schedule(uint64_t t, uint32_t ref_interval, int32_t* out_buf,
                              int32_t* ref_buf, uint64_t* ref_iteration) {
  if (ref_interval < 1 || !out_buf) return TERA_EINVAL;
  const uint64_t K = ref_interval;
  *out_buf = (int32_t)(((t + K - 1) / K) % 2);  // ceil(t / K) mod 2
  if (t == 0) {  // no reference yet
    if (ref_buf) *ref_buf = -1;
    if (ref_iteration) *ref_iteration = 0;
    return TERA_OK;
  }
  const uint64_t ri = K * ((t - 1) / K);  // the latest multiple of K before t
  if (ref_buf) *ref_buf = (int32_t)(((ri + K - 1) / K) % 2);
  if (ref_iteration) *ref_iteration = ri;
  return TERA_OK;
}

uint64_t tera_n_pairs(const tera_ctx* ctx) { return ctx ? ctx->n_pairs : 0; }

uint64_t tera_ctx_launches(const tera_ctx* ctx) { return ctx ? ctx->launches : 0; }

tera_status tera_ctx_create(tera_ctx** out, const tera_grid* grid, int device, uint32_t class_id) {
  if (!out || !grid) return TERA_EINVAL;
  *out = nullptr;
  GridTables t;
  uint64_t ncell_tmp[3] = {1, 1, 1};
  const tera_status gst = grid_tables(grid, &t, ncell_tmp);
  if (gst != TERA_OK) return gst;
  if (cudaSetDevice(device) != cudaSuccess) return TERA_ECUDA;
  tera_ctx* c = new (std::nothrow) tera_ctx();
  if (!c) return TERA_ENOMEM;
  memset(c, 0, sizeof(*c));
  c->device = device;
  c->class_id = class_id;
  c->grid = *grid;
  c->n_boxes = (uint32_t)grid->n[0] * (uint32_t)grid->n[1] * (uint32_t)grid->n[2];
  c->n_pairs = (uint64_t)c->n_boxes * 27u;
  for (int a = 0; a < 3; ++a) c->ncell[a] = ncell_tmp[a];
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (c->num_sms <= 0) c->num_sms = 148;
  tera_status st = TERA_OK;
  if ((st = alloc_dev(c->d_grid, 1)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->d_status, 1)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->d_epoch, 1)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->d_reset, c->n_pairs)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->unit_off, c->n_pairs + 1)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->pair_info, c->n_pairs * 16)) != TERA_OK) goto fail;  // encode + decode
  if ((st = alloc_dev(c->d_total, 8)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->d_units_total, 2)) != TERA_OK) goto fail;
  if ((st = alloc_dev(c->d_stats, 1)) != TERA_OK) goto fail;
  c->prof = new (std::nothrow) ProfState();
  if (cudaMallocHost(reinterpret_cast<void**>(&c->h_status), sizeof(DevStatus)) != cudaSuccess) {
    st = TERA_ENOMEM;
    goto fail;
  }
  cudaMemcpy(c->d_grid, &t, sizeof(t), cudaMemcpyHostToDevice);
  {
    AxisBuckets* hb = new (std::nothrow) AxisBuckets;
    if (!hb) {
      st = TERA_ENOMEM;
      goto fail;
    }
    if (build_axis_buckets(*grid, t, hb)) {
      if ((st = alloc_dev(c->d_buckets, 1)) != TERA_OK) {
        delete hb;
        goto fail;
      }
      cudaMemcpy(c->d_buckets, hb, sizeof(*hb), cudaMemcpyHostToDevice);
    }
    delete hb;
  }
  cudaMemset(c->d_status, 0, sizeof(DevStatus));
  cudaMemset(c->d_epoch, 0, sizeof(uint32_t));
  cudaMemset(c->d_reset, 0, c->n_pairs);
  cudaMemset(c->d_total, 0, 8 * sizeof(uint64_t));
  cudaMemset(c->d_stats, 0, sizeof(DevStats));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    st = TERA_ECUDA;
    goto fail;
  }
  *out = c;
  return TERA_OK;
fail:
  tera_ctx_destroy(c);
  return st;
}

tera_status tera_ctx_destroy(tera_ctx* c) {
  if (!c) return TERA_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  free_dev(c->d_grid);
  free_dev(c->d_buckets);
  free_dev(c->d_status);
  free_dev(c->d_epoch);
  free_dev(c->d_reset);
  free_dev(c->tile_cnt);
  free_dev(c->tile_base);
  free_dev(c->keys_a);
  free_dev(c->ent_agent);
  free_dev(c->ent_dest);
  free_dev(c->keys_b);
  free_dev(c->keys_c);
  free_dev(c->vals_b);
  free_dev(c->vals_c);
  free_dev(c->agents_b);
  free_dev(c->agents_c);
  free_dev(c->rs_hist);
  free_dev(c->scan_part);
  free_dev(c->d_total);
  free_dev(c->seg);
  free_dev(c->matched);
  free_dev(c->slot_src);
  free_dev(c->unit_off);
  free_dev(c->unit_sum);
  free_dev(c->unit_base);
  free_dev(c->unit_pair);
  free_dev(c->pair_info);
  free_dev(c->d_units_total);
  free_dev(c->d_stats);
  free_dev(c->b_scalars);
  if (c->b_side) cudaStreamDestroy(c->b_side);
  if (c->b_fork) cudaEventDestroy(c->b_fork);
  if (c->b_join) cudaEventDestroy(c->b_join);
  free_dev(c->b_ptot);
  free_dev(c->b_items);
  free_dev(c->pscr_dec);
  free_dev(c->b_team);
  free_dev(c->b_tsum);
  free_dev(c->b_tbase);
  free_dev(c->b_part);
  free_dev(c->m_tile_cnt);
  free_dev(c->m_tile_base);
  free_dev(c->m_from);
  free_dev(c->m_before);
  free_dev(c->m_cnt);
  free_dev(c->m_key);
  free_dev(c->m_agent);
  free_dev(c->m_sorted);
  free_dev(c->m_dest);
  free_dev(c->m_keys_b);
  free_dev(c->m_keys_c);
  free_dev(c->m_vals_b);
  free_dev(c->m_vals_c);
  free_dev(c->m_agents_b);
  free_dev(c->m_agents_c);
  free_dev(c->m_hist);
  free_dev(c->cseg_enc);
  free_dev(c->cseg_dec);
  free_dev(c->d_ckeys);
  free_dev(c->pscr);
  free_dev(c->unit_res);
  free_dev(c->mlp_scratch);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (ProfState* p = prof(c)) {
    for (auto& q : p->pending) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
    for (auto e : p->pool) cudaEventDestroy(e);
    if (p->open_a) cudaEventDestroy(p->open_a);
    delete p;
  }
  delete c;
  return TERA_OK;
}

tera_status tera_ctx_reserve(tera_ctx* ctx, int64_t max_agents, uint64_t max_records) {
  if (!ctx || max_agents < 0) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  tera_status st = ensure_agents(ctx, max_agents, 0);
  if (st != TERA_OK) return st;
  st = ensure_records(ctx, max_records, 0);
  if (st != TERA_OK) return st;
  return ensure_units(ctx, 2 * (max_records / kCodecTile) + 4 * ctx->n_pairs + 16, 0);
}

tera_status tera_ctx_status(tera_ctx* ctx, uint64_t* required_capacity, void* stream) {
  if (!ctx) return TERA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess)
    return TERA_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TERA_ECUDA;
  DevStatus h = *ctx->h_status;
  if (required_capacity) *required_capacity = h.required;
  cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), s);
  return (tera_status)h.code;
}

tera_status tera_ctx_stats(tera_ctx* ctx, tera_stats* out, int reset, void* stream) {
  if (!ctx || !out) return TERA_EINVAL;
  static_assert(sizeof(tera_stats) == sizeof(DevStats), "stats layout");
  cudaStream_t s = (cudaStream_t)stream;
  DevStats h;
  if (cudaMemcpyAsync(&h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TERA_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TERA_ECUDA;
  memcpy(out, &h, sizeof(h));
  if (reset) cudaMemsetAsync(ctx->d_stats, 0, sizeof(DevStats), s);
  return TERA_OK;
}

tera_status tera_ctx_profile(tera_ctx* ctx, int enable) {
  if (!ctx || !prof(ctx)) return TERA_EINVAL;
  prof(ctx)->on = enable != 0;
  return TERA_OK;
}

tera_status tera_ctx_profile_collect(tera_ctx* ctx) {
  if (!ctx || !prof(ctx)) return TERA_EINVAL;
  ProfState* p = prof(ctx);
  for (auto& q : p->pending) {
    if (cudaEventSynchronize(q.b) != cudaSuccess) return TERA_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) != cudaSuccess) {
      cudaGetLastError();  // an event pair that was never replayed: no time
      ms = 0.f;
    }
    size_t i = 0;
    while (i < p->names.size() && p->names[i] != q.name) ++i;
    if (i == p->names.size()) {
      p->names.push_back(q.name);
      p->count.push_back(0);
      p->ms.push_back(0.0);
    }
    p->count[i] += 1;
    p->ms[i] += ms;
    p->pool.push_back(q.a);
    p->pool.push_back(q.b);
  }
  p->pending.clear();
  return TERA_OK;
}

int tera_ctx_profile_entries(const tera_ctx* ctx) {
  if (!ctx || !ctx->prof) return 0;
  return (int)reinterpret_cast<const ProfState*>(ctx->prof)->names.size();
}

tera_status tera_ctx_profile_entry(const tera_ctx* ctx, int i, const char** name,
                                   uint64_t* launches, double* total_ms) {
  if (!ctx || !ctx->prof) return TERA_EINVAL;
  const ProfState* p = reinterpret_cast<const ProfState*>(ctx->prof);
  if (i < 0 || (size_t)i >= p->names.size()) return TERA_EINVAL;
  if (name) *name = p->names[(size_t)i].c_str();
  if (launches) *launches = p->count[(size_t)i];
  if (total_ms) *total_ms = p->ms[(size_t)i];
  return TERA_OK;
}

tera_status tera_ctx_profile_reset(tera_ctx* ctx) {
  if (!ctx || !prof(ctx)) return TERA_EINVAL;
  tera_status st = tera_ctx_profile_collect(ctx);
  ProfState* p = prof(ctx);
  p->names.clear();
  p->count.clear();
  p->ms.clear();
  return st;
}

tera_status tera_reset_reference(tera_ctx* ctx, uint32_t pair) {
  if (!ctx || pair >= ctx->n_pairs) return TERA_EINVAL;
  // Rare: a blocking write keeps it ordered before any later launch.
  cudaSetDevice(ctx->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return TERA_ECUDA;
  if (cudaMemset(ctx->d_reset + pair, 1, 1) != cudaSuccess) return TERA_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return TERA_ECUDA;
  return TERA_OK;
}

tera_status tera_unpack_inplace(const uint8_t* buf, uint64_t len, uint32_t class_id, void** view,
                                uint64_t* count, void* stream) {
  if (!buf || !view || !count) return TERA_EINVAL;
  *view = nullptr;
  *count = 0;
  if (len < kHdrBytes) return TERA_ECORRUPT;
  if ((reinterpret_cast<uintptr_t>(buf) & 15u) != 0) return TERA_EINVAL;
  uint8_t h[kHdrBytes];
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h, buf, kHdrBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TERA_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TERA_ECUDA;
  uint32_t magic, cls;
  uint16_t ver, rsz;
  uint64_t n;
  memcpy(&magic, h + 0, 4);
  memcpy(&ver, h + 4, 2);
  memcpy(&rsz, h + 6, 2);
  memcpy(&cls, h + 8, 4);
  memcpy(&n, h + 16, 8);
  if (magic != kTaioMagic || ver != kVersion || rsz != kRecBytes || cls != class_id)
    return TERA_ECORRUPT;
  if (n > (len - kHdrBytes) / kRecBytes) return TERA_ECORRUPT;
  *view = const_cast<uint8_t*>(buf + kHdrBytes);
  *count = n;
  return TERA_OK;
}

tera_status tera_unpack_validate(tera_ctx* ctx, const uint8_t* arena, const uint64_t* off,
                                 void* stream) {
  TERA_CALL_RANGE("tera_unpack_validate");
  if (!ctx || !arena || !off) return TERA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int blocks = (int)((ctx->n_pairs + 255) / 256);
  prof_begin(ctx, s);
  validate_arena_kernel<<<blocks, 256, 0, s>>>(arena, reinterpret_cast<const u64*>(off),
                                               ctx->n_pairs, ctx->class_id, ctx->d_status);
  return check_launch(ctx, "validate_arena_kernel", s);
}

}  // extern "C"

// ---------------- wire messages into host memory ----------------

namespace {

// Grid-stride 16-byte copy of wire[0, wire_off[P]) into host memory; the
// length is read on the device.
__global__ void __launch_bounds__(256)
    wire_to_host_kernel(const uint4* __restrict__ wire, const u64* __restrict__ wire_off, u64 P,
                        uint4* __restrict__ dst, u64 cap, u64* count, DevStatus* st) {
  const u64 n = wire_off[P];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *count = n;
    if (n > cap) {
      latch(st, TERA_ECAPACITY);
      need(st, n);
    }
  }
  if (n > cap) return;
  const u64 n16 = n / 16;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
       i += (u64)gridDim.x * blockDim.x)
    dst[i] = wire[i];
}

}  // namespace

extern "C" tera_status tera_wire_to_host(tera_ctx* ctx, const uint8_t* wire,
                                         const uint64_t* wire_off, uint8_t* host_dst,
                                         uint64_t host_capacity, uint64_t* host_count,
                                         void* stream) {
  TERA_CALL_RANGE("tera_wire_to_host");
  if (!ctx || !wire || !wire_off || !host_dst || !host_count) return TERA_EINVAL;
  if (((uintptr_t)wire | (uintptr_t)host_dst) & 15u) return TERA_EINVAL;
  if ((uintptr_t)host_count & 7u) return TERA_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(ctx, s);
  wire_to_host_kernel<<<(unsigned)grid_for(ctx, 8), 256, 0, s>>>(
      reinterpret_cast<const uint4*>(wire), reinterpret_cast<const u64*>(wire_off),
      ctx->n_pairs, reinterpret_cast<uint4*>(host_dst), host_capacity,
      reinterpret_cast<u64*>(host_count), ctx->d_status);
  return check_launch(ctx, "wire_to_host_kernel", s);
}
