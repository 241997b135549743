// Per-unit device functions of the difference codec (paper Sec. 2.3, steps B,
// C and D, with the significant-byte packer of the compression stage), shared
// by the per-call kernels (encode.cu, decode.cu) and the persistent batched
// kernel (batched.cu).
//
// Work is cut into units of T entries (T = blockDim.x) that never cross a
// pair.  For pair p: ceil(r/T) slot units (reference slots) then ceil(m/T)
// message units (records of the message); decode units cover the r + a
// entries of the received message.
//
// CG = true marks the persistent kernel: data that other blocks of the same
// launch produce is read with ld.global.cg (L2), never from a stale L1 line.
#pragma once

#include "tera_internal.cuh"

namespace tera {

// Per-pair facts of the encode (stride 8 per pair).
enum { PI_R = 0, PI_M = 1, PI_NST = 2, PI_MODE = 3, PI_MATCHED = 4, PI_NEW = 5, PI_SLOTPAY = 6,
       PI_PAY = 7 };
// Per-pair facts of the decode (stride 8 per pair).
enum { DI_NS = 0, DI_NN = 1, DI_NH = 2, DI_PAY = 3, DI_OK = 4, DI_MODE = 5, DI_NT = 6 };

template <bool CG, typename T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <bool CG>
__device__ __forceinline__ U64x2 ldx(const U64x2* p) {
  if constexpr (CG) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p));
    return U64x2{v.x, v.y};
  } else {
    return *p;
  }
}

template <bool CG>
__device__ __forceinline__ Rec load_rec_x(const uint8_t* p) {
  if constexpr (!CG) return load_rec(p);
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
  Rec r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ulonglong2 v = __ldcg(q + i);
    r.w[2 * i] = v.x;
    r.w[2 * i + 1] = v.y;
  }
  return r;
}

// ---------------- learned predictor (not in the paper) ----------------
// MLP 8 -> 64 -> 64 -> 3 (ReLU hidden), float32, weights W1[64][8] b1[64]
// W2[64][64] b2[64] W3[3][64] b3[3]; each neuron: acc = b; for k ascending
// acc = fmaf(W[k], in[k], acc).  Per-slot history (48 bytes): u64 xp[3] (bits
// of the position one iteration before the reference's), u32 d2[3] (bits of
// (float)(xp - position before it)), u32 n (steps known, 0..2), u64 zero.
constexpr int kMlpIn = 8, kMlpH = 64, kMlpOut = 3;
constexpr int kMlpW1 = 0, kMlpB1 = kMlpW1 + kMlpH * kMlpIn, kMlpW2 = kMlpB1 + kMlpH;
constexpr int kMlpB2 = kMlpW2 + kMlpH * kMlpH, kMlpW3 = kMlpB2 + kMlpH;
constexpr int kMlpB3 = kMlpW3 + kMlpOut * kMlpH, kMlpParams = kMlpB3 + kMlpOut;  // 4931
constexpr u32 kHistBytes = 48;
constexpr u32 kModeResidual = 2;
constexpr int kSampleFloats = 12;  // 8 features, 3 target displacements, valid flag

struct PredArgs {
  const float* params;     // MLP weights (device); null: the residual mode is off
  const uint8_t* hist;     // history of the reference (slot j of pair p at index off[p] + j)
  uint8_t* hist_next;      // history of the new reference / receive buffer
  u64* cseg;               // neighbour-count segments: 2 words per entry (key + 1, count)
  u64* pscr;               // per-slot prediction scratch: pred bits x3, ok
  float* samples;          // per-slot training samples (encoder), may be null
  u64* unit_res;           // per-unit residual payload bytes (encoder)
  double lo[3];
  double w;
  u64 ncell[3];
  // per axis, the cell thresholds (ncell + 1 keys: key(lo), the key of the
  // first value of each cell 1 .. ncell - 1, key(hi)); null: no table
  const u64* ck[3];
  float cflo[3], cfs[3];  // float estimate of a cell index: (x - lo) * (1 / w)
  int allow_residual;
  // batched path: the cell counts and every reference slot's prediction were
  // made by the pre-pass (pred_cells_kernel, pred_slots_kernel) into cseg and
  // pscr before the codec kernel
  int pre = 0;
};

struct EncArgs {
  const uint8_t* rec;      // packed messages (TAIO arena laid out with pair_off)
  const u64* pair_off;
  const uint8_t* ref;      // sender reference (may be null)
  const u64* ref_off;
  uint8_t* ref_next;
  uint8_t* wire;
  const u64* wire_off;
  u64* wire_len;
  const u64* unit_off;     // per-call path: units of range pair k start at unit_off[k]
  const u64* units_total;
  const u32* unit_pair;
  U64x2* unit_sum;
  U64x2* unit_base;
  u64* info;
  u32* slot_src;
  u32* matched;
  uint8_t* reset;
  U64x2* seg;              // per-pair hash segments of the message ids
  const u32* epoch;
  u32 p0, p1;
  u32 class_id;
  DevStatus* st;
  DevStats* stats;
  PredArgs pr{};
  // optional id columns (batched path): ids of the packed records by global
  // record index, of the sender reference's slots (index ref_off[p] + j), and
  // of the new sender reference (written, index pair_off[p] + position)
  const u64* msg_ids = nullptr;
  const u64* ref_ids = nullptr;
  u64* ref_ids_next = nullptr;
};

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
  PredArgs pr{};
};

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


// Cell of a reference record: floor((v - lo) / w) per axis, in binary64.
// Values in [lo, hi) take the axis's threshold table: the index is the
// largest i < ncell with key(v) >= ck[i], found from a float estimate by
// exact key comparisons (the table holds the binary64 formula's own
// boundaries, so the result is the formula's, without binary64 division).
__device__ __forceinline__ u64 cell_index(u64 bits, int a, const PredArgs& pr) {
  const u64* T = pr.ck[a];
  if (T) {
    const u64 n = pr.ncell[a];
    const u64 k = key_of(bits);
    if (k >= __ldg(T) && k < __ldg(T + n)) {
      const float f = (approx_f32(bits) - pr.cflo[a]) * pr.cfs[a];
      u64 i = f > 0.0f ? (u64)f : 0;  // the conversion saturates
      i = i < n - 1 ? i : n - 1;
      while (i > 0 && k < __ldg(T + i)) --i;
      while (i + 1 < n && k >= __ldg(T + i + 1)) ++i;
      return i;
    }
  }
  const double q = floor(__ddiv_rn(__dsub_rn(__longlong_as_double((long long)bits), pr.lo[a]), pr.w));
  return (u64)(long long)q;
}

__device__ __forceinline__ u64 cell_key(const Rec& R, const PredArgs& pr) {
  u64 c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = cell_index(R.w[1 + a], a, pr);
  return c[0] + pr.ncell[0] * (c[1] + pr.ncell[1] * c[2]);
}

// Count one reference record in its cell (segment of pair p, zeroed before).
__device__ __forceinline__ void cell_insert(u64* cseg, u64 base, u64 size, u64 key) {
  u64 i = seg_start(key, size);
  for (u64 probe = 0; probe < size; ++probe) {
    u64* e = cseg + 2 * (base + i);
    const u64 k0 = __ldcg(e);
    if (k0 == 0) {
      const u64 prev = atomicCAS(e, 0ull, key + 1);
      if (prev == 0 || prev == key + 1) {
        atomicAdd(e + 1, 1ull);
        return;
      }
    } else if (k0 == key + 1) {
      atomicAdd(e + 1, 1ull);
      return;
    }
    i = (i + 1 == size) ? 0 : i + 1;
  }
}

__device__ __forceinline__ u32 cell_count(const u64* cseg, u64 base, u64 size, u64 key) {
  u64 i = seg_start(key, size);
  for (u64 probe = 0; probe < size; ++probe) {
    const u64* e = cseg + 2 * (base + i);
    const u64 k0 = __ldcg(e);
    if (k0 == key + 1) return (u32)__ldcg(e + 1);
    if (k0 == 0) return 0;
    i = (i + 1 == size) ? 0 : i + 1;
  }
  return 0;
}

// The network on one feature vector; W in shared memory.
__device__ __forceinline__ void mlp_infer(const float* __restrict__ W, const float* f, float* o) {
  float h1[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    float acc = W[kMlpB1 + j];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) acc = __fmaf_rn(W[kMlpW1 + j * kMlpIn + k], f[k], acc);
    h1[j] = acc > 0.0f ? acc : 0.0f;
  }
  o[0] = W[kMlpB3 + 0];
  o[1] = W[kMlpB3 + 1];
  o[2] = W[kMlpB3 + 2];
  for (int j = 0; j < kMlpH; ++j) {
    float acc = W[kMlpB2 + j];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) acc = __fmaf_rn(W[kMlpW2 + j * kMlpH + k], h1[k], acc);
    const float h2 = acc > 0.0f ? acc : 0.0f;
    // output neuron a accumulates its inputs in ascending order, like every layer
#pragma unroll
    for (int a = 0; a < kMlpOut; ++a) o[a] = __fmaf_rn(W[kMlpW3 + a * kMlpH + j], h2, o[a]);
  }
}

struct Hist {
  u64 xp[3];
  u32 d2[3];
  u32 n;
};

__device__ __forceinline__ Hist load_hist(const uint8_t* h) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(h);
  const ulonglong2 a = q[0], b = q[1], c = q[2];
  Hist r;
  r.xp[0] = a.x;
  r.xp[1] = a.y;
  r.xp[2] = b.x;
  r.d2[0] = (u32)b.y;
  r.d2[1] = (u32)(b.y >> 32);
  r.d2[2] = (u32)c.x;
  r.n = (u32)(c.x >> 32);
  return r;
}

// History of a new reference entry made from reference record R with history
// H (hn = nullptr: a new record, no history).
__device__ __forceinline__ void store_hist_next(uint8_t* out, const Rec* R, const Hist* H) {
  ulonglong2* q = reinterpret_cast<ulonglong2*>(out);
  if (!R) {
    q[0] = make_ulonglong2(0, 0);
    q[1] = make_ulonglong2(0, 0);
    q[2] = make_ulonglong2(0, 0);
    return;
  }
  const u32 n = H ? H->n : 0u;
  u32 d2[3] = {0u, 0u, 0u};
  if (n >= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      d2[a] = __float_as_uint(__double2float_rn(
          __dsub_rn(__longlong_as_double((long long)R->w[1 + a]),
                    __longlong_as_double((long long)H->xp[a]))));
  }
  const u32 n2 = n + 1 > 2 ? 2u : n + 1;
  q[0] = make_ulonglong2(R->w[1], R->w[2]);
  q[1] = make_ulonglong2(R->w[3], (u64)d2[0] | ((u64)d2[1] << 32));
  q[2] = make_ulonglong2((u64)d2[2] | ((u64)n2 << 32), 0);
}

// Features of a reference slot; false when it is not predictable.
__device__ __forceinline__ bool features(const Rec& R, const Hist& H, u32 ncount, float* f) {
  if (H.n < 2) return false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f[a] = __double2float_rn(__dsub_rn(__longlong_as_double((long long)R.w[1 + a]),
                                       __longlong_as_double((long long)H.xp[a])));
    f[3 + a] = __uint_as_float(H.d2[a]);
  }
  f[6] = __double2float_rn(__ddiv_rn(__longlong_as_double((long long)R.w[4]), 10.0));
  f[7] = __fmul_rn(__uint2float_rn(ncount), 0.03125f);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) ok &= isfinite(f[i]);
  return ok;
}

// The predicted positions from the network's output: each displacement added
// to the reference position in double precision; false when an output is
// not finite.
__device__ __forceinline__ bool predict_out(const Rec& R, const float* o, u64* pred) {
  bool ok = isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    pred[a] = (u64)__double_as_longlong(
        __dadd_rn(__longlong_as_double((long long)R.w[1 + a]), (double)o[a]));
  return ok;
}

// Predicted position bits from features; false when an output is not finite.
__device__ __forceinline__ bool predict_from(const float* W, const Rec& R, const float* f,
                                             u64* pred) {
  float o[kMlpOut];
  mlp_infer(W, f, o);
  return predict_out(R, o, pred);
}

__device__ __forceinline__ u64 zigzag(u64 d) { return (d << 1) ^ (u64)((long long)d >> 63); }
__device__ __forceinline__ u64 unzigzag(u64 z) { return (z >> 1) ^ (0ull - (z & 1ull)); }

// Predictor arguments from the caller's tera_predictor and the context.
inline void fill_pred(const tera_ctx* ctx, PredArgs* pr, const tera_predictor* pred, u64* cseg) {
  pr->params = pred->params;
  pr->hist = pred->hist_prev;
  pr->hist_next = pred->hist_next;
  pr->cseg = cseg;
  pr->pscr = ctx->pscr;
  pr->samples = nullptr;
  pr->unit_res = ctx->unit_res;
  for (int a = 0; a < 3; ++a) {
    pr->lo[a] = ctx->grid.lo[a];
    pr->ncell[a] = ctx->ncell[a];
    pr->ck[a] = ctx->ck[a];
    pr->cflo[a] = ctx->ck_flo[a];
    pr->cfs[a] = ctx->ck_fs[a];
  }
  pr->w = ctx->grid.w;
  pr->allow_residual = 0;
}

// Slot units of either side: count every reference record in its cell.
__device__ __forceinline__ void cells_unit(const PredArgs& pr, const uint8_t* ref,
                                           const u64* ref_off, u32 p, u64 local, u64 r, int T) {
  const u64 j = local * (u64)T + threadIdx.x;
  if (j >= r) return;
  const Rec R = load_rec(ref + (ref_off[p] + p + 1 + j) * kRecBytes);
  cell_insert(pr.cseg, seg_base(ref_off[p], p), seg_size(r), cell_key(R, pr));
}

// Load the MLP weights into shared memory (all threads).
__device__ __forceinline__ void load_mlp(float* sW, const float* params) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sW[i] = params[i];
  __syncthreads();
}

// Hash entry of a pair's segment: a = tag (epoch << 32 | record index in the
// pair), b = the record's id.  An entry whose tag carries another epoch is
// empty for this iteration, so the segments never need clearing.
//
// Insert: claim the first empty entry on the probe sequence with a CAS of the
// tag, then store the id.  Lookups run only after every insert of the pair
// has finished (a later kernel, or a later phase of the batched kernel).
template <bool CG>
__device__ __forceinline__ void seg_insert_from(U64x2* seg, u64 base, u64 size, u64 id, u64 tag,
                                                u32 epoch, u64 i) {
  for (u64 probe = 0; probe < size; ++probe) {
    U64x2* e = seg + base + i;
    u64 cur = ldx<CG>(&e->a);
    while ((u32)(cur >> 32) != epoch) {  // empty for this iteration: claim it
      const u64 prev = atomicCAS(&e->a, cur, tag);
      if (prev == cur) {
        e->b = id;
        return;
      }
      cur = prev;
    }
    i = (i + 1 == size) ? 0 : i + 1;
  }
}

template <bool CG>
__device__ __forceinline__ void seg_insert(U64x2* seg, u64 base, u64 size, u64 id, u64 tag,
                                           u32 epoch) {
  seg_insert_from<CG>(seg, base, size, id, tag, epoch, seg_start(id, size));
}

// Record index (global) of the message record with this id, probing from
// entry i of the segment [base, base + size), or kNoMatch.
template <bool CG>
__device__ __forceinline__ u32 seg_lookup_from(const U64x2* __restrict__ seg, u32 epoch, u64 base,
                                               u64 size, u64 g_lo, u64 id, u64 i) {
  for (u64 probe = 0; probe < size; ++probe) {
    const U64x2 e = ldx<CG>(seg + base + i);
    if ((u32)(e.a >> 32) != epoch) return kNoMatch;
    if (e.b == id) return (u32)(g_lo + (u32)e.a);
    i = (i + 1 == size) ? 0 : i + 1;
  }
  return kNoMatch;
}

// The same for pair p (one 16-byte load per probe compares the stored id).
template <bool CG>
__device__ __forceinline__ u32 seg_lookup(const U64x2* __restrict__ seg, u32 epoch, u32 p,
                                          u64 g_lo, u64 m, u64 id) {
  const u64 size = seg_size(m);
  return seg_lookup_from<CG>(seg, epoch, seg_base(g_lo, p), size, g_lo, id, seg_start(id, size));
}

// Id of message record g (global record index) of pair p: from the id
// column when there is one, else word 0 of the record in the packed arena.
__device__ __forceinline__ u64 msg_id(const EncArgs& A, u32 p, u64 g) {
  if (A.msg_ids) return A.msg_ids[g];
  return *reinterpret_cast<const u64*>(A.rec + (g + p + 1) * kRecBytes);
}

// Id of slot j of pair p's sender reference (ro = ref_off[p]): from the id
// column when there is one, else word 0 of the reference record.
__device__ __forceinline__ u64 ref_id(const EncArgs& A, u32 p, u64 ro, u64 j) {
  if (A.ref_ids) return A.ref_ids[ro + j];
  return *reinterpret_cast<const u64*>(A.ref + (ro + p + 1 + j) * kRecBytes);
}

// A record of the new sender reference at global index g (pair p), and its
// id in the id column when there is one.
__device__ __forceinline__ void store_ref_next(const EncArgs& A, u32 p, u64 g, const Rec& R) {
  if (!in_bounds(A.st, g, A.pair_off[p], A.pair_off[p + 1])) return;
  store_rec(A.ref_next + (g + p + 1) * kRecBytes, R);
  if (A.ref_ids_next) A.ref_ids_next[g] = R.w[0];
}

// ---------------- encode ----------------

// Message unit: index every record of the pair by id in the pair's segment.
template <int T, bool CG>
__device__ __forceinline__ void enc_build_unit(const EncArgs& A, u32 p, u64 local, u32 epoch) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 nst = pi[PI_NST];
  const u64 m = pi[PI_M];
  const u64 k = (local - nst) * T + threadIdx.x;
  if (k >= m) return;
  const u64 g_lo = A.pair_off[p];
  const u64 id = msg_id(A, p, g_lo + k);
  seg_insert<CG>(A.seg, seg_base(g_lo, p), seg_size(m), id, ((u64)epoch << 32) | k, epoch);
}

// Slot unit: find the message record with the slot's id, write the slot's
// code, and return the unit's (payload bytes, non-placeholder slots).
template <int T, bool CG, bool PR = false>
__device__ __forceinline__ void enc_match_unit(const EncArgs& A, u32 p, u64 local, u64 U,
                                               u32 epoch, U64x2* sm, const float* sW = nullptr) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 r = pi[PI_R];
  const u64 j = local * T + threadIdx.x;
  U64x2 v{0, 0};
  u64 vres = 0;
  if (j < r) {
    if constexpr (PR) {
      if (A.pr.samples) A.pr.samples[(u64)kSampleFloats * (A.ref_off[p] + j) + 11] = 0.0f;
    }
    const u64 g_lo = A.pair_off[p];
    const Rec R = load_rec(A.ref + (A.ref_off[p] + p + 1 + j) * kRecBytes);
    u32 g = seg_lookup<CG>(A.seg, epoch, p, g_lo, pi[PI_M], R.w[0]);
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
      if constexpr (PR) {
        // the slot's prediction, its residual payload, and a training sample
        vres = b;
        u64* ps = A.pr.pscr + 4 * (A.ref_off[p] + j);
        bool ok = false;
        float f[kMlpIn];
        if (A.pr.hist && pi[PI_MODE] == TERA_MODE_XOR) {
          const Hist H = load_hist(A.pr.hist + kHistBytes * (A.ref_off[p] + j));
          const u32 nc = cell_count(A.pr.cseg, seg_base(A.ref_off[p], p), seg_size(r),
                                    cell_key(R, A.pr));
          if (features(R, H, nc, f)) {
            if (A.pr.samples) {
              float* s = A.pr.samples + (u64)kSampleFloats * (A.ref_off[p] + j);
#pragma unroll
              for (int i = 0; i < kMlpIn; ++i) s[i] = f[i];
#pragma unroll
              for (int a = 0; a < 3; ++a)
                s[kMlpIn + a] = __double2float_rn(
                    __dsub_rn(__longlong_as_double((long long)M.w[1 + a]),
                              __longlong_as_double((long long)R.w[1 + a])));
              s[11] = 1.0f;
            }
            if (A.pr.params) {
              u64 pred[3];
              ok = predict_from(sW, R, f, pred);
              if (ok) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                  vres += sig_bytes(zigzag(M.w[1 + a] - pred[a]));
                  vres -= sig_bytes(d.w[1 + a]);
                  ps[a] = pred[a];
                }
              }
            }
          }
        }
        ps[3] = ok ? 1ull : 0ull;
      }
    } else {
      code = 0xFu;  // placeholder
      if constexpr (PR) A.pr.pscr[4 * (A.ref_off[p] + j) + 3] = 0;
    }
    A.slot_src[A.ref_off[p] + j] = g;
    // with the predictor the message mode is chosen later: the slot codes
    // are written when the payload is
    if constexpr (!PR) reinterpret_cast<u32*>(A.wire + A.wire_off[p] + kHdrBytes)[j] = code;
  }
  U64x2 tot;
  block_excl_scan2(v, sm, &tot);
  if (threadIdx.x == 0) A.unit_sum[U] = tot;
  if constexpr (PR) {
    U64x2 tr;
    block_excl_scan2(U64x2{vres, 0}, sm, &tr);
    if (threadIdx.x == 0) A.pr.unit_res[U] = tr.a;
  }
}

// Message unit: records no slot took are new; (payload bytes, new records).
template <int T, bool CG>
__device__ __forceinline__ void enc_new_unit(const EncArgs& A, u32 p, u64 local, u64 U, u32 epoch,
                                             U64x2* sm) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 nst = pi[PI_NST];
  const u64 m = pi[PI_M];
  const u64 k = (local - nst) * T + threadIdx.x;
  U64x2 v{0, 0};
  if (k < m) {
    const u64 g = A.pair_off[p] + k;
    if (ldx<CG>(A.matched + g) != epoch) {
      const Rec M = load_rec(A.rec + (g + p + 1) * kRecBytes);
      // a second record with the same id in this pair would be found instead of this one
      if (seg_lookup<CG>(A.seg, epoch, p, A.pair_off[p], m, M.w[0]) != (u32)g)
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

// One warp: unit prefixes of pair p (units [u0, u0 + n_units)), header,
// padding, the new reference's header and the iteration totals.
template <bool CG, bool PR = false>
__device__ __forceinline__ void enc_scan_pair(const EncArgs& A, u32 p, u64 u0, u64 n_units) {
  const int lane = threadIdx.x & 31;
  u64* pi = A.info + (u64)p * 8;
  const u64 nst = pi[PI_NST];
  const u64 r = pi[PI_R], m = pi[PI_M];
  u64 mode = pi[PI_MODE];
  if constexpr (PR) {
    // residual mode when the predictor makes the slots' payload smaller
    u64 bx = 0, br = 0;
    for (u64 b = 0; b < nst; b += 32) {
      u64 i = b + lane;
      if (i < nst) {
        bx += ldx<CG>(A.unit_sum + u0 + i).a;
        br += ldx<CG>(A.pr.unit_res + u0 + i);
      }
    }
    bx = warp_sum(bx);
    br = warp_sum(br);
    if (A.pr.params && A.pr.allow_residual && mode == TERA_MODE_XOR && br < bx) mode = kModeResidual;
  }
  const bool res = PR && mode == kModeResidual;
  U64x2 run{0, 0};
  for (u64 b = 0; b < nst; b += 32) {
    u64 i = b + lane;
    U64x2 v = i < nst ? ldx<CG>(A.unit_sum + u0 + i) : U64x2{0, 0};
    if constexpr (PR) {
      if (res && i < nst) v.a = ldx<CG>(A.pr.unit_res + u0 + i);
    }
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
  const u64 nmt = n_units - nst;
  for (u64 b = 0; b < nmt; b += 32) {
    u64 i = b + lane;
    U64x2 v = i < nmt ? ldx<CG>(A.unit_sum + u0 + nst + i) : U64x2{0, 0};
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
    pi[PI_MODE] = mode;
    pi[PI_MATCHED] = matched;
    pi[PI_NEW] = n_new;
    pi[PI_SLOTPAY] = slot_pay;
    pi[PI_PAY] = payload;
    ulonglong2* h = reinterpret_cast<ulonglong2*>(w);
    h[0] = make_ulonglong2((u64)kWireMagic | ((u64)kVersion << 32) | ((u64)kRecBytes << 48),
                           (u64)A.class_id | (mode << 32));
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

__device__ __forceinline__ void stage_word(uint8_t* stage, u32& o, u64 v, u32 L) {
  for (u32 b = 0; b < L; ++b) stage[o++] = (uint8_t)(v >> (8 * b));
}

// Store stage[s0, s0 + nbytes) to gA (s0 = gA mod 16): aligned 16-byte stores
// inside, byte stores on the ragged edges shared with neighbouring units.
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

// Any unit: payload bytes (staged), codes of new records, new reference
// (with the predictor: also the slot codes, residual words and histories).
template <int T, bool CG, bool PR = false>
__device__ __forceinline__ void enc_emit_unit(const EncArgs& A, u32 p, u64 local, u64 U, u32 epoch,
                                              U64x2* sm, uint8_t* stage) {
  const u64* pi = A.info + (u64)p * 8;
  const u64 nst = pi[PI_NST], r = pi[PI_R];
  const u64 n_new = ldx<CG>(pi + PI_NEW);
  const bool slot_unit = local < nst;
  const u64 e = slot_unit ? local * T + threadIdx.x : (local - nst) * T + threadIdx.x;
  Rec d, cur, R;
  u32 L[8];
  U64x2 v{0, 0};
  u64 g = 0;
  if (slot_unit) {
    if (e < r) {
      u32 gg = ldx<CG>(A.slot_src + A.ref_off[p] + e);
      if (gg != kNoMatch) {
        g = gg;
        cur = load_rec(A.rec + (g + p + 1) * kRecBytes);
        R = load_rec(A.ref + (A.ref_off[p] + p + 1 + e) * kRecBytes);
#pragma unroll
        for (int w = 0; w < 8; ++w) d.w[w] = cur.w[w] ^ R.w[w];
        if constexpr (PR) {
          if (ldx<CG>(pi + PI_MODE) == kModeResidual) {
            const u64* ps = A.pr.pscr + 4 * (A.ref_off[p] + e);
            if (ldx<CG>(ps + 3)) {
#pragma unroll
              for (int a = 0; a < 3; ++a) d.w[1 + a] = zigzag(cur.w[1 + a] - ldx<CG>(ps + a));
            }
          }
        }
        u32 b = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          L[w] = sig_bytes(d.w[w]);
          b += L[w];
        }
        v = U64x2{b, 1};
      }
      if constexpr (PR) {
        u32 code = 0xFu;
        if (gg != kNoMatch) {
          code = 0;
#pragma unroll
          for (int w = 0; w < 8; ++w) code |= L[w] << (4 * w);
        }
        reinterpret_cast<u32*>(A.wire + A.wire_off[p] + kHdrBytes)[e] = code;
      }
    }
  } else if (e < pi[PI_M]) {
    g = A.pair_off[p] + e;
    if (ldx<CG>(A.matched + g) != epoch) {
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
  const U64x2 base = ldx<CG>(A.unit_base + U);
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
      pos = ldx<CG>(pi + PI_MATCHED) + rank;
    }
    if (in_bounds(A.st, pos, 0, A.pair_off[p + 1] - A.pair_off[p]))
      store_rec(A.ref_next + (A.pair_off[p] + p + 1 + pos) * kRecBytes, cur);
    if constexpr (PR) {
      if (A.pr.hist_next) {
        uint8_t* hn = A.pr.hist_next + kHistBytes * (A.pair_off[p] + pos);
        if (slot_unit) {
          if (A.pr.hist) {
            const Hist H = load_hist(A.pr.hist + kHistBytes * (A.ref_off[p] + e));
            store_hist_next(hn, &R, &H);
          } else {
            store_hist_next(hn, &R, nullptr);
          }
        } else {
          store_hist_next(hn, nullptr, nullptr);
        }
      }
    }
  }
  __syncthreads();
  flush_stage(stage, gA, tot.a);
  __syncthreads();
}

// ---------------- decode ----------------

// Returns false when the code is malformed for entry e; nibbles summed.
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

// Header facts of a received message.
struct DecHdr {
  u64 ns, nn, nh, pay, mode;
};

// Full header check of pair p's message; fills *H and returns the error (0
// when valid).  expect_m: when not ~0, the receive buffer size the caller
// laid out for p, which the header's count must equal.
template <bool CG, bool PR = false>
__device__ __forceinline__ u32 dec_read_header(const DecArgs& A, u32 p, u64 expect_m, DecHdr* H) {
  const u64 avail = A.wire_off[p + 1] - A.wire_off[p];
  const u64* h = reinterpret_cast<const u64*>(A.wire + A.wire_off[p]);
  u32 err = 0;
  u64 ns = 0, nn = 0, nh = 0, pay = 0, mode = 0;
  if (avail < kHdrBytes) {
    err = TERA_ECORRUPT;
  } else {
    const u64 w0 = ldx<CG>(h + 0), w1 = ldx<CG>(h + 1);
    ns = ldx<CG>(h + 2);
    nn = ldx<CG>(h + 3);
    nh = ldx<CG>(h + 4);
    pay = ldx<CG>(h + 5);
    const u64 w6 = ldx<CG>(h + 6), msg = ldx<CG>(h + 7);
    mode = w1 >> 32;
    const u64 r = A.ref ? A.ref_off[p + 1] - A.ref_off[p] : 0;
    if ((u32)w0 != kWireMagic || ((w0 >> 32) & 0xFFFF) != kVersion || (w0 >> 48) != kRecBytes ||
        (u32)w1 != A.class_id || w6 != (u64)p) {
      err = TERA_ECORRUPT;
    } else if (mode == TERA_MODE_XOR || (PR && A.pr.params && mode == kModeResidual)) {
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
      else if (expect_m != ~0ull && ns - nh + nn != expect_m)
        err = TERA_ECORRUPT;
    }
    if (!err && mode != TERA_MODE_RAW && A.ref) {
      // the receiver's reference buffer must be the one this message refers to
      const u64* rh = reinterpret_cast<const u64*>(A.ref + (A.ref_off[p] + p) * kRecBytes);
      if ((u32)rh[0] != kTaioMagic || (u32)rh[1] != A.class_id || (u32)(rh[1] >> 32) != p ||
          rh[2] != r)
        err = TERA_ECORRUPT;
    }
  }
  H->ns = ns;
  H->nn = nn;
  H->nh = nh;
  H->pay = pay;
  H->mode = mode;
  return err;
}

// dec_read_header, with the facts stored in the pair's decode info.
template <bool CG, bool PR = false>
__device__ __forceinline__ u32 dec_check_header(const DecArgs& A, u32 p, u64 expect_m) {
  DecHdr H;
  const u32 err = dec_read_header<CG, PR>(A, p, expect_m, &H);
  u64* pi = A.info + (u64)p * 8;
  pi[DI_NS] = H.ns;
  pi[DI_NN] = H.nn;
  pi[DI_NH] = H.nh;
  pi[DI_PAY] = H.pay;
  pi[DI_OK] = err ? 0 : 1;
  pi[DI_MODE] = H.mode;
  return err;
}

template <int T, bool CG>
__device__ __forceinline__ void dec_sum_unit(const DecArgs& A, u32 p, u64 local, u64 U,
                                             U64x2* sm) {
  u64* pi = A.info + (u64)p * 8;
  const u64 ns = ldx<CG>(pi + DI_NS), n = ns + ldx<CG>(pi + DI_NN);
  const bool ok = ldx<CG>(pi + DI_OK) != 0;
  const u64 e = local * T + threadIdx.x;
  U64x2 v{0, 0};
  if (ok && e < n) {
    const u32 code =
        ldx<CG>(reinterpret_cast<const u32*>(A.wire + A.wire_off[p] + kHdrBytes) + e);
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

// One warp: unit prefixes, totals checked against the header, receive header.
template <bool CG>
__device__ __forceinline__ void dec_scan_pair(const DecArgs& A, u32 p, u64 u0, u64 n_units) {
  const int lane = threadIdx.x & 31;
  u64* pi = A.info + (u64)p * 8;
  U64x2 run{0, 0};
  for (u64 b = 0; b < n_units; b += 32) {
    u64 i = b + lane;
    U64x2 v = i < n_units ? ldx<CG>(A.unit_sum + u0 + i) : U64x2{0, 0};
    U64x2 incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      U64x2 t = shfl_up(incl, o);
      if (lane >= o) incl += t;
    }
    if (i < n_units) A.unit_base[u0 + i] = run + incl - v;
    run += U64x2{__shfl_sync(0xFFFFFFFFu, incl.a, 31), __shfl_sync(0xFFFFFFFFu, incl.b, 31)};
  }
  const u64 m = A.recv_off[p + 1] - A.recv_off[p];
  if (lane == 0) {
    if (ldx<CG>(pi + DI_OK) && (run.a != ldx<CG>(pi + DI_PAY) || run.b != m)) {
      latch(A.st, TERA_ECORRUPT);
      pi[DI_OK] = 0;
    }
    write_taio_header(A.recv + (A.recv_off[p] + p) * kRecBytes, A.class_id, p, m);
  }
}

template <int T, bool CG, bool PR = false>
__device__ __forceinline__ void dec_emit_unit(const DecArgs& A, u32 p, u64 local, u64 U,
                                              U64x2* sm, uint8_t* stage,
                                              const float* sW = nullptr) {
  const u64* pi = A.info + (u64)p * 8;
  if (!ldx<CG>(pi + DI_OK)) return;  // block-uniform
  const u64 ns = ldx<CG>(pi + DI_NS), n = ns + ldx<CG>(pi + DI_NN);
  const u64 e = local * T + threadIdx.x;
  const uint8_t* w8 = A.wire + A.wire_off[p];
  u32 code = 0;
  u32 b = 0;
  bool hole = true;
  if (e < n) {
    code = ldx<CG>(reinterpret_cast<const u32*>(w8 + kHdrBytes) + e);
    check_code(code, e, ns, &hole, &b);
  }
  U64x2 v{b, (e < n && !hole) ? 1ull : 0ull};
  U64x2 tot;
  U64x2 ex = block_excl_scan2(v, sm, &tot);
  const U64x2 base = ldx<CG>(A.unit_base + U);
  // stage [gA, gA + tot.a) with 16-byte loads; the slab is 16-byte aligned and
  // padded, so the rounded range stays inside this pair's slab
  const uint8_t* gA = w8 + kHdrBytes + 4 * n + base.a;
  const u32 s0 = (u32)((uintptr_t)gA & 15u);
  const uint8_t* g16 = gA - s0;
  const u32 nchunks = (u32)((s0 + tot.a + 15u) >> 4);
  for (u32 c = threadIdx.x; c < nchunks; c += blockDim.x)
    *reinterpret_cast<uint4*>(stage + (c << 4)) =
        ldx<CG>(reinterpret_cast<const uint4*>(g16 + (c << 4)));
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
    const u64 pos = base.b + ex.b;
    if (e < ns) {
      const Rec R = load_rec(A.ref + (A.ref_off[p] + p + 1 + e) * kRecBytes);
      bool pred_ok = false;
      u64 pred[3];
      if constexpr (PR) {
        Hist H;
        if (A.pr.hist) H = load_hist(A.pr.hist + kHistBytes * (A.ref_off[p] + e));
        if (A.pr.hist && ldx<CG>(pi + DI_MODE) == kModeResidual) {
          const u64 r = A.ref_off[p + 1] - A.ref_off[p];
          const u32 nc = cell_count(A.pr.cseg, seg_base(A.ref_off[p], p), seg_size(r),
                                    cell_key(R, A.pr));
          float f[kMlpIn];
          if (features(R, H, nc, f)) pred_ok = predict_from(sW, R, f, pred);
        }
        if (A.pr.hist_next)
          store_hist_next(A.pr.hist_next + kHistBytes * (A.recv_off[p] + pos), &R,
                          A.pr.hist ? &H : nullptr);
      }
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        if (pred_ok && w >= 1 && w <= 3) rec.w[w] = pred[w - 1] + unzigzag(rec.w[w]);
        else rec.w[w] ^= R.w[w];
      }
    } else {
      if constexpr (PR) {
        if (A.pr.hist_next)
          store_hist_next(A.pr.hist_next + kHistBytes * (A.recv_off[p] + pos), nullptr, nullptr);
      }
    }
    if (in_bounds(A.st, pos, 0, A.recv_off[p + 1] - A.recv_off[p]))
      store_rec(A.recv + (A.recv_off[p] + p + 1 + pos) * kRecBytes, rec);
  }
  __syncthreads();
}

}  // namespace tera
