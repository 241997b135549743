/*
 * Oracle for the aura-exchange codec.  TEST INFRASTRUCTURE ONLY (see
 * tera_oracle.h): plain loops, one agent or record at a time, in the order the
 * paper describes the steps.  No blocking, fusion or reordering.
 *
 * Paper sections followed:
 *   Sec. 2.1  "Aura Update": partitioning grid, aura = agents within the
 *             interaction distance of a neighbouring box.
 *   Sec. 2.2.1 TeraAgent IO: serialization copies each block into one
 *             contiguous buffer; the class identity is written once; the
 *             receiver reinterprets the buffer in place.
 *   Sec. 2.3  Data transfer minimization: per sender/receiver-pair reference,
 *             matching/reorder (B), difference serialization (C), restore and
 *             defragmentation (D).
 *   Sec. 3.11 compression after the difference (LZ4 in the paper; here the
 *             significant-byte packer defined below).
 */
#define _POSIX_C_SOURCE 199309L
#include "tera_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define REC_WORDS 8
#define REC_BYTES 64
#define TAIO_MAGIC 0x4F494154u /* bytes 'T','A','I','O' */
#define WIRE_MAGIC 0x41524554u /* bytes 'T','E','R','A' */
#define FMT_VERSION 1u
#define HDR_BYTES 64u

/* ---------- little-endian byte helpers (explicit, no type punning) ---------- */

static uint64_t get_le(const uint8_t* p, int nbytes) {
  uint64_t v = 0;
  for (int b = 0; b < nbytes; ++b) v |= (uint64_t)p[b] << (8 * b);
  return v;
}

static void put_le(uint8_t* p, uint64_t v, int nbytes) {
  for (int b = 0; b < nbytes; ++b) p[b] = (uint8_t)(v >> (8 * b));
}

static uint64_t rec_word(const uint8_t* rec, int w) { return get_le(rec + 8 * w, 8); }

static uint64_t f64_bits(double d) {
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
}

/* ---------- grid (Sec. 2.1; Sec. 2.4 "Partitioning Grid") ---------- */

int or_grid_check(const or_grid* g) {
  if (g->reserved != 0 || (g->periodic & ~7u) != 0) return OR_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1) return OR_EINVAL;
    if (!(g->lo[a] < g->hi[a])) return OR_EINVAL;
    /* on a toroidal axis the two neighbours of a box must be two other
     * boxes, so that a neighbour offset names one box */
    if ((g->periodic >> a & 1u) && g->n[a] < 3) return OR_EINVAL;
  }
  /* The aura must be narrower than a partitioning box (Sec. 2.1): w is
   * positive and below the smallest box side on every axis. */
  if (!(g->w > 0.0)) return OR_EINVAL;
  for (int a = 0; a < 3; ++a) {
    int n = g->n[a];
    double* e = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    if (!e) return OR_ENOMEM;
    or_axis_edges(g, a, e);
    for (int k = 0; k < n; ++k) {
      if (!(g->w < e[k + 1] - e[k])) {
        free(e);
        return OR_EINVAL;
      }
    }
    free(e);
  }
  return OR_OK;
}

/* Box edges along one axis: e[k] = lo + ((hi - lo) * k) / n, and e[n] = hi. */
void or_axis_edges(const or_grid* g, int axis, double* e) {
  int n = g->n[axis];
  double lo = g->lo[axis], hi = g->hi[axis];
  for (int k = 0; k < n; ++k) e[k] = lo + ((hi - lo) * (double)k) / (double)n;
  e[n] = hi;
}

/* ---------- O1: classification (Sec. 2.1 "Aura Update") ----------
 * Ownership is half-open [e[i], e[i+1]).  An agent is in the aura of the
 * neighbour box at offset o (per axis -1, 0, +1) when it lies within w of that
 * box in the L-infinity sense: for o = -1, x < e[i] + w; for o = +1,
 * x >= e[i+1] - w; o = 0 always qualifies.  The neighbour must exist: on a
 * closed axis box 0 has no -1 neighbour and box n-1 no +1 neighbour; on a
 * toroidal axis (Sec. 2.5) the neighbour index wraps modulo n. */
int or_classify(const or_grid* g, const double* x, const double* y, const double* z,
                int64_t n, int32_t* owner, uint32_t* mask) {
  int st = or_grid_check(g);
  if (st != OR_OK) return st;
  double* edges[3];
  for (int a = 0; a < 3; ++a) {
    edges[a] = (double*)malloc(sizeof(double) * (size_t)(g->n[a] + 1));
    or_axis_edges(g, a, edges[a]);
  }
  int status = OR_OK;
  for (int64_t i = 0; i < n; ++i) {
    double v[3] = {x[i], y[i], z[i]};
    int idx[3];
    int qual[3][3]; /* qual[axis][o + 1] */
    int inside = 1;
    for (int a = 0; a < 3; ++a) {
      if (!(v[a] >= g->lo[a] && v[a] < g->hi[a])) inside = 0; /* NaN fails too */
    }
    if (!inside) {
      owner[i] = -1;
      mask[i] = 0;
      status = OR_EDOMAIN;
      continue;
    }
    for (int a = 0; a < 3; ++a) {
      const double* e = edges[a];
      int na = g->n[a];
      int cnt = 0;
      for (int k = 1; k <= na - 1; ++k)
        if (v[a] >= e[k]) ++cnt;
      idx[a] = cnt;
      int wrap = (int)(g->periodic >> a & 1u);
      qual[a][0] = (cnt > 0 || wrap) && (v[a] < e[cnt] + g->w);
      qual[a][1] = 1;
      qual[a][2] = (cnt < na - 1 || wrap) && (v[a] >= e[cnt + 1] - g->w);
    }
    owner[i] = idx[0] + g->n[0] * (idx[1] + g->n[1] * idx[2]);
    uint32_t m = 0;
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (ox == 0 && oy == 0 && oz == 0) continue;
          if (qual[0][ox + 1] && qual[1][oy + 1] && qual[2][oz + 1]) {
            int bit = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
            m |= 1u << bit;
          }
        }
    mask[i] = m;
  }
  for (int a = 0; a < 3; ++a) free(edges[a]);
  return status;
}

/* Per-pair lists: for agent i in ascending order and each set bit b in
 * ascending order, append i to the list of pair owner(i)*27 + b. */
int or_pair_lists(const or_grid* g, const int32_t* owner, const uint32_t* mask, int64_t n,
                  uint64_t* pair_count, uint64_t* pair_off, uint32_t* pair_idx,
                  uint64_t idx_capacity) {
  uint64_t n_pairs = (uint64_t)g->n[0] * (uint64_t)g->n[1] * (uint64_t)g->n[2] * 27u;
  for (uint64_t p = 0; p < n_pairs; ++p) pair_count[p] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (owner[i] < 0) continue;
    for (int b = 0; b < 27; ++b)
      if (mask[i] >> b & 1u) pair_count[(uint64_t)owner[i] * 27u + (uint64_t)b] += 1;
  }
  pair_off[0] = 0;
  for (uint64_t p = 0; p < n_pairs; ++p) pair_off[p + 1] = pair_off[p] + pair_count[p];
  if (pair_off[n_pairs] > idx_capacity) return OR_ECAPACITY;
  uint64_t* fill = (uint64_t*)calloc(n_pairs ? n_pairs : 1, sizeof(uint64_t));
  if (!fill) return OR_ENOMEM;
  for (int64_t i = 0; i < n; ++i) {
    if (owner[i] < 0) continue;
    for (int b = 0; b < 27; ++b) {
      if (!(mask[i] >> b & 1u)) continue;
      uint64_t p = (uint64_t)owner[i] * 27u + (uint64_t)b;
      pair_idx[pair_off[p] + fill[p]] = (uint32_t)i;
      fill[p] += 1;
    }
  }
  free(fill);
  return OR_OK;
}

/* ---------- O2: serialization (Sec. 2.2.1 "Serialization") ----------
 * Arena layout: pair p occupies 64-byte units [pair_off[p] + p,
 * pair_off[p+1] + p + 1): one buffer header (class id written once, as the
 * paper replaces the vtable pointer by a class identifier), then its records. */
static void write_taio_header(uint8_t* h, uint32_t class_id, uint32_t pair, uint64_t n) {
  memset(h, 0, HDR_BYTES);
  put_le(h + 0, TAIO_MAGIC, 4);
  put_le(h + 4, FMT_VERSION, 2);
  put_le(h + 6, REC_BYTES, 2);
  put_le(h + 8, class_id, 4);
  put_le(h + 12, pair, 4);
  put_le(h + 16, n, 8);
}

void or_pack(const uint64_t* id, const double* const cols[7], uint64_t n_pairs,
             const uint64_t* pair_off, const uint32_t* pair_idx, uint32_t class_id,
             uint8_t* arena) {
  or_pack_range(id, cols, 0, n_pairs, pair_off, pair_idx, class_id, arena);
}

/* or_pack for pairs [p0, p1) only (the arena layout is that of all pairs). */
void or_pack_range(const uint64_t* id, const double* const cols[7], uint64_t p0, uint64_t p1,
                   const uint64_t* pair_off, const uint32_t* pair_idx, uint32_t class_id,
                   uint8_t* arena) {
  for (uint64_t p = p0; p < p1; ++p) {
    uint8_t* buf = arena + (pair_off[p] + p) * REC_BYTES;
    uint64_t m = pair_off[p + 1] - pair_off[p];
    write_taio_header(buf, class_id, (uint32_t)p, m);
    for (uint64_t k = 0; k < m; ++k) {
      uint32_t i = pair_idx[pair_off[p] + k];
      uint8_t* rec = buf + HDR_BYTES + k * REC_BYTES;
      put_le(rec, id[i], 8);
      for (int c = 0; c < 7; ++c) put_le(rec + 8 * (c + 1), f64_bits(cols[c][i]), 8);
    }
  }
}

/* ---------- O4: significant-byte length of one word ----------
 * L = number of low-order bytes needed to hold the value (0 for zero). */
static int sig_bytes(uint64_t v) {
  int L = 0;
  while (v != 0) {
    L += 1;
    v >>= 8;
  }
  return L;
}

/* ---------- O3 + O4: encode one pair (Sec. 2.3 steps B and C) ---------- */

typedef struct {
  uint64_t id;
  uint64_t k;
} id_pos;

static int cmp_id_pos(const void* a, const void* b) {
  uint64_t x = ((const id_pos*)a)->id, y = ((const id_pos*)b)->id;
  return (x > y) - (x < y);
}

/* Index of the message record with this id, or -1. */
static int64_t find_id(const id_pos* sorted, uint64_t m, uint64_t id) {
  uint64_t lo = 0, hi = m;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (sorted[mid].id < id) lo = mid + 1;
    else hi = mid;
  }
  if (lo < m && sorted[lo].id == id) return (int64_t)sorted[lo].k;
  return -1;
}

static uint64_t round16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

static void write_wire_header(uint8_t* h, uint32_t class_id, uint32_t mode, uint64_t n_slots,
                              uint64_t n_new, uint64_t n_holes, uint64_t payload,
                              uint32_t pair, uint64_t msg_bytes) {
  memset(h, 0, HDR_BYTES);
  put_le(h + 0, WIRE_MAGIC, 4);
  put_le(h + 4, FMT_VERSION, 2);
  put_le(h + 6, REC_BYTES, 2);
  put_le(h + 8, class_id, 4);
  put_le(h + 12, mode, 4);
  put_le(h + 16, n_slots, 8);
  put_le(h + 24, n_new, 8);
  put_le(h + 32, n_holes, 8);
  put_le(h + 40, payload, 8);
  put_le(h + 48, pair, 4);
  put_le(h + 56, msg_bytes, 8);
}

enum { KIND_MATCH = 0, KIND_HOLE = 1, KIND_NEW = 2 };

int or_encode_pair(const uint8_t* msg, uint64_t m, const uint8_t* ref, uint64_t r,
                   uint32_t class_id, uint32_t mode, uint32_t pair, uint8_t* wire,
                   uint64_t wire_cap, uint64_t* wire_len, uint8_t* ref_next) {
  if (mode != OR_MODE_RAW && mode != OR_MODE_XOR) return OR_EINVAL;
  if (mode == OR_MODE_RAW) r = 0; /* no reference: every record is new */

  /* Step B (matching): a map from id to message position. */
  id_pos* sorted = (id_pos*)malloc(sizeof(id_pos) * (size_t)(m ? m : 1));
  uint8_t* matched = (uint8_t*)calloc(m ? m : 1, 1);
  int64_t* src = (int64_t*)malloc(sizeof(int64_t) * (size_t)(r ? r : 1));
  int status = OR_OK;
  if (!sorted || !matched || !src) {
    status = OR_ENOMEM;
    goto done;
  }
  for (uint64_t k = 0; k < m; ++k) {
    sorted[k].id = rec_word(msg + k * REC_BYTES, 0);
    sorted[k].k = k;
  }
  qsort(sorted, (size_t)m, sizeof(id_pos), cmp_id_pos);
  for (uint64_t k = 1; k < m; ++k)
    if (sorted[k].id == sorted[k - 1].id) {
      status = OR_EINVAL; /* ids must be unique within a message */
      goto done;
    }
  /* Reference slot j keeps its position: it is matched with the message
   * record carrying the same id, else it becomes a placeholder (hole). */
  uint64_t n_holes = 0;
  for (uint64_t j = 0; j < r; ++j) {
    int64_t k = find_id(sorted, m, rec_word(ref + j * REC_BYTES, 0));
    src[j] = k;
    if (k < 0) {
      n_holes += 1;
    } else {
      if (matched[k]) {
        status = OR_EINVAL; /* duplicate id in the reference */
        goto done;
      }
      matched[k] = 1;
    }
  }
  /* Records absent from the reference are appended in message order. */
  uint64_t n_new = 0;
  for (uint64_t k = 0; k < m; ++k)
    if (!matched[k]) n_new += 1;
  uint64_t n_codes = r + n_new;

  /* Step C (difference) + byte packing: first the sizes, then the bytes. */
  uint64_t payload = 0;
  for (uint64_t j = 0; j < r; ++j) {
    if (src[j] < 0) continue; /* hole: no payload */
    const uint8_t* cur = msg + (uint64_t)src[j] * REC_BYTES;
    for (int w = 0; w < REC_WORDS; ++w)
      payload += (uint64_t)sig_bytes(rec_word(cur, w) ^ rec_word(ref + j * REC_BYTES, w));
  }
  for (uint64_t k = 0; k < m; ++k) {
    if (matched[k]) continue;
    for (int w = 0; w < REC_WORDS; ++w)
      payload += (uint64_t)sig_bytes(rec_word(msg + k * REC_BYTES, w));
  }
  uint64_t msg_bytes = round16(HDR_BYTES + 4u * n_codes + payload);
  *wire_len = msg_bytes;
  if (msg_bytes > wire_cap) {
    status = OR_ECAPACITY;
    goto done;
  }
  memset(wire, 0, (size_t)msg_bytes);
  write_wire_header(wire, class_id, mode, r, n_new, n_holes, payload, pair, msg_bytes);
  uint8_t* codes = wire + HDR_BYTES;
  uint8_t* pay = wire + HDR_BYTES + 4u * n_codes;
  uint64_t off = 0;
  uint64_t e = 0;
  /* Reference slots, in slot order. */
  for (uint64_t j = 0; j < r; ++j, ++e) {
    if (src[j] < 0) {
      put_le(codes + 4 * e, 0xFu, 4); /* placeholder: word-0 code 0xF */
      continue;
    }
    const uint8_t* cur = msg + (uint64_t)src[j] * REC_BYTES;
    const uint8_t* base = ref + j * REC_BYTES;
    uint32_t code = 0;
    for (int w = 0; w < REC_WORDS; ++w) {
      uint64_t d = rec_word(cur, w) ^ rec_word(base, w);
      int L = sig_bytes(d);
      code |= (uint32_t)L << (4 * w);
      put_le(pay + off, d, L);
      off += (uint64_t)L;
    }
    put_le(codes + 4 * e, code, 4);
  }
  /* New records, in message order, written raw. */
  for (uint64_t k = 0; k < m; ++k) {
    if (matched[k]) continue;
    const uint8_t* cur = msg + k * REC_BYTES;
    uint32_t code = 0;
    for (int w = 0; w < REC_WORDS; ++w) {
      uint64_t d = rec_word(cur, w);
      int L = sig_bytes(d);
      code |= (uint32_t)L << (4 * w);
      put_le(pay + off, d, L);
      off += (uint64_t)L;
    }
    put_le(codes + 4 * e, code, 4);
    e += 1;
  }
  /* New sender reference: matched records (current values) in slot order,
   * then the new records; the same sequence the receiver reconstructs. */
  {
    uint64_t q = 0;
    for (uint64_t j = 0; j < r; ++j) {
      if (src[j] < 0) continue;
      memcpy(ref_next + q * REC_BYTES, msg + (uint64_t)src[j] * REC_BYTES, REC_BYTES);
      q += 1;
    }
    for (uint64_t k = 0; k < m; ++k) {
      if (matched[k]) continue;
      memcpy(ref_next + q * REC_BYTES, msg + k * REC_BYTES, REC_BYTES);
      q += 1;
    }
  }
done:
  free(sorted);
  free(matched);
  free(src);
  return status;
}

/* ---------- O5: decode one pair (Sec. 2.3 step D) ---------- */
int or_decode_pair(const uint8_t* wire, uint64_t wire_avail, const uint8_t* ref, uint64_t r,
                   uint32_t class_id, uint32_t pair, uint8_t* out, uint64_t out_cap,
                   uint64_t* m_out) {
  *m_out = 0;
  if (wire_avail < HDR_BYTES) return OR_ECORRUPT;
  if (get_le(wire + 0, 4) != WIRE_MAGIC) return OR_ECORRUPT;
  if (get_le(wire + 4, 2) != FMT_VERSION) return OR_ECORRUPT;
  if (get_le(wire + 6, 2) != REC_BYTES) return OR_ECORRUPT;
  if (get_le(wire + 8, 4) != class_id) return OR_ECORRUPT;
  if (get_le(wire + 48, 4) != pair) return OR_ECORRUPT;
  uint64_t mode = get_le(wire + 12, 4);
  uint64_t n_slots = get_le(wire + 16, 8);
  uint64_t n_new = get_le(wire + 24, 8);
  uint64_t n_holes = get_le(wire + 32, 8);
  uint64_t payload = get_le(wire + 40, 8);
  uint64_t msg_bytes = get_le(wire + 56, 8);
  if (mode == OR_MODE_RAW) {
    if (n_slots != 0) return OR_ECORRUPT;
  } else if (mode == OR_MODE_XOR) {
    if (n_slots != r) return OR_EREFMISMATCH;
  } else {
    return OR_ECORRUPT;
  }
  if (n_slots > wire_avail || n_new > wire_avail || payload > wire_avail) return OR_ECORRUPT;
  uint64_t n_codes = n_slots + n_new;
  if (msg_bytes != round16(HDR_BYTES + 4u * n_codes + payload)) return OR_ECORRUPT;
  if (msg_bytes > wire_avail) return OR_ECORRUPT;
  const uint8_t* codes = wire + HDR_BYTES;
  const uint8_t* pay = wire + HDR_BYTES + 4u * n_codes;
  uint64_t off = 0, holes = 0, count = 0;
  for (uint64_t e = 0; e < n_codes; ++e) {
    uint32_t code = (uint32_t)get_le(codes + 4 * e, 4);
    if ((code & 0xFu) == 0xFu) {
      /* placeholder: only in a reference slot, and no other nibble set */
      if (e >= n_slots || (code >> 4) != 0) return OR_ECORRUPT;
      holes += 1;
      continue;
    }
    for (int w = 0; w < REC_WORDS; ++w)
      if (((code >> (4 * w)) & 0xFu) > 8u) return OR_ECORRUPT;
    if (e < n_slots && (code & 0xFu) != 0) return OR_ECORRUPT; /* same id => zero delta */
    if (count >= out_cap) return OR_ECAPACITY;
    uint8_t* rec = out + count * REC_BYTES;
    for (int w = 0; w < REC_WORDS; ++w) {
      int L = (int)((code >> (4 * w)) & 0xFu);
      if (off + (uint64_t)L > payload) return OR_ECORRUPT;
      uint64_t d = get_le(pay + off, L); /* zero-extended */
      off += (uint64_t)L;
      uint64_t v = (e < n_slots) ? (d ^ rec_word(ref + e * REC_BYTES, w)) : d;
      put_le(rec + 8 * w, v, 8);
    }
    count += 1;
  }
  if (off != payload) return OR_ECORRUPT;
  if (holes != n_holes) return OR_ECORRUPT;
  *m_out = count;
  return OR_OK;
}

/* ---------- arena drivers ---------- */

/* Wire slab of pair p: an upper bound on its message, so that every message
 * has a fixed place before its size is known:
 *   round16(64 + 4 (r_p + m_p) + 64 m_p). */
void or_wire_slabs(uint64_t n_pairs, const uint64_t* pair_off, const uint64_t* ref_off,
                   uint64_t* wire_off) {
  wire_off[0] = 0;
  for (uint64_t p = 0; p < n_pairs; ++p) {
    uint64_t m = pair_off[p + 1] - pair_off[p];
    uint64_t r = ref_off ? ref_off[p + 1] - ref_off[p] : 0;
    wire_off[p + 1] = wire_off[p] + round16(HDR_BYTES + 4u * (r + m) + REC_BYTES * m);
  }
}

static int check_taio_header(const uint8_t* h, uint32_t class_id, uint32_t pair, uint64_t n) {
  if (get_le(h + 0, 4) != TAIO_MAGIC) return OR_ECORRUPT;
  if (get_le(h + 4, 2) != FMT_VERSION) return OR_ECORRUPT;
  if (get_le(h + 6, 2) != REC_BYTES) return OR_ECORRUPT;
  if (get_le(h + 8, 4) != class_id) return OR_ECORRUPT;
  if (get_le(h + 12, 4) != pair) return OR_ECORRUPT;
  if (get_le(h + 16, 8) != n) return OR_ECORRUPT;
  return OR_OK;
}

int or_encode_all(uint64_t n_pairs, uint32_t class_id, uint32_t mode, const uint8_t* rec_arena,
                  const uint64_t* pair_off, const uint8_t* ref_arena, const uint64_t* ref_off,
                  const uint8_t* reset, uint8_t* wire, const uint64_t* wire_off,
                  uint64_t* wire_len, uint8_t* ref_next) {
  return or_encode_range(0, n_pairs, class_id, mode, rec_arena, pair_off, ref_arena, ref_off,
                         reset, wire, wire_off, wire_len, ref_next);
}

/* or_encode_all for pairs [p0, p1) only; the status of the first failing pair. */
int or_encode_range(uint64_t p0, uint64_t p1, uint32_t class_id, uint32_t mode,
                    const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_arena,
                    const uint64_t* ref_off, const uint8_t* reset, uint8_t* wire,
                    const uint64_t* wire_off, uint64_t* wire_len, uint8_t* ref_next) {
  int status = OR_OK;
  for (uint64_t p = p0; p < p1; ++p) {
    uint64_t m = pair_off[p + 1] - pair_off[p];
    uint64_t r = ref_arena ? ref_off[p + 1] - ref_off[p] : 0;
    const uint8_t* msg_buf = rec_arena + (pair_off[p] + p) * REC_BYTES;
    const uint8_t* ref_buf = ref_arena ? ref_arena + (ref_off[p] + p) * REC_BYTES : NULL;
    int st = check_taio_header(msg_buf, class_id, (uint32_t)p, m);
    if (st == OR_OK && ref_buf && mode != OR_MODE_RAW && !(reset && reset[p]))
      st = check_taio_header(ref_buf, class_id, (uint32_t)p, r);
    uint32_t pm = (reset && reset[p]) ? (uint32_t)OR_MODE_RAW : mode;
    uint8_t* nxt = ref_next + (pair_off[p] + p) * REC_BYTES;
    if (st == OR_OK) {
      write_taio_header(nxt, class_id, (uint32_t)p, m);
      st = or_encode_pair(msg_buf + HDR_BYTES, m, ref_buf ? ref_buf + HDR_BYTES : NULL, r,
                          class_id, pm,
                          (uint32_t)p, wire + wire_off[p], wire_off[p + 1] - wire_off[p],
                          &wire_len[p], nxt + HDR_BYTES);
    } else {
      wire_len[p] = 0;
    }
    if (st != OR_OK && status == OR_OK) status = st;
  }
  return status;
}

/* Receive-buffer sizes come from the headers: m_p = n_slots - n_holes + n_new
 * (0 for a header that cannot be read); recv_off[P+1] is their prefix. */
void or_recv_layout(uint64_t n_pairs, const uint8_t* wire, const uint64_t* wire_off,
                    uint64_t* recv_off) {
  recv_off[0] = 0;
  for (uint64_t p = 0; p < n_pairs; ++p) {
    const uint8_t* h = wire + wire_off[p];
    uint64_t avail = wire_off[p + 1] - wire_off[p];
    uint64_t m = 0;
    if (avail >= HDR_BYTES && get_le(h, 4) == WIRE_MAGIC) {
      uint64_t ns = get_le(h + 16, 8), nn = get_le(h + 24, 8), nh = get_le(h + 32, 8);
      if (nh <= ns && ns <= avail && nn <= avail) m = ns - nh + nn;
    }
    recv_off[p + 1] = recv_off[p] + m;
  }
}

int or_decode_all(uint64_t n_pairs, uint32_t class_id, const uint8_t* wire,
                  const uint64_t* wire_off, const uint8_t* ref_arena, const uint64_t* ref_off,
                  uint8_t* recv, uint64_t recv_cap_units, uint64_t* recv_off) {
  or_recv_layout(n_pairs, wire, wire_off, recv_off);
  if (recv_off[n_pairs] + n_pairs > recv_cap_units) return OR_ECAPACITY;
  return or_decode_range(0, n_pairs, class_id, wire, wire_off, ref_arena, ref_off, recv,
                         recv_off);
}

/* The per-pair part of or_decode_all for pairs [p0, p1), once recv_off is laid
 * out (and checked against the capacity) for all pairs. */
int or_decode_range(uint64_t p0, uint64_t p1, uint32_t class_id, const uint8_t* wire,
                    const uint64_t* wire_off, const uint8_t* ref_arena, const uint64_t* ref_off,
                    uint8_t* recv, const uint64_t* recv_off) {
  int status = OR_OK;
  for (uint64_t p = p0; p < p1; ++p) {
    uint64_t r = ref_arena ? ref_off[p + 1] - ref_off[p] : 0;
    const uint8_t* ref_buf = ref_arena ? ref_arena + (ref_off[p] + p) * REC_BYTES : NULL;
    uint8_t* out = recv + (recv_off[p] + p) * REC_BYTES;
    uint64_t cap = recv_off[p + 1] - recv_off[p];
    uint64_t got = 0;
    int st = OR_OK;
    uint64_t avail = wire_off[p + 1] - wire_off[p];
    int uses_ref = avail >= HDR_BYTES && get_le(wire + wire_off[p] + 12, 4) == OR_MODE_XOR;
    if (ref_buf && uses_ref) st = check_taio_header(ref_buf, class_id, (uint32_t)p, r);
    if (st == OR_OK)
      st = or_decode_pair(wire + wire_off[p], avail, ref_buf ? ref_buf + HDR_BYTES : NULL, r,
                          class_id, (uint32_t)p, out + HDR_BYTES, cap, &got);
    if (st == OR_OK && got != cap) st = OR_ECORRUPT;
    write_taio_header(out, class_id, (uint32_t)p, cap);
    if (st != OR_OK && status == OR_OK) status = st;
  }
  return status;
}

/* ---------- whole iteration (CPU baseline) ---------- */


static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* The difference-serialized message of Sec. 2.3 (steps B and C) before the
 * compression stage: entry e < r is reference slot e, the XOR of the current
 * record with the slot's id and the slot's record, or 64 zero bytes for a
 * placeholder; entries r .. r+a-1 are the records absent from the
 * reference, raw, in message order.  This is what a general-purpose
 * compressor (LZ4 in the paper, Sec. 3.11) is given after the difference
 * encoding.  out holds r + m entries at most; *n_entries = r + a. */
int or_delta_records(const uint8_t* msg, uint64_t m, const uint8_t* ref, uint64_t r,
                     uint8_t* out, uint64_t* n_entries) {
  id_pos* sorted = (id_pos*)malloc(sizeof(id_pos) * (size_t)(m ? m : 1));
  uint8_t* matched = (uint8_t*)calloc(m ? m : 1, 1);
  int status = OR_OK;
  if (!sorted || !matched) {
    status = OR_ENOMEM;
    goto done;
  }
  for (uint64_t k = 0; k < m; ++k) {
    sorted[k].id = rec_word(msg + k * REC_BYTES, 0);
    sorted[k].k = k;
  }
  qsort(sorted, (size_t)m, sizeof(id_pos), cmp_id_pos);
  uint64_t e = 0;
  for (uint64_t j = 0; j < r; ++j, ++e) {
    uint8_t* o = out + e * REC_BYTES;
    int64_t k = find_id(sorted, m, rec_word(ref + j * REC_BYTES, 0));
    if (k < 0) {
      memset(o, 0, REC_BYTES);
      continue;
    }
    matched[k] = 1;
    for (int w = 0; w < REC_WORDS; ++w)
      put_le(o + 8 * w, rec_word(msg + (uint64_t)k * REC_BYTES, w) ^ rec_word(ref + j * REC_BYTES, w),
             8);
  }
  for (uint64_t k = 0; k < m; ++k) {
    if (matched[k]) continue;
    memcpy(out + e * REC_BYTES, msg + k * REC_BYTES, REC_BYTES);
    e += 1;
  }
  *n_entries = e;
done:
  free(sorted);
  free(matched);
  return status;
}

/* ---------- agent migration (Sec. 2.1 "Agent Migration") ----------
 * Agents whose new position lies in another box move to that box; they are
 * sent as raw TeraAgent IO records (Sec. 2.2.1), the difference encoding of
 * Sec. 2.3 being for the aura only.  On one grid the destination of every
 * agent is its owner box by the classification rule, so the paper's second
 * case (a collective lookup for positions outside the locally available boxes)
 * reduces to the same rule; such agents use the inbox side b = 13. */

static void box_coords(const or_grid* g, int32_t b, int c[3]) {
  c[0] = b % g->n[0];
  c[1] = (b / g->n[0]) % g->n[1];
  c[2] = b / (g->n[0] * g->n[1]);
}

/* Side of box d that an agent from box s arrives from: the neighbour bit of
 * the offset s - d (per axis -1, 0 or +1, taken modulo n on a toroidal axis),
 * or 13 when s is not one of d's 26 neighbours. */
int or_migrate_inbox_bit(const or_grid* g, int32_t s, int32_t d) {
  int cs[3], cd[3], o[3];
  box_coords(g, s, cs);
  box_coords(g, d, cd);
  for (int a = 0; a < 3; ++a) {
    int diff = cs[a] - cd[a];
    if (g->periodic >> a & 1u) {
      int na = g->n[a];
      if (diff == na - 1) diff = -1;
      else if (diff == -(na - 1)) diff = 1;
    }
    if (diff < -1 || diff > 1) return 13;
    o[a] = diff;
  }
  return (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
}

static int check_box_off(const uint64_t* box_off, uint64_t n_boxes, int64_t n) {
  if (box_off[0] != 0 || box_off[n_boxes] != (uint64_t)n) return OR_EINVAL;
  for (uint64_t b = 0; b < n_boxes; ++b)
    if (box_off[b + 1] < box_off[b]) return OR_EINVAL;
  return OR_OK;
}

int or_migrate_send(const or_grid* g, const uint64_t* id, const double* const cols[7],
                    int64_t n, const uint64_t* box_off_prev, uint32_t class_id,
                    uint64_t* inbox_off, uint8_t* arena, uint64_t arena_units,
                    uint64_t* box_off_next, uint64_t* id_next, double* const cols_next[7]) {
  int st = or_grid_check(g);
  if (st != OR_OK) return st;
  const uint64_t n_boxes = (uint64_t)g->n[0] * (uint64_t)g->n[1] * (uint64_t)g->n[2];
  const uint64_t n_inbox = n_boxes * 27u;
  if ((st = check_box_off(box_off_prev, n_boxes, n)) != OR_OK) return st;
  int32_t* owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  uint32_t* mask = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
  uint64_t* count = (uint64_t*)calloc((size_t)n_inbox, sizeof(uint64_t));
  uint64_t* fill = (uint64_t*)calloc((size_t)n_inbox, sizeof(uint64_t));
  uint64_t* size_next = (uint64_t*)calloc((size_t)n_boxes, sizeof(uint64_t));
  if (!owner || !mask || !count || !fill || !size_next) {
    st = OR_ENOMEM;
    goto done;
  }
  /* the owner box of every agent's current position */
  st = or_classify(g, cols[0], cols[1], cols[2], n, owner, mask);
  if (st != OR_OK) goto done;
  /* count the leavers of every inbox, and the agents of every next box */
  for (uint64_t s = 0; s < n_boxes; ++s) {
    for (uint64_t i = box_off_prev[s]; i < box_off_prev[s + 1]; ++i) {
      int32_t d = owner[i];
      size_next[d] += 1;
      if ((uint64_t)d != s) count[(uint64_t)d * 27u + (uint64_t)or_migrate_inbox_bit(g, (int32_t)s, d)] += 1;
    }
  }
  inbox_off[0] = 0;
  for (uint64_t q = 0; q < n_inbox; ++q) inbox_off[q + 1] = inbox_off[q] + count[q];
  box_off_next[0] = 0;
  for (uint64_t d = 0; d < n_boxes; ++d) box_off_next[d + 1] = box_off_next[d] + size_next[d];
  if (inbox_off[n_inbox] + n_inbox > arena_units) {
    st = OR_ECAPACITY;
    goto done;
  }
  /* serialize: one TAIO header per inbox, then its leavers in agent order */
  for (uint64_t q = 0; q < n_inbox; ++q)
    write_taio_header(arena + (inbox_off[q] + q) * REC_BYTES, class_id, (uint32_t)q, count[q]);
  for (uint64_t s = 0; s < n_boxes; ++s) {
    for (uint64_t i = box_off_prev[s]; i < box_off_prev[s + 1]; ++i) {
      int32_t d = owner[i];
      if ((uint64_t)d == s) continue;
      uint64_t q = (uint64_t)d * 27u + (uint64_t)or_migrate_inbox_bit(g, (int32_t)s, d);
      uint8_t* rec = arena + (inbox_off[q] + q + 1 + fill[q]) * REC_BYTES;
      fill[q] += 1;
      put_le(rec, id[i], 8);
      for (int c = 0; c < 7; ++c) put_le(rec + 8 * (c + 1), f64_bits(cols[c][i]), 8);
    }
  }
  /* the stayers of box d, in their previous order, open its next range */
  for (uint64_t d = 0; d < n_boxes; ++d) {
    uint64_t pos = box_off_next[d];
    for (uint64_t i = box_off_prev[d]; i < box_off_prev[d + 1]; ++i) {
      if ((uint64_t)owner[i] != d) continue;
      id_next[pos] = id[i];
      for (int c = 0; c < 7; ++c) cols_next[c][pos] = cols[c][i];
      pos += 1;
    }
  }
done:
  free(owner);
  free(mask);
  free(count);
  free(fill);
  free(size_next);
  return st;
}

/* Deserialize every inbox into the next state: the records of box d's
 * inboxes, in ascending inbox side and then in message order, follow its
 * stayers.  Each inbox header is checked (magic, version, record size, class
 * id, inbox index, record count). */
int or_migrate_recv(const or_grid* g, const uint8_t* arena, const uint64_t* inbox_off,
                    uint32_t class_id, const uint64_t* box_off_next, uint64_t* id_next,
                    double* const cols_next[7]) {
  const uint64_t n_boxes = (uint64_t)g->n[0] * (uint64_t)g->n[1] * (uint64_t)g->n[2];
  for (uint64_t d = 0; d < n_boxes; ++d) {
    uint64_t immigrants = inbox_off[d * 27u + 27u] - inbox_off[d * 27u];
    uint64_t size = box_off_next[d + 1] - box_off_next[d];
    if (immigrants > size) return OR_ECORRUPT;
    uint64_t pos = box_off_next[d] + (size - immigrants);
    for (uint64_t b = 0; b < 27; ++b) {
      uint64_t q = d * 27u + b;
      const uint8_t* h = arena + (inbox_off[q] + q) * REC_BYTES;
      uint64_t m = inbox_off[q + 1] - inbox_off[q];
      if (get_le(h, 4) != TAIO_MAGIC || get_le(h + 4, 2) != FMT_VERSION ||
          get_le(h + 6, 2) != REC_BYTES || get_le(h + 8, 4) != class_id ||
          get_le(h + 12, 4) != (uint32_t)q || get_le(h + 16, 8) != m)
        return OR_ECORRUPT;
      for (uint64_t k = 0; k < m; ++k) {
        const uint8_t* rec = h + HDR_BYTES + k * REC_BYTES;
        id_next[pos] = rec_word(rec, 0);
        for (int c = 0; c < 7; ++c) {
          uint64_t bits = rec_word(rec, c + 1);
          memcpy(&cols_next[c][pos], &bits, 8);
        }
        pos += 1;
      }
    }
  }
  return OR_OK;
}

int or_exchange_iteration(const or_grid* g, const uint64_t* id, const double* const cols[7],
                          int64_t n, uint32_t class_id, uint32_t mode,
                          const uint8_t* ref_arena, const uint64_t* ref_off,
                          const uint8_t* recv_ref_arena, const uint64_t* recv_ref_off,
                          int32_t* owner, uint32_t* mask, uint64_t* pair_count,
                          uint64_t* pair_off, uint32_t* pair_idx, uint64_t idx_capacity,
                          uint8_t* rec_arena, uint8_t* wire, uint64_t* wire_off,
                          uint64_t* wire_len, uint8_t* ref_next, uint8_t* recv,
                          uint64_t recv_cap_units, uint64_t* recv_off, double* t_steps) {
  uint64_t n_pairs = (uint64_t)g->n[0] * (uint64_t)g->n[1] * (uint64_t)g->n[2] * 27u;
  double t0 = now_s();
  int st = or_classify(g, cols[0], cols[1], cols[2], n, owner, mask);
  if (st != OR_OK) return st;
  st = or_pair_lists(g, owner, mask, n, pair_count, pair_off, pair_idx, idx_capacity);
  if (st != OR_OK) return st;
  double t1 = now_s();
  or_pack(id, cols, n_pairs, pair_off, pair_idx, class_id, rec_arena);
  double t2 = now_s();
  or_wire_slabs(n_pairs, pair_off, ref_off, wire_off);
  st = or_encode_all(n_pairs, class_id, mode, rec_arena, pair_off, ref_arena, ref_off, NULL,
                     wire, wire_off, wire_len, ref_next);
  if (st != OR_OK) return st;
  double t3 = now_s();
  st = or_decode_all(n_pairs, class_id, wire, wire_off, recv_ref_arena, recv_ref_off, recv,
                     recv_cap_units, recv_off);
  double t4 = now_s();
  if (t_steps) {
    t_steps[0] = t1 - t0;
    t_steps[1] = t2 - t1;
    t_steps[2] = t3 - t2;
    t_steps[3] = t4 - t3;
  }
  return st;
}

/* ---------- residual mode with the learned predictor (not in the paper) ----------
 * Same matching and layout as or_encode_pair.  For a message in mode
 * RESIDUAL, the position words (w1..w3) of a matched slot whose history makes
 * it predictable carry zigzag(bits(x_t) - bits(prediction)) (mod 2^64); every
 * other word is the XOR difference, and new records are raw.  The encoder
 * sends RESIDUAL only when its payload is smaller than the XOR payload
 * (allow_residual != 0); it also writes the history of the new reference. */
int or_predict(const float* params, const uint8_t* rec, const uint8_t* hist, uint32_t ncount,
               uint64_t* pred_bits);
void or_hist_next(const uint8_t* rec, const uint8_t* hist, uint8_t* out);
void or_cell_counts(const uint8_t* ref, uint64_t r, const double lo[3], double w,
                    uint32_t* count);
uint64_t or_zigzag(uint64_t d);
uint64_t or_unzigzag(uint64_t z);

static const uint8_t zero_hist[48] = {0};

int or_encode_pair_pred(const uint8_t* msg, uint64_t m, const uint8_t* ref, uint64_t r,
                        const uint8_t* hist, const float* params, const double lo[3], double w,
                        int allow_residual, uint32_t class_id, uint32_t pair, uint8_t* wire,
                        uint64_t wire_cap, uint64_t* wire_len, uint8_t* ref_next,
                        uint8_t* hist_next) {
  id_pos* sorted = (id_pos*)malloc(sizeof(id_pos) * (size_t)(m ? m : 1));
  uint8_t* matched = (uint8_t*)calloc(m ? m : 1, 1);
  int64_t* src = (int64_t*)malloc(sizeof(int64_t) * (size_t)(r ? r : 1));
  uint32_t* ncount = (uint32_t*)calloc(r ? r : 1, sizeof(uint32_t));
  uint8_t* pred_ok = (uint8_t*)calloc(r ? r : 1, 1);
  uint64_t* pred = (uint64_t*)calloc(3 * (r ? r : 1), sizeof(uint64_t));
  int status = OR_OK;
  if (!sorted || !matched || !src || !ncount || !pred_ok || !pred) {
    status = OR_ENOMEM;
    goto done;
  }
  for (uint64_t k = 0; k < m; ++k) {
    sorted[k].id = rec_word(msg + k * REC_BYTES, 0);
    sorted[k].k = k;
  }
  qsort(sorted, (size_t)m, sizeof(id_pos), cmp_id_pos);
  for (uint64_t k = 1; k < m; ++k)
    if (sorted[k].id == sorted[k - 1].id) {
      status = OR_EINVAL;
      goto done;
    }
  uint64_t n_holes = 0;
  for (uint64_t j = 0; j < r; ++j) {
    int64_t k = find_id(sorted, m, rec_word(ref + j * REC_BYTES, 0));
    src[j] = k;
    if (k < 0) {
      n_holes += 1;
    } else {
      if (matched[k]) {
        status = OR_EINVAL;
        goto done;
      }
      matched[k] = 1;
    }
  }
  uint64_t n_new = 0;
  for (uint64_t k = 0; k < m; ++k)
    if (!matched[k]) n_new += 1;
  /* predictions of the matched slots */
  if (params && hist) {
    or_cell_counts(ref, r, lo, w, ncount);
    for (uint64_t j = 0; j < r; ++j)
      if (src[j] >= 0)
        pred_ok[j] = (uint8_t)or_predict(params, ref + j * REC_BYTES, hist + 48 * j, ncount[j],
                                         pred + 3 * j);
  }
  /* the word slot j sends for word w under each mode */
  uint64_t pay_xor = 0, pay_res = 0;
  for (uint64_t j = 0; j < r; ++j) {
    if (src[j] < 0) continue;
    const uint8_t* cur = msg + (uint64_t)src[j] * REC_BYTES;
    for (int wd = 0; wd < REC_WORDS; ++wd) {
      const uint64_t x = rec_word(cur, wd) ^ rec_word(ref + j * REC_BYTES, wd);
      pay_xor += (uint64_t)sig_bytes(x);
      uint64_t v = x;
      if (pred_ok[j] && wd >= 1 && wd <= 3) v = or_zigzag(rec_word(cur, wd) - pred[3 * j + wd - 1]);
      pay_res += (uint64_t)sig_bytes(v);
    }
  }
  uint64_t pay_new = 0;
  for (uint64_t k = 0; k < m; ++k) {
    if (matched[k]) continue;
    for (int wd = 0; wd < REC_WORDS; ++wd)
      pay_new += (uint64_t)sig_bytes(rec_word(msg + k * REC_BYTES, wd));
  }
  const int residual = allow_residual && params && hist && pay_res < pay_xor;
  const uint32_t mode = residual ? (uint32_t)OR_MODE_RESIDUAL : (uint32_t)OR_MODE_XOR;
  const uint64_t payload = (residual ? pay_res : pay_xor) + pay_new;
  const uint64_t n_codes = r + n_new;
  const uint64_t msg_bytes = round16(HDR_BYTES + 4u * n_codes + payload);
  *wire_len = msg_bytes;
  if (msg_bytes > wire_cap) {
    status = OR_ECAPACITY;
    goto done;
  }
  memset(wire, 0, (size_t)msg_bytes);
  write_wire_header(wire, class_id, mode, r, n_new, n_holes, payload, pair, msg_bytes);
  uint8_t* codes = wire + HDR_BYTES;
  uint8_t* pay = wire + HDR_BYTES + 4u * n_codes;
  uint64_t off = 0, e = 0;
  for (uint64_t j = 0; j < r; ++j, ++e) {
    if (src[j] < 0) {
      put_le(codes + 4 * e, 0xFu, 4);
      continue;
    }
    const uint8_t* cur = msg + (uint64_t)src[j] * REC_BYTES;
    uint32_t code = 0;
    for (int wd = 0; wd < REC_WORDS; ++wd) {
      uint64_t d = rec_word(cur, wd) ^ rec_word(ref + j * REC_BYTES, wd);
      if (residual && pred_ok[j] && wd >= 1 && wd <= 3)
        d = or_zigzag(rec_word(cur, wd) - pred[3 * j + wd - 1]);
      const int L = sig_bytes(d);
      code |= (uint32_t)L << (4 * wd);
      put_le(pay + off, d, L);
      off += (uint64_t)L;
    }
    put_le(codes + 4 * e, code, 4);
  }
  for (uint64_t k = 0; k < m; ++k) {
    if (matched[k]) continue;
    const uint8_t* cur = msg + k * REC_BYTES;
    uint32_t code = 0;
    for (int wd = 0; wd < REC_WORDS; ++wd) {
      const uint64_t d = rec_word(cur, wd);
      const int L = sig_bytes(d);
      code |= (uint32_t)L << (4 * wd);
      put_le(pay + off, d, L);
      off += (uint64_t)L;
    }
    put_le(codes + 4 * e, code, 4);
    e += 1;
  }
  {
    uint64_t q = 0;
    for (uint64_t j = 0; j < r; ++j) {
      if (src[j] < 0) continue;
      memcpy(ref_next + q * REC_BYTES, msg + (uint64_t)src[j] * REC_BYTES, REC_BYTES);
      if (hist_next)
        or_hist_next(ref + j * REC_BYTES, hist ? hist + 48 * j : zero_hist, hist_next + 48 * q);
      q += 1;
    }
    for (uint64_t k = 0; k < m; ++k) {
      if (matched[k]) continue;
      memcpy(ref_next + q * REC_BYTES, msg + k * REC_BYTES, REC_BYTES);
      if (hist_next) or_hist_next(NULL, NULL, hist_next + 48 * q);
      q += 1;
    }
  }
done:
  free(sorted);
  free(matched);
  free(src);
  free(ncount);
  free(pred_ok);
  free(pred);
  return status;
}

int or_decode_pair_pred(const uint8_t* wire, uint64_t wire_avail, const uint8_t* ref, uint64_t r,
                        const uint8_t* hist, const float* params, const double lo[3], double w,
                        uint32_t class_id, uint32_t pair, uint8_t* out, uint64_t out_cap,
                        uint64_t* m_out, uint8_t* hist_next) {
  *m_out = 0;
  if (wire_avail < HDR_BYTES) return OR_ECORRUPT;
  if (get_le(wire + 0, 4) != WIRE_MAGIC || get_le(wire + 4, 2) != FMT_VERSION ||
      get_le(wire + 6, 2) != REC_BYTES || get_le(wire + 8, 4) != class_id ||
      get_le(wire + 48, 4) != pair)
    return OR_ECORRUPT;
  const uint64_t mode = get_le(wire + 12, 4);
  const uint64_t n_slots = get_le(wire + 16, 8), n_new = get_le(wire + 24, 8);
  const uint64_t n_holes = get_le(wire + 32, 8), payload = get_le(wire + 40, 8);
  const uint64_t msg_bytes = get_le(wire + 56, 8);
  if (mode == OR_MODE_RAW) {
    if (n_slots != 0) return OR_ECORRUPT;
  } else if (mode == OR_MODE_XOR || mode == OR_MODE_RESIDUAL) {
    if (n_slots != r) return OR_EREFMISMATCH;
    if (mode == OR_MODE_RESIDUAL && (!params || !hist)) return OR_ECORRUPT;
  } else {
    return OR_ECORRUPT;
  }
  if (n_slots > wire_avail || n_new > wire_avail || payload > wire_avail) return OR_ECORRUPT;
  const uint64_t n_codes = n_slots + n_new;
  if (msg_bytes != round16(HDR_BYTES + 4u * n_codes + payload) || msg_bytes > wire_avail)
    return OR_ECORRUPT;
  uint32_t* ncount = NULL;
  if (mode == OR_MODE_RESIDUAL) {
    ncount = (uint32_t*)calloc(r ? r : 1, sizeof(uint32_t));
    or_cell_counts(ref, r, lo, w, ncount);
  }
  const uint8_t* codes = wire + HDR_BYTES;
  const uint8_t* pay = wire + HDR_BYTES + 4u * n_codes;
  uint64_t off = 0, holes = 0, count = 0;
  int status = OR_OK;
  for (uint64_t e = 0; e < n_codes; ++e) {
    const uint32_t code = (uint32_t)get_le(codes + 4 * e, 4);
    if ((code & 0xFu) == 0xFu) {
      if (e >= n_slots || (code >> 4) != 0) {
        status = OR_ECORRUPT;
        break;
      }
      holes += 1;
      continue;
    }
    int bad = 0;
    for (int wd = 0; wd < REC_WORDS; ++wd)
      if (((code >> (4 * wd)) & 0xFu) > 8u) bad = 1;
    if (bad || (e < n_slots && (code & 0xFu) != 0)) {
      status = OR_ECORRUPT;
      break;
    }
    if (count >= out_cap) {
      status = OR_ECAPACITY;
      break;
    }
    uint64_t pred[3];
    int pred_ok = 0;
    if (mode == OR_MODE_RESIDUAL && e < n_slots)
      pred_ok = or_predict(params, ref + e * REC_BYTES, hist + 48 * e, ncount[e], pred);
    uint8_t* rec = out + count * REC_BYTES;
    for (int wd = 0; wd < REC_WORDS; ++wd) {
      const int L = (int)((code >> (4 * wd)) & 0xFu);
      if (off + (uint64_t)L > payload) {
        status = OR_ECORRUPT;
        break;
      }
      const uint64_t d = get_le(pay + off, L);
      off += (uint64_t)L;
      uint64_t v;
      if (e >= n_slots) v = d;
      else if (pred_ok && wd >= 1 && wd <= 3) v = pred[wd - 1] + or_unzigzag(d);
      else v = d ^ rec_word(ref + e * REC_BYTES, wd);
      put_le(rec + 8 * wd, v, 8);
    }
    if (status != OR_OK) break;
    if (hist_next) {
      if (e < n_slots)
        or_hist_next(ref + e * REC_BYTES, hist ? hist + 48 * e : zero_hist,
                     hist_next + 48 * count);
      else
        or_hist_next(NULL, NULL, hist_next + 48 * count);
    }
    count += 1;
  }
  free(ncount);
  if (status != OR_OK) return status;
  if (off != payload || holes != n_holes) return OR_ECORRUPT;
  *m_out = count;
  return OR_OK;
}

/* Arena drivers of the residual mode.  History arenas have no headers: the
 * entry of slot j of pair p is at index off[p] + j (48 bytes each). */
int or_encode_all_pred(uint64_t n_pairs, uint32_t class_id, int allow_residual,
                       const uint8_t* rec_arena, const uint64_t* pair_off,
                       const uint8_t* ref_arena, const uint64_t* ref_off, const uint8_t* hist,
                       const float* params, const double lo[3], double w, uint8_t* wire,
                       const uint64_t* wire_off, uint64_t* wire_len, uint8_t* ref_next,
                       uint8_t* hist_next) {
  int status = OR_OK;
  for (uint64_t p = 0; p < n_pairs; ++p) {
    const uint64_t m = pair_off[p + 1] - pair_off[p];
    const uint64_t r = ref_arena ? ref_off[p + 1] - ref_off[p] : 0;
    const uint8_t* msg_buf = rec_arena + (pair_off[p] + p) * REC_BYTES;
    const uint8_t* ref_buf = ref_arena ? ref_arena + (ref_off[p] + p) * REC_BYTES : NULL;
    uint8_t* nxt = ref_next + (pair_off[p] + p) * REC_BYTES;
    write_taio_header(nxt, class_id, (uint32_t)p, m);
    int st = or_encode_pair_pred(
        msg_buf + HDR_BYTES, m, ref_buf ? ref_buf + HDR_BYTES : NULL, r,
        (ref_arena && hist) ? hist + 48 * ref_off[p] : NULL, params, lo, w, allow_residual,
        class_id, (uint32_t)p, wire + wire_off[p], wire_off[p + 1] - wire_off[p], &wire_len[p],
        nxt + HDR_BYTES, hist_next ? hist_next + 48 * pair_off[p] : NULL);
    if (st != OR_OK && status == OR_OK) status = st;
  }
  return status;
}

int or_decode_all_pred(uint64_t n_pairs, uint32_t class_id, const uint8_t* wire,
                       const uint64_t* wire_off, const uint8_t* ref_arena,
                       const uint64_t* ref_off, const uint8_t* hist, const float* params,
                       const double lo[3], double w, uint8_t* recv, uint64_t recv_cap_units,
                       uint64_t* recv_off, uint8_t* hist_next) {
  int status = OR_OK;
  recv_off[0] = 0;
  for (uint64_t p = 0; p < n_pairs; ++p) {
    const uint8_t* h = wire + wire_off[p];
    const uint64_t avail = wire_off[p + 1] - wire_off[p];
    uint64_t m = 0;
    if (avail >= HDR_BYTES && get_le(h, 4) == WIRE_MAGIC) {
      const uint64_t ns = get_le(h + 16, 8), nn = get_le(h + 24, 8), nh = get_le(h + 32, 8);
      if (nh <= ns && ns <= avail && nn <= avail) m = ns - nh + nn;
    }
    recv_off[p + 1] = recv_off[p] + m;
  }
  if (recv_off[n_pairs] + n_pairs > recv_cap_units) return OR_ECAPACITY;
  for (uint64_t p = 0; p < n_pairs; ++p) {
    const uint64_t r = ref_arena ? ref_off[p + 1] - ref_off[p] : 0;
    const uint8_t* ref_buf = ref_arena ? ref_arena + (ref_off[p] + p) * REC_BYTES : NULL;
    uint8_t* out = recv + (recv_off[p] + p) * REC_BYTES;
    const uint64_t cap = recv_off[p + 1] - recv_off[p];
    uint64_t got = 0;
    int st = or_decode_pair_pred(wire + wire_off[p], wire_off[p + 1] - wire_off[p],
                                 ref_buf ? ref_buf + HDR_BYTES : NULL, r,
                                 (ref_arena && hist) ? hist + 48 * ref_off[p] : NULL, params, lo,
                                 w, class_id, (uint32_t)p, out + HDR_BYTES, cap, &got,
                                 hist_next ? hist_next + 48 * recv_off[p] : NULL);
    if (st == OR_OK && got != cap) st = OR_ECORRUPT;
    write_taio_header(out, class_id, (uint32_t)p, cap);
    if (st != OR_OK && status == OR_OK) status = st;
  }
  return status;
}
