/*
 * TEST INFRASTRUCTURE ONLY (CPU baseline on all host cores).
 *
 * One aura-exchange iteration (Sec. 2.1 classification, Sec. 2.2.1
 * serialization, Sec. 2.3 difference encoding and decoding) with its work
 * spread over host threads.  Nothing here computes anything of its own: every
 * range is handed to the single-threaded oracle functions of tera_oracle.c,
 * which already treat agents (classification) and pairs (packing, encoding,
 * decoding) independently of each other.  Work is claimed in chunks from a
 * shared counter (agents in chunks of 65,536, pairs one box of 27 at a time),
 * and a status is reduced in chunk order, so the result is the one the
 * single-threaded iteration returns.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <time.h>

#include "tera_oracle.h"

enum { PHASE_CLASSIFY = 0, PHASE_PACK = 1, PHASE_ENCODE = 2, PHASE_DECODE = 3 };

typedef struct {
  int phase;
  uint64_t n_chunks, chunk;  /* chunk size in agents or pairs */
  uint64_t total;            /* agents or pairs */
  atomic_ulong next;
  int* status;               /* [n_chunks] */
  /* inputs and outputs of the iteration */
  const or_grid* g;
  const uint64_t* id;
  const double* const* cols;
  uint32_t class_id, mode;
  const uint8_t *ref_arena, *recv_ref_arena;
  const uint64_t *ref_off, *recv_ref_off;
  int32_t* owner;
  uint32_t* mask;
  const uint64_t* pair_off;
  const uint32_t* pair_idx;
  uint8_t *rec_arena, *wire, *ref_next, *recv;
  const uint64_t* wire_off;
  uint64_t* wire_len;
  const uint64_t* recv_off;
} work;

static void* worker(void* arg) {
  work* w = (work*)arg;
  for (;;) {
    uint64_t c = atomic_fetch_add(&w->next, 1ul);
    if (c >= w->n_chunks) break;
    uint64_t a = c * w->chunk, b = a + w->chunk < w->total ? a + w->chunk : w->total;
    int st = OR_OK;
    switch (w->phase) {
      case PHASE_CLASSIFY:
        st = or_classify(w->g, w->cols[0] + a, w->cols[1] + a, w->cols[2] + a, (int64_t)(b - a),
                         w->owner + a, w->mask + a);
        break;
      case PHASE_PACK:
        or_pack_range(w->id, w->cols, a, b, w->pair_off, w->pair_idx, w->class_id, w->rec_arena);
        break;
      case PHASE_ENCODE:
        st = or_encode_range(a, b, w->class_id, w->mode, w->rec_arena, w->pair_off, w->ref_arena,
                             w->ref_off, NULL, w->wire, w->wire_off, w->wire_len, w->ref_next);
        break;
      default:
        st = or_decode_range(a, b, w->class_id, w->wire, w->wire_off, w->recv_ref_arena,
                             w->recv_ref_off, w->recv, w->recv_off);
        break;
    }
    w->status[c] = st;
  }
  return NULL;
}

/* Run one phase over `total` units in chunks on `threads` threads; the status
 * of the first failing chunk (in unit order), or OR_ENOMEM. */
static int run_phase(work* w, int phase, uint64_t total, uint64_t chunk, int threads) {
  w->phase = phase;
  w->total = total;
  w->chunk = chunk;
  w->n_chunks = (total + chunk - 1) / chunk;
  atomic_store(&w->next, 0ul);
  w->status = (int*)calloc(w->n_chunks ? w->n_chunks : 1, sizeof(int));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)(threads > 0 ? threads : 1));
  if (!w->status || !th) {
    free(w->status);
    free(th);
    return OR_ENOMEM;
  }
  int started = 0;
  for (int i = 0; i < threads; ++i)
    if (pthread_create(&th[i], NULL, worker, w) == 0) started += 1;
    else break;
  if (started == 0) worker(w); /* no thread could start: run the chunks here */
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  int st = OR_OK;
  for (uint64_t c = 0; c < w->n_chunks && st == OR_OK; ++c) st = w->status[c];
  free(w->status);
  free(th);
  return st;
}

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int or_exchange_iteration_mt(const or_grid* g, const uint64_t* id, const double* const cols[7],
                             int64_t n, uint32_t class_id, uint32_t mode,
                             const uint8_t* ref_arena, const uint64_t* ref_off,
                             const uint8_t* recv_ref_arena, const uint64_t* recv_ref_off,
                             int32_t* owner, uint32_t* mask, uint64_t* pair_count,
                             uint64_t* pair_off, uint32_t* pair_idx, uint64_t idx_capacity,
                             uint8_t* rec_arena, uint8_t* wire, uint64_t* wire_off,
                             uint64_t* wire_len, uint8_t* ref_next, uint8_t* recv,
                             uint64_t recv_cap_units, uint64_t* recv_off, double* t_steps,
                             int threads) {
  uint64_t n_pairs = (uint64_t)g->n[0] * (uint64_t)g->n[1] * (uint64_t)g->n[2] * 27u;
  int st = or_grid_check(g);
  if (st != OR_OK) return st;
  if (threads < 1) threads = 1;
  work w = {0};
  w.g = g;
  w.id = id;
  w.cols = cols;
  w.class_id = class_id;
  w.mode = mode;
  w.ref_arena = ref_arena;
  w.ref_off = ref_off;
  w.recv_ref_arena = recv_ref_arena;
  w.recv_ref_off = recv_ref_off;
  w.owner = owner;
  w.mask = mask;
  w.pair_off = pair_off;
  w.pair_idx = pair_idx;
  w.rec_arena = rec_arena;
  w.wire = wire;
  w.wire_off = wire_off;
  w.wire_len = wire_len;
  w.ref_next = ref_next;
  w.recv = recv;
  w.recv_off = recv_off;
  double t0 = now_s();
  st = run_phase(&w, PHASE_CLASSIFY, (uint64_t)(n > 0 ? n : 0), 65536u, threads);
  if (st != OR_OK) return st;
  st = or_pair_lists(g, owner, mask, n, pair_count, pair_off, pair_idx, idx_capacity);
  if (st != OR_OK) return st;
  double t1 = now_s();
  st = run_phase(&w, PHASE_PACK, n_pairs, 27u, threads);
  if (st != OR_OK) return st;
  double t2 = now_s();
  or_wire_slabs(n_pairs, pair_off, ref_off, wire_off);
  st = run_phase(&w, PHASE_ENCODE, n_pairs, 27u, threads);
  if (st != OR_OK) return st;
  double t3 = now_s();
  /* receive layout from every header (single-threaded), then the pairs */
  or_recv_layout(n_pairs, wire, wire_off, recv_off);
  if (recv_off[n_pairs] + n_pairs > recv_cap_units) return OR_ECAPACITY;
  st = run_phase(&w, PHASE_DECODE, n_pairs, 27u, threads);
  double t4 = now_s();
  if (t_steps) {
    t_steps[0] = t1 - t0;
    t_steps[1] = t2 - t1;
    t_steps[2] = t3 - t2;
    t_steps[3] = t4 - t3;
  }
  return st;
}
