/*
 * Oracle for the aura-exchange codec: a plain, slow, single-threaded CPU
 * restatement of what the TeraAgent aura update computes (paper Sec. 2.1,
 * Sec. 2.2.1, Sec. 2.3).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg may call it; the product path never does.
 * It shares no header, helper or table with the CUDA library.
 *
 * Records are 64 bytes = 8 little-endian 64-bit words:
 *   w0 id | w1 x | w2 y | w3 z | w4 diameter | w5 volume | w6 adherence | w7 density
 */
#ifndef TERA_ORACLE_H
#define TERA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_OK = 0,
  OR_EINVAL = 1,
  OR_ENOMEM = 2,
  OR_ECAPACITY = 3,
  OR_ECORRUPT = 4,
  OR_EDOMAIN = 5,
  OR_EREFMISMATCH = 6
};

enum { OR_MODE_RAW = 0, OR_MODE_XOR = 1, OR_MODE_RESIDUAL = 2 };

/* periodic: bit a set makes axis a toroidal (Sec. 2.5 names open, closed
 * and toroidal space boundaries): box n-1 and box 0 are neighbours on it. */
typedef struct {
  double lo[3], hi[3];
  int32_t n[3];
  double w;
  uint32_t periodic;
  uint32_t reserved;
} or_grid;

/* Grid edges and parameter check (Sec. 2.1 partitioning grid; Sec. 2.4). */
int or_grid_check(const or_grid* g);
void or_axis_edges(const or_grid* g, int axis, double* e /* n[axis]+1 */);

/* O1: owner box and 26-neighbour aura mask per agent (Sec. 2.1 "Aura Update"). */
int or_classify(const or_grid* g, const double* x, const double* y, const double* z,
                int64_t n, int32_t* owner, uint32_t* mask);

/* Per-pair stable lists (message p = agents of box s whose mask has bit b,
 * ascending agent index; p = s*27 + b). */
int or_pair_lists(const or_grid* g, const int32_t* owner, const uint32_t* mask, int64_t n,
                  uint64_t* pair_count, uint64_t* pair_off, uint32_t* pair_idx,
                  uint64_t idx_capacity);

/* O2: TeraAgent IO serialization of every pair message (Sec. 2.2.1). */
void or_pack(const uint64_t* id, const double* const cols[7], uint64_t n_pairs,
             const uint64_t* pair_off, const uint32_t* pair_idx, uint32_t class_id,
             uint8_t* arena);

/* O3+O4: match, XOR delta and byte packing of one pair message (Sec. 2.3). */
int or_encode_pair(const uint8_t* msg, uint64_t m, const uint8_t* ref, uint64_t r,
                   uint32_t class_id, uint32_t mode, uint32_t pair, uint8_t* wire,
                   uint64_t wire_cap, uint64_t* wire_len, uint8_t* ref_next);

/* O5: decode and defragment one pair message (Sec. 2.3 step D). */
int or_decode_pair(const uint8_t* wire, uint64_t wire_avail, const uint8_t* ref, uint64_t r,
                   uint32_t class_id, uint32_t pair, uint8_t* out, uint64_t out_cap,
                   uint64_t* m_out);

/* Arena-level drivers (every pair of one iteration). */
void or_wire_slabs(uint64_t n_pairs, const uint64_t* pair_off, const uint64_t* ref_off,
                   uint64_t* wire_off);
int or_encode_all(uint64_t n_pairs, uint32_t class_id, uint32_t mode, const uint8_t* rec_arena,
                  const uint64_t* pair_off, const uint8_t* ref_arena, const uint64_t* ref_off,
                  const uint8_t* reset, uint8_t* wire, const uint64_t* wire_off,
                  uint64_t* wire_len, uint8_t* ref_next);
int or_decode_all(uint64_t n_pairs, uint32_t class_id, const uint8_t* wire,
                  const uint64_t* wire_off, const uint8_t* ref_arena, const uint64_t* ref_off,
                  uint8_t* recv, uint64_t recv_cap_units, uint64_t* recv_off);

/* Receive layout of or_decode_all: recv_off[P+1] from the message headers. */
void or_recv_layout(uint64_t n_pairs, const uint8_t* wire, const uint64_t* wire_off,
                    uint64_t* recv_off);

/* The same drivers over pairs [p0, p1) of the arenas (used to spread the
 * pairs of one iteration over host threads; each pair is independent). */
void or_pack_range(const uint64_t* id, const double* const cols[7], uint64_t p0, uint64_t p1,
                   const uint64_t* pair_off, const uint32_t* pair_idx, uint32_t class_id,
                   uint8_t* arena);
int or_encode_range(uint64_t p0, uint64_t p1, uint32_t class_id, uint32_t mode,
                    const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_arena,
                    const uint64_t* ref_off, const uint8_t* reset, uint8_t* wire,
                    const uint64_t* wire_off, uint64_t* wire_len, uint8_t* ref_next);
int or_decode_range(uint64_t p0, uint64_t p1, uint32_t class_id, const uint8_t* wire,
                    const uint64_t* wire_off, const uint8_t* ref_arena, const uint64_t* ref_off,
                    uint8_t* recv, const uint64_t* recv_off);

/* Difference-serialized message before compression (Sec. 2.3 B and C): XOR
 * for matched slots, 64 zero bytes for placeholders, then the new records. */
int or_delta_records(const uint8_t* msg, uint64_t m, const uint8_t* ref, uint64_t r,
                     uint8_t* out, uint64_t* n_entries);

/* Agent migration (Sec. 2.1 "Agent Migration"; records are the raw TeraAgent
 * IO buffers of Sec. 2.2.1).  The state is box-major: box s holds agents
 * [box_off_prev[s], box_off_prev[s+1]).  An agent whose position now lies in
 * box d != s leaves s for inbox q = d*27 + b, b the neighbour bit of the
 * offset from d to s (the side it arrives from), or 13 when s is not a
 * neighbour of d.  Inbox q holds its leavers in ascending agent index, laid
 * out as a TAIO arena with inbox_off[P+1].  The next state of box d is its
 * stayers in their previous order followed by its inboxes in ascending b.
 * or_migrate_send writes inbox_off, the arena, box_off_next and the stayers;
 * or_migrate_recv writes the immigrants from the arena. */
int or_migrate_inbox_bit(const or_grid* g, int32_t s, int32_t d);
int or_migrate_send(const or_grid* g, const uint64_t* id, const double* const cols[7],
                    int64_t n, const uint64_t* box_off_prev, uint32_t class_id,
                    uint64_t* inbox_off, uint8_t* arena, uint64_t arena_units,
                    uint64_t* box_off_next, uint64_t* id_next, double* const cols_next[7]);
int or_migrate_recv(const or_grid* g, const uint8_t* arena, const uint64_t* inbox_off,
                    uint32_t class_id, const uint64_t* box_off_next, uint64_t* id_next,
                    double* const cols_next[7]);

/* Whole iteration, for the CPU baseline timing. */
int or_exchange_iteration(const or_grid* g, const uint64_t* id, const double* const cols[7],
                          int64_t n, uint32_t class_id, uint32_t mode,
                          const uint8_t* ref_arena, const uint64_t* ref_off,
                          const uint8_t* recv_ref_arena, const uint64_t* recv_ref_off,
                          int32_t* owner, uint32_t* mask, uint64_t* pair_count,
                          uint64_t* pair_off, uint32_t* pair_idx, uint64_t idx_capacity,
                          uint8_t* rec_arena, uint8_t* wire, uint64_t* wire_off,
                          uint64_t* wire_len, uint8_t* ref_next, uint8_t* recv,
                          uint64_t recv_cap_units, uint64_t* recv_off, double* t_steps);

/* or_exchange_iteration with its work spread over `threads` host threads
 * (tera_oracle_mt.c): classification over contiguous agent ranges, packing,
 * encoding and decoding over contiguous pair ranges, each range done by the
 * single-threaded functions above; the lists, slabs and receive layout stay
 * single-threaded.  Same outputs, byte for byte. */
int or_exchange_iteration_mt(const or_grid* g, const uint64_t* id, const double* const cols[7],
                             int64_t n, uint32_t class_id, uint32_t mode,
                             const uint8_t* ref_arena, const uint64_t* ref_off,
                             const uint8_t* recv_ref_arena, const uint64_t* recv_ref_off,
                             int32_t* owner, uint32_t* mask, uint64_t* pair_count,
                             uint64_t* pair_off, uint32_t* pair_idx, uint64_t idx_capacity,
                             uint8_t* rec_arena, uint8_t* wire, uint64_t* wire_off,
                             uint64_t* wire_len, uint8_t* ref_next, uint8_t* recv,
                             uint64_t recv_cap_units, uint64_t* recv_off, double* t_steps,
                             int threads);

/* Learned predictor and residual mode (mlp_oracle.c; not in the paper). */
int or_mlp_nparam(void);
void or_mlp_infer_f32(const float* params, const float* in, float* out);
double or_mlp_loss_grad_f64(const double* params, const double* X, const double* Y, int64_t n,
                            double* grad);
void or_mlp_sgd_f64(double* params, const double* grad, double lr);
void or_mlp_sgd_clip_f64(double* params, const double* grad, double lr, double clip);
uint64_t or_zigzag(uint64_t d);
uint64_t or_unzigzag(uint64_t z);
void or_cell_counts(const uint8_t* ref, uint64_t r, const double lo[3], double w,
                    uint32_t* count);
int or_features(const uint8_t* rec, const uint8_t* hist, uint32_t ncount, float* f);
int or_predict(const float* params, const uint8_t* rec, const uint8_t* hist, uint32_t ncount,
               uint64_t* pred_bits);
void or_hist_next(const uint8_t* rec, const uint8_t* hist, uint8_t* out);
int or_sample(const uint8_t* cur, const uint8_t* rec, const uint8_t* hist, uint32_t ncount,
              float* x, float* y);
int or_encode_pair_pred(const uint8_t* msg, uint64_t m, const uint8_t* ref, uint64_t r,
                        const uint8_t* hist, const float* params, const double lo[3], double w,
                        int allow_residual, uint32_t class_id, uint32_t pair, uint8_t* wire,
                        uint64_t wire_cap, uint64_t* wire_len, uint8_t* ref_next,
                        uint8_t* hist_next);
int or_decode_pair_pred(const uint8_t* wire, uint64_t wire_avail, const uint8_t* ref, uint64_t r,
                        const uint8_t* hist, const float* params, const double lo[3], double w,
                        uint32_t class_id, uint32_t pair, uint8_t* out, uint64_t out_cap,
                        uint64_t* m_out, uint8_t* hist_next);
int or_encode_all_pred(uint64_t n_pairs, uint32_t class_id, int allow_residual,
                       const uint8_t* rec_arena, const uint64_t* pair_off,
                       const uint8_t* ref_arena, const uint64_t* ref_off, const uint8_t* hist,
                       const float* params, const double lo[3], double w, uint8_t* wire,
                       const uint64_t* wire_off, uint64_t* wire_len, uint8_t* ref_next,
                       uint8_t* hist_next);
int or_decode_all_pred(uint64_t n_pairs, uint32_t class_id, const uint8_t* wire,
                       const uint64_t* wire_off, const uint8_t* ref_arena,
                       const uint64_t* ref_off, const uint8_t* hist, const float* params,
                       const double lo[3], double w, uint8_t* recv, uint64_t recv_cap_units,
                       uint64_t* recv_off, uint8_t* hist_next);

#ifdef __cplusplus
}
#endif
#endif
