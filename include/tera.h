/*
 * tera.h — C ABI of the GB300 aura-exchange library (libtera.so).
 *
 * The library implements the per-iteration aura (halo) exchange of the
 * TeraAgent distributed engine for spherical agents whose boxes all live in
 * one GPU's memory:
 *
 *   tera_partition     grid classification: owner box + 26-neighbour aura mask
 *                      per agent, per-pair message lists        (paper Sec. 2.1)
 *   tera_pack          TeraAgent IO serialization into flat 64-byte records
 *                      the receiver uses in place             (paper Sec. 2.2.1)
 *   tera_delta_encode  matching against the pair's reference, per-word XOR
 *                      difference and significant-byte packing  (paper Sec. 2.3,
 *                      steps B and C; Sec. 3.11 for the compression stage)
 *   tera_delta_decode  restore from the receiver's reference and defragment
 *                      into the new reference / receive buffer (Sec. 2.3, step D)
 *   tera_unpack_inplace  header check + typed view of a receive buffer, no
 *                      other reads or writes       (Sec. 2.2.1 "Deserialization")
 *   tera_wire_to_host  the wire messages of an iteration into host memory, with
 *                      the length known only on the device (no host wait)
 *   tera_migrate_send / tera_migrate_recv
 *                      agent migration between boxes of a box-major state,
 *                      as raw TAIO records                (paper Sec. 2.1)
 *
 * Conventions shared by every entry point:
 *  - Device pointers are owned by the caller (allocated e.g. by PyTorch); the
 *    library never frees them.  The context owns its own scratch memory, the
 *    per-iteration hash table and a device status word, all released by
 *    tera_ctx_destroy.
 *  - `stream` is a cudaStream_t passed as void*.  Every call that takes a
 *    stream is asynchronous on it and never synchronizes the host (except
 *    tera_unpack_inplace and tera_ctx_status, which read a few bytes back).
 *    Argument errors are returned at once; errors found on the device
 *    (capacity, corrupt message, agent outside the domain) are latched in the
 *    context's status word (first error wins) and read with tera_ctx_status.
 *  - All multi-byte values in buffers are little-endian (native on x86-64 and
 *    aarch64; the paper sends native bytes without conversion, Sec. 2.2).
 *  - No C++ exception crosses this boundary.
 *
 * Buffer formats (all offsets in bytes):
 *
 *  Record (64 B): eight 64-bit words, w0 id | w1 x | w2 y | w3 z | w4 diameter |
 *    w5 volume | w6 adherence | w7 density; floating-point words are the raw
 *    IEEE-754 binary64 bits.
 *
 *  Record arena ("TAIO" buffers): used for packed messages, sender references
 *    and receive buffers.  An arena is an array of 64-byte units; with an
 *    offset array off[P+1] (record counts, exclusive prefix over pairs), pair
 *    p occupies units [off[p] + p, off[p+1] + p + 1): one 64-byte header, then
 *    its off[p+1]-off[p] records.  Header:
 *       0 u32 magic 0x4F494154 ("TAIO")   4 u16 version 1   6 u16 record size 64
 *       8 u32 class id   12 u32 pair p   16 u64 record count   24..63 zero
 *
 *  Wire message of pair p (starts at wire + wire_off[p]):
 *       0 u32 magic 0x41524554 ("TERA")   4 u16 version 1   6 u16 record size 64
 *       8 u32 class id   12 u32 mode (0 raw, 1 xor, 2 residual)   16 u64 n_slots (r)
 *      24 u64 n_new (a)  32 u64 n_holes   40 u64 payload bytes   48 u32 pair p
 *      52 u32 zero       56 u64 message bytes (multiple of 16)
 *      64: u32 code[r + a]; then the payload; then zero padding.
 *    Entry e < r is reference slot e: placeholder (code 0xF) when the agent
 *    of that slot is not in this message, else the XOR of the current record
 *    and the slot's record.  Entries e >= r are the records absent from the
 *    reference, in message order, sent raw.  Nibble w of a code (bits 4w..4w+3)
 *    is L_w = number of significant low bytes of word w (0..8); the payload
 *    is, entry by entry and word by word, the low L_w bytes of each word,
 *    least significant first.
 *    The slab of pair p is sized by an upper bound known before encoding:
 *       wire_off[p+1] - wire_off[p] = round16(64 + 4 (r_p + m_p) + 64 m_p).
 */
#ifndef TERA_H
#define TERA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TERA_OK = 0,
  TERA_EINVAL = 1,       /* bad argument (returned at once) */
  TERA_ENOMEM = 2,       /* cudaMalloc of context scratch failed */
  TERA_ECAPACITY = 3,    /* a caller buffer is too small; see required capacity */
  TERA_ECORRUPT = 4,     /* malformed message or buffer header */
  TERA_EDOMAIN = 5,      /* an agent lies outside [lo, hi) (or is NaN) */
  TERA_EREFMISMATCH = 6, /* message n_slots differs from the receiver's reference */
  TERA_ETIMEOUT = 7,     /* a bounded device-side wait gave up */
  TERA_ECUDA = 8,        /* a CUDA runtime call failed */
  TERA_EBOUNDS = 9       /* debug builds only (TERA_DEBUG_BOUNDS): a write fell outside the
                            range its pair or buffer owns; the write was skipped */
} tera_status;

enum { TERA_MODE_RAW = 0, TERA_MODE_XOR = 1, TERA_MODE_RESIDUAL = 2 };

typedef struct tera_ctx tera_ctx;

/* Struct-of-arrays agent state; device pointers, caller-owned, n < 2^32. */
typedef struct {
  const uint64_t* id;
  const double *x, *y, *z, *diameter, *volume, *adherence, *density;
  int64_t n;
} tera_soa;

/* Writable struct-of-arrays agent state (outputs); device pointers,
 * caller-owned, n < 2^32. */
typedef struct {
  uint64_t* id;
  double *x, *y, *z, *diameter, *volume, *adherence, *density;
  int64_t n;
} tera_soa_mut;

/* Partitioning grid: box edges e[k] = lo + ((hi - lo) * k) / n (k < n),
 * e[n] = hi, per axis; aura width w with 0 < w < every box side.
 * periodic: bit a set makes axis a toroidal (Sec. 2.5 lists open, closed
 * and toroidal space boundaries): box n-1 and box 0 are neighbours along it,
 * so the aura towards offset -1 of box 0 goes to box n-1 and that towards
 * offset +1 of box n-1 to box 0, with the same thresholds as inside the
 * domain.  Records keep their unshifted coordinates.  A periodic axis needs
 * n >= 3 (each neighbour bit then names a distinct box).  reserved must be 0. */
typedef struct {
  double lo[3], hi[3];
  int32_t n[3];
  double w;
  uint32_t periodic;
  uint32_t reserved;
} tera_grid;

/* Outputs of tera_partition; device pointers, caller-owned.
 * P = n[0]*n[1]*n[2]*27 ordered pairs; pair p = s*27 + b with sender box s and
 * neighbour bit b = (ox+1) + 3(oy+1) + 9(oz+1) (b = 13, the box itself, is
 * always empty). */
typedef struct {
  int32_t* owner;        /* [n]  owner box (ix + nx (iy + ny iz)), -1 outside */
  uint32_t* mask;        /* [n]  bit b set when the agent is in the aura of neighbour b */
  uint64_t* pair_count;  /* [P]  m_p, records in message p */
  uint64_t* pair_off;    /* [P+1] exclusive prefix of pair_count */
  uint32_t* pair_idx;    /* [idx_capacity] agent indices of each message, ascending */
  uint64_t idx_capacity;
} tera_partition_out;

/* Create a context on `device` for one grid (Sec. 2.1 partitioning grid).
 * Box edges and aura thresholds are computed here once, in binary64.
 * Returns TERA_EINVAL when a grid axis has n < 1 or n > 256, lo >= hi, or w is
 * not strictly between 0 and every box side, a periodic axis has n < 3, or
 * periodic has bits above 2 or reserved is nonzero.  class_id is written into every
 * buffer header (the paper replaces the vtable pointer by a class id). */
tera_status tera_ctx_create(tera_ctx** out, const tera_grid* grid, int device,
                            uint32_t class_id);
tera_status tera_ctx_destroy(tera_ctx* ctx);

/* Number of ordered pairs P of the context's grid. */
uint64_t tera_n_pairs(const tera_ctx* ctx);

/* Pre-allocate scratch for up to max_agents agents and max_records records
 * per iteration (otherwise done lazily by the first call that needs it;
 * lazy growth synchronizes the device, so call this before graph capture). */
tera_status tera_ctx_reserve(tera_ctx* ctx, int64_t max_agents, uint64_t max_records);

/* Step a1 (Sec. 2.1 "Aura Update"): owner box and aura mask of every agent,
 * and the per-pair stable lists.  Agent i is in the aura of neighbour box at
 * offset o when, on every axis, o = 0, or o = -1 and x < e[i] + w, or o = +1
 * and x >= e[i+1] - w (the neighbour must exist; on a periodic axis it
 * always does, its index taken modulo n).  Agents outside [lo, hi)
 * get owner -1, mask 0 and latch TERA_EDOMAIN.  More than idx_capacity
 * records latch TERA_ECAPACITY (required capacity reported) and leave every
 * pair empty. */
tera_status tera_partition(tera_ctx* ctx, const tera_soa* soa, tera_partition_out* out,
                           void* stream);

/* Step a2 (Sec. 2.2.1 "Serialization"): write the TAIO buffers of pairs
 * [pair_begin, pair_end) into rec_arena (arena_units 64-byte units), laid out
 * with out->pair_off.  Call it after tera_partition of the same iteration on
 * this context (the whole pair range is packed in agent order from the
 * partition's entry list). */
tera_status tera_pack(tera_ctx* ctx, const tera_soa* soa, const tera_partition_out* part,
                      uint32_t pair_begin, uint32_t pair_end, uint8_t* rec_arena,
                      uint64_t arena_units, void* stream);

/* tera_pack of every pair, also writing the id column of the packed records:
 * rec_ids[g] = id (word 0) of record g, g the global record index (pair p's
 * records are g in [pair_off[p], pair_off[p+1])).  rec_ids (device, 8-byte
 * aligned, caller-owned) has room for arena_units entries.  The column lets
 * the batched codec match ids (Sec. 2.3 step B) without reading the 64-byte
 * records a second time (tera_codec_batched_ids).  No counterpart in the paper. */
tera_status tera_pack_ids(tera_ctx* ctx, const tera_soa* soa, const tera_partition_out* part,
                          uint8_t* rec_arena, uint64_t arena_units, uint64_t* rec_ids,
                          void* stream);

/* Steps a3+a4 (Sec. 2.3 B and C): encode messages [pair_begin, pair_end)
 * against the sender reference (ref_prev laid out with ref_off_prev; both
 * NULL means every reference is empty, as at the first iteration).
 *  - writes wire_off[P+1] (slab layout, all pairs), the messages of the
 *    range at wire + wire_off[p], their lengths wire_len[p];
 *  - writes the new sender reference ref_next, laid out with pair_off
 *    (matched records in slot order, then new records in message order).
 * mode TERA_MODE_XOR or TERA_MODE_RAW (raw: the reference is ignored).  A
 * pair marked by tera_reset_reference is sent raw once.  wire_capacity is in
 * bytes; too small latches TERA_ECAPACITY with the required size. */
tera_status tera_delta_encode(tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off,
                              const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                              uint32_t pair_begin, uint32_t pair_end, uint8_t* ref_next,
                              uint8_t* wire, uint64_t wire_capacity, uint64_t* wire_off,
                              uint64_t* wire_len, int mode, void* stream);

/* Step a5 (Sec. 2.3 D): decode messages [pair_begin, pair_end) against the
 * receiver reference (ref_prev/ref_off_prev, NULL = empty) and write the
 * defragmented records into recv (recv_capacity_units 64-byte units), laid
 * out with recv_off[P+1], which this call computes from ALL message headers
 * (m_p = n_slots - n_holes + n_new).  The receive buffer is the receiver's
 * next reference.  Malformed messages latch TERA_ECORRUPT, a slot count
 * differing from the receiver's reference TERA_EREFMISMATCH; the output of
 * such a pair is unspecified. */
tera_status tera_delta_decode(tera_ctx* ctx, const uint8_t* wire, const uint64_t* wire_off,
                              const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                              uint32_t pair_begin, uint32_t pair_end, uint8_t* recv,
                              uint64_t recv_capacity_units, uint64_t* recv_off, void* stream);

/* The decode step for callers that cannot allocate device memory (no
 * counterpart in the paper).  Hosts whose device memory is reserved up front
 * by their own pool, and real-time loops that forbid allocation after
 * start-up, cannot call cudaMalloc, and so cannot create a tera_ctx.  This
 * variant decodes every pair [0, n_pairs) exactly as tera_delta_decode does
 * (same arguments and outputs, same bytes), but takes all of its scratch
 * memory from one fixed array in the library's device memory (about 16.5 MB
 * per GPU that loads the library, held until the process exits); it calls no
 * cudaMalloc, cudaFree or allocating routine.
 *  - Limits: n_pairs <= 32768 (TERA_ECAPACITY beyond, returned at once) and
 *    at most 393216 codec tiles of 256 entries (about 100M slots + new
 *    records).  Beyond the tile limit the call returns TERA_ECAPACITY with
 *    *required_capacity = 0 (no receive capacity would help); a receive
 *    buffer that is too small returns TERA_ECAPACITY with the required units.
 *  - n_pairs must be a multiple of 27 (the grid's box count times 27);
 *    TERA_EINVAL otherwise.
 *  - The first call on a device looks up the array's device address for
 *    that device (with it current) and keeps it for the life of the process;
 *    after cudaDeviceReset on that device, do not call it there again.
 *  - Every call shares the array, which keeps the last call's contents: calls
 *    that overlap on the GPU (other streams, other threads) race on it; the
 *    caller must serialize them.
 *  - Returns the device status of this call: it synchronizes `stream` and
 *    reads the status word back; *required_capacity (optional) is set on
 *    TERA_ECAPACITY as above.  No context status is touched. */
tera_status tera_delta_decode_noalloc(const uint8_t* wire, const uint64_t* wire_off,
                                      const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                                      uint64_t n_pairs, uint32_t class_id, uint8_t* recv,
                                      uint64_t recv_capacity_units, uint64_t* recv_off,
                                      uint64_t* required_capacity, void* stream);

/* ---------------- learned predictor (not in the paper) ----------------
 * A small MLP predicts each agent's next position from its recent motion;
 * a message in mode TERA_MODE_RESIDUAL carries, for the position words
 * (w1..w3) of every matched slot the network can predict, the zigzag of the
 * integer difference of bit patterns, zigzag(bits(x_t) - bits(prediction))
 * (mod 2^64); every other word is the XOR difference.  The encoder sends the
 * residual mode only for messages it makes smaller (plain XOR otherwise).
 *
 * Network: 8 -> 64 -> 64 -> 3, ReLU on the hidden layers, float32.  Params
 * (4931 floats): W1[64][8], b1[64], W2[64][64], b2[64], W3[3][64], b3[3];
 * each neuron computes acc = b; for k ascending acc = fmaf(W[k], in[k], acc)
 * (bit-identical on every device).  Features of reference slot j (position
 * x1 = x_{t-1} from the reference, history xp = x_{t-2}, d2):
 *   (float)(x1 - xp) per axis, d2 per axis, (float)(diameter / 10.0),
 *   (float)ncount * 2^-5 where ncount = reference records of the pair in the
 *   slot's cell floor((x1 - lo) / w) (per axis, the slot itself included).
 * A slot is predictable when its history has two steps and every feature and
 * output is finite; prediction = x1 + (double)output per axis.
 *
 * History (48 bytes per slot, one array per reference, no headers; slot j of
 * pair p at index off[p] + j): u64 xp[3] (bits) | u32 d2[3] (bits of
 * (float)(xp - the position before it)) | u32 n (steps, 0..2) | u64 zero.
 * Both sides keep it; the receiver's decode writes the same histories as the
 * sender's encode. */
typedef struct {
  const float* params;      /* MLP weights (device); NULL: no residual mode (history only) */
  const uint8_t* hist_prev; /* history of the reference; must be NULL iff the reference is */
  uint8_t* hist_next;       /* history of the new reference / receive buffer (may be NULL) */
  float* samples;           /* encoder, may be NULL: 12 floats per reference slot j at
                               index ref_off[p] + j: 8 features, 3 target displacements
                               (float)(x_t - x_{t-1}), valid flag (1 or 0) */
  int allow_residual;       /* encoder: choose the residual mode when smaller */
} tera_predictor;

/* tera_delta_encode / tera_delta_decode with the predictor's histories (and,
 * with params, the residual mode).  Same arguments and outputs otherwise;
 * XOR-mode messages are byte-identical to those of the plain entry points. */
tera_status tera_delta_encode_pred(tera_ctx* ctx, const uint8_t* rec_arena,
                                   const uint64_t* pair_off, const uint8_t* ref_prev,
                                   const uint64_t* ref_off_prev, uint32_t pair_begin,
                                   uint32_t pair_end, uint8_t* ref_next, uint8_t* wire,
                                   uint64_t wire_capacity, uint64_t* wire_off, uint64_t* wire_len,
                                   int mode, const tera_predictor* pred, void* stream);
tera_status tera_delta_decode_pred(tera_ctx* ctx, const uint8_t* wire, const uint64_t* wire_off,
                                   const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                                   uint32_t pair_begin, uint32_t pair_end, uint8_t* recv,
                                   uint64_t recv_capacity_units, uint64_t* recv_off,
                                   const tera_predictor* pred, void* stream);

/* Training of the predictor on the GPU (float32, deterministic).
 * samples: n records of 12 floats as written by the encoder (records with a
 * zero valid flag are skipped; the valid ones are compacted in order).
 * tera_mlp_grad: gradient (4931 floats) of the mean squared error
 *   (1/v) sum_i sum_a (o_ia - y_ia)^2 over all v valid samples.
 * tera_mlp_train: `steps` steps of SGD, params -= lr * c * gradient with
 *   c = min(1, clip / |gradient|) (no clipping when clip <= 0), each on the
 *   next `batch` valid samples (cyclically); *n_valid receives v.
 * Both synchronize `stream` (they read v back). */
tera_status tera_mlp_grad(tera_ctx* ctx, const float* samples, uint64_t n, const float* params,
                          float* grad, uint64_t* n_valid, void* stream);
tera_status tera_mlp_train(tera_ctx* ctx, const float* samples, uint64_t n, float* params,
                           int steps, int batch, float lr, float clip, uint64_t* n_valid,
                           void* stream);

/* Schedule of the batched codec (picked by the autotuner; outputs do not
 * depend on it): threads per block = entries per tile (128, 256, 512 or
 * 1024), blocks per SM of the persistent launch (1..16, block x blocks <=
 * 2048), and the largest message (records) matched in a block's shared-memory
 * hash table: 0 = as large as the shared memory left to the block allows, else
 * a power of two >= 32 (smaller when it does not fit); larger messages use the
 * pair's hash segment in global memory.
 * team_blocks: 0 = a pair far above the average load per block is carried by
 * a team of blocks sized by its load (at most 64, at most half the blocks of
 * the launch); 2..1024 = every such pair is carried by exactly that many
 * blocks.  Team members meet at barriers whose wait is bounded by
 * wait_limit_us microseconds of the GPU's global timer (0 = 1 s; at most
 * 60 s): a team that cannot meet in time (e.g. more members than blocks that
 * can run at once) latches TERA_ETIMEOUT and its pair is abandoned (that
 * pair's outputs are then unspecified; every other pair is still encoded and
 * decoded).  reserved must be 0. */
typedef struct {
  int block;
  int ctas_per_sm;
  int table_records;
  int team_blocks;
  int wait_limit_us;
  int reserved;
} tera_tune;

/* Steps a3-a5 for EVERY pair of one iteration in one persistent launch
 * (batching of uneven subdomain buffers; not in the paper, which batches
 * only large messages, Sec. 2.4 "Communication").  Each block carries whole
 * pairs, one at a time, through encode and decode.  Produces exactly the bytes
 * of tera_delta_encode + tera_delta_decode over all pairs: wire_off, the wire
 * messages, wire_len, the new sender reference ref_next (laid out with
 * pair_off) and the receive buffers recv with recv_off.  The receive layout
 * is the iteration's pair layout (recv_off = pair_off); every message header's
 * record count is checked against it (TERA_ECORRUPT otherwise).  The sender
 * reference is ref_prev/ref_off_prev, the receiver's recv_prev/recv_off_prev
 * (NULL pairs = empty references).  rec_arena is any packed arena laid out
 * with pair_off (record ids are read from the records).  tune == NULL uses
 * {256, 4, 0, 0, 0, 0}.  Asynchronous, no host synchronization (graph-capturable once
 * scratch is reserved); device errors are latched in the status word.  Small
 * pairs (at most 512 slots, records and receiver slots) are carried by a
 * second launch on a stream the context owns, forked from `stream` after the
 * call's first kernel and joined back into it before the call returns (CUDA
 * events), so all of the call's work is ordered on `stream` like one launch;
 * a context is not to be used from two streams at once. */
tera_status tera_codec_batched(tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off,
                               const uint8_t* ref_prev, const uint64_t* ref_off_prev,
                               uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
                               uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
                               const uint64_t* recv_off_prev, uint8_t* recv,
                               uint64_t recv_capacity_units, uint64_t* recv_off, int mode,
                               const tera_tune* tune, void* stream);

/* Id columns of the batched codec (no counterpart in the paper).  The match
 * of Sec. 2.3 (step B) needs the id of every message record and of every
 * reference slot before any difference can be formed; read from the records
 * themselves, every 64-byte record is fetched from memory once for its id and
 * again for the difference.  With these columns (device, 8-byte aligned,
 * caller-owned) the codec reads the ids from compact arrays instead:
 *   msg       [E] id of packed record g (as tera_pack_ids writes it);
 *   ref_prev  [R] ids of the sender reference's records, slot j of pair p at
 *             ref_off_prev[p] + j (NULL exactly when ref_prev is NULL): the
 *             ref_next column of the call that wrote that reference;
 *   ref_next  [E] written: ids of the new sender reference's records (record
 *             k of pair p at pair_off[p] + k).
 * Each column must hold the ids of its arena's records (word 0); the codec
 * trusts them for the match, and a column that disagrees with its records
 * gives unspecified messages (the decoder rejects a matched slot whose id
 * word differs). */
typedef struct {
  const uint64_t* msg;
  const uint64_t* ref_prev;
  uint64_t* ref_next;
} tera_ids;

/* tera_codec_batched with the id columns above (same arguments and outputs,
 * same bytes; also writes ids->ref_next). */
tera_status tera_codec_batched_ids(tera_ctx* ctx, const uint8_t* rec_arena,
                                   const uint64_t* pair_off, const uint8_t* ref_prev,
                                   const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire,
                                   uint64_t wire_capacity, uint64_t* wire_off, uint64_t* wire_len,
                                   const uint8_t* recv_prev, const uint64_t* recv_off_prev,
                                   uint8_t* recv, uint64_t recv_capacity_units, uint64_t* recv_off,
                                   int mode, const tera_tune* tune, const tera_ids* ids,
                                   void* stream);

/* tera_codec_batched with the predictor: enc_pred for the sender side (its
 * hist_prev / hist_next travel with ref_prev / ref_next), dec_pred for the
 * receiver (recv_prev / recv).  Either may be NULL (no history on that side). */
tera_status tera_codec_batched_pred(
    tera_ctx* ctx, const uint8_t* rec_arena, const uint64_t* pair_off, const uint8_t* ref_prev,
    const uint64_t* ref_off_prev, uint8_t* ref_next, uint8_t* wire, uint64_t wire_capacity,
    uint64_t* wire_off, uint64_t* wire_len, const uint8_t* recv_prev,
    const uint64_t* recv_off_prev, uint8_t* recv, uint64_t recv_capacity_units,
    uint64_t* recv_off, int mode, const tera_tune* tune, const tera_predictor* enc_pred,
    const tera_predictor* dec_pred, void* stream);

/* Copy the wire messages of one iteration, wire[0, wire_off[P]) with P the
 * context's pair count, into host memory host_dst, and the byte count into
 * *host_count.  The paper sends the buffers over MPI (Sec. 2.4); here a
 * kernel writes them into host memory the device can address (pinned memory
 * from cudaHostAlloc / cudaHostRegister, or memory the system lets the device
 * access), so the length never has to be read back before the copy is issued.
 * host_dst must be 16-byte aligned; wire_off[P] is a multiple of 16.  A
 * length above host_capacity latches TERA_ECAPACITY (required = the length)
 * and copies nothing; *host_count is written in every case.  Asynchronous on
 * `stream`: host_dst and *host_count are valid once the stream has reached
 * this point (e.g. after an event recorded behind it completes).  The paper
 * has no counterpart (it sends from host memory). */
tera_status tera_wire_to_host(tera_ctx* ctx, const uint8_t* wire, const uint64_t* wire_off,
                              uint8_t* host_dst, uint64_t host_capacity, uint64_t* host_count,
                              void* stream);

/* Sec. 2.2.1 "Deserialization": check the TAIO header of ONE pair buffer
 * (device pointer `buf`, `len` bytes available) on the host and return a
 * device pointer to its first record and the record count.  Reads the
 * 64-byte header back (synchronizing `stream`); reads or writes nothing
 * else.  TERA_ECORRUPT for a wrong magic, version, record size or class id,
 * or a count that does not fit in len. */
tera_status tera_unpack_inplace(const uint8_t* buf, uint64_t len, uint32_t class_id,
                                void** view, uint64_t* count, void* stream);

/* Device-side form of the same check for every pair of an arena (for use
 * inside captured graphs): latches TERA_ECORRUPT when a header's magic,
 * version, size, class id, pair or count (off[p+1]-off[p]) is wrong. */
tera_status tera_unpack_validate(tera_ctx* ctx, const uint8_t* arena, const uint64_t* off,
                                 void* stream);

/* Agent migration (Sec. 2.1 "Agent Migration"): agents whose position now
 * lies in another box move there, as raw TeraAgent IO records (Sec. 2.2.1;
 * no difference encoding, which is for the aura).
 *
 * The state is box-major: box s holds agents [box_off_prev[s],
 * box_off_prev[s+1]) of `prev` (box_off_prev[0] = 0, non-decreasing,
 * box_off_prev[B] = n; B = n[0]*n[1]*n[2]).  The destination of an agent is
 * the owner box of its position by the rule of tera_partition.  Leavers of
 * box s for box d go to inbox q = d*27 + b, b the neighbour bit of the offset
 * from d to s (the side they arrive from; on a toroidal axis modulo n), or
 * b = 13 when s is not a neighbour of d (the paper's case of a destination
 * outside the locally available boxes, whose lookup here is the same rule).
 * An inbox holds its leavers in ascending agent index.
 *
 * tera_migrate_send writes inbox_off[Q+1] (Q = 27 B; records per inbox,
 * exclusive prefix), the inboxes into `arena` as a TAIO arena (inbox q at
 * units [inbox_off[q] + q, inbox_off[q+1] + q + 1): header with pair field q,
 * then its records), box_off_next[B+1], and every stayer into `next`: box d
 * starts with its stayers in their previous order.  More than arena_units
 * units latch TERA_ECAPACITY (required units reported) and abort the step;
 * a box_off_prev that breaks the rules above latches TERA_EINVAL.  An agent
 * outside [lo, hi) latches TERA_EDOMAIN and is kept in its box.
 * tera_migrate_recv deserializes every inbox of the arena into `next`: the
 * records of box d's inboxes, in ascending side and message order, follow
 * its stayers.  Headers are checked (TERA_ECORRUPT), and so is every index
 * against the arena and the state; nothing outside them is touched.
 * prev and next (n agents each) must not overlap; columns and the arena are
 * 16-byte aligned.  Both calls are asynchronous on `stream`. */
tera_status tera_migrate_send(tera_ctx* ctx, const tera_soa* prev, const uint64_t* box_off_prev,
                              uint8_t* arena, uint64_t arena_units, uint64_t* inbox_off,
                              const tera_soa_mut* next, uint64_t* box_off_next, void* stream);
tera_status tera_migrate_recv(tera_ctx* ctx, const uint8_t* arena, uint64_t arena_units,
                              const uint64_t* inbox_off, const uint64_t* box_off_next,
                              const tera_soa_mut* next, void* stream);

/* Reference interval (Sec. 2.3: the reference is updated "at regular
 * intervals"; every K-th iteration here, K = ref_interval >= 1).  The message
 * of iteration 0 and of every multiple of K becomes the reference of the
 * following iterations, so iteration t >= 1 encodes (and decodes) against the
 * message of iteration K * floor((t - 1) / K).  A caller keeps two reference
 * buffers on each side (sender reference + its offsets, receive buffer + its
 * offsets); iteration t writes its outputs into buffer *out_buf =
 * ceil(t / K) mod 2, and reads its references from buffer *ref_buf (the
 * out_buf of that reference iteration; -1 at t = 0, which has no reference).
 * *ref_iteration (optional) receives K * floor((t - 1) / K) (0 at t = 0).
 * Host-only arithmetic; TERA_EINVAL when ref_interval is 0 or out_buf is NULL. */
tera_status tera_ref_schedule(uint64_t t, uint32_t ref_interval, int32_t* out_buf,
                              int32_t* ref_buf, uint64_t* ref_iteration);

/* Buckets per axis of the classification tables (tera_axis_buckets). */
#define TERA_AXIS_BUCKETS 8192

/* The classification tables a context of this grid uses in tera_partition
 * (Sec. 2.1, "Aura Update": an agent's owner box and the neighbours whose
 * aura holds it, per axis; Sec. 2.4.1: the partitioning grid).  Host-only
 * arithmetic, no device work; the result of the classification never depends
 * on them.  Axis a's domain [lo, hi) is cut into TERA_AXIS_BUCKETS buckets.
 * The device places a coordinate v (only when 2^-126 <= |v| < 2^128) in bucket
 * j = trunc((f - flo[a]) * fs[a]), in float32 arithmetic, f being v's binary64
 * value with its mantissa cut to 20 bits.  tab[a * TERA_AXIS_BUCKETS + j] is
 * 0x80 when the exact comparisons decide for the values placed in bucket j,
 * else (i << 2) | q for every value placed there: i the box index along the
 * axis, q bit 0 when the aura of the neighbour at offset -1 holds v, bit 1 for
 * offset +1.  *on = 0 (tab, flo, fs untouched) when the grid gets no tables:
 * an axis of more than 32 boxes, or a domain whose float estimate is too
 * coarse for its bucket width.  tab (3 * TERA_AXIS_BUCKETS bytes), flo and fs
 * (3 floats each) and on are caller-owned.  TERA_EINVAL when a pointer is
 * NULL or tera_ctx_create would reject the grid. */
tera_status tera_axis_buckets(const tera_grid* grid, uint8_t* tab, float* flo, float* fs, int* on);

/* Cell boundaries of one axis of the predictor's cell grid (the ncount
 * feature above; cells of width w from lo, cell(x) = floor((x - lo) / w) in
 * binary64).  Host-only arithmetic, no device work: the library builds these
 * tables once per context (for axes of at most 65536 cells) so that the
 * device finds a cell by integer comparisons instead of binary64 division.
 * n must be floor((hi - lo) / w) + 1 (the context's cell count of the axis);
 * T (caller-owned, n + 1 entries) receives T[0] = key(lo), T[n] = key(hi)
 * and, for 1 <= k < n, T[k] = key of the smallest binary64 x with
 * cell(x) >= k, where key(x) is the order-preserving map of x's bits
 * (b ^ 0x8000000000000000 for a non-negative x, ~b for a negative one,
 * -0.0 taken as +0.0).  A value x in [lo, hi) then lies in the largest cell
 * k < n with key(x) >= T[k].  TERA_EINVAL when T is NULL, lo, hi or w is
 * not finite, lo >= hi, w <= 0, or n is not that count. */
tera_status tera_cell_thresholds(double lo, double hi, double w, uint64_t n, uint64_t* T);

/* Read (and clear) the latched device status; synchronizes `stream`.
 * *required_capacity (optional) receives the largest capacity a call asked
 * for when the status is TERA_ECAPACITY. */
tera_status tera_ctx_status(tera_ctx* ctx, uint64_t* required_capacity, void* stream);

/* Send pair p raw (against an empty reference) at the next tera_delta_encode
 * that covers it.  Use after mutating a received view, which invalidates the
 * pair's reference on the receiving side. */
tera_status tera_reset_reference(tera_ctx* ctx, uint32_t pair);

/* Totals accumulated on the device by every call of the context since the
 * last reset: iterations (tera_partition calls), agents classified, records
 * packed into messages (sum of m_p), reference slots encoded against (sum of
 * r_p), placeholders, new records, payload bytes and wire-message bytes
 * (sum of message lengths) written by tera_delta_encode.  No counterpart in
 * the paper; used for bytes-per-agent and bandwidth accounting. */
typedef struct {
  uint64_t iterations, agents, records, ref_slots, holes, new_records, payload_bytes,
      wire_bytes;
} tera_stats;

/* Read the totals (synchronizes `stream`); reset != 0 zeroes them afterwards. */
tera_status tera_ctx_stats(tera_ctx* ctx, tera_stats* out, int reset, void* stream);

/* Kernels this context has launched so far (for launch accounting). */
uint64_t tera_ctx_launches(const tera_ctx* ctx);

/* Measurement support (no counterpart in the paper).  When enabled, every
 * kernel launch of the context is bracketed by a pair of CUDA events on its
 * stream.  tera_ctx_profile_collect waits for the recorded events and adds
 * their durations into a per-kernel table (kernel name, launches, total ms);
 * tera_ctx_profile_entries / tera_ctx_profile_entry read the table (names stay
 * valid until tera_ctx_profile_reset or tera_ctx_destroy); reset collects and
 * clears it. */
tera_status tera_ctx_profile(tera_ctx* ctx, int enable);
tera_status tera_ctx_profile_collect(tera_ctx* ctx);
int tera_ctx_profile_entries(const tera_ctx* ctx);
tera_status tera_ctx_profile_entry(const tera_ctx* ctx, int i, const char** name,
                                   uint64_t* launches, double* total_ms);
tera_status tera_ctx_profile_reset(tera_ctx* ctx);

/* Library version string. */
const char* tera_version(void);

#ifdef __cplusplus
}
#endif
#endif
