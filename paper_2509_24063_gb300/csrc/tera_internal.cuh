// Internal definitions shared by the CUDA translation units of libtera: the
// device-side helpers (tera_device.cuh) and the host-side context.
#pragma once

#include <cstddef>

#include <nvtx3/nvToolsExt.h>

#include "tera_device.cuh"

namespace tera {
// One NVTX range around a library call, named after the entry point (shown by
// Nsight Systems on the calling thread; nothing happens when no tool is
// attached).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};
}  // namespace tera

#define TERA_CALL_RANGE(name) ::tera::CallRange tera_call_range_(name)

namespace tera {
// Classification by table (the partition's classify_kernel).  Each axis's
// domain [lo, hi) is cut into kAxisBuckets equal buckets.  The device places
// a coordinate v in bucket j = trunc((approx_f32(v) - flo) * fs); the host
// bounds how far that estimate can stray from v's true place and stores, for
// every bucket that no threshold value (lo, hi, a box edge, e[k] + w,
// e[k+1] - w) can reach within that bound, what every v placed there gets:
// the box index (bits 2..6) and the aura offsets -1 (bit 0) and +1 (bit 1).
// Other buckets hold kBucketExact, and those agents take the exact key
// comparisons.  The table exists when every axis has at most 32 boxes and the
// estimate's error stays under a quarter bucket (on == 0 otherwise).
constexpr int kAxisBuckets = TERA_AXIS_BUCKETS;
constexpr uint8_t kBucketExact = 0x80;
struct AxisBuckets {
  int on;
  float flo[3], fs[3];
  alignas(16) uint8_t tab[3][kAxisBuckets];  // copied to shared memory in 16-byte pieces
};
static_assert(offsetof(AxisBuckets, tab) % 16 == 0, "bucket tables are read as 16-byte vectors");
}  // namespace tera

// The context (host side).
struct tera_ctx {
  int device;
  uint32_t class_id;
  tera_grid grid;
  uint32_t n_boxes;
  uint64_t n_pairs;
  int num_sms;
  uint64_t launches;
  uint64_t iterations;

  tera::GridTables* d_grid;
  tera::AxisBuckets* d_buckets;  // null when classification has no table
  tera::DevStatus* d_status;
  tera::DevStatus* h_status;  // pinned
  uint32_t* d_epoch;
  uint8_t* d_reset;  // [P] pairs to send raw once

  // partition scratch
  int64_t cap_agents;
  uint64_t cap_records;
  uint32_t* tile_cnt;      // [runs + 1] entries per run of 64 agents
  tera::u64* tile_base;     // [runs + 1] entries before each run
  // entries (agent, pair) of the last partition in agent order, and where
  // each went in the pair-sorted order (pack reads them in agent order)
  uint32_t* keys_a;        // [cap_records] pair of entry e
  uint32_t* ent_agent;     // [cap_records] agent of entry e
  uint32_t* ent_dest;      // [cap_records] record index of entry e
  uint32_t* keys_b;        // sort passes
  uint32_t* keys_c;
  uint32_t* vals_b;
  uint32_t* vals_c;
  uint32_t* agents_b;      // agents carried through the sort passes
  uint32_t* agents_c;
  uint32_t* rec_pair;      // pair of each record of the last partition (sorted keys)
  int64_t pack_n;          // agents of the last partition (its runs cover them)
  uint32_t* rs_hist;       // [kRadix * sort tiles]
  tera::u64* scan_part;     // partials of the generic scan
  uint64_t scan_part_cap;
  tera::u64* d_total;       // [4] scalars: total records, ...

  // per-pair hash segments + codec scratch
  tera::U64x2* seg;      // [2 cap_records + 2 P] hash entries {tag, id}
  uint32_t* matched;     // [cap_records] epoch of the iteration in which a slot took the record
  uint32_t* slot_src;  // [cap_records]
  tera::u64* unit_off;  // [P + 1]
  uint64_t cap_units;
  tera::U64x2* unit_sum;   // [cap_units]
  uint32_t* unit_pair;     // [cap_units] pair of each codec unit
  tera::U64x2* unit_base;  // [cap_units]
  tera::u64* pair_info;     // [P * 8] per-pair codec facts
  tera::u64* d_units_total;
  void* prof;  // per-kernel CUDA-event timing (ctx.cu)
  tera::DevStats* d_stats;


  // learned predictor (cell counts of both sides, per-slot predictions)
  uint64_t ncell[3];
  tera::u64* d_ckeys;       // cell thresholds of the axes that have a table
  const tera::u64* ck[3];   // axis a's table in d_ckeys (null: none)
  float ck_flo[3], ck_fs[3];
  uint64_t pred_cap;
  tera::u64* cseg_enc;
  tera::u64* cseg_dec;
  tera::u64* pscr;
  tera::u64* pscr_dec;      // the receiver's predictions (batched pre-pass)
  tera::u64* unit_res;
  uint64_t unit_res_cap;
  float* mlp_scratch;       // training: compacted samples + gradient partials
  uint64_t mlp_scratch_cap;
  // batched codec (batched.cu)
  cudaStream_t b_side;     // the small-pair launch runs on it, forked from and joined to the
  cudaEvent_t b_fork, b_join;  // caller's stream by these events
  tera::u64* b_scalars;  // [0] work items, [1] ticket, [2] abort flag, [3] first small-pair
                         // item, [4] ticket of the small-pair launch
  tera::u64* b_ptot;     // [P * 4] per-pair totals of the match step
  tera::u64* b_items;    // work list (team items first)
  uint64_t b_items_cap;
  uint32_t* b_team;      // [P * 8] barrier counters of the teams
  tera::U64x2* b_tsum;   // per-tile totals of the team pairs
  uint64_t b_tsum_cap;
  tera::u64* b_tbase;    // [P] first tile total of each team pair
  tera::u64* b_part;     // [4 * (P / 1024 + 1)] block sums of the setup's first launch
  // agent migration (migrate.cu)
  uint64_t m_cap_agents;   // agents the tile arrays cover
  uint64_t m_cap_leavers;  // leavers the list and sort buffers hold
  uint32_t* m_tile_cnt;    // [warp tiles + 1] leavers per warp tile of 256 agents
  tera::u64* m_tile_base;  // [warp tiles + 1] leavers before each warp tile (total last)
  tera::u64* m_from;       // [boxes] leavers per source box
  tera::u64* m_before;     // [boxes] leavers of the boxes before each box
  tera::u64* m_cnt;        // [boxes * 27] leavers per inbox
  uint32_t* m_key;         // [m_cap_leavers] inbox of leaver k (agent order)
  uint32_t* m_agent;       // [m_cap_leavers] agent of leaver k
  uint32_t* m_sorted;      // [m_cap_leavers] agent of inbox record j
  uint32_t* m_dest;        // [m_cap_leavers] inbox-order position of leaver k
  uint32_t* m_keys_b;
  uint32_t* m_keys_c;
  uint32_t* m_vals_b;
  uint32_t* m_vals_c;
  uint32_t* m_agents_b;
  uint32_t* m_agents_c;
  uint32_t* m_hist;
};

namespace tera {
// ctx.cu
void prof_begin(tera_ctx* ctx, cudaStream_t s);
tera_status check_launch(tera_ctx* ctx, const char* name, cudaStream_t s);
tera_status ensure_agents(tera_ctx* ctx, int64_t n, cudaStream_t s);
tera_status ensure_records(tera_ctx* ctx, uint64_t cap, cudaStream_t s);
tera_status ensure_units(tera_ctx* ctx, uint64_t cap, cudaStream_t s);
// Exclusive scan of n u32 values into n+1 outputs (total last), any n.
tera_status scan_u32(tera_ctx* ctx, const u32* in, u64* out64, u32* out32, u64 n, cudaStream_t s);
int grid_for(tera_ctx* ctx, int blocks_per_sm);
// unit_pair[u] = p0 + k for every unit u of range pair k (skipped when
// units_total[1] flags an aborted call).
tera_status launch_unit_map(tera_ctx* ctx, u32 p0, u64 npr, cudaStream_t s);
// Scratch of the learned predictor for the current record capacity.
tera_status ensure_pred(tera_ctx* ctx);
// Scratch of the batched codec.
tera_status ensure_batched(tera_ctx* ctx);
// Scratch of agent migration for n agents and up to `leavers` leavers.
tera_status ensure_migrate(tera_ctx* ctx, uint64_t n, uint64_t leavers);

// partition.cu: stable LSD radix sort of entries by u32 key.
struct SortBufs {
  u32* keys_b;
  u32* keys_c;
  u32* vals_b;
  u32* vals_c;
  u32* agents_b;  // agents carried with the entries between passes
  u32* agents_c;
  u32* hist;  // [kRadix * sort tiles + 1]
};
tera_status radix_sort_entries(tera_ctx* ctx, const SortBufs& b, const u32* keys_in,
                               const u32* agent, u32* dest, u32* vals_final, const u64* total_ptr,
                               u64 cap, u64 key_limit, const u32** sorted_keys, cudaStream_t s);
}  // namespace tera
