// tera_delta_decode_noalloc — the decode step with no allocation at all.
//
// Some callers cannot allocate device memory at the point where they decode:
// hosts whose device memory is reserved up front by their own pool, so that
// third-party code may not call cudaMalloc, and real-time loops that forbid
// allocation after start-up.  They cannot create a tera_ctx either (context
// creation allocates).  This entry point runs the same decode kernels as
// tera_delta_decode with every piece of scratch memory — unit layout, per-pair
// facts, per-unit sums and bases, status word — taken from one file-scope
// device array of fixed size, so it calls no cudaMalloc, cudaFree or
// allocating routine.  The caller still passes the inputs and outputs.
//
// The array (kScratchBytes below, about 16.5 MB) exists on every GPU that
// loads this library, until the process exits.  Every call shares it and it
// keeps the last call's contents; calls that overlap on the GPU (from two
// streams or two threads) race on it and must be serialized by the caller.
//
// The array's device address is looked up once per device, by the first call
// made with that device current, and kept for the life of the process; after
// cudaDeviceReset on that device the kept address is stale, so the library
// must not be called there again.
#define TERA_DECODE_KERNELS_ONLY
#include "decode.cu"

#include <mutex>

namespace {

constexpr tera::u64 kStaticMaxPairs = 32768;   // grids up to 1213 boxes (27 pairs each)
constexpr tera::u64 kStaticMaxUnits = 393216;  // codec tiles of 256 entries (~100M entries)

constexpr tera::u64 kOffStatus = 0;
constexpr tera::u64 kOffUnitsTotal = 128;
constexpr tera::u64 kOffUnitOff = 256;
constexpr tera::u64 kOffInfo = kOffUnitOff + 8 * (kStaticMaxPairs + 1) + 248;  // 256-aligned
constexpr tera::u64 kOffUnitPair = kOffInfo + 64 * kStaticMaxPairs;
constexpr tera::u64 kOffUnitSum = kOffUnitPair + 4 * kStaticMaxUnits;
constexpr tera::u64 kOffUnitBase = kOffUnitSum + 16 * kStaticMaxUnits;
constexpr tera::u64 kScratchBytes = kOffUnitBase + 16 * kStaticMaxUnits;

static_assert(kOffInfo % 256 == 0 && kOffUnitPair % 256 == 0 && kOffUnitSum % 256 == 0 &&
                  kOffUnitBase % 256 == 0,
              "scratch regions are 256-byte aligned");

// The scratch.  Host code never uses this name as an address: in host code it
// is only a stand-in, and the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_decode_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, under a lock; not looked up again after a device reset).
tera_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return TERA_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_decode_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return TERA_ECUDA;
    }
    g_scratch_addr[device] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_addr[device];
  return TERA_OK;
}

__global__ void static_unit_map_kernel(const tera::u64* __restrict__ unit_off, tera::u64 npr,
                                       tera::u32* __restrict__ unit_pair,
                                       const tera::u64* __restrict__ units_total) {
  if (units_total[1]) return;
  const int lane = threadIdx.x & 31;
  const tera::u64 warp = ((tera::u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const tera::u64 nwarps = ((tera::u64)gridDim.x * blockDim.x) >> 5;
  for (tera::u64 k = warp; k < npr; k += nwarps)
    for (tera::u64 u = unit_off[k] + lane; u < unit_off[k + 1]; u += 32)
      unit_pair[u] = (tera::u32)k;
}

}  // namespace

extern "C" tera_status tera_delta_decode_noalloc(const uint8_t* wire, const uint64_t* wire_off,
                                                 const uint8_t* ref_prev,
                                                 const uint64_t* ref_off_prev, uint64_t n_pairs,
                                                 uint32_t class_id, uint8_t* recv,
                                                 uint64_t recv_capacity_units, uint64_t* recv_off,
                                                 uint64_t* required_capacity, void* stream) {
  using namespace tera;
  if (required_capacity) *required_capacity = 0;
  if (!wire || !wire_off || !recv || !recv_off) return TERA_EINVAL;
  if ((ref_prev == nullptr) != (ref_off_prev == nullptr)) return TERA_EINVAL;
  if (n_pairs == 0 || n_pairs % 27 != 0) return TERA_EINVAL;
  if (n_pairs > kStaticMaxPairs) return TERA_ECAPACITY;  // beyond the fixed scratch
  if (((uintptr_t)wire | (uintptr_t)recv | (uintptr_t)(ref_prev ? ref_prev : recv)) & 15u)
    return TERA_EINVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return TERA_ECUDA;
  unsigned char* base = nullptr;
  tera_status st = scratch_address(device, &base);
  if (st != TERA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DevStatus* status = reinterpret_cast<DevStatus*>(base + kOffStatus);
  u64* units_total = reinterpret_cast<u64*>(base + kOffUnitsTotal);
  // the status word must start at zero; everything else is written before it is read
  if (cudaMemsetAsync(status, 0, sizeof(DevStatus), s) != cudaSuccess) return TERA_ECUDA;
  DecArgs A;
  A.wire = wire;
  A.wire_off = reinterpret_cast<const u64*>(wire_off);
  A.ref = ref_prev;
  A.ref_off = reinterpret_cast<const u64*>(ref_off_prev);
  A.recv = recv;
  A.recv_off = reinterpret_cast<u64*>(recv_off);
  A.unit_off = reinterpret_cast<const u64*>(base + kOffUnitOff);
  A.units_total = units_total;
  A.unit_pair = reinterpret_cast<const u32*>(base + kOffUnitPair);
  A.unit_sum = reinterpret_cast<U64x2*>(base + kOffUnitSum);
  A.unit_base = reinterpret_cast<U64x2*>(base + kOffUnitBase);
  A.info = reinterpret_cast<u64*>(base + kOffInfo);
  A.p0 = 0;
  A.p1 = (u32)n_pairs;
  A.class_id = class_id;
  A.st = status;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (sms <= 0) sms = 148;
  dec_setup_kernel<false><<<1, 1024, 0, s>>>(A, n_pairs, recv_capacity_units, units_total,
                                             kStaticMaxUnits);
  static_unit_map_kernel<<<(unsigned)((n_pairs + 7) / 8), 256, 0, s>>>(
      A.unit_off, n_pairs, reinterpret_cast<u32*>(base + kOffUnitPair), units_total);
  const unsigned g = (unsigned)sms * 8u;
  dec_sum_kernel<<<g, kCodecTile, 0, s>>>(A);
  dec_scan_kernel<<<(unsigned)((n_pairs + 7) / 8), 256, 0, s>>>(A);
  dec_emit_kernel<false><<<g, kCodecTile, 0, s>>>(A);
  if (cudaGetLastError() != cudaSuccess) return TERA_ECUDA;
  DevStatus h;
  if (cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TERA_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TERA_ECUDA;
  if (required_capacity) *required_capacity = h.required;
  return (tera_status)h.code;
}
