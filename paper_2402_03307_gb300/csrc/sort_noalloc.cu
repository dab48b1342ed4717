// r4g_sort_pairs_noalloc: the stable radix sort of r4g_sort_pairs for callers
// that cannot allocate device memory and so cannot provide a scratch buffer
// (for example a plug-in running inside a host application that owns the
// GPU's memory budget, or a real-time loop where an allocator call and its
// synchronisation are not acceptable). Its scratch -- the ping-pong key and
// value buffers and the per-pass digit counts -- lives in one file-scope
// device array of fixed size, so the call performs no allocation at all.
//
// Properties a caller must know:
//  * the array is R4G_SORT_NOALLOC_SCRATCH_BYTES (about 12.3 MiB) and every
//    GPU that loads the library holds it until the process exits;
//  * n is limited to R4G_SORT_NOALLOC_MAX_PAIRS; larger n is rejected with
//    R4G_EINVAL before anything is enqueued;
//  * every call on a device shares the same array, which keeps the previous
//    call's contents: calls that can overlap on the GPU (different streams
//    without ordering between them) race on it and corrupt each other's
//    results -- serialise them on one stream or with events;
//  * nothing in the array has to start at zero: each pass writes every digit
//    count and every buffer element it later reads;
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current and caches it; make
//    that first call before any stream capture is started. The cache belongs
//    to the device's primary context and does not survive cudaDeviceReset.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "r4g.h"
#include "r4g_internal.cuh"

namespace r4g {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t al(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr int64_t kMaxPairs = R4G_SORT_NOALLOC_MAX_PAIRS;
constexpr int kMaxCtas = kSortMaxCtas;  // upper bound of sort_ctas_for()
constexpr size_t kKeysOff = 0;
constexpr size_t kValsOff = al(sizeof(uint64_t) * kMaxPairs);
constexpr size_t kCntOff = kValsOff + al(sizeof(uint32_t) * kMaxPairs);
constexpr size_t kBytes = kCntOff + al(sizeof(uint32_t) * kSortRadix * kMaxCtas);
static_assert(kBytes == R4G_SORT_NOALLOC_SCRATCH_BYTES, "header constant out of date");

// The scratch itself. In host code this name is only a host-side handle: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

r4g_status err(r4g_status st, const char* msg) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "r4g_sort_pairs_noalloc: %s", msg);
  set_last_error(buf);  // readable through r4g_last_error(NULL)
  return st;
}

// Device address of g_sort_scratch on the current device (looked up once per
// device, with that device current).
r4g_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(R4G_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return err(R4G_EDEVICE, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p) return err(R4G_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return R4G_OK;
}

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

}  // namespace
}  // namespace r4g

extern "C" r4g_status r4g_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* values_in,
                                             uint64_t* keys_out, uint32_t* values_out, int64_t n,
                                             int32_t begin_bit, int32_t end_bit, void* stream) {
  using namespace r4g;
  if (n < 0) return err(R4G_EINVAL, "n is negative");
  if (n > kMaxPairs) return err(R4G_EINVAL, "n exceeds R4G_SORT_NOALLOC_MAX_PAIRS (1048576 pairs)");
  if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit) return err(R4G_EINVAL, "bad bit range");
  if (n == 0) return R4G_OK;
  if (!keys_in || !values_in || !keys_out || !values_out) return err(R4G_EINVAL, "NULL buffer");
  if (!aligned8(keys_in) || !aligned8(keys_out)) return err(R4G_EINVAL, "keys must be 8-byte aligned");
  if (keys_in == keys_out || values_in == values_out) return err(R4G_EINVAL, "outputs alias inputs");
  void* base = nullptr;
  const r4g_status st = scratch_address(&base);
  if (st != R4G_OK) return st;
  uint64_t* tk = reinterpret_cast<uint64_t*>(static_cast<char*>(base) + kKeysOff);
  uint32_t* tv = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + kValsOff);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + kCntOff);
  const int passes = (end_bit - begin_bit + kSortRadixBits - 1) / kSortRadixBits;
  const bool last_even = (passes - 1) % 2 == 0;  // the last pass writes buffer 1 when even
  int which = 0;
  const cudaError_t e = launch_sort(keys_in, values_in, last_even ? keys_out : tk, last_even ? values_out : tv,
                                    last_even ? tk : keys_out, last_even ? tv : values_out, nullptr,
                                    static_cast<uint32_t>(n), n, begin_bit, end_bit, cnt, sort_ctas_for(n),
                                    static_cast<cudaStream_t>(stream), &which);
  if (e != cudaSuccess) return err(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}
