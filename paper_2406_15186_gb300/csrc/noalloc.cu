// Allocation-free variant of the per-(segment, width) maxima.
//
// Some callers cannot call cudaMalloc: a real-time pipeline that hands out all
// device memory from its own pool (a cudaMalloc would synchronise the device
// and stall the stream that carries the telescope data), a process under a
// hard device-memory cap, or code that must not allocate while other work is
// being captured.  pulscan_segment_maxima_noalloc serves them: the caller
// passes the power spectrum and the two output arrays, and the only other
// device memory the call touches is one file-scope static __device__ array
// (kNoAllocWords 64-bit words, 8 MiB plus a small header), which every GPU
// that loads the library holds until the process exits.
//
// The first call on a device does a one-time set-up with that device current:
// it looks up the array's device address with cudaGetSymbolAddress (in host
// code the symbol's name is only a host-side stand-in, not a device address)
// and sets the kernel's shared-memory limit.  Make that first call before any
// stream capture.  Every call shares the one array: calls whose work overlaps
// on the GPU (other streams, other host threads) race and must be serialised
// by the caller.  The slots a call uses are cleared at its start, and the
// kernel that reads them clears them again.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace ps {

namespace {

constexpr int64_t kNoAllocSlots = int64_t(1) << 20;        // segments x z_max at most
constexpr int kNoAllocMaxW = 4096;                          // z_max at most
constexpr int64_t kHeaderWords = 16;                        // series descriptor, tile offsets, counters
constexpr int64_t kNoAllocWords = kNoAllocSlots + kHeaderWords;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

// Header layout (after the slots): SeriesDev (7 words), tile_off[2], counters (2 words).
__global__ void noalloc_header_kernel(SeriesDev *series, int64_t *tile_off, uint32_t *counters, SeriesDev value,
                                      int64_t tiles) {
  if (threadIdx.x == 0) {
    *series = value;
    tile_off[0] = 0;
    tile_off[1] = tiles;
    counters[0] = counters[1] = counters[2] = counters[3] = 0u;
  }
}

int scratch_for_current_device(unsigned long long **out) {
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PULSCAN_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *ptr = nullptr;
    PS_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    // the kernel's shared-memory limit for the largest accepted shape
    const int rc = prepare_bank_raw(kNoAllocMaxW, 4);
    if (rc) return rc;
    g_scratch_ptr[dev] = static_cast<unsigned long long *>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return PULSCAN_OK;
}

}  // namespace

}  // namespace ps

using namespace ps;

extern "C" int pulscan_segment_maxima_noalloc(const float *d_power, int64_t n, int32_t z_max, int32_t segment_len,
                                              float *d_max, uint64_t *d_argmax, pulscan_stream stream) {
  if (!d_power || !d_max || !d_argmax) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if ((reinterpret_cast<uintptr_t>(d_power) & 15u) != 0u)
    return fail(PULSCAN_ERR_INVALID_ARG, "power buffer must be 16-byte aligned");
  if (n < 2 || (n & 1)) return fail(PULSCAN_ERR_INVALID_ARG, "series length must be even and >= 2");
  // bins are 32-bit in the (power, bin) merge keys: M = n/2 + 1 <= 2^32
  if (n >= (int64_t(1) << 33)) return fail(PULSCAN_ERR_UNSUPPORTED, "series of 2^33 samples or more");
  const int64_t m = n / 2 + 1;
  if (z_max < 1 || segment_len < z_max || segment_len > m)
    return fail(PULSCAN_ERR_INVALID_ARG, "need 1 <= z_max <= segment_len <= n/2 + 1");
  if (z_max > kNoAllocMaxW) return fail(PULSCAN_ERR_UNSUPPORTED, "z_max above 4096 for the allocation-free path");
  const int64_t n_seg = std::max<int64_t>(1, m / segment_len);
  const int64_t n_slots = n_seg * z_max;
  if (n_slots > kNoAllocSlots)
    return fail(PULSCAN_ERR_UNSUPPORTED, "segments x z_max above 2^20 for the allocation-free path");
  unsigned long long *base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // tile width as a plan would choose it: the widest giving >= 4 CTAs per SM
  int dev = 0, n_sm = 152;
  PS_CUDA(cudaGetDevice(&dev));
  PS_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  int warps = 1;
  for (int wp = 4; wp >= 1; wp >>= 1) {
    if ((m + search_tile_bins(wp) - 1) / search_tile_bins(wp) >= 4LL * n_sm) {
      warps = wp;
      break;
    }
  }
  const int64_t tiles = (m + search_tile_bins(warps) - 1) / search_tile_bins(warps);
  unsigned long long *slots = base;
  SeriesDev *series = reinterpret_cast<SeriesDev *>(base + kNoAllocSlots);
  int64_t *tile_off = reinterpret_cast<int64_t *>(base + kNoAllocSlots + 8);
  uint32_t *counters = reinterpret_cast<uint32_t *>(base + kNoAllocSlots + 10);
  const SeriesDev sd{m, n_seg, 0, 0, 0, 0, 0u, 0u};
  noalloc_header_kernel<<<1, 32, 0, s>>>(series, tile_off, counters, sd, tiles);
  PS_CUDA(cudaGetLastError());
  PS_CUDA(cudaMemsetAsync(slots, 0, static_cast<size_t>(n_slots) * sizeof(unsigned long long), s));
  return launch_segmax_raw(d_power, series, tile_off, tiles, warps, z_max, segment_len, slots, counters, n_slots,
                           d_max, d_argmax, s);
}
