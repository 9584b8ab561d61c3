// Internal definitions shared by the library's translation units: the plan,
// error reporting, and thin inline-PTX wrappers for mbarrier and TMA bulk
// copies (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/pulscan.h"

namespace ps {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define PS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) return ps::cuda_fail(e__, #call); \
  } while (0)

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes on
// the current device.  The limit is never lowered, so plans of different
// sizes (and the allocation-free entry point) can share a kernel.
struct SmemLimit {
  int set[64] = {};
  std::mutex m;
};

template <class K>
inline int ensure_smem(K kernel, int smem, SmemLimit &lim) {
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PULSCAN_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(lim.m);
  if (lim.set[dev] >= smem) return PULSCAN_OK;
  PS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  lim.set[dev] = smem;
  return PULSCAN_OK;
}

// device error flags (bit set by kernels, read by pulscan_candidates)
enum : uint32_t { kErrTimeout = 1u };

// ---------------------------------------------------------------- tiling
// Boxcar search: each lane owns kR consecutive start bins; a warp owns
// 32 * kR bins; a CTA of 1..4 warps owns one tile of 32 * kR * warps bins.
constexpr int kR = 33;                   // bins per lane (odd: conflict-free smem)
constexpr int kMaxThreads = 128;         // at most 4 warps (tiles of 1056..4224 bins)
constexpr int kMinBlocks = 4;            // resident CTAs per SM the register budget targets
constexpr int kSub = 11;                 // early sub-block edge (kR = 3 * kSub)
constexpr int kEarlyBlocks = 4;          // widths <= 132 use the finer bound

// Normalisation kernel
constexpr int kNormThreads = 256;
constexpr int kHistBins = 2048;

// ---------------------------------------------------------------- plan
struct Series {
  int64_t n;          // samples
  int64_t m;          // bins = n/2 + 1
  int64_t n_seg;      // segments
  int64_t x_off;      // floats
  int64_t spec_off;   // complex bins
  int64_t p_off;      // floats (16-byte aligned)
  int64_t seg_off;    // first global segment
  int64_t tile_off;   // first global search tile
  uint32_t user_index;
  uint32_t harm = 1;  // harmonics summed (1: the series' own power; H >= 2: a stage spectrum, n = 0)
};

// device-side view of one series (what the kernels need)
struct SeriesDev {
  int64_t m;
  int64_t n_seg;
  int64_t p_off;
  int64_t spec_off;
  int64_t seg_off;
  int64_t tile_off;
  uint32_t user_index;
  uint32_t harm;      // harmonics summed: a width-w sum has gamma shape H(H+1)/2 * w
};

struct FftClass {
  int64_t n;
  int count;
  int64_t x_off;      // first series of the class
  int64_t spec_off;
  int64_t spec_stride;  // complex bins between series of the class
  cufftHandle handle;
};

struct GraphCache {
  const void *x = nullptr, *spec = nullptr, *power = nullptr;
  cudaStream_t capture = nullptr;   // plan-owned stream the graph is captured on
  cudaStream_t side = nullptr;      // high-priority stream of a pipelined capture (FFT + normalisation)
  std::vector<cudaEvent_t> ev;      // fork / join events of a pipelined capture
  cudaGraphExec_t exec = nullptr;
};

// A part of a pipelined batch: layout series [s_lo, s_hi), all of one length,
// transformed by chunk_fft[fft].
struct Chunk {
  int64_t s_lo, s_hi;
  int fft;
};

#ifdef __CUDACC__
// The normalised power of Eq. 8 from a bin's deviations d = x - med of both
// components and the block's 1 / (kappa MAD) pair: a = d_re inv_re,
// b = d_im inv_im, P = (a^2 + b^2) / 2, every rounding fixed (no
// contraction), so the normalisation and the fused bank form the same bits.
__device__ __forceinline__ float power_of_dev(float d_re, float d_im, float inv_re, float inv_im) {
  const float a = __fmul_rn(d_re, inv_re), b = __fmul_rn(d_im, inv_im);
  return __fmul_rn(0.5f, __fmaf_rn(a, a, __fmul_rn(b, b)));
}

// The same from the bin itself and the block's (med_re, inv_re, med_im, inv_im).
__device__ __forceinline__ float power_of(float re, float im, float4 nrm) {
  return power_of_dev(__fsub_rn(re, nrm.x), __fsub_rn(im, nrm.z), nrm.y, nrm.w);
}
#endif

}  // namespace ps

struct pulscan_plan_s {
  int32_t z_max = 0;
  int32_t seg_len = 0;
  double sigma_thr = 0.0;
  std::vector<ps::Series> series;   // the series (layout order), then their harmonic stages
  int32_t numharm = 1;              // harmonics summed up to (1: none)
  int64_t n_base = 0;               // entries of `series` that are series (the rest are stages)
  int64_t base_seg = 0;             // segments of those (normalised); stage segments follow
  std::vector<ps::FftClass> fft;
  std::vector<double> n_trials;     // per series (layout order)
  std::vector<uint8_t> searched;    // per width: compared and reported (1) or only summed (0)
  bool trials_fixed = false;        // n_trials set by the caller (kept when the widths change)
  int64_t rblock = 0;               // > 0: candidates report floor(bin / rblock)
  int32_t fidelity = 0;             // PULSCAN_FIDELITY_*: exact, or the paper's GPU approximations
  uint8_t *d_searched = nullptr;    // device copy of `searched`
  std::vector<int> layout_of_user;  // user series index -> layout index
  std::vector<float> h_thresh;      // n_series * z_max, layout order
  int64_t x_floats = 0, spec_bins = 0, p_floats = 0, total_seg = 0, total_tiles = 0;
  int64_t max_cands = 0;
  int search_warps = 4;            // warps per boxcar CTA
  int search_groups = 1;           // 1056-bin slices per warp: 1 scalar adds, 2 packed (tile = 1056 * warps * groups)
  uint32_t wait_test_us = 0;       // > 0: the next search tests its timeout path (no copy issued; limit in us)
  // device scratch
  ps::SeriesDev *d_series = nullptr;
  int64_t *d_tile_off = nullptr;   // n_series + 1, for tile -> series search
  int64_t *d_seg_off = nullptr;    // n_series + 1, for segment -> series search
  float *d_thresh = nullptr;       // n_series * z_max
  float *d_thresh_bound = nullptr; // same, scaled down slightly for bound checks
  double *d_ln_trials = nullptr;   // ln(n_trials) per series
  float *d_gtab = nullptr;         // g(a) = a ln a - a - ln Gamma(a), a = H(H+1)/2 w: [H - 1][w - 1]
  float *d_stats = nullptr;        // 4 * total_seg
  unsigned long long *d_slots = nullptr;  // total_seg * z_max keys, 0 at rest
  uint32_t *d_dirty = nullptr;     // one bit per slot touched by the search, 0 at rest
  uint32_t *d_word_off = nullptr;  // per bitmap word: set bits before it in its 2048-word block
  uint32_t *d_block_off = nullptr; // per 2048-word block: set bits before it
  uint32_t *d_counters = nullptr;  // [0] deferred items, [1] candidates, [2] error flags, [3] finaliser scan,
                                   // [4, 4 + n_ranges) tile claim counters of the persistent bank
  int n_ranges = 1;                // tile ranges of the persistent bank (one per SM)
  int64_t *d_ranges = nullptr;     // their first tiles, n_ranges + 1 entries
  int persist_grid[2] = {0, 0};    // persistent bank grid: [0] search, [1] maxima (0: one CTA per tile)
  int persist_mode = -1;           // -1: persistent for grids of >= 3 waves; 0: never; 1: always
  unsigned long long *d_items = nullptr;  // deferred boxcar blocks
  float *d_snaps = nullptr;        // their running-sum snapshots (33 x 32 floats each)
  int64_t item_cap = 0;           // deferred items in use (<= alloc_item_cap)
  int64_t alloc_item_cap = 0;
  int defer_grid = 1;          // CTAs of the three-warp-per-item deferred kernel (and of the short-segment one)
  int defer_grid_warp = 1;     // CTAs of the one-warp-per-item deferred kernel
  int defer_form = 0;          // deferred blocks: 0 = three warps per item, 1 = one warp per item
  pulscan_cand *d_cands = nullptr;
  // device buffers owned by the plan for pulscan_search_host
  float *own_x = nullptr, *own_spec = nullptr, *own_power = nullptr;
  // logsumexp path (allocated on first use)
  int64_t *d_x_off = nullptr, *d_x_len = nullptr;   // per layout series
  float *d_dp = nullptr;           // dL/dP (power layout)
  float *d_tail = nullptr;         // per segment, W-1 bins spilling into the next segment
  float *d_gspec = nullptr;        // C2R input (spectrum layout)
  double *d_amp_part = nullptr;    // dL/dA partial sums, 16 per series
  std::vector<ps::FftClass> ifft;  // C2R plans per length class
  // timing
  int timing = 0;                  // 0 off, 1 every stage's events, 2 the bank kernel's pair only
  cudaEvent_t ev[14] = {};
  bool ran[7] = {};
  ps::GraphCache graph;
  // pipelined batch (pulscan_plan_set_pipeline): parts of about pipe_bins bins
  int64_t pipe_bins = 0;           // 0: off
  std::vector<ps::Chunk> chunks;
  std::vector<ps::FftClass> chunk_fft;   // R2C plans per (length, series count) of the parts
  void *d_fft_work = nullptr;      // their shared work area (the parts' transforms run one at a time)
  // fused search (pulscan_plan_set_fused): per segment (med_re, 1 / (kappa
  // MAD_re), med_im, 1 / (kappa MAD_im)); P is formed in the bank
  bool fused = false;
  float *d_norm = nullptr;
};

namespace ps {
// launchers (defined in the kernel translation units)
int launch_normalise(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats,
                     cudaStream_t s);
// same, also recording per segment the selected order statistics
// [med_lo, med_hi, dev_lo, dev_hi] of Re then Im (8 floats) into d_sel
int launch_normalise_sel(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats, float *d_sel,
                         cudaStream_t s);
// d_spec != nullptr: the fused search, P formed on the fly from the spectrum
// and p->d_norm (launch_normalise_stats); d_power is then not used
int launch_search(pulscan_plan p, const float *d_power, cudaStream_t s, const float *d_spec = nullptr);
int launch_normalise_stats(pulscan_plan p, const float *d_spec, cudaStream_t s);
int launch_finalize(pulscan_plan p, cudaStream_t s);
int launch_harmonic_sums(pulscan_plan p, float *d_power, cudaStream_t s);   // stage spectra X_H
// paper-GPU fidelity mode
bool is_power_of_four(int64_t v);
int launch_normalise_mom(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats, cudaStream_t s);
int launch_maxima_only(pulscan_plan p, const float *d_power, cudaStream_t s);   // all maxima into the slots
int launch_poly_finalize(pulscan_plan p, cudaStream_t s);
double host_log_sf_normal(double s);   // ln Phi_c(s), FP64 on the host
int launch_segmax(pulscan_plan p, const float *d_power, float *d_max, uint64_t *d_argmax,
                  cudaStream_t s);
void record(pulscan_plan p, int idx, cudaStream_t s);  // timing event helper
int search_smem_bytes(int W, int warps, int groups, int *buf_len_out);
int search_tile_bins(int warps, int groups = 1);
int prepare_bank(pulscan_plan p);       // one-time kernel attributes (before any capture)
int prepare_bank_raw(int W, int warps);
int launch_segmax_raw(const float *d_power, const SeriesDev *d_series, const int64_t *d_tile_off, int64_t tiles,
                      int warps, int W, int seg_len, unsigned long long *d_slots, uint32_t *d_counters,
                      int64_t n_slots, float *d_max, uint64_t *d_argmax, cudaStream_t s);
int prepare_normalise(pulscan_plan p);
// pipelined batch parts: normalisation of segments [seg_lo, seg_lo + n_seg)
// (register kernel only), the search bank over tiles [tile_lo, tile_lo +
// n_tiles), and the deferred blocks after the last part
bool normalise_range_ok(pulscan_plan p);
int launch_normalise_range(pulscan_plan p, const float *d_spec, float *d_power, int64_t seg_lo, int64_t n_seg,
                           cudaStream_t s);
int launch_search_tiles(pulscan_plan p, const float *d_power, int64_t tile_lo, int64_t n_tiles, cudaStream_t s);
int launch_deferred(pulscan_plan p, const float *d_power, cudaStream_t s, const float *d_spec = nullptr);
}  // namespace ps
