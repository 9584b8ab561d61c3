// Candidate finaliser: per-(segment, width) slots -> candidate records with
// FP64 significance (paper §2.2.3, Eq. 9, and the candidate write-out at the
// end of Algorithm 4).
//
// The search kernel leaves, for every (segment, width) whose maximum reached
// T_w, a 64-bit key (power bits << 32 | ~bin) in its slot and sets the slot's
// bit in a dirty bitmap.  Every set bit is one record, so an exclusive scan
// of the words' bit counts (word_scan_kernel: per 2048-word block, then the
// last block over the block totals) gives each record its place in slot
// order -- (series, segment, width) in the plan's layout -- and the total.
// The finaliser then scans the bitmap (one word per warp, one slot per
// lane, grid-stride), visits the slots whose bits are set, converts each to a
// record, computes
// ln p = ln Q(a, S) + ln n_trials (Bonferroni, capped at 0; a = w, or
// H(H+1)/2 w for the H-harmonic sum of §2.3) and the
// Gaussian-equivalent sigma (FP32, cancellation-free form, see signif.cuh),
// appends the record, and clears the slot
// and the bitmap word so both are zero again for the next search.
#include <algorithm>

#include "common.cuh"
#include "signif.cuh"

namespace ps {

namespace {

constexpr int kScanThreads = 256;
constexpr int kWordsPerThread = 8;
constexpr int kWordsPerBlock = kScanThreads * kWordsPerThread;

// word_off[j] = set bits in the words before j within its 2048-word block;
// block_off[b] = set bits of the blocks before b.  Each CTA scans its block
// and publishes its total; the CTA that finishes last (a counter, no
// waiting) scans the totals in place and writes the record count to
// counters[1], then resets the counter for the next search.
__global__ void __launch_bounds__(kScanThreads) word_scan_kernel(const uint32_t *__restrict__ dirty, int64_t n_words,
                                                                  uint32_t *__restrict__ word_off,
                                                                  uint32_t *__restrict__ block_off,
                                                                  uint32_t *__restrict__ counters) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  __shared__ uint32_t last;
  const int64_t j0 = blockIdx.x * static_cast<int64_t>(kWordsPerBlock) + threadIdx.x * kWordsPerThread;
  uint32_t c[kWordsPerThread];
  uint32_t mine = 0;
#pragma unroll
  for (int k = 0; k < kWordsPerThread; ++k) {
    c[k] = (j0 + k < n_words) ? static_cast<uint32_t>(__popc(dirty[j0 + k])) : 0u;
    mine += c[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t base = incl - mine;
  for (int v = 0; v < warp; ++v) base += wsum[v];
#pragma unroll
  for (int k = 0; k < kWordsPerThread; ++k) {
    if (j0 + k < n_words) word_off[j0 + k] = base;
    base += c[k];
  }
  if (threadIdx.x == kScanThreads - 1) {
    block_off[blockIdx.x] = base;
    __threadfence();
    last = (atomicAdd(counters + 3, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  // the last CTA: exclusive scan of the block totals
  __threadfence();
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  const int64_t n_blocks = gridDim.x;
  for (int64_t b0 = 0; b0 < n_blocks; b0 += blockDim.x) {
    const int64_t bb = b0 + threadIdx.x;
    const uint32_t v = (bb < n_blocks) ? __ldcg(block_off + bb) : 0u;
    uint32_t in2 = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, in2, o);
      if (lane >= o) in2 += u;
    }
    if (lane == 31) wsum[warp] = in2;
    __syncthreads();
    uint32_t bs = carry + in2 - v;
    for (int w = 0; w < warp; ++w) bs += wsum[w];
    if (bb < n_blocks) block_off[bb] = bs;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = bs + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counters[1] = carry;
    counters[3] = 0u;
  }
}

__global__ void finalize_kernel(unsigned long long *__restrict__ slots, uint32_t *__restrict__ dirty,
                                int64_t n_words, const uint32_t *__restrict__ word_off,
                                const uint32_t *__restrict__ block_off, int W,
                                const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off,
                                int n_series, const double *__restrict__ ln_trials,
                                const float *__restrict__ gtab,
                                pulscan_cand *__restrict__ cands, uint32_t max_cands) {
  // one warp per bitmap word, one lane per bit: the FP64 significance of
  // neighbouring (segment, width) slots is evaluated in parallel
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); j < n_words;
       j += warps) {
    const uint32_t bits = dirty[j];
    if (bits == 0u) continue;
    if (lane == 0) dirty[j] = 0u;
    const bool mine = (bits >> lane) & 1u;
    const uint64_t idx = static_cast<uint64_t>(j) * 32u + static_cast<uint64_t>(lane);
    const unsigned long long key = mine ? slots[idx] : 0ull;
    // the word's place in slot order, from the scans
    const unsigned act = bits;
    const uint32_t base = block_off[j / kWordsPerBlock] + word_off[j];
    if (key == 0ull) continue;
    slots[idx] = 0ull;
    const int64_t gseg = static_cast<int64_t>(idx / static_cast<uint64_t>(W));
    const int w = static_cast<int>(idx % static_cast<uint64_t>(W)) + 1;
    int lo = 0, hi = n_series - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg_off[mid] <= gseg) lo = mid; else hi = mid - 1;
    }
    const float pw = __uint_as_float(static_cast<uint32_t>(key >> 32));
    const uint32_t bin = 0xffffffffu - static_cast<uint32_t>(key & 0xffffffffull);
    // gamma shape of a width-w sum: w, or H(H+1)/2 w for harmonic stage H
    const uint32_t hh = series[lo].harm;
    const float a = static_cast<float>(hh * (hh + 1) / 2) * static_cast<float>(w);
    const float lp = fminf(0.0f, log_q_f32(a, pw, gtab[(hh - 1) * static_cast<uint32_t>(W) + (w - 1)]) +
                                     static_cast<float>(ln_trials[lo]));
    const float sg = sigma_from_log_p_f32(lp);
    const uint32_t o = base + static_cast<uint32_t>(__popc(act & ((1u << lane) - 1u)));
    if (o < max_cands) {
      pulscan_cand c;
      c.series = series[lo].user_index;
      c.width = static_cast<uint32_t>(w);
      c.bin = bin;
      c.power = pw;
      c.sigma = sg;
      c.harmonics = hh;
      c.reserved = 0u;
      cands[o] = c;
    }
  }
}

}  // namespace

int launch_finalize(pulscan_plan p, cudaStream_t s) {
  const int64_t words = (p->total_seg * static_cast<int64_t>(p->z_max) + 31) / 32;
  const int64_t blocks = (words + kWordsPerBlock - 1) / kWordsPerBlock;
  word_scan_kernel<<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(p->d_dirty, words, p->d_word_off,
                                                                           p->d_block_off, p->d_counters);
  PS_CUDA(cudaGetLastError());
  const int grid = static_cast<int>(std::min<int64_t>(std::max<int64_t>((words + 7) / 8, 1), 2432));
  finalize_kernel<<<grid, 256, 0, s>>>(p->d_slots, p->d_dirty, words, p->d_word_off, p->d_block_off, p->z_max, p->d_series,
                                       p->d_seg_off, static_cast<int>(p->series.size()), p->d_ln_trials,
                                       p->d_gtab, p->d_cands, static_cast<uint32_t>(p->max_cands));
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
