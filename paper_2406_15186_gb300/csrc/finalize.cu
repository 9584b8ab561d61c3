// Candidate finaliser: per-(segment, width) slots -> candidate records with
// FP64 significance (paper §2.2.3, Eq. 9, and the candidate write-out at the
// end of Algorithm 4).
//
// The search kernel leaves, for every (segment, width) whose maximum reached
// T_w, a 64-bit key (power bits << 32 | ~bin) in its slot and the slot's index
// in a "touched" list.  This kernel visits the touched slots (or, if the list
// overflowed, every slot), converts each to a record, computes
// ln p = ln Q(w, S) + ln n_trials (Bonferroni, capped at 0) and the
// Gaussian-equivalent sigma in FP64, appends the record, and clears the slot
// so the slot array is zero again for the next search.
#include "common.cuh"
#include "signif.cuh"

namespace ps {

namespace {

__global__ void finalize_kernel(unsigned long long *__restrict__ slots, const uint32_t *__restrict__ touched,
                                uint32_t touched_cap, uint32_t *__restrict__ counters, int64_t total_slots,
                                int W, const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off,
                                int n_series, const double *__restrict__ ln_trials,
                                pulscan_cand *__restrict__ cands, uint32_t max_cands) {
  const uint32_t nt = counters[0];
  const bool full = nt > touched_cap;
  const int64_t n = full ? total_slots : static_cast<int64_t>(nt);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint64_t idx = full ? static_cast<uint64_t>(i) : static_cast<uint64_t>(touched[i]);
    const unsigned long long key = slots[idx];
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
    const double lp = fmin(0.0, log_q_gamma(static_cast<double>(w), static_cast<double>(pw)) + ln_trials[lo]);
    const double sg = sigma_from_log_p(lp);
    const uint32_t o = atomicAdd(counters + 1, 1u);
    if (o < max_cands) {
      pulscan_cand c;
      c.series = series[lo].user_index;
      c.width = static_cast<uint32_t>(w);
      c.bin = bin;
      c.power = pw;
      c.sigma = static_cast<float>(sg);
      cands[o] = c;
    }
  }
}

}  // namespace

int launch_finalize(pulscan_plan p, cudaStream_t s) {
  const int64_t total = p->total_seg * static_cast<int64_t>(p->z_max);
  finalize_kernel<<<304, 256, 0, s>>>(p->d_slots, p->d_touched, static_cast<uint32_t>(p->touched_cap),
                                       p->d_counters, total, p->z_max, p->d_series, p->d_seg_off,
                                       static_cast<int>(p->series.size()), p->d_ln_trials, p->d_cands,
                                       static_cast<uint32_t>(p->max_cands));
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
