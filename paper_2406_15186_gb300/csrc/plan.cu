// Host runtime of the C ABI: plan creation (layout, threshold tables, cuFFT
// plans, device scratch), argument checking, the whole-path CUDA graph, timing
// events and candidate read-back.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#include "common.cuh"
#include "signif.cuh"

namespace ps {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PULSCAN_ERR_NOMEM : PULSCAN_ERR_CUDA;
}

static int cuda_ok_or(cudaError_t e) { return e == cudaSuccess ? PULSCAN_OK : cuda_fail(e, "plan setup"); }

static int cufft_fail(cufftResult r, const char *what) {
  set_error(std::string(what) + ": cuFFT error " + std::to_string(static_cast<int>(r)));
  return r == CUFFT_ALLOC_FAILED ? PULSCAN_ERR_NOMEM : PULSCAN_ERR_CUDA;
}

void record(pulscan_plan p, int idx, cudaStream_t s) {
  // mode 2 keeps only the bank kernel's pair (4, 5): every event between
  // kernels costs a few microseconds of pipeline drain
  if (p->timing == 1 || (p->timing == 2 && (idx == 4 || idx == 5))) {
    // inside a stream capture the record becomes a node of the graph (an
    // external event record), re-recorded by every launch
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(p->ev[idx], s, cudaEventRecordExternal);
    else
      cudaEventRecord(p->ev[idx], s);
    p->ran[idx / 2] = true;
  }
}

// ln Phi_c(s) on the host: erfc while it is representable, else the
// asymptotic (Mills-ratio) series phi(s)/s (1 - 1/s^2 + 3/s^4 - 15/s^6 + 105/s^8).
double host_log_sf_normal(double s) {
  if (s < 30.0) return std::log(0.5 * std::erfc(s / std::sqrt(2.0)));
  const double s2 = s * s;
  const double series = 1.0 - 1.0 / s2 + 3.0 / (s2 * s2) - 15.0 / (s2 * s2 * s2) + 105.0 / (s2 * s2 * s2 * s2);
  return -0.5 * s2 - std::log(s) - 0.5 * std::log(2.0 * M_PI) + std::log(series);
}

// Smallest float T with ln Q(a, T) <= y (bisection on the FP64 ln Q); a is
// the gamma shape of a width-w sum: w, or H(H+1)/2 w for harmonic stage H.
static float threshold_for(double w, double y) {
  if (y >= 0.0) return 0.0f;
  double lo = 0.0, hi = w + 1.0;
  while (log_q_gamma(w, hi) > y) hi *= 2.0;
  for (int it = 0; it < 300 && hi - lo > 1e-13 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (log_q_gamma(w, mid) > y) lo = mid; else hi = mid;
  }
  float f = static_cast<float>(hi);
  if (static_cast<double>(f) < hi) f = std::nextafter(f, INFINITY);
  return f;
}

static void compute_thresholds(pulscan_plan p) {
  const int W = p->z_max;
  const size_t ns = p->series.size();
  p->h_thresh.assign(ns * W, 0.0f);
  std::map<std::pair<double, uint32_t>, std::vector<float>> cache;
  const double lsf = host_log_sf_normal(p->sigma_thr);
  for (size_t i = 0; i < ns; ++i) {
    const double nt = p->n_trials[i];
    const uint32_t h = p->series[i].harm;
    auto it = cache.find({nt, h});
    if (it == cache.end()) {
      std::vector<float> t(W);
      const double y = lsf - std::log(nt);
      const double c = 0.5 * h * (h + 1);   // gamma shape per unit width
      for (int w = 1; w <= W; ++w) t[w - 1] = p->searched[w - 1] ? threshold_for(c * w, y) : INFINITY;
      it = cache.emplace(std::make_pair(nt, h), std::move(t)).first;
    }
    std::copy(it->second.begin(), it->second.end(), p->h_thresh.begin() + i * W);
  }
}

// Threshold tables to the device: exact T_w, and for the block bounds the
// running minimum over widths >= w scaled by (1 - 2^-10), a margin that covers
// FP32 rounding of the bound and of the running sums.
static int upload_thresholds(pulscan_plan p) {
  const int W = p->z_max;
  const size_t ns = p->series.size();
  std::vector<float> tb(ns * W);
  std::vector<double> lt(ns);
  for (size_t i = 0; i < ns; ++i) {
    float run = INFINITY;
    for (int w = W; w >= 1; --w) {
      run = std::min(run, p->h_thresh[i * W + w - 1]);
      tb[i * W + w - 1] = run * (1.0f - 1.0f / 1024.0f);
    }
    lt[i] = std::log(p->n_trials[i]);
  }
  PS_CUDA(cudaMemcpy(p->d_thresh, p->h_thresh.data(), ns * W * sizeof(float), cudaMemcpyHostToDevice));
  PS_CUDA(cudaMemcpy(p->d_thresh_bound, tb.data(), ns * W * sizeof(float), cudaMemcpyHostToDevice));
  PS_CUDA(cudaMemcpy(p->d_ln_trials, lt.data(), ns * sizeof(double), cudaMemcpyHostToDevice));
  PS_CUDA(cudaMemcpy(p->d_searched, p->searched.data(), W * sizeof(uint8_t), cudaMemcpyHostToDevice));
  return PULSCAN_OK;
}

static void free_chunks(pulscan_plan p) {
  for (auto &f : p->chunk_fft)
    if (f.handle) cufftDestroy(f.handle);
  p->chunk_fft.clear();
  p->chunks.clear();
  if (p->d_fft_work) cudaFree(p->d_fft_work);
  p->d_fft_work = nullptr;
  p->pipe_bins = 0;
}

static void free_plan(pulscan_plan p) {
  if (!p) return;
  for (auto &f : p->fft)
    if (f.handle) cufftDestroy(f.handle);
  for (auto &f : p->ifft)
    if (f.handle) cufftDestroy(f.handle);
  void *ptrs[] = {p->d_series, p->d_tile_off, p->d_seg_off, p->d_thresh, p->d_thresh_bound, p->d_ln_trials,
                  p->d_stats,  p->d_slots,    p->d_dirty,   p->d_counters, p->d_cands,     p->own_x,
                  p->own_spec, p->own_power, p->d_items, p->d_snaps,    p->d_gtab,     p->d_x_off,
                  p->d_x_len,  p->d_dp,      p->d_tail,     p->d_gspec,   p->d_ranges,  p->d_searched, p->d_word_off, p->d_block_off,
                  p->d_norm,   p->d_amp_part};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  for (auto &e : p->ev)
    if (e) cudaEventDestroy(e);
  free_chunks(p);
  for (auto &e : p->graph.ev)
    if (e) cudaEventDestroy(e);
  if (p->graph.exec) cudaGraphExecDestroy(p->graph.exec);
  if (p->graph.capture) cudaStreamDestroy(p->graph.capture);
  if (p->graph.side) cudaStreamDestroy(p->graph.side);
  delete p;
}

template <class T>
static int dalloc(T **out, size_t count) {
  *out = nullptr;
  if (count == 0) count = 1;
  PS_CUDA(cudaMalloc(reinterpret_cast<void **>(out), count * sizeof(T)));
  return PULSCAN_OK;
}

static int check_shape(int64_t n, int32_t z_max, int32_t seg_len, double sigma) {
  if (n < 2 || (n & 1)) return fail(PULSCAN_ERR_INVALID_ARG, "series length must be even and >= 2");
  // bins are 32-bit in the (power, bin) merge keys: M = n/2 + 1 <= 2^32
  if (n >= (int64_t(1) << 33)) return fail(PULSCAN_ERR_UNSUPPORTED, "series of 2^33 samples or more");
  const int64_t m = n / 2 + 1;
  if (z_max < 1) return fail(PULSCAN_ERR_INVALID_ARG, "z_max must be >= 1");
  if (seg_len < z_max) return fail(PULSCAN_ERR_INVALID_ARG, "segment_len must be >= z_max");
  if (seg_len > m) return fail(PULSCAN_ERR_INVALID_ARG, "segment_len must be <= n/2 + 1");
  if (!std::isfinite(sigma) || sigma < 0.0)
    return fail(PULSCAN_ERR_INVALID_ARG, "threshold_sigma must be finite and >= 0");
  return PULSCAN_OK;
}

// Device copies of the series table, the tile offsets and the per-SM tile
// ranges (after the layout or the tile width changed).
static int upload_layout(pulscan_plan p) {
  const size_t ns = p->series.size();
  std::vector<SeriesDev> sd(ns);
  std::vector<int64_t> to(ns + 1), so(ns + 1);
  for (size_t i = 0; i < ns; ++i) {
    const Series &s = p->series[i];
    sd[i] = SeriesDev{s.m, s.n_seg, s.p_off, s.spec_off, s.seg_off, s.tile_off, s.user_index, s.harm};
    to[i] = s.tile_off;
    so[i] = s.seg_off;
  }
  to[ns] = p->total_tiles;
  so[ns] = p->total_seg;
  PS_CUDA(cudaMemcpy(p->d_series, sd.data(), ns * sizeof(SeriesDev), cudaMemcpyHostToDevice));
  PS_CUDA(cudaMemcpy(p->d_tile_off, to.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  PS_CUDA(cudaMemcpy(p->d_seg_off, so.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  std::vector<int64_t> rl(static_cast<size_t>(p->n_ranges) + 1);
  for (int r = 0; r <= p->n_ranges; ++r) rl[r] = p->total_tiles * r / p->n_ranges;   // equal ranges, one per SM
  PS_CUDA(cudaMemcpy(p->d_ranges, rl.data(), rl.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  return PULSCAN_OK;
}

// Re-tile the bank with `warps` warps per CTA and `groups` 1056-bin slices
// per warp (tile = 1056 x warps x groups bins; groups = 2: packed adds).
static int relayout_tiles(pulscan_plan p, int warps, int groups) {
  p->search_warps = warps;
  p->search_groups = groups;
  const int64_t tb = search_tile_bins(warps, groups);
  int64_t tl = 0;
  for (auto &se : p->series) {
    se.tile_off = tl;
    tl += (se.m + tb - 1) / tb;
  }
  p->total_tiles = tl;
  const int64_t nb = (p->z_max + kR - 1) / kR;
  p->item_cap = std::min<int64_t>(std::min<int64_t>(tl * warps * groups * nb, 65536), p->alloc_item_cap);
  int rc = upload_layout(p);
  if (!rc) rc = prepare_bank(p);
  if (p->graph.exec) {
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  return rc;
}

// Parts of a pipelined batch: consecutive series (layout order) of one length,
// about `bins` bins each, with one R2C plan per (length, series count); the
// plans share one work area, since the parts' transforms run one after
// another on one stream.  Fewer than two parts: no pipeline.
static int build_chunks(pulscan_plan p, int64_t bins) {
  free_chunks(p);
  if (p->graph.exec) {
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  if (bins <= 0 || p->numharm != 1) return PULSCAN_OK;
  std::vector<Chunk> ch;
  for (int64_t i = 0; i < p->n_base;) {
    const int64_t n = p->series[i].n;
    int64_t j = i, acc = 0;
    while (j < p->n_base && p->series[j].n == n && (j == i || acc + p->series[j].m <= bins)) acc += p->series[j++].m;
    ch.push_back(Chunk{i, j, -1});
    i = j;
  }
  if (ch.size() < 2) return PULSCAN_OK;
  size_t work_max = 0;
  int rc = PULSCAN_OK;
  for (auto &c : ch) {
    const Series &s0 = p->series[c.s_lo];
    const int count = static_cast<int>(c.s_hi - c.s_lo);
    for (size_t k = 0; k < p->chunk_fft.size(); ++k)
      if (p->chunk_fft[k].n == s0.n && p->chunk_fft[k].count == count) c.fft = static_cast<int>(k);
    if (c.fft >= 0) continue;
    FftClass f{};
    f.n = s0.n;
    f.count = count;
    f.spec_stride = (s0.m + 31) / 32 * 32;
    long long nn = f.n, inembed = f.n, onembed = f.spec_stride;
    size_t work = 0;
    cufftResult r = cufftCreate(&f.handle);
    if (r == CUFFT_SUCCESS) r = cufftSetAutoAllocation(f.handle, 0);
    if (r == CUFFT_SUCCESS)
      r = cufftMakePlanMany64(f.handle, 1, &nn, &inembed, 1, f.n, &onembed, 1, f.spec_stride, CUFFT_R2C, count,
                              &work);
    if (r != CUFFT_SUCCESS) {
      rc = cufft_fail(r, "cufftMakePlanMany64");
      if (f.handle) cufftDestroy(f.handle);
      break;
    }
    work_max = std::max(work_max, work);
    c.fft = static_cast<int>(p->chunk_fft.size());
    p->chunk_fft.push_back(f);
  }
  if (!rc && work_max > 0 && cudaMalloc(&p->d_fft_work, work_max) != cudaSuccess) {
    cudaGetLastError();
    rc = fail(PULSCAN_ERR_NOMEM, "cuFFT work area");
  }
  for (size_t k = 0; !rc && k < p->chunk_fft.size(); ++k) {
    const cufftResult r = cufftSetWorkArea(p->chunk_fft[k].handle, p->d_fft_work);
    if (r != CUFFT_SUCCESS) rc = cufft_fail(r, "cufftSetWorkArea");
  }
  if (rc) {
    free_chunks(p);
    return rc;
  }
  p->chunks = ch;
  p->pipe_bins = bins;
  return PULSCAN_OK;
}

static int build_plan(pulscan_plan *out, const int64_t *lengths, int32_t n_series, int32_t z_max,
                      int32_t seg_len, double sigma, int32_t numharm = 1) {
  if (!out) return fail(PULSCAN_ERR_INVALID_ARG, "null plan pointer");
  *out = nullptr;
  if (n_series < 1 || !lengths) return fail(PULSCAN_ERR_INVALID_ARG, "need at least one series");
  if (numharm < 1 || numharm > 8) return fail(PULSCAN_ERR_INVALID_ARG, "numharm must be in 1..8");
  for (int32_t i = 0; i < n_series; ++i) {
    const int rc = check_shape(lengths[i], z_max, seg_len, sigma);
    if (rc) return rc;
    if (seg_len > (lengths[i] / 2 + 1) / numharm)
      return fail(PULSCAN_ERR_INVALID_ARG, "segment_len must be <= floor(M / numharm)");
  }
  pulscan_plan p = new (std::nothrow) pulscan_plan_s();
  if (!p) return fail(PULSCAN_ERR_NOMEM, "host allocation failed");
  p->z_max = z_max;
  p->seg_len = seg_len;
  p->sigma_thr = sigma;
  p->numharm = numharm;
  // layout: series grouped by length (stable in the caller's order) so every
  // length class is one strided batched FFT
  std::vector<int> order(n_series);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lengths[a] < lengths[b]; });
  p->layout_of_user.assign(n_series, 0);
  // warps per boxcar CTA: the widest tile that still gives >= 4 CTAs per SM
  int n_sm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  p->search_warps = 1;
  for (int wp = 4; wp >= 1; wp >>= 1) {
    int64_t tiles = 0;
    for (int32_t i = 0; i < n_series; ++i) tiles += (lengths[i] / 2 + 1 + search_tile_bins(wp) - 1) / search_tile_bins(wp);
    if (tiles >= 4LL * n_sm) {
      p->search_warps = wp;
      break;
    }
  }
  const int64_t tile_bins = search_tile_bins(p->search_warps);
  int64_t x = 0, sp = 0, pw = 0, sg = 0, tl = 0;
  for (int li = 0; li < n_series; ++li) {
    const int ui = order[li];
    Series s{};
    s.n = lengths[ui];
    s.m = s.n / 2 + 1;
    s.n_seg = std::max<int64_t>(1, s.m / seg_len);
    s.x_off = x;
    s.spec_off = sp;
    s.p_off = pw;
    s.seg_off = sg;
    s.tile_off = tl;
    s.user_index = static_cast<uint32_t>(ui);
    p->series.push_back(s);
    p->layout_of_user[ui] = li;
    x += s.n;
    const int64_t mpad = (s.m + 31) / 32 * 32;
    const bool last = li + 1 == n_series;
    sp += last ? s.m : mpad;
    pw += (last && numharm == 1) ? s.m : mpad;
    sg += s.n_seg;
    tl += (s.m + tile_bins - 1) / tile_bins;
  }
  p->n_base = n_series;
  p->base_seg = sg;
  // harmonic stages H = 2..numharm of every series (layout order): spectra of
  // floor(M / H) bins in the power buffer after the series' powers
  for (int h = 2; h <= numharm; ++h) {
    for (int li = 0; li < n_series; ++li) {
      const Series &b = p->series[li];
      Series s{};
      s.n = 0;
      s.m = b.m / h;
      s.n_seg = std::max<int64_t>(1, s.m / seg_len);
      s.x_off = b.x_off;
      s.spec_off = b.spec_off;
      s.p_off = pw;
      s.seg_off = sg;
      s.tile_off = tl;
      s.user_index = b.user_index;
      s.harm = static_cast<uint32_t>(h);
      p->series.push_back(s);
      const bool last = h == numharm && li + 1 == n_series;
      pw += last ? s.m : (s.m + 31) / 32 * 32;
      sg += s.n_seg;
      tl += (s.m + tile_bins - 1) / tile_bins;
    }
  }
  p->x_floats = x;
  p->spec_bins = sp;
  p->p_floats = pw;
  p->total_seg = sg;
  p->total_tiles = tl;
  const int64_t total_slots = sg * static_cast<int64_t>(z_max);
  if (total_slots >= (int64_t(1) << 32)) {
    free_plan(p);
    return fail(PULSCAN_ERR_UNSUPPORTED, "segments x z_max exceeds 2^32 slots");
  }
  p->max_cands = std::min<int64_t>(total_slots, int64_t(1) << 24);
  const int64_t dirty_words = (total_slots + 31) / 32;
  // deferred-block list: at most one item per (warp, block), capped at 2^16
  // items (277 MB of snapshots); an overflowing block is run exactly by its
  // own warp, which is far slower when whole regions are hot (the harmonic
  // stages of strong tones flag tens of thousands of blocks)
  const int64_t total_warps = tl * p->search_warps * p->search_groups;
  const int64_t nb = (z_max + kR - 1) / kR;
  p->item_cap = std::min<int64_t>(total_warps * nb, 65536);
  p->alloc_item_cap = p->item_cap;
  p->defer_grid = 8 * n_sm;        // 3-warp CTAs, one item each at a time: 24 warps per SM
  p->defer_grid_warp = 4 * n_sm;   // 4-warp CTAs, one item per warp: 16 warps per SM
  // one warp per item wins when the items fill the GPU several times over
  // (a 2^27-sample series: 0.19 against 0.31 ms), three warps per item when
  // few items leave the per-item step chain exposed (2^23: 33 against 23 us);
  // the autotuner times both on the caller's data
  p->defer_form = pw >= (int64_t(1) << 25) ? 1 : 0;
  p->searched.assign(z_max, 1);
  for (auto &s : p->series) p->n_trials.push_back(static_cast<double>(s.m) * z_max);
  compute_thresholds(p);

  int rc = PULSCAN_OK;
  auto ok = [&](int r) {
    if (r && !rc) rc = r;
    return rc == PULSCAN_OK;
  };
  const size_t ns = p->series.size();
  if (ok(dalloc(&p->d_series, ns)) && ok(dalloc(&p->d_tile_off, ns + 1)) && ok(dalloc(&p->d_seg_off, ns + 1)) &&
      ok(dalloc(&p->d_thresh, ns * z_max)) && ok(dalloc(&p->d_thresh_bound, ns * z_max)) &&
      ok(dalloc(&p->d_ln_trials, ns)) && ok(dalloc(&p->d_stats, 4 * sg)) &&
      ok(dalloc(&p->d_slots, total_slots)) && ok(dalloc(&p->d_dirty, dirty_words)) &&
      ok(dalloc(&p->d_word_off, dirty_words)) && ok(dalloc(&p->d_block_off, dirty_words / 2048 + 1)) &&
      ok(dalloc(&p->d_counters, 4 + static_cast<size_t>(n_sm))) && ok(dalloc(&p->d_cands, p->max_cands)) &&
      ok(dalloc(&p->d_items, p->item_cap)) && ok(dalloc(&p->d_snaps, p->item_cap * kR * 32)) &&
      ok(dalloc(&p->d_gtab, static_cast<size_t>(numharm) * z_max)) && ok(dalloc(&p->d_x_off, ns)) &&
      ok(dalloc(&p->d_x_len, ns)) &&
      ok(dalloc(&p->d_ranges, static_cast<size_t>(n_sm) + 1)) && ok(dalloc(&p->d_searched, z_max))) {
    p->n_ranges = n_sm;
    ok(upload_layout(p));
    std::vector<int64_t> xo(ns), xl(ns);
    for (size_t i = 0; i < ns; ++i) {
      xo[i] = p->series[i].x_off;
      xl[i] = p->series[i].n;
    }
    ok(cuda_ok_or(cudaMemcpy(p->d_x_off, xo.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice)));
    ok(cuda_ok_or(cudaMemcpy(p->d_x_len, xl.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice)));
    ok(cuda_ok_or(cudaMemset(p->d_slots, 0, total_slots * sizeof(unsigned long long))));
    ok(cuda_ok_or(cudaMemset(p->d_dirty, 0, dirty_words * sizeof(uint32_t))));
    ok(cuda_ok_or(cudaMemset(p->d_counters, 0, (4 + static_cast<size_t>(n_sm)) * sizeof(uint32_t))));
    ok(upload_thresholds(p));
    std::vector<float> gt(static_cast<size_t>(numharm) * z_max);
    for (int h = 1; h <= numharm; ++h)
      for (int w = 1; w <= z_max; ++w)
        gt[(h - 1) * static_cast<size_t>(z_max) + w - 1] = static_cast<float>(g_of(0.5 * h * (h + 1) * w));
    ok(cuda_ok_or(cudaMemcpy(p->d_gtab, gt.data(), gt.size() * sizeof(float), cudaMemcpyHostToDevice)));
    ok(prepare_bank(p));
    ok(prepare_normalise(p));
  }
  // cuFFT: one strided batched plan per length class (the series only)
  const size_t nb_fft = static_cast<size_t>(p->n_base);
  for (size_t i = 0; rc == PULSCAN_OK && i < nb_fft;) {
    size_t j = i;
    while (j < nb_fft && p->series[j].n == p->series[i].n) ++j;
    FftClass f{};
    f.n = p->series[i].n;
    f.count = static_cast<int>(j - i);
    f.x_off = p->series[i].x_off;
    f.spec_off = p->series[i].spec_off;
    f.spec_stride = (p->series[i].m + 31) / 32 * 32;
    long long nn = f.n, inembed = f.n, onembed = f.spec_stride;
    size_t work = 0;
    cufftResult r = cufftCreate(&f.handle);
    if (r == CUFFT_SUCCESS)
      r = cufftMakePlanMany64(f.handle, 1, &nn, &inembed, 1, f.n, &onembed, 1, f.spec_stride, CUFFT_R2C,
                              f.count, &work);
    if (r != CUFFT_SUCCESS) {
      rc = cufft_fail(r, "cufftMakePlanMany64");
      if (f.handle) cufftDestroy(f.handle);
      break;
    }
    p->fft.push_back(f);
    i = j;
  }
  if (rc != PULSCAN_OK) {
    free_plan(p);
    return rc;
  }
  *out = p;
  return PULSCAN_OK;
}

static bool aligned16(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0u; }

}  // namespace ps

using namespace ps;

extern "C" {

int pulscan_version(void) { return 10000; }

const char *pulscan_last_error(void) { return g_last_error.c_str(); }

int pulscan_plan_create(pulscan_plan *out, int64_t n, int32_t z_max, int32_t segment_len,
                        double threshold_sigma) {
  return build_plan(out, &n, 1, z_max, segment_len, threshold_sigma);
}

int pulscan_plan_create_batch(pulscan_plan *out, const int64_t *h_lengths, int32_t n_series, int32_t z_max,
                              int32_t segment_len, double threshold_sigma) {
  return build_plan(out, h_lengths, n_series, z_max, segment_len, threshold_sigma);
}

int pulscan_plan_create_harmonic(pulscan_plan *out, const int64_t *h_lengths, int32_t n_series, int32_t z_max,
                                 int32_t segment_len, double threshold_sigma, int32_t numharm) {
  return build_plan(out, h_lengths, n_series, z_max, segment_len, threshold_sigma, numharm);
}

void pulscan_plan_destroy(pulscan_plan plan) { free_plan(plan); }

int pulscan_plan_get_info(pulscan_plan p, pulscan_plan_info *info) {
  if (!p || !info) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  info->n_series = p->n_base;
  info->x_floats = p->x_floats;
  info->spec_floats = 2 * p->spec_bins;
  info->power_floats = p->p_floats;
  info->total_segments = p->total_seg;
  info->z_max = p->z_max;
  info->segment_len = p->seg_len;
  info->threshold_sigma = p->sigma_thr;
  info->max_candidates = p->max_cands;
  return PULSCAN_OK;
}

int pulscan_plan_offsets(pulscan_plan p, int64_t *x_off, int64_t *spec_off, int64_t *power_off,
                         int64_t *seg_off) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  const size_t ns = static_cast<size_t>(p->n_base);
  // offsets are reported in the caller's series order; entry ns is the end
  // of the series' own data (harmonic stages follow it)
  for (size_t u = 0; u < ns; ++u) {
    const Series &s = p->series[p->layout_of_user[u]];
    if (x_off) x_off[u] = s.x_off;
    if (spec_off) spec_off[u] = s.spec_off;
    if (power_off) power_off[u] = s.p_off;
    if (seg_off) seg_off[u] = s.seg_off;
  }
  if (x_off) x_off[ns] = p->x_floats;
  if (spec_off) spec_off[ns] = p->spec_bins;
  if (power_off) power_off[ns] = (p->numharm > 1) ? p->series[ns].p_off : p->p_floats;
  if (seg_off) seg_off[ns] = p->base_seg;
  return PULSCAN_OK;
}

int pulscan_plan_set_trials(pulscan_plan p, double n_trials) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (!(n_trials >= 1.0) || !std::isfinite(n_trials)) return fail(PULSCAN_ERR_INVALID_ARG, "n_trials must be >= 1");
  for (auto &t : p->n_trials) t = n_trials;
  p->trials_fixed = true;
  compute_thresholds(p);
  return upload_thresholds(p);
}

int pulscan_plan_set_widths(pulscan_plan p, int32_t mode, int32_t step) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (mode != PULSCAN_WIDTHS_ALL && mode != PULSCAN_WIDTHS_STEP && mode != PULSCAN_WIDTHS_LOG2)
    return fail(PULSCAN_ERR_INVALID_ARG, "unknown width mode");
  if (mode == PULSCAN_WIDTHS_STEP && step < 1) return fail(PULSCAN_ERR_INVALID_ARG, "step must be >= 1");
  std::vector<uint8_t> sel(p->z_max, 0);
  int64_t n_sel = 0;
  for (int w = 1; w <= p->z_max; ++w) {
    const int z = w - 1;
    bool on = true;
    if (mode == PULSCAN_WIDTHS_STEP) on = (z % step) == 0;
    if (mode == PULSCAN_WIDTHS_LOG2) on = z > 0 && (z & (z - 1)) == 0;
    sel[w - 1] = on ? 1 : 0;
    n_sel += on ? 1 : 0;
  }
  if (n_sel == 0) return fail(PULSCAN_ERR_INVALID_ARG, "no width searched");
  p->searched = sel;
  if (!p->trials_fixed)
    for (size_t i = 0; i < p->series.size(); ++i) p->n_trials[i] = static_cast<double>(p->series[i].m) * n_sel;
  compute_thresholds(p);
  return upload_thresholds(p);
}

int pulscan_plan_set_fidelity(pulscan_plan p, int32_t mode) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (mode != PULSCAN_FIDELITY_EXACT && mode != PULSCAN_FIDELITY_PAPER_GPU)
    return fail(PULSCAN_ERR_INVALID_ARG, "unknown fidelity mode");
  if (mode == PULSCAN_FIDELITY_PAPER_GPU && !is_power_of_four(p->seg_len))
    return fail(PULSCAN_ERR_INVALID_ARG, "median of medians needs segment_len = 4^k");
  if (mode == PULSCAN_FIDELITY_PAPER_GPU && p->seg_len > 16384)
    return fail(PULSCAN_ERR_UNSUPPORTED, "median of medians over more than 16384 bins");
  p->fidelity = mode;
  if (p->graph.exec) {   // the captured graph holds the other mode's kernels
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  return PULSCAN_OK;
}

static int search_impl(pulscan_plan p, const float *d_power, cudaStream_t s, const float *d_spec = nullptr);

int pulscan_plan_autotune(pulscan_plan p, const float *d_power, pulscan_stream stream) {
  if (!p || !d_power) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!aligned16(d_power)) return fail(PULSCAN_ERR_INVALID_ARG, "power buffer must be 16-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int timing = p->timing;
  p->timing = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PS_CUDA(cudaEventCreate(&e0));
  PS_CUDA(cudaEventCreate(&e1));
  float best = INFINITY;
  int best_w = p->search_warps, best_m = p->persist_mode, best_g = p->search_groups;
  int rc = PULSCAN_OK;
  for (int wg = 0; wg < 8 && !rc; ++wg) {
    const int w = 1 + (wg & 3), g = 1 + (wg >> 2);
    rc = relayout_tiles(p, w, g);
    for (int mode : {0, 1}) {
      if (rc) break;
      p->persist_mode = mode;
      rc = search_impl(p, d_power, s);   // warm-up (and the kernels' first-use costs)
      float tot = 0.0f;
      for (int r = 0; r < 3 && !rc; ++r) {
        cudaEventRecord(e0, s);
        rc = search_impl(p, d_power, s);
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
          tot += ms;
        else if (!rc)
          rc = fail(PULSCAN_ERR_CUDA, "event timing failed");
      }
      if (!rc && tot < best) {
        best = tot;
        best_w = w;
        best_g = g;
        best_m = mode;
      }
    }
  }
  p->persist_mode = best_m;
  const int rc2 = relayout_tiles(p, best_w, best_g);
  // then the deferred blocks' form, on the chosen launch shape
  float best_f = INFINITY;
  int form = p->defer_form;
  for (int f = 0; f < 2 && !rc && !rc2; ++f) {
    p->defer_form = f;
    rc = search_impl(p, d_power, s);
    float tot = 0.0f;
    for (int r = 0; r < 3 && !rc; ++r) {
      cudaEventRecord(e0, s);
      rc = search_impl(p, d_power, s);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        tot += ms;
      else if (!rc)
        rc = fail(PULSCAN_ERR_CUDA, "event timing failed");
    }
    if (!rc && tot < best_f) {
      best_f = tot;
      form = f;
    }
  }
  p->defer_form = form;
  if (p->graph.exec) {   // a graph captured before holds the other form's kernel
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PS_CUDA(cudaMemsetAsync(p->d_counters, 0, (4 + static_cast<size_t>(p->n_ranges)) * sizeof(uint32_t), s));
  PS_CUDA(cudaStreamSynchronize(s));
  p->timing = timing;
  return rc ? rc : rc2;
}

int pulscan_plan_set_tiling(pulscan_plan p, int32_t warps, int32_t persistent, int32_t packed) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (warps < 1 || warps > 4) return fail(PULSCAN_ERR_INVALID_ARG, "warps must be 1, 2, 3 or 4");
  if (persistent < -1 || persistent > 1) return fail(PULSCAN_ERR_INVALID_ARG, "persistent must be -1, 0 or 1");
  if (packed < 0 || packed > 1) return fail(PULSCAN_ERR_INVALID_ARG, "packed must be 0 or 1");
  PS_CUDA(cudaDeviceSynchronize());
  p->persist_mode = persistent;
  return relayout_tiles(p, warps, packed ? 2 : 1);
}

int pulscan_plan_tiling(pulscan_plan p, int32_t *warps, int32_t *persistent, int32_t *packed) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (warps) *warps = p->search_warps;
  if (persistent) *persistent = p->persist_mode;
  if (packed) *packed = p->search_groups == 2 ? 1 : 0;
  return PULSCAN_OK;
}

int pulscan_plan_test_wait_timeout(pulscan_plan p, int32_t limit_us) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (limit_us < 1 || limit_us > 1000) return fail(PULSCAN_ERR_INVALID_ARG, "limit_us must be 1..1000");
  p->wait_test_us = static_cast<uint32_t>(limit_us);
  return PULSCAN_OK;
}

int pulscan_plan_set_rblock(pulscan_plan p, int64_t block_width) {
  if (!p || block_width < 0) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  p->rblock = block_width;
  return PULSCAN_OK;
}

int pulscan_plan_stage_offsets(pulscan_plan p, int32_t harmonics, int64_t *h_power_off, int64_t *h_seg_off,
                               int64_t *h_bins) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (harmonics < 1 || harmonics > p->numharm) return fail(PULSCAN_ERR_INVALID_ARG, "no such harmonic stage");
  const size_t nb = static_cast<size_t>(p->n_base);
  const size_t first = nb * static_cast<size_t>(harmonics - 1);   // stage entries follow the layout order
  for (size_t u = 0; u < nb; ++u) {
    const Series &s = p->series[first + p->layout_of_user[u]];
    if (h_power_off) h_power_off[u] = s.p_off;
    if (h_seg_off) h_seg_off[u] = s.seg_off;
    if (h_bins) h_bins[u] = s.m;
  }
  const Series &last = p->series[first + nb - 1];
  if (h_power_off) h_power_off[nb] = last.p_off + last.m;
  if (h_seg_off) h_seg_off[nb] = last.seg_off + last.n_seg;
  if (h_bins) h_bins[nb] = 0;
  return PULSCAN_OK;
}

int pulscan_threshold_power(double shape, double n_trials, double sigma_thr, float *t_out) {
  if (!t_out || !(shape > 0.0) || !(n_trials >= 1.0) || !(sigma_thr >= 0.0) || !std::isfinite(sigma_thr) ||
      !std::isfinite(shape) || !std::isfinite(n_trials))
    return fail(PULSCAN_ERR_INVALID_ARG, "shape > 0, n_trials >= 1 and a finite sigma_thr >= 0 are required");
  *t_out = threshold_for(shape, host_log_sf_normal(sigma_thr) - std::log(n_trials));
  return PULSCAN_OK;
}

int pulscan_plan_thresholds(pulscan_plan p, int32_t series, float *h_thresh) {
  if (!p || !h_thresh) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (series < 0 || series >= static_cast<int32_t>(p->n_base))
    return fail(PULSCAN_ERR_INVALID_ARG, "series index out of range");
  const int li = p->layout_of_user[series];
  std::memcpy(h_thresh, p->h_thresh.data() + static_cast<size_t>(li) * p->z_max, p->z_max * sizeof(float));
  return PULSCAN_OK;
}

int pulscan_rfft(pulscan_plan p, const float *d_x, float *d_spec, pulscan_stream stream) {
  if (!p || !d_x || !d_spec) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!aligned16(d_x) || !aligned16(d_spec)) return fail(PULSCAN_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  record(p, 0, s);
  for (auto &f : p->fft) {
    cufftResult r = cufftSetStream(f.handle, s);
    if (r == CUFFT_SUCCESS)
      r = cufftExecR2C(f.handle, const_cast<cufftReal *>(d_x + f.x_off),
                       reinterpret_cast<cufftComplex *>(d_spec) + f.spec_off);
    if (r != CUFFT_SUCCESS) return cufft_fail(r, "cufftExecR2C");
  }
  record(p, 1, s);
  return PULSCAN_OK;
}

int pulscan_power_normalise(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats,
                            pulscan_stream stream) {
  if (!p || !d_spec || !d_power) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!aligned16(d_spec) || !aligned16(d_power)) return fail(PULSCAN_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  if (d_stats && !aligned16(d_stats)) return fail(PULSCAN_ERR_INVALID_ARG, "stats buffer must be 16-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  record(p, 2, s);
  int rc = launch_normalise(p, d_spec, d_power, d_stats, s);
  record(p, 3, s);
  if (rc || p->numharm <= 1) return rc;
  record(p, 12, s);
  rc = launch_harmonic_sums(p, d_power, s);
  record(p, 13, s);
  return rc;
}

static int search_impl(pulscan_plan p, const float *d_power, cudaStream_t s, const float *d_spec) {
  PS_CUDA(cudaMemsetAsync(p->d_counters, 0, (4 + static_cast<size_t>(p->n_ranges)) * sizeof(uint32_t), s));
  if (p->fidelity == PULSCAN_FIDELITY_PAPER_GPU) {
    // every (segment, width) maximum, then the polynomial significance of each
    record(p, 4, s);
    int rc = launch_maxima_only(p, d_power, s);
    if (rc) return rc;
    record(p, 5, s);
    record(p, 8, s);
    rc = launch_poly_finalize(p, s);
    record(p, 9, s);
    return rc;
  }
  record(p, 4, s);
  int rc = launch_search(p, d_power, s, d_spec);   // records 5, 6, 7 around the deferred kernel
  if (rc) return rc;
  record(p, 8, s);
  rc = launch_finalize(p, s);
  record(p, 9, s);
  return rc;
}

int pulscan_boxcar_search(pulscan_plan p, const float *d_power, pulscan_stream stream) {
  if (!p || !d_power) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!aligned16(d_power)) return fail(PULSCAN_ERR_INVALID_ARG, "power buffer must be 16-byte aligned");
  return search_impl(p, d_power, reinterpret_cast<cudaStream_t>(stream));
}

int pulscan_candidates(pulscan_plan p, pulscan_cand *h_out, int64_t cap, int64_t *n_out, pulscan_stream stream) {
  if (!p || !n_out || cap < 0 || (cap > 0 && !h_out)) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t ctr[4];
  PS_CUDA(cudaMemcpyAsync(ctr, p->d_counters, sizeof(ctr), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  const int64_t count = ctr[1];
  *n_out = count;
  const int64_t have = std::min<int64_t>(count, p->max_cands);
  std::vector<pulscan_cand> tmp(static_cast<size_t>(have));
  if (have > 0) {
    PS_CUDA(cudaMemcpyAsync(tmp.data(), p->d_cands, have * sizeof(pulscan_cand), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
  }
  // order by (series, harmonics, segment, width): integer keys formed once
  // per candidate ((series << 36 | harmonics << 32 | segment), (width << 32 |
  // index)); series < 2^28, harmonics <= 8, segments and widths < 2^32, the
  // index below 2^24
  std::vector<std::pair<uint64_t, uint64_t>> key(static_cast<size_t>(have));
  for (int64_t i = 0; i < have; ++i) {
    const pulscan_cand &c = tmp[i];
    const size_t e = static_cast<size_t>(p->n_base) * (c.harmonics - 1) + p->layout_of_user[c.series];
    const Series &se = p->series[e];
    const int64_t seg = std::min<int64_t>(static_cast<int64_t>(c.bin) / p->seg_len, se.n_seg - 1);
    key[i] = {(static_cast<uint64_t>(c.series) << 36) | (static_cast<uint64_t>(c.harmonics) << 32) |
                  static_cast<uint64_t>(seg),
              (static_cast<uint64_t>(c.width) << 32) | static_cast<uint64_t>(i)};
  }
  // the finaliser writes slot order, which is this order whenever the
  // layout keeps the caller's series order; sort only otherwise
  if (!std::is_sorted(key.begin(), key.end())) std::sort(key.begin(), key.end());
  const int64_t ncopy = std::min<int64_t>(have, cap);
  for (int64_t i = 0; i < ncopy; ++i) {
    h_out[i] = tmp[key[i].second & 0xffffffffull];
    if (p->rblock > 0) h_out[i].bin /= static_cast<uint64_t>(p->rblock);   // R-Block: the block index
  }
  if (ctr[2] & kErrTimeout) return fail(PULSCAN_ERR_TIMEOUT, "a bounded device wait timed out");
  if (count > cap || count > p->max_cands)
    return fail(PULSCAN_ERR_CAPACITY, "more candidates than the output capacity");
  return PULSCAN_OK;
}

int pulscan_segment_maxima(pulscan_plan p, const float *d_power, float *d_max, uint64_t *d_argmax,
                           pulscan_stream stream) {
  if (!p || !d_power || !d_max || !d_argmax) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!aligned16(d_power)) return fail(PULSCAN_ERR_INVALID_ARG, "power buffer must be 16-byte aligned");
  return launch_segmax(p, d_power, d_max, d_argmax, reinterpret_cast<cudaStream_t>(stream));
}

// The fused search applies: exact mode, no harmonic stages, blocks within
// the register normalisation kernel.
static bool fused_ok(pulscan_plan p) {
  return p->fused && p->numharm == 1 && p->fidelity == PULSCAN_FIDELITY_EXACT && normalise_range_ok(p);
}

// rfft, the block statistics, the fused search (P formed in the bank).
static int enqueue_fused(pulscan_plan p, const float *d_x, float *d_spec, cudaStream_t s) {
  int rc = pulscan_rfft(p, d_x, d_spec, reinterpret_cast<pulscan_stream>(s));
  if (rc) return rc;
  record(p, 2, s);
  rc = launch_normalise_stats(p, d_spec, s);
  record(p, 3, s);
  return rc ? rc : search_impl(p, nullptr, s, d_spec);
}

int pulscan_plan_set_fused(pulscan_plan p, int32_t on) {
  if (!p || on < 0 || on > 1) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  if (on && (p->numharm != 1 || p->fidelity != PULSCAN_FIDELITY_EXACT || !normalise_range_ok(p)))
    return fail(PULSCAN_ERR_UNSUPPORTED, "the fused search needs the exact mode, no harmonic stages and blocks of "
                                         "at most 16385 bins");
  if (on && !p->d_norm) {
    const int rc = dalloc(&p->d_norm, 4 * static_cast<size_t>(p->base_seg));
    if (rc) return rc;
  }
  PS_CUDA(cudaDeviceSynchronize());
  p->fused = on != 0;
  if (p->graph.exec) {
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  return PULSCAN_OK;
}

// A captured search of a batch runs pipelined: parts of about pipe_bins
// bins (series of one length), whose R2C transform and normalisation go on a
// high-priority side stream while the bank runs the previous part on the
// capture stream, so the memory-bound transforms and the latency-bound
// selects overlap the FP32-add-bound bank; the deferred blocks and the
// finaliser follow the last part.
static bool pipelined(pulscan_plan p) {
  return p->pipe_bins > 0 && p->chunks.size() >= 2 && p->numharm == 1 && p->fidelity == PULSCAN_FIDELITY_EXACT &&
         !p->fused && normalise_range_ok(p);
}

// Stream and events of a pipelined capture (created before the capture).
static int prepare_pipeline(pulscan_plan p) {
  GraphCache &g = p->graph;
  if (!g.side) {
    int least = 0, greatest = 0;
    PS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    PS_CUDA(cudaStreamCreateWithPriority(&g.side, cudaStreamNonBlocking, greatest));
  }
  while (g.ev.size() < p->chunks.size() + 1) {
    cudaEvent_t e = nullptr;
    PS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    g.ev.push_back(e);
  }
  return PULSCAN_OK;
}

// The pipelined search, enqueued on the capture stream `a` (and the side
// stream, forked from and joined back into `a`).
static int enqueue_pipelined(pulscan_plan p, const float *d_x, float *d_spec, float *d_power, cudaStream_t a) {
  GraphCache &g = p->graph;
  PS_CUDA(cudaMemsetAsync(p->d_counters, 0, (4 + static_cast<size_t>(p->n_ranges)) * sizeof(uint32_t), a));
  PS_CUDA(cudaEventRecord(g.ev[0], a));
  PS_CUDA(cudaStreamWaitEvent(g.side, g.ev[0], 0));
  const int64_t ns = static_cast<int64_t>(p->series.size());
  for (size_t i = 0; i < p->chunks.size(); ++i) {
    const Chunk &c = p->chunks[i];
    const Series &s0 = p->series[c.s_lo];
    const FftClass &f = p->chunk_fft[c.fft];
    cufftResult r = cufftSetStream(f.handle, g.side);
    if (r == CUFFT_SUCCESS)
      r = cufftExecR2C(f.handle, const_cast<cufftReal *>(d_x + s0.x_off),
                       reinterpret_cast<cufftComplex *>(d_spec) + s0.spec_off);
    if (r != CUFFT_SUCCESS) return cufft_fail(r, "cufftExecR2C");
    const int64_t seg_hi = c.s_hi < p->n_base ? p->series[c.s_hi].seg_off : p->base_seg;
    int rc = launch_normalise_range(p, d_spec, d_power, s0.seg_off, seg_hi - s0.seg_off, g.side);
    if (rc) return rc;
    PS_CUDA(cudaEventRecord(g.ev[i + 1], g.side));
    PS_CUDA(cudaStreamWaitEvent(a, g.ev[i + 1], 0));
    const int64_t tile_hi = c.s_hi < ns ? p->series[c.s_hi].tile_off : p->total_tiles;
    rc = launch_search_tiles(p, d_power, s0.tile_off, tile_hi - s0.tile_off, a);
    if (rc) return rc;
  }
  int rc = launch_deferred(p, d_power, a);
  if (!rc) rc = launch_finalize(p, a);
  return rc;
}

int pulscan_plan_set_pipeline(pulscan_plan p, int64_t part_bins) {
  if (!p || part_bins < 0) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  PS_CUDA(cudaDeviceSynchronize());
  return build_chunks(p, part_bins);
}

int pulscan_plan_pipeline_parts(pulscan_plan p, int64_t *n_parts) {
  if (!p || !n_parts) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  *n_parts = pipelined(p) ? static_cast<int64_t>(p->chunks.size()) : 0;
  return PULSCAN_OK;
}

int pulscan_search(pulscan_plan p, const float *d_x, float *d_spec, float *d_power, int use_graph,
                   pulscan_stream stream) {
  if (!p || !d_x || !d_spec || !d_power) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // an armed timeout test runs outside the graph (a captured graph would
  // keep the test in every replay)
  if (!use_graph || p->wait_test_us != 0u) {
    if (fused_ok(p) && p->wait_test_us == 0u) return enqueue_fused(p, d_x, d_spec, s);
    int rc = pulscan_rfft(p, d_x, d_spec, stream);
    if (!rc) rc = pulscan_power_normalise(p, d_spec, d_power, nullptr, stream);
    if (!rc) rc = pulscan_boxcar_search(p, d_power, stream);
    return rc;
  }
  // The work is captured once on a plan-owned stream (the legacy default
  // stream cannot be captured) and the graph is launched on the caller's.
  GraphCache &g = p->graph;
  if (!(g.exec && g.x == d_x && g.spec == d_spec && g.power == d_power)) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (!g.capture) PS_CUDA(cudaStreamCreateWithFlags(&g.capture, cudaStreamNonBlocking));
    // with timing on, the stage events are captured as event-record nodes and
    // re-recorded by every launch of the graph
    const pulscan_stream cs = reinterpret_cast<pulscan_stream>(g.capture);
    const bool pipe = pipelined(p);
    if (pipe) {
      const int rp = prepare_pipeline(p);
      if (rp) return rp;
    }
    PS_CUDA(cudaStreamBeginCapture(g.capture, cudaStreamCaptureModeThreadLocal));
    int rc = PULSCAN_OK;
    if (pipe) {
      rc = enqueue_pipelined(p, d_x, d_spec, d_power, g.capture);
    } else if (fused_ok(p)) {
      rc = enqueue_fused(p, d_x, d_spec, g.capture);
    } else {
      rc = pulscan_rfft(p, d_x, d_spec, cs);
      if (!rc) rc = pulscan_power_normalise(p, d_spec, d_power, nullptr, cs);
      if (!rc) rc = pulscan_boxcar_search(p, d_power, cs);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g.capture, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
    // the side stream's priority is kept per node (its parts start first on SMs that free up)
    const cudaError_t ei =
        cudaGraphInstantiateWithFlags(&g.exec, graph, pipe ? cudaGraphInstantiateFlagUseNodePriority : 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
    g.x = d_x;
    g.spec = d_spec;
    g.power = d_power;
  }
  PS_CUDA(cudaGraphLaunch(g.exec, s));
  return PULSCAN_OK;
}

int pulscan_search_host_async(pulscan_plan p, const float *h_x, int use_graph, pulscan_stream stream) {
  if (!p || !h_x) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!p->own_x) {
    int rc = dalloc(&p->own_x, p->x_floats);
    if (!rc) rc = dalloc(&p->own_spec, 2 * p->spec_bins);
    if (!rc) rc = dalloc(&p->own_power, p->p_floats);
    if (rc) return rc;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  PS_CUDA(cudaMemcpyAsync(p->own_x, h_x, p->x_floats * sizeof(float), cudaMemcpyHostToDevice, s));
  return pulscan_search(p, p->own_x, p->own_spec, p->own_power, use_graph, stream);
}

int pulscan_search_host(pulscan_plan p, const float *h_x, pulscan_cand *h_out, int64_t cap, int64_t *n_out,
                        int use_graph, pulscan_stream stream) {
  if (!p || !h_x || !n_out) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  const int rc = pulscan_search_host_async(p, h_x, use_graph, stream);
  if (rc) return rc;
  return pulscan_candidates(p, h_out, cap, n_out, stream);
}

int pulscan_plan_counters(pulscan_plan p, int64_t *h_out, int32_t n) {
  if (!p || !h_out || n < 0) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  uint32_t ctr[4];
  PS_CUDA(cudaMemcpy(ctr, p->d_counters, sizeof(ctr), cudaMemcpyDeviceToHost));
  const int64_t vals[4] = {ctr[0], p->item_cap, ctr[1], p->max_cands};
  for (int i = 0; i < std::min(n, 4); ++i) h_out[i] = vals[i];
  return PULSCAN_OK;
}

int pulscan_plan_set_defer_capacity(pulscan_plan p, int64_t cap) {
  if (!p || cap < 0 || cap > (int64_t(1) << 24)) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  if (cap > p->alloc_item_cap) {
    // grow the list (the captured graph holds the old pointers: drop it)
    PS_CUDA(cudaDeviceSynchronize());
    unsigned long long *items = nullptr;
    float *snaps = nullptr;
    if (dalloc(&items, static_cast<size_t>(cap)) || dalloc(&snaps, static_cast<size_t>(cap) * kR * 32)) {
      if (items) cudaFree(items);
      return fail(PULSCAN_ERR_NOMEM, "deferred-block list allocation failed");
    }
    cudaFree(p->d_items);
    cudaFree(p->d_snaps);
    p->d_items = items;
    p->d_snaps = snaps;
    p->alloc_item_cap = cap;
  }
  // the captured graph holds the old list and capacity in its launches
  if (p->graph.exec && cap != p->item_cap) {
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  p->item_cap = cap;
  return PULSCAN_OK;
}

int pulscan_plan_set_defer_form(pulscan_plan p, int32_t form) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (form != 0 && form != 1) return fail(PULSCAN_ERR_INVALID_ARG, "form must be 0 or 1");
  if (p->graph.exec && form != p->defer_form) {   // the captured graph launches the other kernel
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  p->defer_form = form;
  return PULSCAN_OK;
}

int pulscan_plan_defer_form(pulscan_plan p, int32_t *form) {
  if (!p || !form) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  *form = p->defer_form;
  return PULSCAN_OK;
}

int pulscan_plan_enable_timing(pulscan_plan p, int on) {
  if (!p) return fail(PULSCAN_ERR_INVALID_ARG, "null plan");
  if (on) {
    for (auto &e : p->ev)
      if (!e) PS_CUDA(cudaEventCreate(&e));
  }
  p->timing = (on == 2) ? 2 : (on != 0 ? 1 : 0);
  for (bool &r : p->ran) r = false;
  // a captured graph holds the event records of the setting it was captured
  // with: the next pulscan_search captures anew (an in-flight launch finishes)
  if (p->graph.exec) {
    cudaGraphExecDestroy(p->graph.exec);
    p->graph.exec = nullptr;
  }
  return PULSCAN_OK;
}

int pulscan_plan_timings(pulscan_plan p, float *h_ms, int32_t n) {
  if (!p || !h_ms || n < 0) return fail(PULSCAN_ERR_INVALID_ARG, "bad argument");
  for (int i = 0; i < std::min(n, 7); ++i) {
    h_ms[i] = -1.0f;
    if (!p->ran[i] || !p->ev[2 * i]) continue;
    PS_CUDA(cudaEventSynchronize(p->ev[2 * i + 1]));
    float ms = 0.0f;
    PS_CUDA(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]));
    h_ms[i] = ms;
  }
  return PULSCAN_OK;
}

}  // extern "C"
