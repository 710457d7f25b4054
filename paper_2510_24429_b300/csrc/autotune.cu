// Layout autotuner (pdhg_autotune). The step kernels' speed on a given LP
// depends on three layout choices: the threads per block (step_block), the
// most rows one thread reduces at once in the short-row slices
// (rows_per_thread), and the row length from which a row gets a whole warp
// (long_row_min). The tuner times candidates with the engine's own CUDA-event
// kernel timing, by coordinate search (long_row_min first, then
// rows_per_thread, then step_block, each around the best so far), and keeps
// the fastest. Choices are remembered per LP profile in a plain text file,
// one line per profile, so that LPs of the same shape are not timed again.
//
// The profile of an LP (or batch): precision, the number of instances, m, n
// and nnz on a log2 scale (steps of 1/2), and for A and for A^T the share of
// rows in each power-of-two length class, rounded to 10%.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/pdhg.h"

void pdhg_set_global_error(const char* msg);

namespace {

constexpr int NCLS = 34;  // length classes: 0 = empty row, k >= 1 = lengths in [2^(k-1), 2^k)

int length_class(int64_t len) {
  int k = 0;
  while (len > 0 && k < NCLS - 1) {
    ++k;
    len >>= 1;
  }
  return k;
}

std::string shares(const std::vector<int64_t>& cls, int64_t rows) {
  std::ostringstream o;
  bool first = true;
  for (int k = 0; k < NCLS; ++k) {
    const long tenths = lround(10.0 * (double)cls[k] / (double)std::max<int64_t>(1, rows));  // units of 10%
    if (!tenths) continue;
    o << (first ? "" : ",") << k << ":" << tenths * 10;
    first = false;
  }
  return o.str();
}

long half_log2(int64_t v) { return lround(2.0 * log2((double)std::max<int64_t>(1, v))); }

pdhg_status fail(pdhg_status s, const std::string& msg) {
  pdhg_set_global_error(msg.c_str());
  return s;
}

pdhg_status check_lps(int count, const pdhg_lp_desc* lps) {
  if (count < 1 || !lps) return fail(PDHG_ERR_INVALID, "count < 1 or lps is NULL");
  for (int i = 0; i < count; ++i) {
    const pdhg_lp_desc& L = lps[i];
    if (L.m < 1 || L.n < 1 || L.nnz < 0 || !L.row_ptr || (L.nnz > 0 && !L.col_idx))
      return fail(PDHG_ERR_INVALID, "instance " + std::to_string(i) + ": bad sizes or NULL arrays");
    if (L.row_ptr[0] != 0 || L.row_ptr[L.m] != L.nnz)
      return fail(PDHG_ERR_INVALID, "instance " + std::to_string(i) + ": row_ptr[0] != 0 or row_ptr[m] != nnz");
    for (int64_t r = 0; r < L.m; ++r)
      if (L.row_ptr[r + 1] < L.row_ptr[r])
        return fail(PDHG_ERR_INVALID, "instance " + std::to_string(i) + ": row_ptr not non-decreasing");
    for (int64_t k = 0; k < L.nnz; ++k)
      if (L.col_idx[k] < 0 || L.col_idx[k] >= L.n)
        return fail(PDHG_ERR_INVALID, "instance " + std::to_string(i) + ": column index out of range");
  }
  return PDHG_OK;
}

std::string profile_key(int count, const pdhg_lp_desc* lps, int precision) {
  std::vector<int64_t> ca(NCLS, 0), ct(NCLS, 0);
  int64_t M = 0, N = 0, Z = 0;
  for (int i = 0; i < count; ++i) {
    const pdhg_lp_desc& L = lps[i];
    M += L.m;
    N += L.n;
    Z += L.nnz;
    for (int64_t r = 0; r < L.m; ++r) ca[length_class(L.row_ptr[r + 1] - L.row_ptr[r])] += 1;
    std::vector<int64_t> colcnt(L.n, 0);
    for (int64_t k = 0; k < L.nnz; ++k) colcnt[L.col_idx[k]] += 1;
    for (int64_t j = 0; j < L.n; ++j) ct[length_class(colcnt[j])] += 1;
  }
  std::ostringstream o;
  o << "p" << precision << "/b" << half_log2(count) << "/m" << half_log2(M) << "/n" << half_log2(N) << "/z"
    << half_log2(Z) << "/A" << shares(ca, M) << "/T" << shares(ct, N);
  return o.str();
}

struct Choice {
  int step_block = 256, rows_per_thread = 4, long_row_min = 128;
  double ms = 0.0;
};

// the last stored choice for key, if any
bool cache_lookup(const char* path, const std::string& key, Choice* out) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    Choice c;
    if (!(is >> k >> c.step_block >> c.rows_per_thread >> c.long_row_min >> c.ms)) continue;
    if (k != key) continue;
    const bool valid = (c.step_block == 128 || c.step_block == 256 || c.step_block == 512) &&
                       (c.rows_per_thread == 1 || c.rows_per_thread == 2 || c.rows_per_thread == 4) &&
                       c.long_row_min >= 1;
    if (valid) {
      *out = c;
      found = true;
    }
  }
  return found;
}

bool cache_append(const char* path, const std::string& key, const Choice& c) {
  std::ofstream f(path, std::ios::app);
  if (!f) return false;
  f << key << " " << c.step_block << " " << c.rows_per_thread << " " << c.long_row_min << " " << c.ms << "\n";
  return (bool)f;
}

// mean milliseconds per iteration of the two step kernels under options o
pdhg_status time_candidate(int count, const pdhg_lp_desc* lps, pdhg_options o, void* stream, double* ms) {
  o.kernel_timing = 1;
  o.persistent = 0;
  o.use_graphs = 0;
  o.snapshot_every = 0;
  o.eps_cross = 0.0;
  o.record_for_backward = 0;
  o.inputs_on_device = 0;
  pdhg_ctx* ctx = nullptr;
  pdhg_status s = count == 1 ? pdhg_create(lps[0].m, lps[0].n, lps[0].nnz, lps[0].row_ptr, lps[0].col_idx, lps[0].val,
                                           lps[0].b, lps[0].c, nullptr, nullptr, &o, stream, &ctx)
                             : pdhg_create_batch(count, lps, &o, stream, &ctx);
  if (s != PDHG_OK) return s;
  pdhg_info i0{}, i1{};
  // warm-up, then a first measurement that sizes the final one to ~20 ms of kernels
  int64_t iters = 64;
  s = pdhg_iterate(ctx, 64, 0.0, nullptr);
  if (s == PDHG_OK) s = pdhg_get_info(ctx, &i0);
  if (s == PDHG_OK) s = pdhg_iterate(ctx, iters, 0.0, nullptr);
  if (s == PDHG_OK) s = pdhg_get_info(ctx, &i1);
  if (s == PDHG_OK) {
    const double per = (i1.kernel_ms_primal + i1.kernel_ms_dual - i0.kernel_ms_primal - i0.kernel_ms_dual) /
                       (double)std::max<int64_t>(1, i1.kernel_launches_primal - i0.kernel_launches_primal);
    iters = std::min<int64_t>(4096, std::max<int64_t>(64, (int64_t)(20.0 / std::max(per, 1e-4))));
    i0 = i1;
    s = pdhg_iterate(ctx, iters, 0.0, nullptr);
  }
  if (s == PDHG_OK) s = pdhg_get_info(ctx, &i1);
  if (s == PDHG_OK)
    *ms = (i1.kernel_ms_primal + i1.kernel_ms_dual - i0.kernel_ms_primal - i0.kernel_ms_dual) /
          (double)std::max<int64_t>(1, i1.kernel_launches_primal - i0.kernel_launches_primal);
  if (s != PDHG_OK) pdhg_set_global_error(pdhg_last_error(ctx));
  pdhg_destroy(ctx);
  return s;
}

}  // namespace

extern "C" {

PDHG_API pdhg_status pdhg_profile_key(int count, const pdhg_lp_desc* lps, int precision, char* buf, int64_t cap) {
  if (!buf || cap < 1) return fail(PDHG_ERR_INVALID, "buf is NULL or cap < 1");
  pdhg_status s = check_lps(count, lps);
  if (s != PDHG_OK) return s;
  const std::string key = profile_key(count, lps, precision);
  if ((int64_t)key.size() + 1 > cap) return fail(PDHG_ERR_INVALID, "buf too small for the profile key");
  std::copy(key.begin(), key.end(), buf);
  buf[key.size()] = '\0';
  return PDHG_OK;
}

PDHG_API pdhg_status pdhg_autotune(int count, const pdhg_lp_desc* lps, const pdhg_options* opt,
                                   const char* cache_path, void* cuda_stream, pdhg_options* tuned,
                                   int* from_cache) {
  if (!tuned) return fail(PDHG_ERR_INVALID, "tuned is NULL");
  if (from_cache) *from_cache = 0;
  pdhg_options base;
  if (opt)
    base = *opt;
  else
    pdhg_default_options(&base);
  if (base.inputs_on_device) return fail(PDHG_ERR_INVALID, "pdhg_autotune takes host inputs");
  pdhg_status s = check_lps(count, lps);
  if (s != PDHG_OK) return s;
  const std::string key = profile_key(count, lps, base.precision);
  Choice best;
  if (cache_path && cache_lookup(cache_path, key, &best)) {
    *tuned = base;
    tuned->step_block = best.step_block;
    tuned->rows_per_thread = best.rows_per_thread;
    tuned->long_row_min = best.long_row_min;
    if (from_cache) *from_cache = 1;
    return PDHG_OK;
  }
  best.step_block = base.step_block ? base.step_block : 256;
  best.rows_per_thread = base.rows_per_thread;
  best.long_row_min = base.long_row_min;
  best.ms = -1.0;
  auto run = [&](Choice c) -> pdhg_status {
    pdhg_options o = base;
    o.step_block = c.step_block;
    o.rows_per_thread = c.rows_per_thread;
    o.long_row_min = c.long_row_min;
    double ms = 0.0;
    pdhg_status r = time_candidate(count, lps, o, cuda_stream, &ms);
    if (r != PDHG_OK) return r;
    if (best.ms < 0.0 || ms < best.ms) {
      best = c;
      best.ms = ms;
    }
    return PDHG_OK;
  };
  // coordinate search: the heavy-row threshold, then rows per thread, then block size
  for (int lrm : {32, 64, 128, 256, 512}) {
    Choice c = best;
    c.long_row_min = lrm;
    if ((s = run(c)) != PDHG_OK) return s;
  }
  const Choice after_lrm = best;
  for (int rpt : {1, 2, 4}) {
    if (rpt == after_lrm.rows_per_thread) continue;
    Choice c = after_lrm;
    c.rows_per_thread = rpt;
    if ((s = run(c)) != PDHG_OK) return s;
  }
  const Choice after_rpt = best;
  for (int blk : {128, 256, 512}) {
    if (blk == after_rpt.step_block) continue;
    Choice c = after_rpt;
    c.step_block = blk;
    if ((s = run(c)) != PDHG_OK) return s;
  }
  *tuned = base;
  tuned->step_block = best.step_block;
  tuned->rows_per_thread = best.rows_per_thread;
  tuned->long_row_min = best.long_row_min;
  if (cache_path && !cache_append(cache_path, key, best))
    return fail(PDHG_ERR_INVALID, std::string("cannot append to the cache file ") + cache_path);
  return PDHG_OK;
}

}  // extern "C"
