// Autotuner of the probe solver's block width R (the number of right-hand
// sides that share one pass over the band).
//
// For a band and a probe count K the tuner times one block-PCG iteration
// (k_blk_it, CUDA events) at each candidate R in {8, 16, 32} (R not wider
// than K rounded up to 8) and picks the R that minimises ceil(K / R) x t(R),
// the cost of one iteration sweep over all probes.  Choices are cached in the
// context by (floor(log2 N), K class) and, when the environment variable
// BFSDF_TUNE_CACHE names a file, in that file as JSON lines
//   {"device": "...", "sms": 152, "n_log2": 19, "k_class": 32, "R": 32, "ms": [t8, t16, t32]}
// read when the first choice is looked up and appended when a new one is
// measured.  Entries of other GPU models are ignored.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "internal.cuh"

namespace {

int n_log2(int64_t N) {
  int k = 0;
  while (k < 62 && (int64_t(1) << (k + 1)) <= N) ++k;
  return k;
}

int k_class(int K) { return K >= 32 ? 32 : (K >= 16 ? 16 : 8); }

std::string device_key(int dev, int* sms) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    *sms = 0;
    return "unknown";
  }
  *sms = p.multiProcessorCount;
  return std::string(p.name);
}

// one line of the cache file, in the fixed format written by append_file
bool parse_line(const char* s, std::string* dev, int* sms, int* nl, int* kc, int* R, double ms[3]) {
  const char* d = strstr(s, "\"device\": \"");
  if (!d) return false;
  d += 11;
  const char* e = strchr(d, '"');
  if (!e) return false;
  dev->assign(d, e - d);
  return sscanf(e, "\", \"sms\": %d, \"n_log2\": %d, \"k_class\": %d, \"R\": %d, \"ms\": [%lf, %lf, %lf]", sms, nl, kc,
                R, &ms[0], &ms[1], &ms[2]) == 7;
}

void remember(bf_ctx* ctx, const TuneEntry& t) {
  for (auto& x : ctx->tune)
    if (x.n_log2 == t.n_log2 && x.k_class == t.k_class) {
      x = t;
      return;
    }
  ctx->tune.push_back(t);
}

void load_file(bf_ctx* ctx) {
  ctx->tune_loaded = true;
  const char* path = getenv("BFSDF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  int sms0 = 0;
  const std::string dev0 = device_key(ctx->device, &sms0);
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    std::string dev;
    int sms, nl, kc, R;
    double ms[3];
    if (!parse_line(line, &dev, &sms, &nl, &kc, &R, ms) || dev != dev0 || sms != sms0) continue;
    if (R != 8 && R != 16 && R != 32) continue;
    remember(ctx, TuneEntry{nl, kc, R, {ms[0], ms[1], ms[2]}});
  }
  fclose(f);
}

void append_file(bf_ctx* ctx, const TuneEntry& t) {
  const char* path = getenv("BFSDF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  int sms = 0;
  const std::string dev = device_key(ctx->device, &sms);
  fprintf(f,
          "{\"device\": \"%s\", \"sms\": %d, \"n_log2\": %d, \"k_class\": %d, \"R\": %d, \"ms\": [%.6g, %.6g, "
          "%.6g]}\n",
          dev.c_str(), sms, t.n_log2, t.k_class, t.R, t.ms[0], t.ms[1], t.ms[2]);
  fclose(f);
}

}  // namespace

bf_status autotune_rhs_block(bf_ctx* ctx, bf_band* b, int K, bool force, int* R_out, double ms_out[3]) {
  if (!ctx->tune_loaded) load_file(ctx);
  const int nl = n_log2(b->N > 0 ? b->N : 1), kc = k_class(K);
  if (!force)
    for (const auto& t : ctx->tune)
      if (t.n_log2 == nl && t.k_class == kc) {
        *R_out = t.R;
        if (ms_out) memcpy(ms_out, t.ms, sizeof(t.ms));
        return BF_OK;
      }
  const int cand[3] = {8, 16, 32};
  double ms[3] = {0.0, 0.0, 0.0};
  int best = 8;
  double best_cost = INFINITY;
  for (int i = 0; i < 3; ++i) {
    const int R = cand[i];
    if (R > 8 && R > ((K + 7) / 8) * 8) continue;  // wider than the probes need
    double t = 0.0;
    BF_TRY(bench_block_iter(ctx, b, R, 1, &t));  // warm-up
    BF_TRY(bench_block_iter(ctx, b, R, 5, &t));
    ms[i] = t;
    const double cost = std::ceil((double)K / R) * t;
    if (cost < best_cost) {
      best_cost = cost;
      best = R;
    }
  }
  const TuneEntry t{nl, kc, best, {ms[0], ms[1], ms[2]}};
  remember(ctx, t);
  append_file(ctx, t);
  *R_out = best;
  if (ms_out) memcpy(ms_out, ms, sizeof(ms));
  return BF_OK;
}

extern "C" bf_status bf_autotune_rhs_block(bf_ctx* ctx, bf_band* band, int K, int force, int* rhs_block,
                                           double* ms_per_iter) {
  BF_ENTER(ctx);
  if (!ctx || !band || !rhs_block || K < 1) return BF_EINVAL;
  if (!band->integrated) return bf_fail(ctx, BF_ESTATE, "bf_autotune_rhs_block: call bf_integrate_depth first");
  if (band->obs_mode == 3) return bf_fail(ctx, BF_ESTATE, "bf_autotune_rhs_block: the band holds trilinear rows");
  if (band->N == 0) {
    *rhs_block = 8;
    if (ms_per_iter) memset(ms_per_iter, 0, 3 * sizeof(double));
    return BF_OK;
  }
  return autotune_rhs_block(ctx, band, K, force != 0, rhs_block, ms_per_iter);
}
