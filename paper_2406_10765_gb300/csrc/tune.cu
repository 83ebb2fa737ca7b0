// Autotuner for the FFT plan of the local part of H psi (Sec. III-D picks,
// per execution step, the fastest of the process counts that fit in memory;
// here the candidates are the register line-FFT factorisations N = L R of
// the cell's grid, the Stockham passes, and the band batch of the z-pencils).
// The K split of the tensor-core GEMMs is tuned in tc_gemm.cu.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pw_internal.cuh"

namespace {

// deterministic scratch bands: entries in [-0.5, 0.5) + i [-0.5, 0.5) from a
// 64-bit integer hash of the index (timing input only)
__global__ void k_fill_scratch(double2 *x, long n) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double re = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  const double im = (double)((z << 21) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  x[i] = make_double2(re, im);
}

int plan_index(const pw_cell *c, int L, int R, int fp32, int compact) {
  const int np = pw_reg_plan_count();
  for (int i = 0; i < np; ++i) {
    const pw_reg_plan *p = pw_reg_plan_at(i);
    if (p->L == L && p->R == R && pw_reg_plan_fits(c, i, fp32, compact)) return i;
  }
  return -2;
}

void describe(const pw_cell *c, int fp32, pw_fft_plan *out) {
  const pw_reg_plan *p = pw_reg_plan_at(pw_cell_fft_plan(c, fp32));
  out->L = p ? p->L : 0;
  out->R = p ? p->R : 0;
  out->compact = p ? pw_cell_fft_compact(c, fp32) : 0;
  out->batch_bytes = pw_cell_fft_batch_bytes(c, fp32);
}

}  // namespace

extern "C" int pw_fft_plans(int n, pw_fft_plan *plans, int max) {
  int k = 0;
  const int np = pw_reg_plan_count();
  for (int i = 0; i < np; ++i) {
    const pw_reg_plan *p = pw_reg_plan_at(i);
    if (p->N != n) continue;
    if (plans && k < max) plans[k] = pw_fft_plan{p->L, p->R, 0, 0};
    ++k;
  }
  return k;
}

extern "C" pw_status pw_cell_set_fft_plan(pw_cell *c, int precision, const pw_fft_plan *plan) {
  if (!c || !plan || (precision != PW_FP64 && precision != PW_MIXED)) return PW_ERR_ARG;
  const int fp32 = precision == PW_MIXED;
  int idx = -1;
  if (plan->compact != 0 && plan->compact != 1) return PW_ERR_ARG;
  if (plan->L != 0 || plan->R != 0) {
    idx = plan_index(c, plan->L, plan->R, fp32, plan->compact);
    if (idx < 0) return PW_ERR_ARG;
  } else {
    // the Stockham passes: full plane only
    if (plan->compact || (size_t)c->N[1] * (c->N[0] + 1) * (fp32 ? 8 : 16) > 227 * 1024) return PW_ERR_ARG;
  }
  c->fft_plan[fp32] = idx;
  c->fft_compact[fp32] = idx >= 0 ? plan->compact : 0;
  c->fft_batch[fp32] = plan->batch_bytes;
  return PW_OK;
}

extern "C" pw_status pw_cell_get_fft_plan(const pw_cell *c, int precision, pw_fft_plan *plan) {
  if (!c || !plan || (precision != PW_FP64 && precision != PW_MIXED)) return PW_ERR_ARG;
  describe(c, precision == PW_MIXED, plan);
  return PW_OK;
}

extern "C" pw_status pw_cell_autotune_fft(pw_cell *c, int nb, int precision, void *stream,
                                          pw_fft_tune_report *rep) {
  if (!c || nb < 1 || (precision != PW_FP64 && precision != PW_MIXED)) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int fp32 = precision == PW_MIXED;
  const int npw = c->npw;
  const size_t per_band = (size_t)c->N[2] * c->ncol * (fp32 ? sizeof(float2) : sizeof(double2));
  // candidates: every fitting register plan in both plane layouts, the
  // Stockham passes; three batch sizes
  std::vector<std::pair<int, int>> plans;
  const int np = pw_reg_plan_count();
  for (int cp = 0; cp < 2; ++cp)
    for (int i = 0; i < np; ++i)
      if (pw_reg_plan_fits(c, i, fp32, cp)) plans.push_back({i, cp});
  // the Stockham passes hold one x-y plane in shared memory
  if ((size_t)c->N[1] * (c->N[0] + 1) * (fp32 ? sizeof(float2) : sizeof(double2)) <= 227 * 1024)
    plans.push_back({-1, 0});
  if (plans.empty()) return PW_ERR_ARG;
  const size_t batches[3] = {(size_t)32 << 20, (size_t)64 << 20, (size_t)128 << 20};

  const int saved_plan = c->fft_plan[fp32], saved_cp = c->fft_compact[fp32];
  const size_t saved_batch = c->fft_batch[fp32];
  pw_fft_tune_report r{};
  c->fft_plan[fp32] = -2;
  c->fft_batch[fp32] = 0;
  describe(c, fp32, &r.dflt);
  const int dflt_idx = pw_cell_fft_plan(c, fp32), dflt_cp = pw_cell_fft_compact(c, fp32);
  const size_t dflt_batch = pw_cell_fft_batch_bytes(c, fp32);
  const int dflt_nbatch = (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, dflt_batch / per_band));

  double2 *psi = nullptr, *hpsi = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pw_status s = PW_OK;
  const size_t bytes = (size_t)npw * nb * sizeof(double2);
  if (cudaMalloc((void **)&psi, bytes) != cudaSuccess || cudaMalloc((void **)&hpsi, bytes) != cudaSuccess) {
    cudaGetLastError();
    s = PW_ERR_OOM;
  }
  if (s == PW_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) s = PW_ERR_CUDA;
  if (s == PW_OK) {
    const long n = (long)npw * nb;
    pw_count_launch();
    k_fill_scratch<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(psi, n);
    s = pw_check_launch("autotune fill");
  }
  std::string log;
  double best = 1e300;
  int best_plan = dflt_idx, best_cp = dflt_cp;
  size_t best_batch = dflt_batch;
  for (int pi = 0; pi < (int)plans.size() && s == PW_OK; ++pi) {
    int last_batch = -1;
    for (int bi = 0; bi < 3 && s == PW_OK; ++bi) {
      // batches that give the same band count per pass are the same candidate
      const int nbatch = (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, batches[bi] / per_band));
      if (nbatch == last_batch) continue;
      last_batch = nbatch;
      c->fft_plan[fp32] = plans[pi].first;
      c->fft_compact[fp32] = plans[pi].second;
      c->fft_batch[fp32] = batches[bi];
      double ms = 1e300;
      for (int rep_i = 0; rep_i < 4 && s == PW_OK; ++rep_i) {
        cudaEventRecord(e0, st);
        s = pw_apply_local(c, psi, npw, nb, hpsi, precision, st);
        cudaEventRecord(e1, st);
        if (s != PW_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { s = PW_ERR_CUDA; break; }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep_i > 0) ms = std::min(ms, (double)t);   // first run: warm-up
      }
      if (s != PW_OK) break;
      ++r.ncand;
      {
        const pw_reg_plan *rp = pw_reg_plan_at(plans[pi].first);
        char line[160];
        snprintf(line, sizeof line, "L=%d R=%d compact=%d batch_mib=%zu bands_per_batch=%d ms=%.4f\n",
                 rp ? rp->L : 0, rp ? rp->R : 0, plans[pi].second, batches[bi] >> 20, nbatch, ms);
        log += line;
      }
      const bool is_default = plans[pi].first == dflt_idx && plans[pi].second == dflt_cp && nbatch == dflt_nbatch;
      if (is_default) r.ms_default = ms;
      if (ms < best) {
        best = ms;
        best_plan = plans[pi].first;
        best_cp = plans[pi].second;
        best_batch = batches[bi];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (psi) cudaFree(psi);
  if (hpsi) cudaFree(hpsi);
  if (s != PW_OK) {
    c->fft_plan[fp32] = saved_plan;
    c->fft_compact[fp32] = saved_cp;
    c->fft_batch[fp32] = saved_batch;
    return s;
  }
  c->fft_plan[fp32] = best_plan;
  c->fft_compact[fp32] = best_cp;
  c->fft_batch[fp32] = best_batch;
  c->fft_tune_log = log;
  describe(c, fp32, &r.best);
  r.ms_best = best;
  if (rep) *rep = r;
  return PW_OK;
}

extern "C" int pw_cell_fft_tune_log(const pw_cell *c, char *buf, size_t len) {
  if (!c) return 0;
  const std::string &s = c->fft_tune_log;
  if (buf && len) {
    const size_t n = std::min(len - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return (int)s.size();
}
