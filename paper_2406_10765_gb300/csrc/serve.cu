// Continuous-batching request loop over fixed-potential eigensolves.
//
// Requests (diamond Si or C supercells of n^3 cubic cells, an Ecut, a band
// count, a seed, an arrival time) are admitted while both a slot and device
// memory are free: the admission test uses the footprint model below against
// the caller's budget.  Each admitted request runs on its own CUDA stream from
// a worker thread (cell setup, LOBPCG to tolerance, FP64 finish in mixed
// precision), so the kernels of concurrent requests overlap on the GPU and a
// request that arrives while others run starts as soon as a slot and memory
// free up.  Each request's inputs are regenerated from its seed (SplitMix64,
// same counter layout as the seeded input generator of the tests), and every
// kernel is deterministic, so a request's result does not depend on what else
// is running.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "dense.cuh"
#include "pw_internal.cuh"

namespace {

double uniform01(uint64_t seed, uint64_t i) { return (double)(splitmix64(seed, i) >> 11) * 0x1.0p-53; }

const double kBasis[8][3] = {{0.00, 0.00, 0.00}, {0.00, 0.50, 0.50}, {0.50, 0.00, 0.50},
                             {0.50, 0.50, 0.00}, {0.25, 0.25, 0.25}, {0.25, 0.75, 0.75},
                             {0.75, 0.25, 0.75}, {0.75, 0.75, 0.25}};

struct CellInputs {
  double L;
  std::vector<double> tau, depth, dkb;
};

// diamond supercell, atoms ordered by cell (ix, iy, iz) then basis atom;
// depth[a] = -1 + 0.1 (2u - 1) with u = draw a; D[a][k] = 0.5 + u, u = draw natom + 4a + k
CellInputs make_inputs(const pw_request &r) {
  CellInputs c;
  const double a = r.species == 1 ? 6.74 : 10.26;
  const int n = r.ncell;
  c.L = n * a;
  for (int ix = 0; ix < n; ++ix)
    for (int iy = 0; iy < n; ++iy)
      for (int iz = 0; iz < n; ++iz)
        for (int b = 0; b < 8; ++b) {
          c.tau.push_back((ix + kBasis[b][0]) * a);
          c.tau.push_back((iy + kBasis[b][1]) * a);
          c.tau.push_back((iz + kBasis[b][2]) * a);
        }
  const int natom = 8 * n * n * n;
  for (int i = 0; i < natom; ++i) c.depth.push_back(-1.0 + 0.1 * (2.0 * uniform01(r.seed, i) - 1.0));
  for (int i = 0; i < 4 * natom; ++i) c.dkb.push_back(0.5 + uniform01(r.seed, natom + i));
  return c;
}

// smallest 2^a 3^b >= x
int smooth_at_least(double x) {
  long best = -1;
  for (long p2 = 1; p2 < 1L << 20; p2 *= 2)
    for (long p = p2; p < 1L << 20; p *= 3)
      if (p >= x && (best < 0 || p < best)) best = p;
  return (int)best;
}

}  // namespace

// Device-memory model of one request: cell (beta, V, tables, FFT scratch) +
// solver blocks (S, S2, HS, HS2 of npw x 3nb, P, HP, dense workspace) + the
// split-FP16 operands in mixed precision.  npw is estimated from the sphere
// volume (+3%).
extern "C" size_t pw_request_footprint(const pw_request *r, int precision) {
  if (!r || r->ncell < 1 || r->nbands < 1 || !(r->ecut > 0)) return 0;
  const double a = r->species == 1 ? 6.74 : 10.26;
  const double L = r->ncell * a;
  const double R = sqrt(2.0 * r->ecut) * L / (2.0 * M_PI);
  const double npw = 1.03 * 4.0 / 3.0 * M_PI * R * R * R + 64;
  const int N = smooth_at_least(1.5 * sqrt(2.0 * r->ecut) * L / M_PI);
  const double natom = 8.0 * r->ncell * r->ncell * r->ncell;
  const double nproj = 4 * natom, nb = r->nbands, n3 = 3 * nb;
  double b = npw * nproj * 16 + (double)N * N * N * 12 + npw * 40;        // cell
  b += 64.0 * 1048576;                                                     // FFT z-pencils (cap)
  b += (4 * npw * n3 + 2 * npw * nb) * 16;                                  // S, S2, HS, HS2, P, HP
  b += n3 * n3 * 16 * 6 + n3 * n3 * 8 * 3;                                  // G, A, dense workspace
  b += (double)pw_hs_bytes((int)n3);                                        // Householder digit slices
  if (precision == PW_MIXED)
    b += (npw * 2 * n3 * 2 * 3 + nproj * 2 * npw * 4 * 2) * 2.0;            // split operands
  return (size_t)(1.1 * b);
}

namespace {

std::atomic<unsigned long long> g_batch_launches{0}, g_batch_jobs{0};

// The local parts of H psi of concurrent requests that share a grid size,
// FFT plan and precision run in one launch per kernel (fft_reg.cuh
// run_multi).  A request thread that reaches its FFT becomes the leader for
// its key if none is gathering: it waits until every request solving with the
// same key has a job pending, or the window has passed, then launches all
// pending jobs of the key (at most PW_FFT_BATCH_MAX) on the batch stream,
// ordered after each job's stream (events) and before its continuation.
// Other threads wait until their job is done.  Every band's arithmetic is
// that of the one-cell launch, so results do not depend on the batching.
struct FftBatcher {
  typedef std::tuple<const pw_reg_plan *, int, int> Key;
  struct Job {
    pw_fft_job job;
    Key key;
    cudaStream_t st;
    bool taken;       // in a leader's launch (no longer pending)
    bool done;        // that launch is ordered on st; status set
    pw_status status;
  };
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Job *> pending;
  std::map<Key, bool> leading;
  std::map<Key, int> solving;   // requests solving with this key (expected participants)
  cudaStream_t bst = nullptr;
  double window_s = 100e-6;

  int count(const Key &k) const {
    int n = 0;
    for (const Job *j : pending) n += j->key == k;
    return n;
  }
  pw_status launch(const std::vector<Job *> &take) {
    const Job &j0 = *take[0];
    std::vector<pw_fft_job> jobs;
    for (const Job *t : take) {
      cudaEvent_t e;
      PW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      PW_CUDA(cudaEventRecord(e, t->st));
      PW_CUDA(cudaStreamWaitEvent(bst, e, 0));
      cudaEventDestroy(e);
      jobs.push_back(t->job);
    }
    const pw_reg_plan *plan = std::get<0>(j0.key);
    const int fp32 = std::get<1>(j0.key), cp = std::get<2>(j0.key);
    PW_TRY((fp32 ? plan->multi32[cp] : plan->multi64[cp])(jobs.data(), (int)jobs.size(), bst));
    cudaEvent_t done;
    PW_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    PW_CUDA(cudaEventRecord(done, bst));
    for (const Job *t : take) PW_CUDA(cudaStreamWaitEvent(t->st, done, 0));
    cudaEventDestroy(done);
    g_batch_launches.fetch_add(1);
    g_batch_jobs.fetch_add(take.size());
    return PW_OK;
  }
};

pw_status fft_hook(void *ctx, const pw_fft_job &job, const pw_reg_plan *plan, int fp32, int cp, cudaStream_t st) {
  FftBatcher &B = *(FftBatcher *)ctx;
  FftBatcher::Job me{job, FftBatcher::Key(plan, fp32, cp), st, false, false, PW_OK};
  std::unique_lock<std::mutex> lk(B.mu);
  B.pending.push_back(&me);
  B.cv.notify_all();
  for (;;) {
    if (me.done) return me.status;
    // a job another leader has taken waits for that launch, whatever the
    // leader flag says meanwhile
    if (!me.taken && !B.leading[me.key]) {
      B.leading[me.key] = true;
      const int want = std::min(PW_FFT_BATCH_MAX, std::max(1, B.solving[me.key]));
      const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(B.window_s);
      B.cv.wait_until(lk, deadline, [&] { return B.count(me.key) >= want; });
      // this job first, then the others of the key in arrival order
      std::vector<FftBatcher::Job *> take{&me};
      for (FftBatcher::Job *j : B.pending)
        if (j != &me && j->key == me.key && (int)take.size() < PW_FFT_BATCH_MAX) take.push_back(j);
      for (FftBatcher::Job *t : take) {
        B.pending.erase(std::find(B.pending.begin(), B.pending.end(), t));
        t->taken = true;
      }
      B.leading[me.key] = false;
      lk.unlock();
      const pw_status r = B.launch(take);
      lk.lock();
      for (FftBatcher::Job *t : take) {
        t->status = r;
        t->done = true;
      }
      B.cv.notify_all();
      continue;
    }
    B.cv.wait(lk, [&] { return me.done || (!me.taken && !B.leading[me.key]); });
  }
}

struct Job {
  int idx;
};

struct Server {
  const pw_serve_opts *opts;
  const pw_request *req;
  pw_result *res;
  int nreq;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> ready;        // admitted, waiting for a worker
  size_t in_use = 0;
  int running = 0;
  bool closing = false;
  std::chrono::steady_clock::time_point t0;
  // FFT plans tuned per grid (N0, N1, N2); a grid being tuned is marked with
  // L = -1 and later requests use the default plan meanwhile
  std::mutex plan_mu;
  std::map<std::array<int, 3>, pw_fft_plan> plans;
  FftBatcher batcher;           // used when opts->batch_fft
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

void run_one(Server &sv, int i, int device) {
  cudaSetDevice(device);
  const pw_request &r = sv.req[i];
  pw_result &out = sv.res[i];
  cudaStream_t st = nullptr;
  pw_status s = PW_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    out.status = PW_ERR_CUDA;
    return;
  }
  CellInputs ci = make_inputs(r);
  pw_cell_desc d;
  memset(&d, 0, sizeof d);
  d.lattice[0] = d.lattice[4] = d.lattice[8] = ci.L;
  d.natom = (int)ci.depth.size();
  d.tau = ci.tau.data();
  d.vdepth = ci.depth.data();
  d.vwidth = 1.2;
  d.pwidth = 1.2;
  d.dkb = ci.dkb.data();
  d.ecut = r.ecut;
  d.precision = sv.opts->precision;
  pw_cell *cell = nullptr;
  s = pw_setup_cell(&d, st, &cell);
  if (s == PW_OK && sv.opts->autotune) {
    const std::array<int, 3> g{cell->N[0], cell->N[1], cell->N[2]};
    bool tune = false, have = false;
    pw_fft_plan p{};
    {
      std::lock_guard<std::mutex> lk(sv.plan_mu);
      auto it = sv.plans.find(g);
      if (it == sv.plans.end()) {
        sv.plans[g] = pw_fft_plan{-1, 0, 0, 0};
        tune = true;
      } else if (it->second.L >= 0) {
        p = it->second;
        have = true;
      }
    }
    if (tune) {
      pw_fft_tune_report tr;
      s = pw_cell_autotune_fft(cell, r.nbands, sv.opts->precision, st, &tr);
      std::lock_guard<std::mutex> lk(sv.plan_mu);
      if (s == PW_OK) sv.plans[g] = tr.best;
      else sv.plans.erase(g);
    } else if (have) {
      s = pw_cell_set_fft_plan(cell, sv.opts->precision, &p);
    }
  }
  // the cell's mixed-precision FFTs join launches shared with other requests
  FftBatcher::Key key(nullptr, 1, 0);
  const bool batched = s == PW_OK && sv.opts->batch_fft && sv.opts->precision == PW_MIXED &&
                       pw_reg_plan_at(pw_cell_fft_plan(cell, 1)) != nullptr;
  if (batched) {
    key = FftBatcher::Key(pw_reg_plan_at(pw_cell_fft_plan(cell, 1)), 1, pw_cell_fft_compact(cell, 1));
    cell->fft_hook = fft_hook;
    cell->fft_hook_ctx = &sv.batcher;
    std::lock_guard<std::mutex> lk(sv.batcher.mu);
    sv.batcher.solving[key] += 1;
  }
  pw_solve_report rep;
  memset(&rep, 0, sizeof rep);
  if (s == PW_OK) {
    if (3 * r.nbands > cell->npw) {
      s = PW_ERR_ARG;
    } else {
      pw_solve_opts o;
      memset(&o, 0, sizeof o);
      o.nbands = r.nbands;
      o.tol = r.tol > 0 ? r.tol : (sv.opts->precision == PW_MIXED ? 5e-6 : 1e-8);
      o.maxit = r.maxit > 0 ? r.maxit : 300;
      o.seed = r.seed;
      o.precision = sv.opts->precision;
      s = pw_eigsolve(cell, &o, out.eig, nullptr, 0, &rep, st);
    }
  }
  if (batched) {
    std::lock_guard<std::mutex> lk(sv.batcher.mu);
    sv.batcher.solving[key] -= 1;
    sv.batcher.cv.notify_all();
  }
  out.iters = rep.iters;
  out.max_resid = rep.max_resid;
  out.orth_err = rep.orth_err;
  out.npw = cell ? cell->npw : 0;
  out.status = s;
  pw_destroy_cell(cell);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" void pw_fft_batch_stats(uint64_t *launches, uint64_t *jobs) {
  if (launches) *launches = g_batch_launches.load();
  if (jobs) *jobs = g_batch_jobs.load();
}

extern "C" pw_status pw_serve(const pw_serve_opts *opts, const pw_request *req, int nreq,
                              pw_result *res) {
  if (!opts || nreq < 0 || (nreq > 0 && (!req || !res)) || opts->max_slots < 1 ||
      (opts->precision != PW_FP64 && opts->precision != PW_MIXED))
    return PW_ERR_ARG;
  for (int i = 0; i < nreq; ++i)
    if (!res[i].eig || req[i].ncell < 1 || req[i].nbands < 1 || !(req[i].ecut > 0)) return PW_ERR_ARG;
  int device = 0;
  PW_CUDA(cudaGetDevice(&device));
  size_t budget = opts->hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    PW_CUDA(cudaMemGetInfo(&fr, &tot));
    budget = fr / 10 * 8;
  }
  Server sv;
  sv.opts = opts;
  if (opts->batch_fft) {
    PW_CUDA(cudaStreamCreateWithFlags(&sv.batcher.bst, cudaStreamNonBlocking));
    if (opts->batch_window_us > 0) sv.batcher.window_s = opts->batch_window_us * 1e-6;
  }
  sv.req = req;
  sv.res = res;
  sv.nreq = nreq;
  // arrival order
  std::vector<int> order(nreq);
  for (int i = 0; i < nreq; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return req[a].t_arrival < req[b].t_arrival; });
  std::vector<size_t> need(nreq);
  for (int i = 0; i < nreq; ++i) {
    need[i] = pw_request_footprint(&req[i], opts->precision);
    res[i].hbm_bytes = need[i];
    res[i].status = PW_OK;
    res[i].t_admit = res[i].t_done = res[i].latency = -1.0;
  }
  sv.t0 = std::chrono::steady_clock::now();
  // workers
  std::vector<std::thread> workers;
  for (int w = 0; w < opts->max_slots; ++w)
    workers.emplace_back([&sv, device, &need]() {
      for (;;) {
        int i;
        {
          std::unique_lock<std::mutex> lk(sv.mu);
          sv.cv.wait(lk, [&] { return sv.closing || !sv.ready.empty(); });
          if (sv.ready.empty()) return;
          i = sv.ready.front();
          sv.ready.pop_front();
        }
        run_one(sv, i, device);
        {
          std::lock_guard<std::mutex> lk(sv.mu);
          sv.res[i].t_done = sv.now();
          sv.res[i].latency = sv.res[i].t_done - sv.req[i].t_arrival;
          sv.in_use -= need[i];
          sv.running -= 1;
        }
        sv.cv.notify_all();
      }
    });
  // admission loop: FIFO in arrival order, a request waits for its arrival
  // time, a free slot and room under the budget (one larger than the whole
  // budget is refused with PW_ERR_BUSY)
  const double scale = opts->time_scale > 0 ? opts->time_scale : 1.0;
  for (int q = 0; q < nreq; ++q) {
    const int i = order[q];
    if (need[i] > budget) {
      std::lock_guard<std::mutex> lk(sv.mu);
      res[i].status = PW_ERR_BUSY;
      res[i].t_admit = res[i].t_done = sv.now();
      res[i].latency = 0.0;
      continue;
    }
    const double ta = req[i].t_arrival * scale;
    for (;;) {
      const double dt = ta - sv.now();
      if (dt <= 0) break;
      std::this_thread::sleep_for(std::chrono::duration<double>(std::min(dt, 0.05)));
    }
    std::unique_lock<std::mutex> lk(sv.mu);
    sv.cv.wait(lk, [&] { return sv.running < opts->max_slots && sv.in_use + need[i] <= budget; });
    sv.in_use += need[i];
    sv.running += 1;
    res[i].t_admit = sv.now();
    sv.ready.push_back(i);
    lk.unlock();
    sv.cv.notify_all();
  }
  {
    std::lock_guard<std::mutex> lk(sv.mu);
    sv.closing = true;
  }
  sv.cv.notify_all();
  for (auto &t : workers) t.join();
  if (sv.batcher.bst) {
    cudaStreamSynchronize(sv.batcher.bst);
    cudaStreamDestroy(sv.batcher.bst);
  }
  // latencies are measured against the (scaled) arrival time
  for (int i = 0; i < nreq; ++i)
    if (res[i].t_done >= 0 && res[i].status != PW_ERR_BUSY) res[i].latency = res[i].t_done - req[i].t_arrival * scale;
  return PW_OK;
}
