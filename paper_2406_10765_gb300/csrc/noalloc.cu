// H psi with no device allocation: every scratch byte comes from one
// fixed-size array compiled into the library.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// apply H -- for example a host framework that reserved the whole GPU for its
// own pool allocator at start-up (so a driver allocation would fail or
// fragment its pool), or a latency-critical loop that must not take the
// implicit device synchronisation cudaMalloc/cudaFree can cause.  pw_apply_H
// grows per-cell workspaces on demand; pw_apply_H_noalloc never does.
//
// The scratch is a file-scope __device__ array, so each GPU that loads the
// library holds PW_NOALLOC_SCRATCH_BYTES until the process exits.  Host code
// may not use the array's name as a device address: on first use on each
// device its address is looked up once with cudaGetSymbolAddress (with that
// device current) and cached.  Every call shares the array and leaves its
// contents behind; nothing in it needs to start at zero (each kernel writes
// every scratch element it later reads).  Calls that overlap on the GPU --
// on different streams, or from different host threads -- race on the array.
#include <mutex>

#include "pw_internal.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[PW_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

pw_status scratch_address(void **out) {
  int dev = -1;
  PW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return PW_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    PW_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PW_OK;
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

extern "C" pw_status pw_apply_H_noalloc(pw_cell *c, const void *psi, int ld, int nb, void *hpsi,
                                        void *stream) {
  if (!c || nb < 0) return PW_ERR_ARG;
  if (nb == 0) return PW_OK;
  if (!psi || !hpsi || ld < c->npw) return PW_ERR_ARG;
  if (c->proj_onthefly) return PW_ERR_ARG;   // regenerating beta needs a buffer
  // carve the scratch: projector coefficients B, GEMM partial sums, z-pencils
  // (a cell without atoms has no projectors and needs neither of the first two)
  const bool nonlocal = c->nproj > 0;
  const size_t b_bytes = nonlocal ? round_up((size_t)c->nproj * nb * sizeof(double2)) : 0;
  const size_t ws_elems = nonlocal ? std::max(pw_zgemm_ws_elems(c->nproj, nb, c->npw),
                                              pw_zgemm_ws_elems(c->npw, nb, c->nproj))
                                   : 0;
  const size_t ws_bytes = round_up(ws_elems * sizeof(double2));
  const size_t z_one = pw_local_zbytes_per_band(c);
  if (b_bytes + ws_bytes + z_one > (size_t)PW_NOALLOC_SCRATCH_BYTES) return PW_ERR_ARG;
  void *base = nullptr;
  PW_TRY(scratch_address(&base));
  unsigned char *p = (unsigned char *)base;
  double2 *B = (double2 *)p;
  double2 *ws = (double2 *)(p + b_bytes);
  void *zbuf = p + b_bytes + ws_bytes;
  const size_t zbytes = (size_t)PW_NOALLOC_SCRATCH_BYTES - b_bytes - ws_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  PW_TRY(pw_apply_local_fp64_into(c, (const double2 *)psi, ld, nb, (double2 *)hpsi, zbuf, zbytes, st));
  if (!nonlocal) return PW_OK;
  return pw_apply_nonlocal_fp64_into(c, (const double2 *)psi, ld, nb, (double2 *)hpsi, B, ws,
                                     ws_elems, st);
}
