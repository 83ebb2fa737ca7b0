// H psi = kinetic + local (FFT, fft_h.cu) + nonlocal Kleinman-Bylander term.
//
// Nonlocal term (Sec. III-A): the paper applies each atom's pseudopotential
// to every local wavefunction once it is fetched; on one GPU all atoms are
// resident, so the per-atom loop becomes two dense contractions over all
// projectors at once:  B = beta^H psi  (nproj x nb), B <- D o B,
// H psi += beta B.
#include "pw_internal.cuh"

namespace {
__global__ void k_scale_rows(double2 *B, int nproj, int nb, const double *D) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)nproj * nb) return;
  const double d = D[idx % nproj];
  B[idx].x *= d;
  B[idx].y *= d;
}
}  // namespace

pw_status pw_apply_nonlocal(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                            int precision, cudaStream_t st) {
  (void)precision;
  if (c->nproj == 0 || nb == 0) return PW_OK;
  size_t need = (size_t)c->nproj * nb * sizeof(double2);
  size_t cur = c->B_elems * sizeof(double2);
  PW_TRY(pw_ensure((void **)&c->d_B, &cur, need));
  c->B_elems = cur / sizeof(double2);
  size_t ws = std::max(pw_zgemm_ws_elems(c->nproj, nb, c->npw), pw_zgemm_ws_elems(c->npw, nb, c->nproj));
  size_t wcur = c->gemm_ws_elems * sizeof(double2);
  PW_TRY(pw_ensure((void **)&c->d_gemm_ws, &wcur, ws * sizeof(double2)));
  c->gemm_ws_elems = wcur / sizeof(double2);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  PW_TRY(pw_zgemm('C', 'N', c->nproj, nb, c->npw, one, c->d_beta, c->npw, psi, ld, zero, c->d_B,
                  c->nproj, c->d_gemm_ws, c->gemm_ws_elems, st));
  k_scale_rows<<<(unsigned)(((long)c->nproj * nb + 255) / 256), 256, 0, st>>>(c->d_B, c->nproj, nb, c->d_D);
  PW_TRY(pw_check_launch("scale_rows"));
  return pw_zgemm('N', 'N', c->npw, nb, c->nproj, one, c->d_beta, c->npw, c->d_B, c->nproj, one,
                  hpsi, ld, c->d_gemm_ws, c->gemm_ws_elems, st);
}

extern "C" pw_status pw_apply_H(pw_cell *c, const void *psi, int ld, int nb, void *hpsi,
                                void *stream) {
  if (!c || nb < 0) return PW_ERR_ARG;
  if (nb == 0) return PW_OK;
  if (!psi || !hpsi || ld < c->npw) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  PW_TRY(pw_apply_local(c, (const double2 *)psi, ld, nb, (double2 *)hpsi, c->precision, st));
  return pw_apply_nonlocal(c, (const double2 *)psi, ld, nb, (double2 *)hpsi, c->precision, st);
}
