// Electron density on the FFT grid from a block of bands:
//   rho(r_j) = sum_b w_b |psi_b(r_j)|^2,  psi_b(r_j) = sum_G c_bG exp(i G.r_j)
// (the density that the self-consistent loop of Sec. II-A forms from the
// converged wavefunctions; the paper names the step, not its arithmetic).
// Bands go through the local-part machinery in L2-sized batches: z-pencils
// (K1), then per (z-plane, band group) the inverse plane FFTs and the weighted
// |psi|^2 sum in fixed per-thread points; the group sums are added in a fixed
// order, so the result does not depend on scheduling.
#include "pw_internal.cuh"

namespace {

// rho[i] (+)= sum_g part[g][i], groups in order
__global__ void k_density_reduce(const double *__restrict__ part, int ngroups, long npts, int accumulate,
                                 double *__restrict__ rho) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  double s = accumulate ? rho[i] : 0.0;
  for (int g = 0; g < ngroups; ++g) s += part[g * npts + i];
  rho[i] = s;
}

}  // namespace

extern "C" pw_status pw_density(pw_cell *c, const void *psi, int ld, int nb, const double *occ, double *rho,
                                void *stream) {
  if (!c || nb < 0 || !rho) return PW_ERR_ARG;
  if (nb > 0 && (!psi || ld < c->npw)) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long npts = (long)c->N[0] * c->N[1] * c->N[2];
  if (nb == 0) {
    PW_CUDA(cudaMemsetAsync(rho, 0, npts * sizeof(double), st));
    return PW_OK;
  }
  const int fp32 = c->precision == PW_MIXED;
  const size_t csize = fp32 ? sizeof(float2) : sizeof(double2);
  const size_t per_band = (size_t)c->N[2] * c->ncol * csize;
  // z-pencils of an L2-sized batch of bands (the cell's batch size, default ~64 MB)
  const int batch =
      (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, pw_cell_fft_batch_bytes(c, fp32) / per_band));
  PW_TRY(pw_ensure(&c->d_z, &c->z_bytes, per_band * batch));
  // enough (z-plane, group) blocks for two per SM
  const int ngroups = std::max(1, std::min(8, (2 * 152 + c->N[2] - 1) / c->N[2]));
  PW_TRY(pw_ensure((void **)&c->d_dpart, &c->dpart_bytes, (size_t)ngroups * npts * sizeof(double)));
  const pw_reg_plan *reg = pw_reg_plan_at(pw_cell_fft_plan(c, fp32));
  for (int b0 = 0; b0 < nb; b0 += batch) {
    const int nbb = std::min(batch, nb - b0);
    const double2 *p = (const double2 *)psi + (long)b0 * ld;
    const double *w = occ ? occ + b0 : nullptr;
    const int g = std::min(ngroups, nbb);
    if (reg) PW_TRY((fp32 ? reg->dens32 : reg->dens64)(c, p, ld, nbb, c->d_z, w, g, c->d_dpart, st));
    else PW_TRY(pw_fft_density_batch(c, p, ld, nbb, c->d_z, fp32, w, g, c->d_dpart, st));
    pw_count_launch();
    k_density_reduce<<<(unsigned)((npts + 255) / 256), 256, 0, st>>>(c->d_dpart, g, npts, b0 > 0, rho);
  }
  return pw_check_launch("density");
}
