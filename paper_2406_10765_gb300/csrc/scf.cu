// Self-consistent field outer loop with a model V_Hxc (the loop of Sec. II-A
// that wraps the eigensolver; the paper fixes no exchange-correlation
// functional, so the model is the periodic Hartree potential plus Slater /
// Dirac exchange):
//   n(r) = Omega^-1 sum_b f_b |psi_b(r)|^2                  (pw_density / Omega)
//   V_H: lap V_H = -4 pi (n - <n>), V_H(G) = 4 pi n(G) / |G|^2, V_H(0) = 0
//   v_x = -(3 n / pi)^(1/3)
//   V = V_loc + V_H + v_x;   n_in <- (1 - mix) n_in + mix n_out
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "pw_internal.cuh"

namespace {

__global__ void k_real_to_grid(const double *__restrict__ n, long npts, double2 *__restrict__ g) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < npts) g[i] = make_double2(n[i], 0.0);
}

// g(k) <- 4 pi g(k) / (N^3 |G_k|^2), G = 2 pi k / L with signed k; 0 at k = 0
__global__ void k_poisson(double2 *__restrict__ g, int N0, int N1, int N2, double L0, double L1, double L2) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long npts = (long)N0 * N1 * N2;
  if (i >= npts) return;
  int kx = (int)(i % N0), ky = (int)((i / N0) % N1), kz = (int)(i / ((long)N0 * N1));
  if (2 * kx > N0) kx -= N0;
  if (2 * ky > N1) ky -= N1;
  if (2 * kz > N2) kz -= N2;
  const double two_pi = 6.283185307179586476925;
  const double gx = two_pi * kx / L0, gy = two_pi * ky / L1, gz = two_pi * kz / L2;
  const double g2 = gx * gx + gy * gy + gz * gz;
  const double f = g2 > 0.0 ? 4.0 * 3.141592653589793238463 / ((double)npts * g2) : 0.0;
  g[i] = make_double2(g[i].x * f, g[i].y * f);
}

// v = Re V_H + v_x(n)
__global__ void k_hxc_finish(const double2 *__restrict__ g, const double *__restrict__ n, long npts,
                             double *__restrict__ v) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double nn = fmax(n[i], 0.0);
  v[i] = g[i].x - cbrt(3.0 * nn / 3.141592653589793238463);
}

// V = V0 + add (add may be NULL), and its FP32 copy
__global__ void k_set_v(const double *__restrict__ V0, const double *__restrict__ add, long npts,
                        double *__restrict__ V, float *__restrict__ Vf) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double v = V0[i] + (add ? add[i] : 0.0);
  V[i] = v;
  Vf[i] = (float)v;
}

// n_out = rho / Omega in place; per-block max |n_out - n_in|
__global__ void k_scf_diff(double *__restrict__ nout, const double *__restrict__ nin, long npts,
                           double inv_omega, double *__restrict__ bmax) {
  __shared__ double sh[32];
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double d = 0.0;
  if (i < npts) {
    const double v = nout[i] * inv_omega;
    nout[i] = v;
    d = fabs(v - nin[i]);
  }
  for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x < 32) {
    d = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    if (threadIdx.x == 0) bmax[blockIdx.x] = d;
  }
}

__global__ void k_mix(double *__restrict__ nin, const double *__restrict__ nout, long npts, double mix) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < npts) nin[i] = (1.0 - mix) * nin[i] + mix * nout[i];
}

unsigned blocks(long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

extern "C" pw_status pw_hxc_potential(pw_cell *c, const double *n, double *v, void *stream) {
  if (!c || !n || !v) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long npts = (long)c->N[0] * c->N[1] * c->N[2];
  PW_TRY(pw_ensure((void **)&c->d_grid, &c->grid_bytes, npts * sizeof(double2)));
  pw_count_launch();
  k_real_to_grid<<<blocks(npts), 256, 0, st>>>(n, npts, c->d_grid);
  PW_TRY(pw_grid_fft(c, c->d_grid, 0, st));
  pw_count_launch();
  k_poisson<<<blocks(npts), 256, 0, st>>>(c->d_grid, c->N[0], c->N[1], c->N[2], c->L[0], c->L[1], c->L[2]);
  PW_TRY(pw_grid_fft(c, c->d_grid, 1, st));
  pw_count_launch();
  k_hxc_finish<<<blocks(npts), 256, 0, st>>>(c->d_grid, n, npts, v);
  return pw_check_launch("hxc potential");
}

extern "C" pw_status pw_cell_set_hxc(pw_cell *c, const double *v_hxc, void *stream) {
  if (!c) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long npts = (long)c->N[0] * c->N[1] * c->N[2];
  if (!c->d_V0) {
    if (!v_hxc) return PW_OK;                 // already the cell's own V_loc
    if (cudaMalloc(&c->d_V0, npts * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->d_V0 = nullptr;
      return PW_ERR_OOM;
    }
    PW_CUDA(cudaMemcpyAsync(c->d_V0, c->d_V, npts * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  pw_count_launch();
  k_set_v<<<blocks(npts), 256, 0, st>>>(c->d_V0, v_hxc, npts, c->d_V, c->d_Vf);
  return pw_check_launch("set potential");
}

extern "C" pw_status pw_scf(pw_cell *c, const pw_scf_opts *o, double *eig, double *n_out, pw_scf_report *rep,
                            void *stream) {
  if (!c || !o || !eig || o->nocc < 1 || o->nbands < o->nocc || !(o->mix > 0.0) || o->mix > 1.0 ||
      o->maxiter < 1)
    return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long npts = (long)c->N[0] * c->N[1] * c->N[2];
  const double omega = c->L[0] * c->L[1] * c->L[2];
  const int nb = o->nbands, npw = c->npw;
  double *nin = nullptr, *nout = nullptr, *vhxc = nullptr, *bmax = nullptr, *occ = nullptr;
  void *X = nullptr;
  const unsigned nblk = blocks(npts);
  auto cleanup = [&]() {
    void *ptrs[] = {nin, nout, vhxc, bmax, occ, X};
    for (void *p : ptrs)
      if (p) cudaFree(p);
  };
  if (cudaMalloc(&nin, npts * 8) != cudaSuccess || cudaMalloc(&nout, npts * 8) != cudaSuccess ||
      cudaMalloc(&vhxc, npts * 8) != cudaSuccess || cudaMalloc(&bmax, nblk * 8) != cudaSuccess ||
      cudaMalloc(&occ, nb * 8) != cudaSuccess || cudaMalloc(&X, (size_t)npw * nb * 16) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return PW_ERR_OOM;
  }
  std::vector<double> occ_h(nb, 0.0);
  for (int j = 0; j < o->nocc; ++j) occ_h[j] = o->fill;
  pw_status r = PW_OK;
  if (cudaMemcpyAsync(occ, occ_h.data(), nb * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(nin, 0, npts * 8, st) != cudaSuccess)
    r = PW_ERR_CUDA;
  std::vector<double> bm(nblk);
  double dn = 0.0;
  int it = 0, eig_iters = 0;
  bool conv = false;
  for (; r == PW_OK && it < o->maxiter; ++it) {
    // V = V_loc + V_Hxc[n_in]
    if ((r = pw_hxc_potential(c, nin, vhxc, st)) != PW_OK) break;
    if ((r = pw_cell_set_hxc(c, vhxc, st)) != PW_OK) break;
    // eigenpairs of this H, started from the previous block
    pw_solve_opts so = {};
    so.nbands = nb;
    so.tol = o->eig_tol;
    so.maxit = o->eig_maxit;
    so.seed = o->seed;
    so.x0 = it > 0 ? X : nullptr;
    so.precision = o->precision;
    if (cudaStreamSynchronize(st) != cudaSuccess) { r = PW_ERR_CUDA; break; }
    pw_solve_report sr;
    r = pw_eigsolve(c, &so, eig, X, npw, &sr, st);
    eig_iters += sr.iters;
    if (r == PW_ERR_NOCONV) r = PW_OK;         // the next SCF iteration continues from this block
    if (r != PW_OK) break;
    // n_out and max |n_out - n_in|
    if ((r = pw_density(c, X, npw, nb, occ, nout, st)) != PW_OK) break;
    pw_count_launch();
    k_scf_diff<<<nblk, 256, 0, st>>>(nout, nin, npts, 1.0 / omega, bmax);
    if ((r = pw_check_launch("scf diff")) != PW_OK) break;
    if (cudaMemcpyAsync(bm.data(), bmax, nblk * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      r = PW_ERR_CUDA;
      break;
    }
    dn = *std::max_element(bm.begin(), bm.end());
    if (dn <= o->tol) { conv = true; ++it; break; }
    pw_count_launch();
    k_mix<<<nblk, 256, 0, st>>>(nin, nout, npts, o->mix);
  }
  if (r == PW_OK && n_out)
    if (cudaMemcpyAsync(n_out, nout, npts * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) r = PW_ERR_CUDA;
  if (rep) {
    rep->iters = it;
    rep->eig_iters = eig_iters;
    rep->max_dn = dn;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && r == PW_OK) r = PW_ERR_CUDA;
  cleanup();
  if (r != PW_OK) return r;
  return conv ? PW_OK : PW_ERR_NOCONV;
}
