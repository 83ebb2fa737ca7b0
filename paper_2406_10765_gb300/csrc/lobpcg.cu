// LOBPCG block eigensolver (Knyazev 2001) for H X = X Lambda (Sec. II-A,
// Eq. 1), one of the inner eigensolvers the paper names (Sec. II-A).
//
// One step:
//   R = H X - X Lambda, column norms (FP64, deterministic block reductions);
//   active set: bands with ||r|| > tol stay active (once locked, locked);
//   W = K(R_act), K the Teter-Payne-Allan ratio on 1/2|G|^2 / E_kin(band);
//   H W (the FFT + projector operator, hamiltonian.cu);
//   S = [X, W, P_act], Gram G = S^H S and A = S^H (H S) (Sec. II-B row scheme);
//   Rayleigh-Ritz in FP64 (dense.cu): Jacobi-scaled Cholesky (a failing pivot
//   drops P and retries), Hermitian eigensolve (Syevd, Sec. III-D);
//   X' = S C, P' = [0, W, P_act] C (Hetmaniuk-Lehoucq), and the matching H
//   blocks, so H is applied once per step.
//
// Device layout: S and H S are npw x 3nb complex128 column blocks [X | W | P]
// (ld = npw), ping-ponged between two buffers; P and H P (npw x nb) keep all
// nb columns.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "dense.cuh"
#include "oz_gemm.cuh"
#include "pw_internal.cuh"
#include "tc_gemm.cuh"

struct pw_solver {
  pw_cell *cell = nullptr;
  int nb = 0, npw = 0, maxit = 0, precision = PW_FP64;
  double tol = 0.0;
  cudaStream_t st = nullptr;
  double2 *S = nullptr, *S2 = nullptr, *HS = nullptr, *HS2 = nullptr, *P = nullptr, *HP = nullptr;
  double2 *G = nullptr, *A = nullptr, *C = nullptr;
  double *lam = nullptr, *theta = nullptr, *stats = nullptr;
  int *act = nullptr;
  double2 *gws = nullptr; size_t gws_elems = 0;
  bool haveP = false;
  std::vector<char> active;
  std::vector<double> lam_h, resid_h;
  int iter = 0, dropped = 0;
  pw_dense_ws dws;
  pw_oz_ws oz;               // FP64-accurate tensor-core products of the tall FP64 blocks
  size_t bytes = 0;
  cudaEvent_t ev[12] = {};   // stage boundaries of the last step (7-10: H X and H P)
  int hx_applied = 0;        // H X was recomputed in the last refresh
  // mixed precision: split-FP16 operands of S, H S and the coefficients
  pw_tc_operand opSA, opSB, opST, opHST, opC, opCP, opM;
  double2 *Mx = nullptr;     // mixed: d o L^-H of the current Gram (3nb x 3nb)
  bool st_split_valid = false;   // opST holds the split of the current S
  int chunk_rows = 0;            // rows per chunk of the tall split products (0: automatic)
  float *rmax = nullptr;
  int *d_err = nullptr;
  // mixed precision applies H to the whole basis [X W P] every step instead of
  // carrying H X and H P through the rotations (their split-precision errors
  // would be amplified by ill-conditioned coefficients near convergence)
  bool fresh_h = false;
  // mixed precision with fresh H: the Rayleigh-Ritz left Y in the dense
  // workspace and S~ = S M in S2, and the rotation writes X' = S~ Y to HS2
  bool ytilde = false, x_in_hs2 = false;
  bool xh_swapped = false;        // carried rotation left X' in HS and H X' in S
  bool hst_split_valid = false;   // opHST holds the split of the current H S
  bool hx_valid = true;    // HS[:, 0:nb] == H X for the current X
  // mixed precision: 0 recompute H X and H P every step; 1 carry them
  // through the rotations while the largest residual is above kCarryTol,
  // then recompute; 2 always carry
  int h_blocks = 0;
};

// Residual level below which the mixed solve stops carrying H X and H P
// through the split-precision rotations and applies H to [X W P] afresh: the
// carried blocks hold the split products' error (~1e-6 of |HS| |C|, larger
// when the basis is ill-conditioned near convergence), harmless against
// residuals well above it.
constexpr double kCarryTol = 1e-3;

namespace {

__device__ __forceinline__ double bsum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// per column j: |HX_j - lam_j X_j|^2, sum kin |x|^2, sum |x|^2
__global__ void __launch_bounds__(256) k_stats(const double2 *X, const double2 *HX, int ld, int npw,
                                               const double *lam, const double *kin, double *stats,
                                               int nb) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const double l = lam[j];
  const double2 *x = X + (long)j * ld, *hx = HX + (long)j * ld;
  double r2 = 0.0, kx = 0.0, x2 = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 a = x[g], h = hx[g];
    const double rx = h.x - l * a.x, ry = h.y - l * a.y;
    const double aa = a.x * a.x + a.y * a.y;
    r2 += rx * rx + ry * ry;
    kx += kin[g] * aa;
    x2 += aa;
  }
  r2 = bsum(r2, sh);
  kx = bsum(kx, sh);
  x2 = bsum(x2, sh);
  if (threadIdx.x == 0) {
    stats[j] = r2;
    stats[nb + j] = kx;
    stats[2 * nb + j] = x2;
  }
}

// W[:, a] = K(kin / E_kin(j)) (HX_j - lam_j X_j), j = act[a]
// f32k: the preconditioner factor in FP32 (mixed precision; it only shapes the
// search direction, and FP64 divisions are scarce on this part)
__global__ void k_precond(const double2 *X, const double2 *HX, int ld, int npw, const double *lam,
                          const double *kin, const double *stats, int nb, const int *act, int k,
                          double2 *W, int f32k) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)npw * k) return;
  const int g = (int)(idx % npw), a = (int)(idx / npw);
  const int j = act[a];
  double K;
  if (f32k) {
    const float x = (float)kin[g] * ((float)stats[2 * nb + j] / (float)stats[nb + j]);
    const float p = 27.0f + x * (18.0f + x * (12.0f + 8.0f * x));
    K = (double)(p / (p + 16.0f * x * x * x * x));
  } else {
    const double ek = stats[nb + j] / stats[2 * nb + j];
    const double x = kin[g] / ek;
    const double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
    K = p / (p + 16.0 * x * x * x * x);
  }
  const double2 xv = X[g + (long)j * ld], h = HX[g + (long)j * ld];
  const double l = lam[j];
  W[g + (long)a * ld] = make_double2(K * (h.x - l * xv.x), K * (h.y - l * xv.y));
}

// scale each column of X (and of HX, if given) to unit 2-norm of X's column;
// zero columns are left unchanged
__global__ void __launch_bounds__(256) k_normalize_cols(double2 *X, double2 *HX, int ld, int npw) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double2 *x = X + (long)j * ld;
  double s2 = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s2 += x[g].x * x[g].x + x[g].y * x[g].y;
  s2 = bsum(s2, sh);
  if (!(s2 > 0.0)) return;
  const double f = 1.0 / sqrt(s2);
  for (int g = threadIdx.x; g < npw; g += blockDim.x) { x[g].x *= f; x[g].y *= f; }
  if (HX) {
    double2 *h = HX + (long)j * ld;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) { h[g].x *= f; h[g].y *= f; }
  }
}

// dst[:, a] = src[:, act[a]]
__global__ void k_gather_cols(const double2 *src, int ld, int npw, const int *act, int k,
                              double2 *dst) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)npw * k) return;
  const int g = (int)(idx % npw), a = (int)(idx / npw);
  dst[g + (long)a * ld] = src[g + (long)act[a] * ld];
}

// random start: entry (g, j) = (u1 - 1/2) + i (u2 - 1/2), counters 5 natom + 2 (j npw + g) (+1)
__global__ void k_random_block(double2 *X, int ld, int npw, int nb, uint64_t seed, uint64_t base) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)npw * nb) return;
  const int g = (int)(idx % npw), j = (int)(idx / npw);
  const uint64_t c = base + 2ull * ((uint64_t)j * npw + g);
  const double u1 = (double)(splitmix64(seed, c) >> 11) * 0x1.0p-53;
  const double u2 = (double)(splitmix64(seed, c + 1) >> 11) * 0x1.0p-53;
  X[g + (long)j * ld] = make_double2(u1 - 0.5, u2 - 0.5);
}

// max |G_ij - delta_ij| of an n x n matrix (single CTA)
__global__ void k_orth_err(const double2 *G, int n, double *out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (long idx = threadIdx.x; idx < (long)n * n; idx += blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    const double2 g = G[idx];
    const double re = g.x - (i == j ? 1.0 : 0.0);
    m = fmax(m, sqrt(re * re + g.y * g.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, sh[q]);
    *out = r;
  }
}

pw_status alloc(void **p, size_t bytes, size_t *acc) {
  if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return PW_ERR_OOM; }
  *acc += bytes;
  return PW_OK;
}

const double2 kOne = {1.0, 0.0}, kZero = {0.0, 0.0};

// run H on ncols columns with the solver's precision
pw_status solver_apply_H(pw_solver *s, const double2 *x, double2 *hx, int ncols) {
  pw_cell *c = s->cell;
  const int saved = c->precision;
  c->precision = s->precision;
  pw_status r = pw_apply_H(c, x, s->npw, ncols, hx, s->st);
  c->precision = saved;
  return r;
}

pw_status gemm(pw_solver *s, char oa, char ob, int m, int n, int k, const double2 *A, int lda,
               const double2 *B, int ldb, double2 beta, double2 *C, int ldc) {
  const size_t need = pw_zgemm_ws_elems(m, n, k);
  if (need > s->gws_elems) {
    size_t cur = s->gws_elems * 16;
    PW_TRY(pw_ensure((void **)&s->gws, &cur, need * 16));
    s->gws_elems = cur / 16;
  }
  return pw_gemm64(&s->oz, oa, ob, m, n, k, kOne, A, lda, B, ldb, beta, C, ldc, s->gws, s->gws_elems, s->st);
}

// Cholesky pivot threshold of the Jacobi-scaled Gram: FP64 products are exact
// to ~1e-16, the split-FP16 products to ~1e-8, so pivots below 1e-6 carry no
// information in mixed precision.
double piv_tol(const pw_solver *s) { return s->precision == PW_MIXED ? 1e-6 : 1e-14; }

// Plane-wave rows per chunk of the tall split-FP16 operands: the largest
// chunk operand (2 ns rows x 2 ng K, two FP16 slices) stays under ~8 GB, so
// the 1,728-atom cell fits in HBM; smaller cells take one chunk.
int tall_chunk(const pw_solver *s, int ns) {
  if (s->chunk_rows > 0) return std::min(s->chunk_rows, s->npw);
  const size_t cap = (size_t)8 << 30;
  size_t ng = cap / ((size_t)2 * ns * 2 * 2 * 2);
  ng = std::max<size_t>(1024, ng / 64 * 64);
  return (int)std::min<size_t>(ng, (size_t)s->npw);
}

// C (ns x ns, ld ldc, Hermitian) = X^H Y over the plane-wave rows, chunk by
// chunk, accumulated in FP64 (opSA, opSB as scratch)
pw_status tall_gram(pw_solver *s, const double2 *X, const double2 *Y, int ns, double2 *C, int ldc) {
  const int npw = s->npw, gc = tall_chunk(s, ns);
  for (int g0 = 0; g0 < npw; g0 += gc) {
    const int ng = std::min(gc, npw - g0);
    PW_TRY(pw_tc_operand_alloc(&s->opSA, 2 * ns, 2 * ng, s->st));
    PW_TRY(pw_tc_operand_alloc(&s->opSB, ns, 2 * ng, s->st));
    PW_TRY(pw_tc_split_rows(X + g0, npw, ng, ns, 1, nullptr, &s->opSA, s->st));
    PW_TRY(pw_tc_split_rows(Y + g0, npw, ng, ns, 0, nullptr, &s->opSB, s->st));
    PW_TRY(pw_tc_gemm(&s->opSA, 2 * ns, &s->opSB, ns, C, ldc, 0, g0 > 0, 1, s->d_err, s->st));
  }
  return PW_OK;
}

// out (npw rows, ld npw) = X (npw x ns) times the split coefficients coef,
// row chunk by row chunk; X's rows are split into op (skipped when op already
// holds the split of all of X).  coef2 (optional): out2 = X coef2 from the
// same split chunk.
pw_status tall_times_coef(pw_solver *s, const double2 *X, int ns, pw_tc_operand *op, bool presplit,
                          const pw_tc_operand *coef, int ncols2, double2 *out, int kb_lo, int tri,
                          const pw_tc_operand *coef2 = nullptr, double2 *out2 = nullptr, int kb_lo2 = 0) {
  const int npw = s->npw, gc = tall_chunk(s, ns);
  for (int g0 = 0; g0 < npw; g0 += gc) {
    const int ng = std::min(gc, npw - g0);
    if (!(presplit && gc >= npw)) {
      PW_TRY(pw_tc_operand_alloc(op, ng, 2 * ns, s->st));
      PW_TRY(pw_tc_split_trans(X + g0, npw, ng, ns, s->rmax, op, s->st));
    }
    PW_TRY(pw_tc_gemm(op, ng, coef, ncols2, out + g0, npw, 1, 0, 0, s->d_err, s->st, kb_lo, tri));
    if (coef2)
      PW_TRY(pw_tc_gemm(op, ng, coef2, ncols2, out2 + g0, npw, 1, 0, 0, s->d_err, s->st, kb_lo2));
  }
  return PW_OK;
}

// Mixed precision: from the Gram in s->G (order ns), factor G in FP64
// (scaling, Cholesky, L^-1, M = d L^-H), orthonormalise the basis on the
// tensor cores (S~ = S M, H S~ = H S M into S2, HS2), form A~ = S~^H H S~
// there too, and finish in FP64 (eigensolve, C = M Y).
pw_status rr_mixed_from_gram(pw_solver *s, int ns, int *chol_ok) {
  const int npw = s->npw, nb = s->nb, ldg = 3 * nb;
  s->hst_split_valid = false;
  PW_TRY(pw_rr_factor(&s->dws, ns, s->G, ldg, s->Mx, ldg, chol_ok, s->st, piv_tol(s)));
  if (!*chol_ok) return PW_OK;
  PW_TRY(pw_tc_operand_alloc(&s->opM, 2 * ns, 2 * ns, s->st));
  PW_TRY(pw_tc_split_coef(s->Mx, ldg, ns, ns, nullptr, &s->opM, s->st));
  // S~ = S M, H S~ = HS M; M is upper triangular: output columns j need K rows t <= j only
  PW_TRY(tall_times_coef(s, s->S, ns, &s->opST, false, &s->opM, 2 * ns, s->S2, 0, 1));
  s->st_split_valid = tall_chunk(s, ns) >= npw;   // opST holds the split of all of S
  PW_TRY(tall_times_coef(s, s->HS, ns, &s->opHST, false, &s->opM, 2 * ns, s->HS2, 0, 1));
  s->hst_split_valid = tall_chunk(s, ns) >= npw;  // opHST holds the split of all of H S
  // A~ = S~^H (H S~)
  PW_TRY(tall_gram(s, s->S2, s->HS2, ns, s->A, ldg));
  // X' = S~ Y (and H X' = H S~ Y) on the tensor cores; only the P part of
  // C = M Y in FP64
  s->ytilde = true;
  return pw_rr_finish_tall(&s->dws, ns, nb, s->A, ldg, s->Mx, ldg, s->theta, s->C, ldg, s->st);
}

// Rayleigh-Ritz on the first ns columns of (S, HS) -> theta, C (ns x nb, ld 3nb).
// Events ev[3] / ev[4] bracket the Gram products.
pw_status subspace_rr(pw_solver *s, int ns, int *chol_ok) {
  const int ldg = 3 * s->nb;
  cudaEventRecord(s->ev[3], s->st);
  if (s->precision == PW_MIXED) {
    PW_TRY(tall_gram(s, s->S, s->S, ns, s->G, ldg));
    cudaEventRecord(s->ev[4], s->st);
    return rr_mixed_from_gram(s, ns, chol_ok);
  }
  // Hermitian products: upper-triangle tiles, mirrored
  const size_t need = pw_zgemm_ws_elems(ns, ns, s->npw);
  if (need > s->gws_elems) {
    size_t cur = s->gws_elems * 16;
    PW_TRY(pw_ensure((void **)&s->gws, &cur, need * 16));
    s->gws_elems = cur / 16;
  }
  PW_TRY(pw_gemm64(&s->oz, 'C', 'N', ns, ns, s->npw, kOne, s->S, s->npw, s->S, s->npw, kZero, s->G, ldg, s->gws,
                   s->gws_elems, s->st, 1));
  PW_TRY(pw_gemm64(&s->oz, 'C', 'N', ns, ns, s->npw, kOne, s->S, s->npw, s->HS, s->npw, kZero, s->A, ldg,
                   s->gws, s->gws_elems, s->st, 1));
  cudaEventRecord(s->ev[4], s->st);
  return pw_rayleigh_ritz(&s->dws, ns, s->nb, s->G, ldg, s->A, ldg, s->theta, s->C, ldg, chol_ok, s->st,
                          piv_tol(s));
}

// after a rotation the new block becomes S (and HS): X' sits in S2 (H X' in
// HS2), or, after the tensor-core S~ Y rotation, in HS2
void swap_rotated(pw_solver *s) {
  if (s->xh_swapped) {
    std::swap(s->S, s->HS);
    s->xh_swapped = false;
  } else if (s->x_in_hs2) {
    std::swap(s->S, s->HS2);
    s->x_in_hs2 = false;
  } else {
    std::swap(s->S, s->S2);
    std::swap(s->HS, s->HS2);
  }
}

// X' = S C and H X' = HS C into S2, HS2; with_p: P' = S C_P, HP' = HS C_P
// where C_P is C with its first nb rows zeroed (the [0, W, P] combination)
pw_status rotate(pw_solver *s, int ns, bool with_p) {
  const int npw = s->npw, nb = s->nb, n3 = 3 * nb;
  if (s->precision == PW_MIXED && s->ytilde) {
    s->ytilde = false;
    PW_TRY(pw_tc_operand_alloc(&s->opC, 2 * nb, 2 * ns, s->st));
    if (with_p) {
      // P' = S C_P, C_P = C with its first nb rows zero (opST may still hold
      // the split of S); the first nb coefficient rows are zero: skip their K blocks
      PW_TRY(pw_tc_operand_alloc(&s->opCP, 2 * nb, 2 * ns, s->st));
      PW_TRY(pw_tc_split_coef(s->C, n3, ns, nb, nullptr, &s->opCP, s->st));
      PW_TRY(tall_times_coef(s, s->S, ns, &s->opST, s->st_split_valid, &s->opCP, 2 * nb, s->P,
                             (2 * nb) / 64, 0));
      // carried H blocks: H P' = H S C_P (opHST may still hold the split of H S)
      if (!s->fresh_h)
        PW_TRY(tall_times_coef(s, s->HS, ns, &s->opHST, s->hst_split_valid, &s->opCP, 2 * nb, s->HP,
                               (2 * nb) / 64, 0));
    }
    PW_TRY(pw_tc_split_coef(s->dws.Y, ns, ns, nb, nullptr, &s->opC, s->st));
    s->st_split_valid = false;
    s->hst_split_valid = false;
    if (!s->fresh_h) {
      // X' = S~ Y into HS and H X' = H S~ Y into S (both consumed above); the
      // swap that follows makes them the new S and H S
      PW_TRY(tall_times_coef(s, s->S2, ns, &s->opST, false, &s->opC, 2 * nb, s->HS, 0, 0));
      PW_TRY(tall_times_coef(s, s->HS2, ns, &s->opHST, false, &s->opC, 2 * nb, s->S, 0, 0));
      s->xh_swapped = true;
      return PW_OK;
    }
    // X' = S~ Y into HS2 (H S~ is no longer needed)
    PW_TRY(tall_times_coef(s, s->S2, ns, &s->opST, false, &s->opC, 2 * nb, s->HS2, 0, 0));
    s->x_in_hs2 = true;
    return PW_OK;
  }
  if (with_p && ns > nb) {
    // P' = [W P] C[nb:], then X' = X C[:nb] + P' (the W, P part is shared)
    PW_TRY(gemm(s, 'N', 'N', npw, nb, ns - nb, s->S + (size_t)nb * npw, npw, s->C + nb, n3, kZero, s->P, npw));
    PW_TRY(gemm(s, 'N', 'N', npw, nb, ns - nb, s->HS + (size_t)nb * npw, npw, s->C + nb, n3, kZero, s->HP, npw));
    PW_CUDA(cudaMemcpyAsync(s->S2, s->P, (size_t)npw * nb * 16, cudaMemcpyDeviceToDevice, s->st));
    PW_CUDA(cudaMemcpyAsync(s->HS2, s->HP, (size_t)npw * nb * 16, cudaMemcpyDeviceToDevice, s->st));
    PW_TRY(gemm(s, 'N', 'N', npw, nb, nb, s->S, npw, s->C, n3, kOne, s->S2, npw));
    PW_TRY(gemm(s, 'N', 'N', npw, nb, nb, s->HS, npw, s->C, n3, kOne, s->HS2, npw));
    return PW_OK;
  }
  PW_TRY(gemm(s, 'N', 'N', npw, nb, ns, s->S, npw, s->C, n3, kZero, s->S2, npw));
  PW_TRY(gemm(s, 'N', 'N', npw, nb, ns, s->HS, npw, s->C, n3, kZero, s->HS2, npw));
  return PW_OK;
}

pw_status check_tc_err(pw_solver *s) {
  PW_TRY(pw_oz_check(&s->oz, s->st));
  PW_TRY(pw_oz_check(&s->dws.oz, s->st));
  if (s->precision != PW_MIXED) return PW_OK;
  int e = 0;
  PW_CUDA(cudaMemcpyAsync(&e, s->d_err, 4, cudaMemcpyDeviceToHost, s->st));
  int ec = 0;
  if (s->cell->d_tc_err) PW_CUDA(cudaMemcpyAsync(&ec, s->cell->d_tc_err, 4, cudaMemcpyDeviceToHost, s->st));
  PW_CUDA(cudaStreamSynchronize(s->st));
  return (e || ec) ? PW_ERR_TIMEOUT : PW_OK;
}

// make HS[:, 0:nb] = H X current (mixed precision recomputes it)
pw_status ensure_hx(pw_solver *s) {
  s->hx_applied = 0;
  if (s->hx_valid) return PW_OK;
  cudaEventRecord(s->ev[7], s->st);
  PW_TRY(solver_apply_H(s, s->S, s->HS, s->nb));
  cudaEventRecord(s->ev[8], s->st);
  s->hx_valid = true;
  s->hx_applied = 1;
  return PW_OK;
}

// residual statistics of the current block to the host
pw_status refresh_stats(pw_solver *s, std::vector<double> &st_h) {
  PW_TRY(ensure_hx(s));
  pw_count_launch();
  k_stats<<<s->nb, 256, 0, s->st>>>(s->S, s->HS, s->npw, s->npw, s->lam, s->cell->d_kin, s->stats, s->nb);
  PW_TRY(pw_check_launch("stats"));
  st_h.resize(3 * (size_t)s->nb);
  PW_CUDA(cudaMemcpyAsync(st_h.data(), s->stats, st_h.size() * 8, cudaMemcpyDeviceToHost, s->st));
  PW_CUDA(cudaMemcpyAsync(s->lam_h.data(), s->lam, s->nb * 8, cudaMemcpyDeviceToHost, s->st));
  PW_CUDA(cudaStreamSynchronize(s->st));
  for (int j = 0; j < s->nb; ++j) {
    s->resid_h[j] = sqrt(st_h[j]);
    if (!isfinite(s->resid_h[j]) || !isfinite(s->lam_h[j])) return PW_ERR_NUMERIC;
  }
  return PW_OK;
}

}  // namespace

extern "C" void pw_solver_destroy(pw_solver *s) {
  if (!s) return;
  void *ptrs[] = {s->S, s->S2, s->HS, s->HS2, s->P, s->HP, s->G, s->A, s->C, s->lam, s->theta,
                  s->stats, s->act, s->gws};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  pw_tc_operand *ops[] = {&s->opSA, &s->opSB, &s->opST, &s->opHST, &s->opC, &s->opCP,
                          &s->opM};
  if (s->Mx) cudaFree(s->Mx);
  for (pw_tc_operand *o : ops) pw_tc_operand_free(o);
  if (s->rmax) cudaFree(s->rmax);
  if (s->d_err) cudaFree(s->d_err);
  pw_dense_free(&s->dws);
  pw_oz_free(&s->oz);
  delete s;
}

extern "C" pw_status pw_solver_create(pw_cell *cell, const pw_solve_opts *o, void *stream,
                                      pw_solver **out) {
  if (!out) return PW_ERR_ARG;
  *out = nullptr;
  if (!cell || !o || o->nbands < 1 || 3 * o->nbands > cell->npw || !(o->tol >= 0.0) ||
      (o->precision != PW_FP64 && o->precision != PW_MIXED) || o->chunk_rows < 0 || o->h_blocks < 0 ||
      o->h_blocks > 2)
    return PW_ERR_ARG;
  pw_solver *s = new pw_solver();
  s->cell = cell;
  s->nb = o->nbands;
  s->npw = cell->npw;
  s->tol = o->tol;
  s->maxit = o->maxit;
  s->precision = o->precision;
  s->h_blocks = o->h_blocks;
  // mixed: carried H blocks from the start in modes 1 and 2
  s->fresh_h = o->precision == PW_MIXED && o->h_blocks == 0;
  s->chunk_rows = o->chunk_rows;
  s->st = (cudaStream_t)stream;
  const int nb = s->nb, npw = s->npw, n3 = 3 * nb;
  const size_t blk3 = (size_t)npw * n3 * 16, blk = (size_t)npw * nb * 16;
  size_t acc = 0;
  pw_status r = PW_OK;
  if ((r = alloc((void **)&s->S, blk3, &acc)) || (r = alloc((void **)&s->S2, blk3, &acc)) ||
      (r = alloc((void **)&s->HS, blk3, &acc)) || (r = alloc((void **)&s->HS2, blk3, &acc)) ||
      (r = alloc((void **)&s->P, blk, &acc)) || (r = alloc((void **)&s->HP, blk, &acc)) ||
      (r = alloc((void **)&s->G, (size_t)n3 * n3 * 16, &acc)) ||
      (r = alloc((void **)&s->A, (size_t)n3 * n3 * 16, &acc)) ||
      (r = alloc((void **)&s->C, (size_t)n3 * nb * 16, &acc)) ||
      (r = alloc((void **)&s->lam, nb * 8, &acc)) || (r = alloc((void **)&s->theta, nb * 8, &acc)) ||
      (r = alloc((void **)&s->stats, 3 * (size_t)nb * 8, &acc)) ||
      (r = alloc((void **)&s->act, nb * 4, &acc)) || (r = alloc((void **)&s->rmax, (size_t)npw * 4, &acc)) ||
      (r = alloc((void **)&s->d_err, 16, &acc)) ||
      (r = pw_dense_alloc(&s->dws, n3, nb))) {
    pw_solver_destroy(s);
    return r;
  }
  if (s->precision == PW_MIXED && (r = alloc((void **)&s->Mx, (size_t)n3 * n3 * 16, &acc))) {
    pw_solver_destroy(s);
    return r;
  }
  s->bytes = acc + s->dws.bytes;
  for (cudaEvent_t &e : s->ev)
    if (cudaEventCreate(&e) != cudaSuccess) { pw_solver_destroy(s); return PW_ERR_CUDA; }
  cudaMemsetAsync(s->d_err, 0, 16, s->st);
  s->active.assign(nb, 1);
  s->lam_h.assign(nb, 0.0);
  s->resid_h.assign(nb, 0.0);
  // start block X0 in S[:, 0:nb]
  if (o->x0) {
    // host or device memory (unified addressing decides the direction)
    if (cudaMemcpyAsync(s->S, o->x0, blk, cudaMemcpyDefault, s->st) != cudaSuccess) {
      pw_solver_destroy(s); return PW_ERR_CUDA;
    }
  } else {
    pw_count_launch();
    k_random_block<<<(unsigned)(((long)npw * nb + 255) / 256), 256, 0, s->st>>>(
        s->S, npw, npw, nb, o->seed, 5ull * (uint64_t)cell->natom);
  }
  // H X0, then Cholesky-QR + Rayleigh-Ritz on span(X0)
  int ok = 1;
  if ((r = solver_apply_H(s, s->S, s->HS, nb)) || (r = subspace_rr(s, nb, &ok))) {
    pw_solver_destroy(s); return r;
  }
  if (!ok) { pw_solver_destroy(s); return PW_ERR_CHOL; }
  if ((r = rotate(s, nb, false)) || (r = check_tc_err(s))) { pw_solver_destroy(s); return r; }
  swap_rotated(s);
  s->hx_valid = !s->fresh_h;
  s->st_split_valid = false;
  cudaMemcpyAsync(s->lam, s->theta, nb * 8, cudaMemcpyDeviceToDevice, s->st);
  if (cudaStreamSynchronize(s->st) != cudaSuccess) { pw_solver_destroy(s); return PW_ERR_CUDA; }
  *out = s;
  return PW_OK;
}

extern "C" pw_status pw_subspace_step(pw_cell *cell, pw_solver *s, pw_step_report *rep) {
  if (!cell || !s || cell != s->cell) return PW_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  const int nb = s->nb, npw = s->npw, n3 = 3 * nb;
  std::vector<double> st_h;
  PW_TRY(refresh_stats(s, st_h));
  if (s->precision == PW_MIXED && s->h_blocks == 1 && !s->fresh_h) {
    double r0 = 0.0;
    for (int j = 0; j < nb; ++j) r0 = fmax(r0, s->resid_h[j]);
    if (r0 <= kCarryTol) {
      // from here on H is applied afresh each step (and once now to X)
      s->fresh_h = true;
      s->hx_valid = false;
      PW_TRY(refresh_stats(s, st_h));
    }
  }
  double rmax = 0.0;
  std::vector<int> act;
  for (int j = 0; j < nb; ++j) {
    rmax = fmax(rmax, s->resid_h[j]);
    // carried H X gives residual norms only to the split products' error
    // (~1e-4): no band locks on them; locking starts with fresh H
    const bool carried = s->precision == PW_MIXED && !s->fresh_h;
    s->active[j] = s->active[j] && (carried || s->resid_h[j] > s->tol);
    if (s->active[j]) act.push_back(j);
  }
  const int k = (int)act.size();
  if (rep) {
    memset(rep, 0, sizeof *rep);
    rep->iter = s->iter;
    rep->nactive = k;
    rep->max_resid = rmax;
  }
  if (k == 0) return PW_OK;
  cudaEventRecord(s->ev[0], s->st);
  PW_CUDA(cudaMemcpyAsync(s->act, act.data(), k * 4, cudaMemcpyHostToDevice, s->st));
  double2 *W = s->S + (size_t)nb * npw, *HW = s->HS + (size_t)nb * npw;
  pw_count_launch();
  k_precond<<<(unsigned)(((long)npw * k + 255) / 256), 256, 0, s->st>>>(
      s->S, s->HS, npw, npw, s->lam, cell->d_kin, s->stats, nb, s->act, k, W, s->precision == PW_MIXED);
  // unit columns: the Rayleigh-Ritz is invariant to column scaling, and the
  // split-precision operands need W on the scale of X
  pw_count_launch();
  k_normalize_cols<<<k, 256, 0, s->st>>>(W, nullptr, npw, npw);
  PW_TRY(pw_check_launch("precond"));
  cudaEventRecord(s->ev[1], s->st);
  PW_TRY(solver_apply_H(s, W, HW, k));
  cudaEventRecord(s->ev[2], s->st);
  int ns = nb + k, hp_applied = 0;
  if (s->haveP) {
    pw_count_launch();
    k_gather_cols<<<(unsigned)(((long)npw * k + 255) / 256), 256, 0, s->st>>>(
        s->P, npw, npw, s->act, k, s->S + (size_t)(nb + k) * npw);
    if (s->fresh_h) {
      cudaEventRecord(s->ev[9], s->st);
      PW_TRY(solver_apply_H(s, s->S + (size_t)(nb + k) * npw, s->HS + (size_t)(nb + k) * npw, k));
      cudaEventRecord(s->ev[10], s->st);
      hp_applied = 1;
    } else {
      pw_count_launch();
      k_gather_cols<<<(unsigned)(((long)npw * k + 255) / 256), 256, 0, s->st>>>(
          s->HP, npw, npw, s->act, k, s->HS + (size_t)(nb + k) * npw);
    }
    PW_TRY(pw_check_launch("gather P"));
    ns = nb + 2 * k;
  }
  int ok = 1;
  PW_TRY(subspace_rr(s, ns, &ok));
  int dropped = 0;
  if (!ok && s->haveP) {
    ns = nb + k;
    dropped = 1;
    if (s->precision == PW_MIXED) {
      PW_TRY(rr_mixed_from_gram(s, ns, &ok));
    } else {
      PW_TRY(pw_rayleigh_ritz(&s->dws, ns, nb, s->G, n3, s->A, n3, s->theta, s->C, n3, &ok, s->st,
                              piv_tol(s)));
    }
  }
  if (!ok && s->precision == PW_MIXED && !s->fresh_h) {
    // the pencil broke down with carried H blocks: apply H afresh to X (and
    // P) and take the step again, H applied every step from now on
    s->fresh_h = true;
    PW_TRY(solver_apply_H(s, s->S, s->HS, nb));
    hp_applied = 0;
    ns = nb + k;
    dropped = 0;
    if (s->haveP) {
      PW_TRY(solver_apply_H(s, s->S + (size_t)(nb + k) * npw, s->HS + (size_t)(nb + k) * npw, k));
      hp_applied = 1;
      ns = nb + 2 * k;
    }
    PW_TRY(subspace_rr(s, ns, &ok));
    if (!ok && s->haveP) {
      ns = nb + k;
      dropped = 1;
      PW_TRY(rr_mixed_from_gram(s, ns, &ok));
    }
  }
  if (!ok) return PW_ERR_CHOL;
  cudaEventRecord(s->ev[5], s->st);
  // X' = S C, HX' = HS C, P' = S[:, nb:ns] C[nb:ns], HP' likewise
  PW_TRY(rotate(s, ns, true));
  pw_count_launch();
  k_normalize_cols<<<nb, 256, 0, s->st>>>(s->P, s->HP, npw, npw);
  PW_TRY(pw_check_launch("normalize P"));
  cudaEventRecord(s->ev[6], s->st);
  swap_rotated(s);
  s->hx_valid = !s->fresh_h;
  s->st_split_valid = false;
  PW_CUDA(cudaMemcpyAsync(s->lam, s->theta, nb * 8, cudaMemcpyDeviceToDevice, s->st));
  PW_CUDA(cudaStreamSynchronize(s->st));
  PW_TRY(check_tc_err(s));
  s->haveP = true;
  s->iter++;
  s->dropped += dropped;
  if (rep) {
    rep->iter = s->iter;
    rep->dropped_p = dropped;
    rep->nsub = ns;
    rep->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    float t[6] = {0, 0, 0, 0, 0, 0};
    cudaEventElapsedTime(&t[0], s->ev[0], s->ev[1]);
    cudaEventElapsedTime(&t[1], s->ev[1], s->ev[2]);
    cudaEventElapsedTime(&t[2], s->ev[3], s->ev[4]);
    cudaEventElapsedTime(&t[3], s->ev[4], s->ev[5]);
    cudaEventElapsedTime(&t[4], s->ev[5], s->ev[6]);
    rep->ms_resid = t[0];
    float thx = 0.f, thp = 0.f;
    if (s->hx_applied) cudaEventElapsedTime(&thx, s->ev[7], s->ev[8]);
    if (hp_applied) cudaEventElapsedTime(&thp, s->ev[9], s->ev[10]);
    rep->ms_hpsi = t[1] + thx + thp;
    rep->hpsi_cols = k + (s->hx_applied ? nb : 0) + (hp_applied ? k : 0);
    rep->ms_gram = t[2];
    rep->ms_rr = t[3];
    rep->ms_rot = t[4];
    float part[5];
    pw_dense_stage_ms(&s->dws, part);
    for (int i = 0; i < 5; ++i) rep->ms_rr_part[i] = part[i];
  }
  return PW_OK;
}

extern "C" pw_status pw_solver_polish(pw_solver *s) {
  if (!s) return PW_ERR_ARG;
  const int nb = s->nb, npw = s->npw, n3 = 3 * nb;
  const int saved = s->precision;
  s->precision = PW_FP64;
  pw_status r = solver_apply_H(s, s->S, s->HS, nb);
  int ok = 1;
  if (r == PW_OK) r = subspace_rr(s, nb, &ok);
  if (r == PW_OK && !ok) r = PW_ERR_CHOL;
  if (r == PW_OK) r = rotate(s, nb, false);
  s->precision = saved;
  PW_TRY(r);
  swap_rotated(s);
  s->hx_valid = true;
  PW_CUDA(cudaMemcpyAsync(s->lam, s->theta, nb * 8, cudaMemcpyDeviceToDevice, s->st));
  PW_CUDA(cudaStreamSynchronize(s->st));
  (void)npw; (void)n3;
  // P no longer matches the rotated block
  s->haveP = false;
  return PW_OK;
}

extern "C" pw_status pw_solver_eigs(pw_solver *s, double *eig, double *resid) {
  if (!s) return PW_ERR_ARG;
  std::vector<double> st_h;

  PW_TRY(refresh_stats(s, st_h));
  if (eig) memcpy(eig, s->lam_h.data(), s->nb * 8);
  if (resid) memcpy(resid, s->resid_h.data(), s->nb * 8);
  return PW_OK;
}

extern "C" pw_status pw_solver_block(pw_solver *s, void *psi, int ld) {
  if (!s || !psi || ld < s->npw) return PW_ERR_ARG;
  PW_CUDA(cudaMemcpy2DAsync(psi, (size_t)ld * 16, s->S, (size_t)s->npw * 16, (size_t)s->npw * 16,
                            s->nb, cudaMemcpyDeviceToDevice, s->st));
  PW_CUDA(cudaStreamSynchronize(s->st));
  return PW_OK;
}

extern "C" pw_status pw_solver_set_p(pw_solver *s, const void *p, int ld) {
  if (!s || !p || ld < s->npw) return PW_ERR_ARG;
  const int nb = s->nb, npw = s->npw;
  // host or device memory (unified addressing decides the direction)
  PW_CUDA(cudaMemcpy2DAsync(s->P, (size_t)npw * 16, p, (size_t)ld * 16, (size_t)npw * 16, nb,
                            cudaMemcpyDefault, s->st));
  // the FP64 step carries H P through the rotations, so form it here (in the
  // solver's precision); the mixed step recomputes H P itself
  if (!s->fresh_h) PW_TRY(solver_apply_H(s, s->P, s->HP, nb));
  pw_count_launch();
  k_normalize_cols<<<nb, 256, 0, s->st>>>(s->P, s->fresh_h ? nullptr : s->HP, npw, npw);
  PW_TRY(pw_check_launch("set P"));
  PW_CUDA(cudaStreamSynchronize(s->st));
  s->haveP = true;
  return PW_OK;
}

extern "C" pw_status pw_solver_get_p(pw_solver *s, void *p, int ld, int *have_p) {
  if (!s || !p || ld < s->npw) return PW_ERR_ARG;
  if (have_p) *have_p = s->haveP ? 1 : 0;
  PW_CUDA(cudaMemcpy2DAsync(p, (size_t)ld * 16, s->P, (size_t)s->npw * 16, (size_t)s->npw * 16, s->nb,
                            cudaMemcpyDefault, s->st));
  PW_CUDA(cudaStreamSynchronize(s->st));
  return PW_OK;
}

// FP64 steps after a mixed solve: the split-precision floor leaves a few
// bands just above tol, which one or two FP64 steps finish; more than this
// means the mixed solve did not converge and FP64 (~20x slower) would not help
constexpr int kMaxFp64Refine = 8;

extern "C" pw_status pw_eigsolve(pw_cell *cell, const pw_solve_opts *o, double *eig, void *psi_out,
                                 int ld, pw_solve_report *rep, void *stream) {
  if (!cell || !o || !eig || (psi_out && ld < cell->npw)) return PW_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  pw_solver *s = nullptr;
  PW_TRY(pw_solver_create(cell, o, stream, &s));
  pw_status r = PW_OK;
  std::vector<double> st_h;
  bool conv = false;
  for (;;) {
    if ((r = refresh_stats(s, st_h)) != PW_OK) break;
    double rmax = 0.0;
    for (int j = 0; j < s->nb; ++j) rmax = fmax(rmax, s->resid_h[j]);
    if (rmax <= s->tol) { conv = true; break; }
    if (s->iter >= s->maxit) break;
    pw_step_report sr;
    if ((r = pw_subspace_step(cell, s, &sr)) != PW_OK) break;
    // every band locked: nothing left to iterate (a locked band whose residual
    // drifted above tol leaves the solve unconverged)
    if (sr.nactive == 0) break;
  }
  int fp64_iters = 0;
  if (r == PW_OK && s->precision == PW_MIXED) {
    // FP64 Rayleigh-Ritz on the converged block: FP64 overlap, eigensolve,
    // residual norms and orthonormality
    r = pw_solver_polish(s);
    if (r == PW_OK) r = refresh_stats(s, st_h);
    double rmax = 0.0;
    for (int j = 0; j < s->nb; ++j) rmax = fmax(rmax, s->resid_h[j]);
    if (r == PW_OK && rmax > s->tol && s->iter < s->maxit) {
      // bands the split-precision floor left above tol: continue in FP64 from
      // the polished block (P was dropped by the polish; H X is FP64)
      s->precision = PW_FP64;
      s->fresh_h = false;
      for (int j = 0; j < s->nb; ++j) s->active[j] = s->resid_h[j] > s->tol;
      for (;;) {
        if ((r = refresh_stats(s, st_h)) != PW_OK) break;
        rmax = 0.0;
        for (int j = 0; j < s->nb; ++j) rmax = fmax(rmax, s->resid_h[j]);
        if (rmax <= s->tol || s->iter >= s->maxit || fp64_iters >= kMaxFp64Refine) break;
        pw_step_report sr;
        if ((r = pw_subspace_step(cell, s, &sr)) != PW_OK) break;
        ++fp64_iters;
        if (sr.nactive == 0) break;
      }
      s->precision = PW_MIXED;
    }
    if (r == PW_OK) conv = rmax <= s->tol;
  }
  if (r == PW_OK || r == PW_ERR_CHOL) {
    memcpy(eig, s->lam_h.data(), s->nb * 8);
    if (psi_out) pw_solver_block(s, psi_out, ld);
  }
  if (rep) {
    rep->iters = s->iter;
    double rmax = 0.0;
    for (int j = 0; j < s->nb; ++j) rmax = fmax(rmax, s->resid_h[j]);
    rep->max_resid = rmax;
    rep->device_bytes = s->bytes;
    // orthonormality of the final block, FP64
    double oe = -1.0;
    if (gemm(s, 'C', 'N', s->nb, s->nb, s->npw, s->S, s->npw, s->S, s->npw, kZero, s->G, s->nb) == PW_OK) {
      pw_count_launch();
      k_orth_err<<<1, 1024, 0, s->st>>>(s->G, s->nb, s->theta);
      cudaMemcpyAsync(&oe, s->theta, 8, cudaMemcpyDeviceToHost, s->st);
      cudaStreamSynchronize(s->st);
    }
    rep->orth_err = oe;
    rep->fp64_iters = fp64_iters;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  pw_solver_destroy(s);
  if (r != PW_OK) return r;
  return conv ? PW_OK : PW_ERR_NOCONV;
}
