// FP64 dense linear algebra of the Rayleigh-Ritz step (the paper's Syevd hot
// spot, Sec. III-D), all on the GPU in FP64:
//
//  * Jacobi scaling and blocked Cholesky of the Gram matrix, with the pivot
//    test that drives the drop-P fallback;
//  * triangular inverse L^-1 (recursive, GEMM based);
//  * Hermitian eigensolver: Householder reduction to a real symmetric
//    tridiagonal T, Cuppen's divide and conquer on T (deflation, secular
//    equation solved per root with a two-pole rational model, eigenvectors
//    from the Gu-Eisenstat (Lowner) recomputed z), and back-transformation of
//    the wanted eigenvectors.
//
// The divide and conquer runs level by level over a binary tree with leaves
// of size 1; every node of a level is handled by the same few batched
// launches.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <vector>

#include <atomic>

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

#include "dense.cuh"
#include "house.cuh"

namespace {

constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ double warp_prod(double v) {
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ double block_max(double v, double *sh) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = -1.7976931348623157e308;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : -1.7976931348623157e308;
    r = warp_max(r);
    if (threadIdx.x == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// ======================================================================
// Cholesky, scaling, triangular inverse
// ======================================================================

// dscale_i = Re(G_ii)^-1/2; flag[0] |= 1 if a diagonal is not positive
__global__ void k_diag_scale(const double2 *G, int ld, int n, double *dscale, int *flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double g = G[i + (long)i * ld].x;
  // a diagonal entry sum_g |s_g|^2 is finite for any finite basis column, so a
  // NaN / Inf here means NaN / Inf in the basis (or in its split operands)
  if (!isfinite(g)) atomicOr(flag, 8);
  if (!(g > 0.0)) { atomicOr(flag, 1); dscale[i] = 0.0; return; }
  dscale[i] = 1.0 / sqrt(g);
}

// out = d o (0.5 (M + M^H)) o d  (n x n, out ld n)
__global__ void k_scale_herm(const double2 *M, int ld, int n, const double *d, double2 *out) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n) return;
  const double2 a = M[i + (long)j * ld], b = M[j + (long)i * ld];
  const double s = 0.5 * d[i] * d[j];
  out[i + (long)j * n] = make_double2(s * (a.x + b.x), s * (a.y - b.y));
}

// lower triangle <- conj(upper), diagonal made real (n x n, ld n)
__global__ void k_mirror_upper_to_lower(double2 *M, int n) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n || i < j) return;
  if (i == j) { M[i + (long)i * n].y = 0.0; return; }
  const double2 u = M[j + (long)i * n];
  M[i + (long)j * n] = make_double2(u.x, -u.y);
}

// out (ld n) = 0.5 (M + M^H) of an n x n matrix (ld)
__global__ void k_copy_herm(const double2 *M, int ld, int n, double2 *out) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n) return;
  const double2 a = M[i + (long)j * ld], b = M[j + (long)i * ld];
  out[i + (long)j * n] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
}

constexpr int CB = 32;   // Cholesky / inverse block
constexpr int DC_TC_MIN_HALF = 512;   // merge levels with larger halves: products on the tensor cores

// unblocked Cholesky of the diagonal block at j0 (size b <= 32), in place
// Li (b x b, ld CB) = L11^-1 as well, for the row solves of the panel below
__global__ void k_potf2(double2 *A, int n, int j0, int b, double *piv, int *flag, double2 *Li) {
  __shared__ double2 L[CB][CB + 1];
  __shared__ double s_inv;
  __shared__ int bad;
  const int t = threadIdx.x;
  for (int e = t; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    L[i][j] = A[(j0 + i) + (long)(j0 + j) * n];
  }
  if (t == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    // the pivot's square root and reciprocal once, by one thread (FP64
    // division runs on the narrow FP64 pipe of this part)
    if (t == 0) {
      const double p = L[c][c].x;
      piv[j0 + c] = p;
      const double d = p > 0.0 ? sqrt(p) : 1.0;
      if (!(p > 0.0)) bad = 1;
      L[c][c] = make_double2(d, 0.0);
      s_inv = 1.0 / d;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = c + 1 + t; i < b; i += blockDim.x) { L[i][c].x *= inv; L[i][c].y *= inv; }
    __syncthreads();
    for (int e = t; e < b * b; e += blockDim.x) {
      const int i = e % b, j = e / b;
      if (j > c && i >= j) {
        const double2 li = L[i][c], lj = L[j][c];
        // L[i][j] -= li * conj(lj)
        L[i][j].x -= li.x * lj.x + li.y * lj.y;
        L[i][j].y -= li.y * lj.x - li.x * lj.y;
      }
    }
    __syncthreads();
  }
  for (int e = t; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    if (i >= j) A[(j0 + i) + (long)(j0 + j) * n] = L[i][j];
  }
  if (t == 0 && bad) atomicOr(flag, 2);
  // L11^-1 by row elimination of [L11 | I]: step l scales row l by 1/L_ll and
  // removes L_il (i > l) from the rows below; only the original L entries are
  // read, and each step's updates are spread over the whole block
  __shared__ double2 X[CB][CB + 1];
  __shared__ double s_dinv[CB];
  for (int e = t; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    X[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (t < b) s_dinv[t] = 1.0 / L[t][t].x;
  __syncthreads();
  for (int l = 0; l < b; ++l) {
    if (t <= l) {
      const double inv = s_dinv[l];
      X[l][t].x *= inv;
      X[l][t].y *= inv;
    }
    __syncthreads();
    const int cnt = (b - 1 - l) * (l + 1);
    for (int e = t; e < cnt; e += blockDim.x) {
      const int i = l + 1 + e / (l + 1), j = e % (l + 1);
      X[i][j] = csub(X[i][j], cmul(L[i][l], X[l][j]));
    }
    __syncthreads();
  }
  for (int e = t; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    Li[i + j * CB] = X[i][j];
  }
}

// rows i >= j0 + b:  A[i, j0:j0+b] <- A[i, j0:j0+b] L11^-H, as products with
// the inverse Li = L11^-1 from k_potf2: x_c = sum_{l <= c} a_l conj(Li[c][l]).
// 16 rows per block, thread (row r, r + 8; column c), so every SM gets work.
constexpr int TRSM_ROWS = 16;
__global__ void __launch_bounds__(256) k_trsm_inv(double2 *A, int n, int j0, int b, const double2 *Li) {
  __shared__ double2 Ls[CB][CB + 1], As[TRSM_ROWS][CB + 1];
  const int r0 = j0 + b + blockIdx.x * TRSM_ROWS;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    Ls[i][j] = Li[i + j * CB];
  }
  for (int e = threadIdx.x; e < TRSM_ROWS * b; e += blockDim.x) {
    const int rr = e % TRSM_ROWS, c = e / TRSM_ROWS, i = r0 + rr;
    As[rr][c] = i < n ? A[i + (long)(j0 + c) * n] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int c = threadIdx.x & 31, rq = threadIdx.x >> 5;
  if (c >= b) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int rr = rq + 8 * h, i = r0 + rr;
    if (i >= n) continue;
    double2 x = make_double2(0.0, 0.0);
    for (int l = 0; l <= c; ++l) {
      const double2 a = As[rr][l], li = Ls[c][l];
      // x += a conj(li)
      x.x = fma(a.x, li.x, x.x);
      x.x = fma(a.y, li.y, x.x);
      x.y = fma(a.y, li.x, x.y);
      x.y = fma(-a.x, li.y, x.y);
    }
    A[i + (long)(j0 + c) * n] = x;
  }
}

__global__ void k_zero_upper(double2 *A, int n) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i < n && j < n && i < j) A[i + (long)j * n] = make_double2(0.0, 0.0);
}

// flag |= 4 if min pivot <= tol * max pivot or a pivot is not finite (a tiny
// pivot can overflow the columns after it, so a non-finite pivot is a
// breakdown, not evidence of NaN / Inf input: k_diag_scale reports those)
__global__ void k_chol_check(const double *piv, int n, double tol, int *flag) {
  __shared__ double sh[32];
  double mn = 1e300, mx = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double p = piv[i];
    if (!isfinite(p)) bad = 1;
    mn = fmin(mn, p);
    mx = fmax(mx, p);
  }
  mx = block_max(mx, sh);
  mn = -block_max(-mn, sh);
  if (bad) atomicOr(flag, 4);
  if (threadIdx.x == 0 && !(mn > tol * mx)) atomicOr(flag, 4);
}

// inverse of lower-triangular diagonal blocks (size <= 32), one CTA per block
__global__ void k_trinv_small(const double2 *L, double2 *X, int n, const int *blk_lo,
                              const int *blk_sz) {
  __shared__ double2 Ls[CB][CB + 1];
  const int lo = blk_lo[blockIdx.x], b = blk_sz[blockIdx.x];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    Ls[i][j] = L[(lo + i) + (long)(lo + j) * n];
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= b) return;
  double2 x[CB];
  for (int i = 0; i < b; ++i) {
    if (i < j) { x[i] = make_double2(0.0, 0.0); continue; }
    double2 s = (i == j) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
    for (int l = j; l < i; ++l) s = csub(s, cmul(Ls[i][l], x[l]));
    const double inv = 1.0 / Ls[i][i].x;
    x[i] = make_double2(s.x * inv, s.y * inv);
  }
  for (int i = 0; i < b; ++i) X[(lo + i) + (long)(lo + j) * n] = x[i];
}

__global__ void k_scale_rows_real(double2 *C, int ld, int n, int nb, const double *d) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)n * nb) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  double2 &c = C[i + (long)j * ld];
  c.x *= d[i];
  c.y *= d[i];
}

// ======================================================================
// Householder tridiagonalisation, complex Hermitian (lower triangle)
// ======================================================================

// ----------------------------------------------------------------------
// Blocked Householder reduction (panels of TPB columns, lower triangle).
// Inside a panel the trailing matrix is not updated: column c first receives
// the panel's previous rank-2 updates, A22 v is a pure Hermitian product of
// the not-yet-updated lower triangle, corrected by V (W^H v) + W (V^H v);
// after the panel, A22 -= V W^H + W V^H is one rank-2 TPB GEMM on the lower
// tiles.  Panel buffer P = [V | W | V] (ld n), so [V W] and [W V] are both
// column ranges of it.
//
// Per column c (panel index i) three kernels:
//   k_pcol   finish W[:, i-1], update column c, norm partials; the block that
//            finishes last forms beta, tau and the scale s of the reflector
//            (v = x s below its unit head) -- scalars only;
//   k_phemv  lower-tile partial products of A22 v (v formed on the fly from
//            x and s), the dots W^H v and V^H v, and the V columns of v;
//   k_prows  sum the partials, subtract the corrections, p = tau y, store v
//            in place of x and the partial dots p^H v.
// FP64 runs at about two FMAs per clock per SM on this part, so the products
// are written as four FMAs per complex multiply-add.
// ----------------------------------------------------------------------
constexpr int TT = 32;
constexpr int TPB = 32;

// The per-column kernels are chained with programmatic dependent launch: a
// kernel may start while its predecessor finishes, waits (griddepcontrol.wait)
// before it reads anything the predecessor wrote, and only then lets its own
// successor launch.  So before its wait a kernel may read data written two or
// more launches back (k_phemv loads its tile of the trailing matrix there).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}
constexpr int PCOL_THREADS = 128;

// 32 rows per block; the four warps split the panel's previous updates
// (q = warp mod 4) so that the FP64 work lands on all four SM sub-partitions
__global__ void __launch_bounds__(PCOL_THREADS) k_pcol(double2 *A, int n, int c, int i, double2 *P, int b,
                                                       const double2 *p, const double2 *dotpart, int ndot,
                                                       double2 *tau, double *d, double *e, double *nrm_part,
                                                       double2 *hscal, unsigned *ticket) {
  __shared__ double sh[32];
  __shared__ unsigned s_ticket;
  __shared__ double2 s_vc[TPB], s_wc[TPB], s_u[4][33];
  double2 *V = P, *W = P + (long)b * n;
  const int rl = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int r = c + blockIdx.x * 32 + rl;
  // Before the wait: what the panel's earlier columns wrote two or more
  // launches back — V[:, q < i], W[:, q < i-1] and, for i > 0, column c of A
  // (last written by the previous panel's update).  p and the dots (and from
  // them W[:, i-1]) come from the predecessor.
  constexpr int QMAX = (TPB + 3) / 4;
  double2 vq_r[QMAX], wq_r[QMAX];
  double2 a = make_double2(0.0, 0.0);
  if (i > 0) {
    if (threadIdx.x < i) {
      const int q = threadIdx.x;
      s_vc[q] = V[c + (long)q * n];
      if (q < i - 1) s_wc[q] = W[c + (long)q * n];
    }
#pragma unroll
    for (int t = 0; t < QMAX; ++t) {
      const int q = g + 4 * t;
      const bool ok = r < n && q < i;
      vq_r[t] = ok ? V[r + (long)q * n] : make_double2(0.0, 0.0);
      wq_r[t] = ok && q < i - 1 ? W[r + (long)q * n] : make_double2(0.0, 0.0);
    }
    if (g == 0 && r < n) a = A[r + (long)c * n];
  }
  pdl_wait();
  pdl_trigger();
  double2 al = make_double2(0.0, 0.0);
  if (i > 0) {
    al = panel_alpha(dotpart, ndot, tau[c - 1], sh);
    // W[c, i-1] = p_{c-1}[0] + alpha v_{c-1}[row c], the head of v_{c-1} being 1
    if (threadIdx.x == 0) s_wc[i - 1] = cadd(__ldcg(&p[0]), al);
  }
  __syncthreads();
  if (i > 0) {
    double2 u = make_double2(0.0, 0.0);   // sum_q v_rq conj(w_cq) + w_rq conj(v_cq), q = g mod 4
    if (r < n) {
#pragma unroll
      for (int t = 0; t < QMAX; ++t) {
        const int q = g + 4 * t;
        if (q >= i) break;
        const double2 vq = vq_r[t];
        double2 wq = wq_r[t];
        if (q == i - 1) {
          wq = __ldcg(&p[r - c]);
          cmac(wq, al, vq);
          W[r + (long)q * n] = wq;
        }
        cmacc(u, s_wc[q], vq);
        cmacc(u, s_vc[q], wq);
      }
    }
    s_u[g][rl] = u;
    __syncthreads();
  }
  if (g == 0 && r < n) {
    if (i == 0) a = A[r + (long)c * n];
    if (i > 0) {
      a = csub(a, cadd(cadd(s_u[0][rl], s_u[1][rl]), cadd(s_u[2][rl], s_u[3][rl])));
      A[r + (long)c * n] = a;
    }
  }
  if (g != 0) return;
  double nrm = 0.0;
  if (r < n && r > c + 1) nrm = a.x * a.x + a.y * a.y;
  nrm = warp_sum(nrm);
  if (rl == 0) {
    nrm_part[blockIdx.x] = nrm;
    __threadfence();
    s_ticket = atomicAdd(ticket, 1u);
  }
  __syncwarp();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  // last block: reflector scalars from x = A[c+1:, c]
  double xn2 = 0.0;
  for (int q = rl; q < (int)gridDim.x; q += 32) xn2 += __ldcg(&nrm_part[q]);
  xn2 = warp_sum(xn2);
  if (rl != 0) return;
  *ticket = 0u;
  const double2 alpha = __ldcg(&A[(c + 1) + (long)c * n]);
  double beta;
  double2 tk, scal;
  reflector_scalars(xn2, alpha, beta, tk, scal);
  d[c] = __ldcg(&A[c + (long)c * n]).x;
  tau[c] = tk;
  e[c] = beta;
  *hscal = scal;
}

// y = A22 v as lower-tile partials (A22 = rows/cols >= c+1, not yet updated
// by this panel); 2i extra blocks: u[2q] = W[:, q]^H v, u[2q+1] = V[:, q]^H v;
// nwr more blocks write v into V[:, i] and its copy
__global__ void __launch_bounds__(256) k_phemv(const double2 *A, int n, int c, int i, double2 *P, int b,
                                               int ntiles, double2 *part, int nmax, double2 *ucorr,
                                               const double2 *hscal) {
  __shared__ double2 tile[TT][TT + 1];
  __shared__ double2 vrow[TT], vcol[TT], rpart[4][TT + 1], cpart[4][TT + 1];
  __shared__ double sh[32];
  const int o = c + 1, m = n - o;
  const double2 *xk = A + o + (long)c * n;   // x of column c, x[0] at row o
  const int blk = blockIdx.x;
  int I = 0, J = 0, x0 = 0, y0 = 0;
  if (blk < ntiles) {
    // tile (I, J) of the lower triangle; FP32 estimate (FP64 is scarce), fixed up exactly
    const int t = blk;
    I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    J = t - I * (I + 1) / 2;
    x0 = TT * I;
    y0 = TT * J;   // tile rows x0.., columns y0.. (offsets from o)
    // the trailing matrix was last written before the predecessor's wait: load it now
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int yc = y0 + lane;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rl = wq * 4 + q, xr = x0 + rl;
      double2 a = make_double2(0.0, 0.0);
      if (xr < m && yc < m && (I != J || yc <= xr)) a = A[(o + xr) + (long)(o + yc) * n];
      tile[rl][lane] = a;
    }
  }
  pdl_wait();
  pdl_trigger();
  const double2 scal = *hscal;
  if (blk >= ntiles + 2 * i) {   // writer blocks
    const int x = (blk - ntiles - 2 * i) * blockDim.x + threadIdx.x;
    if (x < m) {
      const double2 v = refl_entry(xk, x, scal);
      P[o + x + (long)i * n] = v;
      P[o + x + (long)(2 * b + i) * n] = v;
    }
    return;
  }
  if (blk >= ntiles) {
    const int q2 = blk - ntiles, q = q2 >> 1;
    const double2 *col = P + (long)((q2 & 1) ? q : b + q) * n;   // odd: V[:, q], even: W[:, q]
    double2 s = make_double2(0.0, 0.0);
    for (int x = threadIdx.x; x < m; x += blockDim.x) cmacc(s, col[o + x], refl_entry(xk, x, scal));
    s.x = block_sum(s.x, sh);
    s.y = block_sum(s.y, sh);
    if (threadIdx.x == 0) ucorr[q2] = s;
    return;
  }
  if (threadIdx.x < TT) {
    const int xr = x0 + threadIdx.x, yc = y0 + threadIdx.x;
    vrow[threadIdx.x] = xr < m ? refl_entry(xk, xr, scal) : make_double2(0.0, 0.0);
    vcol[threadIdx.x] = yc < m ? refl_entry(xk, yc, scal) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // warps 0-3: quarter row sums A v; warps 4-7: quarter column sums A^H v
  // (strictly below the diagonal in a diagonal tile)
  {
    const int k = (threadIdx.x >> 5) & 3, l = threadIdx.x & 31;
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x < 128) {
#pragma unroll
      for (int cl = 8 * k; cl < 8 * k + 8; ++cl) cmac(s, tile[l][cl], vcol[cl]);
      rpart[k][l] = s;
    } else {
#pragma unroll
      for (int rr = 8 * k; rr < 8 * k + 8; ++rr)
        if (I != J || rr > l) cmacc(s, tile[rr][l], vrow[rr]);
      cpart[k][l] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < TT) {
    const int l = threadIdx.x;
    const double2 rs = cadd(cadd(rpart[0][l], rpart[1][l]), cadd(rpart[2][l], rpart[3][l]));
    const double2 cs = cadd(cadd(cpart[0][l], cpart[1][l]), cadd(cpart[2][l], cpart[3][l]));
    if (I != J) {
      if (x0 + l < m) part[(long)J * nmax + x0 + l] = rs;
      if (y0 + l < m) part[(long)I * nmax + y0 + l] = cs;
    } else if (x0 + l < m) {
      part[(long)J * nmax + x0 + l] = cadd(rs, cs);
    }
  }
}

// 32 rows per block, 8 thread groups over the partial slots s0..nT-1 and the
// corrections: y = sum of partials - V[:, <i] u_W - W[:, <i] u_V, p = tau_c y,
// v stored in place of x, partial dots p^H v.  part[s * nmax + x] holds slot
// s of row o + x.
__global__ void __launch_bounds__(256) k_prows(double2 *A, int n, int c, int i, const double2 *P, int b,
                                               const double2 *part, int s0, int nT, int nmax, const double2 *ucorr,
                                               const double2 *tau, const double2 *hscal, double2 *p,
                                               double2 *dotpart) {
  __shared__ double2 red[8][33];
  const int o = c + 1, m = n - o;
  const int rl = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int x = blockIdx.x * 32 + rl;
  // Before the wait: the panel columns V[:, q < i], W[:, q < i] (written two
  // or more launches back); the partial products and corrections come from
  // the predecessor.
  constexpr int QMAX = (TPB + 7) / 8;
  double2 vq_r[QMAX], wq_r[QMAX];
#pragma unroll
  for (int t = 0; t < QMAX; ++t) {
    const int q = g + 8 * t;
    const bool ok = x < m && q < i;
    vq_r[t] = ok ? P[o + x + (long)q * n] : make_double2(0.0, 0.0);
    wq_r[t] = ok ? P[o + x + (long)(b + q) * n] : make_double2(0.0, 0.0);
  }
  pdl_wait();
  pdl_trigger();
  double2 y = make_double2(0.0, 0.0);
  if (x < m) {
    for (int s = s0 + g; s < nT; s += 8) y = cadd(y, part[(long)s * nmax + x]);
#pragma unroll
    for (int t = 0; t < QMAX; ++t) {
      const int q = g + 8 * t;
      if (q >= i) break;
      const double2 uw = ucorr[2 * q], uv = ucorr[2 * q + 1];
      cmac(y, vq_r[t], make_double2(-uw.x, -uw.y));   // - V[r,q] (W^H v)_q
      cmac(y, wq_r[t], make_double2(-uv.x, -uv.y));   // - W[r,q] (V^H v)_q
    }
  }
  red[g][rl] = y;
  __syncthreads();
  if (g != 0) return;
  double2 pv = make_double2(0.0, 0.0);
  if (x < m) {
#pragma unroll
    for (int q = 1; q < 8; ++q) y = cadd(y, red[q][rl]);
    const double2 pr = cmul(tau[c], y);
    p[x] = pr;
    double2 *xc = A + o + (long)c * n;
    const double2 v = refl_entry(xc, x, *hscal);
    xc[x] = v;
    cmacc(pv, pr, v);
  }
  pv.x = warp_sum(pv.x);
  pv.y = warp_sum(pv.y);
  if (rl == 0) dotpart[blockIdx.x] = pv;
}

// W[:, i] = p + alpha v for the panel's last column (rows >= c+1)
__global__ void __launch_bounds__(256) k_pfinal(const double2 *A, int n, int c, int i, double2 *P, int b,
                                                const double2 *p, const double2 *dotpart, int ndot,
                                                const double2 *tau) {
  __shared__ double sh[32];
  pdl_wait();
  pdl_trigger();
  const double2 al = panel_alpha(dotpart, ndot, tau[c], sh);
  const int o = c + 1;
  const int r = o + blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) {
    double2 w = p[r - o];
    cmac(w, al, A[r + (long)c * n]);
    P[r + (long)(b + i) * n] = w;
  }
}

// ----------------------------------------------------------------------
// One panel in one cooperative launch: the per-column work of k_pcol,
// k_phemv and k_prows (and k_pfinal after the panel's last column) as phases
// of a persistent grid separated by grid-wide barriers, so the chain of three
// dependent launches per column becomes three barriers.  Same arithmetic as
// the chained kernels; every block derives the reflector scalars itself from
// the norm partials (one barrier fewer than a leader block would need).
// ----------------------------------------------------------------------
constexpr int CO_THREADS = 256;
constexpr int CO_QMAX = (TPB + 7) / 8;     // panel columns per thread, 8 warps (phase C)
constexpr int CO_QMAX4 = (TPB + 3) / 4;    // the same with 4 warps (phase A, k_pcol's split)

__global__ void __launch_bounds__(CO_THREADS) k_panel_coop(double2 *A, int n, int j0, int b, double2 *P,
                                                           double2 *p, double2 *dotpart, double2 *tau, double *d,
                                                           double *e, double *nrm_part, double2 *hscal_g,
                                                           double2 *part, int nmax, double2 *ucorr) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32];
  __shared__ double2 tile[TT][TT + 1];
  __shared__ double2 vrow[TT], vcol[TT], rpart[4][TT + 1], cpart[4][TT + 1];
  __shared__ double2 s_vc[TPB], s_wc[TPB], s_u[8][33];
  double2 *V = P, *W = P + (long)b * n;
  const int nblk = gridDim.x;
  const int rl = threadIdx.x & 31, g = threadIdx.x >> 5;
  int ndot = 0;
  double2 tk = make_double2(0.0, 0.0), scal = make_double2(0.0, 0.0);
  for (int i = 0; i < b; ++i) {
    const int c = j0 + i, o = c + 1, m = n - o;
    // ---- phase A: column c receives the panel's earlier rank-2 updates.
    // Two 32-row blocks per pass, four warps each, in k_pcol's order.
    double2 al = make_double2(0.0, 0.0);
    if (i > 0) {
      al = panel_alpha(dotpart, ndot, tk, sh, PCOL_THREADS);   // tk: tau of column c - 1
      if (threadIdx.x < i) {
        const int q = threadIdx.x;
        s_vc[q] = V[c + (long)q * n];
        if (q < i - 1) s_wc[q] = W[c + (long)q * n];
      }
      if (threadIdx.x == 0) s_wc[i - 1] = cadd(__ldcg(&p[0]), al);
    }
    __syncthreads();
    const int nrb = (n - c + 31) / 32;
    const int half = g >> 2, gq = g & 3;
    for (int rb0 = 2 * blockIdx.x; rb0 < nrb; rb0 += 2 * nblk) {
      const int rb = rb0 + half;
      const int r = c + rb * 32 + rl;
      double2 u = make_double2(0.0, 0.0);
      if (i > 0 && rb < nrb && r < n) {
#pragma unroll
        for (int t = 0; t < CO_QMAX4; ++t) {
          const int q = gq + 4 * t;
          if (q >= i) break;
          const double2 vq = V[r + (long)q * n];
          double2 wq;
          if (q == i - 1) {
            wq = __ldcg(&p[r - c]);
            cmac(wq, al, vq);
            W[r + (long)q * n] = wq;
          } else {
            wq = W[r + (long)q * n];
          }
          cmacc(u, s_wc[q], vq);
          cmacc(u, s_vc[q], wq);
        }
      }
      s_u[g][rl] = u;
      __syncthreads();
      if (gq == 0 && rb < nrb) {
        double nrm = 0.0;
        if (r < n) {
          double2 a = A[r + (long)c * n];
          if (i > 0) {
            const int h4 = 4 * half;
            a = csub(a, cadd(cadd(s_u[h4][rl], s_u[h4 + 1][rl]), cadd(s_u[h4 + 2][rl], s_u[h4 + 3][rl])));
            A[r + (long)c * n] = a;
          }
          if (r > c + 1) nrm = a.x * a.x + a.y * a.y;
        }
        nrm = warp_sum(nrm);
        if (rl == 0) nrm_part[rb] = nrm;
      }
      __syncthreads();
    }
    grid.sync();
    // reflector scalars from x = A[c+1:, c] (every block, one warp, in the
    // order of k_pcol's last block)
    {
      if (g == 0) {
        double xn2 = 0.0;
        for (int q = rl; q < nrb; q += 32) xn2 += __ldcg(&nrm_part[q]);
        xn2 = warp_sum(xn2);
        if (rl == 0) sh[0] = xn2;
      }
      __syncthreads();
      const double xn2 = sh[0];
      __syncthreads();
      const double2 alpha = __ldcg(&A[(c + 1) + (long)c * n]);
      double beta;
      if (xn2 == 0.0 && alpha.y == 0.0) {
        beta = alpha.x;
        tk = make_double2(0.0, 0.0);
        scal = make_double2(0.0, 0.0);
      } else {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
        tk = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double qq = 1.0 / (den.x * den.x + den.y * den.y);
        scal = make_double2(den.x * qq, -den.y * qq);
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        d[c] = __ldcg(&A[c + (long)c * n]).x;
        tau[c] = tk;
        e[c] = beta;
        *hscal_g = scal;
      }
    }
    // ---- phase B: lower-tile partials of A22 v, the corrections W^H v and
    // V^H v, and the copy of v into the panel
    const double2 *xk = A + o + (long)c * n;
    const int nT = (m + TT - 1) / TT, ntiles = nT * (nT + 1) / 2, nwr = (m + 255) / 256;
    const int tasks = ntiles + 2 * i + nwr;
    for (int task = blockIdx.x; task < tasks; task += nblk) {
      if (task >= ntiles + 2 * i) {
        const int x = (task - ntiles - 2 * i) * blockDim.x + threadIdx.x;
        if (x < m) {
          const double2 v = refl_entry(xk, x, scal);
          P[o + x + (long)i * n] = v;
          P[o + x + (long)(2 * b + i) * n] = v;
        }
        continue;
      }
      if (task >= ntiles) {
        const int q2 = task - ntiles, q = q2 >> 1;
        const double2 *col = P + (long)((q2 & 1) ? q : b + q) * n;   // odd: V[:, q], even: W[:, q]
        double2 sacc = make_double2(0.0, 0.0);
        for (int x = threadIdx.x; x < m; x += blockDim.x) cmacc(sacc, col[o + x], refl_entry(xk, x, scal));
        sacc.x = block_sum(sacc.x, sh);
        sacc.y = block_sum(sacc.y, sh);
        if (threadIdx.x == 0) ucorr[q2] = sacc;
        continue;
      }
      int I = (int)((sqrtf(8.0f * task + 1.0f) - 1.0f) * 0.5f);
      while ((I + 1) * (I + 2) / 2 <= task) ++I;
      while (I * (I + 1) / 2 > task) --I;
      const int J = task - I * (I + 1) / 2;
      const int x0 = TT * I, y0 = TT * J;
      {
        const int wq = threadIdx.x >> 5, yc = y0 + rl;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = wq * 4 + q, xr = x0 + rr;
          double2 a = make_double2(0.0, 0.0);
          if (xr < m && yc < m && (I != J || yc <= xr)) a = A[(o + xr) + (long)(o + yc) * n];
          tile[rr][rl] = a;
        }
      }
      if (threadIdx.x < TT) {
        const int xr = x0 + threadIdx.x, yc = y0 + threadIdx.x;
        vrow[threadIdx.x] = xr < m ? refl_entry(xk, xr, scal) : make_double2(0.0, 0.0);
        vcol[threadIdx.x] = yc < m ? refl_entry(xk, yc, scal) : make_double2(0.0, 0.0);
      }
      __syncthreads();
      {
        const int k = g & 3;
        double2 sacc = make_double2(0.0, 0.0);
        if (threadIdx.x < 128) {
#pragma unroll
          for (int cl = 8 * k; cl < 8 * k + 8; ++cl) cmac(sacc, tile[rl][cl], vcol[cl]);
          rpart[k][rl] = sacc;
        } else {
#pragma unroll
          for (int rr = 8 * k; rr < 8 * k + 8; ++rr)
            if (I != J || rr > rl) cmacc(sacc, tile[rr][rl], vrow[rr]);
          cpart[k][rl] = sacc;
        }
      }
      __syncthreads();
      if (threadIdx.x < TT) {
        const int l = threadIdx.x;
        const double2 rs = cadd(cadd(rpart[0][l], rpart[1][l]), cadd(rpart[2][l], rpart[3][l]));
        const double2 cs = cadd(cadd(cpart[0][l], cpart[1][l]), cadd(cpart[2][l], cpart[3][l]));
        if (I != J) {
          if (x0 + l < m) part[(long)J * nmax + x0 + l] = rs;
          if (y0 + l < m) part[(long)I * nmax + y0 + l] = cs;
        } else if (x0 + l < m) {
          part[(long)J * nmax + x0 + l] = cadd(rs, cs);
        }
      }
      __syncthreads();
    }
    grid.sync();
    // ---- phase C: y = partial sums - V (W^H v) - W (V^H v), p = tau y, v in
    // place of x, partial dots p^H v
    ndot = (m + 31) / 32;
    double2 *xc = A + o + (long)c * n;
    for (int rb = blockIdx.x; rb < ndot; rb += nblk) {
      const int x = rb * 32 + rl;
      double2 y = make_double2(0.0, 0.0);
      if (x < m) {
        for (int q = g; q < nT; q += 8) y = cadd(y, __ldcg(&part[(long)q * nmax + x]));
#pragma unroll
        for (int t = 0; t < CO_QMAX; ++t) {
          const int q = g + 8 * t;
          if (q >= i) break;
          const double2 uw = __ldcg(&ucorr[2 * q]), uv = __ldcg(&ucorr[2 * q + 1]);
          cmac(y, P[o + x + (long)q * n], make_double2(-uw.x, -uw.y));         // - V[r,q] (W^H v)_q
          cmac(y, P[o + x + (long)(b + q) * n], make_double2(-uv.x, -uv.y));   // - W[r,q] (V^H v)_q
        }
      }
      s_u[g][rl] = y;
      __syncthreads();
      if (g == 0) {
        double2 pv = make_double2(0.0, 0.0);
        if (x < m) {
#pragma unroll
          for (int q = 1; q < 8; ++q) y = cadd(y, s_u[q][rl]);
          const double2 pr = cmul(tk, y);
          p[x] = pr;
          const double2 v = refl_entry(xc, x, scal);
          xc[x] = v;
          cmacc(pv, pr, v);
        }
        pv.x = warp_sum(pv.x);
        pv.y = warp_sum(pv.y);
        if (rl == 0) dotpart[rb] = pv;
      }
      __syncthreads();
    }
    grid.sync();
  }
  // W[:, b-1] = p + alpha v for the panel's last column
  {
    const int cl = j0 + b - 1, o = cl + 1;
    const double2 al = panel_alpha(dotpart, ndot, tk, sh);
    for (int r = o + blockIdx.x * blockDim.x + threadIdx.x; r < n; r += nblk * blockDim.x) {
      double2 w = __ldcg(&p[r - o]);
      cmac(w, al, A[r + (long)cl * n]);
      W[r + (long)(b - 1) * n] = w;
    }
  }
}

__global__ void k_last_diag_plain(const double2 *A, int n, double *d) {
  d[n - 1] = A[(n - 1) + (long)(n - 1) * n].x;
}

// ======================================================================
// divide and conquer on the symmetric tridiagonal (d, e)
// ======================================================================

// leaves of size 1: every boundary is a split, so d_i loses |e_{i-1}| + |e_i|
__global__ void k_dc_init(const double *d, const double *e, int n, double *lam, double *Z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = d[i];
  if (i > 0) v -= fabs(e[i - 1]);
  if (i < n - 1) v -= fabs(e[i]);
  lam[i] = v;
}
__global__ void k_identity(double *Z, int n) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  Z[idx] = (idx % n == idx / n) ? 1.0 : 0.0;
}

struct DcArrays {
  double *lam, *Z, *W, *U;
  double *Ds, *zs, *DK, *zK, *tauK, *zh, *lamK, *dD, *lnew;
  int *perm, *colK, *orig, *dcol, *src, *defl;
  int *knode;
  double *rhonode;
  int *ctype, *qL, *qR, *kLR, *kneed;
};

// exclusive prefix over the block of per-thread counts (blockDim <= 256);
// returns this thread's offset, *total the sum
__device__ int block_excl_scan(int v, int *s_scan, int *total) {
  __syncthreads();
  s_scan[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int c = s_scan[t];
      s_scan[t] = acc;
      acc += c;
    }
    s_scan[blockDim.x] = acc;
  }
  __syncthreads();
  *total = s_scan[blockDim.x];
  return s_scan[threadIdx.x];
}

// sort, z-vector, deflation and compaction for one node per CTA.  The merge
// of the two sorted halves places each value by its rank in the other half
// (ties: left first); the deflation scan (each decision depends on the
// previous surviving index) runs on one thread over the node's arrays and
// records its rotations, which the block then applies in order; the
// compactions are block-wide prefix sums.
__global__ void __launch_bounds__(256) k_dc_deflate(const int *nodes, int n, const double *e,
                                                    DcArrays a) {
  __shared__ double sh[32];
  __shared__ int s_scan[257];
  __shared__ int s_nrot;
  const int node = blockIdx.x;
  const int lo = nodes[3 * node], mid = nodes[3 * node + 1], hi = nodes[3 * node + 2];
  const int size = hi - lo, m1 = mid - lo;
  const double beta = e[mid - 1];
  const double rho = fabs(beta), sgn = beta >= 0.0 ? 1.0 : -1.0;
  // 1. merge: left value -> its index + #(right < v); right -> index + #(left <= v)
  for (int p = threadIdx.x; p < size; p += blockDim.x) {
    const double v = a.lam[lo + p];
    int out;
    if (p < m1) {
      int l = 0, r = size - m1;
      while (l < r) {
        const int mm = (l + r) >> 1;
        if (a.lam[lo + m1 + mm] < v) l = mm + 1; else r = mm;
      }
      out = p + l;
    } else {
      int l = 0, r = m1;
      while (l < r) {
        const int mm = (l + r) >> 1;
        if (a.lam[lo + mm] <= v) l = mm + 1; else r = mm;
      }
      out = (p - m1) + l;
    }
    a.perm[lo + out] = p;
  }
  __syncthreads();
  double dmax = 0.0;
  for (int c = lo + threadIdx.x; c < hi; c += blockDim.x) a.ctype[c] = c < mid ? 0 : 1;
  for (int p = threadIdx.x; p < size; p += blockDim.x) {
    const int li = a.perm[lo + p];
    const double Dv = a.lam[lo + li];
    const double z = li < m1 ? a.Z[(mid - 1) + (long)(lo + li) * n]
                             : sgn * a.Z[mid + (long)(lo + li) * n];
    a.Ds[lo + p] = Dv;
    a.zs[lo + p] = z * 0.70710678118654752440;
    a.defl[lo + p] = 0;
    dmax = fmax(dmax, fabs(Dv));
  }
  dmax = block_max(dmax, sh);
  const double rho2 = 2.0 * rho;
  const double tol = 8.0 * kEps * fmax(dmax, rho2);
  // 2. deflation scan; rotation list in this node's own columns of W (W is
  // rewritten by k_dc_gemm later in the level)
  double *rot = a.W + (long)lo * n;
  if (threadIdx.x == 0) {
    int prev = -1, nrot = 0;
    for (int p = 0; p < size; ++p) {
      const double zp = a.zs[lo + p];
      if (rho2 * fabs(zp) <= tol) { a.defl[lo + p] = 1; continue; }
      if (prev >= 0) {
        const int j = prev;
        const double zj = a.zs[lo + j];
        const double r = hypot(zp, zj);
        const double c = zp / r, s = -zj / r;
        const double Dj = a.Ds[lo + j], Dp = a.Ds[lo + p];
        if (fabs(c * s * (Dp - Dj)) <= tol) {
          const int cj = lo + a.perm[lo + j], ci = lo + a.perm[lo + p];
          if (a.ctype[cj] != a.ctype[ci]) a.ctype[cj] = a.ctype[ci] = 2;
          rot[4 * nrot] = cj;
          rot[4 * nrot + 1] = ci;
          rot[4 * nrot + 2] = c;
          rot[4 * nrot + 3] = s;
          ++nrot;
          a.Ds[lo + j] = c * c * Dj + s * s * Dp;
          a.Ds[lo + p] = s * s * Dj + c * c * Dp;
          a.zs[lo + j] = 0.0;
          a.zs[lo + p] = r;
          a.defl[lo + j] = 1;
        }
      }
      prev = p;
    }
    s_nrot = nrot;
  }
  __syncthreads();
  const int nrot = s_nrot;
  for (int k = 0; k < nrot; ++k) {           // in order: a column may take part in two
    const int cj = (int)rot[4 * k], ci = (int)rot[4 * k + 1];
    const double c = rot[4 * k + 2], s = rot[4 * k + 3];
    double *Qj = a.Z + (long)cj * n, *Qi = a.Z + (long)ci * n;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
      const double qj = Qj[r], qi = Qi[r];
      Qj[r] = c * qj + s * qi;
      Qi[r] = -s * qj + c * qi;
    }
    __syncthreads();
  }
  // 3. compaction: survivors -> (DK, zK, colK), deflated -> (dD, dcol), in order
  const bool all_defl = !(rho2 > 0.0);   // no coupling: everything deflates
  const int chunk = (size + blockDim.x - 1) / blockDim.x;
  const int p0 = min(size, (int)threadIdx.x * chunk), p1 = min(size, p0 + chunk);
  int cnt = 0;
  for (int p = p0; p < p1; ++p) cnt += (!all_defl && !a.defl[lo + p]);
  int k_total;
  int t = block_excl_scan(cnt, s_scan, &k_total);
  int q = p0 - t;
  for (int p = p0; p < p1; ++p) {
    const int col = lo + a.perm[lo + p];
    if (!all_defl && !a.defl[lo + p]) {
      a.DK[lo + t] = a.Ds[lo + p];
      a.zK[lo + t] = a.zs[lo + p];
      a.colK[lo + t] = col;
      ++t;
    } else {
      a.dD[lo + q] = a.Ds[lo + p];
      a.dcol[lo + q] = col;
      ++q;
    }
  }
  __syncthreads();
  // root columns the upper rows need (types 0, 2) and the lower rows (2, 1)
  const int kk = k_total;
  const int c0 = min(kk, (int)threadIdx.x * ((kk + blockDim.x - 1) / blockDim.x));
  const int c1 = min(kk, c0 + (kk + blockDim.x - 1) / blockDim.x);
  int nl = 0, nr = 0;
  for (int q2 = c0; q2 < c1; ++q2) {
    const int ty = a.ctype[a.colK[lo + q2]];
    nl += ty != 1;
    nr += ty != 0;
  }
  int nl_total, nr_total;
  int ol = block_excl_scan(nl, s_scan, &nl_total);
  int orr = block_excl_scan(nr, s_scan, &nr_total);
  for (int q2 = c0; q2 < c1; ++q2) {
    const int ty = a.ctype[a.colK[lo + q2]];
    if (ty != 1) a.qL[lo + ol++] = q2;
    if (ty != 0) a.qR[lo + orr++] = q2;
  }
  if (threadIdx.x == 0) {
    a.knode[node] = kk;
    a.kLR[2 * node] = nl_total;
    a.kLR[2 * node + 1] = nr_total;
    a.kneed[node] = 0;
    a.rhonode[node] = rho2;
  }
}

// one warp per root t of the secular equation 1 + rho sum z_i^2 / (D_i - lam) = 0
__global__ void __launch_bounds__(256) k_dc_roots(const int *nodes, DcArrays a) {
  const int node = blockIdx.y;
  const int lo = nodes[3 * node];
  const int k = a.knode[node];
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= k) return;
  const double rho = a.rhonode[node];
  const double *D = a.DK + lo, *z = a.zK + lo;
  int o;
  double blo, bhi;
  if (t < k - 1) {
    const double half = 0.5 * (D[t + 1] - D[t]);
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s += z[i] * z[i] / ((D[i] - D[t]) - half);
    s = warp_sum(s);
    if (1.0 + rho * s >= 0.0) { o = t; blo = 0.0; bhi = half; }
    else { o = t + 1; blo = -half; bhi = 0.0; }
  } else {
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s += z[i] * z[i];
    s = warp_sum(s);
    o = t; blo = 0.0; bhi = rho * s;
  }
  const double Do = D[o];
  const double da = D[t] - Do;                          // left pole
  const double db = (t < k - 1) ? D[t + 1] - Do : 0.0;  // right pole (if any)
  double tau = 0.5 * (blo + bhi);
  for (int it = 0; it < 100; ++it) {
    double psi = 0.0, dpsi = 0.0, phi = 0.0, dphi = 0.0;
    for (int i = lane; i < k; i += 32) {
      // one reciprocal per term (FP64 divisions are the costly part here)
      const double r = __drcp_rn((D[i] - Do) - tau);
      const double term = z[i] * z[i] * r;
      if (i <= t) { psi += term; dpsi = fma(term, r, dpsi); }
      else { phi += term; dphi = fma(term, r, dphi); }
    }
    psi = rho * warp_sum(psi);
    dpsi = rho * warp_sum(dpsi);
    phi = rho * warp_sum(phi);
    dphi = rho * warp_sum(dphi);
    const double f = 1.0 + psi + phi;
    if (f < 0.0) blo = fmax(blo, tau); else bhi = fmin(bhi, tau);
    if (f == 0.0 || bhi - blo <= 4.0 * kEps * fmax(fabs(blo), fabs(bhi))) break;
    const double q = dpsi * (da - tau) * (da - tau);
    const double pp = psi - dpsi * (da - tau);
    double x;
    if (t < k - 1) {
      const double s = dphi * (db - tau) * (db - tau);
      const double r = phi - dphi * (db - tau);
      const double Cc = 1.0 + pp + r;
      const double A2 = Cc, B2 = -(Cc * (da + db) + q + s), C2 = Cc * da * db + q * db + s * da;
      x = 0.5 * (blo + bhi);
      if (A2 == 0.0) {
        if (B2 != 0.0) x = -C2 / B2;
      } else {
        const double disc = fmax(B2 * B2 - 4.0 * A2 * C2, 0.0);
        const double sq = sqrt(disc);
        const double r1 = (B2 >= 0.0) ? (-B2 - sq) / (2.0 * A2) : (-B2 + sq) / (2.0 * A2);
        const double r2 = (r1 != 0.0) ? C2 / (A2 * r1) : r1;
        if (r1 > da && r1 < db) x = r1;
        else if (r2 > da && r2 < db) x = r2;
      }
    } else {
      const double Cc = 1.0 + pp + phi;
      x = (Cc > 0.0) ? da + q / Cc : 0.5 * (blo + bhi);
    }
    if (!(x > blo && x < bhi)) x = 0.5 * (blo + bhi);
    if (fabs(x - tau) <= 2.0 * kEps * fabs(x)) { tau = x; break; }
    tau = x;
  }
  if (lane == 0) {
    a.orig[lo + t] = o;
    a.tauK[lo + t] = tau;
    a.lamK[lo + t] = Do + tau;
  }
}

// Lowner: rho zh_i^2 = prod_j (lam_j - D_i) / prod_{j != i} (D_j - D_i)
__global__ void __launch_bounds__(256) k_dc_zhat(const int *nodes, DcArrays a) {
  const int node = blockIdx.y;
  const int lo = nodes[3 * node];
  const int k = a.knode[node];
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= k) return;
  const double *D = a.DK + lo;
  const double Di = D[i];
  double prod = 1.0;
  for (int j = lane; j < k; j += 32) {
    const double num = (D[a.orig[lo + j]] - Di) + a.tauK[lo + j];
    prod *= (j == i) ? num : num / (D[j] - Di);
  }
  prod = warp_prod(prod);
  if (lane == 0) {
    const double zi = a.zK[lo + i];
    a.zh[lo + i] = copysign(sqrt(fmax(prod, 0.0) / a.rhonode[node]), zi);
  }
}

// eigenvectors of the secular problem: u_t[i] = zh_i / (D_i - lam_t), normalised
__global__ void __launch_bounds__(256) k_dc_vectors(const int *nodes, int n, DcArrays a) {
  const int node = blockIdx.y;
  const int lo = nodes[3 * node];
  const int k = a.knode[node];
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= k) return;
  const double *D = a.DK + lo;
  const double Do = D[a.orig[lo + t]], tau = a.tauK[lo + t];
  double s = 0.0;
  for (int i = lane; i < k; i += 32) {
    const double u = a.zh[lo + i] / ((D[i] - Do) - tau);
    s += u * u;
  }
  const double inv = 1.0 / sqrt(warp_sum(s));
  double *Ucol = a.U + (long)(lo + t) * n + lo;
  for (int i = lane; i < k; i += 32) Ucol[i] = inv * a.zh[lo + i] / ((D[i] - Do) - tau);
}

// W[rows, lo + t] = Z[rows, colK] U[:, t]  (node rows lo..hi-1).  Z is block
// diagonal apart from the columns a deflating rotation mixed, so row tiles of
// the upper half run over the root columns qL only, those of the lower half
// over qR; only the roots t < kneed are formed.
__global__ void __launch_bounds__(256) k_dc_gemm(const int *nodes, int n, DcArrays a) {
  const int node = blockIdx.z;
  const int lo = nodes[3 * node], mid = nodes[3 * node + 1], hi = nodes[3 * node + 2];
  const int tl = (mid - lo + 63) / 64;
  const bool upper = (int)blockIdx.x < tl;
  const int rbeg = upper ? lo + (int)blockIdx.x * 64 : mid + ((int)blockIdx.x - tl) * 64;
  const int rend = upper ? mid : hi;
  const int kneed = a.kneed[node];
  const int t0 = blockIdx.y * 64;
  if (rbeg >= rend || t0 >= kneed) return;
  const int *ql = upper ? a.qL + lo : a.qR + lo;
  const int kq = a.kLR[2 * node + (upper ? 0 : 1)];
  __shared__ double As[16][65], Bs[16][65];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < kq; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e & 63, kk = e >> 6;
      double v = 0.0;
      if (rbeg + r < rend && k0 + kk < kq) v = a.Z[(rbeg + r) + (long)a.colK[lo + ql[k0 + kk]] * n];
      As[kk][r] = v;
      const int kb = e & 15, tt = e >> 4;
      double u = 0.0;
      if (k0 + kb < kq && t0 + tt < kneed) u = a.U[(lo + ql[k0 + kb]) + (long)(lo + t0 + tt) * n];
      Bs[kb][tt] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = As[kk][tx + 16 * q]; bv[q] = Bs[kk][ty + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] = fma(av[q], bv[r], acc[q][r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = rbeg + tx + 16 * q, t = t0 + ty + 16 * r;
      if (row < rend && t < kneed) a.W[row + (long)(lo + t) * n] = acc[q][r];
    }
}

// The merge product of k_dc_gemm for one node and half (upper rows lo..mid
// or lower rows mid..hi) as a dense real product on zero-padded operands, for
// the FP64-accurate tensor-core path: Zg[r, k] = Z[row0 + r, colK[lo + ql[k]]]
// (k < kq), Ug[k, t] = U[lo + ql[k], lo + t] (k < kq, t < kneed), zero beyond;
// kq and kneed stay on the device (kmax, tmax bound them)
__global__ void k_dc_gather_z(int lo, int mid, int hi, int node, int half, int n, DcArrays a, int kmax,
                              double *Zg) {
  const int rows = half ? hi - mid : mid - lo, row0 = half ? mid : lo;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)rows * kmax) return;
  const int r = (int)(idx % rows), k = (int)(idx / rows);
  const int kq = a.kLR[2 * node + half];
  const int *ql = (half ? a.qR : a.qL) + lo;
  Zg[idx] = k < kq ? a.Z[(row0 + r) + (long)a.colK[lo + ql[k]] * n] : 0.0;
}
__global__ void k_dc_gather_u(int lo, int node, int half, int n, DcArrays a, int kmax, int tmax, double *Ug) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)kmax * tmax) return;
  const int k = (int)(idx % kmax), t = (int)(idx / kmax);
  const int kq = a.kLR[2 * node + half], kneed = a.kneed[node];
  const int *ql = (half ? a.qR : a.qL) + lo;
  Ug[idx] = (k < kq && t < kneed) ? a.U[(lo + ql[k]) + (long)(lo + t) * n] : 0.0;
}
// W[row0 + r, lo + t] = Wt[r, t] for t < kneed (k_dc_gemm's output columns)
__global__ void k_dc_scatter_w(int lo, int mid, int hi, int node, int half, int n, DcArrays a, int tmax,
                               const double *Wt) {
  const int rows = half ? hi - mid : mid - lo, row0 = half ? mid : lo;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)rows * tmax) return;
  const int r = (int)(idx % rows), t = (int)(idx / rows);
  if (t < a.kneed[node]) a.W[(row0 + r) + (long)(lo + t) * n] = Wt[idx];
}

// final order: rank of each (value, source index) among the node's eigenvalues;
// kneed = roots among the `keep` lowest (the roots are in increasing order)
__global__ void k_dc_rank(const int *nodes, DcArrays a, int keep) {
  const int node = blockIdx.y;
  const int lo = nodes[3 * node], hi = nodes[3 * node + 2];
  const int size = hi - lo, k = a.knode[node];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= size) return;
  const double v = e < k ? a.lamK[lo + e] : a.dD[lo + e - k];
  int rank = 0;
  for (int f = 0; f < size; ++f) {
    const double w = f < k ? a.lamK[lo + f] : a.dD[lo + f - k];
    rank += (w < v) || (w == v && f < e);
  }
  a.lnew[lo + rank] = v;
  a.src[lo + rank] = lo + e;     // W column: roots at lo..lo+k-1, deflated copied after them
  if (e < k && rank < keep) atomicMax(&a.kneed[node], e + 1);
}

// copy deflated columns of Z into W after the roots' columns
__global__ void k_dc_copy_defl(const int *nodes, int n, DcArrays a) {
  const int node = blockIdx.y;
  const int lo = nodes[3 * node], hi = nodes[3 * node + 2];
  const int size = hi - lo, k = a.knode[node];
  const int q = blockIdx.x;
  if (q >= size - k) return;
  const double *src = a.Z + (long)a.dcol[lo + q] * n;
  double *dst = a.W + (long)(lo + k + q) * n;
  for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) dst[r] = src[r];
}

__global__ void k_dc_write(const int *nodes, int n, DcArrays a, int keep) {
  const int node = blockIdx.y;
  const int lo = nodes[3 * node], hi = nodes[3 * node + 2];
  const int p = blockIdx.x;
  if (p >= hi - lo) return;
  if (threadIdx.x == 0) a.lam[lo + p] = a.lnew[lo + p];
  if (p >= keep) return;   // every eigenvalue, only the kept vectors
  const double *src = a.W + (long)a.src[lo + p] * n;
  double *dst = a.Z + (long)(lo + p) * n;
  for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) dst[r] = src[r];
}

// ======================================================================
// back-transformation  Y = H_0 H_1 ... H_{n-2} Z
// ======================================================================
__global__ void k_bt_init(const double *Z, int n, int nb, double2 *Y) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)n * nb) return;
  Y[idx] = make_double2(Z[idx], 0.0);
}

constexpr int BTB = 128;  // reflectors per compact-WY block

// Vb (mb x b, ld mb) = reflectors j0..j0+b-1 with explicit zeros above their unit
// entries; reflector j lives in A[j+1:, j] and Vb row q is matrix row j0+1+q
__global__ void k_copy_panel(const double2 *A, int n, int j0, int b, double2 *Vb, int mb) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)mb * b) return;
  const int q = (int)(idx % mb), c = (int)(idx / mb);
  const int row = j0 + 1 + q, j = j0 + c;
  Vb[idx] = row >= j + 1 ? A[row + (long)j * n] : make_double2(0.0, 0.0);
}

// T (b x b, upper, ld b): T_ii = tau_i; T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i],
// G = Vb^H Vb.  Row r of T depends only on itself (T[r, i] = -tau_i
// sum_{m=r}^{i-1} T[r, m] G[m, i]), so each warp owns one row: the lanes split
// the sum, the row is kept in shared memory, and the next column of G is
// fetched while the current one is reduced.
constexpr int BT_WARPS = 4;
__global__ void __launch_bounds__(32 * BT_WARPS) k_build_T(const double2 *G, const double2 *tau, int j0, int b,
                                                           double2 *T) {
  __shared__ double2 trow[BT_WARPS][BTB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * BT_WARPS + w;
  if (r >= b) return;
  double2 *tr = trow[w];
  constexpr int KMAX = BTB / 32;
  double2 gnext[KMAX];
  auto fetch = [&](int col) {
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int m = r + lane + 32 * k;
      gnext[k] = (col < b && m < col) ? G[m + (long)col * b] : make_double2(0.0, 0.0);
    }
  };
  if (lane == 0) tr[r] = tau[j0 + r];
  fetch(r + 1);
  __syncwarp();
  for (int c = r + 1; c < b; ++c) {
    double2 g[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) g[k] = gnext[k];
    fetch(c + 1);
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int m = r + lane + 32 * k;
      if (m < c) cmac(s, tr[m], g[k]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    if (lane == 0) {
      const double2 t = cmul(tau[j0 + c], s);
      tr[c] = make_double2(-t.x, -t.y);
    }
    __syncwarp();
  }
  for (int c = lane; c < b; c += 32) T[r + (long)c * b] = c >= r ? tr[c] : make_double2(0.0, 0.0);
}

void build_tree(pw_dense_ws *ws, int n, cudaStream_t st) {
  ws->levels.clear();
  std::function<void(int, int, int)> rec = [&](int lo, int hi, int depth) {
    if (hi - lo <= 1) return;
    const int mid = lo + (hi - lo) / 2;
    if ((int)ws->levels.size() <= depth) ws->levels.resize(depth + 1);
    ws->levels[depth].push_back(lo);
    ws->levels[depth].push_back(mid);
    ws->levels[depth].push_back(hi);
    rec(lo, mid, depth + 1);
    rec(mid, hi, depth + 1);
  };
  rec(0, n, 0);
  ws->level_off.assign(ws->levels.size(), 0);
  std::vector<int> flat;
  ws->max_level_nodes = 0;
  for (size_t l = 0; l < ws->levels.size(); ++l) {
    ws->level_off[l] = (int)flat.size() / 3;
    flat.insert(flat.end(), ws->levels[l].begin(), ws->levels[l].end());
    ws->max_level_nodes = std::max(ws->max_level_nodes, (int)ws->levels[l].size() / 3);
  }
  // ordered on the solve's stream (after the kernels that read the previous
  // tree, before the ones that read this one)
  if (!flat.empty()) {
    cudaMemcpyAsync(ws->nodes, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  ws->tree_n = n;
}

}  // namespace

// ======================================================================
// products of the dense solve
// ======================================================================
int pw_dense_products_mode() { return pw_f64_products_mode(); }

pw_status pw_dense_gemm(pw_dense_ws *ws, char opA, char opB, int m, int n, int k, double2 alpha,
                        const double2 *A, int lda, const double2 *B, int ldb, double2 beta, double2 *C,
                        int ldc, cudaStream_t st, int herm) {
  if (m <= 0 || n <= 0) return PW_OK;
  if (pw_use_oz(m, n, k)) {
    if (ws->oz.bytes == 0) {
      // reserve the largest product of an order-nmax solve at once (the
      // L^-1 A L^-H blocks and C = M Y), so later products reuse it
      const size_t big = std::max(pw_oz_ws_bytes(256, ws->nmax, ws->nmax),
                                  std::max(pw_oz_ws_bytes(ws->nmax, 256, ws->nmax),
                                           pw_oz_ws_bytes(ws->nmax, ws->nbmax, ws->nmax)));
      void *p = nullptr;
      if (cudaMalloc(&p, big) == cudaSuccess) { ws->oz.buf = p; ws->oz.bytes = big; ++ws->oz.gen; }
      else cudaGetLastError();
    }
    return pw_zgemm_oz(&ws->oz, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st, herm);
  }
  return pw_zgemm_ex(opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws->gemm_ws, ws->gemm_ws_elems,
                     st, herm);
}

// ======================================================================
// workspace
// ======================================================================
pw_status pw_dense_alloc(pw_dense_ws *ws, int nmax, int nbmax) {
  if (ws->nmax >= nmax && ws->nbmax >= nbmax) return PW_OK;
  pw_dense_free(ws);
  const size_t n2 = (size_t)nmax * nmax;
  size_t total = 0;
  auto get = [&](void **p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return false; }
    total += bytes;
    return true;
  };
  bool ok = get((void **)&ws->G, n2 * 16) && get((void **)&ws->A, n2 * 16) &&
            get((void **)&ws->T, n2 * 16) && get((void **)&ws->Linv, n2 * 16) &&
            get((void **)&ws->Y, (size_t)nmax * nbmax * 16) &&
            get((void **)&ws->dscale, nmax * 8) && get((void **)&ws->piv, nmax * 8) &&
            get((void **)&ws->flag, 64) && get((void **)&ws->d, nmax * 8) &&
            get((void **)&ws->e, nmax * 8) && get((void **)&ws->lam, nmax * 8) &&
            get((void **)&ws->tau, nmax * 16) && get((void **)&ws->p, nmax * 16) &&
            get((void **)&ws->w, nmax * 16) &&
            get((void **)&ws->part, (size_t)((nmax + TT - 1) / TT) * nmax * 16) &&
            get((void **)&ws->Z, n2 * 8) && get((void **)&ws->W, n2 * 8) && get((void **)&ws->U, n2 * 8);
  double **dbl[] = {&ws->Ds, &ws->zs, &ws->DK, &ws->zK, &ws->tauK, &ws->zh, &ws->lamK, &ws->dD, &ws->lnew};
  for (double **q : dbl) ok = ok && get((void **)q, nmax * 8);
  int **ints[] = {&ws->perm, &ws->colK, &ws->orig, &ws->dcol, &ws->src};
  for (int **q : ints) ok = ok && get((void **)q, nmax * 4);
  ok = ok && get((void **)&ws->nodes, (size_t)3 * nmax * 4 + 64) &&
       get((void **)&ws->knode, (size_t)nmax * 4 + 64) &&
       get((void **)&ws->rhonode, (size_t)nmax * 8 + 64) && get((void **)&ws->ctype, (size_t)nmax * 4) &&
       get((void **)&ws->qL, (size_t)nmax * 4) && get((void **)&ws->qR, (size_t)nmax * 4) &&
       get((void **)&ws->kLR, (size_t)nmax * 8 + 64) && get((void **)&ws->kneed, (size_t)nmax * 4 + 64);
  ok = ok && get((void **)&ws->ticket, 64) && get((void **)&ws->panel, (size_t)nmax * 3 * TPB * 16) &&
       get((void **)&ws->ucorr, 2 * TPB * 16) && get((void **)&ws->hscal, 16) && get((void **)&ws->Li, CB * CB * 16) &&
       get((void **)&ws->nrm_part, (size_t)(nmax / 32 + 2) * 8) &&
       get((void **)&ws->hsmax, (size_t)(nmax / TPB + 2) * 8);
  if (ok && pw_hs_bytes(nmax)) {
    // zeroed once: a slice tile is only read where the panel's slicing wrote it
    ok = get(&ws->hsl, pw_hs_bytes(nmax)) && cudaMemset(ws->hsl, 0, pw_hs_bytes(nmax)) == cudaSuccess;
  }
  if (ok && !ws->oz.err) {
    ok = cudaMalloc((void **)&ws->oz.err, 16) == cudaSuccess && cudaMemset(ws->oz.err, 0, 16) == cudaSuccess;
    if (!ok) { cudaGetLastError(); ws->oz.err = nullptr; }
  }
  ok = ok && get((void **)&ws->Vb, (size_t)nmax * BTB * 16) && get((void **)&ws->Gv, BTB * BTB * 16) &&
       get((void **)&ws->Tb, BTB * BTB * 16) && get((void **)&ws->Wk, (size_t)BTB * nbmax * 16) &&
       get((void **)&ws->Wk2, (size_t)BTB * nbmax * 16);
  ws->gemm_ws_elems = std::max(pw_zgemm_ws_elems(nmax, nmax, nmax), pw_zgemm_ws_elems(nmax, nbmax, nmax));
  ws->gemm_ws_elems = std::max(ws->gemm_ws_elems, pw_zgemm_ws_elems(BTB, nbmax, nmax));
  ws->gemm_ws_elems = std::max(ws->gemm_ws_elems, pw_zgemm_ws_elems(BTB, BTB, nmax));
  if (ok && ws->gemm_ws_elems) ok = get((void **)&ws->gemm_ws, ws->gemm_ws_elems * 16);
  if (!ok) { pw_dense_free(ws); return PW_ERR_OOM; }
  for (cudaEvent_t &e : ws->ev)
    if (!e && cudaEventCreate(&e) != cudaSuccess) { pw_dense_free(ws); return PW_ERR_CUDA; }
  ws->nmax = nmax;
  ws->nbmax = nbmax;
  ws->bytes = total;
  ws->tree_n = -1;
  return PW_OK;
}

void pw_dense_free(pw_dense_ws *ws) {
  for (auto &g : ws->graphs) cudaGraphExecDestroy(g.exec);
  ws->graphs.clear();
  pw_oz_free(&ws->oz);
  void *ptrs[] = {ws->G, ws->A, ws->T, ws->Linv, ws->Y, ws->dscale, ws->piv, ws->flag, ws->d, ws->e,
                  ws->lam, ws->tau, ws->p, ws->w, ws->part, ws->Z, ws->W, ws->U, ws->Ds, ws->zs,
                  ws->DK, ws->zK, ws->tauK, ws->zh, ws->lamK, ws->dD, ws->lnew, ws->perm, ws->colK,
                  ws->orig, ws->dcol, ws->src, ws->nodes, ws->knode, ws->rhonode, ws->ctype, ws->qL, ws->qR,
                  ws->kLR, ws->kneed, ws->gemm_ws,
                  ws->Vb, ws->Gv, ws->Tb, ws->Wk, ws->Wk2, ws->ticket, ws->panel, ws->ucorr,
                  ws->hscal, ws->nrm_part, ws->Li, ws->hsl, ws->hsmax};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : ws->ev)
    if (e) cudaEventDestroy(e);
  *ws = pw_dense_ws();
}

void pw_dense_stage_ms(pw_dense_ws *ws, float out[5]) {
  for (int i = 0; i < 5; ++i) {
    out[i] = 0.0f;
    if (ws->ev[i] && ws->ev[i + 1]) cudaEventElapsedTime(&out[i], ws->ev[i], ws->ev[i + 1]);
  }
}

// ======================================================================
// Hermitian eigensolver
// ======================================================================
// Cooperative grids fill the device; two of them partly resident at once
// (concurrent solves on other streams) could each wait at a grid barrier for
// blocks that only the other's exit would make room for.  So every
// cooperative launch on a device is ordered after the previous one, through
// one event recorded behind each launch (host mutex, then stream wait).
pw_status pw_coop_ordered(cudaStream_t st, const std::function<pw_status()> &launch) {
  static std::mutex mu;
  static cudaEvent_t last[64] = {};
  int dev = 0;
  PW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return PW_ERR_ARG;
  std::lock_guard<std::mutex> lk(mu);
  if (!last[dev]) PW_CUDA(cudaEventCreateWithFlags(&last[dev], cudaEventDisableTiming));
  else PW_CUDA(cudaStreamWaitEvent(st, last[dev], 0));
  PW_TRY(launch());
  PW_CUDA(cudaEventRecord(last[dev], st));
  return PW_OK;
}

namespace {
// The three stages of the eigensolver, each a fixed launch sequence for a
// given (n, nb) on a given workspace (so each can be captured as a graph).
// measured slower than the chained kernels at n = 3,456 (277 against 204 ms:
// two 256-thread blocks per SM leave the FP64 pipe short of warps, and
// three grid barriers per column cost more than PDL's launch overlap)
std::atomic<int> g_coop{0};

// grid of the cooperative panel kernel on the current device (0: not
// available): blocks that fit at once, at most two per SM
int coop_grid() {
  static std::mutex mu;
  static int grid[64];
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    int coop = 0, sms = 0, per = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_panel_coop, CO_THREADS, 0) != cudaSuccess) {
      cudaGetLastError();
      per = 0;
    }
    grid[dev] = coop ? std::min(per, 2) * sms : 0;
    done[dev] = true;
  }
  return grid[dev];
}

pw_status launch_panel_coop(cudaLaunchConfig_t &cfg, double2 *A, int n, int j0, int b, pw_dense_ws *ws) {
  return pw_coop_ordered(cfg.stream, [&]() -> pw_status {
    pw_count_launch();
    PW_CUDA(cudaLaunchKernelEx(&cfg, k_panel_coop, A, n, j0, b, ws->panel, ws->p, ws->w, ws->tau, ws->d, ws->e,
                               ws->nrm_part, ws->hscal, ws->part, ws->nmax, ws->ucorr));
    return PW_OK;
  });
}

// the reduction with one cooperative launch per panel (three grid barriers
// per column) and the panel's rank-64 update
pw_status tridiag_coop(pw_dense_ws *ws, int n, double2 *A, int grid, cudaStream_t st) {
  const double2 mone = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
  for (int j0 = 0; j0 + 1 < n; j0 += TPB) {
    const int b = std::min(TPB, n - 1 - j0);
    PW_CUDA(cudaMemsetAsync(ws->panel, 0, (size_t)n * 3 * b * sizeof(double2), st));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(CO_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PW_TRY(launch_panel_coop(cfg, A, n, j0, b, ws));
    const int t = j0 + b, m2 = n - t;
    if (m2 > 0)
      PW_TRY(pw_dense_gemm(ws, 'N', 'C', m2, m2, 2 * b, mone, ws->panel + t, n, ws->panel + (long)b * n + t, n,
                           one, A + t + (long)t * n, n, st, 2));
  }
  pw_count_launch();
  k_last_diag_plain<<<1, 1, 0, st>>>(A, n, ws->d);
  return pw_check_launch("tridiag (cooperative panels)");
}

pw_status stage_tridiag(pw_dense_ws *ws, int n, double2 *A, cudaStream_t st) {
  const int mode = g_coop.load();
  const int grid = mode == 1 ? coop_grid() : 0;
  if (grid > 0) return tridiag_coop(ws, n, A, grid, st);
  // Hermitian products on the tensor cores for the panels of trailing order
  // >= PW_HS_MIN_ORDER (slices of each such panel's trailing matrix first):
  // chained per column (mode 0) or one cooperative launch per panel (mode 3)
  const bool hs = (mode == 0 || mode == 3) && ws->hsl && pw_dense_products_mode() == 1 &&
                  n - 1 >= PW_HS_MIN_ORDER;
  const int hgrid = hs && mode == 3 ? pw_hs_panel_grid() : 0;
  // 1. Householder tridiagonalisation: panels of TPB columns (lower triangle)
  PW_CUDA(cudaMemsetAsync(ws->ticket, 0, sizeof(unsigned), st));
  if (hs) PW_CUDA(cudaMemsetAsync(ws->hsmax, 0, (size_t)(n / TPB + 2) * 8, st));
  {
    const double2 mone = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
    double2 *dotpart = ws->w;
    for (int j0 = 0; j0 + 1 < n; j0 += TPB) {
      const int b = std::min(TPB, n - 1 - j0);
      const bool ptc = hs && n - j0 - 1 >= PW_HS_MIN_ORDER;
      PW_CUDA(cudaMemsetAsync(ws->panel, 0, (size_t)n * 3 * b * sizeof(double2), st));
      if (ptc) PW_TRY(pw_hs_slice(ws, A, n, j0, st));
      if (ptc && hgrid > 0) {
        PW_TRY(pw_hs_panel(ws, A, n, j0, b, hgrid, st));
        const int t = j0 + b, m2 = n - t;
        if (m2 > 0)
          PW_TRY(pw_dense_gemm(ws, 'N', 'C', m2, m2, 2 * b, mone, ws->panel + t, n, ws->panel + (long)b * n + t,
                               n, one, A + t + (long)t * n, n, st, 2));
        continue;
      }
      int ndot = 0;
      for (int i = 0; i < b; ++i) {
        const int c = j0 + i, m = n - c - 1;
        const int npcol = (n - c + 31) / 32;
        pw_count_launch();
        PW_CUDA(launch_pdl(k_pcol, npcol, PCOL_THREADS, st, A, n, c, i, ws->panel, b,
                           (const double2 *)ws->p, (const double2 *)dotpart, ndot, ws->tau, ws->d, ws->e,
                           ws->nrm_part, ws->hscal, ws->ticket));
        int s0 = 0, nT = (m + TT - 1) / TT;
        const double2 *part = ws->part;
        if (ptc) {
          PW_TRY(pw_hs_hemv(ws, A, n, c, i, b, j0, &nT, st));
          part = ws->part + (c + 1);
        } else {
          const int ntiles = nT * (nT + 1) / 2, nwr = (m + 255) / 256;
          pw_count_launch();
          PW_CUDA(launch_pdl(k_phemv, ntiles + 2 * i + nwr, 256, st, (const double2 *)A, n, c, i, ws->panel,
                             b, ntiles, ws->part, ws->nmax, ws->ucorr, (const double2 *)ws->hscal));
        }
        ndot = (m + 31) / 32;
        pw_count_launch();
        PW_CUDA(launch_pdl(k_prows, ndot, 256, st, A, n, c, i, (const double2 *)ws->panel, b, part, s0, nT,
                           ws->nmax, (const double2 *)ws->ucorr, (const double2 *)ws->tau,
                           (const double2 *)ws->hscal, ws->p, dotpart));
      }
      const int cl = j0 + b - 1, ml = n - cl - 1;
      pw_count_launch();
      PW_CUDA(launch_pdl(k_pfinal, (ml + 255) / 256, 256, st, (const double2 *)A, n, cl, b - 1, ws->panel, b,
                         (const double2 *)ws->p, (const double2 *)dotpart, ndot, (const double2 *)ws->tau));
      const int t = j0 + b, m2 = n - t;
      if (m2 > 0)
        PW_TRY(pw_dense_gemm(ws, 'N', 'C', m2, m2, 2 * b, mone, ws->panel + t, n, ws->panel + (long)b * n + t,
                             n, one, A + t + (long)t * n, n, st, 2));
    }
    pw_count_launch();
    k_last_diag_plain<<<1, 1, 0, st>>>(A, n, ws->d);
  }
  PW_TRY(pw_check_launch("tridiag"));

  return PW_OK;
}

pw_status stage_dc(pw_dense_ws *ws, int n, int nb, double *lam, cudaStream_t st) {
  // 2. divide and conquer
  DcArrays a{lam, ws->Z, ws->W, ws->U, ws->Ds, ws->zs, ws->DK, ws->zK, ws->tauK, ws->zh,
             ws->lamK, ws->dD, ws->lnew, ws->perm, ws->colK, ws->orig, ws->dcol, ws->src,
             (int *)ws->p /* defl scratch: n ints fit in n double2 */, ws->knode, ws->rhonode,
             ws->ctype, ws->qL, ws->qR, ws->kLR, ws->kneed};
  pw_count_launch();
  k_dc_init<<<(n + 255) / 256, 256, 0, st>>>(ws->d, ws->e, n, lam, ws->Z);
  pw_count_launch();
  k_identity<<<(unsigned)(((long)n * n + 255) / 256), 256, 0, st>>>(ws->Z, n);
  for (int l = (int)ws->levels.size() - 1; l >= 0; --l) {
    const int nn = (int)ws->levels[l].size() / 3;
    const int *nodes = ws->nodes + 3 * ws->level_off[l];
    int maxsize = 0;
    for (int q = 0; q < nn; ++q) maxsize = std::max(maxsize, ws->levels[l][3 * q + 2] - ws->levels[l][3 * q]);
    pw_count_launch();
    k_dc_deflate<<<nn, 256, 0, st>>>(nodes, n, ws->e, a);
    const dim3 gw((maxsize + 7) / 8, nn);
    pw_count_launch();
    k_dc_roots<<<gw, 256, 0, st>>>(nodes, a);
    pw_count_launch();
    k_dc_zhat<<<gw, 256, 0, st>>>(nodes, a);
    pw_count_launch();
    k_dc_vectors<<<gw, 256, 0, st>>>(nodes, n, a);
    // the root merge keeps only the nb lowest eigenpairs
    const int keep = l == 0 ? nb : n;
    pw_count_launch();
    k_dc_rank<<<dim3((maxsize + 127) / 128, nn), 128, 0, st>>>(nodes, a, keep);
    // levels whose halves all have >= 512 rows: their merge products on the
    // FP64-accurate tensor-core path (real operands gathered into ws->T)
    int minhalf = n;
    bool fits = true;   // the gathered operands and the product fit in ws->T (2 nmax^2 doubles)
    for (int q = 0; q < nn; ++q) {
      const int lo = ws->levels[l][3 * q], mid = ws->levels[l][3 * q + 1], hi = ws->levels[l][3 * q + 2];
      minhalf = std::min(minhalf, std::min(mid - lo, hi - mid));
      const size_t sz = hi - lo, rows = std::max(mid - lo, hi - mid), tm = std::min<size_t>(sz, keep);
      fits = fits && rows * sz + sz * tm + rows * tm <= 2 * (size_t)ws->nmax * ws->nmax;
    }
    if (pw_dense_products_mode() == 1 && minhalf >= DC_TC_MIN_HALF && fits) {
      for (int q = 0; q < nn; ++q) {
        const int lo = ws->levels[l][3 * q], mid = ws->levels[l][3 * q + 1], hi = ws->levels[l][3 * q + 2];
        const int node = q, size = hi - lo;   // per-node arrays are indexed within the level
        const int kmax = size, tmax = std::min(size, keep);
        for (int half = 0; half < 2; ++half) {
          const int rows = half ? hi - mid : mid - lo;
          double *Zg = (double *)ws->T, *Ug = Zg + (size_t)rows * kmax, *Wt = Ug + (size_t)kmax * tmax;
          pw_count_launch();
          k_dc_gather_z<<<(unsigned)(((long)rows * kmax + 255) / 256), 256, 0, st>>>(lo, mid, hi, node, half, n, a,
                                                                                     kmax, Zg);
          pw_count_launch();
          k_dc_gather_u<<<(unsigned)(((long)kmax * tmax + 255) / 256), 256, 0, st>>>(lo, node, half, n, a, kmax,
                                                                                     tmax, Ug);
          PW_TRY(pw_dgemm_oz(&ws->oz, rows, tmax, kmax, Zg, rows, Ug, kmax, Wt, rows, st));
          pw_count_launch();
          k_dc_scatter_w<<<(unsigned)(((long)rows * tmax + 255) / 256), 256, 0, st>>>(lo, mid, hi, node, half, n,
                                                                                      a, tmax, Wt);
        }
      }
    } else {
      pw_count_launch();
      k_dc_gemm<<<dim3((maxsize + 63) / 64 + 1, (maxsize + 63) / 64, nn), 256, 0, st>>>(nodes, n, a);
    }
    pw_count_launch();
    k_dc_copy_defl<<<dim3(maxsize, nn), 128, 0, st>>>(nodes, n, a);
    pw_count_launch();
    k_dc_write<<<dim3(maxsize, nn), 128, 0, st>>>(nodes, n, a, keep);
  }
  PW_TRY(pw_check_launch("divide and conquer"));

  return PW_OK;
}

pw_status stage_backtransform(pw_dense_ws *ws, int n, int nb, const double2 *A, double2 *Y, cudaStream_t st) {
  // 3. back-transformation of the wanted columns
  pw_count_launch();
  k_bt_init<<<(unsigned)(((long)n * nb + 255) / 256), 256, 0, st>>>(ws->Z, n, nb, Y);
  // Y = H_0 H_1 ... H_{n-2} Z, blocks of BTB reflectors from the last:
  // H_j0 ... H_j1-1 = I - V T V^H  ->  Y[j0+1:, :] -= V (T (V^H Y[j0+1:, :]))
  {
    const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0),
                  mone = make_double2(-1.0, 0.0);
    for (int j1 = n - 1; j1 > 0;) {
      const int j0 = std::max(0, j1 - BTB), b = j1 - j0, mb = n - j0 - 1;
      pw_count_launch();
      k_copy_panel<<<(unsigned)(((long)mb * b + 255) / 256), 256, 0, st>>>(A, n, j0, b, ws->Vb, mb);
      PW_TRY(pw_dense_gemm(ws, 'C', 'N', b, b, mb, one, ws->Vb, mb, ws->Vb, mb, zero, ws->Gv, b, st));
      pw_count_launch();
      k_build_T<<<(b + BT_WARPS - 1) / BT_WARPS, 32 * BT_WARPS, 0, st>>>(ws->Gv, ws->tau, j0, b, ws->Tb);
      double2 *Yb = Y + (j0 + 1);
      PW_TRY(pw_dense_gemm(ws, 'C', 'N', b, nb, mb, one, ws->Vb, mb, Yb, n, zero, ws->Wk, b, st));
      PW_TRY(pw_dense_gemm(ws, 'N', 'N', b, nb, b, one, ws->Tb, b, ws->Wk, b, zero, ws->Wk2, b, st));
      PW_TRY(pw_dense_gemm(ws, 'N', 'N', mb, nb, b, mone, ws->Vb, mb, ws->Wk2, b, one, Yb, n, st));
      j1 = j0;
    }
  }
  return pw_check_launch("back-transform");
}

std::atomic<int> g_graphs{1};

// what a captured stage depends on besides its key: the product buffers'
// generation, the product mode and the panel mode
unsigned stage_gen(const pw_dense_ws *ws) {
  return (2 * ws->oz.gen + (unsigned)pw_dense_products_mode()) * 4 + (unsigned)g_coop.load();
}

// A stage through the workspace's graph cache: the first call of a key runs
// directly (and grows any workspace it needs); a key seen twice in a row is
// captured (thread-local capture mode) and then replayed.  Graphs bake in
// buffer addresses: an entry is dropped when the workspace's product buffers
// were reallocated since its capture (generation).  Not on the legacy default
// stream (which cannot be captured) or a stream already being captured.
template <typename F>
pw_status run_stage(pw_dense_ws *ws, int stage, int n, int nb, const void *p0, const void *p1, cudaStream_t st,
                    F &&fn) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!g_graphs.load() || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread ||
      cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return fn();
  // the product buffers' generation and the product mode both decide what a
  // capture holds
  const unsigned gen = stage_gen(ws);
  for (auto it = ws->graphs.begin(); it != ws->graphs.end(); ++it) {
    if (it->stage == stage && it->n == n && it->nb == nb && it->p0 == p0 && it->p1 == p1) {
      if (it->gen == gen) {
        PW_CUDA(cudaGraphLaunch(it->exec, st));
        pw_count_launches(it->kernels);
        return PW_OK;
      }
      cudaGraphExecDestroy(it->exec);
      ws->graphs.erase(it);
      break;
    }
  }
  const bool repeat = ws->last_key[stage][0] == n && ws->last_key[stage][1] == nb;
  ws->last_key[stage][0] = n;
  ws->last_key[stage][1] = nb;
  if (!repeat) return fn();
  cudaGraph_t g = nullptr;
  PW_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const uint64_t k0 = pw_thread_launches();
  const pw_status r = fn();
  const uint64_t nk = pw_thread_launches() - k0;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  cudaGraphExec_t exec = nullptr;
  if (r != PW_OK || ce != cudaSuccess || !g || stage_gen(ws) != gen ||
      cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
    // capture did not work out: clear the error and run the stage directly
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fn();
  }
  cudaGraphDestroy(g);
  if (ws->graphs.size() >= 6) {
    cudaGraphExecDestroy(ws->graphs.front().exec);
    ws->graphs.erase(ws->graphs.begin());
  }
  ws->graphs.push_back({stage, n, nb, p0, p1, gen, exec, nk});
  PW_CUDA(cudaGraphLaunch(exec, st));
  return PW_OK;
}
}  // namespace

extern "C" pw_status pw_householder_panels(int mode) {
  if (mode < 0 || mode > 3) return PW_ERR_ARG;
  g_coop.store(mode);
  return PW_OK;
}

extern "C" pw_status pw_dense_graphs(int on) {
  if (on != 0 && on != 1) return PW_ERR_ARG;
  g_graphs.store(on);
  return PW_OK;
}

pw_status pw_heev_lowest(pw_dense_ws *ws, int n, int nb, double2 *A, double *lam, double2 *Y,
                         cudaStream_t st) {
  if (n <= 0 || nb <= 0 || nb > n || n > ws->nmax || nb > ws->nbmax) return PW_ERR_ARG;
  // 1. Householder tridiagonalisation: panels of TPB columns (lower triangle)
  if (ws->ev[2]) cudaEventRecord(ws->ev[2], st);
  // with cooperative panels the stage is ~5 launches per 32 columns and is
  // ordered across streams by an event, so it runs uncaptured
  if ((g_coop.load() == 1 && coop_grid() > 0) || g_coop.load() == 3) PW_TRY(stage_tridiag(ws, n, A, st));
  else PW_TRY(run_stage(ws, 0, n, nb, A, nullptr, st, [&] { return stage_tridiag(ws, n, A, st); }));
  // 2. divide and conquer (the merge tree is built and uploaded outside any capture)
  if (ws->ev[3]) cudaEventRecord(ws->ev[3], st);
  if (ws->tree_n != n) build_tree(ws, n, st);
  PW_TRY(run_stage(ws, 1, n, nb, lam, nullptr, st, [&] { return stage_dc(ws, n, nb, lam, st); }));
  // 3. back-transformation of the wanted columns
  if (ws->ev[4]) cudaEventRecord(ws->ev[4], st);
  return run_stage(ws, 2, n, nb, A, Y, st, [&] { return stage_backtransform(ws, n, nb, A, Y, st); });
}

// ======================================================================
// Rayleigh-Ritz
// ======================================================================
namespace {
pw_status cholesky(pw_dense_ws *ws, double2 *A, int n, cudaStream_t st) {
  const double2 mone = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int b = std::min(CB, n - j0);
    pw_count_launch();
    k_potf2<<<1, 256, 0, st>>>(A, n, j0, b, ws->piv, ws->flag, ws->Li);
    const int rest = n - j0 - b;
    if (rest > 0) {
      pw_count_launch();
      k_trsm_inv<<<(rest + TRSM_ROWS - 1) / TRSM_ROWS, 256, 0, st>>>(A, n, j0, b, ws->Li);
      // A22 -= L21 L21^H on the lower tiles only (the factorisation reads the
      // lower triangle; the upper one is cleared at the end)
      PW_TRY(pw_dense_gemm(ws, 'N', 'C', rest, rest, b, mone, A + (j0 + b) + (long)j0 * n, n,
                           A + (j0 + b) + (long)j0 * n, n, one, A + (j0 + b) + (long)(j0 + b) * n, n, st, 2));
    }
  }
  pw_count_launch();
  k_zero_upper<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 32), 0, st>>>(A, n);
  return pw_check_launch("cholesky");
}

// X = L^-1 for lower-triangular L (n x n, ld n); T is scratch
pw_status trinv(pw_dense_ws *ws, const double2 *L, double2 *X, int n, cudaStream_t st) {
  PW_CUDA(cudaMemsetAsync(X, 0, (size_t)n * n * 16, st));
  // leaves: blocks of CB along the diagonal
  std::vector<int> lo, sz;
  for (int j = 0; j < n; j += CB) { lo.push_back(j); sz.push_back(std::min(CB, n - j)); }
  int *dlo = ws->src, *dsz = ws->dcol;   // int scratch (n entries each, >= n/CB needed)
  PW_CUDA(cudaMemcpyAsync(dlo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, st));
  PW_CUDA(cudaMemcpyAsync(dsz, sz.data(), sz.size() * 4, cudaMemcpyHostToDevice, st));
  pw_count_launch();
  k_trinv_small<<<(unsigned)lo.size(), 32, 0, st>>>(L, X, n, dlo, dsz);
  PW_TRY(pw_check_launch("trinv_small"));
  // combine: [L11 0; L21 L22]^-1 = [X11 0; -X22 L21 X11, X22], bottom-up over
  // block widths 32, 64, 128, ...; the pairs of one width go in one batched
  // launch, and the triangular X11, X22 bound each tile's K range
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0),
                zero = make_double2(0.0, 0.0);
  const long dstep = (long)n + 1;
  for (int w = CB; w < n; w *= 2) {
    const int full = n / (2 * w);            // pairs of two complete w-blocks
    double2 *T = ws->T;
    if (full > 0) {
      const long s2 = 2 * (long)w * dstep;   // from one pair's corner to the next
      if (pw_use_oz(w, w, w)) {
        // few large pairs: one tensor-core product each
        for (int q = 0; q < full; ++q) {
          PW_TRY(pw_dense_gemm(ws, 'N', 'N', w, w, w, one, L + w + q * s2, n, X + q * s2, n, zero,
                               T + (long)q * w * w, w, st, 4));
          PW_TRY(pw_dense_gemm(ws, 'N', 'N', w, w, w, mone, X + w * dstep + q * s2, n, T + (long)q * w * w, w,
                               zero, X + w + q * s2, n, st, 5));
        }
      } else {
        // T_p = L21 X11 (w x w, ld w)
        PW_TRY(pw_zgemm_batched('N', 'N', w, w, w, one, L + w, n, s2, X, n, s2, zero, T, w, (long)w * w,
                                full, st, 4));
        // X21 = -X22 T_p
        PW_TRY(pw_zgemm_batched('N', 'N', w, w, w, mone, X + w * dstep, n, s2, T, w, (long)w * w, zero,
                                X + w, n, s2, full, st, 5));
      }
    }
    const int off = full * 2 * w;
    if (off + w < n) {                       // a last pair with a shorter second block
      const int h1 = w, h2 = n - off - w;
      PW_TRY(pw_dense_gemm(ws, 'N', 'N', h2, h1, h1, one, L + (off + h1) + (long)off * n, n, X + off * dstep,
                           n, zero, T, h2, st, 4));
      PW_TRY(pw_dense_gemm(ws, 'N', 'N', h2, h1, h2, mone, X + (off + h1) * dstep, n, T, h2, zero,
                           X + (off + h1) + (long)off * n, n, st, 5));
    }
  }
  return PW_OK;
}
}  // namespace

pw_status pw_rayleigh_ritz(pw_dense_ws *ws, int n, int nb, const double2 *G, int ldg,
                           const double2 *A, int lda, double *theta, double2 *C, int ldc,
                           int *chol_ok, cudaStream_t st, double piv_tol) {
  if (n > ws->nmax || nb > ws->nbmax || nb > n) return PW_ERR_ARG;
  *chol_ok = 1;
  cudaEventRecord(ws->ev[0], st);
  PW_CUDA(cudaMemsetAsync(ws->flag, 0, 16, st));
  pw_count_launch();
  k_diag_scale<<<(n + 127) / 128, 128, 0, st>>>(G, ldg, n, ws->dscale, ws->flag);
  const dim3 g2((n + 31) / 32, (n + 31) / 32), b2(32, 32);
  pw_count_launch();
  k_scale_herm<<<g2, b2, 0, st>>>(G, ldg, n, ws->dscale, ws->G);
  pw_count_launch();
  k_scale_herm<<<g2, b2, 0, st>>>(A, lda, n, ws->dscale, ws->A);
  PW_TRY(pw_check_launch("scale"));
  PW_TRY(cholesky(ws, ws->G, n, st));
  pw_count_launch();
  k_chol_check<<<1, 256, 0, st>>>(ws->piv, n, piv_tol, ws->flag);
  int flag = 0;
  PW_CUDA(cudaMemcpyAsync(&flag, ws->flag, 4, cudaMemcpyDeviceToHost, st));
  PW_CUDA(cudaStreamSynchronize(st));
  if (flag & 8) return PW_ERR_NUMERIC;
  if (flag) { *chol_ok = 0; return PW_OK; }
  PW_TRY(trinv(ws, ws->G, ws->Linv, n, st));
  cudaEventRecord(ws->ev[1], st);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  // At = Linv As Linv^H, using the triangle of Linv: row block I of T = Linv As
  // needs columns < I_end of Linv; column block J of At = T Linv^H needs
  // rows < J_end of T and, At being Hermitian, only its rows <= J_end
  constexpr int TB = 256;
  for (int i0 = 0; i0 < n; i0 += TB) {
    const int ib = std::min(TB, n - i0), kend = i0 + ib;
    PW_TRY(pw_dense_gemm(ws, 'N', 'N', ib, n, kend, one, ws->Linv + i0, n, ws->A, n, zero, ws->T + i0, n, st));
  }
  for (int j0 = 0; j0 < n; j0 += TB) {
    const int jb = std::min(TB, n - j0), kend = j0 + jb;
    PW_TRY(pw_dense_gemm(ws, 'N', 'C', kend, jb, kend, one, ws->T, n, ws->Linv + j0, n, zero,
                         ws->A + (long)j0 * n, n, st));
  }
  pw_count_launch();
  k_mirror_upper_to_lower<<<g2, b2, 0, st>>>(ws->A, n);
  PW_TRY(pw_heev_lowest(ws, n, nb, ws->A, ws->lam, ws->Y, st));
  PW_CUDA(cudaMemcpyAsync(theta, ws->lam, nb * 8, cudaMemcpyDeviceToDevice, st));
  // C = d o (Linv^H Y); Linv^H is upper triangular
  PW_TRY(pw_dense_gemm(ws, 'C', 'N', n, nb, n, one, ws->Linv, n, ws->Y, n, zero, C, ldc, st, 3));
  pw_count_launch();
  k_scale_rows_real<<<(unsigned)(((long)n * nb + 255) / 256), 256, 0, st>>>(C, ldc, n, nb, ws->dscale);
  cudaEventRecord(ws->ev[5], st);
  return pw_check_launch("rayleigh_ritz");
}

extern "C" pw_status pw_heev(int n, int nb, void *A, double *w, void *Y, void *stream) {
  if (n < 1 || nb < 1 || nb > n || !A || !w || !Y) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  pw_dense_ws ws;
  PW_TRY(pw_dense_alloc(&ws, n, nb));
  pw_status r = pw_heev_lowest(&ws, n, nb, (double2 *)A, w, (double2 *)Y, st);
  if (r == PW_OK && cudaStreamSynchronize(st) != cudaSuccess) r = PW_ERR_CUDA;
  if (r == PW_OK) r = pw_oz_check(&ws.oz, st);
  pw_dense_free(&ws);
  return r;
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz in two halves, for callers that orthonormalise the basis
// themselves (the mixed path does S L^-H on the tensor cores)
// ---------------------------------------------------------------------------
namespace {
// M = d o Linv^H   (M[i][j] = d_i conj(Linv[j][i]), upper triangular)
__global__ void k_make_M(const double2 *Linv, int n, const double *d, double2 *M, int ldm) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n) return;
  const double2 l = Linv[j + (long)i * n];
  M[i + (long)j * ldm] = i <= j ? make_double2(d[i] * l.x, -d[i] * l.y) : make_double2(0.0, 0.0);
}
}  // namespace

pw_status pw_rr_factor(pw_dense_ws *ws, int n, const double2 *G, int ldg, double2 *M, int ldm,
                       int *chol_ok, cudaStream_t st, double piv_tol) {
  if (n > ws->nmax) return PW_ERR_ARG;
  *chol_ok = 1;
  cudaEventRecord(ws->ev[0], st);
  PW_CUDA(cudaMemsetAsync(ws->flag, 0, 16, st));
  pw_count_launch();
  k_diag_scale<<<(n + 127) / 128, 128, 0, st>>>(G, ldg, n, ws->dscale, ws->flag);
  const dim3 g2((n + 31) / 32, (n + 31) / 32), b2(32, 32);
  pw_count_launch();
  k_scale_herm<<<g2, b2, 0, st>>>(G, ldg, n, ws->dscale, ws->G);
  PW_TRY(pw_check_launch("scale"));
  PW_TRY(cholesky(ws, ws->G, n, st));
  pw_count_launch();
  k_chol_check<<<1, 256, 0, st>>>(ws->piv, n, piv_tol, ws->flag);
  int flag = 0;
  PW_CUDA(cudaMemcpyAsync(&flag, ws->flag, 4, cudaMemcpyDeviceToHost, st));
  PW_CUDA(cudaStreamSynchronize(st));
  if (flag & 8) return PW_ERR_NUMERIC;
  if (flag) { *chol_ok = 0; return PW_OK; }
  PW_TRY(trinv(ws, ws->G, ws->Linv, n, st));
  pw_count_launch();
  k_make_M<<<g2, b2, 0, st>>>(ws->Linv, n, ws->dscale, M, ldm);
  cudaEventRecord(ws->ev[1], st);
  return pw_check_launch("rr_factor");
}

pw_status pw_rr_finish_tall(pw_dense_ws *ws, int n, int nb, const double2 *At, int lda, const double2 *M,
                            int ldm, double *theta, double2 *Cp, int ldc, cudaStream_t st) {
  if (n > ws->nmax || nb > ws->nbmax || nb > n) return PW_ERR_ARG;
  pw_count_launch();
  const dim3 g2((n + 31) / 32, (n + 31) / 32), b2(32, 32);
  k_copy_herm<<<g2, b2, 0, st>>>(At, lda, n, ws->A);
  PW_TRY(pw_heev_lowest(ws, n, nb, ws->A, ws->lam, ws->Y, st));
  PW_CUDA(cudaMemcpyAsync(theta, ws->lam, nb * 8, cudaMemcpyDeviceToDevice, st));
  PW_CUDA(cudaMemset2DAsync(Cp, (size_t)ldc * 16, 0, (size_t)nb * 16, nb, st));
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  if (n > nb)
    PW_TRY(pw_dense_gemm(ws, 'N', 'N', n - nb, nb, n - nb, one, M + nb + (long)nb * ldm, ldm, ws->Y + nb, n,
                         zero, Cp + nb, ldc, st, 3));
  cudaEventRecord(ws->ev[5], st);
  return pw_check_launch("rr_finish_tall");
}

pw_status pw_rr_finish(pw_dense_ws *ws, int n, int nb, const double2 *At, int lda, const double2 *M,
                       int ldm, double *theta, double2 *C, int ldc, cudaStream_t st) {
  if (n > ws->nmax || nb > ws->nbmax || nb > n) return PW_ERR_ARG;
  // Hermitian order-n matrix into the workspace (ld n), eigensolve, C = M Y
  pw_count_launch();
  const dim3 g2((n + 31) / 32, (n + 31) / 32), b2(32, 32);
  k_copy_herm<<<g2, b2, 0, st>>>(At, lda, n, ws->A);
  PW_TRY(pw_heev_lowest(ws, n, nb, ws->A, ws->lam, ws->Y, st));
  PW_CUDA(cudaMemcpyAsync(theta, ws->lam, nb * 8, cudaMemcpyDeviceToDevice, st));
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  // M is upper triangular: each row tile skips the zero part of its K range
  PW_TRY(pw_dense_gemm(ws, 'N', 'N', n, nb, n, one, M, ldm, ws->Y, n, zero, C, ldc, st, 3));
  cudaEventRecord(ws->ev[5], st);
  return pw_check_launch("rr_finish");
}
