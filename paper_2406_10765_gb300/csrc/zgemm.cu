// Complex FP64 GEMM on the FP64 pipe (no tensor-core FP64 on this part):
// C = alpha op(A) op(B) + beta C, column-major, op in {N, C}.
//
// Used for the FP64 path's contractions: the projector products B = beta^H
// psi and H psi += beta (D B) (Sec. III-A), the subspace matrices S^H S and
// S^H (H S) (Sec. II-B row scheme), the rotations, and the small dense
// triangular / back-transform products of the Rayleigh-Ritz solve.
//
// 64 x 64 output tile per 256-thread CTA, each thread 4 x 4 outputs strided
// by 16 (conflict-free shared-memory reads), K staged 8 at a time.  Long
// contractions are split over grid.z with deterministic partial sums reduced
// by a second kernel (no floating-point atomics).
#include <algorithm>

#include "pw_internal.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 8;

template <char OPA, char OPB>
__global__ void __launch_bounds__(256) k_zgemm(int m, int n, int k, int kchunk, double2 alpha,
                                               const double2 *__restrict__ A, int lda,
                                               const double2 *__restrict__ B, int ldb,
                                               double2 beta, double2 *__restrict__ C, int ldc,
                                               double2 *__restrict__ ws, int herm, long sA, long sB,
                                               long sC) {
  // herm 1: upper-triangle tiles (mirrored later); herm 2: lower-triangle tiles only
  if (herm == 1 && blockIdx.y < blockIdx.x) return;
  if (herm == 2 && blockIdx.y > blockIdx.x) return;
  // batched: blockIdx.z picks the problem (operands at multiples of the strides)
  const bool batched = (sA | sB | sC) != 0;
  if (batched) {
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
  }
  __shared__ double2 As[BK][BM + 1];
  __shared__ double2 Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = batched ? 0 : blockIdx.z * kchunk;
  const int ke = batched ? k : min(k, kb + kchunk);
  // triangular operands (explicit zeros) bound the K range of a tile:
  // herm 3: op(A) upper, rows m0.. need K >= m0; herm 4: op(B) lower,
  // columns n0.. need K >= n0; herm 5: op(A) lower, rows < m0 + BM need K < m0 + BM
  int ks = kb, kl = ke;
  if (herm == 3) ks = max(kb, m0 - m0 % BK);
  if (herm == 4) ks = max(kb, n0 - n0 % BK);
  if (herm == 5) kl = min(ke, m0 + BM);
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = ks; k0 < kl; k0 += BK) {
    // A tile: op(A)(mm, kk), 64 x 8 = 512 elements, 2 per thread
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = threadIdx.x + t * 256;
      int mm, kk;
      if (OPA == 'N') { mm = e & 63; kk = e >> 6; } else { kk = e & 7; mm = e >> 3; }
      const int gm = m0 + mm, gk = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (gm < m && gk < ke) {
        if (OPA == 'N') v = A[gm + (long)gk * lda];
        else { v = A[gk + (long)gm * lda]; v.y = -v.y; }
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = threadIdx.x + t * 256;
      int nn, kk;
      if (OPB == 'N') { kk = e & 7; nn = e >> 3; } else { nn = e & 63; kk = e >> 6; }
      const int gn = n0 + nn, gk = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (gn < n && gk < ke) {
        if (OPB == 'N') v = B[gk + (long)gn * ldb];
        else { v = B[gn + (long)gk * ldb]; v.y = -v.y; }
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  const bool split = !batched && gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
      if (gm >= m || gn >= n) continue;
      if (split) {
        ws[((long)blockIdx.z * n + gn) * m + gm] = acc[i][j];
      } else {
        double2 r = cmul(alpha, acc[i][j]);
        if (beta.x != 0.0 || beta.y != 0.0) r = cadd(r, cmul(beta, C[gm + (long)gn * ldc]));
        C[gm + (long)gn * ldc] = r;
      }
    }
}

// lower triangle <- conj(upper) (n x n, ld)
__global__ void k_zmirror(double2 *C, int ldc, int n) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n || i <= j) return;
  const double2 u = C[j + (long)i * ldc];
  C[i + (long)j * ldc] = make_double2(u.x, -u.y);
}

__global__ void k_zgemm_reduce(int m, int n, int splits, double2 alpha, const double2 *__restrict__ ws,
                               double2 beta, double2 *__restrict__ C, int ldc, int herm) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)m * n) return;
  const int gm = (int)(idx % m), gn = (int)(idx / m);
  // same tile selection as k_zgemm (the skipped tiles have no partial sums)
  if (herm == 1 && gn / BN < gm / BM) return;
  if (herm == 2 && gn / BN > gm / BM) return;
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < splits; ++z) s = cadd(s, ws[(long)z * m * n + idx]);
  double2 r = cmul(alpha, s);
  if (beta.x != 0.0 || beta.y != 0.0) r = cadd(r, cmul(beta, C[gm + (long)gn * ldc]));
  C[gm + (long)gn * ldc] = r;
}

int choose_splits(int m, int n, int k) {
  if (m <= 0 || n <= 0 || k <= 0) return 1;   // empty product: nothing to split
  const long tiles = (long)((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  long s = (2 * 152 + tiles - 1) / tiles;
  // K chunks of at least 128, or of 32 when the tiles alone leave half the SMs idle
  s = std::min<long>(s, std::max(1, k / (tiles < 76 ? 32 : 128)));
  s = std::min<long>(s, 64);
  return (int)std::max<long>(1, s);
}

}  // namespace

size_t pw_zgemm_ws_elems(int m, int n, int k) {
  const int s = choose_splits(m, n, k);
  return s > 1 ? (size_t)s * m * n : 0;
}

pw_status pw_zgemm_herm(int n, int k, const double2 *A, int lda, const double2 *B, int ldb,
                        double2 *C, int ldc, double2 *ws, size_t ws_elems, cudaStream_t st) {
  return pw_zgemm_ex('C', 'N', n, n, k, make_double2(1.0, 0.0), A, lda, B, ldb,
                     make_double2(0.0, 0.0), C, ldc, ws, ws_elems, st, 1);
}

pw_status pw_zgemm(char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A, int lda,
                   const double2 *B, int ldb, double2 beta, double2 *C, int ldc, double2 *ws,
                   size_t ws_elems, cudaStream_t st) {
  return pw_zgemm_ex(opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, st, 0);
}

pw_status pw_zgemm_ex(char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A, int lda,
                      const double2 *B, int ldb, double2 beta, double2 *C, int ldc, double2 *ws,
                      size_t ws_elems, cudaStream_t st, int herm) {
  if (m <= 0 || n <= 0) return PW_OK;
  if (k <= 0) {
    // C = beta C
    if (beta.x == 1.0 && beta.y == 0.0) return PW_OK;
    // reuse the reduce kernel with zero partial sums
    pw_count_launch();
    k_zgemm_reduce<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, st>>>(m, n, 0, alpha, ws, beta, C, ldc,
                                                                          0);
    return pw_check_launch("zgemm k=0");
  }
  int splits = choose_splits(m, n, k);
  if ((size_t)splits * m * n > ws_elems || !ws) splits = 1;
  int kchunk = (k + splits - 1) / splits;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  splits = (k + kchunk - 1) / kchunk;
  dim3 grid((m + BM - 1) / BM, (n + BN - 1) / BN, splits);
#define L(a, b) k_zgemm<a, b><<<grid, 256, 0, st>>>(m, n, k, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, ws, herm, \
                                                   0L, 0L, 0L)
  pw_count_launch();
  if (opA == 'N' && opB == 'N') L('N', 'N');
  else if (opA == 'C' && opB == 'N') L('C', 'N');
  else if (opA == 'N' && opB == 'C') L('N', 'C');
  else if (opA == 'C' && opB == 'C') L('C', 'C');
  else return PW_ERR_ARG;
#undef L
  if (splits > 1)
    {
      pw_count_launch();
      k_zgemm_reduce<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, st>>>(m, n, splits, alpha, ws,
                                                                          beta, C, ldc, herm);
    }
  if (herm == 1) {
    pw_count_launch();
    k_zmirror<<<dim3((m + 31) / 32, (m + 31) / 32), dim3(32, 32), 0, st>>>(C, ldc, m);
  }
  return pw_check_launch("zgemm");
}

pw_status pw_zgemm_batched(char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                           int lda, long sA, const double2 *B, int ldb, long sB, double2 beta,
                           double2 *C, int ldc, long sC, int batch, cudaStream_t st, int mode) {
  if (m <= 0 || n <= 0 || batch <= 0) return PW_OK;
  if (k <= 0 || (sA | sB | sC) == 0 || mode == 1) return PW_ERR_ARG;
  dim3 grid((m + BM - 1) / BM, (n + BN - 1) / BN, batch);
#define L(a, b) k_zgemm<a, b><<<grid, 256, 0, st>>>(m, n, k, k, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, \
                                                   mode, sA, sB, sC)
  pw_count_launch();
  if (opA == 'N' && opB == 'N') L('N', 'N');
  else if (opA == 'C' && opB == 'N') L('C', 'N');
  else if (opA == 'N' && opB == 'C') L('N', 'C');
  else if (opA == 'C' && opB == 'C') L('C', 'C');
  else return PW_ERR_ARG;
#undef L
  return pw_check_launch("zgemm batched");
}
