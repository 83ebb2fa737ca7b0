// FP64-accurate complex GEMM on the FP16 tensor cores (an Ozaki-type split
// of each operand into short integer slices), for the dense products of the
// Rayleigh-Ritz step -- the Cholesky and triangular-inverse updates, the
// Householder panel updates and the back-transformation of the small
// eigensolve (Syevd, Sec. III-D) -- which the FP64 pipe of this part runs at
// only ~1.2 TFLOP/s.
//
// Arithmetic (C = op(A) op(B), complex, K = inner dimension):
//   * Real form: row i of op(A) becomes one real row over K' = 2K,
//     (re_k, im_k) interleaved; column j of op(B) becomes two real rows,
//     (re, -im) and (im, re), so D[i][2j] = Re C_ij and D[i][2j+1] = Im C_ij.
//   * Each real row r is scaled by a power of two 2^e_r so that its largest
//     entry lies in [1/2, 1), and the scaled entry x is written exactly (to
//     2^-56) as x = sum_{p=1..S} d_p 2^(-BETA p) with integer digits,
//     |d_1| <= 2^BETA, |d_p| <= 2^(BETA-1), stored as FP16 (S = 8, BETA = 7).
//   * The slice products d_p(a) d_q(b) with p + q = g are summed in one FP32
//     tensor-memory accumulator per group g (g = 2..S+1; the pairs with
//     p + q > S + 1 are below 2^-55 of the largest product and dropped).  Over
//     a chunk of 64 real K every partial sum is an integer below 2^22, so the
//     FP32 accumulation is exact whatever its rounding.
//   * After each chunk the epilogue adds every group, shifted to a common
//     binary point 2^-L, into a 64-bit integer per output (exact except for
//     a rounding of the lowest groups below 2^-L), and at the end converts
//     to FP64 and removes the row and column scales.
// The error is at most 5.5 K' 2^-55 max|a_i| max|b_j| per entry (the row and
// column maxima; each real term is off by at most 1.375 2^-55 in scaled
// units -- the 2^-57 roundings of both digit expansions and the dropped
// pairs -- and the scales add a factor of at most 4), plus the final
// rounding to FP64: inside the usual FP64 bound K' u |a||b| for rows
// without large internal dynamic range.
//
// Kernel: tile of 128 complex rows x 32 complex columns (128 x 64 real) per
// CTA; warp 0 = TMA producer, warp 1 = MMA issuer (one thread), warps 2..9 =
// epilogue.  Two shared-memory stages of 32 real K, each holding all S slices
// of the A and B tiles (64-byte swizzle); eight 64-column FP32 accumulators
// fill the 512 tensor-memory columns.  Every mbarrier wait is bounded; on
// timeout the CTA records an error word, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "oz_gemm.cuh"
#include "pw_internal.cuh"
#include "umma.cuh"

namespace {

using namespace pw_umma;

constexpr int NG = S;                 // accumulator groups g = 2..S+1
constexpr int BM = 128, BN = 64, BK = 32;   // real rows, real columns, real K per stage
constexpr int A_T = BM * BK * 2;      // 8 KB per slice
constexpr int B_T = BN * BK * 2;      // 4 KB per slice
constexpr int STAGE = S * (A_T + B_T);   // 96 KB
constexpr int NSTAGE = 2;
constexpr int CHUNK_KB = 2;           // K blocks per exact accumulation chunk (64 real K)
constexpr int SMEM_BYTES = NSTAGE * STAGE + 1024 + 512;
constexpr int TMEM_COLS = 512;
constexpr int EPI_WARPS = 8;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 32
// FP16), 8-row groups 512 B apart
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) { return smem_desc(addr, 16, 512, 4); }
// instruction descriptor, kind::f16: FP16 A and B, FP32 D, both K-major, M = 128, N = 64
__host__ __device__ constexpr uint32_t idesc_oz() { return idesc_f16(BM, BN, false); }
__global__ void __launch_bounds__(NTHREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              int a_slice_rows, int b_slice_rows, int m, int n, int kblocks, int mtiles, int ntiles,
              const int *__restrict__ ea, const int *__restrict__ eb, double2 alpha, double2 beta,
              double2 *__restrict__ C, int ldc, int herm, int ioff, int joff, double2 *__restrict__ part,
              int *__restrict__ err, int real_out) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + NSTAGE * STAGE);
  uint64_t *empty = full + NSTAGE;
  uint64_t *accf = empty + NSTAGE;     // [NG] group accumulator ready
  uint64_t *acce = accf + NG;          // [NG] group accumulator drained
  uint32_t *tmem_slot = (uint32_t *)(acce + NG);

  const int tile = blockIdx.x;
  const int mt = tile / ntiles, nt = tile % ntiles;
  if (mt >= mtiles) return;
  const int m0 = mt * BM;              // complex rows m0 .. m0 + 127 (of this block)
  // complex columns j0 .. j0 + 31, or with real_out (real operands: one
  // slice row per real column of B, output real, ld ldc in doubles) real
  // columns j0 .. j0 + 63
  const int j0 = nt * (real_out ? BN : BN / 2);
  const int gm0 = ioff + m0, gj0 = joff + j0;   // the same in the whole product
  // Hermitian output, upper part (mirrored later): skip tiles strictly below
  // the diagonal; lower part: tiles holding no element with j/64 <= i/64
  if (herm == 1 && gm0 > gj0 + BN / 2 - 1) return;
  if (herm == 2 && (gj0 >> 6) > ((gm0 + BM - 1) >> 6)) return;
  // K range of the tile (real K blocks): triangular operands are zero outside
  int kb_lo = 0, kb_hi = kblocks;
  if (herm == 3) kb_lo = min(kblocks, (2 * gm0) / BK);
  if (herm == 4) kb_lo = min(kblocks, (2 * gj0) / BK);
  if (herm == 5) kb_hi = min(kblocks, (2 * (gm0 + BM) + BK - 1) / BK);
  // K split: part z of gridDim.y takes an equal share, in whole chunks
  const int ntot = max(0, kb_hi - kb_lo);
  const int nch = (ntot + CHUNK_KB - 1) / CHUNK_KB;
  const int per = (nch + (int)gridDim.y - 1) / (int)gridDim.y;
  const int c0 = min(nch, (int)blockIdx.y * per), c1 = min(nch, c0 + per);
  const int kb_beg = kb_lo + c0 * CHUNK_KB;
  const int nkb = max(0, min(kb_hi, kb_lo + c1 * CHUNK_KB) - kb_beg);
  const int nchunk = (nkb + CHUNK_KB - 1) / CHUNK_KB;
  // binary point of the fixed-point sum: |sum| <= K' (scaled entries < 1)
  int lg = 0;
  while ((1 << lg) < max(1, nkb * BK)) ++lg;
  const int Lfix = min(56, 62 - lg);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int g = 0; g < NG; ++g) { mbar_init(&accf[g], 1); mbar_init(&acce[g], EPI_WARPS); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: all S slices of the A and B tiles per stage
      for (int i = 0; i < nkb; ++i) {
        const int s = i % NSTAGE;
        const uint32_t u = i / NSTAGE;
        if (!mbar_wait(&empty[s], (u & 1) ^ 1)) { atomicOr(err, 1); break; }
        unsigned char *st = smem + s * STAGE;
        mbar_expect_tx(&full[s], STAGE);
        const int x = (kb_beg + i) * BK;
#pragma unroll
        for (int p = 0; p < S; ++p) {
          tma_load_2d(st + p * A_T, &mapA, &full[s], x, p * a_slice_rows + m0);
          tma_load_2d(st + S * A_T + p * B_T, &mapB, &full[s], x, p * b_slice_rows + (real_out ? j0 : 2 * j0));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t idesc = idesc_oz();
      bool ok = true;
      for (int i = 0; i < nkb && ok; ++i) {
        const int s = i % NSTAGE;
        const uint32_t u = i / NSTAGE;
        const int ch = i / CHUNK_KB;
        const bool first = (i % CHUNK_KB) == 0;
        const bool last = (i % CHUNK_KB) == CHUNK_KB - 1 || i == nkb - 1;
        if (!mbar_wait(&full[s], u & 1)) { atomicOr(err, 2); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + s * STAGE);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            const int d = g + 2;
            if (first && kk == 0) {
              // the epilogue has read this group's previous chunk
              if (!mbar_wait(&acce[g], ((uint32_t)ch & 1) ^ 1)) { atomicOr(err, 8); ok = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const int plo = max(1, d - S), phi = min(S, d - 1);
#pragma unroll
            for (int p = plo; p <= phi; ++p) {
              const int q = d - p;
              const uint64_t da = smem_desc_sw64(base + (p - 1) * A_T) + 2 * kk;
              const uint64_t db = smem_desc_sw64(base + S * A_T + (q - 1) * B_T) + 2 * kk;
              mma_f16(tmem + (uint32_t)(g * BN), da, db, idesc, !(first && kk == 0 && p == plo));
            }
            if (last && kk == BK / 16 - 1) mma_commit(&accf[g]);
          }
          if (!ok) break;
        }
        mma_commit(&empty[s]);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; lane quarter q, column half h
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    long long acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0;
    bool ok = true;
    for (int ch = 0; ch < nchunk && ok; ++ch) {
#pragma unroll 1
      for (int g = 0; g < NG; ++g) {
        if (!mbar_wait(&accf[g], (uint32_t)ch & 1)) { atomicOr(err, 4); ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t v[32];
        tmem_ld32(tmem + lanes + (uint32_t)(g * BN + h * 32), v);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[g]);
        const int sh = Lfix - BETA * (g + 2);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] += shifted(f2i_exact(v[i]), sh);
      }
    }
    const int i = m0 + q * 32 + lane;              // complex output row
    if (ok && i < m && real_out) {
      double *Cr = (double *)C;
      const int ka = -Lfix - ea[i];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int j = j0 + h * 32 + t;
        if (j >= n) continue;
        double r = alpha.x * scale_pow2((double)acc[t], ka - eb[j]);
        if (beta.x != 0.0) r += beta.x * Cr[i + (long)j * ldc];
        Cr[i + (long)j * ldc] = r;
      }
    } else if (ok && i < m) {
      const int jb = j0 + h * 16;                  // first complex column of this thread
      const int ka = -Lfix - ea[i];
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int j = jb + t;
        if (j >= n) continue;
        if (herm == 2 && ((joff + j) >> 6) > ((ioff + i) >> 6)) continue;
        const int k = ka - eb[j];
        const double re = scale_pow2((double)acc[2 * t], k);
        const double im = scale_pow2((double)acc[2 * t + 1], k);
        if (part) {
          part[(long)blockIdx.y * m * n + i + (long)j * m] = make_double2(re, im);
        } else {
          double2 r = make_double2(alpha.x * re - alpha.y * im, alpha.x * im + alpha.y * re);
          if (beta.x != 0.0 || beta.y != 0.0) {
            const double2 c = C[i + (long)j * ldc];
            r.x += beta.x * c.x - beta.y * c.y;
            r.y += beta.x * c.y + beta.y * c.x;
          }
          C[i + (long)j * ldc] = r;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// sum of the K-split parts (in part order), then alpha, beta; same element
// selection as the single-part epilogue
__global__ void k_oz_reduce(const double2 *__restrict__ part, int splits, int m, int n, double2 alpha,
                            double2 beta, double2 *__restrict__ C, int ldc) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)m * n) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < splits; ++z) {
    const double2 v = part[(long)z * m * n + idx];
    s.x += v.x;
    s.y += v.y;
  }
  double2 r = make_double2(alpha.x * s.x - alpha.y * s.y, alpha.x * s.y + alpha.y * s.x);
  if (beta.x != 0.0 || beta.y != 0.0) {
    const double2 c = C[i + (long)j * ldc];
    r.x += beta.x * c.x - beta.y * c.y;
    r.y += beta.x * c.y + beta.y * c.x;
  }
  C[i + (long)j * ldc] = r;
}

// lower triangle <- conj(upper) (n x n, ld)
__global__ void k_oz_mirror(double2 *C, int ldc, int n) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n || i <= j) return;
  const double2 u = C[j + (long)i * ldc];
  C[i + (long)j * ldc] = make_double2(u.x, -u.y);
}

// ------------------------------------------------------------- slicing ----
// Slices of the real rows of an operand.  The complex "row" r over k is
//   contiguous:  v_kappa = X[kappa + r ld]      (a column of X)
//   strided:     v_kappa = X[r + kappa ld]      (a row of X)
// conjugated if conj.  bside = 0: one real row r = (re, im) over K' = 2k;
// bside = 1: two real rows 2r = (re, -im), 2r + 1 = (im, re).
// out: [S][rows_total][kpad] FP16, e: row exponents (one per complex row).
__global__ void __launch_bounds__(256) k_oz_slice_contig(const double2 *__restrict__ X, int ld, int k, int conj,
                                                         int bside, int kpad, int rows_total,
                                                         __half *__restrict__ out, int *__restrict__ e) {
  __shared__ unsigned long long shm[8];
  const int r = blockIdx.x;
  const double2 *x = X + (long)r * ld;
  unsigned long long mb = 0;
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    const double2 v = x[t];
    const unsigned long long a = abs_bits(v.x), c = abs_bits(v.y);
    mb = max(mb, max(a, c));
  }
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mb;
  __syncthreads();
  mb = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mb = max(mb, shm[w]);
  const int ex = row_exp(mb);
  if (threadIdx.x == 0) e[r] = ex;
  const long slice = (long)rows_total * kpad;
  for (int t = threadIdx.x; t < kpad / 2; t += blockDim.x) {
    double re = 0.0, im = 0.0;
    if (t < k) {
      const double2 v = x[t];
      re = v.x;
      im = conj ? -v.y : v.y;
    }
    __half dr[S], di[S];
    digits(re, ex, dr);
    digits(im, ex, di);
    if (!bside) {
      __half *o = out + (long)r * kpad + 2 * t;
#pragma unroll
      for (int p = 0; p < S; ++p) *(__half2 *)(o + p * slice) = __halves2half2(dr[p], di[p]);
    } else {
      __half *o0 = out + (long)(2 * r) * kpad + 2 * t, *o1 = o0 + kpad;
#pragma unroll
      for (int p = 0; p < S; ++p) {
        *(__half2 *)(o0 + p * slice) = __halves2half2(dr[p], __hneg(di[p]));
        *(__half2 *)(o1 + p * slice) = __halves2half2(di[p], dr[p]);
      }
    }
  }
}

// row maxima of the strided rows as ordered bits: block (32 rows, 8 warps)
// over a 256-long K range, lane = row (reads coalesced across rows), the
// warps' maxima combined in shared memory, then one atomicMax per row into mx
// (cleared before)
constexpr int RX_K = 256;
__global__ void __launch_bounds__(256) k_oz_rowmax(const double2 *__restrict__ X, int ld, int nrows, int k,
                                                   unsigned long long *__restrict__ mx) {
  __shared__ unsigned long long sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const int t0 = blockIdx.y * RX_K, t1 = min(k, t0 + RX_K);
  unsigned long long m = 0;
  if (r < nrows)
    for (int t = t0 + w; t < t1; t += 8) {
      const double2 v = X[r + (long)t * ld];
      m = max(m, max(abs_bits(v.x), abs_bits(v.y)));
    }
  sh[w][lane] = m;
  __syncthreads();
  if (w == 0 && r < nrows) {
#pragma unroll
    for (int q = 1; q < 8; ++q) m = max(m, sh[q][lane]);
    atomicMax(&mx[r], m);
  }
}

// strided rows: 32 rows x 64 K tile through shared memory (reads along r,
// writes along K)
__global__ void __launch_bounds__(256) k_oz_slice_strided(const double2 *__restrict__ X, int ld, int nrows, int k,
                                                          int conj, int bside, int kpad, int rows_total,
                                                          const unsigned long long *__restrict__ mx,
                                                          int *__restrict__ e, __half *__restrict__ out) {
  __shared__ double2 tileS[64][33];
  const int r0 = blockIdx.x * 32, t0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int tt = ty; tt < 64; tt += 8) {
    const int r = r0 + tx, t = t0 + tt;
    double2 v = make_double2(0.0, 0.0);
    if (r < nrows && t < k) v = X[r + (long)t * ld];
    if (conj) v.y = -v.y;
    tileS[tt][tx] = v;
  }
  __syncthreads();
  const long slice = (long)rows_total * kpad;
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr;
    if (r >= nrows) continue;
    const int ex = row_exp(mx[r]);
    if (blockIdx.y == 0 && tx == 0) e[r] = ex;
    for (int tt = tx; tt < 64; tt += 32) {
      const int t = t0 + tt;
      if (2 * t >= kpad) continue;
      const double2 v = tileS[tt][rr];
      __half dr[S], di[S];
      digits(v.x, ex, dr);
      digits(v.y, ex, di);
      if (!bside) {
        __half *o = out + (long)r * kpad + 2 * t;
#pragma unroll
        for (int p = 0; p < S; ++p) *(__half2 *)(o + p * slice) = __halves2half2(dr[p], di[p]);
      } else {
        __half *o0 = out + (long)(2 * r) * kpad + 2 * t, *o1 = o0 + kpad;
#pragma unroll
        for (int p = 0; p < S; ++p) {
          *(__half2 *)(o0 + p * slice) = __halves2half2(dr[p], __hneg(di[p]));
          *(__half2 *)(o1 + p * slice) = __halves2half2(di[p], dr[p]);
        }
      }
    }
  }
}

// Slices of real rows (the real mode, C = A B with real A, B): row r of A
// is strided (A[r + t lda]), row j of the B side is column j of B,
// contiguous (B[t + j ldb]); out: [S][rows_total][kpad] FP16, e: row
// exponents.  Row maxima of the strided rows come from k_ozr_rowmax (mx,
// cleared before).
__global__ void __launch_bounds__(256) k_ozr_slice_contig(const double *__restrict__ X, int ld, int k, int kpad,
                                                          int rows_total, __half *__restrict__ out,
                                                          int *__restrict__ e) {
  __shared__ unsigned long long shm[8];
  const int r = blockIdx.x;
  const double *x = X + (long)r * ld;
  unsigned long long mb = 0;
  for (int t = threadIdx.x; t < k; t += blockDim.x) mb = max(mb, abs_bits(x[t]));
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mb;
  __syncthreads();
  mb = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mb = max(mb, shm[w]);
  const int ex = row_exp(mb);
  if (threadIdx.x == 0) e[r] = ex;
  const long slice = (long)rows_total * kpad;
  for (int t2 = threadIdx.x; t2 < kpad / 2; t2 += blockDim.x) {
    const int t = 2 * t2;
    __half d0[S], d1[S];
    digits(t < k ? x[t] : 0.0, ex, d0);
    digits(t + 1 < k ? x[t + 1] : 0.0, ex, d1);
    __half *o = out + (long)r * kpad + t;
#pragma unroll
    for (int p = 0; p < S; ++p) *(__half2 *)(o + p * slice) = __halves2half2(d0[p], d1[p]);
  }
}
__global__ void __launch_bounds__(256) k_ozr_rowmax(const double *__restrict__ X, int ld, int nrows, int k,
                                                    unsigned long long *__restrict__ mx) {
  __shared__ unsigned long long sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const int t0 = blockIdx.y * RX_K, t1 = min(k, t0 + RX_K);
  unsigned long long m = 0;
  if (r < nrows)
    for (int t = t0 + w; t < t1; t += 8) m = max(m, abs_bits(X[r + (long)t * ld]));
  sh[w][lane] = m;
  __syncthreads();
  if (w == 0 && r < nrows) {
#pragma unroll
    for (int q = 1; q < 8; ++q) m = max(m, sh[q][lane]);
    atomicMax(&mx[r], m);
  }
}
__global__ void __launch_bounds__(256) k_ozr_slice_strided(const double *__restrict__ X, int ld, int nrows, int k,
                                                           int kpad, int rows_total,
                                                           const unsigned long long *__restrict__ mx,
                                                           int *__restrict__ e, __half *__restrict__ out) {
  __shared__ double tileS[64][33];
  const int r0 = blockIdx.x * 32, t0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int tt = ty; tt < 64; tt += 8) {
    const int r = r0 + tx, t = t0 + tt;
    tileS[tt][tx] = (r < nrows && t < k) ? X[r + (long)t * ld] : 0.0;
  }
  __syncthreads();
  const long slice = (long)rows_total * kpad;
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr;
    if (r >= nrows) continue;
    const int ex = row_exp(mx[r]);
    if (blockIdx.y == 0 && tx == 0) e[r] = ex;
    const int t = t0 + 2 * tx;
    if (t >= kpad) continue;
    __half d0[S], d1[S];
    digits(tileS[2 * tx][rr], ex, d0);
    digits(tileS[2 * tx + 1][rr], ex, d1);
    __half *o = out + (long)r * kpad + t;
#pragma unroll
    for (int p = 0; p < S; ++p) *(__half2 *)(o + p * slice) = __halves2half2(d0[p], d1[p]);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map(CUtensorMap *map, const void *base, int kpad, long rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// slices of op(X)'s rows (bside 0) or of op(X)'s columns (bside 1):
//   A side: op = 'N': rows of X (m x k) -> strided; op = 'C': columns of X (k x m) -> contiguous, conj
//   B side: op = 'N': columns of X (k x n) -> contiguous; op = 'C': rows of X (n x k) -> strided, conj
pw_status slice_operand(char op, int bside, const double2 *X, int ld, int nrows, int k, int kpad,
                        int rows_total, __half *out, int *e, unsigned long long *mx, cudaStream_t st) {
  const bool contig = bside ? op == 'N' : op == 'C';
  const int conj = op == 'C';
  if (contig) {
    pw_count_launch();
    k_oz_slice_contig<<<nrows, 256, 0, st>>>(X, ld, k, conj, bside, kpad, rows_total, out, e);
  } else {
    PW_CUDA(cudaMemsetAsync(mx, 0, (size_t)nrows * sizeof(unsigned long long), st));
    pw_count_launch();
    k_oz_rowmax<<<dim3((nrows + 31) / 32, (k + RX_K - 1) / RX_K), 256, 0, st>>>(X, ld, nrows, k, mx);
    pw_count_launch();
    k_oz_slice_strided<<<dim3((nrows + 31) / 32, (kpad / 2 + 63) / 64), 256, 0, st>>>(
        X, ld, nrows, k, conj, bside, kpad, rows_total, mx, e, out);
  }
  return pw_check_launch("oz slice");
}

int g_max_parts = 16;

// the kernel's shared-memory opt-in, once per device (outside any later
// stream capture: the first product on a device runs uncaptured)
pw_status allow_smem() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return PW_ERR_ARG;
  std::lock_guard<std::mutex> g(mu);
  if (!done[dev]) {
    PW_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    done[dev] = true;
  }
  return PW_OK;
}

}  // namespace

size_t pw_oz_ws_bytes(int m, int n, int k) {
  const size_t kpad = ((size_t)2 * k + BK - 1) / BK * BK;
  const size_t arows = ((size_t)m + BM - 1) / BM * BM, brows = (2 * (size_t)n + BN - 1) / BN * BN;
  return (size_t)S * (arows + brows) * kpad * 2 + (arows + brows) * 4 + std::max(arows, brows) * 8 + 4096;
}

void pw_oz_free(pw_oz_ws *w) {
  if (w->buf) cudaFree(w->buf);
  if (w->part) cudaFree(w->part);
  if (w->err) cudaFree(w->err);
  *w = pw_oz_ws();
}

pw_status pw_oz_check(pw_oz_ws *w, cudaStream_t st) {
  if (!w->err) return PW_OK;
  int e = 0;
  PW_CUDA(cudaMemcpyAsync(&e, w->err, 4, cudaMemcpyDeviceToHost, st));
  PW_CUDA(cudaStreamSynchronize(st));
  return e ? PW_ERR_TIMEOUT : PW_OK;
}

namespace {
// One block of the product: rows [i0, i0 + mb) of op(A), columns [j0, j0 + nb)
// of op(B), the whole K (given operand pointers already offset); herm
// predicates use the global offsets.
pw_status oz_block(pw_oz_ws *w, char opA, char opB, int mb, int nb, int k, double2 alpha, const double2 *A,
                   int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc, cudaStream_t st,
                   int herm, int ioff, int joff) {
  const int kpad = (2 * k + BK - 1) / BK * BK;
  const int kblocks = kpad / BK;
  // slice storage: rows padded to the tile (the tensor map of the last slice
  // then never reads another slice's rows)
  const int arows = (mb + BM - 1) / BM * BM, brows = (2 * nb + BN - 1) / BN * BN;
  const size_t abytes = (size_t)S * arows * kpad * 2, bbytes = (size_t)S * brows * kpad * 2;
  const size_t mxrows = (size_t)std::max(arows, brows);
  const size_t need = abytes + bbytes + ((size_t)arows + brows) * 4 + 256 + mxrows * 8 + 1024;
  if (need > w->bytes) {
    if (w->buf) cudaFree(w->buf);
    w->buf = nullptr;
    w->bytes = 0;
    ++w->gen;
    if (cudaMalloc(&w->buf, need) != cudaSuccess) { cudaGetLastError(); return PW_ERR_OOM; }
    w->bytes = need;
  }
  if (!w->err) {
    if (cudaMalloc((void **)&w->err, 16) != cudaSuccess) { cudaGetLastError(); return PW_ERR_OOM; }
    PW_CUDA(cudaMemsetAsync(w->err, 0, 16, st));
    ++w->gen;
  }
  unsigned char *p = (unsigned char *)w->buf;
  __half *sa = (__half *)p, *sb = (__half *)(p + abytes);
  int *ea = (int *)(p + abytes + bbytes), *eb = ea + arows;
  unsigned long long *mx =
      (unsigned long long *)(((uintptr_t)(eb + brows) + 255) & ~(uintptr_t)255);   // strided row maxima
  PW_TRY(slice_operand(opA, 0, A, lda, mb, k, kpad, arows, sa, ea, mx, st));
  PW_TRY(slice_operand(opB, 1, B, ldb, nb, k, kpad, brows, sb, eb, mx, st));
  CUtensorMap ma, mbm;
  if (!make_map(&ma, sa, kpad, (long)S * arows, BM) || !make_map(&mbm, sb, kpad, (long)S * brows, BN))
    return PW_ERR_CUDA;
  PW_TRY(allow_smem());
  const int mtiles = arows / BM, ntiles = brows / BN, tiles = mtiles * ntiles;
  // K split when the tiles alone leave SMs idle (>= 8 chunks per part)
  const int nch = (kblocks + CHUNK_KB - 1) / CHUNK_KB;
  int parts = 1;
  if (herm == 0 && tiles < 152) {
    parts = std::min({(2 * 152 + tiles - 1) / tiles, std::max(1, nch / 8), g_max_parts});
    const size_t pbytes = (size_t)parts * mb * nb * 16;
    if (parts > 1 && pbytes > w->part_bytes) {
      if (w->part) cudaFree(w->part);
      w->part = nullptr;
      w->part_bytes = 0;
      ++w->gen;
      if (cudaMalloc((void **)&w->part, pbytes) != cudaSuccess) { cudaGetLastError(); parts = 1; }
      else w->part_bytes = pbytes;
    }
  }
  pw_count_launch();
  k_oz_gemm<<<dim3(tiles, parts), NTHREADS, SMEM_BYTES, st>>>(ma, mbm, arows, brows, mb, nb, kblocks, mtiles,
                                                               ntiles, ea, eb, alpha, beta, C, ldc, herm, ioff,
                                                               joff, parts > 1 ? w->part : nullptr, w->err, 0);
  PW_TRY(pw_check_launch("oz gemm"));
  if (parts > 1) {
    pw_count_launch();
    k_oz_reduce<<<(unsigned)(((long)mb * nb + 255) / 256), 256, 0, st>>>(w->part, parts, mb, nb, alpha, beta, C,
                                                                          ldc);
    PW_TRY(pw_check_launch("oz reduce"));
  }
  return PW_OK;
}

// operand pointer of op(X) at (row r, K index t): op 'N' -> X[r + t ld],
// op 'C' -> X[t + r ld]
const double2 *at(const double2 *X, char op, int ld, long r, long t) {
  return op == 'N' ? X + r + t * (long)ld : X + t + r * (long)ld;
}
}  // namespace

pw_status pw_dgemm_oz(pw_oz_ws *w, int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                      double *C, int ldc, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0 || lda < m || ldb < k || ldc < m) return PW_ERR_ARG;
  const int kpad = (k + BK - 1) / BK * BK;
  const int kblocks = kpad / BK;
  const int arows = (m + BM - 1) / BM * BM, brows = (n + BN - 1) / BN * BN;
  const size_t abytes = (size_t)S * arows * kpad * 2, bbytes = (size_t)S * brows * kpad * 2;
  const size_t need = abytes + bbytes + ((size_t)arows + brows) * 4 + 256 + (size_t)arows * 8 + 1024;
  if (need > w->bytes) {
    if (w->buf) cudaFree(w->buf);
    w->buf = nullptr;
    w->bytes = 0;
    ++w->gen;
    if (cudaMalloc(&w->buf, need) != cudaSuccess) { cudaGetLastError(); return PW_ERR_OOM; }
    w->bytes = need;
  }
  if (!w->err) {
    if (cudaMalloc((void **)&w->err, 16) != cudaSuccess) { cudaGetLastError(); return PW_ERR_OOM; }
    PW_CUDA(cudaMemsetAsync(w->err, 0, 16, st));
    ++w->gen;
  }
  unsigned char *p = (unsigned char *)w->buf;
  __half *sa = (__half *)p, *sb = (__half *)(p + abytes);
  int *ea = (int *)(p + abytes + bbytes), *eb = ea + arows;
  unsigned long long *mx = (unsigned long long *)(((uintptr_t)(eb + brows) + 255) & ~(uintptr_t)255);
  // A: strided rows (row maxima first); B: its columns, contiguous.  Slice
  // rows past m and n are never written: they only feed output rows and
  // columns that are not stored
  PW_CUDA(cudaMemsetAsync(mx, 0, (size_t)m * 8, st));
  pw_count_launch();
  k_ozr_rowmax<<<dim3((m + 31) / 32, (k + RX_K - 1) / RX_K), 256, 0, st>>>(A, lda, m, k, mx);
  pw_count_launch();
  k_ozr_slice_strided<<<dim3((m + 31) / 32, (kpad + 63) / 64), 256, 0, st>>>(A, lda, m, k, kpad, arows, mx, ea, sa);
  pw_count_launch();
  k_ozr_slice_contig<<<n, 256, 0, st>>>(B, ldb, k, kpad, brows, sb, eb);
  PW_TRY(pw_check_launch("oz real slices"));
  CUtensorMap ma, mbm;
  if (!make_map(&ma, sa, kpad, (long)S * arows, BM) || !make_map(&mbm, sb, kpad, (long)S * brows, BN))
    return PW_ERR_CUDA;
  PW_TRY(allow_smem());
  const int mtiles = arows / BM, ntiles = brows / BN;
  pw_count_launch();
  k_oz_gemm<<<dim3(mtiles * ntiles, 1), NTHREADS, SMEM_BYTES, st>>>(
      ma, mbm, arows, brows, m, n, kblocks, mtiles, ntiles, ea, eb, make_double2(1.0, 0.0), make_double2(0.0, 0.0),
      (double2 *)C, ldc, 0, 0, 0, nullptr, w->err, 1);
  return pw_check_launch("oz gemm (real)");
}

pw_status pw_zgemm_oz(pw_oz_ws *w, char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                      int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc, cudaStream_t st,
                      int herm) {
  if ((opA != 'N' && opA != 'C') || (opB != 'N' && opB != 'C') || herm < 0 || herm > 5) return PW_ERR_ARG;
  if (m <= 0 || n <= 0) return PW_OK;
  if (k <= 0) return PW_ERR_ARG;
  if (herm == 1 && m != n) return PW_ERR_ARG;
  // Blocks of rows, columns and (for the modes whose predicates do not
  // depend on K) K, so that the slices of one block stay under the cap; K
  // blocks after the first accumulate into C (beta = 1).
  const size_t cap = std::max(w->bytes, (size_t)PW_OZ_SLICE_CAP);
  const double per_k = (double)S * 2 * 2;     // slice bytes per real row per complex K index
  int kc = k, mc = m, nc = n;
  auto bytes = [&]() { return per_k * ((double)mc + 2.0 * nc) * kc; };
  auto shrink_k = [&]() {
    if (herm <= 2)
      while (kc > 512 && bytes() > (double)cap) kc = (kc + 1) / 2;
  };
  // K longest (Gram-type products): K blocks first; otherwise rows and
  // columns first (K blocks cost a pass over C each)
  if ((double)k > (double)m + 2.0 * n) shrink_k();
  while (bytes() > (double)cap && (mc > BM || nc > BN / 2)) {
    if ((double)mc >= 2.0 * nc && mc > BM) mc = ((mc + 1) / 2 + BM - 1) / BM * BM;
    else if (nc > BN / 2) nc = ((nc + 1) / 2 + BN / 2 - 1) / (BN / 2) * (BN / 2);
    else mc = ((mc + 1) / 2 + BM - 1) / BM * BM;
  }
  shrink_k();
  const double2 one = make_double2(1.0, 0.0);
  for (int k0 = 0; k0 < k; k0 += kc) {
    const int kb = std::min(kc, k - k0);
    const double2 bt = k0 == 0 ? beta : one;
    for (int i0 = 0; i0 < m; i0 += mc) {
      const int mb = std::min(mc, m - i0);
      for (int j0 = 0; j0 < n; j0 += nc) {
        const int nb = std::min(nc, n - j0);
        // skip blocks the Hermitian modes leave alone
        if (herm == 1 && i0 > j0 + nb - 1) continue;
        if (herm == 2 && (j0 >> 6) > ((i0 + mb - 1) >> 6)) continue;
        PW_TRY(oz_block(w, opA, opB, mb, nb, kb, alpha, at(A, opA, lda, i0, k0), lda,
                        at(B, opB == 'N' ? 'C' : 'N', ldb, j0, k0), ldb, bt, C + i0 + (long)j0 * ldc, ldc, st,
                        herm, i0, j0));
      }
    }
  }
  if (herm == 1) {
    pw_count_launch();
    k_oz_mirror<<<dim3((m + 31) / 32, (m + 31) / 32), dim3(32, 32), 0, st>>>(C, ldc, m);
    PW_TRY(pw_check_launch("oz mirror"));
  }
  return PW_OK;
}

namespace {
std::atomic<int> g_f64_products{1};
// complex multiply-adds below which the FP64 pipe beats slicing the operands
constexpr double kOzMinMacs = 8.0 * (1 << 20);
}  // namespace

int pw_f64_products_mode() { return g_f64_products.load(); }

extern "C" pw_status pw_dense_products(int mode) {
  if (mode != 0 && mode != 1) return PW_ERR_ARG;
  g_f64_products.store(mode);
  return PW_OK;
}

bool pw_use_oz(int m, int n, int k) {
  return k > 0 && g_f64_products.load() == 1 && (double)m * n * k >= kOzMinMacs;
}

pw_status pw_gemm64(pw_oz_ws *w, char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                    int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc, double2 *ws,
                    size_t ws_elems, cudaStream_t st, int herm) {
  if (m <= 0 || n <= 0) return PW_OK;
  if (w && pw_use_oz(m, n, k))
    return pw_zgemm_oz(w, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st, herm);
  return pw_zgemm_ex(opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, st, herm);
}

extern "C" pw_status pw_zgemm_f64tc(char opA, char opB, int m, int n, int k, const double *alpha,
                                    const void *A, int lda, const void *B, int ldb, const double *beta, void *C,
                                    int ldc, void *stream) {
  if (!alpha || !beta || m < 0 || n < 0 || k < 1 || !A || !B || !C) return PW_ERR_ARG;
  if (ldc < m || lda < (opA == 'N' ? m : k) || ldb < (opB == 'N' ? k : n)) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  pw_oz_ws w;
  pw_status r = pw_zgemm_oz(&w, opA, opB, m, n, k, make_double2(alpha[0], alpha[1]), (const double2 *)A, lda,
                            (const double2 *)B, ldb, make_double2(beta[0], beta[1]), (double2 *)C, ldc, st, 0);
  if (r == PW_OK) r = pw_oz_check(&w, st);
  if (r == PW_OK && cudaStreamSynchronize(st) != cudaSuccess) r = PW_ERR_CUDA;
  pw_oz_free(&w);
  return r;
}
