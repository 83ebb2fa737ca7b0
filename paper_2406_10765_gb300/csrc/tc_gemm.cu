// Split-FP16 tensor-core GEMM for the mixed-precision path (tcgen05 + TMA,
// sm_103a).  These are the dense contractions of the step: the projector
// products of Sec. III-A and the subspace products S^H S, S^H (H S) and the
// rotations of Sec. II-B.
//
// Real core:  D[m][n] = sum_k sum_{(s,t) in pairs} A_s[m][k] B_t[n][k]
//   A_s, B_t: FP16 slices of scaled operands, K-major, rows padded, K a
//   multiple of 64; x * 2^e_row = hi + lo with hi = fp16(x 2^e), lo =
//   fp16(x 2^e - hi), |x 2^e| < 2^14.  Pairs (hi,hi), (hi,lo), (lo,hi) keep
//   ~22 significant bits of every product; accumulation is FP32 in TMEM.
//   Complex products use interleaved rows (re-row, im-row) so one real GEMM
//   yields the complex result; the epilogue removes the row scales in FP64.
//
// Kernel: one 128 x 128 output tile per CTA (and, with a K split, one of
// gridDim.y equal K ranges of it, partial sums reduced in FP64 by a second
// kernel in a fixed order); warp 0 = TMA producer, warp 1 =
// MMA issuer (one thread), warps 2-9 = epilogue (tcgen05.ld from TMEM).
// Three shared-memory stages of (A_hi, A_lo, B_hi, B_lo) = 64 KB each,
// 128-byte swizzle.  Each 64-wide K-block accumulates in a fresh TMEM buffer
// (two buffers), folded by the epilogue into compensated FP32 sums.  Every
// mbarrier wait is bounded (~1 s of clock); on timeout the CTA records an
// error, still frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "pw_internal.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int A_TILE = BM * BK * 2;          // 16 KB
constexpr int B_TILE = BN * BK * 2;          // 16 KB
constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;
constexpr int NSTAGE = 3;
constexpr int SMEM_BYTES = NSTAGE * STAGE + 1024 + 256;
constexpr int TMEM_COLS = 4 * BN;            // 2 accumulator buffers + compensation (+ spare)
constexpr int CMP_COL = 2 * BN;              // TMEM column of the compensation terms
constexpr int EPI_WARPS = 8;                 // 4 lane quarters x 2 column halves
constexpr int EPI_COLS = BN / 2;
// K blocks per TMEM accumulator buffer (K = 128): the tensor-core FP32
// accumulation rounds toward zero, so longer chunks bias positive sums
// (~2.5e-8 relative per MMA); two blocks keep the bias below ~1e-6
constexpr int CHUNK_KB = 2;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int GROUP_M = 16;                  // tile rows per group of the launch order
constexpr long long WAIT_CYCLES = 2000000000ll;   // ~1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after `limit` clocks without the phase completing
__device__ __forceinline__ bool mbar_wait_limit(uint64_t *bar, uint32_t parity, long long limit) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  return mbar_wait_limit(bar, parity, WAIT_CYCLES);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                          // swizzle: 128B
  return d;
}

// instruction descriptor, kind::f16: FP16 A and B, FP32 D, both K-major, M=128, N=BN
__host__ __device__ constexpr uint32_t idesc_f16() {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// two 32-column TMEM loads (accumulator and compensation) under one wait
__device__ __forceinline__ void tmem_ld32x2(uint32_t ta, uint32_t tb, float *va, float *vb) {
  uint32_t a[32], b[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]), "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31]),
        "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]), "=r"(b[16]), "=r"(b[17]), "=r"(b[18]), "=r"(b[19]), "=r"(b[20]), "=r"(b[21]), "=r"(b[22]), "=r"(b[23]), "=r"(b[24]), "=r"(b[25]), "=r"(b[26]), "=r"(b[27]), "=r"(b[28]), "=r"(b[29]), "=r"(b[30]), "=r"(b[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    va[i] = __uint_as_float(a[i]);
    vb[i] = __uint_as_float(b[i]);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 columns into TMEM; the caller waits (tcgen05.wait::st) before the
// columns are read again
__device__ __forceinline__ void tmem_st32_async(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// error-free sums s + x = t + err (Knuth's two-sum: t = s + x, z = t - s,
// err = (s - (t - z)) + (x - z)), err accumulated into e, on two lanes of
// packed FP32: one instruction per two round-to-nearest additions
__device__ __forceinline__ void two_sum_acc2(float &s0, float &s1, float &e0, float &e1, float x0, float x1) {
  const float2 s = make_float2(s0, s1), x = make_float2(x0, x1);
  const float2 t = __fadd2_rn(s, x);
  const float2 z = __fadd2_rn(t, make_float2(-s.x, -s.y));
  const float2 u = __fadd2_rn(t, make_float2(-z.x, -z.y));
  const float2 a = __fadd2_rn(s, make_float2(-u.x, -u.y));
  const float2 b = __fadd2_rn(x, make_float2(-z.x, -z.y));
  const float2 e = __fadd2_rn(make_float2(e0, e1), __fadd2_rn(a, b));
  s0 = t.x;
  s1 = t.y;
  e0 = e.x;
  e1 = e.y;
}

// Epilogue destinations (complex128 output, column-major, ldc):
//  ROWPAIR: real row r = 2i + c  ->  C[i + n ldc].{re,im}[c]   (A^H B products)
//  COLPAIR: real col n = 2j + c  ->  C[r + j ldc].{re,im}[c]   (A B products)
//
// Accumulation: every BK-wide K-block goes into a fresh TMEM accumulator
// (double-buffered); epilogue warps fold each block into compensated
// (two-sum) FP32 register sums, so the FP32 rounding of the tensor-core
// accumulator covers only 12 MMAs.
// Epilogue conversions on integer bits (FP64 issues at about two operations
// per clock per SM on this part).
// float -> double, exact; float subnormals (far below anything the FP16
// slices produce) flush to zero
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ed = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
// exponent k of a power-of-two row scale 2^k held as a float; a zero (or
// subnormal) scale gives a large negative k, so the product flushes to zero
__device__ __forceinline__ int pow2_exp(float s) {
  const int e = (int)((__float_as_uint(s) >> 23) & 0xFFu);
  return e == 0 ? -4096 : e - 127;
}
// x 2^k by exponent arithmetic; results below the normal range become zero
__device__ __forceinline__ double scale_pow2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return __longlong_as_double(b & (long long)0x8000000000000000ull);
  const int en = ex + k;
  if (en <= 0) return __longlong_as_double(b & (long long)0x8000000000000000ull);
  if (en >= 0x7FF) return __longlong_as_double((b & (long long)0x8000000000000000ull) | 0x7FF0000000000000ll);
  return __longlong_as_double(b + ((long long)k << 52));
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              int a_slice_rows, int b_slice_rows, int m, int n, int kblocks, int mtiles,
              int ntiles, const float *__restrict__ inv_sa, const float *__restrict__ inv_sb,
              double2 *__restrict__ C, int ldc, int mode, int accumulate, int herm_skip,
              int kb_lo, int tri_b, double *__restrict__ part, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + NSTAGE * STAGE);
  uint64_t *empty = full + NSTAGE;
  uint64_t *accf = empty + NSTAGE;       // [2] accumulator ready
  uint64_t *acce = accf + 2;             // [2] accumulator drained
  uint32_t *tmem_slot = (uint32_t *)(acce + 2);

  // grouped tile order: GROUP_M tile rows at a time, the row index varying
  // fastest, so that a wave of CTAs shares a few A row blocks and B column
  // blocks (its operands stay in L2) instead of sweeping all of B
  const int tile = blockIdx.x;
  const int grp = tile / (GROUP_M * ntiles), m_first = grp * GROUP_M;
  const int gsz = min(GROUP_M, mtiles - m_first), rem = tile - grp * GROUP_M * ntiles;
  const int mt = m_first + rem % gsz, nt = rem / gsz;
  if (mt >= mtiles || nt >= ntiles) return;
  const int m0 = mt * BM, n0 = nt * BN;
  // Hermitian products: skip tiles strictly below the diagonal (rows are
  // interleaved re/im pairs of output row i = r / 2)
  if (herm_skip && n0 + BN - 1 < m0 / 2) return;
  // K blocks of this tile: kb_lo.. (B zero below), and with tri_b (B rows
  // from an upper-triangular coefficient matrix) only K < n0 + BN is nonzero
  const int kb_end = tri_b ? min(kblocks, (n0 + BN + BK - 1) / BK) : kblocks;
  const int ntot = max(0, kb_end - kb_lo);
  // K split: part z of gridDim.y takes an equal share of the tile's K blocks
  const int per = (ntot + (int)gridDim.y - 1) / (int)gridDim.y;
  const int z0 = min(ntot, (int)blockIdx.y * per), z1 = min(ntot, z0 + per);
  const int kb_beg = kb_lo + z0;
  const int nkb = z1 - z0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], EPI_WARPS); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      for (int i = 0; i < nkb; ++i) {
        const int s = i % NSTAGE;
        const uint32_t u = i / NSTAGE;
        if (!mbar_wait(&empty[s], (u & 1) ^ 1)) { atomicOr(err, 1); break; }
        unsigned char *st = smem + s * STAGE;
        mbar_expect_tx(&full[s], STAGE);
        const int x = (kb_beg + i) * BK;
        tma_load_2d(st, &mapA, &full[s], x, m0);
        tma_load_2d(st + A_TILE, &mapA, &full[s], x, a_slice_rows + m0);
        tma_load_2d(st + 2 * A_TILE, &mapB, &full[s], x, n0);
        tma_load_2d(st + 2 * A_TILE + B_TILE, &mapB, &full[s], x, b_slice_rows + n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: CHUNK_KB K-blocks per accumulator buffer
      const uint32_t idesc = idesc_f16();
      const int nchunk = (nkb + CHUNK_KB - 1) / CHUNK_KB;
      // operand descriptors of every stage, formed once; a K step of 16
      // (32 bytes) adds 2 to the start-address field
      uint64_t dA0[NSTAGE], dA1[NSTAGE], dB0[NSTAGE], dB1[NSTAGE];
#pragma unroll
      for (int s = 0; s < NSTAGE; ++s) {
        const uint32_t a0 = smem_u32(smem + s * STAGE);
        dA0[s] = smem_desc(a0);
        dA1[s] = smem_desc(a0 + A_TILE);
        dB0[s] = smem_desc(a0 + 2 * A_TILE);
        dB1[s] = smem_desc(a0 + 2 * A_TILE + B_TILE);
      }
      bool ok = true;
      for (int ch = 0; ch < nchunk && ok; ++ch) {
        const int b = ch & 1;
        const uint32_t ub = ch >> 1;
        if (!mbar_wait(&acce[b], (ub & 1) ^ 1)) { atomicOr(err, 8); break; }
        const uint32_t d = tmem + (uint32_t)(b * BN);
        const int kb1 = min(nkb, (ch + 1) * CHUNK_KB);
        for (int kb = ch * CHUNK_KB; kb < kb1; ++kb) {
          const int s = kb % NSTAGE;
          const uint32_t u = kb / NSTAGE;
          if (!mbar_wait(&full[s], u & 1)) { atomicOr(err, 2); ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          uint64_t a0, a1, b0, b1;
          // stage s of a runtime index: select among the precomputed descriptors
#pragma unroll
          for (int t = 0; t < NSTAGE; ++t)
            if (t == s) { a0 = dA0[t]; a1 = dA1[t]; b0 = dB0[t]; b1 = dB1[t]; }
          const bool first = kb == ch * CHUNK_KB;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t o = 2 * kk;
            mma_f16(d, a0 + o, b0 + o, idesc, !(first && kk == 0));
            mma_f16(d, a0 + o, b1 + o, idesc, 1);
            mma_f16(d, a1 + o, b0 + o, idesc, 1);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&accf[b]);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; lane quarter q, column half h.
    // Running sums live in registers, their compensation terms in TMEM.
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    const uint32_t cmp_base = tmem + lanes + (uint32_t)(CMP_COL + h * EPI_COLS);
    float sum[EPI_COLS];
#pragma unroll
    for (int i = 0; i < EPI_COLS; ++i) sum[i] = 0.0f;
    {
      float z[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) z[i] = 0.0f;
#pragma unroll
      for (int c0 = 0; c0 < EPI_COLS; c0 += 32) tmem_st32(cmp_base + c0, z);
    }
    bool ok = true;
    const int nchunk = (nkb + CHUNK_KB - 1) / CHUNK_KB;
    for (int ch = 0; ch < nchunk; ++ch) {
      const int b = ch & 1;
      const uint32_t ub = ch >> 1;
      if (!mbar_wait(&accf[b], ub & 1)) { atomicOr(err, 4); ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = tmem + lanes + (uint32_t)(b * BN + h * EPI_COLS);
#pragma unroll
      for (int c0 = 0; c0 < EPI_COLS; c0 += 32) {
        float v[32], e[32];
        tmem_ld32x2(base + c0, cmp_base + c0, v, e);
#pragma unroll
        for (int i = 0; i < 32; i += 2) two_sum_acc2(sum[c0 + i], sum[c0 + i + 1], e[i], e[i + 1], v[i], v[i + 1]);
        tmem_st32_async(cmp_base + c0, e);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
    float cmp[EPI_COLS];
#pragma unroll
    for (int c0 = 0; c0 < EPI_COLS; c0 += 32) tmem_ld32(cmp_base + c0, cmp + c0);
    const int r = m0 + q * 32 + lane;            // output (real) row of this thread
    if (ok && r < m && part) {
      // K split: this part's sums, real layout part[z][col][r], scaled
      const int ka = pow2_exp(inv_sa[r]);
      const int cb = n0 + h * EPI_COLS;
      double *pz = part + (long)blockIdx.y * n * m;
#pragma unroll
      for (int t = 0; t < EPI_COLS; ++t) {
        const int col = cb + t;
        if (col < n)
          pz[(long)col * m + r] = scale_pow2(f2d_bits(sum[t]) + f2d_bits(cmp[t]), ka + pow2_exp(inv_sb[col]));
      }
    } else if (ok && r < m) {
      // value = (sum + cmp) 2^(ka + kb): one FP64 add, the rest on integer bits
      const int ka = pow2_exp(inv_sa[r]);
      const int cb = n0 + h * EPI_COLS;
      if (mode == 0) {                         // ROWPAIR
        const int i = r >> 1, c = r & 1;
#pragma unroll
        for (int t = 0; t < EPI_COLS; ++t) {
          const int col = cb + t;
          if (col < n) {
            double *dst = (double *)&C[i + (long)col * ldc] + c;
            const double val = scale_pow2(f2d_bits(sum[t]) + f2d_bits(cmp[t]), ka + pow2_exp(inv_sb[col]));
            *dst = accumulate ? *dst + val : val;
          }
        }
      } else {                                 // COLPAIR
#pragma unroll
        for (int t = 0; t < EPI_COLS; t += 2) {
          const int col = cb + t;
          if (col < n) {
            double2 *dst = &C[r + (long)(col >> 1) * ldc];
            const double re = scale_pow2(f2d_bits(sum[t]) + f2d_bits(cmp[t]), ka + pow2_exp(inv_sb[col]));
            const double im =
                scale_pow2(f2d_bits(sum[t + 1]) + f2d_bits(cmp[t + 1]), ka + pow2_exp(inv_sb[col + 1]));
            if (accumulate) { double2 o = *dst; o.x += re; o.y += im; *dst = o; }
            else *dst = make_double2(re, im);
          }
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

// -------------------------------------------------------------- splits ----
// The splits below run on integer and FP32 arithmetic only: FP64 issues at
// about two operations per clock per SM on this part, which made the split
// kernels FP64-bound at several times their memory time.

// |x| as ordered integer bits (for non-negative doubles the integer order is
// the numeric order)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// x 2^sh rounded to the nearest float, ties to even, from the bit pattern;
// magnitudes below the smallest normal float become a signed zero (they are
// far below what the two FP16 slices can hold after the row scaling)
__device__ __forceinline__ float d2f_pow2(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return __uint_as_float(sign);
  e += sh - 1023 + 127;
  unsigned m = (unsigned)((b >> 29) & 0x7FFFFFu);      // top 23 of the 52 fraction bits
  const unsigned rest = (unsigned)(b & 0x1FFFFFFFu);    // the 29 dropped bits
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) {
    if (++m == 0x800000u) { m = 0; ++e; }
  }
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | m);
}

// hi = fp16(x), lo = fp16(x - hi); x - hi is exact in FP32
__device__ __forceinline__ void split2f(float x, __half &hi, __half &lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn(x - __half2float(hi));
}

__device__ __forceinline__ unsigned long long warp_maxu(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ unsigned long long block_maxu(unsigned long long v) {
  __shared__ unsigned long long shm[32];
  v = warp_maxu(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = shm[w] > r ? shm[w] : r;
  __syncthreads();
  return r;
}

// exponent sh of the power-of-two row scale 2^sh (max 2^sh in [2^13, 2^14))
__device__ __forceinline__ int pow2_shift(double mx, float *inv) {
  if (!(mx > 0.0)) { *inv = 1.0f; return 0; }
  int e;
  frexp(mx, &e);
  const int sh = 14 - e;
  *inv = ldexpf(1.0f, -sh);
  return sh;
}

// Rows from columns: for each column c of X (npw x ncols, ld), real rows
//   conj=0:  row c       = (re, im) interleaved over g
//   conj=1:  row 2c      = (re, im),   row 2c + 1 = (-im, re)
// out: slices [2][rows_total][kpad] (hi then lo), inv scale per row.
__global__ void __launch_bounds__(256) k_split_rows(const double2 *__restrict__ X, int ld, int npw,
                                                    int ncols, int conj, int kpad, int rows_total,
                                                    __half *__restrict__ out,
                                                    float *__restrict__ inv_scale,
                                                    const double *__restrict__ colscale) {
  const int c = blockIdx.x;
  const double2 *x = X + (long)c * ld;
  const double cs = colscale ? colscale[c] : 1.0;
  unsigned long long mb = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 v = x[g];
    const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
    const unsigned long long t = a > b ? a : b;
    mb = t > mb ? t : mb;
  }
  mb = block_maxu(mb);
  float inv;
  const int sh = pow2_shift(__longlong_as_double((long long)mb) * fabs(cs) * 1.0000001, &inv);
  const long slice = (long)rows_total * kpad;
  const int r0 = conj ? 2 * c : c;
  if (threadIdx.x == 0) { inv_scale[r0] = inv; if (conj) inv_scale[r0 + 1] = inv; }
  __half *o0 = out + (long)r0 * kpad;
  for (int g = threadIdx.x; g < kpad / 2; g += blockDim.x) {
    float re = 0.0f, im = 0.0f;
    if (g < npw) {
      double2 v = x[g];
      if (colscale) { v.x *= cs; v.y *= cs; }
      re = d2f_pow2(v.x, sh);
      im = d2f_pow2(v.y, sh);
    }
    __half h, l;
    split2f(re, h, l); o0[2 * g] = h; o0[slice + 2 * g] = l;
    split2f(im, h, l); o0[2 * g + 1] = h; o0[slice + 2 * g + 1] = l;
    if (conj) {
      __half *o1 = o0 + kpad;
      split2f(-im, h, l); o1[2 * g] = h; o1[slice + 2 * g] = l;
      split2f(re, h, l); o1[2 * g + 1] = h; o1[slice + 2 * g + 1] = l;
    }
  }
}

// Transposed rows: for each g of X (npw x ncols), row g = (re, im) over the
// columns t (K = 2 ncols).  Per-row scale from the row maximum.
__global__ void __launch_bounds__(256) k_rowmax(const double2 *__restrict__ X, int ld, int npw,
                                                int ncols, float *__restrict__ rmax) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npw) return;
  unsigned long long m = 0;
  for (int t = 0; t < ncols; ++t) {
    const double2 v = X[g + (long)t * ld];
    const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
    const unsigned long long u = a > b ? a : b;
    m = u > m ? u : m;
  }
  // rounded up to a float so that the scale never undercounts the maximum
  const double md = __longlong_as_double((long long)m);
  float mf = d2f_pow2(md, 0);
  if ((double)mf < md) mf = __uint_as_float(__float_as_uint(mf) + 1u);
  rmax[g] = mf;
}

__global__ void __launch_bounds__(256) k_split_trans(const double2 *__restrict__ X, int ld, int npw,
                                                     int ncols, int kpad, int rows_total,
                                                     const float *__restrict__ rmax,
                                                     __half *__restrict__ out,
                                                     float *__restrict__ inv_scale) {
  // tile: 32 rows (g) x 64 columns (t); read coalesced along g, write along t
  __shared__ double2 tileS[64][33];
  const int g0 = blockIdx.x * 32, t0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8
  for (int tt = ty; tt < 64; tt += 8) {
    const int g = g0 + tx, t = t0 + tt;
    double2 v = make_double2(0.0, 0.0);
    if (g < npw && t < ncols) v = X[g + (long)t * ld];
    tileS[tt][tx] = v;
  }
  __syncthreads();
  const long slice = (long)rows_total * kpad;
  for (int gg = ty; gg < 32; gg += 8) {
    const int g = g0 + gg;
    if (g >= npw) continue;
    float inv;
    const int sh = pow2_shift((double)rmax[g] * 1.0000001, &inv);
    if (blockIdx.y == 0 && tx == 0) inv_scale[g] = inv;
    __half *o = out + (long)g * kpad;
    for (int tt = tx; tt < 64; tt += 32) {
      const int t = t0 + tt;
      if (2 * t >= kpad) continue;
      const double2 v = tileS[tt][gg];
      __half h, l;
      split2f(d2f_pow2(v.x, sh), h, l); o[2 * t] = h; o[slice + 2 * t] = l;
      split2f(d2f_pow2(v.y, sh), h, l); o[2 * t + 1] = h; o[slice + 2 * t + 1] = l;
    }
  }
}

// Coefficient rows for A B products: for column j of Cm (kdim x ncols, ld):
//   row 2j = (re, -im) over t,  row 2j + 1 = (im, re)
// optional per-row (t) real factor d[t] applied first.
__global__ void __launch_bounds__(256) k_split_coef(const double2 *__restrict__ Cm, int ld, int kdim,
                                                    int ncols, const double *__restrict__ d,
                                                    int kpad, int rows_total,
                                                    __half *__restrict__ out,
                                                    float *__restrict__ inv_scale) {
  const int j = blockIdx.x;
  const double2 *x = Cm + (long)j * ld;
  unsigned long long mb = 0;
  for (int t = threadIdx.x; t < kdim; t += blockDim.x) {
    double2 v = x[t];
    if (d) { v.x *= d[t]; v.y *= d[t]; }
    const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
    const unsigned long long u = a > b ? a : b;
    mb = u > mb ? u : mb;
  }
  mb = block_maxu(mb);
  float inv;
  const int sh = pow2_shift(__longlong_as_double((long long)mb) * 1.0000001, &inv);
  if (threadIdx.x == 0) { inv_scale[2 * j] = inv; inv_scale[2 * j + 1] = inv; }
  const long slice = (long)rows_total * kpad;
  __half *o0 = out + (long)(2 * j) * kpad, *o1 = o0 + kpad;
  for (int t = threadIdx.x; t < kpad / 2; t += blockDim.x) {
    float re = 0.0f, im = 0.0f;
    if (t < kdim) {
      double2 v = x[t];
      if (d) { v.x *= d[t]; v.y *= d[t]; }
      re = d2f_pow2(v.x, sh);
      im = d2f_pow2(v.y, sh);
    }
    __half h, l;
    split2f(re, h, l); o0[2 * t] = h; o0[slice + 2 * t] = l;
    split2f(-im, h, l); o0[2 * t + 1] = h; o0[slice + 2 * t + 1] = l;
    split2f(im, h, l); o1[2 * t] = h; o1[slice + 2 * t] = l;
    split2f(re, h, l); o1[2 * t + 1] = h; o1[slice + 2 * t + 1] = l;
  }
}

// The bounded wait of the GEMM pipeline on a barrier that nothing arrives
// on: it must give up after `limit` clocks and report, leaving the context
// usable (failure detection without a fault or a hang).
__global__ void k_wait_selftest(long long limit, int *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_limit(&bar, 0, limit)) atomicOr(err, 16);
}

// sum of the K-split parts (in part order) into C, same destinations and
// tile selection as the single-part epilogue
__global__ void k_tc_reduce(const double *__restrict__ part, int splits, int m, int n,
                            double2 *__restrict__ C, int ldc, int mode, int accumulate, int herm_skip) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)m * n) return;
  const int r = (int)(idx % m), col = (int)(idx / m);
  if (herm_skip && (col / BN) * BN + BN - 1 < ((r / BM) * BM) / 2) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[(long)z * m * n + idx];
  double *dst = mode == 0 ? (double *)&C[(r >> 1) + (long)col * ldc] + (r & 1)
                          : (double *)&C[r + (long)(col >> 1) * ldc] + (col & 1);
  *dst = accumulate ? *dst + s : s;
}

// lower triangle <- conj(upper) for an n x n complex matrix (ld)
__global__ void k_mirror_lower(double2 *G, int ld, int n) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= n || j >= n || i <= j) return;
  const double2 u = G[j + (long)i * ld];
  G[i + (long)j * ld] = make_double2(u.x, -u.y);
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

bool make_map(CUtensorMap *map, const void *base, int kpad, int rows_total, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// ------------------------------------------------------------------ host ----

int pw_tc_kpad(int kreal) { return (kreal + BK - 1) / BK * BK; }

pw_status pw_tc_split_rows(const double2 *X, int ld, int npw, int ncols, int conj, const double *colscale,
                           pw_tc_operand *op, cudaStream_t st) {
  if (op->rows_total < (conj ? 2 : 1) * ncols || op->kpad < 2 * npw) return PW_ERR_ARG;
  pw_count_launch();
  k_split_rows<<<ncols, 256, 0, st>>>(X, ld, npw, ncols, conj, op->kpad, op->rows_total, op->data,
                                      op->inv_scale, colscale);
  return pw_check_launch("split_rows");
}

pw_status pw_tc_split_trans(const double2 *X, int ld, int npw, int ncols, float *rmax_ws,
                            pw_tc_operand *op, cudaStream_t st) {
  if (op->rows_total < npw || op->kpad < 2 * ncols) return PW_ERR_ARG;
  pw_count_launch();
  k_rowmax<<<(npw + 255) / 256, 256, 0, st>>>(X, ld, npw, ncols, rmax_ws);
  pw_count_launch();
  k_split_trans<<<dim3((npw + 31) / 32, (op->kpad / 2 + 63) / 64), 256, 0, st>>>(
      X, ld, npw, ncols, op->kpad, op->rows_total, rmax_ws, op->data, op->inv_scale);
  return pw_check_launch("split_trans");
}

pw_status pw_tc_split_coef(const double2 *Cm, int ld, int kdim, int ncols, const double *d,
                           pw_tc_operand *op, cudaStream_t st) {
  if (op->rows_total < 2 * ncols || op->kpad < 2 * kdim) return PW_ERR_ARG;
  pw_count_launch();
  k_split_coef<<<ncols, 256, 0, st>>>(Cm, ld, kdim, ncols, d, op->kpad, op->rows_total, op->data,
                                      op->inv_scale);
  return pw_check_launch("split_coef");
}

// ------------------------------------------------------- K-split tuning ----
// A product shape with few output tiles and long K leaves SMs idle; splitting
// K over gridDim.y fills them at the cost of an FP64 partial-sum pass.  The
// split is a tile-shape choice (128 x 128 x K/s): fixed at 1, forced, or
// picked per shape by timing the candidates on first use (the autotuner).
namespace {

constexpr int kWaveTiles = 4 * 152;                 // shapes with fewer tiles are tuned
constexpr size_t kPartBytesMax = (size_t)256 << 20; // partial sums of one product

// shape class of a product: output tiles, K blocks rounded up to a power of
// two (cells of nearby sizes share a choice), the K bounds and the layout
struct GemmKey {
  int mtiles, ntiles, kclass, kb_lo, tri_b, herm, mode;
  bool operator<(const GemmKey &o) const {
    return std::tie(mtiles, ntiles, kclass, kb_lo, tri_b, herm, mode) <
           std::tie(o.mtiles, o.ntiles, o.kclass, o.kb_lo, o.tri_b, o.herm, o.mode);
  }
};
GemmKey make_key(int m, int n, int kblocks, int kb_lo, int tri_b, int herm, int mode) {
  int kc = 1;
  while (kc < kblocks - kb_lo) kc *= 2;
  return GemmKey{(m + BM - 1) / BM, (n + BN - 1) / BN, kc, kb_lo, tri_b, herm, mode};
}
struct GemmChoice {
  int split;
  float ms_one, ms_best;   // timed at split 1 and at the chosen split
};

std::mutex g_tune_mu;
int g_tune_mode = 0, g_tune_split = 1;
std::map<GemmKey, GemmChoice> g_tune_table;

// largest split worth trying: at least 4 K blocks per part, bounded partial sums
int max_split(int m, int n, int kblocks, int kb_lo) {
  const int ntot = kblocks - kb_lo;
  int s = std::min(16, std::max(1, ntot / 4));
  while (s > 1 && (size_t)s * m * n * sizeof(double) > kPartBytesMax) --s;
  return s;
}

// keep freed partial-sum buffers in the device's stream-ordered pool
void pool_keep() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> g(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = kPartBytesMax;   // keep partial-sum buffers between calls
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

pw_status launch_gemm(const CUtensorMap &ma, const CUtensorMap &mb, const pw_tc_operand *A,
                      const pw_tc_operand *B, int m, int n, double2 *C, int ldc, int mode, int accumulate,
                      int herm, int *d_err, cudaStream_t st, int kb_lo, int tri_b, int split) {
  const int mtiles = (m + BM - 1) / BM, ntiles = (n + BN - 1) / BN;
  double *part = nullptr;
  if (split > 1) {
    pool_keep();
    PW_CUDA(cudaMallocAsync((void **)&part, (size_t)split * m * n * sizeof(double), st));
  }
  pw_count_launch();
  k_tc_gemm<<<dim3(mtiles * ntiles, split), NTHREADS, SMEM_BYTES, st>>>(
      ma, mb, A->rows_total, B->rows_total, m, n, A->kpad / BK, mtiles, ntiles, A->inv_scale, B->inv_scale, C,
      ldc, mode, accumulate, herm, kb_lo, tri_b, part, d_err);
  pw_status r = pw_check_launch("tc_gemm");
  if (split > 1) {
    if (r == PW_OK) {
      pw_count_launch();
      k_tc_reduce<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, st>>>(part, split, m, n, C, ldc, mode,
                                                                          accumulate, herm);
      r = pw_check_launch("tc_gemm reduce");
    }
    cudaFreeAsync(part, st);
  }
  PW_TRY(r);
  if (herm) {
    const int ni = m / 2;
    pw_count_launch();
    k_mirror_lower<<<dim3((ni + 31) / 32, (ni + 31) / 32), dim3(32, 32), 0, st>>>(C, ldc, ni);
    PW_TRY(pw_check_launch("mirror"));
  }
  return PW_OK;
}

// times every candidate split on a scratch output; returns the fastest
pw_status tune_split(const GemmKey &key, int m, int n, int smax, const CUtensorMap &ma, const CUtensorMap &mb,
                     const pw_tc_operand *A, const pw_tc_operand *B, int *d_err, cudaStream_t st,
                     GemmChoice *out) {
  const int ldc = key.mode == 0 ? (m + 1) / 2 : m;
  const size_t cols = key.mode == 0 ? (size_t)n : (size_t)(n + 1) / 2;
  double2 *Cs = nullptr;
  PW_CUDA(cudaMallocAsync((void **)&Cs, (size_t)ldc * cols * sizeof(double2), st));
  cudaEvent_t e0, e1;
  PW_CUDA(cudaEventCreate(&e0));
  PW_CUDA(cudaEventCreate(&e1));
  pw_status r = PW_OK;
  GemmChoice best{1, 0.0f, 0.0f};
  for (int s = 1; s <= smax && r == PW_OK; s = s < 4 ? s + 1 : s * 2) {
    float ms = 1e30f;
    pw_status rs = PW_OK;
    for (int rep = 0; rep < 3 && rs == PW_OK; ++rep) {
      cudaEventRecord(e0, st);
      rs = launch_gemm(ma, mb, A, B, m, n, Cs, ldc, key.mode, 0, key.herm, d_err, st, key.kb_lo, key.tri_b, s);
      cudaEventRecord(e1, st);
      float t = 0.0f;
      if (rs == PW_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
          rep > 0)
        ms = std::min(ms, t);
    }
    if (s == 1) {
      r = rs;   // the single-part product must run
      best = GemmChoice{1, ms, ms};
    } else if (rs != PW_OK) {
      cudaGetLastError();   // e.g. no room for the partial sums: stop at the splits that ran
      break;
    } else if (ms < best.ms_best) {
      best.split = s;
      best.ms_best = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(Cs, st);
  if (r == PW_OK) *out = best;
  return r;
}

}  // namespace

extern "C" pw_status pw_autotune_gemm(int mode, int split) {
  if (mode < 0 || mode > 2 || (mode == 2 && split < 1)) return PW_ERR_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_mode = mode;
  g_tune_split = mode == 2 ? split : 1;
  if (mode == 0) g_tune_table.clear();
  return PW_OK;
}

extern "C" int pw_autotune_gemm_table(char *buf, size_t len) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  std::string s;
  for (const auto &kv : g_tune_table) {
    const GemmKey &k = kv.first;
    char line[256];
    snprintf(line, sizeof line,
             "mtiles=%d ntiles=%d k<=%d k_lo=%d tri_b=%d herm=%d mode=%d split=%d ms1=%.4f ms=%.4f\n",
             k.mtiles, k.ntiles, k.kclass * BK, k.kb_lo * BK, k.tri_b, k.herm, k.mode, kv.second.split, kv.second.ms_one,
             kv.second.ms_best);
    s += line;
  }
  if (buf && len) {
    const size_t c = std::min(len - 1, s.size());
    memcpy(buf, s.data(), c);
    buf[c] = 0;
  }
  return (int)g_tune_table.size();
}

extern "C" int pw_autotune_gemm_load(const char *text) {
  if (!text) return -1;
  // parse into a local table first: a dump with a bad line changes nothing
  std::map<GemmKey, GemmChoice> parsed;
  int added = 0;
  const char *p = text;
  while (*p) {
    const char *e = strchr(p, '\n');
    const std::string line(p, e ? (size_t)(e - p) : strlen(p));
    p = e ? e + 1 : p + line.size();
    if (line.empty()) continue;
    GemmKey k{};
    int kmax = 0, klo = 0, split = 0;
    float ms1 = 0.0f, ms = 0.0f;
    if (sscanf(line.c_str(), "mtiles=%d ntiles=%d k<=%d k_lo=%d tri_b=%d herm=%d mode=%d split=%d ms1=%f ms=%f",
               &k.mtiles, &k.ntiles, &kmax, &klo, &k.tri_b, &k.herm, &k.mode, &split, &ms1, &ms) != 10 ||
        k.mtiles < 1 || k.ntiles < 1 || kmax < BK || kmax % BK || klo < 0 || klo % BK || split < 1 || split > 16)
      return -1;
    k.kclass = kmax / BK;
    k.kb_lo = klo / BK;
    parsed[k] = GemmChoice{split, ms1, ms};
    ++added;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (const auto &kv : parsed) g_tune_table[kv.first] = kv.second;
  return added;
}

pw_status pw_tc_gemm(const pw_tc_operand *A, int m, const pw_tc_operand *B, int n, double2 *C, int ldc,
                     int mode, int accumulate, int herm, int *d_err, cudaStream_t st, int kb_lo, int tri_b) {
  if (A->kpad != B->kpad || m > A->rows_total || n > B->rows_total || m <= 0 || n <= 0) return PW_ERR_ARG;
  if (kb_lo < 0 || kb_lo > A->kpad / BK) return PW_ERR_ARG;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A->data, A->kpad, 2 * A->rows_total, BM) ||
      !make_map(&mb, B->data, B->kpad, 2 * B->rows_total, BN))
    return PW_ERR_CUDA;
  // per-device kernel attribute (set on every call: cheap, thread-safe, and
  // correct on every device the caller uses)
  PW_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  const GemmKey key = make_key(m, n, A->kpad / BK, kb_lo, tri_b, herm, mode);
  const int tiles = key.mtiles * key.ntiles;
  const int smax = max_split(m, n, A->kpad / BK, kb_lo);
  int split = 1, tmode;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tmode = g_tune_mode;
    if (tmode == 2) split = g_tune_split;
    if (tmode == 1) {
      auto it = g_tune_table.find(key);
      if (it != g_tune_table.end()) { split = it->second.split; tmode = 0; }
    }
  }
  if (tmode == 1) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (tiles < kWaveTiles && smax > 1 && cs == cudaStreamCaptureStatusNone) {
      GemmChoice ch;
      PW_TRY(tune_split(key, m, n, smax, ma, mb, A, B, d_err, st, &ch));
      split = ch.split;
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tune_table[key] = ch;
    }
  }
  split = std::max(1, std::min(split, smax));
  return launch_gemm(ma, mb, A, B, m, n, C, ldc, mode, accumulate, herm, d_err, st, kb_lo, tri_b, split);
}

pw_status pw_tc_operand_alloc(pw_tc_operand *op, int rows, int kreal, cudaStream_t st) {
  const int kpad = pw_tc_kpad(kreal);
  const int rows_pad = (rows + 255) / 256 * 256;
  const size_t bytes = (size_t)2 * rows_pad * kpad * sizeof(__half);   // rows padded to 256
  if (op->data && op->cap_bytes >= bytes && op->scale_cap >= rows_pad) {
    op->rows_total = rows_pad;
    op->kpad = kpad;
    return PW_OK;
  }
  pw_tc_operand_free(op);
  if (cudaMalloc(&op->data, bytes) != cudaSuccess ||
      cudaMalloc(&op->inv_scale, (size_t)rows_pad * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    pw_tc_operand_free(op);
    return PW_ERR_OOM;
  }
  // padded rows and K must read as zeros: cleared on the caller's stream so
  // the clearing is ordered before the kernels that fill the operand
  PW_CUDA(cudaMemsetAsync(op->data, 0, bytes, st));
  PW_CUDA(cudaMemsetAsync(op->inv_scale, 0, (size_t)rows_pad * sizeof(float), st));
  op->cap_bytes = bytes;
  op->scale_cap = rows_pad;
  op->rows_total = rows_pad;
  op->kpad = kpad;
  return PW_OK;
}

void pw_tc_operand_free(pw_tc_operand *op) {
  if (op->data) cudaFree(op->data);
  if (op->inv_scale) cudaFree(op->inv_scale);
  *op = pw_tc_operand();
}

extern "C" pw_status pw_zgemm_tc(char opA, int m, int n, int k, const void *A, int lda, const void *B,
                                 int ldb, double beta, void *C, int ldc, void *stream) {
  if ((opA != 'C' && opA != 'N') || m < 1 || n < 1 || k < 1 || !A || !B || !C ||
      (beta != 0.0 && beta != 1.0) || ldc < m)
    return PW_ERR_ARG;
  if (opA == 'C' ? (lda < k || ldb < k) : (lda < m || ldb < k)) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  pw_tc_operand a, b;
  int *err = nullptr;
  float *rmax = nullptr;
  pw_status r = PW_OK;
  const double2 *Ad = (const double2 *)A, *Bd = (const double2 *)B;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return PW_ERR_OOM; }
  cudaMemsetAsync(err, 0, sizeof(int), st);
  if (opA == 'C') {
    if ((r = pw_tc_operand_alloc(&a, 2 * m, 2 * k, st)) == PW_OK &&
        (r = pw_tc_operand_alloc(&b, n, 2 * k, st)) == PW_OK &&
        (r = pw_tc_split_rows(Ad, lda, k, m, 1, nullptr, &a, st)) == PW_OK &&
        (r = pw_tc_split_rows(Bd, ldb, k, n, 0, nullptr, &b, st)) == PW_OK)
      r = pw_tc_gemm(&a, 2 * m, &b, n, (double2 *)C, ldc, 0, beta != 0.0, 0, err, st);
  } else {
    if (cudaMalloc(&rmax, (size_t)m * sizeof(float)) != cudaSuccess) { cudaGetLastError(); r = PW_ERR_OOM; }
    if (r == PW_OK && (r = pw_tc_operand_alloc(&a, m, 2 * k, st)) == PW_OK &&
        (r = pw_tc_operand_alloc(&b, 2 * n, 2 * k, st)) == PW_OK &&
        (r = pw_tc_split_trans(Ad, lda, m, k, rmax, &a, st)) == PW_OK &&
        (r = pw_tc_split_coef(Bd, ldb, k, n, nullptr, &b, st)) == PW_OK)
      r = pw_tc_gemm(&a, m, &b, 2 * n, (double2 *)C, ldc, 1, beta != 0.0, 0, err, st);
  }
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    r = PW_ERR_CUDA;
  if (r == PW_OK && herr) r = PW_ERR_TIMEOUT;
  cudaFree(err);
  if (rmax) cudaFree(rmax);
  pw_tc_operand_free(&a);
  pw_tc_operand_free(&b);
  return r;
}

extern "C" pw_status pw_selftest_bounded_wait(long long cycles, void *stream) {
  if (cycles < 1 || cycles > WAIT_CYCLES) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int *d_err = nullptr, herr = 0;
  PW_CUDA(cudaMalloc(&d_err, sizeof(int)));
  pw_status r = PW_OK;
  if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) r = PW_ERR_CUDA;
  if (r == PW_OK) {
    pw_count_launch();
    k_wait_selftest<<<1, 32, 0, st>>>(cycles, d_err);
    r = pw_check_launch("wait selftest");
  }
  if (r == PW_OK && (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
    r = PW_ERR_CUDA;
  cudaFree(d_err);
  if (r != PW_OK) return r;
  return herr ? PW_ERR_TIMEOUT : PW_ERR_NUMERIC;   // the wait must have run out
}
