// Device helpers shared by the tensor-core kernels that compute FP64-accurate
// products from integer slices on the FP16 tensor cores (tcgen05 MMA with
// tensor-memory accumulators, mbarrier-paced shared-memory stages): inline
// PTX wrappers, bounded mbarrier waits, shared-memory matrix descriptors, and
// the integer digit split of an FP64 value.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "oz_gemm.cuh"

namespace pw_umma {

constexpr int S = PW_OZ_SLICES;        // digits per FP64 value
constexpr int BETA = 7;                // bits per digit
constexpr long long WAIT_CYCLES = 2000000000ll;   // ~1 s at the top SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// bounded wait: false after WAIT_CYCLES clocks without the phase completing
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > WAIT_CYCLES) return false;
  return true;
}
// contiguous global -> shared copy completing on an mbarrier (both addresses
// 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor (sm_100 family): start address, leading and
// stride byte offsets, swizzle mode (2 = 128 B, 4 = 64 B)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)swz << 61;
  return d;
}
// instruction descriptor, kind::f16: FP16 A and B, FP32 D, M x N; A read
// MN-major when a_mn (B always K-major)
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n, bool a_mn) {
  return (1u << 4) | ((a_mn ? 1u : 0u) << 15) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r) {
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
}

// x 2^k by exponent arithmetic (x finite); results below the normal range are zero
__device__ __forceinline__ double scale_pow2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return __longlong_as_double(b & (long long)0x8000000000000000ull);
  const int en = ex + k;
  if (en <= 0) return __longlong_as_double(b & (long long)0x8000000000000000ull);
  if (en >= 0x7FF) return __longlong_as_double((b & (long long)0x8000000000000000ull) | 0x7FF0000000000000ll);
  return __longlong_as_double(b + ((long long)k << 52));
}

// An FP32 accumulator value holding an integer |v| < 2^22, as an int: adding
// 1.5 * 2^23 puts the integer into the low mantissa bits
__device__ __forceinline__ int f2i_exact(uint32_t bits) {
  const float v = __uint_as_float(bits) + 12582912.0f;
  return __float_as_int(v) - 0x4B400000;
}

// v 2^sh into a 64-bit fixed-point sum (sh < 0: rounded to nearest)
__device__ __forceinline__ long long shifted(int v, int sh) {
  if (sh >= 0) return (long long)v << sh;
  return ((long long)v + (1ll << (-sh - 1))) >> (-sh);
}

// |x| as ordered integer bits
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// exponent e with max 2^e in [1/2, 1) from the bits of a maximum
__device__ __forceinline__ int row_exp(unsigned long long mb) {
  const int ex = (int)(mb >> 52);
  if (ex == 0) return 0;                 // zero (or subnormal): any scale works
  return 1022 - ex;                      // max in [2^(ex-1023), 2^(ex-1022)) -> [1/2, 1)
}
// the S digits of x 2^e (|x 2^e| < 1): the fixed-point value
// F = round(x 2^(e + 56)) is peeled from the top, BETA bits at a time, each
// digit rounded to nearest (integer arithmetic only); |d_1| <= 2^BETA,
// |d_p| <= 2^(BETA-1) after it, and x 2^e = sum_p d_p 2^(-BETA p) to 2^-57
__device__ __forceinline__ void digits_i(double x, int e, int *out) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  long long F = 0;
  if (ex != 0) {
    const long long mant = (b & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;   // 53 bits
    const int sa = ex - 1075 + e + 56;                                     // F = mant 2^sa
    if (sa >= 0) F = mant << sa;
    else if (sa > -64) F = (mant + (1ll << (-sa - 1))) >> (-sa);
    if (b < 0) F = -F;
  }
#pragma unroll
  for (int p = 1; p <= S; ++p) {
    const int sh = 56 - BETA * p;
    long long dgt;
    if (sh > 0) {
      dgt = (F + (1ll << (sh - 1))) >> sh;
      F -= dgt << sh;
    } else {
      dgt = F;
      F = 0;
    }
    out[p - 1] = (int)dgt;
  }
}
__device__ __forceinline__ void digits(double x, int e, __half *out) {
  int d[S];
  digits_i(x, e, d);
#pragma unroll
  for (int p = 0; p < S; ++p) out[p] = __int2half_rn(d[p]);
}

}  // namespace pw_umma
