// Hermitian products y = A22 v of the blocked Householder reduction (the
// tridiagonalisation inside Syevd, Sec. III-D) on the FP16 tensor cores at
// FP64 accuracy.
//
// Inside a panel of 32 columns the trailing matrix A22 is not updated (the
// panel's rank-2 corrections are applied through V and W), so it is split
// once per panel into integer digit slices and every column's product reads
// the slices instead of the FP64 matrix:
//   * A22 / 2^-eA = sum_p a_p 2^(-7p) (p = 1..8, the digit split of the FP64
//     oz product with one scale for the whole trailing matrix), and
//     v / 2 = sum_q b_q 2^(-7q) (|v| <= 1 for a Householder vector whose head
//     is 1);
//   * the products a_p b_q with p + q = g (g = 2..9) are summed in one FP32
//     tensor-memory accumulator per g: the B operand for slice p holds the
//     digit q = g - p of v in its row for g, so all slices p of a tile
//     accumulate into the same 16 columns (8 groups x real/imaginary part of
//     v); the eight B operands are 16-row windows of one digit array.  Over
//     64 K every partial sum is an integer below 2^22 (exact in FP32);
//   * the epilogue adds the groups into a 64-bit fixed-point sum per output
//     and writes one FP64 partial per tile, summed with the other tiles'
//     partials in FP64 by the row kernel of the reduction.
// The error per output is at most ~K 2^-55 max|A22| (normwise FP64).
//
// Storage: the lower-triangle tiles of 128 x 128 (anchored at row and column
// 0, so every tile starts on a 256-byte boundary) are written per panel in
// the exact byte image of the kernel's shared-memory stage: one 32 KB
// sub-tile per (tile, real/imaginary part, slice), 128-byte swizzled.  A
// sub-tile is one contiguous bulk copy.  Its layout, for tile element
// (r, c) (r = row, c = column, both 0..127):
//   byte = (c / 8) 2048 + (r / 64) 1024 + (c % 8) 128 + swz(r % 64)
// so that the same bytes are the MN-major operand of A v (M = r, K = c:
// 64-row atoms 1 KB apart, 8-column groups 2 KB apart) and the K-major
// operand of A^H v (M = c: 8-row groups 2 KB apart, K = r along the
// swizzled 128-byte rows, the second 64 rows 1 KB further).  Diagonal tiles
// are stored as full Hermitian blocks and give only A v; off-diagonal tiles
// give A v for their rows and A^H v for their columns.
//
// Kernel: persistent, one CTA per SM, each CTA a contiguous range of work
// units (tile, real or imaginary part: eight sub-tiles each).  Warp 0 =
// bulk-copy producer (six 32 KB stages), warp 1 = MMA issuer (one thread),
// warps 2..5 = B-operand builders and epilogue; B operands and accumulators
// are double-buffered, so a unit's MMAs run while the previous unit's sums
// are read and the next unit's digits of v are written.  Every mbarrier wait
// is bounded; on timeout the CTA records an error word and leaves in order.
#include <cuda_fp16.h>

#include <mutex>

#include "dense.cuh"
#include "pw_internal.cuh"
#include "umma.cuh"

namespace {

using namespace pw_umma;

constexpr int HT = 128;                      // tile edge
constexpr int SUB = HT * HT * 2;             // bytes of one slice of one part of a tile (32 KB)
constexpr int UNIT = S * SUB;                // one part of a tile, all slices (256 KB)
constexpr int NST = 6;                       // shared-memory stages
// B operand of one direction: 32 rows x 128 K, no swizzle, K-major: 8-row x
// 16-byte core matrices, rows 16 B apart, the 16 K chunks of 8 elements 512 B
// apart.  Row 2t (Re v) / 2t + 1 (Im v) holds digit t - 6 of v for t = 7..14
// and zeros below, so the 16-row window starting at row 14 - 2p is slice
// p's operand: its row 2j (2j + 1) holds digit j + 1 - p, the partner of
// slice p + 1 in group g = j + 2.
constexpr int BROWS = 32;
constexpr int BKC = BROWS * 16;              // bytes per K chunk (512)
constexpr int BDIR = (HT / 8) * BKC;         // 8 KB
constexpr int OFF_B = NST * SUB;             // [buffer 2][dir 2] B operands
constexpr int OFF_RED = OFF_B + 4 * BDIR;    // block-sum scratch (8 doubles)
constexpr int OFF_BAR = OFF_RED + 64;
constexpr int NBAR = 2 * NST + 5;            // full[], empty[], bready[2], mdone[2], fin
constexpr int SMEM = OFF_BAR + NBAR * 8 + 16 + 1024;
constexpr int NTHR = 192;
constexpr int TMEM_COLS = 128;               // per buffer: D_row[h], D_col[h] (two 64-K halves), 16 columns each
constexpr int LFIX = 54;                     // binary point of the per-tile fixed-point sums
constexpr int DOT_LD = 64;                   // partial dots per k_pcol block (2 x 32 panel columns)
static_assert(SMEM <= 232448, "shared memory per CTA");

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// lower-triangle tile (I, J) of the trailing tiles from the triangular index t
__device__ __forceinline__ void tri_decode(int t, int &I, int &J) {
  int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}
__device__ __forceinline__ long tile_index(int I, int J) { return (long)I * (I + 1) / 2 + J; }

// work unit u: trailing tile (I, J) (relative to the first trailing tile),
// real (0) or imaginary (1) part of its slices, and the slices p0..p1-1
// (piece of ks equal shares); its partial sums go to slot
// (2 tile + part) ks + piece of the row (A v) or column (A^H v) outputs
struct Unit {
  int I, J, part, piece, p0, p1;
};
__device__ __forceinline__ Unit unit_of(long u, int ks) {
  Unit w;
  w.piece = (int)(u % ks);
  const long r = u / ks;
  w.part = (int)(r & 1);
  tri_decode((int)(r >> 1), w.I, w.J);
  w.p0 = w.piece * (S / ks);
  w.p1 = w.p0 + S / ks;
  return w;
}

// byte offset of tile element (r, c) (r in a group of 8 rows r8 = r / 8)
__device__ __forceinline__ uint32_t sub_off(int r8, int c) {
  const int cin = c & 7;
  return (uint32_t)((c >> 3) * 2048 + (r8 >> 3) * 1024 + cin * 128 + (((r8 & 7) ^ cin) << 4));
}

// ------------------------------------------------------------ slicing ----
// largest |Re|, |Im| over the lower triangle of rows and columns >= j0, as
// ordered bits (atomicMax into *slot, cleared before)
__global__ void __launch_bounds__(256) k_hs_max(const double2 *__restrict__ A, int n, int j0,
                                                unsigned long long *slot) {
  __shared__ unsigned long long sh[8];
  const int c = j0 + blockIdx.x;
  unsigned long long mb = 0;
  for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
    const double2 v = A[r + (long)c * n];
    mb = max(mb, max(abs_bits(v.x), abs_bits(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mb = max(mb, sh[w]);
    atomicMax(slot, mb);
  }
}

// digit slices of the trailing tiles (I >= J >= J0): block = (tile, 16
// columns), thread = (column, 8 consecutive rows); entries outside rows and
// columns [j0, n) are zero, the strict upper part of a diagonal tile is the
// conjugate of its lower part
__global__ void __launch_bounds__(256) k_hs_slice(const double2 *__restrict__ A, int n, int j0, int J0,
                                                  const unsigned long long *__restrict__ slot,
                                                  unsigned char *__restrict__ hsl) {
  int I, J;
  tri_decode(blockIdx.x >> 3, I, J);
  I += J0;
  J += J0;
  const int e = row_exp(*slot);
  const int cl = (blockIdx.x & 7) * 16 + (threadIdx.x >> 4), r8 = threadIdx.x & 15;
  const int c = J * HT + cl;
  uint32_t wr[S][4], wi[S][4];
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    int dr[2][S], di[2][S];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = I * HT + r8 * 8 + k + h;
      double2 z = make_double2(0.0, 0.0);
      if (r < n && c < n && r >= j0 && c >= j0) {
        if (r >= c) z = A[r + (long)c * n];
        else {
          z = A[c + (long)r * n];
          z.y = -z.y;
        }
      }
      digits_i(z.x, e, dr[h]);
      digits_i(z.y, e, di[h]);
    }
#pragma unroll
    for (int p = 0; p < S; ++p) {
      wr[p][k >> 1] = (uint32_t)__half_as_ushort(__int2half_rn(dr[0][p])) |
                      ((uint32_t)__half_as_ushort(__int2half_rn(dr[1][p])) << 16);
      wi[p][k >> 1] = (uint32_t)__half_as_ushort(__int2half_rn(di[0][p])) |
                      ((uint32_t)__half_as_ushort(__int2half_rn(di[1][p])) << 16);
    }
  }
  const uint32_t off = sub_off(r8, cl);
  unsigned char *base = hsl + (size_t)tile_index(I, J) * 2 * UNIT + off;
#pragma unroll
  for (int p = 0; p < S; ++p) {
    *(uint4 *)(base + (size_t)p * SUB) = make_uint4(wr[p][0], wr[p][1], wr[p][2], wr[p][3]);
    *(uint4 *)(base + UNIT + (size_t)p * SUB) = make_uint4(wi[p][0], wi[p][1], wi[p][2], wi[p][3]);
  }
}

// --------------------------------------------------------- the product ----
struct HsArgs {
  const double2 *A;            // the matrix being reduced (column c holds x after k_pcol)
  int n, c, i, b;              // order, column, its index in the panel, panel width
  double2 *P;                  // panel [V | W | V] (ld n)
  const unsigned char *hsl;    // slices of the panel's trailing tiles
  const unsigned long long *slot;   // max bits of the trailing matrix (its scale)
  const double2 *dotp;         // k_pcol's partial dots, DOT_LD per block
  int ndotblk;
  double2 *ucorr;              // W^H v, V^H v per panel column
  const double2 *hscal;        // reflector scale s (v = x s below the unit head)
  double2 *part;               // tile partials [slot][nmax]
  int nmax;
  int J0, ntp, ks, units;      // first trailing tile, trailing tiles per side, pieces per (tile, part), units
  int *err;
};

__device__ __forceinline__ double2 refl_v(const double2 *xcol, int x, int m, double2 s) {
  if (x < 0 || x >= m) return make_double2(0.0, 0.0);
  return x == 0 ? make_double2(1.0, 0.0) : cmul(xcol[x], s);
}

// sum over the 128 epilogue threads (named barrier 1), result in every thread
__device__ double epi_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  epi_sync();
  if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) - 2] = v;
  epi_sync();
  return (red[0] + red[1]) + (red[2] + red[3]);
}

__global__ void __launch_bounds__(NTHR, 1) k_hemv_tc(const __grid_constant__ HsArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + OFF_BAR);
  uint64_t *empty = full + NST;
  uint64_t *bready = empty + NST;    // [2] B operands of a unit built, its accumulators free
  uint64_t *mdone = bready + 2;      // [2] a unit's MMAs complete
  uint64_t *fin = mdone + 2;
  uint32_t *tmem_slot = (uint32_t *)(fin + 1);
  double *red = (double *)(smem + OFF_RED);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long ub = (long)blockIdx.x * a.units / gridDim.x, ue = (long)(blockIdx.x + 1) * a.units / gridDim.x;
  const int nunit = (int)(ue - ub);
  const int o = a.c + 1, m = a.n - o;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&bready[b], 128); mbar_init(&mdone[b], 1); }
    mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero rows of the B operands (never rewritten)
  for (int w = threadIdx.x; w < 4 * BDIR / 16; w += NTHR) ((uint4 *)(smem + OFF_B))[w] = make_uint4(0u, 0u, 0u, 0u);
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
      // ------------- producer: the slices were written before the panel's
      // first column, two or more launches back, so no dependency wait
      int k = 0;
      uint32_t issued = 0, last_ph = 0;   // per stage: a copy issued, parity of its last phase
      bool ok = true;
      for (int u = 0; u < nunit && ok; ++u) {
        const Unit w = unit_of(ub + u, a.ks);
        const unsigned char *src =
            a.hsl + ((size_t)tile_index(w.I + a.J0, w.J + a.J0) * 2 + w.part) * UNIT;
        for (int p = w.p0; p < w.p1; ++p, ++k) {
          const int s = k % NST;
          const uint32_t ph = (uint32_t)(k / NST) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1)) { atomicOr(a.err, 1); ok = false; break; }
          mbar_expect_tx(&full[s], SUB);
          bulk_load(smem + s * SUB, src + (size_t)p * SUB, SUB, &full[s]);
          issued |= 1u << s;
          last_ph = (last_ph & ~(1u << s)) | (ph << s);
        }
      }
      // leave no copy in flight
      for (int s = 0; s < NST; ++s)
        if (((issued >> s) & 1) && !mbar_wait(&full[s], (last_ph >> s) & 1)) atomicOr(a.err, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------- MMA issuer
      const uint32_t id_mn = idesc_f16(128, 16, true), id_k = idesc_f16(128, 16, false);
      // stage 0's A operand: MN-major (64-row atoms 1 KB apart, 8-column
      // groups 2 KB apart) and K-major (8-row groups 2 KB apart)
      const uint64_t dmn0 = smem_desc(smem_u32(smem), 1024, 2048, 2), dk0 = smem_desc(smem_u32(smem), 16, 2048, 2);
      int k = 0;
      bool ok = true;
      for (int u = 0; u < nunit && ok; ++u) {
        const Unit w = unit_of(ub + u, a.ks);
        const bool diag = w.I == w.J;
        const int bf = u & 1;
        if (!mbar_wait(&bready[bf], (uint32_t)(u >> 1) & 1)) { atomicOr(a.err, 2); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // descriptors are formed once; the K steps, slices and stages only
        // move their start address (16-byte units in the low 14 bits, which
        // cover all of shared memory, so the additions never carry out)
        const uint64_t db0 = smem_desc(smem_u32(smem + OFF_B + (2 * bf) * BDIR), BKC, 128, 0);
        const uint64_t db1 = db0 + (BDIR >> 4);
        const uint32_t d0 = tmem + (uint32_t)(bf * 64);
        for (int p = w.p0; p < w.p1; ++p, ++k) {
          const int s = k % NST;
          if (!mbar_wait(&full[s], (uint32_t)(k / NST) & 1)) { atomicOr(a.err, 2); ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da_mn = dmn0 + (uint64_t)(s * (SUB >> 4)), da_k = dk0 + (uint64_t)(s * (SUB >> 4));
          const uint64_t win = (uint64_t)(14 - 2 * p);          // slice p's 16-row window of B
#pragma unroll
          for (int kk = 0; kk < HT / 16; ++kk) {
            const int h = kk >> 2;
            const uint32_t acc = (p == w.p0 && (kk & 3) == 0) ? 0u : 1u;
            const uint64_t bo = (uint64_t)(kk * (2 * BKC >> 4)) + win;
            // A v: M = tile rows, K = tile columns (MN-major A)
            mma_f16(d0 + (uint32_t)(h * 16), da_mn + (uint64_t)(kk * (4096 >> 4)), db0 + bo, id_mn, acc);
            // A^H v: M = tile columns, K = tile rows (K-major A)
            if (!diag)
              mma_f16(d0 + (uint32_t)(32 + h * 16), da_k + (uint64_t)(h * (1024 >> 4) + (kk & 3) * 2), db1 + bo,
                      id_k, acc);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&mdone[bf]);
      }
      // every MMA of this CTA complete before the teardown
      mma_commit(fin);
      if (!mbar_wait(fin, 0)) atomicOr(a.err, 2);
    }
  } else {
    // ------------- warps 2..5: B operands, epilogue, side work
    const int et = threadIdx.x - 64;            // 0..127: K entry of the B operands
    const int q4 = warp & 3;                    // tensor-memory lane quarter
    const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
    pdl_wait();
    pdl_trigger();
    const double2 scal = *a.hscal;
    const int eA = row_exp(*a.slot);
    const double2 *xk = a.A + o + (long)a.c * a.n;   // x of column c, x[0] at row o
    const int ksc = -LFIX - eA + 1;             // value = acc 2^ksc (digits of v / 2)
    // digits of v over the unit's tile columns (dir 0, A v) and rows (dir 1,
    // A^H v) into buffer u & 1: rows 14..29 of the window layout
    auto build = [&](int u) {
      const Unit w = unit_of(ub + u, a.ks);
      const int ndir = w.I == w.J ? 1 : 2;
      const int I = w.I + a.J0, J = w.J + a.J0;
      for (int dir = 0; dir < ndir; ++dir) {
        const double2 v = refl_v(xk, (dir == 0 ? J : I) * HT + et - o, m, scal);
        int dr[S], di[S];
        digits_i(v.x, -1, dr);
        digits_i(v.y, -1, di);
        __half *col = (__half *)(smem + OFF_B + (2 * (u & 1) + dir) * BDIR + (et >> 3) * BKC) + (et & 7);
#pragma unroll
        for (int t = 0; t < S; ++t) {
          col[(2 * (t + 7)) * 8] = __int2half_rn(dr[t]);
          col[(2 * (t + 7) + 1) * 8] = __int2half_rn(di[t]);
        }
      }
      // the B operands (generic-proxy writes) to the tensor core, and the
      // buffer's accumulators free
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&bready[u & 1]);
    };
    auto epilogue = [&](int u) -> bool {
      if (!mbar_wait(&mdone[u & 1], (uint32_t)(u >> 1) & 1)) { atomicOr(a.err, 4); return false; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const Unit w = unit_of(ub + u, a.ks);
      const int part = w.part;
      const int I = w.I + a.J0, J = w.J + a.J0;
      uint32_t r[32];
#pragma unroll
      for (int dir = 0; dir < 2; ++dir) {
        if (dir == 1 && I == J) break;
        tmem_ld32(tmem + lanes + (uint32_t)((u & 1) * 64 + dir * 32), r);
        long long R = 0, Q = 0;                   // Re v part, Im v part
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int sh = LFIX - BETA * (j + 2);
            R += shifted(f2i_exact(r[h * 16 + 2 * j]), sh);
            Q += shifted(f2i_exact(r[h * 16 + 2 * j + 1]), sh);
          }
        // A = Ar + i Ai, v = vr + i vi; rows (dir 0): Ar v -> (R, Q), i Ai v -> (-Q, R);
        // columns (dir 1, conj(A)^T v): Ar -> (R, Q), -i Ai -> (Q, -R)
        long long yr, yi;
        if (part == 0) { yr = R; yi = Q; }
        else if (dir == 0) { yr = -Q; yi = R; }
        else { yr = Q; yi = -R; }
        const int x = (dir == 0 ? I : J) * HT + q4 * 32 + lane;
        const int sl = (2 * (dir == 0 ? w.J : w.I) + part) * a.ks + w.piece;
        if (x >= o && x < a.n)
          a.part[(long)sl * a.nmax + x] = make_double2(scale_pow2((double)yr, ksc), scale_pow2((double)yi, ksc));
      }
      return true;
    };
    if (nunit > 0) build(0);
    if (nunit > 1) build(1);
    // v into V[:, i] and its copy (a share of the rows per CTA)
    {
      const int per = (m + gridDim.x - 1) / gridDim.x;
      const int x0 = blockIdx.x * per, x1 = min(m, x0 + per);
      for (int x = x0 + et; x < x1; x += 128) {
        const double2 v = refl_v(xk, x, m, scal);
        a.P[o + x + (long)a.i * a.n] = v;
        a.P[o + x + (long)(2 * a.b + a.i) * a.n] = v;
      }
    }
    // ucorr[d] = col^H v with col = W[:, q] (d = 2q) or V[:, q] (d = 2q + 1):
    // s times k_pcol's partial dots over the rows below the head, plus the head
    for (int d = blockIdx.x; d < 2 * a.i; d += gridDim.x) {
      double sr = 0.0, si = 0.0;
      for (int t = et; t < a.ndotblk; t += 128) {
        const double2 v = a.dotp[(long)t * DOT_LD + d];
        sr += v.x;
        si += v.y;
      }
      sr = epi_sum(sr, red);
      si = epi_sum(si, red);
      if (et == 0) {
        const int q = d >> 1;
        const double2 hv = a.P[o + (long)((d & 1) ? q : a.b + q) * a.n];
        const double2 u = cmul(scal, make_double2(sr, si));
        a.ucorr[d] = make_double2(u.x + hv.x, u.y - hv.y);
      }
    }
    // unit u's accumulators are read before the B operands of unit u + 2
    // replace its buffer
    bool ok = true;
    for (int u = 0; u < nunit && ok; ++u) {
      ok = epilogue(u);
      if (ok && u + 2 < nunit) build(u + 2);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

int sm_count() {
  static std::mutex mu;
  static int cnt[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (!cnt[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cnt[dev] = v > 0 ? v : 148;
  }
  return cnt[dev];
}

pw_status allow_smem() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return PW_ERR_ARG;
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    PW_CUDA(cudaFuncSetAttribute(k_hemv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    done[dev] = true;
  }
  return PW_OK;
}

}  // namespace

size_t pw_hs_bytes(int nmax) {
  if (nmax < PW_HS_MIN_ORDER) return 0;
  const size_t nt = (size_t)(nmax + HT - 1) / HT;
  return nt * (nt + 1) / 2 * 2 * (size_t)UNIT;
}

pw_status pw_hs_slice(pw_dense_ws *ws, const double2 *A, int n, int j0, cudaStream_t st) {
  unsigned long long *slot = ws->hsmax + j0 / 32;
  pw_count_launch();
  k_hs_max<<<n - j0, 256, 0, st>>>(A, n, j0, slot);
  const int J0 = j0 / HT, ntp = (n + HT - 1) / HT - J0;
  pw_count_launch();
  k_hs_slice<<<ntp * (ntp + 1) / 2 * 8, 256, 0, st>>>(A, n, j0, J0, slot, (unsigned char *)ws->hsl);
  return pw_check_launch("householder slices");
}

pw_status pw_hs_hemv(pw_dense_ws *ws, const double2 *A, int n, int c, int i, int b, int j0, int ndotblk,
                     int *nslots, cudaStream_t st) {
  PW_TRY(allow_smem());
  HsArgs a;
  a.A = A;
  a.n = n;
  a.c = c;
  a.i = i;
  a.b = b;
  a.P = ws->panel;
  a.hsl = (const unsigned char *)ws->hsl;
  a.slot = ws->hsmax + j0 / 32;
  a.dotp = ws->dotp;
  a.ndotblk = ndotblk;
  a.ucorr = ws->ucorr;
  a.hscal = ws->hscal;
  a.part = ws->part;
  a.nmax = ws->nmax;
  a.J0 = (c + 1) / HT;
  a.ntp = (n + HT - 1) / HT - a.J0;
  // pieces per (tile, part): enough units for every SM, within the partial
  // slots ws->part holds ((nmax + 31) / 32)
  const int sms = sm_count(), tiles2 = a.ntp * (a.ntp + 1), slots = (ws->nmax + 31) / 32;
  a.ks = 1;
  while (a.ks < S && tiles2 * a.ks < sms && 2 * a.ntp * a.ks * 2 <= slots) a.ks *= 2;
  a.units = tiles2 * a.ks;
  a.err = ws->oz.err;
  *nslots = 2 * a.ntp * a.ks;
  const int grid = std::min(a.units, sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  pw_count_launch();
  PW_CUDA(cudaLaunchKernelEx(&cfg, k_hemv_tc, a));
  return PW_OK;
}
