// Hermitian products y = A22 v of the blocked Householder reduction (the
// tridiagonalisation inside Syevd, Sec. III-D) on the FP16 tensor cores at
// FP64 accuracy.
//
// Inside a panel of 32 columns the trailing matrix A22 is not updated (the
// panel's rank-2 corrections are applied through V and W), so it is split
// once per panel into integer digit slices and every column's product reads
// the slices instead of the FP64 matrix:
//   * A22 2^eA = sum_p a_p 2^(-7p) (p = 1..8, the digit split of the
//     FP64-accurate product, one scale for the whole trailing matrix), and
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
// The error per output is at most 10 K 2^-55 max|A22| for trailing order K
// (2K real terms, each off by at most 1.25 2^-55 in scaled units: the
// digit roundings and the dropped pairs; the scales add a factor of 4):
// normwise FP64.
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
// Kernel (k_hemv_tc, one column per launch, chained with k_pcol and k_prows
// by programmatic dependent launch): persistent, one CTA per SM, each CTA a
// contiguous range of work units (tile, real or imaginary part, and for
// short trailing orders a piece of its eight slices, so that every SM has
// work).  Warp 0 = bulk-copy producer (six 32 KB stages), warp 1 = MMA
// issuer (one thread), warps 2..5 = B-operand builders and epilogue, warps
// 6..7 = v into the panel and the panel's correction dots; B operands and
// accumulators are double-buffered, so a unit's MMAs run while the previous
// unit's sums are read and the next unit's digits of v are written.  The
// same roles run inside k_panel_tc, one cooperative launch per panel.
// Every mbarrier wait is bounded; on timeout the CTA records an error word
// and leaves in order.
#include <cuda_fp16.h>

#include <mutex>

#include <cooperative_groups.h>

#include "dense.cuh"
#include "house.cuh"
#include "pw_internal.cuh"
#include "umma.cuh"

namespace {

using namespace pw_umma;

constexpr int HT = 128;                      // tile edge
constexpr int SUB = HT * HT * 2;             // bytes of one slice of one part of a tile (32 KB)
constexpr int UNIT = S * SUB;                // one part of a tile, all slices (256 KB)
// B operand of one direction: 32 rows x 128 K, no swizzle, K-major: 8-row x
// 16-byte core matrices, rows 16 B apart, the 16 K chunks of 8 elements 512 B
// apart.  Row 2t (Re v) / 2t + 1 (Im v) holds digit t - 6 of v for t = 7..14
// and zeros below, so the 16-row window starting at row 14 - 2p is slice
// p's operand: its row 2j (2j + 1) holds digit j + 1 - p, the partner of
// slice p + 1 in group g = j + 2.
constexpr int BROWS = 32;
constexpr int BKC = BROWS * 16;              // bytes per K chunk (512)
constexpr int BDIR = (HT / 8) * BKC;         // 8 KB
constexpr int TMEM_COLS = 128;               // per buffer: D_row[h], D_col[h] (two 64-K halves), 16 columns each
constexpr int LFIX = 54;                     // binary point of the per-tile fixed-point sums
constexpr int TPB_HS = 32;                   // panel width of the reduction
constexpr int NBAR_FIXED = 5;                // bready[2], mdone[2], fin
// dynamic shared memory of a CTA running the product with NS stages of one
// sub-tile: stages, [buffer 2][dir 2] B operands, block-sum scratch, barriers
template <int NS>
struct HsL {
  static constexpr int OFF_B = NS * SUB;
  static constexpr int OFF_RED = OFF_B + 4 * BDIR;
  static constexpr int OFF_BAR = OFF_RED + 64;
  static constexpr int SMEM = OFF_BAR + (2 * NS + NBAR_FIXED) * 8 + 16 + 1024;
};
constexpr int NST_HEMV = 6;                  // one column per launch
constexpr int NST_PANEL = 5;                 // cooperative panel (its column phases need static scratch)
constexpr int NTHR = 256;                    // producer, MMA, 4 epilogue warps, 2 side warps
constexpr int NTHR_PANEL = 256;
static_assert(HsL<NST_HEMV>::SMEM <= 232448, "shared memory per CTA");
static_assert(HsL<NST_PANEL>::SMEM + 8 * 1024 <= 232448, "shared memory per CTA");

__device__ __forceinline__ void named_sync(int id, int nthr) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
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
// Shared-memory view of a CTA running the product with NS stages.
template <int NS>
struct HsSmem {
  unsigned char *base;
  uint64_t *full, *empty;      // [NS] stage filled / stage read by the MMAs
  uint64_t *bready, *mdone;    // [2] a unit's B operands built (and its accumulators free) / its MMAs done
  uint64_t *fin;
  uint32_t *tmem_slot;
  double *red;                 // block-sum scratch
  __device__ explicit HsSmem(unsigned char *smem) {
    base = smem;
    full = (uint64_t *)(smem + HsL<NS>::OFF_BAR);
    empty = full + NS;
    bready = empty + NS;
    mdone = bready + 2;
    fin = mdone + 2;
    tmem_slot = (uint32_t *)(fin + 1);
    red = (double *)(smem + HsL<NS>::OFF_RED);
  }
};

// barriers, the B operands' zero rows (never rewritten) and the tensor
// memory (warp 0); the caller synchronises the block afterwards
template <int NS>
__device__ void hs_setup(const HsSmem<NS> &m) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&m.full[s], 1); mbar_init(&m.empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&m.bready[b], 128); mbar_init(&m.mdone[b], 1); }
    mbar_init(m.fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int w = threadIdx.x; w < 4 * BDIR / 16; w += blockDim.x)
    ((uint4 *)(m.base + HsL<NS>::OFF_B))[w] = make_uint4(0u, 0u, 0u, 0u);
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(m.tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
}

// one CTA's share of one column's product
struct HsCol {
  const double2 *A;            // column c holds x (rows c + 1..)
  int n, c;
  long ub;                     // first unit of this CTA
  int nunit;                   // its units
  int J0, ks;                  // first trailing tile, pieces per (tile, part)
  const unsigned char *hsl;    // slices of the panel's trailing tiles
  double2 *part;               // tile partials [slot][nmax], global row index
  int nmax;
  int *err;
};
__device__ __forceinline__ int hs_subtiles(const HsCol &w) { return w.nunit * (S / w.ks); }

// the column's units of a CTA: `units` spread over the grid in contiguous ranges
__device__ __forceinline__ void hs_range(int units, long &ub, int &nunit) {
  ub = (long)blockIdx.x * units / gridDim.x;
  nunit = (int)((long)(blockIdx.x + 1) * units / gridDim.x - ub);
}

// pieces per (tile, part): enough units for the grid, within the slots of
// the partial sums; the host's count of slots uses the same rule
__host__ __device__ __forceinline__ int hs_pieces(int ntp, int grid, int slots) {
  int ks = 1;
  while (ks < S && ntp * (ntp + 1) * ks < grid && 2 * ntp * ks * 2 <= slots) ks *= 2;
  return ks;
}

// an error word another role of the CTA (or another CTA) may have set
__device__ __forceinline__ bool hs_failed(const int *err) { return *(const volatile int *)err != 0; }

// producer: sub-tiles [pos, end) of the CTA's sequence for the column; k
// counts every sub-tile the CTA has issued (stage k % NS, phase k / NS)
template <int NS>
__device__ bool hs_produce(const HsCol &w, const HsSmem<NS> &m, int pos, int end, int &k, uint32_t &issued,
                           uint32_t &last_ph) {
  const int spu = S / w.ks;
  for (; pos < end; ++pos, ++k) {
    if (pos % spu == 0 && hs_failed(w.err)) return false;
    const Unit u = unit_of(w.ub + pos / spu, w.ks);
    const int p = u.p0 + pos % spu;
    const unsigned char *src =
        w.hsl + ((size_t)tile_index(u.I + w.J0, u.J + w.J0) * 2 + u.part) * UNIT + (size_t)p * SUB;
    const int s = k % NS;
    const uint32_t ph = (uint32_t)(k / NS) & 1;
    if (!mbar_wait(&m.empty[s], ph ^ 1)) { atomicOr(w.err, 1); return false; }
    mbar_expect_tx(&m.full[s], SUB);
    bulk_load(m.base + s * SUB, src, SUB, &m.full[s]);
    issued |= 1u << s;
    last_ph = (last_ph & ~(1u << s)) | (ph << s);
  }
  return true;
}
// before the CTA leaves: every issued copy has landed
template <int NS>
__device__ void hs_produce_drain(const HsSmem<NS> &m, uint32_t issued, uint32_t last_ph, int *err) {
  for (int s = 0; s < NS; ++s)
    if (((issued >> s) & 1) && !mbar_wait(&m.full[s], (last_ph >> s) & 1)) atomicOr(err, 1);
}

// MMA issuer: all units of the column.  k counts the sub-tiles read, ug the
// CTA's units over all columns (B buffer and accumulators ug & 1).  The
// descriptors are formed once; K steps, slices and stages only move their
// start address (16-byte units in the low 14 bits, which cover all of shared
// memory, so the additions never carry out).
template <int NS>
__device__ bool hs_mma(const HsCol &w, const HsSmem<NS> &m, uint32_t tmem, int &k, int &ug) {
  const uint32_t id_mn = idesc_f16(128, 16, true), id_k = idesc_f16(128, 16, false);
  // stage 0's A operand: MN-major (64-row atoms 1 KB apart, 8-column groups
  // 2 KB apart) and K-major (8-row groups 2 KB apart)
  const uint64_t dmn0 = smem_desc(smem_u32(m.base), 1024, 2048, 2), dk0 = smem_desc(smem_u32(m.base), 16, 2048, 2);
  for (int u = 0; u < w.nunit; ++u, ++ug) {
    if (hs_failed(w.err)) return false;
    const Unit un = unit_of(w.ub + u, w.ks);
    const bool diag = un.I == un.J;
    const int bf = ug & 1;
    if (!mbar_wait(&m.bready[bf], (uint32_t)(ug >> 1) & 1)) { atomicOr(w.err, 2); return false; }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint64_t db0 = smem_desc(smem_u32(m.base + HsL<NS>::OFF_B + (2 * bf) * BDIR), BKC, 128, 0);
    const uint64_t db1 = db0 + (BDIR >> 4);
    const uint32_t d0 = tmem + (uint32_t)(bf * 64);
    for (int p = un.p0; p < un.p1; ++p, ++k) {
      const int s = k % NS;
      if (!mbar_wait(&m.full[s], (uint32_t)(k / NS) & 1)) { atomicOr(w.err, 2); return false; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da_mn = dmn0 + (uint64_t)(s * (SUB >> 4)), da_k = dk0 + (uint64_t)(s * (SUB >> 4));
      const uint64_t win = (uint64_t)(14 - 2 * p);          // slice p's 16-row window of B
#pragma unroll
      for (int kk = 0; kk < HT / 16; ++kk) {
        const int h = kk >> 2;
        const uint32_t acc = (p == un.p0 && (kk & 3) == 0) ? 0u : 1u;
        const uint64_t bo = (uint64_t)(kk * (2 * BKC >> 4)) + win;
        // A v: M = tile rows, K = tile columns (MN-major A)
        mma_f16(d0 + (uint32_t)(h * 16), da_mn + (uint64_t)(kk * (4096 >> 4)), db0 + bo, id_mn, acc);
        // A^H v: M = tile columns, K = tile rows (K-major A)
        if (!diag)
          mma_f16(d0 + (uint32_t)(32 + h * 16), da_k + (uint64_t)(h * (1024 >> 4) + (kk & 3) * 2), db1 + bo,
                  id_k, acc);
      }
      mma_commit(&m.empty[s]);
    }
    mma_commit(&m.mdone[bf]);
  }
  return true;
}
// every MMA of the CTA complete before the teardown
template <int NS>
__device__ void hs_mma_finish(const HsSmem<NS> &m, int *err) {
  mma_commit(m.fin);
  if (!mbar_wait(m.fin, 0)) atomicOr(err, 2);
}

// entry x of v = x s below its unit head (zero outside 0..m-1); x may have
// been written by another CTA of the same cooperative launch
__device__ __forceinline__ double2 refl_v(const double2 *xcol, int x, int m, double2 s) {
  if (x < 0 || x >= m) return make_double2(0.0, 0.0);
  return x == 0 ? make_double2(1.0, 0.0) : cmul(__ldcg(&xcol[x]), s);
}

// Warps 2..5 (et = threadIdx.x - 64, the K entry of the B operands):
// digits of v over unit u's tile columns (dir 0, A v) and rows (dir 1, A^H v)
// into buffer ug & 1, rows 14..29 of the window layout
template <int NS>
__device__ void hs_build(const HsCol &w, const HsSmem<NS> &m, int u, int ug, double2 scal) {
  const int et = threadIdx.x - 64;
  const int o = w.c + 1, mm = w.n - o;
  const double2 *xk = w.A + o + (long)w.c * w.n;
  const Unit un = unit_of(w.ub + u, w.ks);
  const int ndir = un.I == un.J ? 1 : 2;
  const int I = un.I + w.J0, J = un.J + w.J0;
  for (int dir = 0; dir < ndir; ++dir) {
    const double2 v = refl_v(xk, (dir == 0 ? J : I) * HT + et - o, mm, scal);
    int dr[S], di[S];
    digits_i(v.x, -1, dr);
    digits_i(v.y, -1, di);
    __half *col = (__half *)(m.base + HsL<NS>::OFF_B + (2 * (ug & 1) + dir) * BDIR + (et >> 3) * BKC) + (et & 7);
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
  mbar_arrive(&m.bready[ug & 1]);
}

// warps 2..5: unit u's sums (buffer ug & 1) into the partial slots
template <int NS>
__device__ bool hs_epilogue(const HsCol &w, const HsSmem<NS> &m, uint32_t tmem, int u, int ug, int eA) {
  if (!mbar_wait(&m.mdone[ug & 1], (uint32_t)(ug >> 1) & 1)) { atomicOr(w.err, 4); return false; }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int q4 = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;   // tensor-memory lane quarter
  const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
  const int o = w.c + 1;
  const int ksc = -LFIX - eA + 1;               // value = acc 2^ksc (digits of v / 2)
  const Unit un = unit_of(w.ub + u, w.ks);
  const int part = un.part;
  const int I = un.I + w.J0, J = un.J + w.J0;
  uint32_t r[32];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    if (dir == 1 && I == J) break;
    tmem_ld32(tmem + lanes + (uint32_t)((ug & 1) * 64 + dir * 32), r);
    long long R = 0, Q = 0;                     // Re v part, Im v part
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
    const int sl = (2 * (dir == 0 ? un.J : un.I) + part) * w.ks + un.piece;
    if (x >= o && x < w.n)
      w.part[(long)sl * w.nmax + x] = make_double2(scale_pow2((double)yr, ksc), scale_pow2((double)yi, ksc));
  }
  return true;
}

// warps 2..5 over the column: the first two units' B operands, then each
// unit's sums before the B operands of the unit two later replace its buffer
template <int NS>
__device__ void hs_epi_start(const HsCol &w, const HsSmem<NS> &m, double2 scal, int ug) {
  if (w.nunit > 0) hs_build(w, m, 0, ug, scal);
  if (w.nunit > 1) hs_build(w, m, 1, ug + 1, scal);
}
template <int NS>
__device__ void hs_epi_rest(const HsCol &w, const HsSmem<NS> &m, uint32_t tmem, double2 scal, int eA, int &ug) {
  for (int u = 0; u < w.nunit; ++u) {
    if (hs_failed(w.err) || !hs_epilogue(w, m, tmem, u, ug + u, eA)) break;
    if (u + 2 < w.nunit) hs_build(w, m, u + 2, ug + u + 2, scal);
  }
  ug += w.nunit;
}

// sum over nthr threads (tid 0..nthr-1, whole warps) at named barrier id
__device__ double group_sum(double v, double *red, int id, int nthr, int tid) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  named_sync(id, nthr);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  named_sync(id, nthr);
  double r = 0.0;
  for (int q = 0; q < (nthr >> 5); ++q) r += red[q];
  named_sync(id, nthr);
  return r;
}

// v into V[:, i] and its copy (a share of the rows per CTA), and
// ucorr[d] = col^H v with col = W[:, q] (d = 2q) or V[:, q] (d = 2q + 1), one
// CTA per dot, on the FP64 pipe (which the tensor-core product leaves idle)
struct HsSide {
  const double2 *A;
  int n, c, i, b;
  double2 *P;
  double2 *ucorr;
};
__device__ void hs_side(const HsSide &a, double2 scal, double *red, int id, int nthr, int tid) {
  const int o = a.c + 1, m = a.n - o;
  const double2 *xk = a.A + o + (long)a.c * a.n;
  const int per = (m + gridDim.x - 1) / gridDim.x;
  const int x0 = blockIdx.x * per, x1 = min(m, x0 + per);
  for (int x = x0 + tid; x < x1; x += nthr) {
    const double2 v = refl_v(xk, x, m, scal);
    a.P[o + x + (long)a.i * a.n] = v;
    a.P[o + x + (long)(2 * a.b + a.i) * a.n] = v;
  }
  for (int d = blockIdx.x; d < 2 * a.i; d += gridDim.x) {
    const int q = d >> 1;
    const double2 *col = a.P + o + (long)((d & 1) ? q : a.b + q) * a.n;
    double2 sacc = make_double2(0.0, 0.0);
    for (int x = tid; x < m; x += nthr) cmacc(sacc, __ldcg(&col[x]), refl_v(xk, x, m, scal));
    sacc.x = group_sum(sacc.x, red, id, nthr, tid);
    sacc.y = group_sum(sacc.y, red, id, nthr, tid);
    if (tid == 0) a.ucorr[d] = sacc;
  }
}

// ------------------------------------------------ one column per launch ----
struct HsArgs {
  HsSide side;
  const unsigned char *hsl;    // slices of the panel's trailing tiles
  const unsigned long long *slot;   // max bits of the trailing matrix (its scale)
  const double2 *hscal;        // reflector scale s (v = x s below the unit head)
  double2 *part;               // tile partials [slot][nmax]
  int nmax;
  int J0, ks, units;           // first trailing tile, pieces per (tile, part), units
  int *err;
};

__global__ void __launch_bounds__(NTHR, 1) k_hemv_tc(const __grid_constant__ HsArgs a) {
  constexpr int NS = NST_HEMV;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const HsSmem<NS> m((unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  HsCol w;
  w.A = a.side.A;
  w.n = a.side.n;
  w.c = a.side.c;
  hs_range(a.units, w.ub, w.nunit);
  w.J0 = a.J0;
  w.ks = a.ks;
  w.hsl = a.hsl;
  w.part = a.part;
  w.nmax = a.nmax;
  w.err = a.err;

  hs_setup(m);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *m.tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // the slices were written before the panel's first column, two or more
      // launches back, so the producer needs no dependency wait
      int k = 0;
      uint32_t issued = 0, last_ph = 0;
      hs_produce(w, m, 0, hs_subtiles(w), k, issued, last_ph);
      hs_produce_drain(m, issued, last_ph, w.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int k = 0, ug = 0;
      hs_mma(w, m, tmem, k, ug);
      hs_mma_finish(m, w.err);
    }
  } else if (warp < 6) {
    pdl_wait();
    pdl_trigger();
    const double2 scal = *a.hscal;
    const int eA = row_exp(*a.slot);
    int ug = 0;
    hs_epi_start(w, m, scal, ug);
    hs_epi_rest(w, m, tmem, scal, eA, ug);
  } else {
    pdl_wait();
    pdl_trigger();
    hs_side(a.side, *a.hscal, m.red, 1, 64, threadIdx.x - 192);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// --------------------------------------------- one cooperative panel ----
// All the columns of a panel (32 from j0) in one cooperative launch, one CTA
// per SM, the phases of each column separated by grid-wide barriers:
//   A  (all threads) column c receives the panel's earlier rank-2 updates;
//      norm partials of x per 32-row block;
//   -- barrier --
//      reflector scalars (every CTA, from the norm partials); then the
//      tensor-core product (warp 0 copies, warp 1 MMAs, warps 2..5 B
//      operands and sums) while warps 6..7 store v and form the panel's
//      correction dots W^H v, V^H v;
//   -- barrier --
//   C  (all threads) y = partial sums - corrections, p = tau y, v in place
//      of x, partial dots p^H v;
//   -- barrier --
// The first stages of a column's slices are requested during its phase A.
// The same arithmetic as the chained kernels (k_pcol, the product, k_prows)
// up to the order of the column update's sums.
struct PanelArgs {
  double2 *A;
  int n, j0, b;
  double2 *P;                  // panel [V | W | V] (ld n)
  double2 *p, *dotpart;        // p of the previous column, its partial dots p^H v
  double2 *tau;
  double *d, *e, *nrm_part;
  double2 *hscal;
  double2 *ucorr;
  const unsigned char *hsl;
  const unsigned long long *slot;
  double2 *part;
  int nmax, slots;
  int *err;
};

constexpr int CO_Q8 = (TPB_HS + 7) / 8;        // panel columns per warp of an 8-warp row block

__global__ void __launch_bounds__(NTHR_PANEL, 1) k_panel_tc(const __grid_constant__ PanelArgs a) {
  constexpr int NS = NST_PANEL;
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const HsSmem<NS> m((unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023));
  __shared__ double sh[32];
  __shared__ double2 s_vc[TPB_HS], s_wc[TPB_HS], s_u[8][33];
  const int n = a.n, b = a.b, nblk = gridDim.x;
  double2 *V = a.P, *W = a.P + (long)b * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, rl = lane, g = warp;

  hs_setup(m);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *m.tmem_slot;

  const int eA = row_exp(*a.slot);
  const int nT = (n + HT - 1) / HT;
  int kprod = 0, kmma = 0, ug_mma = 0, ug_epi = 0, pos0 = 0;
  uint32_t issued = 0, last_ph = 0;
  int ndot = 0;
  double2 tk = make_double2(0.0, 0.0), scal = make_double2(0.0, 0.0);
  for (int i = 0; i < b; ++i) {
    const int c = a.j0 + i, o = c + 1, mrow = n - o;
    HsCol w;
    w.A = a.A;
    w.n = n;
    w.c = c;
    w.J0 = o / HT;
    const int ntp = nT - w.J0;
    w.ks = hs_pieces(ntp, nblk, a.slots);
    hs_range(ntp * (ntp + 1) * w.ks, w.ub, w.nunit);
    w.hsl = a.hsl;
    w.part = a.part;
    w.nmax = a.nmax;
    w.err = a.err;
    const int nslots = 2 * ntp * w.ks;
    // the first stages of this column's slices, while phase A runs
    if (warp == 0 && lane == 0) {
      pos0 = min(NS, hs_subtiles(w));
      hs_produce(w, m, 0, pos0, kprod, issued, last_ph);
    }
    // ---- phase A: column c receives the panel's earlier rank-2 updates.
    // Two 32-row blocks per pass, four warps each, in k_pcol's order.
    double2 al = make_double2(0.0, 0.0);
    if (i > 0) {
      al = panel_alpha(a.dotpart, ndot, tk, sh, 128);   // tk: tau of column c - 1
      if (threadIdx.x < i) {
        const int q = threadIdx.x;
        s_vc[q] = __ldcg(&V[c + (long)q * n]);
        if (q < i - 1) s_wc[q] = __ldcg(&W[c + (long)q * n]);
      }
      if (threadIdx.x == 0) s_wc[i - 1] = cadd(__ldcg(&a.p[0]), al);
    }
    __syncthreads();
    // one 32-row block per CTA and pass, the eight warps splitting the
    // panel's columns (q = warp mod 8)
    const int nrb = (n - c + 31) / 32;
    for (int rb = blockIdx.x; rb < nrb; rb += nblk) {
      const int r = c + rb * 32 + rl;
      double2 u = make_double2(0.0, 0.0);
      if (i > 0 && r < n) {
#pragma unroll
        for (int t = 0; t < CO_Q8; ++t) {
          const int q = g + 8 * t;
          if (q >= i) break;
          const double2 vq = __ldcg(&V[r + (long)q * n]);
          double2 wq;
          if (q == i - 1) {
            wq = __ldcg(&a.p[r - c]);
            cmac(wq, al, vq);
            W[r + (long)q * n] = wq;
          } else {
            wq = __ldcg(&W[r + (long)q * n]);
          }
          cmacc(u, s_wc[q], vq);
          cmacc(u, s_vc[q], wq);
        }
      }
      s_u[g][rl] = u;
      __syncthreads();
      if (g == 0) {
        double nrm = 0.0;
        if (r < n) {
          double2 av = __ldcg(&a.A[r + (long)c * n]);
          if (i > 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) av = csub(av, s_u[q][rl]);
            a.A[r + (long)c * n] = av;
          }
          if (r > c + 1) nrm = av.x * av.x + av.y * av.y;
        }
        nrm = warp_sum(nrm);
        if (rl == 0) a.nrm_part[rb] = nrm;
      }
      __syncthreads();
    }
    grid.sync();
    // reflector scalars from x = A[c+1:, c] (every block, in the order of
    // k_pcol's last block)
    {
      const double2 alpha = __ldcg(&a.A[(c + 1) + (long)c * n]);
      if (g == 0) {
        double xn2 = 0.0;
        for (int q = rl; q < nrb; q += 32) xn2 += __ldcg(&a.nrm_part[q]);
        xn2 = warp_sum(xn2);
        if (rl == 0) sh[0] = xn2;
      }
      __syncthreads();
      const double xn2 = sh[0];
      __syncthreads();
      double beta;
      reflector_scalars(xn2, alpha, beta, tk, scal);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.d[c] = __ldcg(&a.A[c + (long)c * n]).x;
        a.tau[c] = tk;
        a.e[c] = beta;
        *a.hscal = scal;
      }
    }
    // ---- phase B: the tensor-core product, v into the panel, the dots
    if (warp == 0) {
      if (lane == 0) hs_produce(w, m, pos0, hs_subtiles(w), kprod, issued, last_ph);
    } else if (warp == 1) {
      if (lane == 0) hs_mma(w, m, tmem, kmma, ug_mma);
    } else if (warp < 6) {
      hs_epi_start(w, m, scal, ug_epi);
      hs_epi_rest(w, m, tmem, scal, eA, ug_epi);
    } else {
      HsSide sd;
      sd.A = a.A;
      sd.n = n;
      sd.c = c;
      sd.i = i;
      sd.b = b;
      sd.P = a.P;
      sd.ucorr = a.ucorr;
      hs_side(sd, scal, m.red, 2, 64, threadIdx.x - 192);
    }
    grid.sync();
    // ---- phase C: y = partial sums - V (W^H v) - W (V^H v), p = tau y, v in
    // place of x, partial dots p^H v
    ndot = (mrow + 31) / 32;
    double2 *xc = a.A + o + (long)c * n;
    for (int rb = blockIdx.x; rb < ndot; rb += nblk) {
      const int x = rb * 32 + rl;
      double2 y = make_double2(0.0, 0.0);
      if (x < mrow) {
        for (int q = g; q < nslots; q += 8) y = cadd(y, __ldcg(&a.part[(long)q * a.nmax + o + x]));
#pragma unroll
        for (int t = 0; t < CO_Q8; ++t) {
          const int q = g + 8 * t;
          if (q >= i) break;
          const double2 uw = __ldcg(&a.ucorr[2 * q]), uv = __ldcg(&a.ucorr[2 * q + 1]);
          cmac(y, __ldcg(&a.P[o + x + (long)q * n]), make_double2(-uw.x, -uw.y));         // - V[r,q] (W^H v)_q
          cmac(y, __ldcg(&a.P[o + x + (long)(b + q) * n]), make_double2(-uv.x, -uv.y));   // - W[r,q] (V^H v)_q
        }
      }
      s_u[g][rl] = y;
      __syncthreads();
      if (g == 0) {
        double2 pv = make_double2(0.0, 0.0);
        if (x < mrow) {
#pragma unroll
          for (int q = 1; q < 8; ++q) y = cadd(y, s_u[q][rl]);
          const double2 pr = cmul(tk, y);
          a.p[x] = pr;
          const double2 v = x == 0 ? make_double2(1.0, 0.0) : cmul(__ldcg(&xc[x]), scal);
          xc[x] = v;
          cmacc(pv, pr, v);
        }
        pv.x = warp_sum(pv.x);
        pv.y = warp_sum(pv.y);
        if (rl == 0) a.dotpart[rb] = pv;
      }
      __syncthreads();
    }
    grid.sync();
  }
  // W[:, b-1] = p + alpha v for the panel's last column
  {
    const int cl = a.j0 + b - 1, o = cl + 1;
    const double2 al = panel_alpha(a.dotpart, ndot, tk, sh);
    for (int r = o + blockIdx.x * blockDim.x + threadIdx.x; r < n; r += nblk * blockDim.x) {
      double2 wv = __ldcg(&a.p[r - o]);
      cmac(wv, al, __ldcg(&a.A[r + (long)cl * n]));
      W[r + (long)(b - 1) * n] = wv;
    }
  }
  if (warp == 0 && lane == 0) hs_produce_drain(m, issued, last_ph, a.err);
  if (warp == 1 && lane == 0) hs_mma_finish(m, a.err);
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
    PW_CUDA(cudaFuncSetAttribute(k_hemv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, HsL<NST_HEMV>::SMEM));
    PW_CUDA(cudaFuncSetAttribute(k_panel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, HsL<NST_PANEL>::SMEM));
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

pw_status pw_hs_hemv(pw_dense_ws *ws, const double2 *A, int n, int c, int i, int b, int j0, int *nslots,
                     cudaStream_t st) {
  PW_TRY(allow_smem());
  HsArgs a;
  a.side.A = A;
  a.side.n = n;
  a.side.c = c;
  a.side.i = i;
  a.side.b = b;
  a.side.P = ws->panel;
  a.side.ucorr = ws->ucorr;
  a.hsl = (const unsigned char *)ws->hsl;
  a.slot = ws->hsmax + j0 / 32;
  a.hscal = ws->hscal;
  a.part = ws->part;
  a.nmax = ws->nmax;
  a.J0 = (c + 1) / HT;
  const int ntp = (n + HT - 1) / HT - a.J0;
  // pieces per (tile, part): enough units for every SM, within the partial
  // slots ws->part holds ((nmax + 31) / 32)
  const int sms = sm_count();
  a.ks = hs_pieces(ntp, sms, (ws->nmax + 31) / 32);
  a.units = ntp * (ntp + 1) * a.ks;
  a.err = ws->oz.err;
  *nslots = 2 * ntp * a.ks;
  const int grid = std::min(a.units, sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = HsL<NST_HEMV>::SMEM;
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

int pw_hs_panel_grid() {
  // one CTA per SM, all resident (cooperative launch): the occupancy check
  // confirms one fits
  int per = 0;
  if (allow_smem() != PW_OK ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_panel_tc, NTHR_PANEL, HsL<NST_PANEL>::SMEM) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per >= 1 ? sm_count() : 0;
}

pw_status pw_hs_panel(pw_dense_ws *ws, double2 *A, int n, int j0, int b, int grid, cudaStream_t st) {
  PW_TRY(allow_smem());
  PanelArgs a;
  a.A = A;
  a.n = n;
  a.j0 = j0;
  a.b = b;
  a.P = ws->panel;
  a.p = ws->p;
  a.dotpart = ws->w;
  a.tau = ws->tau;
  a.d = ws->d;
  a.e = ws->e;
  a.nrm_part = ws->nrm_part;
  a.hscal = ws->hscal;
  a.ucorr = ws->ucorr;
  a.hsl = (const unsigned char *)ws->hsl;
  a.slot = ws->hsmax + j0 / 32;
  a.part = ws->part;
  a.nmax = ws->nmax;
  a.slots = (ws->nmax + 31) / 32;
  a.err = ws->oz.err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHR_PANEL);
  cfg.dynamicSmemBytes = HsL<NST_PANEL>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return pw_coop_ordered(st, [&]() -> pw_status {
    pw_count_launch();
    PW_CUDA(cudaLaunchKernelEx(&cfg, k_panel_tc, a));
    return PW_OK;
  });
}
