// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "pw.h"

#define PW_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      pw_last_cuda_error(e_, __FILE__, __LINE__);                       \
      return PW_ERR_CUDA;                                               \
    }                                                                   \
  } while (0)

#define PW_TRY(call)                                                    \
  do {                                                                  \
    pw_status s_ = (call);                                              \
    if (s_ != PW_OK) return s_;                                         \
  } while (0)

void pw_last_cuda_error(cudaError_t e, const char *file, int line);
// count of kernel launches issued by the library (diagnostics; see pw_kernel_launches)
void pw_count_launch();
void pw_count_launches(uint64_t n);
uint64_t pw_thread_launches();   // this thread's count (captures count their kernels)
pw_status pw_check_launch(const char *what);

// --------------------------------------------------------------------------
// complex helpers (double2 / float2)
// --------------------------------------------------------------------------
template <typename T> struct cpx_t;
template <> struct cpx_t<double> { typedef double2 type; };
template <> struct cpx_t<float> { typedef float2 type; };

// SplitMix64 (Steele, Lea and Flood 2014) in counter form: output i of the
// stream `seed`; the seeded synthetic inputs (start blocks, serving
// requests) draw from it on the host and on the device
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {  // conj(a) * b
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
  C r; r.x = a.x + b.x; r.y = a.y + b.y; return r;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
  C r; r.x = a.x - b.x; r.y = a.y - b.y; return r;
}

// --------------------------------------------------------------------------
// the cell
// --------------------------------------------------------------------------
#define PW_MAX_PASSES 12

struct pw_fft_axis {
  int n;
  int npass;
  int radix[PW_MAX_PASSES];
  double2 *tw64;   // device, n entries exp(-2 pi i k / n)
  float2 *tw32;
};

struct pw_cell;
// Bands of one cell for a launch that covers several cells (fft_reg.cuh
// run_multi): the cell, its bands psi / hpsi (ld), its z-pencil buffer.
#define PW_FFT_BATCH_MAX 16
struct pw_fft_job {
  pw_cell *c;
  const double2 *psi;
  double2 *hpsi;
  int ld, nb;
  void *Z;
  double scale;
};
struct pw_cell {
  int precision;
  double L[3];
  int N[3];
  double ecut, vwidth, pwidth;
  int natom, nproj, npw, ncol;
  int mxmax;                 // x-extent of the sphere: mx in [-mxmax, mxmax]
  std::vector<int> m_host;   // npw*3
  std::vector<double> tau_host, depth_host, dkb_host;
  // device tables
  int *d_gcol = nullptr;      // npw: column index of each plane wave
  int *d_gz = nullptr;        // npw: mz mod Nz
  int *d_colstart = nullptr;  // ncol+1: first plane wave of each column
  int *d_colxy = nullptr;     // ncol: (my mod Ny) * Nx + (mx mod Nx)
  double *d_kin = nullptr;    // npw: 1/2 |G|^2
  double *d_V = nullptr;      // Nz*Ny*Nx real potential, index (z*Ny + y)*Nx + x
  float *d_Vf = nullptr;
  double2 *d_beta = nullptr;  // npw x nproj (ld = npw); NULL while generated on the fly
  // projector generation: plane-wave indices and per-axis phase tables
  // exp(-i 2 pi m tau_a / L), kept for regenerating beta (chunks or whole)
  int *d_m = nullptr;
  double2 *d_ph[3] = {nullptr, nullptr, nullptr};
  int Mext[3] = {0, 0, 0};
  double proj_ns = 0, proj_np = 0;
  int proj_onthefly = 0;      // 1: beta generated per chunk of atoms in each H psi
  double2 *d_bchunk = nullptr; size_t bchunk_bytes = 0;
  struct pw_tc_operand *op_bc_rows = nullptr, *op_bc_t = nullptr, *op_psi_c = nullptr;
  double *d_D = nullptr;      // nproj
  pw_fft_axis ax[3];
  // apply_H workspace (grown on demand)
  void *d_z = nullptr; size_t z_bytes = 0;
  // FFT plan per precision ([0] FP64, [1] FP32): register line-FFT plan index,
  // -1 for the Stockham passes, -2 for the default; z-pencil batch bytes (0: default)
  int fft_plan[2] = {-2, -2};
  int fft_compact[2] = {0, 0};
  size_t fft_batch[2] = {0, 0};
  std::string fft_tune_log;   // candidates and times of the last FFT tuning
  double *d_dpart = nullptr; size_t dpart_bytes = 0;   // density partial sums
  double *d_V0 = nullptr;                              // the cell's own V_loc while another V is set
  double2 *d_grid = nullptr; size_t grid_bytes = 0;    // full-grid FFT scratch
  double2 *d_B = nullptr; size_t B_elems = 0;   // nproj x nb projections
  double2 *d_gemm_ws = nullptr; size_t gemm_ws_elems = 0;
  struct pw_oz_ws *oz = nullptr;   // FP64-accurate tensor-core products (FP64 projector terms)
  // set by the serving loop: the local part of H psi goes to a launch shared
  // with other requests' cells (register plans only); returns once that
  // launch is ordered on `st`
  pw_status (*fft_hook)(void *ctx, const pw_fft_job &job, const struct pw_reg_plan *plan, int fp32, int cp,
                        cudaStream_t st) = nullptr;
  void *fft_hook_ctx = nullptr;
  size_t bytes = 0;
  // mixed-precision operands (split FP16), built on first use: beta as rows
  // over G (for beta^H psi) and as rows over projectors (for beta (D B))
  struct pw_tc_operand *op_beta_rows = nullptr, *op_beta_t = nullptr;
  struct pw_tc_operand *op_psi = nullptr, *op_db = nullptr;
  float *d_rmax = nullptr;
  int *d_tc_err = nullptr;
  void *d_beta_split = nullptr; size_t beta_split_bytes = 0;
};

// beta columns 4 a0 .. 4 (a0 + na) - 1 into out (npw x 4 na, ld npw)
pw_status pw_beta_chunk(pw_cell *c, int a0, int na, double2 *out, cudaStream_t st);
// beta rows g0 .. g0+ng-1 of every projector, FP32 arithmetic, into out (ng x nproj, ld ng)
pw_status pw_beta_rows_f32(pw_cell *c, int g0, int ng, double2 *out, cudaStream_t st);

// apply_H pieces
pw_status pw_apply_local(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                         int precision, cudaStream_t st);
pw_status pw_apply_nonlocal(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                            int precision, cudaStream_t st);

// FP64 H pieces writing only into caller-provided scratch (no allocation)
size_t pw_local_zbytes_per_band(const pw_cell *c);
// Register line-FFT plans for cubic grids N = L R (fft_reg_*.cu).  run*: one
// batch of nbb bands through K1-K3 via the z-pencil buffer Z; dens*: the
// density of one batch (z-pencils into Z, then per (z-plane, band group) the
// inverse plane FFTs and sum_j occ[j] |psi_j(r)|^2 into part[group][z][y][x]).
// run*[compact]: plane kernel with the full N x N plane (0) or only the
// sphere's x-columns (1) in shared memory; smem: its shared-memory bytes.
typedef pw_status (*pw_reg_run_fn)(pw_cell *, const double2 *, int, int, double2 *, void *, double,
                                   cudaStream_t);
typedef pw_status (*pw_reg_multi_fn)(const pw_fft_job *, int, cudaStream_t);
struct pw_reg_plan {
  int N, L, R;
  pw_reg_run_fn run64[2], run32[2];
  pw_status (*dens64)(pw_cell *, const double2 *, int, int, void *, const double *, int, double *,
                      cudaStream_t);
  pw_status (*dens32)(pw_cell *, const double2 *, int, int, void *, const double *, int, double *,
                      cudaStream_t);
  size_t (*smem)(const pw_cell *, int fp32, int compact);
  pw_reg_multi_fn multi64[2], multi32[2];
};
int pw_reg_plan_count();
const pw_reg_plan *pw_reg_plan_at(int i);
// plan i can run this cell's grid in this precision and plane layout (cubic
// grid of size N, plane in shared memory, sphere columns that do not wrap)
bool pw_reg_plan_fits(const pw_cell *c, int i, int fp32, int compact);
// the cell's FFT plan for a precision (resolving the default): a plan index,
// or -1 for the Stockham passes; its plane layout; its z-pencil batch bytes
int pw_cell_fft_plan(const pw_cell *c, int fp32);
int pw_cell_fft_compact(const pw_cell *c, int fp32);
size_t pw_cell_fft_batch_bytes(const pw_cell *c, int fp32);
// unscaled 3-D FFT of a complex grid g[(z N1 + y) N0 + x] in place (sign -1
// forward, +1 inverse)
pw_status pw_grid_fft(pw_cell *c, double2 *g, int inverse, cudaStream_t st);
pw_status pw_fft_density_batch(pw_cell *c, const double2 *psi, int ld, int nbb, void *Z, int fp32,
                               const double *occ, int ngroups, double *part, cudaStream_t st);
pw_status pw_apply_local_fp64_into(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                                   void *zbuf, size_t zbytes, cudaStream_t st);
pw_status pw_apply_nonlocal_fp64_into(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                                      double2 *B, double2 *ws, size_t ws_elems, cudaStream_t st);

// dense complex FP64 GEMM: C = alpha op(A) op(B) + beta C, column-major.
// opA: 'N' (A is m x k) or 'C' (A is k x m, conjugate-transposed);
// opB: 'N' (B is k x n) or 'C' (B is n x k, conjugate-transposed).
pw_status pw_zgemm(char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                   int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc,
                   double2 *ws, size_t ws_elems, cudaStream_t st);
size_t pw_zgemm_ws_elems(int m, int n, int k);
// herm = 1: C is Hermitian (A^H B with A == B up to H-symmetry); only the
// upper-triangle tiles are computed, then mirrored.  herm = 2: only the tiles
// on and below the diagonal are computed (the caller keeps a lower triangle).
// herm = 3: op(A) is upper triangular (explicit zeros below the diagonal), so
// each row tile skips the K range left of its first row; herm = 4: op(B) is
// lower triangular (column tiles skip K below their first column); herm = 5:
// op(A) is lower triangular (row tiles stop K after their last row).
pw_status pw_zgemm_ex(char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                      int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc,
                      double2 *ws, size_t ws_elems, cudaStream_t st, int herm);
// batch independent products, operand i at A + i sA, B + i sB, C + i sC
// (element strides); mode as herm above except 1 (no mirror pass)
pw_status pw_zgemm_batched(char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                           int lda, long sA, const double2 *B, int ldb, long sB, double2 beta,
                           double2 *C, int ldc, long sC, int batch, cudaStream_t st, int mode);
// C (n x n) = A^H B, Hermitian result (upper tiles + mirror)
pw_status pw_zgemm_herm(int n, int k, const double2 *A, int lda, const double2 *B, int ldb,
                        double2 *C, int ldc, double2 *ws, size_t ws_elems, cudaStream_t st);

// grow a device buffer
pw_status pw_ensure(void **ptr, size_t *cur_bytes, size_t need_bytes);
