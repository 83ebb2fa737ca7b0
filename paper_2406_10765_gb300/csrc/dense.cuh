// FP64 dense linear algebra of the Rayleigh-Ritz step, on the GPU.
#pragma once
#include <functional>

#include "oz_gemm.cuh"
#include "pw_internal.cuh"

// Workspace for Rayleigh-Ritz problems up to order nmax with up to nbmax wanted pairs.
struct pw_dense_ws {
  int nmax = 0, nbmax = 0;
  double2 *G = nullptr, *A = nullptr, *T = nullptr, *Linv = nullptr;  // nmax^2 each
  double2 *Y = nullptr;       // nmax x nbmax
  double *dscale = nullptr;   // nmax
  double *piv = nullptr;      // nmax
  int *flag = nullptr;        // device status words
  // tridiagonal eigensolver
  double *d = nullptr, *e = nullptr, *lam = nullptr;  // nmax
  double2 *tau = nullptr;                             // nmax
  double2 *p = nullptr, *w = nullptr;                 // nmax
  double2 *part = nullptr;                            // hemv partial sums
  double *Z = nullptr, *W = nullptr, *U = nullptr;    // nmax^2 real
  double *Ds = nullptr, *zs = nullptr, *DK = nullptr, *zK = nullptr, *tauK = nullptr,
         *zh = nullptr, *lamK = nullptr, *dD = nullptr, *lnew = nullptr;
  int *perm = nullptr, *colK = nullptr, *orig = nullptr, *dcol = nullptr, *src = nullptr;
  int *nodes = nullptr;       // per-level node tables (lo, mid, hi) for nmax
  int *knode = nullptr;       // per node: nondeflated count
  // per column: which half of the node it is nonzero in (0 upper, 1 lower,
  // 2 both after a deflating rotation); per node: the root columns each half
  // of the merge product needs, their counts and the roots the caller keeps
  int *ctype = nullptr, *qL = nullptr, *qR = nullptr, *kLR = nullptr, *kneed = nullptr;
  double *rhonode = nullptr;
  double2 *gemm_ws = nullptr; size_t gemm_ws_elems = 0;
  pw_oz_ws oz;                // FP64-accurate tensor-core products (slices, partial sums)
  // captured eigensolver stages (tridiagonalisation, divide and conquer,
  // back-transformation) keyed by stage, order, wanted pairs and buffers
  struct graph_entry {
    int stage, n, nb;
    const void *p0, *p1;
    unsigned gen;
    cudaGraphExec_t exec;
    uint64_t kernels;         // kernel launches the capture holds
  };
  std::vector<graph_entry> graphs;
  int last_key[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
  // blocked back-transformation: reflector panel, its Gram, T, two work blocks
  double2 *Vb = nullptr, *Gv = nullptr, *Tb = nullptr, *Wk = nullptr, *Wk2 = nullptr;
  unsigned *ticket = nullptr;   // last-block-done counter of the Householder steps
  // blocked Householder reduction: panel [V | W | V] (nmax x 3*32), partial
  // norms of a column, the panel correction dots
  double2 *panel = nullptr, *ucorr = nullptr, *hscal = nullptr;
  double2 *Li = nullptr;      // inverse of the current Cholesky diagonal block (CB x CB)
  // tensor-core Hermitian products of the reduction: digit slices of the
  // panel's trailing tiles, the trailing matrix's maximum per panel (ordered
  // bits)
  void *hsl = nullptr;
  unsigned long long *hsmax = nullptr;
  double *nrm_part = nullptr;
  // host side tree for the current n
  int tree_n = -1;
  std::vector<std::vector<int>> levels;   // per level: flat (lo, mid, hi) triples
  std::vector<int> level_off;             // offset of each level in `nodes` (in triples)
  int max_level_nodes = 0;
  size_t bytes = 0;
  // sub-stage timing of the last Rayleigh-Ritz: events at the boundaries of
  // scale+Cholesky+L^-1 | L^-1 A L^-H | tridiagonal | divide & conquer |
  // back-transform + coefficients
  cudaEvent_t ev[6] = {};
  float ms[5] = {0, 0, 0, 0, 0};
};

// Products of the dense solve: FP64-accurate tensor-core product
// (pw_zgemm_oz) when the process-wide mode (pw_dense_products) is 1 and the
// product is large enough to pay for its operand slicing, else the FP64 pipe.
pw_status pw_dense_gemm(pw_dense_ws *ws, char opA, char opB, int m, int n, int k, double2 alpha,
                        const double2 *A, int lda, const double2 *B, int ldb, double2 beta, double2 *C,
                        int ldc, cudaStream_t st, int herm = 0);
int pw_dense_products_mode();

// elapsed times of the last pw_rayleigh_ritz (after its stream synchronised)
void pw_dense_stage_ms(pw_dense_ws *ws, float out[5]);

pw_status pw_dense_alloc(pw_dense_ws *ws, int nmax, int nbmax);

// Hermitian products of the Householder reduction on the tensor cores
// (hemv_tc.cu): used for the panels whose trailing order is at least
// PW_HS_MIN_ORDER when the product mode is 1.  pw_hs_bytes: slice buffer
// bytes for order nmax (0 below the threshold).  pw_hs_slice: the slices of
// the trailing matrix of the panel starting at column j0.  pw_hs_hemv: the
// product for column c (panel index i, width b): partials into ws->part
// (*nslots slots per row, part[s * nmax + row] with the global row index),
// ucorr and v into the panel, as the FP64 k_phemv does.
#define PW_HS_MIN_ORDER 1024
size_t pw_hs_bytes(int nmax);
pw_status pw_hs_slice(pw_dense_ws *ws, const double2 *A, int n, int j0, cudaStream_t st);
pw_status pw_hs_hemv(pw_dense_ws *ws, const double2 *A, int n, int c, int i, int b, int j0, int *nslots,
                     cudaStream_t st);
// All columns of the panel at j0 (width b, trailing order >= PW_HS_MIN_ORDER,
// its slices written) in one cooperative launch of `grid` CTAs (from
// pw_hs_panel_grid, 0 when the device cannot hold one per SM), leaving the
// panel [V | W | V], tau, d, e as the chained kernels and k_pfinal do.
int pw_hs_panel_grid();
pw_status pw_hs_panel(pw_dense_ws *ws, double2 *A, int n, int j0, int b, int grid, cudaStream_t st);
// Runs `launch` (one cooperative launch on st) after the previous
// cooperative launch on the current device, whatever its stream.
pw_status pw_coop_ordered(cudaStream_t st, const std::function<pw_status()> &launch);
void pw_dense_free(pw_dense_ws *ws);

// Lowest nb Ritz pairs of the pencil (A, G), both n x n Hermitian (device,
// leading dims ldg, lda).  theta: device nb doubles; C: device n x nb (ldc)
// coefficients.  *chol_ok (host) = 0 on a Cholesky breakdown (a pivot of the
// Jacobi-scaled Gram <= piv_tol times the largest).  Synchronises `st`.
pw_status pw_rayleigh_ritz(pw_dense_ws *ws, int n, int nb, const double2 *G, int ldg,
                           const double2 *A, int lda, double *theta, double2 *C, int ldc,
                           int *chol_ok, cudaStream_t st, double piv_tol = 1e-14);

// Rayleigh-Ritz in two halves.  pw_rr_factor: Jacobi scaling d and Cholesky
// of G (same pivot test), L^-1, and M = d o L^-H (n x n upper triangular,
// ld ldm); synchronises.  pw_rr_finish: eigensolve of the Hermitian matrix
// At = M^H A M (given, ld lda), theta (nb), C = M Y (n x nb, ldc).  The
// sub-stage events are recorded as for pw_rayleigh_ritz.
pw_status pw_rr_factor(pw_dense_ws *ws, int n, const double2 *G, int ldg, double2 *M, int ldm,
                       int *chol_ok, cudaStream_t st, double piv_tol);
pw_status pw_rr_finish(pw_dense_ws *ws, int n, int nb, const double2 *At, int lda, const double2 *M,
                       int ldm, double *theta, double2 *C, int ldc, cudaStream_t st);
// Variant for callers that hold the orthonormalised basis S~ = S M: leaves
// the eigenvectors Y (n x nb, ld n) in ws->Y for X' = S~ Y and forms only
// the rows nb..n-1 of C = M Y (= M[nb:, nb:] Y[nb:], M upper triangular) in
// Cp, whose rows 0..nb-1 are set to zero: P' = S Cp.
pw_status pw_rr_finish_tall(pw_dense_ws *ws, int n, int nb, const double2 *At, int lda, const double2 *M,
                            int ldm, double *theta, double2 *Cp, int ldc, cudaStream_t st);

// Hermitian eigensolver: lowest nb eigenpairs of the n x n matrix A (device,
// destroyed).  lam: device n doubles (all eigenvalues, ascending); Y: device
// n x nb (ld n) eigenvectors.
pw_status pw_heev_lowest(pw_dense_ws *ws, int n, int nb, double2 *A, double *lam, double2 *Y,
                         cudaStream_t st);
