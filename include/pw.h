/*
 * pw.h -- C ABI of the GB300 plane-wave block-eigensolver library.
 *
 * The library solves the fixed-potential plane-wave Kohn-Sham eigenproblem
 * H X = X Lambda (Sec. II-A, Eq. 1) for the lowest nb bands with LOBPCG,
 * one of the inner eigensolvers of Sec. II-A.  One step applies H to a block
 * of bands by FFT (the column scheme of Sec. II-B) plus the Kleinman-Bylander
 * projector contractions (the pseudopotential application of Sec. III-A),
 * forms the subspace matrices S^H S and S^H (H S) (Sec. II-B), and solves the
 * small dense eigenproblem (Syevd, Sec. III-D) on the GPU in FP64.
 *
 * Conventions shared by every entry point:
 *  - Units: Hartree atomic units (bohr, Ha).
 *  - Wavefunction blocks are complex128 (interleaved re, im doubles),
 *    column-major npw x nb with leading dimension ld >= npw: column j is band
 *    j, entry g is the coefficient of plane wave G_g = 2 pi m_g / L.  The
 *    plane-wave order is the library's canonical sphere order: integer
 *    vectors m with 1/2 |G|^2 <= Ecut, sorted lexicographically by
 *    (m_x, m_y, m_z), so each z-column of the sphere is contiguous.
 *    pw_cell_info() returns that order.
 *  - Device pointers are plain CUDA device addresses (for example from
 *    torch.Tensor.data_ptr()); host pointers are plain host memory.  The
 *    caller owns every buffer it passes; the library owns pw_cell and
 *    pw_solver objects and their device workspaces.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - No exceptions cross the ABI.  Every call returns a pw_status;
 *    pw_strerror() names it.  Calls on the same pw_cell must not overlap.
 */
#ifndef PW_H
#define PW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pw_cell pw_cell;
typedef struct pw_solver pw_solver;

typedef enum {
  PW_OK = 0,
  PW_ERR_ARG = -1,      /* invalid argument or unsupported size */
  PW_ERR_OOM = -2,      /* device allocation failed */
  PW_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  PW_ERR_CHOL = -4,     /* overlap matrix not positive definite, even without P */
  PW_ERR_NOCONV = -5,   /* maxit reached; partial results are filled in */
  PW_ERR_TIMEOUT = -6,  /* a bounded device wait ran out */
  PW_ERR_BUSY = -7,     /* admission refused: not enough device memory */
  PW_ERR_NUMERIC = -8   /* NaN/Inf met in a residual norm or eigensolve */
} pw_status;

enum { PW_FP64 = 0, PW_MIXED = 1 };

/* Cell description.  All pointers are caller-owned host memory, copied by
 * pw_setup_cell.  Inputs follow the synthetic Si/C workloads: Gaussian local
 * wells V(r) = sum_a d_a sum_R exp(-|r - tau_a - R|^2 / (2 vwidth^2)) and,
 * per atom, four Gaussian KB projectors (s, p_x, p_y, p_z) of radial width
 * pwidth with diagonal coefficients dkb. */
typedef struct {
  double lattice[9];    /* bohr, column-major 3x3 (columns a1 a2 a3); must be
                           diagonal (orthorhombic cell) */
  int natom;
  const double *tau;    /* natom*3 Cartesian positions, bohr */
  const double *vdepth; /* natom well depths d_a, Ha */
  double vwidth;        /* sigma, bohr */
  double pwidth;        /* r_p, bohr */
  const double *dkb;    /* natom*4: D_s, D_px, D_py, D_pz, Ha */
  double ecut;          /* Ha */
  int grid[3];          /* FFT grid; 0 -> smallest 2^a 3^b >= 1.5 sqrt(2 Ecut) L_i / pi
                           (the grid rule of Sec. II-A times 1.5) */
  int precision;        /* PW_FP64 or PW_MIXED */
} pw_cell_desc;

/* Builds the plane-wave sphere, the FFT grid, V_loc(r) on the grid, the
 * kinetic table and the projector matrix beta (npw x 4 natom) on the device
 * of the calling thread, on `stream` (the call synchronises it).
 * Errors: PW_ERR_ARG (non-orthorhombic lattice, Ecut <= 0, natom < 0, a plane
 * wave within 1e-9 Ha of Ecut, grid too small for the sphere or not 2^a 3^b,
 * plane too large for shared memory), PW_ERR_OOM, PW_ERR_CUDA.  On error
 * *out is NULL. */
pw_status pw_setup_cell(const pw_cell_desc *desc, void *stream, pw_cell **out);

/* npw, grid and a host pointer to the npw*3 integer vectors m (owned by the
 * cell, valid until pw_destroy_cell).  Any output pointer may be NULL. */
pw_status pw_cell_info(const pw_cell *cell, int *npw, int grid[3], const int **mvec);

/* Number of projectors (4 natom) and bytes of device memory held by the cell. */
pw_status pw_cell_sizes(const pw_cell *cell, int *nproj, size_t *device_bytes);

/* Selects the arithmetic of later pw_apply_H calls on this cell: PW_FP64, or
 * PW_MIXED (FP32 FFTs and split-FP16 tensor-core projector contractions --
 * two FP16 slices per row-scaled operand, the reading of "split-BF16" that
 * keeps 22 bits -- FP64 kinetic term and FP64 accumulation of the result). */
pw_status pw_cell_set_precision(pw_cell *cell, int precision);

/* hpsi = H psi for nb bands (Sec. II-A Eq. 1; FFT local term per Sec. II-B,
 * nonlocal term per Sec. III-A).  psi, hpsi: device complex128 npw x nb,
 * leading dimension ld >= npw; they must not overlap.  nb = 0 is a no-op.
 * Errors: PW_ERR_ARG (NULL pointer with nb > 0, ld < npw, nb < 0),
 * PW_ERR_OOM (workspace growth), PW_ERR_CUDA. */
pw_status pw_apply_H(pw_cell *cell, const void *psi, int ld, int nb, void *hpsi, void *stream);

/* Projector storage of a cell.  onthefly = 0 (default): beta (npw x 4 natom
 * complex128, and in mixed precision its split-FP16 copies) stays resident.
 * onthefly = 1: beta is freed and pw_apply_H regenerates it in chunks of
 * atoms (at most 256 MB of beta at a time) from the plane-wave indices and
 * per-axis structure-factor tables: the same operator (Sec. III-A), FP64
 * values, the projection summed chunk by chunk.  Trades the resident
 * projector memory for one projector evaluation per H psi.  Synchronises
 * `stream`.  Errors: PW_ERR_ARG, PW_ERR_OOM (switching back), PW_ERR_CUDA. */
pw_status pw_cell_set_projectors(pw_cell *cell, int onthefly, void *stream);

/* Size of the fixed device scratch array used by pw_apply_H_noalloc. */
#define PW_NOALLOC_SCRATCH_BYTES (16u << 20)

/* H psi without allocating any device memory.  The paper has no counterpart:
 * this is a library convenience for callers that cannot call cudaMalloc when
 * they apply H, e.g. a host framework whose pool allocator reserved the GPU,
 * or a latency-critical loop that must avoid cudaMalloc's implicit
 * synchronisation.  Same operator and arguments as pw_apply_H, always in FP64
 * arithmetic; all scratch (FFT z-pencils, projector coefficients, GEMM partial
 * sums) lives in one static device array of PW_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  The cell must
 * already exist (pw_setup_cell allocates).  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Calls share the
 * array: calls that overlap on the GPU (other streams, other threads) race.
 * Errors: PW_ERR_ARG as pw_apply_H, for a cell that generates its
 * projectors on the fly (pw_cell_set_projectors), and when the scratch would exceed
 * PW_NOALLOC_SCRATCH_BYTES (projector coefficients, partial sums and one
 * band's z-pencils must fit: roughly nb <= 400 for a 2,048-projector cell,
 * fewer at small nb-independent limits); PW_ERR_CUDA. */
pw_status pw_apply_H_noalloc(pw_cell *cell, const void *psi, int ld, int nb, void *hpsi,
                             void *stream);

/* Solver options. */
typedef struct {
  int nbands;           /* nb >= 1, nb <= npw / 3 */
  double tol;           /* residual-norm tolerance (bands below it are locked) */
  int maxit;            /* maximum LOBPCG steps for pw_eigsolve */
  uint64_t seed;        /* SplitMix64 stream of the random start when x0 == NULL */
  const void *x0;       /* optional complex128 npw x nbands start (ld = npw), host
                           or device memory */
  int precision;        /* PW_FP64 or PW_MIXED */
  int chunk_rows;       /* PW_MIXED: plane-wave rows per chunk of the tall
                           split-FP16 products (Gram, S M, rotations); 0 picks
                           chunks whose split operands stay under ~8 GB.  Bounds
                           the solver's scratch; results agree to rounding. */
  int h_blocks;         /* PW_MIXED: 0 (default) apply H to [X W P] every
                           step; 1 carry H X and H P through the split-FP16
                           rotations (one H application per step, to W) while
                           the largest residual norm is above 1e-3, then apply
                           H to [X W P], no band locks while carrying; 2 always
                           carry (stalls near 1e-4: the carried blocks hold the
                           split products' error).  FP64 always carries. */
} pw_solve_opts;

typedef struct {
  int iter;             /* steps taken so far */
  int nactive;          /* active (unlocked) bands used in this step */
  int dropped_p;        /* 1 if P was dropped after a Cholesky breakdown */
  int nsub;             /* order of the Rayleigh-Ritz problem (nb + k or nb + 2k) */
  double max_resid;     /* max_i ||H x_i - theta_i x_i|| of the block the step started from */
  double ms;            /* wall time of the step (host clock, synchronised) */
  /* device time per stage (CUDA events on the solver's stream), ms: */
  double ms_resid;      /* residual norms + preconditioner */
  double ms_hpsi;       /* every H application of the step (FFT local part +
                           projector contractions): H W, and in mixed precision
                           also H X and H P, which are recomputed each step */
  double ms_gram;       /* S^H S and S^H (H S) */
  double ms_rr;         /* Cholesky, L^-1, eigensolve, coefficients (FP64) */
  double ms_rot;        /* rotations X', H X', P', H P' */
  /* inside ms_rr: scale + Cholesky + L^-1 | L^-1 A L^-H | Householder
   * tridiagonalisation | divide and conquer | back-transform + coefficients */
  double ms_rr_part[5];
  int hpsi_cols;        /* columns H was applied to in the step */
} pw_step_report;

typedef struct {
  int iters;            /* LOBPCG steps taken (all precisions) */
  int fp64_iters;       /* of which FP64 refinement steps after a mixed solve */
  double max_resid;     /* final max residual norm (FP64) */
  double orth_err;      /* max |X^H X - I| of the final block (FP64) */
  double seconds;
  size_t device_bytes;  /* solver workspace */
} pw_solve_report;

/* Creates LOBPCG state for `opts->nbands` bands: draws or copies the start
 * block, applies H, and performs the initial Cholesky-QR + Rayleigh-Ritz.
 * Synchronises `stream`.  Errors: PW_ERR_ARG, PW_ERR_OOM, PW_ERR_CHOL,
 * PW_ERR_NUMERIC, PW_ERR_CUDA. */
pw_status pw_solver_create(pw_cell *cell, const pw_solve_opts *opts, void *stream,
                           pw_solver **out);

/* One LOBPCG step (residual, preconditioner, H W, S^H S and S^H H S,
 * Cholesky, Rayleigh-Ritz, rotation), Knyazev's method with the
 * Hetmaniuk-Lehoucq P.  Synchronises the solver's stream.  rep may be NULL.
 * Errors: PW_ERR_CHOL (overlap not positive definite even without P),
 * PW_ERR_NUMERIC, PW_ERR_CUDA. */
pw_status pw_subspace_step(pw_cell *cell, pw_solver *solver, pw_step_report *rep);

/* FP64 Rayleigh-Ritz refinement of the current block: H X, X^H X and
 * X^H (H X) in FP64, FP64 Cholesky and eigensolve, FP64 rotation.  Used to
 * finish mixed-precision solves (FP64 overlap, eigenvalues, residual norms
 * and orthonormality).  Drops P.  Synchronises the solver's stream. */
pw_status pw_solver_polish(pw_solver *solver);

/* Current Ritz values (host, nb) and residual norms of the current block
 * (host, nb; computed in FP64).  Either pointer may be NULL. */
pw_status pw_solver_eigs(pw_solver *solver, double *eig, double *resid);

/* Copies the current block X (device complex128 npw x nb, leading dim ld). */
pw_status pw_solver_block(pw_solver *solver, void *psi, int ld);

/* Search directions of Knyazev's method (the block P of the LOBPCG step,
 * Sec. II-A names LOBPCG as an inner eigensolver).  pw_solver_set_p replaces
 * P by the nb columns of p (complex128 npw x nb, leading dimension ld >= npw,
 * host or device memory; columns are normalised, and in FP64 the matching
 * H P is formed); the next pw_subspace_step then uses S = [X, W, P].  With
 * pw_solver_get_p (copies P into p, same layout; *have_p = 1 once a step or
 * set_p has defined it, may be NULL) and pw_solver_block, a solve can be saved
 * and resumed: pw_solver_create with x0 = the saved block, then set_p.  A P
 * that makes the overlap singular (for example columns inside span(X)) is
 * dropped by the next step's Cholesky pivot test (pw_step_report.dropped_p).
 * Both synchronise the solver's stream.  Errors: PW_ERR_ARG (NULL, ld < npw),
 * PW_ERR_OOM, PW_ERR_CUDA. */
pw_status pw_solver_set_p(pw_solver *solver, const void *p, int ld);
pw_status pw_solver_get_p(pw_solver *solver, void *p, int ld, int *have_p);

void pw_solver_destroy(pw_solver *solver);

/* Runs LOBPCG to max residual <= tol or maxit steps.  eig: host nb doubles
 * (required); psi_out: device complex128 npw x nb (ld) or NULL.  With
 * opts->precision == PW_MIXED the block converged in mixed precision is
 * finished by pw_solver_polish (FP64); bands still above tol then continue in
 * FP64 (rep->fp64_iters, at most 8 steps) within maxit, and the reported
 * residuals are FP64.  Returns PW_ERR_NOCONV with eig / psi_out filled if
 * maxit (or the FP64 step limit) is reached. */
pw_status pw_eigsolve(pw_cell *cell, const pw_solve_opts *opts, double *eig, void *psi_out,
                      int ld, pw_solve_report *rep, void *stream);

/* ---------------------------------------------------------------- serving
 * A request is a fixed-potential eigensolve of a synthetic diamond supercell:
 * Si (a = 10.26 bohr) or C (a = 6.74 bohr), n x n x n cubic cells (8 n^3
 * atoms), Gaussian wells and KB projectors as in pw_cell_desc (widths 1.2
 * bohr) with depths and D drawn from the request's SplitMix64 stream (depth
 * a: draw a, d = -1 + 0.1 (2u - 1); D[a][k]: draw 8n^3 + 4a + k, 0.5 + u) and
 * the random start block of pw_solve_opts.seed. */
typedef struct {
  int species;          /* 0 = Si, 1 = C */
  int ncell;            /* n >= 1 */
  double ecut;          /* Ha */
  int nbands;
  uint64_t seed;
  double t_arrival;     /* seconds after pw_serve starts (times opts.time_scale) */
  double tol;           /* 0 -> 1e-8 (FP64) or 5e-6 (mixed) */
  int maxit;            /* 0 -> 300 */
} pw_request;

typedef struct {
  double *eig;          /* caller-owned host buffer of nbands doubles (filled) */
  int status;           /* pw_status of this request (PW_ERR_BUSY: larger than the budget) */
  int iters, npw;
  double max_resid, orth_err;
  double t_admit, t_done, latency;   /* seconds; latency = t_done - arrival */
  size_t hbm_bytes;     /* footprint used for admission */
} pw_result;

typedef struct {
  int max_slots;        /* requests on the GPU at once (worker threads / streams) */
  size_t hbm_budget;    /* bytes admitted at once; 0 -> 80% of free device memory */
  int precision;        /* PW_FP64 or PW_MIXED */
  double time_scale;    /* multiplies arrival times; 0 -> 1 */
  int autotune;         /* 1: the first request of each grid size tunes the FFT
                           plan (pw_cell_autotune_fft on its bands) and later
                           requests of that grid reuse it; the tensor-core K
                           splits follow pw_autotune_gemm's process-wide mode */
  int batch_fft;        /* PW_MIXED, 1: the FFT local parts of H psi of the
                           requests running at once that share a grid size and
                           plan run in one launch per kernel (up to 16 cells'
                           band blocks, uneven band counts and spheres); a
                           request waits at most batch_window_us for partners.
                           Results are the same as unbatched. */
  double batch_window_us;  /* 0 -> 100 */
} pw_serve_opts;

/* Launches of the cross-request FFT batching of pw_serve in this process and
 * the band blocks (one per request per launch) they carried. */
void pw_fft_batch_stats(uint64_t *launches, uint64_t *jobs);

/* Device-memory footprint model used to admit a request (bytes). */
size_t pw_request_footprint(const pw_request *req, int precision);

/* Serves a stream of requests with continuous batching on the current
 * device: a request is admitted at its arrival time once a slot is free and
 * its footprint fits under the budget next to the requests already running;
 * admitted requests run concurrently on their own streams, so their kernels
 * overlap; results[i] receives the eigenvalues, status and timings of
 * req[i].  Each request's result is independent of the mix (inputs from its
 * seed, deterministic kernels).  Blocks until every request has finished.
 * Errors: PW_ERR_ARG (bad options or request fields, NULL eig buffer),
 * PW_ERR_CUDA; per-request failures are reported in results[i].status. */
pw_status pw_serve(const pw_serve_opts *opts, const pw_request *req, int nreq, pw_result *results);

/* Electron density of a block of bands on the cell's FFT grid, the quantity
 * the self-consistent loop of Sec. II-A forms from the converged
 * wavefunctions: rho(r_j) = sum_b occ_b |psi_b(r_j)|^2 with psi_b(r_j) =
 * sum_G c_bG exp(i G.r_j), r_j = L j / N (no normalisation factor).
 * psi: device complex128 npw x nb, leading dimension ld >= npw, sphere order
 * of pw_cell_info.  occ: device nb doubles, or NULL for all ones.  rho:
 * device N0*N1*N2 doubles, x fastest: rho[(jz*N1 + jy)*N0 + jx]; overwritten.
 * Uses the cell's precision for the FFTs (FP32 in mixed mode) and sums in
 * FP64 across band groups; the result is independent of scheduling.  Shares
 * the cell's FFT workspace with pw_apply_H (no concurrent calls on one cell).
 * Asynchronous on `stream`.  Errors: PW_ERR_ARG (nb < 0, ld < npw, NULL
 * pointer, a grid whose plane exceeds shared memory), PW_ERR_OOM, PW_ERR_CUDA. */
pw_status pw_density(pw_cell *cell, const void *psi, int ld, int nb, const double *occ, double *rho,
                     void *stream);

/* Model exchange-correlation step of the self-consistent loop of Sec. II-A
 * (the paper fixes no functional): v(r) = V_H(r) + v_x(r) from an electron
 * density n(r), with V_H the periodic solution of lap V_H = -4 pi (n - <n>)
 * (V_H(G) = 4 pi n(G) / |G|^2, G = 2 pi k / L, V_H(0) = 0) and the
 * Slater/Dirac exchange v_x = -(3 n / pi)^(1/3).  n, v: device N0*N1*N2
 * doubles, x fastest ([z][y][x], as rho of pw_density); n is not changed.
 * FP64.  Asynchronous on `stream`.  Errors: PW_ERR_ARG (NULL pointer),
 * PW_ERR_OOM, PW_ERR_CUDA. */
pw_status pw_hxc_potential(pw_cell *cell, const double *n, double *v, void *stream);

/* Local potential of the cell becomes V_loc + v_hxc (device N0*N1*N2
 * doubles, [z][y][x]; copied), in both the FP64 and FP32 copies used by
 * pw_apply_H; v_hxc == NULL restores the cell's own V_loc.  Asynchronous on
 * `stream`.  Errors: PW_ERR_ARG, PW_ERR_OOM, PW_ERR_CUDA. */
pw_status pw_cell_set_hxc(pw_cell *cell, const double *v_hxc, void *stream);

typedef struct {
  int nbands;           /* bands solved for (>= nocc) */
  int nocc;             /* occupied bands */
  double fill;          /* occupation of each occupied band (2 for spin pairs) */
  double mix;           /* linear density mixing, 0 < mix <= 1 */
  int maxiter;          /* SCF iterations at most */
  double tol;           /* stop when max_r |n_out - n_in| <= tol */
  double eig_tol;       /* pw_eigsolve tolerance of each iteration */
  int eig_maxit;        /* pw_eigsolve step limit of each iteration */
  uint64_t seed;        /* random start block of the first iteration */
  int precision;        /* PW_FP64 | PW_MIXED (eigensolves and FFTs) */
} pw_scf_opts;

typedef struct {
  int iters;            /* SCF iterations taken */
  int eig_iters;        /* LOBPCG steps over all iterations */
  double max_dn;        /* max |n_out - n_in| of the last iteration */
} pw_scf_report;

/* Self-consistent field loop with the model V_Hxc of pw_hxc_potential:
 * starting from n_in = 0, iteration k sets V = V_loc + V_Hxc[n_in]
 * (pw_cell_set_hxc), solves for the lowest nbands eigenpairs (pw_eigsolve,
 * started from the previous iteration's block), forms
 * n_out = Omega^-1 sum_{b < nocc} fill |psi_b|^2 (pw_density) and mixes
 * n_in <- (1 - mix) n_in + mix n_out, until max |n_out - n_in| <= tol or
 * maxiter.  eig: host nbands doubles (last iteration).  n_out: device
 * N0*N1*N2 doubles or NULL (last output density).  The cell keeps the last
 * V = V_loc + V_Hxc[n_in].  Synchronises `stream`.  Returns PW_ERR_NOCONV
 * (results filled) if maxiter is reached; errors as pw_eigsolve. */
pw_status pw_scf(pw_cell *cell, const pw_scf_opts *opts, double *eig, double *n_out, pw_scf_report *rep,
                 void *stream);

/* FP64 Hermitian eigensolver used by the Rayleigh-Ritz step (the small dense
 * eigensolve, Syevd in Sec. III-D): Householder reduction to a real
 * tridiagonal, divide and conquer, back-transformation.  A: device complex128
 * n x n Hermitian, column-major, ld n; destroyed.  w: device n doubles (all
 * eigenvalues, ascending).  Y: device complex128 n x nb (ld n), eigenvectors
 * of the nb lowest.  Synchronises `stream`.  Errors: PW_ERR_ARG (n < 1,
 * nb < 1, nb > n, NULL pointer), PW_ERR_OOM, PW_ERR_CUDA. */
pw_status pw_heev(int n, int nb, void *A, double *w, void *Y, void *stream);

/* Complex matrix product on the tensor cores in split-FP16 arithmetic (the
 * mixed-precision form of the dense contractions: projector products of
 * Sec. III-A, S^H S, S^H (H S) and the rotations of Sec. II-B).  Each operand
 * row is scaled by a power of two and split into two FP16 slices (hi, lo);
 * the products hi*hi + hi*lo + lo*hi accumulate in FP32 and the result is
 * rescaled in FP64 (relative error ~1e-6 of |A||B|).
 *   opA = 'C': C (m x n) = A^H B, A: k x m (lda), B: k x n (ldb)
 *   opA = 'N': C (m x n) = A B,   A: m x k (lda), B: k x n (ldb)
 * All device complex128, column-major.  beta: 0 (overwrite) or 1 (C += ...).
 * Allocates and frees its own operand buffers; synchronises `stream`.
 * Errors: PW_ERR_ARG (bad op, sizes < 1, ld too small, beta not 0/1),
 * PW_ERR_OOM, PW_ERR_CUDA, PW_ERR_TIMEOUT (a bounded device wait ran out). */
pw_status pw_zgemm_tc(char opA, int m, int n, int k, const void *A, int lda, const void *B,
                      int ldb, double beta, void *C, int ldc, void *stream);

/* Complex FP64 matrix product on the FP16 tensor cores, FP64-accurate: the
 * dense products of the Rayleigh-Ritz solve (Syevd, Sec. III-D, and the
 * Cholesky and back-transformation around it) without the FP64 pipe.  Each
 * real row of op(A) and each real column of op(B) is scaled by a power of
 * two and written exactly as 8 integer slices of 7 bits (FP16 values); the
 * slice products whose weights reach 2^-63 are accumulated exactly (FP32
 * tensor-core sums over 64-wide K chunks are integers below 2^22) into a
 * 64-bit fixed-point sum and converted to FP64 once.  Error per entry at
 * most 11K 2^-55 max_k |op(A)_ik| max_k |op(B)_kj|, within the FP64 product
 * bound for rows without large internal range.
 *   C (m x n) = alpha op(A) op(B) + beta C,  op in {'N', 'C'}:
 *   op(A) = A (m x k, lda >= m) or A^H (A k x m, lda >= k);
 *   op(B) = B (k x n, ldb >= k) or B^H (B n x k, ldb >= n).
 * All device complex128, column-major; alpha, beta: host pointers to
 * (re, im).  Allocates and frees its slice buffers; synchronises `stream`.
 * Errors: PW_ERR_ARG (bad op, sizes, leading dimensions, NULL), PW_ERR_OOM,
 * PW_ERR_CUDA, PW_ERR_TIMEOUT (a bounded device wait ran out). */
pw_status pw_zgemm_f64tc(char opA, char opB, int m, int n, int k, const double *alpha, const void *A,
                         int lda, const void *B, int ldb, const double *beta, void *C, int ldc,
                         void *stream);

/* Products of the FP64 Rayleigh-Ritz solve (Cholesky updates, triangular
 * inverse, L^-1 A L^-H, Householder panel updates, back-transformation),
 * process-wide: mode 1 (default) runs the large ones with the FP64-accurate
 * tensor-core product of pw_zgemm_f64tc, mode 0 keeps every one on the FP64
 * pipe.  Results agree to FP64 rounding.  Errors: PW_ERR_ARG. */
pw_status pw_dense_products(int mode);

/* Captured CUDA graphs for the eigensolver of the Rayleigh-Ritz step (its
 * three stages: Householder tridiagonalisation, divide and conquer,
 * back-transformation), process-wide: with on = 1 (default) a stage whose
 * order and wanted-pair count repeat on the same workspace is captured once
 * and replayed (thousands of kernel launches per stage become one graph
 * launch); with 0 every launch is issued directly.  Graphs are used only on
 * streams other than the legacy default stream.  Results are the same.
 * Errors: PW_ERR_ARG. */
pw_status pw_dense_graphs(int on);

/* Householder reduction of the eigensolver (Syevd, Sec. III-D),
 * process-wide.  mode = 0 (default) chains three kernels per column with
 * programmatic dependent launch; while the product mode (pw_dense_products)
 * is 1, the Hermitian products A22 v of panels whose trailing order is at
 * least 1024 run on the FP16 tensor cores at FP64 accuracy (the panel's
 * trailing matrix split once into integer digit slices), the others on the
 * FP64 pipe.  mode = 2: the same chain with every Hermitian product on the
 * FP64 pipe.  mode = 1 (where the device supports cooperative launch): each
 * panel of 32 columns as one cooperative launch whose phases (column update,
 * Hermitian product on the FP64 pipe, row sums) are separated by grid-wide
 * barriers.  mode = 3: as mode 0, with each panel that uses the tensor-core
 * products run as one cooperative launch (one CTA per SM; column update,
 * tensor-core product, row sums separated by grid-wide barriers).
 * Cooperative launches are ordered one after another across streams.  All
 * modes give the same tridiagonal matrix to FP64 rounding.
 * Errors: PW_ERR_ARG. */
pw_status pw_householder_panels(int mode);

/* ---- Autotuner: the plan and tile-shape choices of the hot kernels ----
 * Sec. III-D picks, for each execution step, the process count that runs it
 * fastest among the candidates that fit in memory.  On one GPU the matching
 * choices are how a step's work is cut into kernel work units: the
 * factorisation of the FFT lines and the band batch of the local part of
 * H psi, and the K extent of the tensor-core GEMM tiles. */

/* A plan for the local part of H psi: register line FFTs with N = L R per
 * axis (L lanes, R values per lane), or L = R = 0 for the Stockham passes in
 * shared memory; compact = 1 keeps only the x-columns that meet the sphere
 * in shared memory (register plans only: smaller planes, e.g. the FP64 plane
 * at N = 128, more blocks per SM); batch_bytes: z-pencil bytes per batch of
 * bands (0: 64 MiB). */
typedef struct {
  int L, R;
  int compact;
  size_t batch_bytes;
} pw_fft_plan;

/* Register line-FFT plans compiled for grid size n: writes up to `max` of
 * them to `plans` (may be NULL) and returns how many exist (0: the grid size
 * runs on the Stockham passes only). */
int pw_fft_plans(int n, pw_fft_plan *plans, int max);

/* The cell's plan for one precision (PW_FP64, or PW_MIXED for its FP32
 * FFTs).  Set: L = R = 0 selects the Stockham passes.  Results agree to
 * rounding across plans.  Errors: PW_ERR_ARG (NULL, unknown precision, or an
 * (L, R, compact) that is not a plan for the cell's cubic grid, or whose
 * plane does not fit in shared memory in that precision). */
pw_status pw_cell_set_fft_plan(pw_cell *cell, int precision, const pw_fft_plan *plan);
pw_status pw_cell_get_fft_plan(const pw_cell *cell, int precision, pw_fft_plan *plan);

typedef struct {
  int ncand;            /* candidates timed */
  pw_fft_plan best;     /* the fastest, now set on the cell */
  pw_fft_plan dflt;     /* the default plan */
  double ms_best;       /* local part of H psi on nb bands with `best` (CUDA events, best of 3) */
  double ms_default;    /* the same with the default plan */
} pw_fft_tune_report;

/* Times the local part of H psi (FFT, V_loc, kinetic) on nb scratch bands
 * for every register plan that fits the cell's grid (full and compact plane)
 * and for the Stockham passes, each with z-pencil batches of 32, 64 and
 * 128 MiB, and sets the fastest on the cell for that precision.  Allocates and frees 2 npw nb
 * complex128 of scratch; synchronises `stream`.  Errors: PW_ERR_ARG (nb < 1,
 * precision), PW_ERR_OOM, PW_ERR_CUDA. */
pw_status pw_cell_autotune_fft(pw_cell *cell, int nb, int precision, void *stream,
                               pw_fft_tune_report *rep);
/* The candidates and times of the cell's last pw_cell_autotune_fft, one line
 * each ("L= R= compact= batch_mib= bands_per_batch= ms="), into buf (len
 * bytes, NUL-terminated, truncated); returns the full text length (0 if the
 * cell was never tuned). */
int pw_cell_fft_tune_log(const pw_cell *cell, char *buf, size_t len);

/* K split of the split-FP16 tensor-core GEMMs (tiles of 128 x 128 x K/s,
 * partial sums reduced in FP64 in a fixed order), process-wide:
 *   mode 0: s = 1 for every product (the default; clears the table);
 *   mode 1: each new product shape class (output tiles, K blocks rounded up
 *           to a power of two, K bounds, layout) with fewer than 608 output
 *           tiles is timed on its first call at s = 1, 2, 3, 4, 8, 16 (within
 *           limits: K >= 256 per part, partial sums <= 256 MiB) on
 *           a scratch output, and the fastest s is kept for the class (not
 *           under stream capture; that call synchronises its stream);
 *   mode 2: s = `split` wherever those limits allow it.
 * Results agree to rounding across splits.  Errors: PW_ERR_ARG. */
pw_status pw_autotune_gemm(int mode, int split);
/* The tuned shape classes as text, one line each ("mtiles= ntiles= k<= k_lo=
 * ... split= ms1= ms="), into buf (len bytes, NUL-terminated, truncated);
 * returns the number of shapes. */
int pw_autotune_gemm_table(char *buf, size_t len);
/* Adds shape classes in the text format of pw_autotune_gemm_table (a table
 * saved by an earlier process), so mode 1 uses them without timing again.
 * Returns the number of lines added, or -1 for a malformed line, in which
 * case nothing from `text` is added (the table is unchanged).  Host only: no
 * device work. */
int pw_autotune_gemm_load(const char *text);

/* Failure-detection self-test: one kernel waits, with the bounded wait of
 * the tensor-core GEMM pipeline and a limit of `cycles` SM clocks (1 ..
 * ~2e9), on a shared-memory barrier that nothing arrives on.  Returns
 * PW_ERR_TIMEOUT when the wait gave up and reported as designed (the
 * expected result; the context stays usable), PW_ERR_NUMERIC if it did not,
 * PW_ERR_ARG, PW_ERR_CUDA.  Synchronises `stream`. */
pw_status pw_selftest_bounded_wait(long long cycles, void *stream);

/* Number of CUDA kernel launches the library has issued in this process
 * (all devices, all threads); a diagnostic counter for launch accounting. */
uint64_t pw_kernel_launches(void);

void pw_destroy_cell(pw_cell *cell);
const char *pw_strerror(pw_status status);

#ifdef __cplusplus
}
#endif
#endif /* PW_H */
