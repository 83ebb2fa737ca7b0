// H psi = kinetic + local (FFT, fft_h.cu) + nonlocal Kleinman-Bylander term.
//
// Nonlocal term (Sec. III-A): the paper applies each atom's pseudopotential
// to every local wavefunction once it is fetched; on one GPU all atoms are
// resident, so the per-atom loop becomes two dense contractions over all
// projectors at once:  B = beta^H psi  (nproj x nb), B <- D o B,
// H psi += beta B.
#include <algorithm>

#include "oz_gemm.cuh"
#include "pw_internal.cuh"
#include "tc_gemm.cuh"

namespace {
__global__ void k_scale_rows(double2 *B, int nproj, int nb, const double *D) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)nproj * nb) return;
  const double d = D[idx % nproj];
  B[idx].x *= d;
  B[idx].y *= d;
}
}  // namespace

// the cell's workspace of the FP64-accurate tensor-core products (made on first use)
static pw_oz_ws *cell_oz(pw_cell *c) {
  if (!c->oz) c->oz = new pw_oz_ws();
  return c->oz;
}

// mixed precision: split-FP16 tensor-core products, FP64 accumulation into hpsi
static pw_status nonlocal_tc(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                             cudaStream_t st) {
  if (!c->op_beta_rows) {
    c->op_beta_rows = new pw_tc_operand();
    c->op_beta_t = new pw_tc_operand();
    c->op_psi = new pw_tc_operand();
    c->op_db = new pw_tc_operand();
    size_t cur = 0;
    PW_TRY(pw_ensure((void **)&c->d_tc_err, &cur, 16));
    cur = 0;
    PW_TRY(pw_ensure((void **)&c->d_rmax, &cur, (size_t)c->npw * sizeof(float)));
    PW_CUDA(cudaMemsetAsync(c->d_tc_err, 0, 16, st));
    PW_TRY(pw_tc_operand_alloc(c->op_beta_rows, 2 * c->nproj, 2 * c->npw, st));
    PW_TRY(pw_tc_operand_alloc(c->op_beta_t, c->npw, 2 * c->nproj, st));
    PW_TRY(pw_tc_split_rows(c->d_beta, c->npw, c->npw, c->nproj, 1, nullptr, c->op_beta_rows, st));
    PW_TRY(pw_tc_split_trans(c->d_beta, c->npw, c->npw, c->nproj, c->d_rmax, c->op_beta_t, st));
  }
  PW_TRY(pw_tc_operand_alloc(c->op_psi, nb, 2 * c->npw, st));
  PW_TRY(pw_tc_operand_alloc(c->op_db, 2 * nb, 2 * c->nproj, st));
  PW_TRY(pw_tc_split_rows(psi, ld, c->npw, nb, 0, nullptr, c->op_psi, st));
  // B = beta^H psi  (nproj x nb)
  PW_TRY(pw_tc_gemm(c->op_beta_rows, 2 * c->nproj, c->op_psi, nb, c->d_B, c->nproj, 0, 0, 0,
                    c->d_tc_err, st));
  // hpsi += beta (D o B)
  PW_TRY(pw_tc_split_coef(c->d_B, c->nproj, c->nproj, nb, c->d_D, c->op_db, st));
  return pw_tc_gemm(c->op_beta_t, c->npw, c->op_db, 2 * nb, hpsi, ld, 1, 1, 0, c->d_tc_err, st);
}

// Projectors generated on the fly into a bounded buffer instead of kept
// resident.  FP64: chunks of atoms, each adding beta_c (D_c o beta_c^H psi).
// Mixed: chunks of plane waves, so every tensor-core product keeps all
// projectors (B accumulated over chunks in FP64, then hpsi_c += beta_c (D B)).
constexpr size_t BCHUNK_BYTES = 256u << 20;
static pw_status nonlocal_onthefly(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                                   int precision, cudaStream_t st) {
  const int npw = c->npw;
  const int ca = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->natom,
                                                            BCHUNK_BYTES / ((size_t)npw * 4 * sizeof(double2))));
  const int npc = 4 * ca;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  if (precision == PW_MIXED) {
    // mixed: chunks of plane waves (every projector in each chunk keeps the
    // tensor-core products wide), beta generated in FP32 twice per call
    const int np = c->nproj;
    const int gc = (int)std::max<size_t>(64, std::min<size_t>((size_t)npw, BCHUNK_BYTES / ((size_t)np * sizeof(double2))));
    PW_TRY(pw_ensure((void **)&c->d_bchunk, &c->bchunk_bytes, (size_t)gc * np * sizeof(double2)));
    if (!c->op_bc_rows) {
      c->op_bc_rows = new pw_tc_operand();
      c->op_bc_t = new pw_tc_operand();
      c->op_psi_c = new pw_tc_operand();
      if (!c->op_db) c->op_db = new pw_tc_operand();
      size_t cur = 0;
      if (!c->d_tc_err) {
        PW_TRY(pw_ensure((void **)&c->d_tc_err, &cur, 16));
        PW_CUDA(cudaMemsetAsync(c->d_tc_err, 0, 16, st));
      }
      cur = 0;
      if (!c->d_rmax) PW_TRY(pw_ensure((void **)&c->d_rmax, &cur, (size_t)npw * sizeof(float)));
    }
    // B = sum over chunks of beta_c^H psi_c (FP64 accumulation)
    for (int g0 = 0; g0 < npw; g0 += gc) {
      const int ng = std::min(gc, npw - g0);
      PW_TRY(pw_beta_rows_f32(c, g0, ng, c->d_bchunk, st));
      PW_TRY(pw_tc_operand_alloc(c->op_bc_rows, 2 * np, 2 * ng, st));
      PW_TRY(pw_tc_operand_alloc(c->op_psi_c, nb, 2 * ng, st));
      PW_TRY(pw_tc_split_rows(c->d_bchunk, ng, ng, np, 1, nullptr, c->op_bc_rows, st));
      PW_TRY(pw_tc_split_rows(psi + g0, ld, ng, nb, 0, nullptr, c->op_psi_c, st));
      PW_TRY(pw_tc_gemm(c->op_bc_rows, 2 * np, c->op_psi_c, nb, c->d_B, np, 0, g0 > 0, 0, c->d_tc_err, st));
    }
    // hpsi_c += beta_c (D o B)
    PW_TRY(pw_tc_operand_alloc(c->op_db, 2 * nb, 2 * np, st));
    PW_TRY(pw_tc_split_coef(c->d_B, np, np, nb, c->d_D, c->op_db, st));
    for (int g0 = 0; g0 < npw; g0 += gc) {
      const int ng = std::min(gc, npw - g0);
      PW_TRY(pw_beta_rows_f32(c, g0, ng, c->d_bchunk, st));
      PW_TRY(pw_tc_operand_alloc(c->op_bc_t, ng, 2 * np, st));
      PW_TRY(pw_tc_split_trans(c->d_bchunk, ng, ng, np, c->d_rmax, c->op_bc_t, st));
      PW_TRY(pw_tc_gemm(c->op_bc_t, ng, c->op_db, 2 * nb, hpsi + g0, ld, 1, 1, 0, c->d_tc_err, st));
    }
    return PW_OK;
  }
  // FP64: chunks of atoms, beta generated in FP64 (the operator of the resident path)
  PW_TRY(pw_ensure((void **)&c->d_bchunk, &c->bchunk_bytes, (size_t)npw * npc * sizeof(double2)));
  {
    size_t ws = std::max(pw_zgemm_ws_elems(npc, nb, npw), pw_zgemm_ws_elems(npw, nb, npc));
    size_t wcur = c->gemm_ws_elems * sizeof(double2);
    PW_TRY(pw_ensure((void **)&c->d_gemm_ws, &wcur, ws * sizeof(double2)));
    c->gemm_ws_elems = wcur / sizeof(double2);
  }
  for (int a0 = 0; a0 < c->natom; a0 += ca) {
    const int na = std::min(ca, c->natom - a0), np = 4 * na;
    PW_TRY(pw_beta_chunk(c, a0, na, c->d_bchunk, st));
    PW_TRY(pw_gemm64(cell_oz(c), 'C', 'N', np, nb, npw, one, c->d_bchunk, npw, psi, ld, zero, c->d_B, np,
                     c->d_gemm_ws, c->gemm_ws_elems, st));
    pw_count_launch();
    k_scale_rows<<<(unsigned)(((long)np * nb + 255) / 256), 256, 0, st>>>(c->d_B, np, nb, c->d_D + 4 * a0);
    PW_TRY(pw_check_launch("scale_rows"));
    PW_TRY(pw_gemm64(cell_oz(c), 'N', 'N', npw, nb, np, one, c->d_bchunk, npw, c->d_B, np, one, hpsi, ld,
                     c->d_gemm_ws, c->gemm_ws_elems, st));
  }
  return PW_OK;
}

pw_status pw_apply_nonlocal(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                            int precision, cudaStream_t st) {
  if (c->nproj == 0 || nb == 0) return PW_OK;
  size_t need = (size_t)c->nproj * nb * sizeof(double2);
  size_t cur = c->B_elems * sizeof(double2);
  PW_TRY(pw_ensure((void **)&c->d_B, &cur, need));
  c->B_elems = cur / sizeof(double2);
  if (c->proj_onthefly) return nonlocal_onthefly(c, psi, ld, nb, hpsi, precision, st);
  if (precision == PW_MIXED) return nonlocal_tc(c, psi, ld, nb, hpsi, st);
  size_t ws = std::max(pw_zgemm_ws_elems(c->nproj, nb, c->npw), pw_zgemm_ws_elems(c->npw, nb, c->nproj));
  size_t wcur = c->gemm_ws_elems * sizeof(double2);
  PW_TRY(pw_ensure((void **)&c->d_gemm_ws, &wcur, ws * sizeof(double2)));
  c->gemm_ws_elems = wcur / sizeof(double2);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  PW_TRY(pw_gemm64(cell_oz(c), 'C', 'N', c->nproj, nb, c->npw, one, c->d_beta, c->npw, psi, ld, zero, c->d_B,
                   c->nproj, c->d_gemm_ws, c->gemm_ws_elems, st));
  pw_count_launch();
  k_scale_rows<<<(unsigned)(((long)c->nproj * nb + 255) / 256), 256, 0, st>>>(c->d_B, c->nproj, nb, c->d_D);
  PW_TRY(pw_check_launch("scale_rows"));
  return pw_gemm64(cell_oz(c), 'N', 'N', c->npw, nb, c->nproj, one, c->d_beta, c->npw, c->d_B, c->nproj, one,
                   hpsi, ld, c->d_gemm_ws, c->gemm_ws_elems, st);
}

// FP64 nonlocal term with caller-provided buffers: B (nproj x nb) and GEMM
// split-K partial sums (ws, ws_elems); no allocation
pw_status pw_apply_nonlocal_fp64_into(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                                      double2 *B, double2 *ws, size_t ws_elems, cudaStream_t st) {
  if (c->nproj == 0 || nb == 0) return PW_OK;
  if (!c->d_beta) return PW_ERR_ARG;   // projectors generated on the fly: not without allocation
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  PW_TRY(pw_zgemm('C', 'N', c->nproj, nb, c->npw, one, c->d_beta, c->npw, psi, ld, zero, B, c->nproj,
                  ws, ws_elems, st));
  pw_count_launch();
  k_scale_rows<<<(unsigned)(((long)c->nproj * nb + 255) / 256), 256, 0, st>>>(B, c->nproj, nb, c->d_D);
  PW_TRY(pw_check_launch("scale_rows"));
  return pw_zgemm('N', 'N', c->npw, nb, c->nproj, one, c->d_beta, c->npw, B, c->nproj, one, hpsi, ld,
                  ws, ws_elems, st);
}

extern "C" pw_status pw_apply_H(pw_cell *c, const void *psi, int ld, int nb, void *hpsi,
                                void *stream) {
  if (!c || nb < 0) return PW_ERR_ARG;
  if (nb == 0) return PW_OK;
  if (!psi || !hpsi || ld < c->npw) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  PW_TRY(pw_apply_local(c, (const double2 *)psi, ld, nb, (double2 *)hpsi, c->precision, st));
  return pw_apply_nonlocal(c, (const double2 *)psi, ld, nb, (double2 *)hpsi, c->precision, st);
}
