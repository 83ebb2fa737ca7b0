// Split-FP16 tcgen05 GEMM operands and entry points (mixed-precision path).
#pragma once
#include <cuda_fp16.h>

#include "pw_internal.cuh"

// An operand: two FP16 slices (hi, lo) of rows_total x kpad each (K-major,
// slice 1 follows slice 0), plus the inverse power-of-two scale of each row.
struct pw_tc_operand {
  __half *data = nullptr;
  float *inv_scale = nullptr;
  int rows_total = 0, kpad = 0;
  size_t cap_bytes = 0;
  int scale_cap = 0;
};

int pw_tc_kpad(int kreal);
// (re)allocates when larger; new storage is cleared on `st`
pw_status pw_tc_operand_alloc(pw_tc_operand *op, int rows, int kreal, cudaStream_t st);
void pw_tc_operand_free(pw_tc_operand *op);

// rows from the columns of X (npw x ncols): conj=0 -> ncols rows (re, im);
// conj=1 -> 2 ncols rows, pairs (re, im) / (-im, re).  colscale (device, optional)
// multiplies column c before splitting.
pw_status pw_tc_split_rows(const double2 *X, int ld, int npw, int ncols, int conj,
                           const double *colscale, pw_tc_operand *op, cudaStream_t st);
// rows g of X (npw rows), (re, im) over the ncols columns; rmax_ws: npw floats
pw_status pw_tc_split_trans(const double2 *X, int ld, int npw, int ncols, float *rmax_ws,
                            pw_tc_operand *op, cudaStream_t st);
// coefficient rows for A B products: rows 2j (re, -im), 2j+1 (im, re) over t < kdim;
// d (device, optional) scales entry t first
pw_status pw_tc_split_coef(const double2 *Cm, int ld, int kdim, int ncols, const double *d,
                           pw_tc_operand *op, cudaStream_t st);

// C (complex128, ld) from the m real rows of A and n real rows of B.
// mode 0 (rows pair re/im: A^H B products) or 1 (columns pair: A B products);
// accumulate: add to C; herm: compute the upper triangle only and mirror it.
// d_err: device int, OR-ed with a nonzero code if a bounded wait ran out.
// kb_lo: the first kb_lo 64-wide K blocks of B are zero (skipped); tri_b: B's
// rows come from an upper-triangular coefficient matrix (split_coef of M with
// M[t][j] = 0 for t > j), so an output tile of real columns n0.. stops at K
// block (n0 + 128) / 64.
pw_status pw_tc_gemm(const pw_tc_operand *A, int m, const pw_tc_operand *B, int n, double2 *C,
                     int ldc, int mode, int accumulate, int herm, int *d_err, cudaStream_t st,
                     int kb_lo = 0, int tri_b = 0);
