// FP64-accurate complex GEMM on the FP16 tensor cores (integer-slice split of
// both operands, exact slice products, 64-bit fixed-point accumulation).
#pragma once
#include "pw_internal.cuh"

#define PW_OZ_SLICES 8
// slice bytes of one block of a product; larger products run in blocks of
// rows, columns or K
#define PW_OZ_SLICE_CAP ((size_t)2 << 30)

// Workspace of the product (grown on demand, owned by the caller's object).
struct pw_oz_ws {
  void *buf = nullptr;        // operand slices and row exponents
  size_t bytes = 0;
  double2 *part = nullptr;    // K-split partial results
  size_t part_bytes = 0;
  int *err = nullptr;         // device error word (a bounded wait ran out)
  unsigned gen = 0;           // bumped whenever buf or part is reallocated
};

// C = alpha op(A) op(B) + beta C, column-major complex128, op in {N, C};
// herm as pw_zgemm_ex (0 plain, 1 Hermitian upper + mirror, 2 tiles with
// j/64 <= i/64 only, 3 op(A) upper triangular, 4 op(B) lower triangular,
// 5 op(A) lower triangular).  Error per entry <= 11K 2^-55 max_k|op(A)_ik|
// max_k|op(B)_kj|.  Asynchronous on st.
pw_status pw_zgemm_oz(pw_oz_ws *w, char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                      int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc, cudaStream_t st,
                      int herm);
// C = A B for real column-major A (m x k, lda), B (k x n, ldb), C (m x n,
// ldc): the same slice arithmetic on real rows (A's rows strided, B's
// columns contiguous), error per entry <= 5.5K 2^-55 max_k|a_ik| max_k|b_kj|.
// Asynchronous on st.
pw_status pw_dgemm_oz(pw_oz_ws *w, int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                      double *C, int ldc, cudaStream_t st);
// Dispatch of an FP64 product: the tensor-core path when the process-wide
// mode (pw_dense_products) is 1, w is given and the product has at least
// ~8M complex multiply-adds; else the FP64 pipe (pw_zgemm_ex with ws).
pw_status pw_gemm64(pw_oz_ws *w, char opA, char opB, int m, int n, int k, double2 alpha, const double2 *A,
                    int lda, const double2 *B, int ldb, double2 beta, double2 *C, int ldc, double2 *ws,
                    size_t ws_elems, cudaStream_t st, int herm = 0);
bool pw_use_oz(int m, int n, int k);
int pw_f64_products_mode();
// device bytes of the slices of an m x n x k product (without K-split parts)
size_t pw_oz_ws_bytes(int m, int n, int k);
// PW_ERR_TIMEOUT if a bounded wait of an earlier product ran out (synchronises st)
pw_status pw_oz_check(pw_oz_ws *w, cudaStream_t st);
void pw_oz_free(pw_oz_ws *w);
