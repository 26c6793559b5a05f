// Create-time device work of the single-LP solver (pdlp_setup.cu): the row
// starts of K' and the stable transpose, Sec. 2.2 scaling, the scaled vectors and
// scalars, and small tables.  Separate from pdlp_internal.cuh, which holds
// what the step and check kernels share.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pdlp {

// Fills the Algorithm 2 exponent-factor table: pw[k] = (k + 2)^-0.3 and
// pw[count + k] = (k + 2)^-0.6 for k < count (the same pow() the step test calls).
cudaError_t setup_pow_table(double *pw, long long count, cudaStream_t s);
// Row starts of K' on the device: T_ptr (n + 1) = exclusive
// scan of K's column counts; work[0] = the largest column count; work holds
// col_starts_work_ints(n) ints.
cudaError_t setup_col_starts(int32_t n, int64_t nnz, const int32_t *K_idx, int32_t *T_ptr, int32_t *work,
                             cudaStream_t s);
size_t col_starts_work_ints(int32_t n);
// K' on the device (pdlp_setup.cu), given its row starts T_ptr (already on
// the device): the stable transpose, equal to the host counting sort, for
// columns of at most transpose_max_segment() entries, with
// transpose_work_ints(n, nnz) ints of scratch, which it leaves holding the
// transpose permutation at work + n and the row of every entry of K at
// work + n + nnz.
cudaError_t setup_transpose(int32_t m, int32_t n, int64_t nnz, const int32_t *K_ptr, const int32_t *K_idx,
                            const double *K_val, const int32_t *T_ptr, int32_t *T_idx, double *T_val, int32_t *work,
                            cudaStream_t s);
size_t transpose_work_ints(int32_t n, int64_t nnz);
int transpose_max_segment();

// Sec. 2.2 scaling of K and K' in place (row-wise passes over both).
cudaError_t setup_scale(int32_t m, int32_t n, int64_t nnz, int32_t *K_ptr, int32_t *K_idx, double *K_val,
                        int32_t *T_ptr, int32_t *T_idx, double *T_val, double *D1, double *D2, double *work_m,
                        double *work_n, int ruiz_iters, double pc_alpha, cudaStream_t s);
// The same scaling, bitwise equal, given the row of every entry of K
// (rowid) and the transpose permutation (perm: K' position -> K entry), as
// setup_transpose leaves them in its scratch: the Ruiz maxima come from one
// pass over K's entries (atomic maxima on the IEEE bits), only K's values
// are divided, and K''s values are copied through perm.
cudaError_t setup_scale_perm(int32_t m, int32_t n, int64_t nnz, const int32_t *K_ptr, const int32_t *K_idx,
                             double *K_val, const int32_t *T_ptr, double *T_val, const int32_t *rowid,
                             const int32_t *perm, double *D1, double *D2, double *work_m, double *work_n,
                             double *rcp_m, double *rcp_n, int ruiz_iters, double pc_alpha, cudaStream_t s);
cudaError_t setup_vectors(int32_t m, int32_t n, const double *c0, const double *q0, const double *l0,
                          const double *u0, const double *D1, const double *D2, double *c, double *q, double *l,
                          double *u, cudaStream_t s);
cudaError_t setup_f32(int64_t nnz, const double *val, float *val32, cudaStream_t s);
// rD = 1 / D elementwise (the infeasibility pieces unscale with products)
cudaError_t setup_recip(int32_t count, const double *D, double *rD, cudaStream_t s);
// out[0] = sum (c~)^2, out[1] = sum (q~)^2, out[2] = max |K~|, with
// scalars_work_doubles() doubles of scratch
cudaError_t setup_scalars(int32_t m, int32_t n, int64_t nnz, const double *c, const double *q, const double *val,
                          double *out, double *work, cudaStream_t s);
size_t scalars_work_doubles();
cudaError_t setup_warm(int32_t m, int32_t n, const double *x0, const double *y0, const double *D1,
                       const double *D2, double *x, double *y, cudaStream_t s);

// Sliced-ELL copy of a CSR matrix (layout from sell_layout, pdlp_sell.h):
// inv[perm[r]] = r; then every stored entry is set to column -1 / value 0
// and internal row r's entries (original row perm[r], columns renumbered
// through inv) are written from base[r], 32 apart when lane[r] is 1.
cudaError_t setup_invert(int32_t rows, const int32_t *perm, int32_t *inv, cudaStream_t s);
cudaError_t setup_sell_fill(int32_t rows, int64_t total, const int32_t *perm, const int32_t *base,
                            const uint8_t *lane, const int32_t *ptr, const int32_t *idx, const double *val,
                            const int32_t *inv, int32_t *sidx, double *sval, cudaStream_t s);
// Debug check of a sliced-ELL copy (rows internal rows, column indices of
// the other side in [0, cols)): counts[0] stored entries with a column
// outside [-1, cols) or padding (column -1) with a nonzero value, counts[1]
// work items outside the storage or malformed, counts[2] rows that the items
// do not cover exactly once; waits for the result.
cudaError_t setup_check_sell(int32_t rows, int32_t cols, int64_t total, int32_t nitems, const int4 *items,
                             const int32_t *sidx, const double *sval, const float *sval32, unsigned int counts[3],
                             cudaStream_t s);
// Entries of a CSR matrix on the device: *first = the first nonzero whose
// column lies outside [0, n) or whose value is not finite (nnz if none),
// *col_bad = 1 when that entry's column is the fault; waits for the result.
cudaError_t setup_check_entries(int64_t nnz, const int32_t *idx, const double *val, int32_t n, int64_t *first,
                                int *col_bad, cudaStream_t s);
// QP extension: qd[j] = D2[j] q0[perm_c[j]] D2[j] (scaled Hessian diagonal,
// internal order; q0 in the original order).
cudaError_t setup_qp_diag(int32_t n, const int32_t *perm_c, const double *D2, const double *q0, double *qd,
                          cudaStream_t s);
// dst[r] = src[perm[r]] for r < count (original order -> internal order)
cudaError_t setup_permute(int32_t count, const int32_t *perm, const double *src, double *dst, cudaStream_t s);
// Warm start in the internal order: x[j] = x0[perm_c[j]] / D2[j] (0 without
// x0), y[i] = y0[perm_r[i]] / D1[i], with D1, D2 in the internal order.
cudaError_t setup_warm_perm(int32_t m, int32_t n, const double *x0, const double *y0, const int32_t *perm_r,
                            const int32_t *perm_c, const double *D1, const double *D2, double *x, double *y,
                            cudaStream_t s);

}  // namespace pdlp
