// Launchers of the library's kernels (one translation unit per family).
#pragma once
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_common.cuh"

namespace rs {

// ---- sketch generation (rs_sketch_gen.cu) ----
int sample_cap(int64_t n, int64_t cnt);
// mode 0 subsample, 1 subcount (signs), 2 srht. k0_arg < 0: first slot is ctrl->k.
cudaError_t launch_gen_sample(cudaStream_t st, const Ctrl* ctrl, int64_t k0_arg, int nslots,
                              uint64_t seed, int64_t n, int64_t cnt, int mode, int64_t kk,
                              int64_t tau, int32_t* perm, int64_t perm_stride, int32_t* boff,
                              int64_t boff_stride, int32_t* err);
cudaError_t launch_gen_count(cudaStream_t st, const Ctrl* ctrl, int64_t k0_arg, int nslots,
                             uint64_t seed, int64_t m, int64_t tau, int32_t* perm,
                             int64_t perm_stride, int32_t* boff, int64_t boff_stride);
template <typename T>
cudaError_t launch_gen_gauss(cudaStream_t st, const Ctrl* ctrl, int64_t k_arg, uint64_t seed,
                             int64_t m, int64_t tau, T* S);

// ---- applying the sketch (rs_apply.cu) ----
// Where the tau "sketched rows" S^T A live: rows of A picked by the sample
// (subsample, no copy) or a materialised tau x ld buffer.
template <typename T>
struct RowsView {
  const T* A;        // A, row-major, leading dimension lda
  int64_t lda;
  const T* SA;       // materialised S^T A (tau x ldsa) or nullptr (subsample)
  int64_t ldsa;
};
struct PlanView {    // bucket-row representation of subsample / count / subcount
  const int32_t* perm;  // packed (row | sign bit), grouped by bucket
  const int32_t* boff;  // tau + 1 bucket offsets
  int64_t perm_stride, boff_stride;  // per slot
};
// SA[j, :] = sum_{t in bucket j} sign_t A[row_t, :]   (count, subcount)
template <typename T>
cudaError_t launch_sa_rows(cudaStream_t st, const Ctrl* ctrl, int force, PlanView plan,
                           const T* A, int64_t lda, int64_t m, int64_t tau, T* SA, int64_t ldsa);
// M = S^T A S (tau x tau, FP64 out) and r_S = S^T r for the bucket-row sketches
template <typename T>
cudaError_t launch_msys_rows(cudaStream_t st, const Ctrl* ctrl, int force, PlanView plan,
                             RowsView<T> rows, int64_t m, int64_t tau, const double* r,
                             double* M, double* rS);
// Gaussian: SA = S^T A, M = SA S, r_S = S^T r; u = S delta
template <typename T>
cudaError_t launch_gauss_sa(cudaStream_t st, const Ctrl* ctrl, int force, const T* S, const T* A,
                            int64_t lda, int64_t m, int64_t tau, T* SA, int64_t ldsa);
template <typename T>
cudaError_t launch_gauss_msys(cudaStream_t st, const Ctrl* ctrl, int force, const T* S,
                              const T* SA, int64_t ldsa, int64_t m, int64_t tau, const double* r,
                              double* M, double* rS);
template <typename T>
cudaError_t launch_gauss_u(cudaStream_t st, const Ctrl* ctrl, int force, const T* S, int64_t m,
                           int64_t tau, const double* delta, double* u);
// SRHT (m' = 2^ceil(log2 m)): SA, M, r_S, u through fast Walsh-Hadamard transforms
template <typename T>
cudaError_t launch_srht_sa(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                           uint64_t seed, PlanView C, const T* A, int64_t lda, int64_t m,
                           int64_t mp, int64_t tau, T* SA, int64_t ldsa);
template <typename T>
cudaError_t launch_srht_msys(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                             uint64_t seed, PlanView C, const T* SA, int64_t ldsa, int64_t m,
                             int64_t mp, int64_t tau, const double* r, double* M, double* rS);
cudaError_t launch_srht_u(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                          uint64_t seed, PlanView C, int64_t m, int64_t mp, int64_t tau,
                          const double* delta, double* u);
int64_t srht_max_pad(int elem_bytes);

// ---- small SPD solve (rs_chol.cu) ----
// delta = least-norm solution of M delta = r_S by Cholesky with the pivot rule:
// a pivot below tau * eps * max_i M_ii drops its index (delta_j = 0). When perm /
// boff are given, also scatters u[row_t] = sign_t delta_j over bucket j.
template <typename T>
cudaError_t launch_chol_solve(cudaStream_t st, const Ctrl* ctrl, int force, const double* M,
                              const double* rS, int64_t tau, T* gscratch, double* delta,
                              PlanView plan, double* u, int32_t* ndropped);
template <typename T>
size_t chol_scratch_elems(int64_t tau);

// ---- iterate / residual update (rs_update.cu) ----
struct UpdateArgs {
  const double* gam;  // gamma_k table
  const double* bet;  // beta_k table
  double* w; double* wp; double* r; double* rp;
  double* u;          // dense S delta (reset to 0 after use)
  const double* delta;
  double* partials;   // per-block partial ||r||^2
  double* hist;       // hist[k + 1] written by the last block
  int mixed;          // 1: convergence sets `pending` instead of `stop`
};
template <typename T>
cudaError_t launch_update(cudaStream_t st, Ctrl* ctrl, PlanView plan, RowsView<T> rows,
                          int64_t m, int64_t tau, UpdateArgs a);
int update_blocks(int64_t m);
// w = w_prev = u = 0, r = r_prev = -b, hist[0] = (||b|| > 0)
cudaError_t launch_init_state(cudaStream_t st, int64_t m, const double* b, double* w, double* wp,
                              double* r, double* rp, double* u);
// ctrl->k0 = ctrl->k (first iteration of a chunk)
cudaError_t launch_chunk_begin(cudaStream_t st, Ctrl* ctrl);

// ---- forming A, b; true residuals through X (rs_form.cu) ----
// C (m x ldc) = op(X) op(X)^T + lambda I, primal op(X) = X^T (m = d), dual X (m = n)
template <typename TI, typename TO>
cudaError_t launch_form_A(cudaStream_t st, const TI* X, int64_t n, int64_t d, int dual,
                          double lambda, TO* A, int64_t lda);
// out[j] = sum_i X[i, j] v[i] (j < d), FP64 accumulate; part: scratch of
// ceil(n / rows_per_chunk) * d doubles (xt_part_elems)
// (stop: when non-null and *stop != 0 at run time the kernels do nothing)
template <typename TI>
cudaError_t launch_xt_v(cudaStream_t st, const TI* X, int64_t n, int64_t d, const double* v,
                        double* out, double* part, const int32_t* stop = nullptr);
size_t xt_part_elems(int64_t n, int64_t d);
// out[i] = sum_j X[i, j] v[j] (i < n), FP64 accumulate
template <typename TI>
cudaError_t launch_x_v(cudaStream_t st, const TI* X, int64_t n, int64_t d, const double* v,
                       double* out, const int32_t* stop = nullptr);
// r_true = v + lambda x - b; replaces (r, rp) keeping r - rp, writes hist[k] and the
// convergence decision (mode 1) or only the relative residual (mode 0 -> *rel_out)
cudaError_t launch_refresh_finish(cudaStream_t st, Ctrl* ctrl, int mode, int64_t m,
                                  const double* v, const double* x, const double* b,
                                  double lambda, double* r, double* rp, double* partials,
                                  double* hist, double* rel_out);

}  // namespace rs
