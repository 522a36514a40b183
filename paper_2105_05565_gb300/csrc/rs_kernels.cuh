// Launchers of the library's kernels (one translation unit per family).
#pragma once
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_common.cuh"

namespace rs {

// ---- sketch generation (rs_sketch_gen.cu) ----
int sample_cap(int64_t n, int64_t cnt);
// message returned by rs_last_error(NULL) (entry points without a context)
void set_global_error_msg(const char* msg);
// mode 0 subsample, 1 subcount (signs), 2 srht. k0_arg < 0: first slot is ctrl->k.
cudaError_t launch_gen_sample(cudaStream_t st, const Ctrl* ctrl, int64_t k0_arg, int nslots,
                              uint64_t seed, int64_t n, int64_t cnt, int mode, int64_t kk,
                              int64_t tau, int32_t* perm, int64_t perm_stride, int32_t* boff,
                              int64_t boff_stride, int32_t* err);
cudaError_t launch_gen_count(cudaStream_t st, const Ctrl* ctrl, int64_t k0_arg, int nslots,
                             uint64_t seed, int64_t m, int64_t tau, int32_t* perm,
                             int64_t perm_stride, int32_t* boff, int64_t boff_stride);
// Gaussian S of every slot, stored transposed: ST_s[j * ld + i] = S[i, j]
template <typename T>
cudaError_t launch_gen_gauss(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                             int64_t k0_arg, uint64_t seed, int64_t m, int64_t tau, T* ST,
                             int64_t ld, int64_t st_slot);

// ---- applying the sketch, phase 1 (rs_apply.cu) ----
struct PlanView {    // bucket-row representation of subsample / count / subcount (and SRHT's C)
  const int32_t* perm;  // packed (row | sign bit), grouped by bucket
  const int32_t* boff;  // tau + 1 bucket offsets
  int64_t perm_stride, boff_stride;  // per slot
};
// Where the tau "sketched rows" S^T A of a slot live: rows of A picked by the
// sample (subsample, no copy) or a materialised tau x ldsa buffer per slot;
// ST: transposed Gaussian sketch per slot (Gaussian only).
template <typename T>
struct RowsView {
  const T* A;
  int64_t lda;
  const T* SA;       // nullptr for subsample
  int64_t ldsa, sa_slot;
  const T* ST;       // Gaussian: tau x lda per slot, else nullptr
  int64_t st_slot;
  int64_t bq;        // 0: SA row-major (row stride ldsa); else blocked by bq-row slices
};
template <typename T>
cudaError_t launch_sa_batched(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              PlanView plan, const T* A, int64_t lda, int64_t m, int64_t tau, T* SA,
                              int64_t ldsa, int64_t sa_slot, int64_t bq = 0);
// S^T A and M = S^T A S of the bucket-row sketches in one launch (plan and kJB rows
// of S^T A in shared memory); sa_msys_fits says whether they fit
template <typename T>
bool sa_msys_fits(int64_t m, int64_t tau, int64_t nperm);
template <typename T>
cudaError_t launch_sa_msys(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, PlanView plan,
                           const T* A, int64_t lda, int64_t m, int64_t tau, T* SA, int64_t ldsa,
                           int64_t sa_slot, int64_t bq, double* M, int64_t m_slot,
                           float* Mf = nullptr);
template <typename T>
cudaError_t launch_msys_batched(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                                PlanView plan, RowsView<T> rows, int64_t m, int64_t tau,
                                double* M, int64_t m_slot, float* Mf = nullptr);

template <typename T>
cudaError_t launch_gauss_msys(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              const T* ST, int64_t st_slot, int64_t m, int64_t tau, const T* SA,
                              int64_t ldsa, int64_t sa_slot, double* M, int64_t m_slot,
                              int64_t lda);
template <typename T>
cudaError_t launch_gauss_system(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                                const T* ST, int64_t st_slot, const T* A, int64_t lda, int64_t m,
                                int64_t tau, T* SA, int64_t ldsa, int64_t sa_slot, double* M,
                                int64_t m_slot);
template <typename T>
cudaError_t launch_srht_system(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                               int64_t k0_arg, uint64_t seed, PlanView plan, const T* A,
                               int64_t lda, int64_t m, int64_t mp, int64_t tau, T* SA, int64_t ldsa,
                               int64_t sa_slot, double* M, int64_t m_slot);
int64_t srht_max_pad();

// ---- small SPD system (rs_chol.cu) ----
__host__ __device__ size_t factor_ws_elems(int64_t tau);
template <typename T>
cudaError_t launch_factor_inv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              const double* M, int64_t m_slot, int64_t tau, T* Linv, int64_t l_slot,
                              T* ws, int32_t* ndropped);
// P = M^+ (and, if Linv != nullptr, the zeroed L^{-1}) per slot; ws holds
// potri_ws_elems(tau) elements per slot
__host__ __device__ size_t potri_ws_elems(int64_t tau);
bool potri_needs_ws(int64_t tau, size_t elem);  // false: the tiles fit shared memory
template <typename T, typename TP>
cudaError_t launch_potri(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, const double* M,
                         int64_t m_slot, int64_t tau, T* Linv, int64_t l_slot, TP* P, int64_t pld,
                         int64_t p_slot, T* ws, int32_t* ndropped);
// one problem of a batched small solve: its M per slot, the stored P (type TP of the
// launch) per slot, its drop counter and control block (active slots)
struct PotriJob {
  const double* M;
  int64_t m_slot, tau;
  void* P;
  int64_t pld, p_slot;
  int32_t* ndropped;
  const Ctrl* ctrl;
};
// M^+ of every active slot of the running problems order[0..nrun) of jobs, chunk slots
// each, in one launch; ws holds potri_batch_ctas() x potri_ws_elems(tau_max) elements
int potri_batch_ctas();
template <typename T, typename TP>
cudaError_t launch_potri_batch(cudaStream_t st, const PotriJob* jobs, const int32_t* order,
                               int nrun, int chunk, int64_t tau_max, T* ws);
template <typename T>
struct DeltaArgs {
  int kind;            // 0 bucket rows (subsample, count, subcount), 1 Gaussian, 2 SRHT
  PlanView plan;
  const T* ST; int64_t st_slot, ld;
  uint64_t seed; int64_t mp;
  const double* r; int64_t m, tau;
  const T* Linv; int64_t l_slot;
  double* rS_out;      // may be nullptr
  double* delta_out;
  double* u;           // dense S delta (bucket rows, SRHT)
};
template <typename T>
cudaError_t launch_delta(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                         DeltaArgs<T> g);

// ---- fused iterations of a chunk on a thread-block cluster (rs_iterate.cu) ----
template <typename T, typename TF>
struct IterArgs {
  int kind;            // 0 bucket rows (subsample, count, subcount), 1 Gaussian
  int mixed;           // 1: convergence sets `pending` (FP64 check follows)
  const T* A; int64_t lda;
  const T* SA; int64_t sa_slot;   // sketched rows per slot (nullptr for subsample)
  const T* ST;                    // Gaussian: S^T per slot (stride sa_slot)
  PlanView plan;
  const int32_t* inv; int64_t inv_slot;  // row -> bucket | sign (bucket-row sketches)
  const TF* Linv; int64_t l_slot;
  const double* gam; const double* bet;
  double* w; double* wp; double* r; double* rp;
  double* hist; double* delta_out; double* rS_out;
  int64_t m, tau, chunk;
  int64_t sub_end;  // iterations run while k < k0 + sub_end (sub_end <= chunk)
  int stage;           // set by the launcher: r and the plan staged in shared memory
};
template <typename T, typename TF>
cudaError_t launch_iterate(cudaStream_t st, Ctrl* ctrl, IterArgs<T, TF> g);
// inverse map of the sketch plans: inv[i] = bucket | sign bit, or 0x7FFFFFFF when row i
// is not in the sketch (all_rows = 1: every row is, as in the count sketch)
cudaError_t launch_inv_map(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, PlanView plan,
                           int64_t m, int64_t tau, int all_rows, int32_t* inv, int64_t inv_slot);

// ---- persistent iterations of a chunk over the whole GPU (rs_iterate_wide.cu) ----
// Bucket-row sketches (subsample, count, subcount). Each CTA owns a slice of q rows
// of the m-vectors; delta = M^+ S^T r is assembled from per-CTA partials through a
// deterministic all-reduce (tagged partial words in global memory, then the
// cluster's shared memory).
template <typename T, typename TF>
struct WideArgs {
  int mixed;                       // 1: convergence sets `pending` (FP64 check follows)
  const T* rows;                   // S^T A of slot 0, blocked: CTA c's tau x round_up(q, 4)
                                   // block at c * tau * round_up(q, 4)
  int64_t sa_slot;                 // slot stride of S^T A
  const int32_t* inv; int64_t inv_slot;      // row -> bucket | sign, kNotSketched
  const TF* P; int64_t pld, p_slot;          // M^+ per slot, tau x pld
  const double* gam; const double* bet;
  double* w; double* wp; double* r; double* rp;
  double* hist; double* delta_out;
  uint64_t* part;                  // 2 x nblk x (tau + 1) x 2 tagged words of partials
  uint64_t* epoch;                 // launch counter of the tags
  int32_t* abort_word;             // set by a CTA whose bounded wait ran out
  int64_t m, tau, chunk, q;
  int64_t sub_end;  // iterations run while k < k0 + sub_end (sub_end <= chunk)
  uint64_t wait_ns;  // bound of every device-side wait (global timer)
  int64_t stall_ns;  // fault injection: CTA 0 publishes its first partials this late
  double* wsum;      // nullptr, or the running sum of the iterates w^0..w^k (m)
  int accel;         // 1: Algorithm 3 with (w, v, r_w, r_v) in (w, w_prev, r, r_prev)
  double acc_a, acc_b, acc_g;  // its alpha, beta, gamma
  int nblk;
  int nsab;                        // buffers of the staged S^T A block (2, or 1 when tight)
};
struct WidePlan {
  int nblk;       // CTAs (a multiple of the cluster size)
  int64_t q;      // rows per CTA (a multiple of 4)
  size_t smem;    // dynamic shared memory per CTA
  int nsab;       // S^T A staging buffers
};
// false when the slice buffers do not fit shared memory (the cluster kernel is used)
template <typename T, typename TF>
bool wide_plan(int64_t m, int64_t tau, int max_ctas, int64_t chunk, WidePlan* out);
template <typename T, typename TF>
cudaError_t launch_iterate_wide(cudaStream_t st, Ctrl* ctrl, const WideArgs<T, TF>& g, size_t smem);
// CTAs per cluster of the persistent iteration kernel, a non-portable size: each
// CTA of a cluster gathers a sixteenth of the all-reduced entries from global memory
// and scatters them to its 15 peers through distributed shared memory (16 measured
// 4 % faster per iteration than 8 at m = 4096, tau = 256)
constexpr int kWideCluster = 16;
// P_s = M_s^+ in FP32 by symmetric sweeps, without the triangular factor (tau <= 256)
cudaError_t launch_sweep_inv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                             const float* M, int64_t m_slot, int64_t tau, float* P, int64_t pld,
                             int64_t p_slot, int32_t* ndropped);
constexpr int64_t kSweepMaxTau = 256;
// P_s = L_s^{-T} L_s^{-1} (full, row stride pld) for every active slot
template <typename TF>
cudaError_t launch_pinv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, const TF* Linv,
                        int64_t l_slot, int64_t tau, TF* P, int64_t pld, int64_t p_slot);

// ---- matrix-free sparse X (rs_sparse.cu) ----
constexpr int kPiece = 1024;  // column entries summed by one warp in X^T v
template <typename VT>
struct SparseX {
  int64_t n, d, nnz;
  const int64_t* rowptr; const int32_t* colidx; const VT* val;  // CSR (rows ascending)
  const int64_t* colptr; const int32_t* rowidx; const VT* cval; // CSC (rows ascending)
  const int32_t* pcol; const int64_t* pstart; int64_t npieces;  // pieces of <= kPiece entries
  const int32_t* cpiece;                                        // d + 1: pieces of column c
};
// per-slot XS of a chunk (compact rows that meet the sampled columns) and its scans
struct MfArgs {
  int64_t n, d, tau;
  const int64_t* rowptr; const int32_t* colidx;
  const int32_t* inv; int64_t inv_slot;        // column -> bucket | sign per slot
  int32_t* bsum; int32_t* boffs;               // per slot: nrb x 2 block counts / offsets
  int32_t* tot;                                // per slot: entries E, compact rows R
  int32_t* crow; int32_t* cptr; int32_t* ebuck;  // rows (rcap), offsets (rcap + 1), buckets (ecap)
  int64_t nrb, rcap, ecap;
  double lambda;
};
int64_t mf_row_blocks(int64_t n);
// *err = 1 when the CSR arrays are inconsistent (read-only bounds check)
cudaError_t launch_csr_check(cudaStream_t st, const int64_t* rowptr, int64_t n,
                             const int32_t* colidx, int64_t nnz, int64_t d, int32_t* err);
template <typename VT>
cudaError_t build_csc(cudaStream_t st, const int64_t* rowptr, int64_t n, const int32_t* colidx,
                      const VT* val, int64_t nnz, int64_t d, int32_t* table, int nb,
                      int64_t* colcnt, int64_t* colptr, int32_t* rowidx, VT* cval);
// out = X^T v (FP64, column pieces; pu: npieces doubles); z = X x (FP64)
template <typename VT>
cudaError_t sparse_xtv_d(cudaStream_t st, const SparseX<VT>& X, const double* v, double* out,
                         double* pu, const int32_t* stop);
template <typename VT>
cudaError_t sparse_xv_d(cudaStream_t st, const SparseX<VT>& X, const double* x, double* z,
                        const int32_t* stop);
template <typename VT, typename AT>
cudaError_t launch_mf_phase1(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, MfArgs a,
                             const VT* val, AT* eval, PlanView plan, double* M, int64_t m_slot);
struct UpdateArgs;
template <typename VT, typename AT>
cudaError_t launch_mf_iteration(cudaStream_t st, Ctrl* ctrl, MfArgs a, const SparseX<VT>& X,
                                const AT* eval, PlanView plan, const AT* P, int64_t pld,
                                int64_t p_slot, AT* v, AT* pu, UpdateArgs u, double* rS_out);

// ---- many problems, several right-hand sides each (rs_batch.cu) ----
struct BatchPairs {        // per (problem, right-hand side)
  int32_t* flag;           // 0 active, 1 pending (FP64 check due), 2 converged, 3 failed
  int32_t* skip;           // 1: no refresh (converged or failed)
  int64_t* iters;          // iterations done
  double* r0;              // ||b||
  double* resid;           // last relative residual
};
struct BatchRef {          // state of one pair (plain FP64)
  int64_t d; int pair; double lambda;
  double* w; double* wp; const double* b; double* r; double* rp;
};
struct BatchRefM {        // state of one pair (mixed)
  int64_t d; int pair; double lambda;
  float2* w2; float2* r2; float* dw; float* dr;   // the pair's state
  double* wd; const double* v; const double* b;   // w in FP64, X^T X w, b
};
// what: 0 init state and r0, 1 w -> FP64 (active pairs), 2 w -> FP64 (all), 3 refresh
cudaError_t launch_batch_mixed_aux(cudaStream_t st, int what, const BatchRefM* refs, int npairs,
                                   BatchPairs pairs, const double* tol);
cudaError_t launch_batch_init(cudaStream_t st, const BatchRef* refs, int npairs, BatchPairs pairs);

// one cluster of kBatchCluster CTAs per problem (rs_batch_cluster.cu)
constexpr int kBatchCluster = 8;
template <typename T>
struct BatchProbC {
  int64_t d, tau, bq, sa_slot, pld, p_slot, perm_stride, boff_stride, inv_slot;
  const T* SA;                                    // per slot: tau x bq slices, one per CTA
  const T* P;                                     // per slot: M^+ (tau x pld)
  const int32_t* perm; const int32_t* boff; const int32_t* inv;  // per slot: plan, row map
  T *w, *wp, *r, *rp;                             // plain: nrhs x d each
  float2 *w2, *r2;                                // mixed: nrhs x d float pairs
  float *dw, *dr;                                 // mixed: last increments
  Ctrl* ctrl;
};
// tau_max, bq_max, perm_max, pld_max: maxima over the problems of tau, bq, the plan's
// perm_stride and the row stride of M^+ (they size the shared memory)
template <typename T, bool kMixed>
cudaError_t launch_batch_cluster(cudaStream_t st, const BatchProbC<T>* probs, const int32_t* order,
                                 int nprob, int nrhs, BatchPairs pairs, const double* gam,
                                 const double* bet, int64_t chunk, const double* tol,
                                 int64_t tau_max, int64_t bq_max, int64_t perm_max, int64_t pld_max,
                                 int threads, int32_t* err_word);
template <typename T, bool kMixed>
int batch_cluster_fit(int nrhs, int64_t tau_max, int64_t bq_max, int64_t perm_max, int64_t pld_max,
                      int threads);

cudaError_t launch_batch_finish(cudaStream_t st, Ctrl* const* ctrls, int P, int nrhs,
                                BatchPairs pairs, int32_t* alive, int32_t* out);

// ---- learned sketch proposal (rs_learned.cu) ----
constexpr int kMlpParams = 4545;  // W1 64x4, b1, W2 64x64, b2, w3, b3
// raw: 2 m floats of work space; zstat: 2 m standardised static features
template <typename T>
cudaError_t launch_lp_static(cudaStream_t st, const T* A, int64_t lda, int64_t m, float* raw,
                             float* zstat);
// plans of the chunk's slots drawn from the proposal (w null: uniform); stats: 5
// doubles, score: m floats of work space; last: last visit per row (updated when
// update_age)
cudaError_t launch_collect_pre(cudaStream_t st, Ctrl* ctrl, const double* w, const double* wstar,
                               const double* r, int64_t m, double tol, double* e2_out);
cudaError_t launch_collect_rows(cudaStream_t st, const Ctrl* ctrl, const int32_t* perm,
                                const int32_t* boff, int64_t tau, const float* feat,
                                const double* rS, const double* delta, const double* e2,
                                int64_t m, int64_t cap, float* Z, float* y, int64_t* count);
template <typename T>
cudaError_t launch_lp_diag_score(cudaStream_t st, const T* A, int64_t lda, int64_t m,
                                 float* score);
cudaError_t launch_lp_plans(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, int64_t k0_arg,
                            uint64_t seed, const uint16_t* w, float eps, const float* zstat,
                            float* dyn, double* stats, const double* r, int32_t* last, int64_t m,
                            int64_t tau, float* score, int32_t* perm, int64_t perm_stride,
                            int32_t* boff, int64_t boff_stride, bool update_age,
                            bool fixed_score);
// the m x 4 feature rows at iteration k0 (the network's inputs); dyn: 2 m floats
cudaError_t launch_lp_features(cudaStream_t st, const Ctrl* ctrl, int64_t k0, const float* zstat,
                               float* dyn, double* stats, const double* r, const int32_t* last,
                               int64_t m, float* score, float* feat_out);
cudaError_t launch_mlp_forward(cudaStream_t st, const uint16_t* w, const float* Z, int64_t n,
                               float* s_out);
int mlp_grad_blocks(int64_t n);
// part: mlp_grad_blocks(n) x kMlpParams floats, loss_part: mlp_grad_blocks(n) floats
cudaError_t launch_mlp_grad(cudaStream_t st, const float* theta, const float* Z, const float* y,
                            int64_t n, float* part, float* loss_part, float* grad, double* loss);
cudaError_t launch_mlp_adam(cudaStream_t st, float* theta, float* mom, float* vel, const float* grad,
                            int64_t step, float lr, float b1, float b2, float eps, uint16_t* w_bf16);
cudaError_t launch_f32_to_bf16(cudaStream_t st, const float* x, int64_t n, uint16_t* out);

// ---- iterate / residual update (rs_update.cu) ----
struct UpdateArgs {
  const double* gam;  // gamma_k table
  const double* bet;  // beta_k table
  double* w; double* wp; double* r; double* rp;
  double* u;          // dense S delta (reset to 0 after use); unused with rows.ST
  const double* delta;
  double* partials;   // per-block partial ||r||^2
  double* hist;       // hist[k + 1] written by the last block
  int mixed;          // 1: convergence sets `pending` instead of `stop`
};
template <typename T>
cudaError_t launch_update(cudaStream_t st, Ctrl* ctrl, PlanView plan, RowsView<T> rows,
                          int64_t m, int64_t tau, UpdateArgs a);
int update_blocks(int64_t m);
// w = w_prev = u = 0, r = r_prev = -b
cudaError_t launch_init_state(cudaStream_t st, int64_t m, const double* b, double* w, double* wp,
                              double* r, double* rp, double* u);
// ctrl->k0 = ctrl->k (first iteration of a chunk)
cudaError_t launch_chunk_begin(cudaStream_t st, Ctrl* ctrl, const double* hist = nullptr);
cudaError_t launch_scale(cudaStream_t st, const double* in, double s, int64_t m, double* out);
cudaError_t launch_cast_f64_f32(cudaStream_t st, const double* in, int64_t n, float* out);
// raise (never lower) a kernel's maximum dynamic shared memory on the current device
cudaError_t set_smem_max(const void* func, size_t bytes);

// ---- Conjugate Gradients (rs_cg.cu) ----
struct CgScal {
  double rr;        // r . r of the current residual
  double pv;        // p . A p of the current direction
  double beta;      // coefficient of the next direction update
  uint32_t ticket;  // last-block counter of the grid reductions
  int32_t pad;
};
int cg_blocks(int64_t m);
int cg_matvec_blocks(int64_t m);
cudaError_t launch_cg_dir(cudaStream_t st, const Ctrl* ctrl, const CgScal* cs, int64_t m,
                          const double* r, double* p, float2* p2);
template <typename TA>
cudaError_t launch_cg_matvec(cudaStream_t st, const Ctrl* ctrl, const TA* A, int64_t lda, int64_t m,
                             const double* p, const float2* p2, double* v, CgScal* cs,
                             double* part);
cudaError_t launch_cg_lam_dot(cudaStream_t st, const Ctrl* ctrl, int64_t m, double lambda,
                              const double* p, double* v, CgScal* cs, double* part);
cudaError_t launch_cg_update(cudaStream_t st, Ctrl* ctrl, CgScal* cs, int64_t m, const double* p,
                             const double* v, double* w, double* r, double* part, double* hist,
                             int mixed);
cudaError_t launch_cg_rr(cudaStream_t st, const Ctrl* ctrl, CgScal* cs, int64_t m, const double* r,
                         int init);

// ---- X^T X on the tensor cores (rs_tc_gemm.cu) ----
// A (lower triangle and diagonal, d x lda FP32) = X^T X + lambda I, TF32 inputs, FP32
// accumulation; Xt_ws: gram_tc_ws_floats(n, d) floats; err set on a device timeout
size_t gram_tc_ws_floats(int64_t n, int64_t d);
// the part of rows [r0, r1) of X (r0 a multiple of 32; r1 too, or r1 = n): stored with
// lambda I for r0 = 0, added to A otherwise (row ranges of an upload in pieces)
cudaError_t launch_gram_tc_rows(cudaStream_t st, const float* X, int64_t n, int64_t d,
                                double lambda, float* A, int64_t lda, float* Xt_ws, int32_t* err,
                                int64_t r0, int64_t r1, float* Xcopy = nullptr);
// (Xcopy != nullptr: X is also copied there, row-major, from the same read)
// kernel ridge: the Gaussian kernel matrix on the tensor cores (FP32) or in FP64, and
// A = K^T K + lambda I turned into K^T (K + lambda I)
cudaError_t launch_gauss_sa_tc(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                               const float* ST, int64_t ld, int64_t m, int64_t tau,
                               const float* A, int64_t lda, float* SA, int32_t* err);
size_t rbf_tc_ws_floats(int64_t n, int64_t d);
cudaError_t launch_rbf_tc(cudaStream_t st, const float* P, int64_t n, int64_t d, double sigma,
                          float* K, int64_t ldK, float* ws, int32_t* err);
template <typename TP>
cudaError_t launch_rbf_f64(cudaStream_t st, const TP* P, int64_t n, int64_t d, double sigma,
                           double* K, int64_t ldK);
template <typename T>
cudaError_t launch_add_offdiag(cudaStream_t st, T* A, int64_t lda, const T* K, int64_t ldK,
                               int64_t n, double lambda);
cudaError_t launch_gram_tc(cudaStream_t st, const float* X, int64_t n, int64_t d, double lambda,
                           float* A, int64_t lda, float* Xt_ws, int32_t* err,
                           float* Xcopy = nullptr);
template <typename T>
cudaError_t launch_mirror_lower(cudaStream_t st, T* A, int64_t m, int64_t lda);

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
// the same for FP32 X in float-pair arithmetic (relative error about 1e-12; part as
// for launch_xt_v)
cudaError_t launch_xt_v_pairs(cudaStream_t st, const float* X, int64_t n, int64_t d,
                              const double* v, double* out, double* part,
                              const int32_t* stop = nullptr);
// its three steps, for row ranges of X: the float pairs of v, the sums of the 512-row
// blocks of rows [r0, r1) (r0 a multiple of 512), the sum of all blocks into out
cudaError_t xt_pairs_split(cudaStream_t st, const double* v, int64_t n, int64_t d, double* part,
                           const int32_t* stop = nullptr);
cudaError_t xt_pairs_rows(cudaStream_t st, const float* X, int64_t n, int64_t d, double* part,
                          int64_t r0, int64_t r1, const int32_t* stop = nullptr);
cudaError_t xt_pairs_sum(cudaStream_t st, int64_t n, int64_t d, double* part, double* out,
                         const int32_t* stop = nullptr);
// out[i] = sum_j X[i, j] v[j] (i < n), FP64 accumulate
template <typename TI>
cudaError_t launch_x_v(cudaStream_t st, const TI* X, int64_t n, int64_t d, const double* v,
                       double* out, const int32_t* stop = nullptr);
// out = X^T (X v) for FP32 X in one pass, FP64-accurate (float pairs); d <= 4096;
// part: xtx_df_blocks() * d doubles
cudaError_t launch_xtx_v_df(cudaStream_t st, const float* X, int64_t n, int64_t d, const double* v,
                            double* out, double* part, const int32_t* stop = nullptr);
int xtx_df_blocks();
// out[q] = X^T X V[q] for nv <= 4 vectors (nv x d, vector-major) in one pass over X,
// d <= 4096; part holds xtx_multi_blocks() x nv x d doubles; vectors flagged in skip
// (nv entries) are not written, and nothing runs when all are flagged
cudaError_t launch_xtx_multi_df(cudaStream_t st, const float* X, int64_t n, int64_t d, int nv,
                                const double* V, double* out, double* part, const int32_t* skip);
int xtx_multi_blocks();
// the same product in two passes (U = X W with a warp per row, then X^T U with a thread
// per column): U holds n x 4 float pairs, part xtx_two_pass_part(n, d, nv) doubles
cudaError_t launch_xtx_two_pass(cudaStream_t st, const float* X, int64_t n, int64_t d, int nv,
                                const double* W, double* out, float2* U, double* part,
                                const int32_t* skip);
int64_t xtx_two_pass_part(int64_t n, int64_t d, int nv);
// r_true = v + lambda x - b; replaces (r, rp) keeping r - rp, writes hist[k] and the
// convergence decision (mode 1) or only the relative residual (mode 0 -> *rel_out)
cudaError_t launch_refresh_finish(cudaStream_t st, Ctrl* ctrl, int mode, int64_t m,
                                  const double* v, const double* x, const double* b,
                                  double lambda, double* r, double* rp, double* partials,
                                  double* hist, double* rel_out);

}  // namespace rs
