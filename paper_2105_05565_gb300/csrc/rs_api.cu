// C ABI of the solver (include/ridgesketch.h): context, buffers, the chunked
// device-side iteration loop (one CUDA graph replay per chunk) and parity hooks.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "ridgesketch.h"
#include "rs_kernels.cuh"

using namespace rs;

namespace {

std::mutex g_err_mu;
std::string g_err;

void set_global_error(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = s;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

constexpr int64_t kLdAlign = 128;     // row length padding of m-long rows (elements)
constexpr int kChunksPerGraph = 4;    // chunks of iterations captured in one CUDA graph
constexpr int64_t kMixedChunk = 600;   // default slots per chunk in mixed precision (two waves of two CTAs per SM in the FP64 factor)
constexpr int64_t kMaxSample = 8192;  // largest ordered sample drawn by one CTA
constexpr int64_t kMaxCountTau = 2048;

int64_t pow2_ceil(int64_t m) {
  int64_t p = 1;
  while (p < m) p <<= 1;
  return p;
}

int64_t default_tau(int64_t m) {  // smallest t with t^3 >= m^2
  int64_t t = (int64_t)llround(std::pow((double)m, 2.0 / 3.0));
  if (t < 1) t = 1;
  auto ge = [&](int64_t x) { return (long double)x * x * x >= (long double)m * m; };
  while (!ge(t)) ++t;
  while (t > 1 && ge(t - 1)) --t;
  return t;
}

}  // namespace

namespace rs {
void set_global_error_msg(const char* msg) { set_global_error(msg ? msg : ""); }
}  // namespace rs

namespace {
// set while rs_create_batch creates its member contexts: M^+ per slot is kept for the
// batch's iteration kernel (the persistent single-problem kernel is not used)
thread_local bool t_batch_member = false;
}  // namespace

struct rs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // problem
  int form = 0, sketch = 0, precision = 0, chol_fp64 = 1, refresh_every = 400;
  int64_t n = 0, d = 0, m = 0, tau = 0, s = 0, kk = 0, mp = 0, ld = 0, chunk = 64;
  double lambda = 0.0;
  uint64_t seed = 0;
  rs_mom mom{};
  int xdtype = RS_F64;
  bool xtx_df = true;      // one-pass float-pair X^T X v for FP32 X (primal)
  // device data
  void* X = nullptr;
  double* y = nullptr;
  void* A = nullptr;     // m x ld, double (plain) or float (mixed)
  double* b = nullptr;
  double *w = nullptr, *wp = nullptr, *r = nullptr, *rp = nullptr, *u = nullptr;
  void* SA = nullptr;    // per slot: tau x ld
  void* ST = nullptr;    // gaussian, per slot: tau x ld (S transposed)
  double* M = nullptr;   // per slot: tau x tau (FP64)
  void* Linv = nullptr;  // per slot: tau x tau inverse Cholesky factor (factor precision)
  void* fws = nullptr;   // factor workspace when the factor does not fit shared memory
  double *rS = nullptr, *delta = nullptr;
  int64_t sa_slot = 0, m_slot = 0, l_slot = 0;
  int64_t bq = 0;             // S^T A blocked by slices of bq rows of the iterate (0: row-major)
  // learned proposal of the subsample rows (rs_set_proposal)
  bool learned = false;
  bool lp_uniform = false;     // no network: p_j = 1 / m
  bool lp_fixed = false;       // scores fixed once (importance sampling, rs_set_sampling)
  float lp_eps = 0.1f;
  uint16_t* lp_w = nullptr;    // network weights, bfloat16
  float* lp_raw = nullptr;     // 2 m work space (raw static, then the dynamic features)
  float* lp_zstat = nullptr;   // 2 m standardised static features
  double* lp_stats = nullptr;  // 8
  float* lp_score = nullptr;   // m scores
  float* lp_feat = nullptr;    // m x 4 features (rs_proposal_features)
  int32_t* lp_last = nullptr;  // last iteration whose sample held the row (-1: never)
  int32_t *perm = nullptr, *boff = nullptr;
  int32_t* inv = nullptr;  // per slot (stride ld): row -> bucket | sign (bucket-row sketches)
  // persistent iteration kernel over the whole GPU (bucket-row sketches)
  bool use_wide = false;
  WidePlan wide{};
  void* Pm = nullptr;       // per slot: M^+ = L^{-T} L^{-1}, tau x pld (factor precision)
  int32_t* tc_err = nullptr;  // a tensor-core GEMM of phase 1 gave up a bounded wait
  void* pws = nullptr;      // per slot: tile workspace of k_potri when the tiles pass shared memory
  bool potri = false;       // M^+ by the one-kernel factor, inverse and product
  bool sweep_p = false;     // M^+ by FP32 sweeps from an FP32 M (mixed, FP32 factor)
  bool batch_member = false;  // a problem of an rs_batch (S^T A and M^+ kept per slot)
  float* Mf = nullptr;      // per slot: M in FP32 for the sweeps
  int64_t pld = 0, p_slot = 0;
  uint64_t* xpart = nullptr;   // all-reduce partials, 2 x nblk x (tau + 1) x 2 tagged words
  uint64_t* xflags = nullptr;  // launch counter of the tags
  int32_t* xabort = nullptr;
  uint64_t wait_ns = 2000000000ull;  // bound of the persistent kernel's waits
  int64_t stall_ns = 0;              // fault injection (tests)
  // Conjugate Gradients on the same system (rs_solve_cg)
  double *cg_p = nullptr, *cg_v = nullptr, *cg_part = nullptr;
  float2* cg_p2 = nullptr;  // p as float pairs (mixed, dense A)
  CgScal* cg_s = nullptr;
  cudaGraphExec_t cg_graph = nullptr;
  bool kernel = false;               // kernel ridge: X holds K, A = K^T (K + lambda I)
  bool accel = false;                // Algorithm 3 (rs_set_acceleration)
  double acc_a = 0.5, acc_b = 0.0, acc_g = 1.0;
  bool avg = false;                  // keep the running sum of the iterates (rs_set_averaging)
  double* wsum = nullptr;            // m: sum of w^0..w^k of the current solve
  int64_t last_iters = 0;            // iterations of the last rs_solve
  // matrix-free sparse X (CSR input)
  bool sparse = false;
  int64_t nnz = 0;
  int64_t* sx_rowptr = nullptr; int32_t* sx_colidx = nullptr; void* sx_val = nullptr;
  int64_t* sx_colptr = nullptr; int32_t* sx_rowidx = nullptr; void* sx_cval = nullptr;
  int32_t* sx_pcol = nullptr; int64_t* sx_pstart = nullptr; int32_t* sx_cpiece = nullptr;
  int64_t sx_npieces = 0;
  int32_t *mf_bsum = nullptr, *mf_boffs = nullptr, *mf_tot = nullptr, *mf_crow = nullptr,
          *mf_cptr = nullptr, *mf_ebuck = nullptr;
  void* mf_eval = nullptr;   // per slot: ecap entries (FP32 mixed, FP64 plain)
  void* mf_v = nullptr;      // n: (XS) delta (FP32 mixed, FP64 plain)
  void* mf_pu = nullptr;     // pieces of X^T v, same type
  double* mf_pud = nullptr;  // pieces of the FP64 products
  double* mf_z = nullptr;    // n: X w for the FP64 refresh
  int64_t mf_nrb = 0, mf_rcap = 0, mf_ecap = 0;
  int64_t perm_stride = 0, boff_stride = 0;
  int64_t nslots = 0;
  int32_t* err_flag = nullptr;
  int32_t* ndropped = nullptr;
  double *gam = nullptr, *bet = nullptr;
  int64_t sched_len = 0;
  double* hist = nullptr;
  int64_t hist_len = 0;
  double* partials = nullptr;
  int64_t npartials = 0;
  double *vn = nullptr, *vd = nullptr, *xt_part = nullptr, *rel_dev = nullptr;
  Ctrl* ctrl = nullptr;
  Ctrl* ctrl_h = nullptr;  // pinned
  double* scal_h = nullptr;  // pinned scalar
  double r0 = 0.0;
  // graph of one chunk
  cudaGraphExec_t graph = nullptr;
  bool graph_refresh = false;
  // timing
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double setup_ms = 0.0, solve_ms = 0.0;
  std::string err;

  bool mixed() const { return precision == RS_MIXED; }
  size_t elem() const { return mixed() ? sizeof(float) : sizeof(double); }
  bool f64_factor() const { return !mixed() || chol_fp64 == 1; }
  // CG in mixed precision with dense A: the FP32 A needs the FP64 refresh through X
  bool cg_refresh() const { return mixed() && !sparse; }
};

#define CKC(ctx, call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
      return (e_ == cudaErrorMemoryAllocation) ? RS_ENOMEM : RS_ECUDA;                       \
    }                                                                                       \
  } while (0)

#define FAILC(ctx, code, msg)   \
  do {                          \
    (ctx)->err = (msg);         \
    return (code);              \
  } while (0)

namespace {

// ---- device memory of the contexts ----
// One stream-ordered pool per device that keeps the blocks its contexts free
// (release threshold: unlimited), so creating and destroying a context costs no
// cudaMalloc / cudaFree (and no device-wide synchronisation) once the pool holds
// the sizes; rs_trim_memory returns the unused blocks to the driver. Every access
// to a context's memory is ordered on the context's stream.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaError_t ctx_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool[dev] == nullptr) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

// " (device memory: F GiB free of T GiB)" for out-of-memory messages
std::string mem_note() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return std::string();
  }
  char buf[96];
  std::snprintf(buf, sizeof(buf), " (device memory: %.1f GiB free of %.1f GiB)",
                (double)fr / (1 << 30), (double)tot / (1 << 30));
  return std::string(buf);
}

cudaError_t pmalloc(rs_ctx* c, void** p, size_t bytes) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = ctx_pool(c->device, &pool);
  if (e != cudaSuccess) return e;
  e = cudaMallocFromPoolAsync(p, bytes, pool, c->stream);
  if (e == cudaErrorMemoryAllocation) {
    // out of device memory: let the stream-ordered frees of every context on this
    // device complete (the pool is shared, and a block whose free is still pending
    // is not released by a trim), give the pool's unused blocks back, try once more
    cudaGetLastError();
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone)
      cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, pool, c->stream);
  }
  return e;
}
void pfree(rs_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}
// a blocking copy ordered after the work already on the context's stream
cudaError_t copy_sync(rs_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

template <typename T>
rs_status dalloc(rs_ctx* c, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  CKC(c, pmalloc(c, (void**)p, n * sizeof(T)));
  return RS_OK;
}

void free_all(rs_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cg_graph) cudaGraphExecDestroy(c->cg_graph);
  void* ptrs[] = {c->X, c->y, c->A, c->b, c->w, c->wp, c->r, c->rp, c->u, c->SA, c->ST, c->M,
                  c->Linv, c->fws, c->pws, c->rS, c->delta, c->perm, c->boff, c->inv, c->err_flag,
                  c->ndropped,
                  c->gam, c->bet, c->hist, c->partials, c->vn, c->vd, c->xt_part, c->rel_dev,
                  c->ctrl, c->Pm, c->xpart, c->xflags, c->xabort, c->Mf,
                  c->sx_rowptr, c->sx_colidx, c->sx_val, c->sx_colptr, c->sx_rowidx, c->sx_cval,
                  c->sx_pcol, c->sx_pstart, c->sx_cpiece, c->mf_bsum, c->mf_boffs, c->mf_tot,
                  c->mf_crow, c->mf_cptr, c->mf_ebuck, c->mf_eval, c->mf_v, c->mf_pu, c->mf_pud,
                  c->mf_z, c->lp_w, c->lp_raw, c->lp_zstat, c->lp_stats, c->lp_score, c->lp_feat,
                  c->lp_last, c->wsum, c->cg_p, c->cg_v, c->cg_part, c->cg_s, c->cg_p2,
                  c->tc_err};
  for (void* p : ptrs) pfree(c, p);
  if (c->ctrl_h) {  // the stream may still read the pinned control block
    cudaStreamSynchronize(c->stream);
    cudaFreeHost(c->ctrl_h);
  }
  if (c->scal_h) cudaFreeHost(c->scal_h);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

PlanView plan_view(const rs_ctx* c) {
  PlanView p{};
  if (c->sketch == RS_GAUSSIAN) return p;
  p.perm = c->perm;
  p.boff = (c->sketch == RS_SRHT) ? nullptr : c->boff;
  p.perm_stride = c->perm_stride;
  p.boff_stride = c->boff_stride;
  return p;
}

template <typename T>
RowsView<T> rows_view(const rs_ctx* c) {
  RowsView<T> v{};
  v.A = static_cast<const T*>(c->A);
  v.lda = c->ld;
  v.SA = (c->sketch == RS_SUBSAMPLE && !c->use_wide && !c->batch_member) ? nullptr : static_cast<const T*>(c->SA);
  v.ldsa = c->ld;
  v.sa_slot = c->sa_slot;
  v.ST = (c->sketch == RS_GAUSSIAN) ? static_cast<const T*>(c->ST) : nullptr;
  v.st_slot = c->sa_slot;
  v.bq = c->bq;
  return v;
}

// ---- matrix-free sparse X ----
template <typename VT>
SparseX<VT> sparse_view(const rs_ctx* c) {
  SparseX<VT> X{};
  X.n = c->n; X.d = c->d; X.nnz = c->nnz;
  X.rowptr = c->sx_rowptr; X.colidx = c->sx_colidx; X.val = static_cast<const VT*>(c->sx_val);
  X.colptr = c->sx_colptr; X.rowidx = c->sx_rowidx; X.cval = static_cast<const VT*>(c->sx_cval);
  X.pcol = c->sx_pcol; X.pstart = c->sx_pstart; X.npieces = c->sx_npieces;
  X.cpiece = c->sx_cpiece;
  return X;
}

MfArgs mf_args(const rs_ctx* c) {
  MfArgs a{};
  a.n = c->n; a.d = c->d; a.tau = c->tau;
  a.rowptr = c->sx_rowptr; a.colidx = c->sx_colidx;
  a.inv = c->inv; a.inv_slot = c->ld;
  a.bsum = c->mf_bsum; a.boffs = c->mf_boffs; a.tot = c->mf_tot;
  a.crow = c->mf_crow; a.cptr = c->mf_cptr; a.ebuck = c->mf_ebuck;
  a.nrb = c->mf_nrb; a.rcap = c->mf_rcap; a.ecap = c->mf_ecap;
  a.lambda = c->lambda;
  return a;
}

// calls f(tag) with a null pointer of the sparse value type
template <typename F>
rs_status with_vt(const rs_ctx* c, F&& f) {
  if (c->xdtype == RS_F64) return f(static_cast<double*>(nullptr));
  if (c->xdtype == RS_F32) return f(static_cast<float*>(nullptr));
  return f(static_cast<__nv_bfloat16*>(nullptr));
}

// sketch plan of `nslots` consecutive iterations starting at k0_arg (< 0: ctrl->k)
rs_status enqueue_gen(rs_ctx* c, int64_t k0_arg, int nslots) {
  cudaStream_t st = c->stream;
  if (c->learned) {  // rows drawn from the learned proposal (the chunk's plans at once)
    CKC(c, launch_lp_plans(st, c->ctrl, k0_arg >= 0 ? 1 : 0, nslots, k0_arg, c->seed,
                           c->lp_uniform ? nullptr : c->lp_w, c->lp_eps, c->lp_zstat, c->lp_raw,
                           c->lp_stats, c->r, c->lp_last, c->m, c->tau, c->lp_score, c->perm,
                           c->perm_stride, c->boff, c->boff_stride, k0_arg < 0 && !c->lp_fixed,
                           c->lp_fixed));
    return RS_OK;
  }
  switch (c->sketch) {
    case RS_SUBSAMPLE:
      CKC(c, launch_gen_sample(st, c->ctrl, k0_arg, nslots, c->seed, c->m, c->tau, 0, 1, c->tau,
                               c->perm, c->perm_stride, c->boff, c->boff_stride, c->err_flag));
      break;
    case RS_SUBCOUNT:
      CKC(c, launch_gen_sample(st, c->ctrl, k0_arg, nslots, c->seed, c->m, c->s, 1, c->kk, c->tau,
                               c->perm, c->perm_stride, c->boff, c->boff_stride, c->err_flag));
      break;
    case RS_SRHT:
      CKC(c, launch_gen_sample(st, c->ctrl, k0_arg, nslots, c->seed, c->mp, c->tau, 2, 1, c->tau,
                               c->perm, c->perm_stride, nullptr, 0, c->err_flag));
      break;
    case RS_COUNT:
      CKC(c, launch_gen_count(st, c->ctrl, k0_arg, nslots, c->seed, c->m, c->tau, c->perm,
                              c->perm_stride, c->boff, c->boff_stride));
      break;
    default:
      break;
  }
  return RS_OK;
}

// Phase 1 of a chunk (independent of the iterate): sketch plans, S^T A, M = S^T A S
// and the inverse Cholesky factor of M for `nslots` consecutive iterations. force = 1
// (parity hooks) runs every slot starting at iteration k0_arg; force = 0 starts at
// ctrl->k0 and skips slots the solve will not reach.
// stages of phase 1 (a chunk's profile times them apart): the sketch plans, the
// sketched rows (with M where one pass forms both), M from the sketched rows, and
// the small systems' inverses
constexpr int kP1Plan = 1, kP1Rows = 2, kP1Msys = 4, kP1Inv = 8, kP1All = 15;

// M^+ of every slot in one kernel: FP64 or FP32 arithmetic (the factor's), stored in
// the iteration kernel's type (FP32 in mixed precision: FP64 factor and inverse,
// rounded once to FP32 for the FP32 iterations)
rs_status enqueue_potri(rs_ctx* c, cudaStream_t st, int force, int nslots) {
  double* M = c->M;
  if (c->f64_factor() && c->mixed() && (c->sparse || c->batch_member || c->use_wide))
    CKC(c, (launch_potri<double, float>(st, c->ctrl, force, nslots, M, c->m_slot, c->tau, nullptr,
                                        c->l_slot, static_cast<float*>(c->Pm), c->pld, c->p_slot,
                                        static_cast<double*>(c->pws), c->ndropped)));
  else if (c->f64_factor())
    CKC(c, (launch_potri<double, double>(st, c->ctrl, force, nslots, M, c->m_slot, c->tau, nullptr,
                                         c->l_slot, static_cast<double*>(c->Pm), c->pld, c->p_slot,
                                         static_cast<double*>(c->pws), c->ndropped)));
  else
    CKC(c, (launch_potri<float, float>(st, c->ctrl, force, nslots, M, c->m_slot, c->tau, nullptr,
                                       c->l_slot, static_cast<float*>(c->Pm), c->pld, c->p_slot,
                                       static_cast<float*>(c->pws), c->ndropped)));
  return RS_OK;
}

template <typename T>
rs_status enqueue_phase1_t(rs_ctx* c, int force, int64_t k0_arg, int nslots, bool want_p,
                           int stages = kP1All) {
  cudaStream_t st = c->stream;
  rs_status s;
  const PlanView plan = plan_view(c);
  if (stages & kP1Plan) {
    if ((s = enqueue_gen(c, force ? k0_arg : -1, nslots)) != RS_OK) return s;
    if (c->inv != nullptr)
      CKC(c, launch_inv_map(st, c->ctrl, force, nslots, plan, c->m, c->tau,
                            c->sketch == RS_COUNT ? 1 : 0, c->inv, c->ld));
  }
  const T* A = static_cast<const T*>(c->A);
  T* SA = static_cast<T*>(c->SA);
  if (!(stages & (kP1Rows | kP1Msys))) {
  } else if (c->sparse) {  // XS and M = S^T X^T X S + lambda S^T S without A
    s = with_vt(c, [&](auto tag) -> rs_status {
      using VT = std::remove_pointer_t<decltype(tag)>;
      CKC(c, (launch_mf_phase1<VT, T>(st, c->ctrl, force, nslots, mf_args(c),
                                      static_cast<const VT*>(c->sx_val), static_cast<T*>(c->mf_eval),
                                      plan, c->M, c->m_slot)));
      return RS_OK;
    });
    if (s != RS_OK) return s;
  } else
  switch (c->sketch) {
    case RS_SUBSAMPLE:
    case RS_COUNT:
    case RS_SUBCOUNT:
      if (c->sketch == RS_SUBSAMPLE && !c->use_wide && !c->batch_member) {  // M = A[C, C] gathered
        CKC(c, launch_msys_batched<T>(st, c->ctrl, force, nslots, plan, rows_view<T>(c), c->m,
                                      c->tau, c->M, c->m_slot));
        break;
      }
      if (!(stages & kP1Rows)) break;  // (here M is formed with S^T A)
      if (sa_msys_fits<T>(c->m, c->tau, c->perm_stride)) {  // S^T A and M in one pass
        CKC(c, launch_sa_msys<T>(st, c->ctrl, force, nslots, plan, A, c->ld, c->m, c->tau, SA, c->ld,
                                 c->sa_slot, c->bq, c->M, c->m_slot,
                                 (want_p && c->sweep_p) ? c->Mf : nullptr));
        break;
      }
      CKC(c, launch_sa_batched<T>(st, c->ctrl, force, nslots, plan, A, c->ld, c->m, c->tau, SA,
                                  c->ld, c->sa_slot, c->bq));
      CKC(c, launch_msys_batched<T>(st, c->ctrl, force, nslots, plan, rows_view<T>(c), c->m, c->tau,
                                    c->M, c->m_slot, (want_p && c->sweep_p) ? c->Mf : nullptr));
      break;
    case RS_GAUSSIAN: {
      T* ST = static_cast<T*>(c->ST);
      CKC(c, launch_gen_gauss<T>(st, c->ctrl, force, nslots, k0_arg, c->seed, c->m, c->tau, ST,
                                 c->ld, c->sa_slot));
      if constexpr (sizeof(T) == 4) {
        if (c->tc_err != nullptr && c->sa_slot == c->tau * c->ld) {
          // S^T A of all slots as one TF32 tensor-core product, then M = S^T A S
          CKC(c, launch_gauss_sa_tc(st, c->ctrl, force, nslots, ST, c->ld, c->m, c->tau, A, c->ld,
                                    SA, c->tc_err));
          CKC(c, launch_gauss_msys<T>(st, c->ctrl, force, nslots, ST, c->sa_slot, c->m, c->tau,
                                      SA, c->ld, c->sa_slot, c->M, c->m_slot, c->ld));
          break;
        }
      }
      CKC(c, launch_gauss_system<T>(st, c->ctrl, force, nslots, ST, c->sa_slot, A, c->ld, c->m,
                                    c->tau, SA, c->ld, c->sa_slot, c->M, c->m_slot));
      break;
    }
    case RS_SRHT:
      CKC(c, launch_srht_system<T>(st, c->ctrl, force, nslots, k0_arg, c->seed, plan, A, c->ld, c->m,
                                   c->mp, c->tau, SA, c->ld, c->sa_slot, c->M, c->m_slot));
      break;
  }
  if (!(stages & kP1Inv)) return RS_OK;
  if (want_p && c->sweep_p) {
    // FP32 M^+ directly (symmetric sweeps), no triangular factor
    CKC(c, launch_sweep_inv(st, c->ctrl, force, nslots, c->Mf, c->m_slot, c->tau,
                            static_cast<float*>(c->Pm), c->pld, c->p_slot, c->ndropped));
    return RS_OK;
  }
  if (want_p && c->potri) return enqueue_potri(c, st, force, nslots);
  if (c->f64_factor())
    CKC(c, launch_factor_inv<double>(st, c->ctrl, force, nslots, c->M, c->m_slot, c->tau,
                                     static_cast<double*>(c->Linv), c->l_slot,
                                     static_cast<double*>(c->fws), c->ndropped));
  else
    CKC(c, launch_factor_inv<float>(st, c->ctrl, force, nslots, c->M, c->m_slot, c->tau,
                                    static_cast<float*>(c->Linv), c->l_slot,
                                    static_cast<float*>(c->fws), c->ndropped));
  if (want_p) {
    if (c->f64_factor())
      CKC(c, launch_pinv<double>(st, c->ctrl, force, nslots, static_cast<const double*>(c->Linv),
                                 c->l_slot, c->tau, static_cast<double*>(c->Pm), c->pld, c->p_slot));
    else
      CKC(c, launch_pinv<float>(st, c->ctrl, force, nslots, static_cast<const float*>(c->Linv),
                                c->l_slot, c->tau, static_cast<float*>(c->Pm), c->pld, c->p_slot));
  }
  return RS_OK;
}

// want_p: also M^+ per slot, for the persistent iteration kernel
rs_status enqueue_phase1(rs_ctx* c, int force, int64_t k0_arg, int nslots, bool want_p = false,
                         int stages = kP1All) {
  return c->mixed() ? enqueue_phase1_t<float>(c, force, k0_arg, nslots, want_p, stages)
                    : enqueue_phase1_t<double>(c, force, k0_arg, nslots, want_p, stages);
}

template <typename TF, typename T>
DeltaArgs<TF> delta_args(rs_ctx* c) {
  DeltaArgs<TF> g{};
  g.kind = c->sketch == RS_GAUSSIAN ? 1 : (c->sketch == RS_SRHT ? 2 : 0);
  g.plan = plan_view(c);
  g.ST = nullptr;
  g.st_slot = c->sa_slot;
  g.ld = c->ld;
  g.seed = c->seed;
  g.mp = c->mp;
  g.r = c->r;
  g.m = c->m;
  g.tau = c->tau;
  g.Linv = static_cast<const TF*>(c->Linv);
  g.l_slot = c->l_slot;
  g.rS_out = c->rS;
  g.delta_out = c->delta;
  g.u = c->u;
  return g;
}

// the sketched residual r_S = S^T r, delta = L^{-T} L^{-1} r_S and u = S delta of
// the current (force = 0) or given (force = 1, slot 0) iteration
rs_status enqueue_delta(rs_ctx* c, int force, int64_t k_arg) {
  cudaStream_t st = c->stream;
  if (c->f64_factor()) {
    DeltaArgs<double> g = delta_args<double, double>(c);
    if (c->sketch == RS_GAUSSIAN) {
      if (c->mixed()) return (c->err = "rs: Gaussian sketch with an FP64 factor needs FP64 S in the mixed form", RS_EUNSUPPORTED);
      g.ST = static_cast<const double*>(c->ST);
    }
    CKC(c, launch_delta<double>(st, c->ctrl, force, k_arg, g));
  } else {
    DeltaArgs<float> g = delta_args<float, float>(c);
    if (c->sketch == RS_GAUSSIAN) g.ST = static_cast<const float*>(c->ST);
    CKC(c, launch_delta<float>(st, c->ctrl, force, k_arg, g));
  }
  return RS_OK;
}

rs_status enqueue_update(rs_ctx* c) {
  UpdateArgs a{};
  a.gam = c->gam; a.bet = c->bet;
  a.w = c->w; a.wp = c->wp; a.r = c->r; a.rp = c->rp; a.u = c->u;
  a.delta = c->delta; a.partials = c->partials; a.hist = c->hist;
  a.mixed = c->mixed();
  if (c->mixed())
    CKC(c, launch_update<float>(c->stream, c->ctrl, plan_view(c), rows_view<float>(c), c->m, c->tau, a));
  else
    CKC(c, launch_update<double>(c->stream, c->ctrl, plan_view(c), rows_view<double>(c), c->m, c->tau, a));
  return RS_OK;
}

template <typename T, typename TF>
rs_status enqueue_iterate_t(rs_ctx* c, int64_t sub_end) {
  IterArgs<T, TF> g{};
  g.kind = c->sketch == RS_GAUSSIAN ? 1 : 0;
  g.mixed = c->mixed();
  g.A = static_cast<const T*>(c->A);
  g.lda = c->ld;
  g.SA = c->sketch == RS_SUBSAMPLE ? nullptr : static_cast<const T*>(c->SA);
  g.sa_slot = c->sa_slot;
  g.ST = c->sketch == RS_GAUSSIAN ? static_cast<const T*>(c->ST) : nullptr;
  g.plan = plan_view(c);
  g.inv = c->inv;
  g.inv_slot = c->ld;
  g.Linv = static_cast<const TF*>(c->Linv);
  g.l_slot = c->l_slot;
  g.gam = c->gam; g.bet = c->bet;
  g.w = c->w; g.wp = c->wp; g.r = c->r; g.rp = c->rp;
  g.hist = c->hist; g.delta_out = c->delta; g.rS_out = c->rS;
  g.m = c->m; g.tau = c->tau; g.chunk = c->chunk;
  g.sub_end = sub_end;
  CKC(c, (launch_iterate<T, TF>(c->stream, c->ctrl, g)));
  return RS_OK;
}

template <typename T, typename TF>
rs_status enqueue_wide_t(rs_ctx* c, int64_t sub_end) {
  WideArgs<T, TF> g{};
  g.mixed = c->mixed();
  g.rows = static_cast<const T*>(c->SA);
  g.sa_slot = c->sa_slot;
  g.inv = c->inv;
  g.inv_slot = c->ld;
  g.P = static_cast<const TF*>(c->Pm);
  g.pld = c->pld;
  g.p_slot = c->p_slot;
  g.gam = c->gam; g.bet = c->bet;
  g.w = c->w; g.wp = c->wp; g.r = c->r; g.rp = c->rp;
  g.hist = c->hist; g.delta_out = c->delta;
  g.part = c->xpart;
  g.epoch = c->xflags;
  g.abort_word = c->xabort;
  g.m = c->m; g.tau = c->tau; g.chunk = c->chunk; g.q = c->wide.q;
  g.sub_end = sub_end;
  g.nblk = c->wide.nblk;
  g.nsab = c->wide.nsab;
  g.wait_ns = c->wait_ns;
  g.stall_ns = c->stall_ns;
  g.wsum = c->avg ? c->wsum : nullptr;
  g.accel = c->accel ? 1 : 0;
  g.acc_a = c->acc_a;
  g.acc_b = c->acc_b;
  g.acc_g = c->acc_g;
  CKC(c, (launch_iterate_wide<T, TF>(c->stream, c->ctrl, g, c->wide.smem)));
  return RS_OK;
}

// every iteration of the chunk in one launch (all sketches but SRHT): over the
// whole GPU for the bucket-row sketches, else on one thread-block cluster
// the persistent iterations of the current chunk up to its slot sub_end (default: all)
rs_status enqueue_iterate(rs_ctx* c, int64_t sub_end = -1) {
  if (sub_end < 0 || sub_end > c->chunk) sub_end = c->chunk;
  if (c->use_wide) {
    // mixed: M^+ (FP64-formed or by FP32 sweeps) is stored in FP32 for the FP32 iterations
    if (!c->mixed()) return enqueue_wide_t<double, double>(c, sub_end);
    return enqueue_wide_t<float, float>(c, sub_end);
  }
  if (!c->mixed()) return enqueue_iterate_t<double, double>(c, sub_end);
  return c->f64_factor() ? enqueue_iterate_t<float, double>(c, sub_end)
                         : enqueue_iterate_t<float, float>(c, sub_end);
}

// one matrix-free iteration: delta, (XS) delta, X^T v by column pieces, update
rs_status enqueue_mf_iteration(rs_ctx* c) {
  UpdateArgs a{};
  a.gam = c->gam; a.bet = c->bet;
  a.w = c->w; a.wp = c->wp; a.r = c->r; a.rp = c->rp; a.u = c->u;
  a.delta = c->delta; a.partials = c->partials; a.hist = c->hist;
  a.mixed = c->mixed();
  return with_vt(c, [&](auto tag) -> rs_status {
    using VT = std::remove_pointer_t<decltype(tag)>;
    const SparseX<VT> X = sparse_view<VT>(c);
    if (c->mixed())
      CKC(c, (launch_mf_iteration<VT, float>(c->stream, c->ctrl, mf_args(c), X,
                                             static_cast<const float*>(c->mf_eval), plan_view(c),
                                             static_cast<const float*>(c->Pm), c->pld, c->p_slot,
                                             static_cast<float*>(c->mf_v),
                                             static_cast<float*>(c->mf_pu), a, c->rS)));
    else
      CKC(c, (launch_mf_iteration<VT, double>(c->stream, c->ctrl, mf_args(c), X,
                                              static_cast<const double*>(c->mf_eval), plan_view(c),
                                              static_cast<const double*>(c->Pm), c->pld, c->p_slot,
                                              static_cast<double*>(c->mf_v),
                                              static_cast<double*>(c->mf_pu), a, c->rS)));
    return RS_OK;
  });
}

rs_status enqueue_iteration(rs_ctx* c) {
  rs_status s = enqueue_delta(c, 0, -1);
  if (s != RS_OK) return s;
  return enqueue_update(c);
}

// true residual through X into vn / vd; v is the current iterate vector (m)
rs_status enqueue_true_av(rs_ctx* c, const double* v, const int32_t* stop) {
  cudaStream_t st = c->stream;
  if (c->sparse)  // primal: X^T (X w) + lambda w, FP64 through the stored values
    return with_vt(c, [&](auto tag) -> rs_status {
      using VT = std::remove_pointer_t<decltype(tag)>;
      const SparseX<VT> X = sparse_view<VT>(c);
      CKC(c, sparse_xv_d<VT>(st, X, v, c->mf_z, stop));
      CKC(c, sparse_xtv_d<VT>(st, X, c->mf_z, c->vd, c->mf_pud, stop));
      return RS_OK;
    });
  // primal: A w = X^T (X w) + lambda w; dual: A a = X (X^T a) + lambda a
  if (c->kernel) {  // K w into vn (for the lambda K w term), K^T (K w) into vd, FP64 sums
    if (c->xdtype == RS_F32) {
      CKC(c, launch_x_v<float>(st, static_cast<const float*>(c->X), c->n, c->d, v, c->vn, stop));
      CKC(c, launch_xt_v<float>(st, static_cast<const float*>(c->X), c->n, c->d, c->vn, c->vd,
                                c->xt_part, stop));
    } else {
      CKC(c, launch_x_v<double>(st, static_cast<const double*>(c->X), c->n, c->d, v, c->vn, stop));
      CKC(c, launch_xt_v<double>(st, static_cast<const double*>(c->X), c->n, c->d, c->vn, c->vd,
                                 c->xt_part, stop));
    }
    return RS_OK;
  }
  if (c->xdtype == RS_F32) {
    const float* X = static_cast<const float*>(c->X);
    if (c->form == RS_PRIMAL && c->d <= 4096 && c->xtx_df) {
      CKC(c, launch_xtx_v_df(st, X, c->n, c->d, v, c->vd, c->xt_part, stop));
    } else if (c->form == RS_PRIMAL && c->xtx_df && c->d <= 24576) {
      // wider d: the same float-pair product in two passes (X w into vn as pairs)
      CKC(c, launch_xtx_two_pass(st, X, c->n, c->d, 1, v, c->vd, reinterpret_cast<float2*>(c->vn),
                                 c->xt_part, stop));
    } else if (c->form == RS_PRIMAL) {
      CKC(c, launch_x_v<float>(st, X, c->n, c->d, v, c->vn, stop));
      CKC(c, launch_xt_v<float>(st, X, c->n, c->d, c->vn, c->vd, c->xt_part, stop));
    } else {
      CKC(c, launch_xt_v<float>(st, X, c->n, c->d, v, c->vd, c->xt_part, stop));
      CKC(c, launch_x_v<float>(st, X, c->n, c->d, c->vd, c->vn, stop));
    }
  } else {
    const double* X = static_cast<const double*>(c->X);
    if (c->form == RS_PRIMAL) {
      CKC(c, launch_x_v<double>(st, X, c->n, c->d, v, c->vn, stop));
      CKC(c, launch_xt_v<double>(st, X, c->n, c->d, c->vn, c->vd, c->xt_part, stop));
    } else {
      CKC(c, launch_xt_v<double>(st, X, c->n, c->d, v, c->vd, c->xt_part, stop));
      CKC(c, launch_x_v<double>(st, X, c->n, c->d, c->vd, c->vn, stop));
    }
  }
  return RS_OK;
}

const double* av_out(const rs_ctx* c) { return c->form == RS_PRIMAL ? c->vd : c->vn; }

rs_status enqueue_refresh(rs_ctx* c) {
  rs_status s = enqueue_true_av(c, c->w, &c->ctrl->stop);
  if (s != RS_OK) return s;
  // A w = K^T K w + lambda K w (kernel ridge) or X^T X w + lambda w
  CKC(c, launch_refresh_finish(c->stream, c->ctrl, 1, c->m, av_out(c), c->kernel ? c->vn : c->w,
                               c->b, c->lambda, c->r, c->rp, c->partials, c->hist, nullptr));
  return RS_OK;
}

// one chunk: phase 1 for all its slots, then its iterations; with_refresh (mixed) puts
// an FP64 refresh after every refresh_every iterations (the chunk holds a whole number
// of periods), so the persistent kernel runs in launches of one period each
rs_status enqueue_chunk(rs_ctx* c, bool with_refresh) {
  CKC(c, launch_chunk_begin(c->stream, c->ctrl, c->hist));
  rs_status s = enqueue_phase1(c, 0, -1, (int)c->nslots, c->use_wide || c->sparse);
  if (s != RS_OK) return s;
  const int64_t per = with_refresh ? std::min<int64_t>(c->refresh_every, c->chunk) : c->chunk;
  if (c->sparse || c->sketch == RS_SRHT) {
    for (int64_t i = 0; i < c->chunk; ++i) {
      s = c->sparse ? enqueue_mf_iteration(c) : enqueue_iteration(c);
      if (s != RS_OK) return s;
      if (with_refresh && (i + 1) % per == 0 && i + 1 < c->chunk && (s = enqueue_refresh(c)) != RS_OK)
        return s;
    }
  } else {
    for (int64_t e = per;; e += per) {
      if ((s = enqueue_iterate(c, std::min<int64_t>(e, c->chunk))) != RS_OK) return s;
      if (e >= c->chunk) break;
      if (with_refresh && (s = enqueue_refresh(c)) != RS_OK) return s;
    }
  }
  if (with_refresh) return enqueue_refresh(c);
  return RS_OK;
}

rs_status build_graph(rs_ctx* c, bool with_refresh) {
  if (c->graph && c->graph_refresh == with_refresh) return RS_OK;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  CKC(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
  // several chunks per replay: the host reads the control block once per replay;
  // chunks after the solve has stopped return at once (every kernel checks ctrl)
  rs_status s = RS_OK;
  for (int i = 0; i < kChunksPerGraph && s == RS_OK; ++i) s = enqueue_chunk(c, with_refresh);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (s != RS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) FAILC(c, RS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) FAILC(c, RS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  c->graph_refresh = with_refresh;
  return RS_OK;
}

rs_status ensure_schedule(rs_ctx* c, int64_t K) {
  if (K <= c->sched_len && K + 1 <= c->hist_len) return RS_OK;
  const int64_t L = std::max<int64_t>(K, 1024);
  pfree(c, c->gam);
  pfree(c, c->bet);
  pfree(c, c->hist);
  c->gam = c->bet = c->hist = nullptr;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (c->cg_graph) {  // captured the history buffer too
    cudaGraphExecDestroy(c->cg_graph);
    c->cg_graph = nullptr;
  }
  rs_status s;
  if ((s = dalloc(c, &c->gam, L)) != RS_OK) return s;
  if ((s = dalloc(c, &c->bet, L)) != RS_OK) return s;
  if ((s = dalloc(c, &c->hist, L + 1)) != RS_OK) return s;
  // momentum parameters (Section 8.1), eqs. (38), (40), (50), (66), (67)
  std::vector<double> g(L), bt(L);
  const rs_mom& mo = c->mom;
  if (mo.kind == RS_MOM_NONE) {
    for (int64_t k = 0; k < L; ++k) { g[k] = 1.0; bt[k] = 0.0; }
  } else if (mo.kind == RS_MOM_CONST) {
    for (int64_t k = 0; k < L; ++k) { g[k] = mo.gamma_c; bt[k] = mo.beta_c; }
  } else if (mo.kind == RS_MOM_HEURISTIC && mo.uncapped) {
    for (int64_t k = 0; k < L; ++k) {
      g[k] = 1.0;
      bt[k] = 1.0 - (2.0 - mo.eta) / (((double)k + 1.0) * (1.0 - mo.eta) + 1.0);
    }
  } else {
    double acc = 0.0, eta_k = mo.eta;
    for (int64_t k = 0; k < L; ++k) {
      const double zeta_k = acc / eta_k;
      const double acc_next = acc + eta_k * (1.0 - eta_k);
      const double zeta_next = acc_next / eta_k;
      const double gk = eta_k / (1.0 + zeta_next);
      const double bk = zeta_k / (1.0 + zeta_next);
      g[k] = (mo.kind == RS_MOM_THEORY) ? gk : 1.0;
      bt[k] = bk;
      acc = acc_next;
      if (bk >= mo.beta_switch) eta_k = 1.0;
    }
  }
  CKC(c, copy_sync(c, c->gam, g.data(), L * sizeof(double), cudaMemcpyHostToDevice));
  CKC(c, copy_sync(c, c->bet, bt.data(), L * sizeof(double), cudaMemcpyHostToDevice));
  c->sched_len = L;
  c->hist_len = L + 1;
  return RS_OK;
}

rs_status read_ctrl(rs_ctx* c) {
  CKC(c, cudaMemcpyAsync(c->ctrl_h, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status write_ctrl(rs_ctx* c) {
  CKC(c, cudaMemcpyAsync(c->ctrl, c->ctrl_h, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
  return RS_OK;
}

// run chunks until the device says stop; max_chunks bounds the host loop
rs_status run_loop(rs_ctx* c, bool with_refresh, int64_t max_chunks) {
  rs_status s = build_graph(c, with_refresh);
  if (s != RS_OK) return s;
  for (int64_t q = 0; q < (max_chunks + kChunksPerGraph - 1) / kChunksPerGraph; ++q) {
    CKC(c, cudaGraphLaunch(c->graph, c->stream));
    if ((s = read_ctrl(c)) != RS_OK) return s;
    if (c->ctrl_h->stop) return RS_OK;
  }
  return RS_OK;
}

rs_status copy_out_w(rs_ctx* c, double* w_out, int32_t on_device) {
  if (!w_out) return RS_OK;
  const double* src = c->w;
  if (c->form == RS_DUAL) {  // w = X^T alpha (eq. (3))
    if (c->xdtype == RS_F32)
      CKC(c, launch_xt_v<float>(c->stream, static_cast<const float*>(c->X), c->n, c->d, c->w, c->vd,
                                c->xt_part));
    else
      CKC(c, launch_xt_v<double>(c->stream, static_cast<const double*>(c->X), c->n, c->d, c->w,
                                 c->vd, c->xt_part));
    src = c->vd;
  }
  CKC(c, cudaMemcpyAsync(w_out, src, c->d * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return RS_OK;
}

rs_status true_rel(rs_ctx* c, const double* v_dev, double* rel) {
  rs_status s = enqueue_true_av(c, v_dev, nullptr);
  if (s != RS_OK) return s;
  CKC(c, launch_refresh_finish(c->stream, c->ctrl, 0, c->m, av_out(c), c->kernel ? c->vn : v_dev,
                               c->b, c->lambda, nullptr, nullptr, c->partials, nullptr, c->rel_dev));
  CKC(c, cudaMemcpyAsync(c->scal_h, c->rel_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  *rel = *c->scal_h;
  return RS_OK;
}

// CSR input: device copies, CSC by a stable counting sort, the column pieces of
// X^T v, b = X^T y, and the capacities of the per-slot XS buffers
template <typename VT>
rs_status sparse_setup_t(rs_ctx* c, const rs_matrix* X, const double* y, int32_t y_on_device) {
  cudaStream_t st = c->stream;
  const int64_t n = c->n, d = c->d, nnz = c->nnz;
  const cudaMemcpyKind kind = X->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  rs_status s;
  if ((s = dalloc(c, &c->sx_rowptr, n + 1)) != RS_OK) return s;
  if ((s = dalloc(c, &c->sx_colidx, nnz)) != RS_OK) return s;
  CKC(c, pmalloc(c, (void**)&c->sx_val, std::max<int64_t>(nnz, 1) * sizeof(VT)));
  CKC(c, cudaMemcpyAsync(c->sx_rowptr, X->rowptr, (n + 1) * sizeof(int64_t), kind, st));
  CKC(c, cudaMemcpyAsync(c->sx_colidx, X->colidx, nnz * sizeof(int32_t), kind, st));
  CKC(c, cudaMemcpyAsync(c->sx_val, X->val, nnz * sizeof(VT), kind, st));
  CKC(c, cudaMemsetAsync(c->err_flag, 0, sizeof(int32_t), st));
  CKC(c, launch_csr_check(st, c->sx_rowptr, n, c->sx_colidx, nnz, d, c->err_flag));
  int32_t bad = 0;
  CKC(c, cudaMemcpyAsync(&bad, c->err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKC(c, cudaStreamSynchronize(st));
  if (bad) FAILC(c, RS_EINVAL, "rs_create: inconsistent CSR arrays (rowptr or column indices)");
  // CSC (rows ascending in every column)
  const int nb = 152;
  int32_t* table = nullptr;
  int64_t* colcnt = nullptr;
  if ((s = dalloc(c, &table, (size_t)nb * d)) != RS_OK) return s;
  if ((s = dalloc(c, &colcnt, d)) != RS_OK) { pfree(c, table); return s; }
  if ((s = dalloc(c, &c->sx_colptr, d + 1)) != RS_OK) return s;
  if ((s = dalloc(c, &c->sx_rowidx, nnz)) != RS_OK) return s;
  CKC(c, pmalloc(c, (void**)&c->sx_cval, std::max<int64_t>(nnz, 1) * sizeof(VT)));
  cudaError_t e = build_csc<VT>(st, c->sx_rowptr, n, c->sx_colidx, static_cast<const VT*>(c->sx_val),
                                nnz, d, table, nb, colcnt, c->sx_colptr, c->sx_rowidx,
                                static_cast<VT*>(c->sx_cval));
  std::vector<int64_t> colptr(d + 1);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(colptr.data(), c->sx_colptr, (d + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  pfree(c, table);
  pfree(c, colcnt);
  CKC(c, e);
  // pieces of at most kPiece entries per column, in column order
  std::vector<int32_t> pcol, cpiece(d + 1);
  std::vector<int64_t> pstart;
  for (int64_t col = 0; col < d; ++col) {
    cpiece[col] = (int32_t)pcol.size();
    for (int64_t q = colptr[col]; q < colptr[col + 1]; q += kPiece) {
      pcol.push_back((int32_t)col);
      pstart.push_back(q);
    }
  }
  cpiece[d] = (int32_t)pcol.size();
  c->sx_npieces = (int64_t)pcol.size();
  if ((s = dalloc(c, &c->sx_pcol, pcol.size())) != RS_OK) return s;
  if ((s = dalloc(c, &c->sx_pstart, pstart.size())) != RS_OK) return s;
  if ((s = dalloc(c, &c->sx_cpiece, d + 1)) != RS_OK) return s;
  if (!pcol.empty()) {
    CKC(c, copy_sync(c, c->sx_pcol, pcol.data(), pcol.size() * 4, cudaMemcpyHostToDevice));
    CKC(c, copy_sync(c, c->sx_pstart, pstart.data(), pstart.size() * 8, cudaMemcpyHostToDevice));
  }
  CKC(c, copy_sync(c, c->sx_cpiece, cpiece.data(), (d + 1) * 4, cudaMemcpyHostToDevice));
  // y, b = X^T y (FP64)
  if ((s = dalloc(c, &c->y, n)) != RS_OK) return s;
  CKC(c, cudaMemcpyAsync(c->y, y, n * sizeof(double), y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  if ((s = dalloc(c, &c->mf_pud, std::max<int64_t>(c->sx_npieces, 1))) != RS_OK) return s;
  if ((s = dalloc(c, &c->mf_z, n)) != RS_OK) return s;
  if ((s = dalloc(c, &c->vd, d)) != RS_OK) return s;
  if ((s = dalloc(c, &c->b, d)) != RS_OK) return s;
  CKC(c, sparse_xtv_d<VT>(st, sparse_view<VT>(c), c->y, c->b, c->mf_pud, nullptr));
  // capacity of one slot's XS: the entries of the heaviest sampled columns
  std::vector<int64_t> cnt(d);
  for (int64_t col = 0; col < d; ++col) cnt[col] = colptr[col + 1] - colptr[col];
  const int64_t ns = (c->sketch == RS_COUNT) ? d : (c->sketch == RS_SUBCOUNT ? c->s : c->tau);
  std::nth_element(cnt.begin(), cnt.begin() + std::min<int64_t>(ns, d) - 1, cnt.end(), std::greater<int64_t>());
  int64_t ecap = 0;
  for (int64_t q = 0; q < std::min<int64_t>(ns, d); ++q) ecap += cnt[q];
  c->mf_ecap = std::max<int64_t>(ecap, 1);
  c->mf_rcap = std::max<int64_t>(1, std::min<int64_t>(n, ecap));
  c->mf_nrb = mf_row_blocks(n);
  return RS_OK;
}

}  // namespace

// ===========================================================================
// public API
// ===========================================================================
extern "C" {

void rs_default_opts(rs_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = RS_PLAIN_FP64;
  o->refresh_every = 50;
  o->sub_s = 0;
  o->cuda_stream = nullptr;
  o->device = 0;
  o->chol_fp64 = 1;
  o->chunk = 0;
  o->setup_tc = 1;
  o->iter_ctas = 0;
  o->spin_limit_ns = 0;
  o->stall_ns = 0;
  o->tune_cache = nullptr;
}

void rs_default_mom(rs_mom* m, int32_t kind) {
  if (!m) return;
  std::memset(m, 0, sizeof(*m));
  m->kind = kind;
  m->uncapped = 0;
  m->eta = 0.995;
  m->beta_switch = 0.5;
  m->gamma_c = 1.0;
  m->beta_c = 0.5;
}

const char* rs_last_error(const rs_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err.c_str();
}

constexpr int64_t kPipeMinRows = 16384;
constexpr int kPipePieces = 4;

// Setup of a mixed primal context from FP32 X in host memory: X is copied into c->X
// in kPipePieces row ranges on a copy stream; on the context's stream, each range's
// transposed copy, its part of X^T X + lambda I (tensor cores, added into A) and its
// 512-row blocks of X^T y follow their range's copy event. c->X, y, A (zeroed), b and
// the scratch are allocated on the context's stream before.
rs_status setup_pipelined(rs_ctx* c, const float* Xh, double lambda) {
  cudaStream_t st = c->stream;
  const int64_t n = c->n, d = c->d;
  float* Xf = static_cast<float*>(c->X);
  float* Xt = nullptr;
  CKC(c, pmalloc(c, (void**)&Xt, gram_tc_ws_floats(n, d) * sizeof(float)));
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[kPipePieces + 1] = {};
  auto cleanup = [&]() {
    for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);  // (released once completed)
    if (cs) cudaStreamDestroy(cs);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (int i = 0; i <= kPipePieces && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  // the copies start once the allocations are in place in the context's stream order
  if (e == cudaSuccess) e = cudaEventRecord(ev[kPipePieces], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[kPipePieces], 0);
  if (e == cudaSuccess) e = xt_pairs_split(st, c->y, n, d, c->xt_part);
  const int64_t rows = round_up((n + kPipePieces - 1) / kPipePieces, 512);
  auto piece = [&](int i, int64_t& r0, int64_t& r1) {
    r0 = std::min<int64_t>(n, (int64_t)i * rows);
    r1 = std::min<int64_t>(n, r0 + rows);
  };
  // copy of range i, then the arithmetic of range i - 1 (a host staging a pageable
  // source copies the next range while the device works on the previous one)
  for (int i = 0; i <= kPipePieces && e == cudaSuccess; ++i) {
    int64_t r0, r1;
    if (i < kPipePieces) {
      piece(i, r0, r1);
      if (r1 > r0)
        e = cudaMemcpyAsync(Xf + r0 * d, Xh + r0 * d, (size_t)(r1 - r0) * d * sizeof(float),
                            cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess) e = cudaEventRecord(ev[i], cs);
    }
    if (i >= 1 && e == cudaSuccess) {
      piece(i - 1, r0, r1);
      e = cudaStreamWaitEvent(st, ev[i - 1], 0);
      if (e == cudaSuccess && r1 > r0)
        e = launch_gram_tc_rows(st, Xf, n, d, lambda, static_cast<float*>(c->A), c->ld, Xt,
                                c->err_flag, r0, r1);
      if (e == cudaSuccess && r1 > r0) e = xt_pairs_rows(st, Xf, n, d, c->xt_part, r0, r1);
    }
  }
  if (e == cudaSuccess) e = launch_mirror_lower<float>(st, static_cast<float*>(c->A), d, c->ld);
  if (e == cudaSuccess) e = xt_pairs_sum(st, n, d, c->xt_part, c->b);
  pfree(c, Xt);  // in stream order, after the products
  cleanup();
  CKC(c, e);
  return RS_OK;
}

// bytes the per-slot buffers of one chunk may take: a quarter of the free device
// memory, at least 4 GB and at most 16 GB
int64_t slot_budget() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = (size_t)16e9;
  }
  return std::max<int64_t>((int64_t)4e9, std::min<int64_t>((int64_t)16e9, (int64_t)(fr / 4)));
}

// the largest chunk within `cap` slots; in mixed precision a whole number of refresh
// periods, or (cap below one period) the period itself shortened to cap
int64_t cap_chunk(rs_ctx* c, int64_t cap) {
  if (!c->mixed()) return cap;
  if (cap >= c->refresh_every) return cap / c->refresh_every * c->refresh_every;
  c->refresh_every = (int)cap;
  return cap;
}

rs_status rs_create(const rs_matrix* X, const double* y, int32_t y_on_device, double lambda,
                    int32_t form, int32_t sketch, int64_t tau, const rs_mom* mom, uint64_t seed,
                    const rs_opts* opts, rs_ctx** out) {
  if (out) *out = nullptr;
  if (!X || !y || !out) { set_global_error("rs_create: null argument"); return RS_EINVAL; }
  if (X->n <= 0 || X->d <= 0) { set_global_error("rs_create: empty X"); return RS_EINVAL; }
  if (X->is_csr) {
    if (!X->rowptr || !X->colidx || X->nnz < 0 || (X->nnz > 0 && !X->val)) { set_global_error("rs_create: null or bad CSR arrays"); return RS_EINVAL; }
    if (X->dtype != RS_F64 && X->dtype != RS_F32 && X->dtype != RS_BF16) { set_global_error("rs_create: bad dtype"); return RS_EINVAL; }
    if (X->d > INT32_MAX || X->n > INT32_MAX) { set_global_error("rs_create: sparse X needs n, d < 2^31"); return RS_EINVAL; }
  } else {
    if (!X->val) { set_global_error("rs_create: empty X"); return RS_EINVAL; }
    if (X->dtype != RS_F64 && X->dtype != RS_F32) { set_global_error("rs_create: bad dtype"); return RS_EINVAL; }
  }
  if (!(lambda > 0.0) || !std::isfinite(lambda)) { set_global_error("rs_create: lambda must be > 0"); return RS_EINVAL; }
  if (form != RS_PRIMAL && form != RS_DUAL) { set_global_error("rs_create: bad form"); return RS_EINVAL; }
  if (sketch < RS_GAUSSIAN || sketch > RS_SRHT) { set_global_error("rs_create: bad sketch"); return RS_EINVAL; }
  if (X->is_csr && form != RS_PRIMAL) { set_global_error("rs_create: a sparse X runs matrix-free in the primal form only"); return RS_EUNSUPPORTED; }
  if (X->is_csr && sketch != RS_SUBSAMPLE && sketch != RS_COUNT && sketch != RS_SUBCOUNT) {
    set_global_error("rs_create: a sparse X takes the subsample, count or subcount sketch");
    return RS_EUNSUPPORTED;
  }
  rs_opts o;
  rs_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != RS_PLAIN_FP64 && o.precision != RS_MIXED) { set_global_error("rs_create: bad precision"); return RS_EINVAL; }
  rs_mom mo;
  rs_default_mom(&mo, RS_MOM_NONE);
  if (mom) mo = *mom;
  if (mo.kind < RS_MOM_NONE || mo.kind > RS_MOM_HEURISTIC) { set_global_error("rs_create: bad momentum kind"); return RS_EINVAL; }
  if ((mo.kind == RS_MOM_THEORY || mo.kind == RS_MOM_HEURISTIC) && !(mo.eta > 0.0 && mo.eta <= 1.0)) {
    set_global_error("rs_create: eta must be in (0, 1]");
    return RS_EINVAL;
  }

  rs_ctx* c = new (std::nothrow) rs_ctx();
  if (!c) { set_global_error("rs_create: out of host memory"); return RS_ENOMEM; }
  auto fail = [&](rs_status s) {
    set_global_error(c->err);
    free_all(c);
    delete c;
    return s;
  };
  c->device = o.device;
  DeviceGuard dg(c->device);
  c->form = form;
  c->sketch = sketch;
  c->precision = o.precision;
  c->chol_fp64 = o.chol_fp64 ? 1 : 0;
  c->refresh_every = o.refresh_every > 0 ? o.refresh_every : 50;
  if (o.spin_limit_ns > 0) c->wait_ns = (uint64_t)o.spin_limit_ns;
  c->stall_ns = o.stall_ns > 0 ? o.stall_ns : 0;
  c->n = X->n;
  c->d = X->d;
  c->m = (form == RS_PRIMAL) ? X->d : X->n;
  c->lambda = lambda;
  c->seed = seed;
  c->mom = mo;
  c->xdtype = X->dtype;
  c->sparse = X->is_csr != 0;
  c->batch_member = t_batch_member;
  c->nnz = X->is_csr ? X->nnz : 0;
  const int64_t m = c->m;
  c->tau = tau > 0 ? tau : default_tau(m);
  c->ld = round_up(m, kLdAlign);
  if (c->tau > m && sketch != RS_SRHT) { c->err = "rs_create: tau must be <= m"; return fail(RS_EINVAL); }
  if (sketch == RS_SRHT) {
    c->mp = pow2_ceil(m);
    if (c->mp > srht_max_pad()) { c->err = "rs_create: SRHT needs 2^ceil(log2 m) <= 16384"; return fail(RS_EUNSUPPORTED); }
    if (c->tau > c->mp) { c->err = "rs_create: SRHT needs tau <= 2^ceil(log2 m)"; return fail(RS_EINVAL); }
  }
  if (sketch == RS_SUBCOUNT) {
    if (o.sub_s > 0) {
      if (o.sub_s % c->tau != 0 || o.sub_s > m || o.sub_s < c->tau) { c->err = "rs_create: SubCount s must be a multiple of tau in [tau, m]"; return fail(RS_EINVAL); }
      c->s = o.sub_s;
      c->kk = o.sub_s / c->tau;
    } else {
      c->kk = (10 * c->tau <= m) ? 10 : m / c->tau;
      c->s = c->kk * c->tau;
    }
  }
  const int64_t sample_n = (sketch == RS_SUBCOUNT) ? c->s : c->tau;
  if ((sketch == RS_SUBSAMPLE || sketch == RS_SUBCOUNT || sketch == RS_SRHT) && sample_n > kMaxSample) {
    c->err = "rs_create: sample size above 8192 is not supported";
    return fail(RS_EUNSUPPORTED);
  }
  if (sketch == RS_COUNT && c->tau > kMaxCountTau) { c->err = "rs_create: count sketch tau above 2048 is not supported"; return fail(RS_EUNSUPPORTED); }
  if (c->tau > 8192) { c->err = "rs_create: tau above 8192 is not supported"; return fail(RS_EUNSUPPORTED); }

  if (o.cuda_stream) {
    c->stream = static_cast<cudaStream_t>(o.cuda_stream);
  } else {
    // a blocking stream: its work orders after the work issued before it on the
    // legacy default stream, where device inputs are often produced (a non-blocking
    // stream could read them half-written)
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault) != cudaSuccess) { c->err = "rs_create: stream"; return fail(RS_ECUDA); }
    c->own_stream = true;
  }
  // mixed: a chunk (the slots whose sketched systems phase 1 forms and factors in one
  // batch) holds a whole number of refresh periods; by default the smallest such
  // number of iterations >= kMixedChunk, so that phase 1 keeps every SM busy even
  // when the refresh period is short
  // default chunks: 600 slots for dense A in either precision (the FP64 factor's
  // four CTAs per SM then fill the GPU), 128 for the matrix-free path
  c->chunk = o.chunk > 0 ? o.chunk : ((c->mixed() || !c->sparse) ? kMixedChunk : 128);
  if (c->mixed()) {  // a chunk shorter than the period shortens the period to it
    if (c->chunk < c->refresh_every) c->refresh_every = (int)c->chunk;
    c->chunk = round_up(c->chunk, (int64_t)c->refresh_every);
  }
  if (!c->sparse) {
    // keep the per-slot buffers of one chunk (S^T A is materialised for every sketch
    // once the persistent kernel runs it) within the slot budget where S^T A and M
    // are formed in one pass (bucket-row sketches whose rows fit shared memory): there
    // a full chunk fills the FP64 factor's wave (in FP64 a 4 GB cap held 379 slots of
    // tau = 256 at m = 4096). The other phase-1 paths share reads of A and the
    // factors' work space in L2 between the slots in flight and run faster on smaller
    // chunks (kernel ridge at m = 20640: 2x per slot at 600 slots against 150), so
    // they keep 4 GB.
    const int64_t nperm = round_up(sketch == RS_COUNT ? m : (sketch == RS_SUBCOUNT ? c->s : c->tau), 4);
    const bool one_pass =
        (sketch == RS_SUBSAMPLE || sketch == RS_COUNT || sketch == RS_SUBCOUNT) &&
        (c->mixed() ? sa_msys_fits<float>(m, c->tau, nperm) : sa_msys_fits<double>(m, c->tau, nperm));
    const int64_t per_slot = c->tau * c->ld * (int64_t)c->elem() * (sketch == RS_GAUSSIAN ? 2 : 1) +
                             c->tau * c->tau * 33 + c->ld * 4;
    const int64_t budget = one_pass ? slot_budget() : (int64_t)4e9;
    const int64_t cap = std::max<int64_t>(1, budget / std::max<int64_t>(per_slot, 1));
    if (c->chunk > cap) c->chunk = cap_chunk(c, cap);
  }
  c->nslots = c->chunk;
  cudaStream_t st = c->stream;
  rs_status s;
#define TRY(expr) do { if ((s = (expr)) != RS_OK) return fail(s); } while (0)
#define TRYC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { c->err = std::string(#call) + ": " + cudaGetErrorString(e_) + (e_ == cudaErrorMemoryAllocation ? mem_note() : std::string()); return fail(e_ == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA); } } while (0)
  TRYC(cudaEventCreate(&c->ev0));
  TRYC(cudaEventCreate(&c->ev1));
  TRYC(cudaMallocHost((void**)&c->ctrl_h, sizeof(Ctrl)));
  TRYC(cudaMallocHost((void**)&c->scal_h, sizeof(double)));
  TRY(dalloc(c, &c->ctrl, 1));
  std::memset(c->ctrl_h, 0, sizeof(Ctrl));
  c->ctrl_h->r0 = 1.0;
  TRYC(cudaMemcpyAsync(c->ctrl, c->ctrl_h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));

  TRY(dalloc(c, &c->err_flag, 1));
  TRY(dalloc(c, &c->ndropped, 1));
  TRYC(cudaMemsetAsync(c->err_flag, 0, sizeof(int32_t), st));
  TRYC(cudaMemsetAsync(c->ndropped, 0, sizeof(int32_t), st));
  TRY(dalloc(c, &c->rel_dev, 1));
  if (c->sparse) {
    // matrix-free: CSR + CSC of X on the device, b = X^T y; A is never formed
    TRYC(cudaEventRecord(c->ev0, st));
    s = with_vt(c, [&](auto tag) -> rs_status {
      using VT = std::remove_pointer_t<decltype(tag)>;
      return sparse_setup_t<VT>(c, X, y, y_on_device);
    });
    if (s != RS_OK) return fail(s);
    TRYC(cudaEventRecord(c->ev1, st));
    // the per-slot XS buffers of a chunk, sized for the heaviest sampled columns, stay
    // within the slot budget: a chunk of a few dozen slots would leave most SMs idle in
    // its small solves (one CTA per slot)
    const int64_t per_slot = c->mf_rcap * 8 + c->mf_ecap * (4 + (int64_t)c->elem()) +
                             c->tau * c->tau * 33 + c->ld * 4 + c->mf_nrb * 16;
    const int64_t cap = std::max<int64_t>(1, slot_budget() / std::max<int64_t>(per_slot, 1));
    if (c->chunk > cap) {
      c->chunk = cap_chunk(c, cap);
      c->nslots = c->chunk;
    }
  } else {
  // X, y
  const size_t xel = X->dtype == RS_F32 ? 4 : 8;
  const size_t xbytes = (size_t)X->n * X->d * xel;
  const int dual = (form == RS_DUAL);
  // X from the host for the tensor-core Gram: uploaded in pieces, each piece's part of
  // X^T X and X^T y formed as soon as it has landed (the upload, about 210 GB/s on this
  // machine, overlaps the setup's arithmetic)
  const bool pipe = !X->on_device && X->dtype == RS_F32 && c->mixed() && !dual && o.setup_tc &&
                    c->n >= kPipeMinRows;
  // X on the device for the tensor-core Gram: the transposed copy's kernel also writes
  // the context's copy of X, from one read of the caller's X
  const bool fused_copy = X->on_device && X->dtype == RS_F32 && c->mixed() && !dual && o.setup_tc;
  TRYC(pmalloc(c, (void**)&c->X, xbytes));
  if (!pipe && !fused_copy)
    TRYC(cudaMemcpyAsync(c->X, X->val, xbytes, X->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  TRY(dalloc(c, &c->y, c->n));
  TRYC(cudaMemcpyAsync(c->y, y, c->n * sizeof(double), y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  // scratch of the X products
  TRY(dalloc(c, &c->vn, c->n));
  TRY(dalloc(c, &c->vd, c->d));
  TRY(dalloc(c, &c->xt_part, std::max<size_t>(xt_part_elems(c->n, c->d),
                                               (size_t)xtx_df_blocks() * c->d)));
  // A and b (eqs. (2)-(4))
  TRYC(pmalloc(c, (void**)&c->A, (size_t)m * c->ld * c->elem()));
  TRYC(cudaMemsetAsync(c->A, 0, (size_t)m * c->ld * c->elem(), st));
  TRY(dalloc(c, &c->b, m));
  TRYC(cudaEventRecord(c->ev0, st));
  if (pipe) {
    TRY(setup_pipelined(c, static_cast<const float*>(X->val), lambda));
  } else if (X->dtype == RS_F32) {
    const float* Xf = static_cast<const float*>(c->X);
    if (c->mixed() && !dual && o.setup_tc) {
      // X^T X on the tensor cores through a transposed, padded copy of X
      float* Xt = nullptr;
      TRYC(pmalloc(c, (void**)&Xt, gram_tc_ws_floats(c->n, c->d) * sizeof(float)));
      cudaError_t e1 =
          fused_copy ? launch_gram_tc(st, static_cast<const float*>(X->val), c->n, c->d, lambda,
                                      static_cast<float*>(c->A), c->ld, Xt, c->err_flag,
                                      static_cast<float*>(c->X))
                     : launch_gram_tc(st, Xf, c->n, c->d, lambda, static_cast<float*>(c->A), c->ld,
                                      Xt, c->err_flag);
      if (e1 == cudaSuccess) e1 = launch_mirror_lower<float>(st, static_cast<float*>(c->A), c->d, c->ld);
      pfree(c, Xt);  // in stream order, after the product
      TRYC(e1);
    } else if (c->mixed()) TRYC((launch_form_A<float, float>(st, Xf, c->n, c->d, dual, lambda, static_cast<float*>(c->A), c->ld)));
    else TRYC((launch_form_A<float, double>(st, Xf, c->n, c->d, dual, lambda, static_cast<double*>(c->A), c->ld)));
    if (!dual && c->mixed()) TRYC(launch_xt_v_pairs(st, Xf, c->n, c->d, c->y, c->b, c->xt_part));
    else if (!dual) TRYC(launch_xt_v<float>(st, Xf, c->n, c->d, c->y, c->b, c->xt_part));
  } else {
    const double* Xd = static_cast<const double*>(c->X);
    if (c->mixed()) TRYC((launch_form_A<double, float>(st, Xd, c->n, c->d, dual, lambda, static_cast<float*>(c->A), c->ld)));
    else TRYC((launch_form_A<double, double>(st, Xd, c->n, c->d, dual, lambda, static_cast<double*>(c->A), c->ld)));
    if (!dual) TRYC(launch_xt_v<double>(st, Xd, c->n, c->d, c->y, c->b, c->xt_part));
  }
  if (dual) TRYC(cudaMemcpyAsync(c->b, c->y, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRYC(cudaEventRecord(c->ev1, st));
  }
  // iteration buffers
  TRY(dalloc(c, &c->w, m));
  TRY(dalloc(c, &c->wp, m));
  TRY(dalloc(c, &c->r, m));
  TRY(dalloc(c, &c->rp, m));
  TRY(dalloc(c, &c->u, m));
  TRYC(cudaMemsetAsync(c->u, 0, m * sizeof(double), st));
  TRY(dalloc(c, &c->rS, c->tau));
  TRY(dalloc(c, &c->delta, c->tau));
  if (c->sparse) {
    // M^+ per slot and the per-slot XS of the chunk
    // M^+ is stored in the iteration's type (FP32 in mixed precision); it is formed in
    // the factor's precision by one kernel
    const size_t fel = c->f64_factor() ? 8 : 4;
    const size_t nsl = (size_t)c->nslots;
    c->pld = round_up(c->tau, 4);
    c->p_slot = c->tau * c->pld;
    TRYC(pmalloc(c, (void**)&c->Pm, nsl * c->p_slot * (c->mixed() ? 4 : 8)));
    if (c->tau <= 4096) {
      c->potri = true;
      if (potri_needs_ws(c->tau, fel)) TRYC(pmalloc(c, &c->pws, nsl * potri_ws_elems(c->tau) * fel));
    }
    TRY(dalloc(c, &c->mf_bsum, nsl * c->mf_nrb * 2));
    TRY(dalloc(c, &c->mf_boffs, nsl * c->mf_nrb * 2));
    TRY(dalloc(c, &c->mf_tot, nsl * 2));
    TRYC(cudaMemsetAsync(c->mf_tot, 0, nsl * 2 * sizeof(int32_t), st));
    TRY(dalloc(c, &c->mf_crow, nsl * c->mf_rcap));
    TRY(dalloc(c, &c->mf_cptr, nsl * (c->mf_rcap + 1)));
    TRY(dalloc(c, &c->mf_ebuck, nsl * c->mf_ecap));
    TRYC(pmalloc(c, (void**)&c->mf_eval, nsl * c->mf_ecap * c->elem()));
    TRYC(pmalloc(c, (void**)&c->mf_v, (size_t)c->n * c->elem()));
    TRYC(cudaMemsetAsync(c->mf_v, 0, (size_t)c->n * c->elem(), st));
    TRYC(pmalloc(c, (void**)&c->mf_pu, std::max<int64_t>(c->sx_npieces, 1) * c->elem()));
  }
  if (t_batch_member && !c->sparse) {
    // M^+ in the batch iteration kernel's type (FP32 in mixed precision), formed in
    // the factor's precision
    const size_t fel = c->f64_factor() ? 8 : 4;
    c->pld = round_up(c->tau, 4);
    c->p_slot = c->tau * c->pld;
    TRYC(pmalloc(c, (void**)&c->Pm, (size_t)c->nslots * c->p_slot * (c->mixed() ? 4 : 8)));
    // FP32 M^+ by sweeps (every phase-1 path of a member writes the FP32 M they read)
    c->sweep_p = c->mixed() && !c->f64_factor() && c->tau <= kSweepMaxTau;
    if (c->sweep_p) TRY(dalloc(c, &c->Mf, (size_t)c->nslots * c->tau * c->tau));
    else if (c->tau <= 4096) {
      c->potri = true;
      if (potri_needs_ws(c->tau, fel))
        TRYC(pmalloc(c, &c->pws, (size_t)c->nslots * potri_ws_elems(c->tau) * fel));
    }
  }
  if (!t_batch_member && !c->sparse && (sketch == RS_SUBSAMPLE || sketch == RS_COUNT || sketch == RS_SUBCOUNT) && o.iter_ctas >= 0) {
    // persistent iteration kernel over the whole GPU: S^T A blocked by CTA, M^+ per
    // slot and the all-reduce buffers
    bool fits = false;
    if (!c->mixed()) fits = wide_plan<double, double>(m, c->tau, o.iter_ctas, c->chunk, &c->wide);
    else fits = wide_plan<float, float>(m, c->tau, o.iter_ctas, c->chunk, &c->wide);
    if (fits) {
      const size_t fel = c->f64_factor() ? 8 : 4;
      c->pld = round_up(c->tau, 4);
      c->p_slot = c->tau * c->pld;
      TRYC(pmalloc(c, (void**)&c->Pm, (size_t)c->nslots * c->p_slot * (c->mixed() ? 4 : 8)));
      const size_t nwords = (size_t)2 * c->wide.nblk * (c->tau + 1) * 2;
      TRY(dalloc(c, &c->xpart, nwords));
      TRY(dalloc(c, &c->xflags, 1));
      TRY(dalloc(c, &c->xabort, 1));
      TRYC(cudaMemsetAsync(c->xpart, 0, nwords * sizeof(uint64_t), st));
      TRYC(cudaMemsetAsync(c->xflags, 0, sizeof(uint64_t), st));
      TRYC(cudaMemsetAsync(c->xabort, 0, sizeof(int32_t), st));
      c->use_wide = true;
      // FP32 M^+ by sweeps where S^T A and M are formed in one pass
      c->sweep_p = c->mixed() && !c->f64_factor() && c->tau <= kSweepMaxTau &&
                   sa_msys_fits<float>(m, c->tau, round_up((sketch == RS_COUNT) ? m : (sketch == RS_SUBCOUNT ? c->s : c->tau), 4));
      if (c->sweep_p) TRY(dalloc(c, &c->Mf, (size_t)c->nslots * c->tau * c->tau));
      // otherwise M^+ by factor, inverse and product in one kernel
      if (!c->sweep_p && c->tau <= 4096) {
        c->potri = true;
        if (potri_needs_ws(c->tau, fel))
          TRYC(pmalloc(c, &c->pws, (size_t)c->nslots * potri_ws_elems(c->tau) * fel));
      }
    } else {
      cudaGetLastError();
    }
  }
  {
    // per-slot buffers of phase 1 (sketched rows, M, inverse factor)
    const size_t fel = c->f64_factor() ? 8 : 4;
    if (c->use_wide) c->bq = c->wide.q;
    // batch members: one slice per CTA of the problem's cluster
    if (c->batch_member) c->bq = round_up((m + kBatchCluster - 1) / kBatchCluster, 4);
    if (c->bq > 0)
      c->sa_slot = (m + c->bq - 1) / c->bq * c->tau * round_up(c->bq, 4);
    else
      c->sa_slot = (sketch == RS_SUBSAMPLE && !c->batch_member) ? 0 : c->tau * c->ld;
    c->m_slot = c->tau * c->tau;
    c->l_slot = c->tau * c->tau;
    const size_t nsl = (size_t)c->nslots;
    TRY(dalloc(c, &c->M, nsl * c->m_slot));
    // L^{-1} per slot: for the factor-then-inverse paths and single-slot probes; a
    // batch member forms M^+ in one kernel (or by sweeps) and is never probed
    if (!(c->batch_member && (c->potri || c->sweep_p)))
      TRYC(pmalloc(c, (void**)&c->Linv, nsl * c->l_slot * fel));
    const size_t need_smem = (size_t)factor_ws_elems(c->tau) * fel + 4096;
    if (need_smem > 220 * 1024 || c->tau > 4096)
      TRYC(pmalloc(c, (void**)&c->fws, nsl * factor_ws_elems(c->tau) * fel));
    if (c->sa_slot > 0) {
      TRYC(pmalloc(c, (void**)&c->SA, nsl * c->sa_slot * c->elem()));
      TRYC(cudaMemsetAsync(c->SA, 0, nsl * c->sa_slot * c->elem(), st));
    }
    if (sketch == RS_GAUSSIAN) {
      TRYC(pmalloc(c, (void**)&c->ST, nsl * c->sa_slot * c->elem()));
      TRYC(cudaMemsetAsync(c->ST, 0, nsl * c->sa_slot * c->elem(), st));
      if (c->mixed()) {  // S^T A on the tensor cores
        TRY(dalloc(c, &c->tc_err, 1));
        TRYC(cudaMemsetAsync(c->tc_err, 0, sizeof(int32_t), st));
      }
    }
  }
  if (sketch != RS_GAUSSIAN) {
    c->perm_stride = round_up((sketch == RS_COUNT) ? m : (sketch == RS_SUBCOUNT ? c->s : c->tau), 4);
    c->boff_stride = round_up(c->tau + 1, 4);  // 16-byte aligned slots (bulk copies)
    TRY(dalloc(c, &c->perm, (size_t)c->perm_stride * c->nslots));
    TRY(dalloc(c, &c->boff, (size_t)c->boff_stride * c->nslots));
    // pool memory holds whatever a previous context left: the plans start as valid
    // (all-zero) indices, so that no read of a slot that was not drawn yet can
    // leave its buffers
    TRYC(cudaMemsetAsync(c->perm, 0, (size_t)c->perm_stride * c->nslots * sizeof(int32_t), st));
    TRYC(cudaMemsetAsync(c->boff, 0, (size_t)c->boff_stride * c->nslots * sizeof(int32_t), st));
    if (sketch != RS_SRHT) {
      TRY(dalloc(c, &c->inv, (size_t)c->ld * c->nslots));
      TRYC(cudaMemsetAsync(c->inv, 0, (size_t)c->ld * c->nslots * sizeof(int32_t), st));
    }
  }
  c->npartials = std::max<int64_t>(update_blocks(m), 256);
  TRY(dalloc(c, &c->partials, c->npartials));
  TRY(ensure_schedule(c, 1024));
  // ||b|| = ||r^0||
  {
    // ||b||: evaluate v + lambda x - b with v = x = 0 (u is all zeros here), r0 = 1
    double* zeros = c->u;
    TRYC(launch_refresh_finish(st, c->ctrl, 0, m, zeros, zeros, c->b, 0.0, nullptr, nullptr,
                               c->partials, nullptr, c->rel_dev));
    TRYC(cudaMemcpyAsync(c->scal_h, c->rel_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    TRYC(cudaStreamSynchronize(st));
    c->r0 = *c->scal_h;  // r0 was 1 in ctrl, so rel = ||b||
  }
  float ms = 0.f;
  TRYC(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->setup_ms = ms;
#undef TRY
#undef TRYC
  *out = c;
  return RS_OK;
}

void rs_destroy(rs_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard dg(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
  }
  delete ctx;
}

rs_status rs_trim_memory(int32_t device) {
  if (device < 0 || device >= 64) return RS_EINVAL;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    pool = g_pool[device];
  }
  if (pool == nullptr) return RS_OK;
  DeviceGuard dg(device);
  if (cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    set_global_error("rs_trim_memory: cudaMemPoolTrimTo failed");
    return RS_ECUDA;
  }
  return RS_OK;
}

rs_status rs_get_dims(const rs_ctx* c, int64_t* m, int64_t* tau, int64_t* s, int64_t* k_sum,
                      int64_t* m_pad) {
  if (!c) return RS_EINVAL;
  if (m) *m = c->m;
  if (tau) *tau = c->tau;
  if (s) *s = c->s;
  if (k_sum) *k_sum = c->kk;
  if (m_pad) *m_pad = c->mp;
  return RS_OK;
}

rs_status rs_solve(rs_ctx* c, double tol, int64_t max_iters, double* w_out, int32_t w_on_device,
                   double* hist_out, int64_t* iters_out) {
  if (!c) { set_global_error("rs_solve: null context"); return RS_EINVAL; }
  if (max_iters < 0 || !(tol >= 0.0)) FAILC(c, RS_EINVAL, "rs_solve: bad tol or max_iters");
  DeviceGuard dg(c->device);
  cudaStream_t st = c->stream;
  rs_status s;
  if ((s = ensure_schedule(c, std::max<int64_t>(max_iters, 1))) != RS_OK) return s;
  CKC(c, launch_init_state(st, c->m, c->b, c->w, c->wp, c->r, c->rp, c->u));
  // a timed-out earlier solve left the abort word raised
  if (c->xabort) CKC(c, cudaMemsetAsync(c->xabort, 0, sizeof(int32_t), st));
  if (c->avg) CKC(c, cudaMemsetAsync(c->wsum, 0, c->m * sizeof(double), st));  // w^0 = 0
  if (c->learned) CKC(c, cudaMemsetAsync(c->lp_last, 0xFF, c->m * sizeof(int32_t), st));
  if (!std::isfinite(c->r0)) {
    c->err = "rs_solve: NaN or Inf in b (||b|| is not finite)";
    return RS_ENUMERIC;
  }
  const double h0 = c->r0 > 0.0 ? 1.0 : 0.0;
  CKC(c, cudaMemcpyAsync(c->hist, &h0, sizeof(double), cudaMemcpyHostToDevice, st));
  CKC(c, cudaStreamSynchronize(st));
  int64_t iters = 0;
  rs_status result = RS_OK;
  float ms = 0.f;
  if (c->r0 == 0.0 || max_iters == 0) {
    iters = 0;
    if (c->r0 != 0.0 && tol < 1.0) result = RS_ENOTCONV;
  } else {
    Ctrl* h = c->ctrl_h;
    std::memset(h, 0, sizeof(Ctrl));
    h->max_iters = max_iters;
    h->r0 = c->r0;
    h->tol = tol;
    h->checked_k = -1;
    h->pk = -1;
    h->predict = !c->use_wide ? 0 : (c->mixed() ? 1 : 2);
    if ((s = write_ctrl(c)) != RS_OK) return s;
    CKC(c, cudaEventRecord(c->ev0, st));
    const int64_t max_chunks = (max_iters + c->chunk - 1) / c->chunk + 2;
    if ((s = run_loop(c, c->mixed(), max_chunks)) != RS_OK) return s;
    CKC(c, cudaEventRecord(c->ev1, st));
    CKC(c, cudaEventSynchronize(c->ev1));
    CKC(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    iters = h->k;
    int32_t gen_err = 0;
    CKC(c, copy_sync(c, &gen_err, c->err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (gen_err) FAILC(c, RS_ECUDA, "sketch generation: sample threshold search failed");
    if (c->tc_err != nullptr) {
      int32_t te = 0;
      CKC(c, copy_sync(c, &te, c->tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
      if (te) {
        CKC(c, cudaMemsetAsync(c->tc_err, 0, sizeof(int32_t), c->stream));
        FAILC(c, RS_ETIMEOUT, "rs_solve: a bounded wait of the tensor-core S^T A gave up");
      }
    }
    if (h->status == RS_ETIMEOUT) {
      FAILC(c, RS_ETIMEOUT, "rs_solve: a bounded device-side wait of the iteration kernel gave up");
    } else if (h->status == RS_ENUMERIC) {
      result = RS_ENUMERIC;
      c->err = "rs_solve: NaN or Inf in the residual";
    } else {
      double last = 0.0;
      if (c->mixed() && h->checked_k == iters) {
        // the last refresh already took the FP64 true residual of this iterate
        CKC(c, copy_sync(c, &last, c->hist + iters, sizeof(double), cudaMemcpyDeviceToHost));
      } else if (c->mixed()) {  // final FP64 residual check through X
        if ((s = true_rel(c, c->w, &last)) != RS_OK) return s;
        CKC(c, copy_sync(c, c->hist + iters, &last, sizeof(double), cudaMemcpyHostToDevice));
      } else {
        CKC(c, copy_sync(c, &last, c->hist + iters, sizeof(double), cudaMemcpyDeviceToHost));
      }
      if (!(last <= tol)) result = RS_ENOTCONV;
    }
  }
  c->solve_ms = ms;
  c->last_iters = iters;
  if ((s = copy_out_w(c, w_out, w_on_device)) != RS_OK) return s;
  if (hist_out) CKC(c, cudaMemcpyAsync(hist_out, c->hist, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  CKC(c, cudaStreamSynchronize(st));
  if (iters_out) *iters_out = iters;
  return result;
}

// ---- Conjugate Gradients on the same system (the competitor of Section 8.3) ----
namespace {
constexpr int kCgPlainSeg = 64;  // plain: iterations per captured segment
constexpr int kCgSegs = 4;       // segments per graph replay

// one CG iteration: direction, product with p . v, update with r . r and the stop test
rs_status enqueue_cg_iter(rs_ctx* c) {
  cudaStream_t st = c->stream;
  const int64_t m = c->m;
  float2* p2 = (c->mixed() && !c->sparse) ? c->cg_p2 : nullptr;
  CKC(c, launch_cg_dir(st, c->ctrl, c->cg_s, m, c->r, c->cg_p, p2));
  if (c->sparse) {  // A p = X^T (X p) + lambda p through the stored entries, FP64 sums
    rs_status s = with_vt(c, [&](auto tag) -> rs_status {
      using VT = std::remove_pointer_t<decltype(tag)>;
      const SparseX<VT> X = sparse_view<VT>(c);
      CKC(c, sparse_xv_d<VT>(st, X, c->cg_p, c->mf_z, &c->ctrl->stop));
      CKC(c, sparse_xtv_d<VT>(st, X, c->mf_z, c->cg_v, c->mf_pud, &c->ctrl->stop));
      return RS_OK;
    });
    if (s != RS_OK) return s;
    CKC(c, launch_cg_lam_dot(st, c->ctrl, m, c->lambda, c->cg_p, c->cg_v, c->cg_s, c->cg_part));
  } else if (c->mixed()) {
    CKC(c, launch_cg_matvec<float>(st, c->ctrl, static_cast<const float*>(c->A), c->ld, m, c->cg_p,
                                   p2, c->cg_v, c->cg_s, c->cg_part));
  } else {
    CKC(c, launch_cg_matvec<double>(st, c->ctrl, static_cast<const double*>(c->A), c->ld, m,
                                    c->cg_p, nullptr, c->cg_v, c->cg_s, c->cg_part));
  }
  CKC(c, launch_cg_update(st, c->ctrl, c->cg_s, m, c->cg_p, c->cg_v, c->w, c->r, c->cg_part,
                          c->hist, c->cg_refresh() ? 1 : 0));
  return RS_OK;
}

// a graph of kCgSegs segments; a segment is one refresh period followed by the FP64
// refresh (dense mixed) or kCgPlainSeg iterations (FP64 products)
rs_status build_cg_graph(rs_ctx* c) {
  if (c->cg_graph) return RS_OK;
  const int per = c->cg_refresh() ? c->refresh_every : kCgPlainSeg;
  CKC(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
  rs_status s = RS_OK;
  for (int q = 0; q < kCgSegs && s == RS_OK; ++q) {
    for (int i = 0; i < per && s == RS_OK; ++i) s = enqueue_cg_iter(c);
    if (s == RS_OK && c->cg_refresh()) {
      s = enqueue_refresh(c);  // r = A w - b through X in FP64; decides convergence
      if (s == RS_OK) {
        const cudaError_t e = launch_cg_rr(c->stream, c->ctrl, c->cg_s, c->m, c->r, 0);
        if (e != cudaSuccess) s = (c->err = std::string("cg: ") + cudaGetErrorString(e), RS_ECUDA);
      }
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (s != RS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) FAILC(c, RS_ECUDA, std::string("cg graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&c->cg_graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) FAILC(c, RS_ECUDA, std::string("cg graph: ") + cudaGetErrorString(e2));
  return RS_OK;
}
}  // namespace

rs_status rs_create_kernel(const rs_matrix* P, const double* y, int32_t y_on_device, double lambda,
                           double sigma, int32_t sketch, int64_t tau, const rs_mom* mom,
                           uint64_t seed, const rs_opts* opts, rs_ctx** out) {
  if (out) *out = nullptr;
  if (!P || !y || !out || P->is_csr || !P->val) {
    set_global_error("rs_create_kernel: need dense points, y and out");
    return RS_EINVAL;
  }
  if (!(sigma > 0.0) || !(lambda > 0.0) || P->n < 1 || P->d < 1) {
    set_global_error("rs_create_kernel: need sigma > 0, lambda > 0, n, d >= 1");
    return RS_EINVAL;
  }
  if (P->dtype != RS_F64 && P->dtype != RS_F32) {
    set_global_error("rs_create_kernel: points must be FP64 or FP32");
    return RS_EINVAL;
  }
  rs_opts o;
  rs_default_opts(&o);
  if (opts) o = *opts;
  const bool mixed = o.precision == RS_MIXED;
  const int64_t n = P->n, d = P->d;
  DeviceGuard dg(o.device);
  cudaStream_t st = static_cast<cudaStream_t>(o.cuda_stream);
  // temporary buffers of the set-up (the context copies K)
  const size_t pel = P->dtype == RS_F32 ? 4 : 8;
  const size_t kel = mixed ? 4 : 8;
  void *Pd = nullptr, *K = nullptr, *ws = nullptr;
  int32_t* err = nullptr;
  auto release = [&]() {
    if (Pd && !P->on_device) cudaFree(Pd);
    if (K) cudaFree(K);
    if (ws) cudaFree(ws);
    if (err) cudaFree(err);
  };
  cudaError_t e = cudaSuccess;
  const void* Pv = P->val;
  if (!P->on_device) {
    e = cudaMalloc(&Pd, (size_t)n * d * pel);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Pd, P->val, (size_t)n * d * pel, cudaMemcpyHostToDevice, st);
    Pv = Pd;
  }
  if (e == cudaSuccess) e = cudaMalloc(&K, (size_t)n * n * kel);
  if (e == cudaSuccess && mixed) {
    // FP32 points (a converted copy when given FP64), the tensor-core kernel matrix
    const float* Pf = static_cast<const float*>(Pv);
    float* conv = nullptr;
    if (P->dtype == RS_F64) {
      e = cudaMalloc((void**)&conv, (size_t)n * d * 4);
      if (e == cudaSuccess) e = launch_cast_f64_f32(st, static_cast<const double*>(Pv), (int64_t)n * d, conv);
      Pf = conv;
    }
    if (e == cudaSuccess) e = cudaMalloc(&ws, rbf_tc_ws_floats(n, d) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
      e = launch_rbf_tc(st, Pf, n, d, sigma, static_cast<float*>(K), n, static_cast<float*>(ws), err);
    if (e == cudaSuccess) e = launch_mirror_lower<float>(st, static_cast<float*>(K), n, n);
    int32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (conv) cudaFree(conv);
    if (e == cudaSuccess && bad) e = cudaErrorLaunchTimeout;
  } else if (e == cudaSuccess) {
    e = P->dtype == RS_F64
            ? launch_rbf_f64<double>(st, static_cast<const double*>(Pv), n, d, sigma,
                                     static_cast<double*>(K), n)
            : launch_rbf_f64<float>(st, static_cast<const float*>(Pv), n, d, sigma,
                                    static_cast<double*>(K), n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    release();
    set_global_error(std::string("rs_create_kernel: kernel matrix: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA;
  }
  // the ridge system with X = K (primal): A = K^T K + lambda I, b = K^T y; then
  // A += lambda (K - I) for A = K^T (K + lambda I) (eq. (kernelridge))
  rs_matrix Km{};
  Km.is_csr = 0;
  Km.dtype = mixed ? RS_F32 : RS_F64;
  Km.n = n;
  Km.d = n;
  Km.val = K;
  Km.on_device = 1;
  rs_ctx* c = nullptr;
  rs_status s = rs_create(&Km, y, y_on_device, lambda, RS_PRIMAL, sketch, tau, mom, seed, &o, &c);
  release();
  if (s != RS_OK) return s;
  c->kernel = true;
  cudaError_t e2 = mixed ? launch_add_offdiag<float>(c->stream, static_cast<float*>(c->A), c->ld,
                                                     static_cast<const float*>(c->X), n, n, lambda)
                         : launch_add_offdiag<double>(c->stream, static_cast<double*>(c->A), c->ld,
                                                      static_cast<const double*>(c->X), n, n, lambda);
  if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
  if (e2 != cudaSuccess) {
    set_global_error(std::string("rs_create_kernel: ") + cudaGetErrorString(e2));
    rs_destroy(c);
    return RS_ECUDA;
  }
  *out = c;
  return RS_OK;
}

rs_status rs_get_kernel(rs_ctx* c, double* K_out) {
  if (!c || !K_out) { set_global_error("rs_get_kernel: null argument"); return RS_EINVAL; }
  if (!c->kernel) FAILC(c, RS_EINVAL, "rs_get_kernel: not a kernel ridge context");
  DeviceGuard dg(c->device);
  const size_t nn = (size_t)c->n * c->n;
  if (c->xdtype == RS_F64) {
    CKC(c, copy_sync(c, K_out, c->X, nn * 8, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(nn);
    CKC(c, copy_sync(c, tmp.data(), c->X, nn * 4, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < nn; ++i) K_out[i] = (double)tmp[i];
  }
  return RS_OK;
}

rs_status rs_solve_cg(rs_ctx* c, double tol, int64_t max_iters, double* w_out, int32_t w_on_device,
                      double* hist_out, int64_t* iters_out) {
  if (!c) { set_global_error("rs_solve_cg: null context"); return RS_EINVAL; }
  if (max_iters < 0 || !(tol >= 0.0)) FAILC(c, RS_EINVAL, "rs_solve_cg: bad tol or max_iters");
  if (!c->sparse && c->A == nullptr) FAILC(c, RS_EUNSUPPORTED, "rs_solve_cg: no formed A");
  DeviceGuard dg(c->device);
  cudaStream_t st = c->stream;
  const int64_t m = c->m;
  rs_status s;
  if (!c->cg_p) {
    const int64_t np = std::max<int64_t>(cg_matvec_blocks(m), cg_blocks(m));
    if ((s = dalloc(c, &c->cg_p, m)) != RS_OK) return s;
    if ((s = dalloc(c, &c->cg_v, m)) != RS_OK) return s;
    if ((s = dalloc(c, &c->cg_part, np)) != RS_OK) return s;
    CKC(c, pmalloc(c, (void**)&c->cg_s, sizeof(CgScal)));
    CKC(c, pmalloc(c, (void**)&c->cg_p2, m * sizeof(float2)));
  }
  if ((s = ensure_schedule(c, std::max<int64_t>(max_iters, 1))) != RS_OK) return s;
  if (c->xabort) CKC(c, cudaMemsetAsync(c->xabort, 0, sizeof(int32_t), st));
  CKC(c, launch_init_state(st, m, c->b, c->w, c->wp, c->r, c->rp, c->u));  // w = 0, r = -b
  CKC(c, cudaMemsetAsync(c->cg_p, 0, m * sizeof(double), st));
  const double h0 = c->r0 > 0.0 ? 1.0 : 0.0;
  CKC(c, cudaMemcpyAsync(c->hist, &h0, sizeof(double), cudaMemcpyHostToDevice, st));
  Ctrl* h = c->ctrl_h;
  std::memset(h, 0, sizeof(Ctrl));
  h->max_iters = max_iters;
  h->r0 = c->r0 > 0.0 ? c->r0 : 1.0;
  h->tol = tol;
  h->checked_k = -1;
  h->pk = -1;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  CKC(c, launch_cg_rr(st, c->ctrl, c->cg_s, m, c->r, 1));
  CKC(c, cudaStreamSynchronize(st));
  if (!std::isfinite(c->r0)) {
    c->err = "rs_solve_cg: NaN or Inf in b (||b|| is not finite)";
    return RS_ENUMERIC;
  }
  int64_t iters = 0;
  rs_status result = RS_OK;
  float ms = 0.f;
  if (c->r0 == 0.0 || max_iters == 0) {
    if (c->r0 != 0.0 && tol < 1.0) result = RS_ENOTCONV;
  } else {
    if ((s = build_cg_graph(c)) != RS_OK) return s;
    const int per = c->cg_refresh() ? c->refresh_every : kCgPlainSeg;
    const int64_t per_graph = (int64_t)per * kCgSegs;
    CKC(c, cudaEventRecord(c->ev0, st));
    for (int64_t q = 0; q < max_iters / per_graph + 2; ++q) {
      CKC(c, cudaGraphLaunch(c->cg_graph, st));
      if ((s = read_ctrl(c)) != RS_OK) return s;
      if (h->stop) break;
    }
    CKC(c, cudaEventRecord(c->ev1, st));
    CKC(c, cudaEventSynchronize(c->ev1));
    CKC(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    iters = h->k;
    if (h->status == RS_ENUMERIC) {
      result = RS_ENUMERIC;
      c->err = "rs_solve_cg: NaN or Inf in the residual";
    } else {
      double last = 0.0;
      if (c->cg_refresh() && h->checked_k != iters) {  // final FP64 residual through X
        if ((s = true_rel(c, c->w, &last)) != RS_OK) return s;
        CKC(c, copy_sync(c, c->hist + iters, &last, sizeof(double), cudaMemcpyHostToDevice));
      } else {
        CKC(c, copy_sync(c, &last, c->hist + iters, sizeof(double), cudaMemcpyDeviceToHost));
      }
      if (!(last <= tol)) result = RS_ENOTCONV;
    }
  }
  c->solve_ms = ms;
  c->last_iters = iters;
  if ((s = copy_out_w(c, w_out, w_on_device)) != RS_OK) return s;
  if (hist_out) CKC(c, cudaMemcpyAsync(hist_out, c->hist, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  CKC(c, cudaStreamSynchronize(st));
  if (iters_out) *iters_out = iters;
  return result;
}

rs_status rs_set_acceleration(rs_ctx* c, double mu, double nu) {
  if (!c) { set_global_error("rs_set_acceleration: null context"); return RS_EINVAL; }
  DeviceGuard dg(c->device);
  if (mu == 0.0 && nu == 0.0) {  // back to Algorithm 2
    c->accel = false;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return RS_OK;
  }
  if (!(mu > 0.0 && mu <= 1.0 && nu >= 1.0 && nu * mu <= 1.0 + 1e-12))
    FAILC(c, RS_EINVAL, "rs_set_acceleration: need 0 < mu <= 1 <= nu <= 1 / mu");
  if (!c->use_wide)
    FAILC(c, RS_EUNSUPPORTED, "rs_set_acceleration: needs the persistent iteration kernel "
                              "(subsample, count or subcount sketch of dense A)");
  // Algorithm 3: beta = 1 - sqrt(mu / nu), gamma = sqrt(1 / (mu nu)),
  // alpha = 1 / (1 + sqrt(nu / mu))
  c->acc_b = 1.0 - std::sqrt(mu / nu);
  c->acc_g = std::sqrt(1.0 / (mu * nu));
  c->acc_a = 1.0 / (1.0 + std::sqrt(nu / mu));
  c->accel = true;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return RS_OK;
}

rs_status rs_set_averaging(rs_ctx* c, int32_t on) {
  if (!c) { set_global_error("rs_set_averaging: null context"); return RS_EINVAL; }
  DeviceGuard dg(c->device);
  if (!on) { c->avg = false; return RS_OK; }
  if (!c->use_wide)
    FAILC(c, RS_EUNSUPPORTED, "rs_set_averaging: needs the persistent iteration kernel "
                              "(subsample, count or subcount sketch of dense A)");
  if (!c->wsum) {
    rs_status s = dalloc(c, &c->wsum, c->m);
    if (s != RS_OK) return s;
  }
  c->avg = true;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }  // kernels read wsum
  return RS_OK;
}

rs_status rs_get_average(rs_ctx* c, double* w_out, int32_t w_on_device) {
  if (!c || !w_out) { set_global_error("rs_get_average: null argument"); return RS_EINVAL; }
  if (!c->avg) FAILC(c, RS_EINVAL, "rs_get_average: averaging is off (rs_set_averaging)");
  DeviceGuard dg(c->device);
  // mean of w^0..w^t (t iterations) into u, then out as w (dual: X^T of the mean)
  CKC(c, launch_scale(c->stream, c->wsum, 1.0 / (double)(c->last_iters + 1), c->m, c->u));
  double* keep = c->w;
  c->w = c->u;
  rs_status s = copy_out_w(c, w_out, w_on_device);
  c->w = keep;
  if (s != RS_OK) return s;
  CKC(c, cudaStreamSynchronize(c->stream));
  CKC(c, cudaMemsetAsync(c->u, 0, c->m * sizeof(double), c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status rs_chunking(const rs_ctx* c, int64_t* chunk, int32_t* refresh_every,
                      int32_t* fused_potri) {
  if (!c) return RS_EINVAL;
  if (chunk) *chunk = c->chunk;
  if (refresh_every) *refresh_every = c->mixed() ? c->refresh_every : 0;
  if (fused_potri) *fused_potri = c->potri ? 1 : 0;
  return RS_OK;
}

rs_status rs_iter_plan(const rs_ctx* c, int32_t* ctas, int64_t* q) {
  if (!c) return RS_EINVAL;
  if (ctas) *ctas = c->use_wide ? c->wide.nblk : 0;
  if (q) *q = c->bq;
  return RS_OK;
}

rs_status rs_dump_sketch(rs_ctx* c, int64_t k, int32_t* idx, int8_t* sign, int32_t* bucket) {
  if (!c || k < 0) return RS_EINVAL;
  if (c->sketch == RS_GAUSSIAN) FAILC(c, RS_EINVAL, "rs_dump_sketch: use rs_dump_gaussian");
  DeviceGuard dg(c->device);
  rs_status s = enqueue_gen(c, k, 1);
  if (s != RS_OK) return s;
  std::vector<int32_t> perm(c->perm_stride), boff(c->boff_stride);
  CKC(c, cudaMemcpyAsync(perm.data(), c->perm, perm.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaMemcpyAsync(boff.data(), c->boff, boff.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  int32_t gen_err = 0;
  CKC(c, copy_sync(c, &gen_err, c->err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (gen_err) FAILC(c, RS_ECUDA, "sketch generation: sample threshold search failed");
  auto row = [](int32_t e) { return e & 0x7FFFFFFF; };
  switch (c->sketch) {
    case RS_SUBSAMPLE:
      if (idx) for (int64_t j = 0; j < c->tau; ++j) idx[j] = row(perm[j]);
      break;
    case RS_SUBCOUNT:
      for (int64_t p = 0; p < c->s; ++p) {
        if (idx) idx[p] = row(perm[p]);
        if (sign) sign[p] = perm[p] < 0 ? -1 : 1;
        if (bucket) bucket[p] = (int32_t)(p / c->kk);
      }
      break;
    case RS_SRHT:
      if (idx) for (int64_t j = 0; j < c->tau; ++j) idx[j] = row(perm[j]);
      if (sign)
        for (int64_t i = 0; i < c->m; ++i)
          sign[i] = draw_neg(draw_k(iter_key(c->seed, k), 1, (uint64_t)i)) ? -1 : 1;
      break;
    case RS_COUNT:
      for (int64_t b = 0; b < c->tau; ++b)
        for (int32_t t = boff[b]; t < boff[b + 1]; ++t) {
          const int32_t i = row(perm[t]);
          if (i < 0 || i >= c->m) FAILC(c, RS_ECUDA, "rs_dump_sketch: corrupt count plan");
          if (bucket) bucket[i] = (int32_t)b;
          if (sign) sign[i] = perm[t] < 0 ? -1 : 1;
        }
      if (idx) for (int64_t t = 0; t < c->m; ++t) idx[t] = row(perm[t]);
      break;
  }
  return RS_OK;
}

rs_status rs_dump_gaussian(rs_ctx* c, int64_t k, double* S) {
  if (!c || k < 0 || !S) return RS_EINVAL;
  if (c->sketch != RS_GAUSSIAN) FAILC(c, RS_EINVAL, "rs_dump_gaussian: not a Gaussian sketch");
  DeviceGuard dg(c->device);
  const size_t n = (size_t)c->tau * c->ld;
  std::vector<double> st(n);
  if (c->mixed()) {
    CKC(c, launch_gen_gauss<float>(c->stream, c->ctrl, 1, 1, k, c->seed, c->m, c->tau,
                                   static_cast<float*>(c->ST), c->ld, c->sa_slot));
    std::vector<float> tmp(n);
    CKC(c, cudaMemcpyAsync(tmp.data(), c->ST, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < n; ++i) st[i] = tmp[i];
  } else {
    CKC(c, launch_gen_gauss<double>(c->stream, c->ctrl, 1, 1, k, c->seed, c->m, c->tau,
                                    static_cast<double*>(c->ST), c->ld, c->sa_slot));
    CKC(c, cudaMemcpyAsync(st.data(), c->ST, n * 8, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaStreamSynchronize(c->stream));
  }
  for (int64_t i = 0; i < c->m; ++i)
    for (int64_t j = 0; j < c->tau; ++j) S[i * c->tau + j] = st[j * c->ld + i];
  return RS_OK;
}

rs_status rs_get_state(rs_ctx* c, double* w, double* w_prev, double* r, double* r_prev, int64_t* k) {
  if (!c) return RS_EINVAL;
  DeviceGuard dg(c->device);
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  const size_t bytes = c->m * sizeof(double);
  if (w) CKC(c, cudaMemcpyAsync(w, c->w, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (w_prev) CKC(c, cudaMemcpyAsync(w_prev, c->wp, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (r) CKC(c, cudaMemcpyAsync(r, c->r, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (r_prev) CKC(c, cudaMemcpyAsync(r_prev, c->rp, bytes, cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  if (k) *k = c->ctrl_h->k;
  return RS_OK;
}

rs_status rs_set_state(rs_ctx* c, const double* w, const double* w_prev, const double* r,
                       const double* r_prev, int64_t k) {
  if (!c || !w || !w_prev || !r || !r_prev || k < 0) return RS_EINVAL;
  DeviceGuard dg(c->device);
  const size_t bytes = c->m * sizeof(double);
  CKC(c, cudaMemcpyAsync(c->w, w, bytes, cudaMemcpyHostToDevice, c->stream));
  CKC(c, cudaMemcpyAsync(c->wp, w_prev, bytes, cudaMemcpyHostToDevice, c->stream));
  CKC(c, cudaMemcpyAsync(c->r, r, bytes, cudaMemcpyHostToDevice, c->stream));
  CKC(c, cudaMemcpyAsync(c->rp, r_prev, bytes, cudaMemcpyHostToDevice, c->stream));
  CKC(c, cudaMemsetAsync(c->u, 0, bytes, c->stream));
  if (c->learned) CKC(c, cudaMemsetAsync(c->lp_last, 0xFF, c->m * sizeof(int32_t), c->stream));
  std::memset(c->ctrl_h, 0, sizeof(Ctrl));
  c->ctrl_h->k = k;
  c->ctrl_h->k0 = k;
  c->ctrl_h->max_iters = INT64_MAX;
  c->ctrl_h->r0 = c->r0 > 0.0 ? c->r0 : 1.0;
  c->ctrl_h->no_stop = 1;
  rs_status s = write_ctrl(c);
  if (s != RS_OK) return s;
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status rs_probe_step(rs_ctx* c, double* M, double* r_S, double* delta) {
  if (!c) return RS_EINVAL;
  DeviceGuard dg(c->device);
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  const int64_t k = c->ctrl_h->k;
  if ((s = enqueue_phase1(c, 1, k, 1)) != RS_OK) return s;
  if ((s = enqueue_delta(c, 1, k)) != RS_OK) return s;
  const size_t t = c->tau;
  if (M) CKC(c, cudaMemcpyAsync(M, c->M, t * t * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (r_S) CKC(c, cudaMemcpyAsync(r_S, c->rS, t * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (delta) CKC(c, cudaMemcpyAsync(delta, c->delta, t * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaMemsetAsync(c->u, 0, c->m * sizeof(double), c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status rs_step(rs_ctx* c, int64_t n_iters, double* hist_out) {
  if (!c || n_iters < 0) return RS_EINVAL;
  if (n_iters == 0) return RS_OK;
  DeviceGuard dg(c->device);
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  const int64_t k0 = c->ctrl_h->k;
  if ((s = ensure_schedule(c, k0 + n_iters)) != RS_OK) return s;
  Ctrl* h = c->ctrl_h;
  h->stop = 0;
  h->pending = 0;
  h->status = 0;
  h->ticket = 0;
  h->no_stop = 1;
  h->predict = 0;  // every chunk runs to its end
  h->kcap = 0;
  h->max_iters = k0 + n_iters;
  h->r0 = c->r0 > 0.0 ? c->r0 : 1.0;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  if (c->xabort) CKC(c, cudaMemsetAsync(c->xabort, 0, sizeof(int32_t), c->stream));
  const int64_t chunks = (n_iters + c->chunk - 1) / c->chunk + 1;
  for (int64_t q = 0; q < chunks; ++q) {
    if ((s = enqueue_chunk(c, false)) != RS_OK) return s;
    if ((s = read_ctrl(c)) != RS_OK) return s;
    if (h->stop) break;
  }
  if (h->status == RS_ETIMEOUT) FAILC(c, RS_ETIMEOUT, "rs_step: a bounded device-side wait gave up");
  if (h->status == RS_ENUMERIC) FAILC(c, RS_ENUMERIC, "rs_step: NaN or Inf in the residual");
  if (hist_out)
    CKC(c, copy_sync(c, hist_out, c->hist + k0 + 1, n_iters * sizeof(double), cudaMemcpyDeviceToHost));
  // leave the context ready for further steps or probes
  h->stop = 0;
  h->max_iters = INT64_MAX;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status rs_true_residual(rs_ctx* c, const double* v, double* rel_out) {
  if (!c || !v || !rel_out) return RS_EINVAL;
  DeviceGuard dg(c->device);
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  Ctrl saved = *c->ctrl_h;
  c->ctrl_h->r0 = c->r0 > 0.0 ? c->r0 : 1.0;
  c->ctrl_h->ticket = 0;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  CKC(c, cudaMemcpyAsync(c->u, v, c->m * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  double rel = 0.0;
  if ((s = true_rel(c, c->u, &rel)) != RS_OK) return s;
  CKC(c, cudaMemsetAsync(c->u, 0, c->m * sizeof(double), c->stream));
  *c->ctrl_h = saved;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  CKC(c, cudaStreamSynchronize(c->stream));
  *rel_out = rel;
  return RS_OK;
}

rs_status rs_profile_iteration(rs_ctx* c, int64_t reps, rs_kernel_stat* out, int32_t cap,
                               int32_t* n_out) {
  if (!c || reps <= 0 || !out || !n_out || cap <= 0) return RS_EINVAL;
  DeviceGuard dg(c->device);
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  const int64_t k0 = c->ctrl_h->k;
  if ((s = ensure_schedule(c, k0 + reps + c->chunk + 2)) != RS_OK) return s;
  Ctrl* h = c->ctrl_h;
  h->stop = 0; h->pending = 0; h->status = 0; h->ticket = 0; h->no_stop = 1;
  h->predict = 0; h->kcap = 0;
  // past the profiled iterations, so that no kernel of the last chunk sees the cap
  // (the refresh after it would return at once)
  h->max_iters = k0 + reps + c->chunk + 1;
  h->r0 = c->r0 > 0.0 ? c->r0 : 1.0;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  struct Grp { const char* name; double ms = 0; int64_t n = 0; double bytes = 0, flops = 0; int64_t iters = 0; };
  std::vector<Grp> g;
  auto grp = [&](const char* nm) -> Grp& {
    for (auto& x : g) if (std::strcmp(x.name, nm) == 0) return x;
    g.push_back(Grp{nm});
    return g.back();
  };
  cudaEvent_t e0, e1;
  CKC(c, cudaEventCreate(&e0));
  CKC(c, cudaEventCreate(&e1));
  auto timed = [&](const char* nm, auto&& fn) -> rs_status {
    cudaError_t e = cudaEventRecord(e0, c->stream);
    if (e != cudaSuccess) FAILC(c, RS_ECUDA, "event");
    rs_status r = fn();
    if (r != RS_OK) return r;
    e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) FAILC(c, RS_ECUDA, std::string("profile: ") + cudaGetErrorString(e));
    Grp& x = grp(nm);
    x.ms += ms;
    x.n += 1;
    return RS_OK;
  };
  const double el = (double)c->elem();
  const double fel = c->f64_factor() ? 8.0 : 4.0;
  const double pel = (c->use_wide && c->mixed()) ? 4.0 : fel;  // M^+ as the iterations read it
  const double m = (double)c->m, tau = (double)c->tau;
  const int ns = (int)c->nslots;
  const double rows = c->sketch == RS_COUNT ? m : (c->sketch == RS_SUBCOUNT ? (double)c->s : tau);
  for (int64_t it = 0; it < reps && s == RS_OK; ++it) {
    if (c->sparse) {  // matrix-free: phase 1 of the chunk, then one group per iteration
      if (it % c->chunk == 0) {
        s = timed("phase1", [&]() -> rs_status {
          CKC(c, launch_chunk_begin(c->stream, c->ctrl));
          return enqueue_phase1(c, 0, -1, ns, true);
        });
        if (s != RS_OK) break;
      }
      s = timed("mf_iter", [&]() { return enqueue_mf_iteration(c); });
      // per iteration: X restricted to the sampled columns' rows is touched through
      // the compact rows; X^T v reads every stored entry once
      grp("mf_iter").bytes += (double)c->nnz * (4.0 + (c->xdtype == RS_BF16 ? 2.0 : (c->xdtype == RS_F32 ? 4.0 : 8.0))) + m * 48.0;
      grp("mf_iter").iters += 1;
      if (s == RS_OK && c->mixed() && (it + 1) % c->refresh_every == 0)
        s = timed("refresh", [&]() { return enqueue_refresh(c); });
      continue;
    }
    if (it % c->chunk == 0) {
      const double nsl = (double)std::min<int64_t>(ns, reps - it);
      const PlanView plan = plan_view(c);
      if (c->sketch == RS_GAUSSIAN || c->sketch == RS_SRHT) {
        // one group for the whole phase 1 of these sketches
        s = timed("phase1", [&]() -> rs_status {
          CKC(c, launch_chunk_begin(c->stream, c->ctrl));
          return enqueue_phase1(c, 0, -1, ns);
        });
        if (s != RS_OK) break;
      } else {
        s = timed("gen", [&]() -> rs_status {
          CKC(c, launch_chunk_begin(c->stream, c->ctrl));
          const rs_status r = enqueue_gen(c, -1, ns);
          if (r != RS_OK) return r;
          // the row -> bucket map of the new plans, as in the chunk's phase 1
          if (c->inv != nullptr)
            CKC(c, launch_inv_map(c->stream, c->ctrl, 0, ns, plan, c->m, c->tau,
                                  c->sketch == RS_COUNT ? 1 : 0, c->inv, c->ld));
          return RS_OK;
        });
        if (s != RS_OK) break;
        const bool has_sa = c->sketch == RS_COUNT || c->sketch == RS_SUBCOUNT || c->use_wide;
        const int64_t bq = c->bq;
        const bool fused = has_sa && (c->mixed() ? sa_msys_fits<float>(c->m, c->tau, c->perm_stride)
                                                 : sa_msys_fits<double>(c->m, c->tau, c->perm_stride));
        if (fused) {
          // S^T A and M in one pass: A rows read once per slot, S^T A written once
          s = timed("sa_msys", [&]() -> rs_status {
            if (c->mixed())
              CKC(c, launch_sa_msys<float>(c->stream, c->ctrl, 0, ns, plan, static_cast<const float*>(c->A), c->ld, c->m, c->tau, static_cast<float*>(c->SA), c->ld, c->sa_slot, bq, c->M, c->m_slot, c->sweep_p ? c->Mf : nullptr));
            else
              CKC(c, launch_sa_msys<double>(c->stream, c->ctrl, 0, ns, plan, static_cast<const double*>(c->A), c->ld, c->m, c->tau, static_cast<double*>(c->SA), c->ld, c->sa_slot, bq, c->M, c->m_slot));
            return RS_OK;
          });
          grp("sa_msys").bytes += nsl * (rows * m * el + tau * m * el + rows * 4.0 + tau * tau * 8.0);
          grp("sa_msys").flops += nsl * (rows * m + tau * rows);
          if (s != RS_OK) break;
        } else {
          if (has_sa) {
            s = timed("sa", [&]() -> rs_status {
              if (c->mixed())
                CKC(c, launch_sa_batched<float>(c->stream, c->ctrl, 0, ns, plan, static_cast<const float*>(c->A), c->ld, c->m, c->tau, static_cast<float*>(c->SA), c->ld, c->sa_slot, bq));
              else
                CKC(c, launch_sa_batched<double>(c->stream, c->ctrl, 0, ns, plan, static_cast<const double*>(c->A), c->ld, c->m, c->tau, static_cast<double*>(c->SA), c->ld, c->sa_slot, bq));
              return RS_OK;
            });
            grp("sa").bytes += nsl * (rows * m * el + tau * m * el + rows * 4.0);
            grp("sa").flops += nsl * rows * m;
            if (s != RS_OK) break;
          }
          s = timed("msys", [&]() -> rs_status {
            if (c->mixed()) CKC(c, launch_msys_batched<float>(c->stream, c->ctrl, 0, ns, plan, rows_view<float>(c), c->m, c->tau, c->M, c->m_slot));
            else CKC(c, launch_msys_batched<double>(c->stream, c->ctrl, 0, ns, plan, rows_view<double>(c), c->m, c->tau, c->M, c->m_slot));
            return RS_OK;
          });
          grp("msys").bytes += nsl * ((c->sketch == RS_SUBSAMPLE ? tau * tau * el : tau * m * el + rows * 4.0) + tau * tau * 8.0);
          grp("msys").flops += nsl * (c->sketch == RS_SUBSAMPLE ? 0.0 : tau * rows);
          if (s != RS_OK) break;
        }
        const bool sweep = c->sweep_p;
        if (sweep) {
          s = timed("sweep", [&]() -> rs_status {
            CKC(c, launch_sweep_inv(c->stream, c->ctrl, 0, ns, c->Mf, c->m_slot, c->tau, static_cast<float*>(c->Pm), c->pld, c->p_slot, c->ndropped));
            return RS_OK;
          });
          grp("sweep").bytes += nsl * tau * tau * (8.0 + 4.0);
          grp("sweep").flops += nsl * tau * tau * tau;
          if (s != RS_OK) break;
        }
        if (!sweep && c->use_wide && c->potri) {
          // factor, inverse and M^+ in one kernel
          s = timed("potri", [&]() { return enqueue_potri(c, c->stream, 0, ns); });
          // Cholesky tau^3 / 3, triangular inverse tau^3 / 3, L^{-T} L^{-1} tau^3 / 3
          grp("potri").bytes += nsl * (tau * tau * (8.0 + fel));
          grp("potri").flops += nsl * (tau * tau * tau);
          if (s != RS_OK) break;
        } else {
        if (!sweep) s = timed("factor", [&]() -> rs_status {
          if (c->f64_factor())
            CKC(c, launch_factor_inv<double>(c->stream, c->ctrl, 0, ns, c->M, c->m_slot, c->tau, static_cast<double*>(c->Linv), c->l_slot, static_cast<double*>(c->fws), c->ndropped));
          else
            CKC(c, launch_factor_inv<float>(c->stream, c->ctrl, 0, ns, c->M, c->m_slot, c->tau, static_cast<float*>(c->Linv), c->l_slot, static_cast<float*>(c->fws), c->ndropped));
          return RS_OK;
        });
        if (!sweep) {
          grp("factor").bytes += nsl * (tau * tau * (8.0 + fel));
          grp("factor").flops += nsl * (2.0 * tau * tau * tau / 3.0);
        }
        if (s != RS_OK) break;
        if (c->use_wide && !sweep) {
          s = timed("pinv", [&]() -> rs_status {
            if (c->f64_factor())
              CKC(c, launch_pinv<double>(c->stream, c->ctrl, 0, ns, static_cast<const double*>(c->Linv), c->l_slot, c->tau, static_cast<double*>(c->Pm), c->pld, c->p_slot));
            else
              CKC(c, launch_pinv<float>(c->stream, c->ctrl, 0, ns, static_cast<const float*>(c->Linv), c->l_slot, c->tau, static_cast<float*>(c->Pm), c->pld, c->p_slot));
            return RS_OK;
          });
          grp("pinv").bytes += nsl * (tau * tau * 2.0 * fel);
          grp("pinv").flops += nsl * (2.0 * tau * tau * tau);
          if (s != RS_OK) break;
        }
        }
      }
    }
    if (c->sketch != RS_SRHT) {
      // fused: the chunk's iterations in one launch per refresh period (mixed) or one
      // launch for the whole chunk (plain); every launch runs to its end
      const int64_t per = c->mixed() ? std::min<int64_t>(c->refresh_every, c->chunk) : c->chunk;
      int64_t done = 0;
      for (int64_t off = 0; off < c->chunk && it + done < reps && s == RS_OK; off += per) {
        const int64_t e = std::min<int64_t>(off + per, c->chunk);
        const int64_t nit = e - off;
        s = timed("iterate", [&]() { return enqueue_iterate(c, e); });
        // algorithmic HBM bytes: S^T A (or the sampled rows of A) and the small system
        // of every iteration; the persistent kernel reads and writes w, w_prev, r,
        // r_prev once per launch, the cluster kernel every iteration
        grp("iterate").bytes += c->use_wide
            ? (double)nit * (tau * m * el + tau * tau * pel + 4.0 * m) + 64.0 * m
            : (double)nit * (tau * m * el + tau * tau * fel + 80.0 * m);
        grp("iterate").flops += (double)nit * (2.0 * tau * m + 2.0 * tau * tau + 10.0 * m);
        grp("iterate").iters += nit;
        done += nit;
        if (s == RS_OK && c->mixed()) {
          s = timed("refresh", [&]() { return enqueue_refresh(c); });
          grp("refresh").bytes += (double)c->n * (double)c->d * (c->xdtype == RS_F32 ? 4.0 : 8.0) + m * 48.0;
          grp("refresh").flops += 4.0 * (double)c->n * (double)c->d;
        }
      }
      it += done - 1;
      continue;
    }
    s = timed("delta", [&]() { return enqueue_delta(c, 0, -1); });
    grp("delta").bytes += tau * tau * fel / 2.0 + rows * 12.0 + m * 8.0;
    grp("delta").flops += 2.0 * tau * tau;
    if (s != RS_OK) break;
    s = timed("update", [&]() { return enqueue_update(c); });
    grp("update").bytes += (c->sketch == RS_SUBSAMPLE ? tau * m * el : tau * m * el) + m * 8.0 * 9.0;
    grp("update").flops += 2.0 * tau * m + 10.0 * m;
    if (s == RS_OK && c->mixed() && (it + 1) % c->refresh_every == 0) {
      s = timed("refresh", [&]() { return enqueue_refresh(c); });
      grp("refresh").bytes += 2.0 * (double)c->n * (double)c->d * (c->xdtype == RS_F32 ? 4.0 : 8.0) + m * 48.0;
      grp("refresh").flops += 4.0 * (double)c->n * (double)c->d;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != RS_OK) return s;
  int32_t n = 0;
  for (auto& x : g) {
    if (n >= cap) break;
    rs_kernel_stat& o = out[n++];
    std::memset(&o, 0, sizeof(o));
    std::strncpy(o.name, x.name, sizeof(o.name) - 1);
    o.launches = x.n;
    o.ms = x.n ? x.ms / x.n : 0.0;
    // per launch, averaged like the times (a chunk's last launch may be shorter)
    o.bytes = x.n ? x.bytes / x.n : 0.0;
    o.flops = x.n ? x.flops / x.n : 0.0;
    o.iters = x.iters > 0 ? x.iters : x.n;
  }
  *n_out = n;
  h->stop = 0;
  h->max_iters = INT64_MAX;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

static rs_status lp_alloc(rs_ctx* c);

rs_status rs_set_proposal(rs_ctx* c, const uint16_t* w_bf16, double eps) {
  if (!c) { set_global_error("rs_set_proposal: null context"); return RS_EINVAL; }
  DeviceGuard dg(c->device);
  if (eps < 0.0) {  // back to the plain sampler
    c->learned = false;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return RS_OK;
  }
  if (c->sketch != RS_SUBSAMPLE || c->sparse)
    FAILC(c, RS_EUNSUPPORTED, "rs_set_proposal: the learned proposal draws subsample sketches of dense A");
  if (!(eps <= 1.0)) FAILC(c, RS_EINVAL, "rs_set_proposal: eps must be in [0, 1]");
  int64_t np2 = 1;
  while (np2 < c->m) np2 <<= 1;
  if (np2 * 8 > 200 * 1024) FAILC(c, RS_EUNSUPPORTED, "rs_set_proposal: m > 16384");
  rs_status s0 = lp_alloc(c);
  if (s0 != RS_OK) return s0;
  cudaStream_t st = c->stream;
  c->lp_uniform = (w_bf16 == nullptr);
  if (w_bf16) CKC(c, cudaMemcpyAsync(c->lp_w, w_bf16, kMlpParams * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
  c->lp_eps = (float)eps;
  c->lp_fixed = false;
  c->learned = true;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  CKC(c, cudaStreamSynchronize(st));
  return RS_OK;
}

// buffers of the scored proposal and the static features (once per context)
static rs_status lp_alloc(rs_ctx* c) {
  cudaStream_t st = c->stream;
  const size_t m = (size_t)c->m;
  if (!c->lp_w) {
    CKC(c, pmalloc(c, (void**)&c->lp_w, kMlpParams * sizeof(uint16_t)));
    CKC(c, pmalloc(c, (void**)&c->lp_raw, 2 * m * sizeof(float)));
    CKC(c, pmalloc(c, (void**)&c->lp_zstat, 2 * m * sizeof(float)));
    CKC(c, pmalloc(c, (void**)&c->lp_stats, 8 * sizeof(double)));
    CKC(c, pmalloc(c, (void**)&c->lp_score, m * sizeof(float)));
    CKC(c, pmalloc(c, (void**)&c->lp_feat, m * 4 * sizeof(float)));
    CKC(c, pmalloc(c, (void**)&c->lp_last, m * sizeof(int32_t)));
    CKC(c, cudaMemsetAsync(c->lp_last, 0xFF, m * sizeof(int32_t), st));
    if (c->mixed())
      CKC(c, launch_lp_static<float>(st, static_cast<const float*>(c->A), c->ld, c->m, c->lp_raw,
                                     c->lp_zstat));
    else
      CKC(c, launch_lp_static<double>(st, static_cast<const double*>(c->A), c->ld, c->m, c->lp_raw,
                                      c->lp_zstat));
  }
  return RS_OK;
}

rs_status rs_collect(rs_ctx* c, const double* w_star, int64_t n_iters, double tol, float* Z_out,
                     float* y_out, int64_t* n_rows) {
  if (!c || !w_star || !Z_out || !y_out || !n_rows || n_iters < 0 || !(tol >= 0.0)) {
    set_global_error("rs_collect: bad arguments");
    return RS_EINVAL;
  }
  *n_rows = 0;
  if (!c->learned || c->lp_fixed)
    FAILC(c, RS_EINVAL, "rs_collect: needs a proposal (rs_set_proposal, weights or uniform)");
  if (c->mixed() || c->chunk != 1 || c->mom.kind != RS_MOM_NONE)
    FAILC(c, RS_EINVAL, "rs_collect: needs plain FP64, chunk = 1 and no momentum (the "
                        "projection identity of the labels)");
  if (n_iters == 0) return RS_OK;
  DeviceGuard dg(c->device);
  cudaStream_t st = c->stream;
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  const int64_t k0 = c->ctrl_h->k;
  if ((s = ensure_schedule(c, k0 + n_iters + 2)) != RS_OK) return s;
  const int64_t cap = n_iters * c->tau;
  double *ws = nullptr, *e2 = nullptr;
  float *Zd = nullptr, *yd = nullptr;
  int64_t* cnt = nullptr;
  auto release = [&]() { pfree(c, ws); pfree(c, e2); pfree(c, Zd); pfree(c, yd); pfree(c, cnt); };
  if ((s = dalloc(c, &ws, c->m)) != RS_OK || (s = dalloc(c, &e2, 1)) != RS_OK ||
      (s = dalloc(c, &Zd, cap * 4)) != RS_OK || (s = dalloc(c, &yd, cap)) != RS_OK ||
      (s = dalloc(c, &cnt, 1)) != RS_OK) {
    release();
    return s;
  }
  // the same control state as rs_step: every iteration runs until the collection stops
  Ctrl* h = c->ctrl_h;
  h->stop = 0; h->pending = 0; h->status = 0; h->ticket = 0; h->no_stop = 1;
  h->predict = 0; h->kcap = 0;
  h->max_iters = k0 + n_iters;
  h->r0 = c->r0 > 0.0 ? c->r0 : 1.0;
  cudaError_t e = cudaMemcpyAsync(ws, w_star, c->m * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) { release(); FAILC(c, RS_ECUDA, std::string("rs_collect: ") + cudaGetErrorString(e)); }
  if ((s = write_ctrl(c)) != RS_OK) { release(); return s; }
  for (int64_t it = 0; it < n_iters && s == RS_OK; ++it) {
    const int64_t k = k0 + it;
    // ||e_k||_A^2 and the stop test; the features and the rows drawn at k; the step's
    // r_C and delta; the labels; then the iteration itself
    e = launch_collect_pre(st, c->ctrl, c->w, ws, c->r, c->m, tol, e2);
    if (e == cudaSuccess)
      e = launch_lp_features(st, c->ctrl, k, c->lp_zstat, c->lp_raw, c->lp_stats, c->r, c->lp_last,
                             c->m, c->lp_score, c->lp_feat);
    if (e != cudaSuccess) break;
    if ((s = enqueue_phase1(c, 1, k, 1)) != RS_OK) break;
    if ((s = enqueue_delta(c, 1, k)) != RS_OK) break;
    e = cudaMemsetAsync(c->u, 0, c->m * sizeof(double), st);
    if (e == cudaSuccess)
      e = launch_collect_rows(st, c->ctrl, c->perm, c->boff, c->tau, c->lp_feat, c->rS, c->delta,
                              e2, c->m, cap, Zd, yd, cnt);
    if (e != cudaSuccess) break;
    s = enqueue_chunk(c, false);
    if (s == RS_OK && it % 64 == 63) {  // stop enqueueing once the device has stopped
      if ((s = read_ctrl(c)) != RS_OK) break;
      if (h->stop) break;
    }
  }
  if (s != RS_OK) { release(); return s; }
  if (e != cudaSuccess) { release(); FAILC(c, RS_ECUDA, std::string("rs_collect: ") + cudaGetErrorString(e)); }
  int64_t n = 0;
  e = cudaMemcpyAsync(&n, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(Z_out, Zd, n * 4 * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(y_out, yd, n * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) FAILC(c, RS_ECUDA, std::string("rs_collect: ") + cudaGetErrorString(e));
  if ((s = read_ctrl(c)) != RS_OK) return s;
  if (h->status == RS_ETIMEOUT) FAILC(c, RS_ETIMEOUT, "rs_collect: a bounded device-side wait gave up");
  *n_rows = n;
  // leave the context ready for further steps or probes
  h->stop = 0;
  h->max_iters = INT64_MAX;
  if ((s = write_ctrl(c)) != RS_OK) return s;
  CKC(c, cudaStreamSynchronize(st));
  return RS_OK;
}

rs_status rs_set_sampling(rs_ctx* c, int32_t kind) {
  if (!c) { set_global_error("rs_set_sampling: null context"); return RS_EINVAL; }
  DeviceGuard dg(c->device);
  if (kind == RS_SAMPLE_UNIFORM) {  // the sketch's own uniform draws
    c->learned = false;
    c->lp_fixed = false;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return RS_OK;
  }
  if (kind != RS_SAMPLE_DIAG) FAILC(c, RS_EINVAL, "rs_set_sampling: unknown sampling");
  if (c->sketch != RS_SUBSAMPLE || c->sparse)
    FAILC(c, RS_EUNSUPPORTED, "rs_set_sampling: importance sampling draws subsample sketches of dense A");
  int64_t np2 = 1;
  while (np2 < c->m) np2 <<= 1;
  if (np2 * 8 > 200 * 1024) FAILC(c, RS_EUNSUPPORTED, "rs_set_sampling: m > 16384");
  rs_status s = lp_alloc(c);
  if (s != RS_OK) return s;
  if (c->mixed())
    CKC(c, launch_lp_diag_score<float>(c->stream, static_cast<const float*>(c->A), c->ld, c->m,
                                       c->lp_score));
  else
    CKC(c, launch_lp_diag_score<double>(c->stream, static_cast<const double*>(c->A), c->ld, c->m,
                                        c->lp_score));
  c->lp_uniform = true;  // no network: the scores stay ln A_jj
  c->lp_eps = 0.0f;
  c->lp_fixed = true;
  c->learned = true;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status rs_proposal_features(rs_ctx* c, float* Z_out) {
  if (!c || !Z_out) return RS_EINVAL;
  if (!c->learned || c->lp_fixed) FAILC(c, RS_EINVAL, "rs_proposal_features: no learned proposal set");
  DeviceGuard dg(c->device);
  rs_status s = read_ctrl(c);
  if (s != RS_OK) return s;
  CKC(c, launch_lp_features(c->stream, c->ctrl, c->ctrl_h->k, c->lp_zstat, c->lp_raw, c->lp_stats,
                            c->r, c->lp_last, c->m, c->lp_score, c->lp_feat));
  CKC(c, cudaMemcpyAsync(Z_out, c->lp_feat, c->m * 4 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return RS_OK;
}

rs_status rs_timings(const rs_ctx* c, double* setup_ms, double* solve_ms) {
  if (!c) return RS_EINVAL;
  if (setup_ms) *setup_ms = c->setup_ms;
  if (solve_ms) *solve_ms = c->solve_ms;
  return RS_OK;
}

}  // extern "C"


// ===========================================================================
// batches of problems (rs_create_batch / rs_solve_batch)
//
// Problem p is a member context (A_p, b_p of its first right-hand side, its sketch
// sequence seed + p, per-slot S^T A and M^+); its right-hand sides share them. One
// chunk of the batch, captured once as a CUDA graph:
//   phase 1 of every member (chunk_begin, plans, S^T A and M, M^+), spread over
//   side streams by balanced d^2 (longest first);
//   the batch's persistent iteration kernel (CTA per problem);
//   mixed: w in FP64, X^T X w per pair through X on the member's stream, the FP64
//   refresh of every pair;
//   the finish kernel (problems whose pairs are all done stop; counts for the host).
// The autotuner times whole chunks for each (iteration CTA size, side streams)
// candidate on the first solve and keeps the fastest.
// ===========================================================================
struct rs_batch {
  int P = 0, nrhs = 0;
  int precision = 0;
  int64_t chunk = 50, tau_max = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<rs_ctx*> mem;            // one member context per problem
  std::vector<unsigned char*> state;   // per problem: 48 bytes per (right-hand side, coordinate)
  void* probs = nullptr;               // device BatchProb (plain) or BatchProbM (mixed) array
  void* refs = nullptr;                // device BatchRef or BatchRefM array, P * nrhs
  rs::Ctrl** ctrls = nullptr;          // device: the members' control blocks
  int32_t *flag = nullptr, *skip = nullptr;
  int64_t* iters = nullptr;
  double *r0 = nullptr, *resid = nullptr;
  double* tol = nullptr;               // device: tolerance of the current solve
  int32_t* fin = nullptr;              // device: problems running, failed pairs, timeouts
  int32_t* fin_h = nullptr;            // pinned copy
  int32_t* alive = nullptr;            // device: 1 while problem p runs
  int32_t* order = nullptr;            // device: problems of the captured chunk, largest first
  std::vector<int32_t> order_h;        // host copy; its first nrun entries are captured
  int nrun = 0;
  int32_t* err_word = nullptr;         // device: an iteration kernel gave up a bounded wait
  std::vector<double*> xpart;          // per phase-1 stream: X^T X W partial sums (mixed)
  std::vector<float2*> xu;             // per phase-1 stream: X W as float pairs (mixed)
  int64_t bq_max = 0, d_max = 0, perm_max = 0, pld_max = 0;
  // the small solves of all running problems in one launch (every member forms M^+ by
  // factor, inverse and product): the members' jobs and the launch's tile work space
  bool potri_batch = false;
  rs::PotriJob* pjobs = nullptr;
  void* pbws = nullptr;
  std::vector<cudaStream_t> side;      // phase-1 fan-out streams
  std::vector<cudaEvent_t> evs;        // fork / join events (timing disabled)
  cudaGraphExec_t graph = nullptr;
  const double* graph_gam = nullptr;   // momentum table the graph was captured with
  int graph_threads = 0, graph_streams = 0, graph_nrun = 0;
  bool tuned = false;
  int threads = 256;                   // CTA size of the iteration kernel (tuned)
  int nstreams = 1;                    // side streams of phase 1 (tuned)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double setup_ms = 0.0, solve_ms = 0.0, tune_ms = 0.0;
  std::string tune_cache;              // file of the autotuner's choices ("" = none)
  bool tune_cached = false;            // the choice of this batch came from that file
  int sketch = 0;
  std::string err;
  bool mixed() const { return precision == RS_MIXED; }
};

namespace {

std::string g_batch_err;
constexpr int kBatchMaxStreams = 4;

rs::BatchPairs batch_pairs(const rs_batch* b) {
  rs::BatchPairs p{};
  p.flag = b->flag; p.skip = b->skip; p.iters = b->iters; p.r0 = b->r0; p.resid = b->resid;
  return p;
}

void batch_free(rs_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (rs_ctx* c : b->mem) rs_destroy(c);
  for (unsigned char* p : b->state) if (p) cudaFree(p);
  void* ptrs[] = {b->probs, b->refs, b->ctrls, b->flag, b->skip, b->iters, b->r0, b->resid,
                  b->tol, b->fin, b->alive, b->order, b->err_word, b->pjobs, b->pbws};
  for (void* p : ptrs) if (p) cudaFree(p);
  for (double* p : b->xpart) if (p) cudaFree(p);
  for (float2* p : b->xu) if (p) cudaFree(p);
  if (b->fin_h) cudaFreeHost(b->fin_h);
  for (cudaStream_t s : b->side) if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->evs) if (e) cudaEventDestroy(e);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

#define BKC(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return (e_ == cudaErrorMemoryAllocation) ? RS_ENOMEM : RS_ECUDA;             \
    }                                                                             \
  } while (0)

// byte offsets of the per-problem state (v = nrhs * d entries per array):
//   plain  w, w_prev, r, r_prev, b (FP64 each; the sixth array unused)
//   mixed  w (float pair), r (float pair), Delta_w, Delta_r (FP32), w (FP64), b, X^T X w
rs_status batch_upload(rs_batch* b) {
  const size_t np = (size_t)b->P * b->nrhs;
  std::vector<rs::Ctrl*> ctrls(b->P);
  for (int p = 0; p < b->P; ++p) ctrls[p] = b->mem[p]->ctrl;
  BKC(cudaMalloc(&b->ctrls, b->P * sizeof(rs::Ctrl*)));
  BKC(cudaMemcpy(b->ctrls, ctrls.data(), b->P * sizeof(rs::Ctrl*), cudaMemcpyHostToDevice));
  auto fill = [&](auto& q, const rs_ctx* c) {
    q.d = c->m; q.tau = c->tau; q.bq = c->bq; q.sa_slot = c->sa_slot; q.pld = c->pld;
    q.p_slot = c->p_slot; q.perm_stride = c->perm_stride; q.boff_stride = c->boff_stride;
    q.inv_slot = c->ld;
    q.perm = c->perm; q.boff = c->boff; q.inv = c->inv;
    q.ctrl = c->ctrl;
  };
  if (b->mixed()) {
    std::vector<rs::BatchProbC<float>> h(b->P);
    std::vector<rs::BatchRefM> f(np);
    for (int p = 0; p < b->P; ++p) {
      const rs_ctx* c = b->mem[p];
      const size_t v = (size_t)b->nrhs * c->m;
      unsigned char* base = b->state[p];
      rs::BatchProbC<float>& q = h[p];
      q = {};
      fill(q, c);
      q.SA = static_cast<const float*>(c->SA); q.P = static_cast<const float*>(c->Pm);
      q.w2 = reinterpret_cast<float2*>(base);
      q.r2 = reinterpret_cast<float2*>(base + 8 * v);
      q.dw = reinterpret_cast<float*>(base + 16 * v);
      q.dr = reinterpret_cast<float*>(base + 20 * v);
      for (int r = 0; r < b->nrhs; ++r) {
        rs::BatchRefM& g = f[(size_t)p * b->nrhs + r];
        const size_t o = (size_t)r * c->m;
        g.d = c->m; g.pair = p * b->nrhs + r; g.lambda = c->lambda;
        g.w2 = q.w2 + o; g.r2 = q.r2 + o; g.dw = q.dw + o; g.dr = q.dr + o;
        g.wd = reinterpret_cast<double*>(base + 24 * v) + o;
        g.b = reinterpret_cast<const double*>(base + 32 * v) + o;
        g.v = reinterpret_cast<const double*>(base + 40 * v) + o;
      }
    }
    BKC(cudaMalloc(&b->probs, h.size() * sizeof(h[0])));
    BKC(cudaMemcpy(b->probs, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice));
    BKC(cudaMalloc(&b->refs, f.size() * sizeof(f[0])));
    BKC(cudaMemcpy(b->refs, f.data(), f.size() * sizeof(f[0]), cudaMemcpyHostToDevice));
  } else {
    std::vector<rs::BatchProbC<double>> h(b->P);
    std::vector<rs::BatchRef> f(np);
    for (int p = 0; p < b->P; ++p) {
      const rs_ctx* c = b->mem[p];
      const size_t v = (size_t)b->nrhs * c->m;
      double* base = reinterpret_cast<double*>(b->state[p]);
      rs::BatchProbC<double>& q = h[p];
      q = {};
      fill(q, c);
      q.SA = static_cast<const double*>(c->SA); q.P = static_cast<const double*>(c->Pm);
      q.w = base; q.wp = base + v; q.r = base + 2 * v; q.rp = base + 3 * v;
      for (int r = 0; r < b->nrhs; ++r) {
        rs::BatchRef& g = f[(size_t)p * b->nrhs + r];
        const size_t o = (size_t)r * c->m;
        g.d = c->m; g.pair = p * b->nrhs + r; g.lambda = c->lambda;
        g.w = q.w + o; g.wp = q.wp + o; g.r = q.r + o; g.rp = q.rp + o; g.b = base + 4 * v + o;
      }
    }
    BKC(cudaMalloc(&b->probs, h.size() * sizeof(h[0])));
    BKC(cudaMemcpy(b->probs, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice));
    BKC(cudaMalloc(&b->refs, f.size() * sizeof(f[0])));
    BKC(cudaMemcpy(b->refs, f.data(), f.size() * sizeof(f[0]), cudaMemcpyHostToDevice));
  }
  // one launch for the small solves of all members (each with the same chunk)
  bool all_potri = true;
  for (const rs_ctx* c : b->mem) all_potri = all_potri && c->potri && !c->sweep_p && !c->sparse;
  if (all_potri) {
    std::vector<rs::PotriJob> j(b->P);
    for (int p = 0; p < b->P; ++p) {
      const rs_ctx* c = b->mem[p];
      j[p] = rs::PotriJob{c->M, c->m_slot, c->tau, c->Pm, c->pld, c->p_slot, c->ndropped, c->ctrl};
    }
    BKC(cudaMalloc(&b->pjobs, j.size() * sizeof(j[0])));
    BKC(cudaMemcpy(b->pjobs, j.data(), j.size() * sizeof(j[0]), cudaMemcpyHostToDevice));
    const size_t fel = b->mem[0]->f64_factor() ? 8 : 4;
    BKC(cudaMalloc(&b->pbws, (size_t)rs::potri_batch_ctas() * rs::potri_ws_elems(b->tau_max) * fel));
    b->potri_batch = true;
  }
  return RS_OK;
}

// the small solves of the running problems of a chunk, one launch (potri_batch)
rs_status batch_enqueue_potri(rs_batch* b) {
  const rs_ctx* c0 = b->mem[0];
  if (c0->f64_factor() && b->mixed())
    BKC((rs::launch_potri_batch<double, float>(b->stream, b->pjobs, b->order, b->nrun,
                                               (int)b->chunk, b->tau_max,
                                               static_cast<double*>(b->pbws))));
  else if (c0->f64_factor())
    BKC((rs::launch_potri_batch<double, double>(b->stream, b->pjobs, b->order, b->nrun,
                                                (int)b->chunk, b->tau_max,
                                                static_cast<double*>(b->pbws))));
  else
    BKC((rs::launch_potri_batch<float, float>(b->stream, b->pjobs, b->order, b->nrun,
                                              (int)b->chunk, b->tau_max,
                                              static_cast<float*>(b->pbws))));
  return RS_OK;
}

// the problems a chunk graph covers: those of `alive` (all when null), largest first
rs_status batch_set_order(rs_batch* b, const int32_t* alive) {
  b->order_h.clear();
  for (int p = 0; p < b->P; ++p)
    if (!alive || alive[p]) b->order_h.push_back(p);
  std::stable_sort(b->order_h.begin(), b->order_h.end(),
                   [&](int x, int y) { return b->mem[x]->m > b->mem[y]->m; });
  b->nrun = (int)b->order_h.size();
  if (b->nrun > 0)
    BKC(cudaMemcpy(b->order, b->order_h.data(), b->nrun * sizeof(int32_t), cudaMemcpyHostToDevice));
  return RS_OK;
}

// fresh state of every pair and every member's control block (k = 0)
rs_status batch_reset(rs_batch* b, double tol, int64_t max_iters) {
  const rs::BatchPairs pr = batch_pairs(b);
  const int np = b->P * b->nrhs;
  if (b->mixed())
    BKC(rs::launch_batch_mixed_aux(b->stream, 0, static_cast<const rs::BatchRefM*>(b->refs), np, pr, b->tol));
  else
    BKC(rs::launch_batch_init(b->stream, static_cast<const rs::BatchRef*>(b->refs), np, pr));
  BKC(cudaMemcpyAsync(b->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, b->stream));
  BKC(cudaMemsetAsync(b->err_word, 0, sizeof(int32_t), b->stream));
  for (rs_ctx* c : b->mem) {
    std::memset(c->ctrl_h, 0, sizeof(rs::Ctrl));
    c->ctrl_h->max_iters = max_iters;
    c->ctrl_h->r0 = 1.0;
    c->ctrl_h->tol = tol;
    BKC(cudaMemcpyAsync(c->ctrl, c->ctrl_h, sizeof(rs::Ctrl), cudaMemcpyHostToDevice, b->stream));
  }
  BKC(cudaStreamSynchronize(b->stream));
  return RS_OK;
}

// phase-1 stream of each captured problem: longest processing time first over d_p^2
// (order_h is sorted by d, largest first)
std::vector<int> batch_owners(const rs_batch* b, int ns) {
  std::vector<int> owner(b->P, 0);
  std::vector<double> load(ns, 0.0);
  for (int t = 0; t < b->nrun; ++t) {
    const int p = b->order_h[t];
    int best = 0;
    for (int i = 1; i < ns; ++i) if (load[i] < load[best]) best = i;
    owner[p] = best;
    load[best] += (double)b->mem[p]->m * (double)b->mem[p]->m;
  }
  return owner;
}

rs_status batch_fork(rs_batch* b, int ns, int ev) {
  if (ns <= 1) return RS_OK;
  BKC(cudaEventRecord(b->evs[ev], b->stream));
  for (int i = 1; i < ns; ++i) BKC(cudaStreamWaitEvent(b->side[i - 1], b->evs[ev], 0));
  return RS_OK;
}

rs_status batch_join(rs_batch* b, int ns, int ev) {
  for (int i = 1; i < ns; ++i) {
    BKC(cudaEventRecord(b->evs[ev + i], b->side[i - 1]));
    BKC(cudaStreamWaitEvent(b->stream, b->evs[ev + i], 0));
  }
  return RS_OK;
}

// parts of a chunk (batch_enqueue_chunk)
constexpr int kPartPhase1 = 1, kPartIterate = 2, kPartRefresh = 4, kPartAll = 7;

// one chunk of the captured problems (enqueued on b->stream, or captured from it);
// `parts` selects phase 1, the iterations and the refresh with the end-of-chunk
// bookkeeping
rs_status batch_enqueue_chunk(rs_batch* b, int threads, int ns, int parts = kPartAll,
                              int p1_stages = kP1All) {
  const std::vector<int> owner = batch_owners(b, ns);
  auto stream_of = [&](int p) { return owner[p] == 0 ? b->stream : b->side[owner[p] - 1]; };
  const rs::BatchPairs pr = batch_pairs(b);
  const int np = b->P * b->nrhs;
  rs_status s;
  if (parts & kPartPhase1) {
  // with potri_batch the members stop before their small solves, which then run for
  // all of them in one launch on the batch's stream
  const int mstages = b->potri_batch ? (p1_stages & ~kP1Inv) : p1_stages;
  if (mstages != 0) {
    if ((s = batch_fork(b, ns, 0)) != RS_OK) return s;
    for (int t = 0; t < b->nrun; ++t) {
      const int p = b->order_h[t];
      rs_ctx* c = b->mem[p];
      cudaStream_t st = stream_of(p);
      if (p1_stages & kP1Plan) BKC(launch_chunk_begin(st, c->ctrl));
      c->stream = st;
      s = enqueue_phase1(c, 0, -1, (int)c->nslots, true, mstages);
      c->stream = b->stream;
      if (s != RS_OK) { b->err = c->err; return s; }
    }
    if ((s = batch_join(b, ns, 0)) != RS_OK) return s;
  }
  if (b->potri_batch && (p1_stages & kP1Inv) && (s = batch_enqueue_potri(b)) != RS_OK) return s;
  }
  const double* gam = b->mem[0]->gam;
  const double* bet = b->mem[0]->bet;
  if ((parts & kPartIterate) && b->mixed())
    BKC((rs::launch_batch_cluster<float, true>(
        b->stream, static_cast<const rs::BatchProbC<float>*>(b->probs), b->order, b->nrun, b->nrhs,
        pr, gam, bet, b->chunk, b->tol, b->tau_max, b->bq_max, b->perm_max, b->pld_max, threads,
        b->err_word)));
  if ((parts & kPartIterate) && !b->mixed())
    BKC((rs::launch_batch_cluster<double, false>(
        b->stream, static_cast<const rs::BatchProbC<double>*>(b->probs), b->order, b->nrun,
        b->nrhs, pr, gam, bet, b->chunk, b->tol, b->tau_max, b->bq_max, b->perm_max, b->pld_max,
        threads, b->err_word)));
  if (!(parts & kPartRefresh)) return RS_OK;
  if (b->mixed()) {
    const rs::BatchRefM* refs = static_cast<const rs::BatchRefM*>(b->refs);
    // FP64 refresh: w in FP64, X^T X W of each problem in one pass over X (four
    // right-hand sides at a time), r = X^T X w + lambda w - b
    BKC(rs::launch_batch_mixed_aux(b->stream, 1, refs, np, pr, b->tol));
    if ((s = batch_fork(b, ns, kBatchMaxStreams)) != RS_OK) return s;
    for (int t = 0; t < b->nrun; ++t) {
      const int p = b->order_h[t];
      rs_ctx* c = b->mem[p];
      const size_t v = (size_t)b->nrhs * c->m;
      const double* wd = reinterpret_cast<const double*>(b->state[p] + 24 * v);
      double* xv = reinterpret_cast<double*>(b->state[p] + 40 * v);
      for (int q0 = 0; q0 < b->nrhs; q0 += 4)
        BKC(launch_xtx_two_pass(stream_of(p), static_cast<const float*>(c->X), c->n, c->d,
                                std::min(4, b->nrhs - q0), wd + (size_t)q0 * c->m,
                                xv + (size_t)q0 * c->m, b->xu[owner[p]], b->xpart[owner[p]],
                                b->skip + p * b->nrhs + q0));
    }
    if ((s = batch_join(b, ns, kBatchMaxStreams)) != RS_OK) return s;
    BKC(rs::launch_batch_mixed_aux(b->stream, 3, refs, np, pr, b->tol));
  }
  BKC(rs::launch_batch_finish(b->stream, b->ctrls, b->P, b->nrhs, pr, b->alive, b->fin));
  return RS_OK;
}

// capture `parts` of one chunk into *out
rs_status batch_capture(rs_batch* b, int threads, int ns, int parts, cudaGraphExec_t* out,
                        int p1_stages = kP1All) {
  BKC(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
  const rs_status s = batch_enqueue_chunk(b, threads, ns, parts, p1_stages);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (s != RS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    b->err = std::string("batch graph capture: ") + cudaGetErrorString(e);
    return RS_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    *out = nullptr;
    b->err = std::string("batch graph instantiate: ") + cudaGetErrorString(ei);
    return RS_ECUDA;
  }
  return RS_OK;
}

rs_status batch_build_graph(rs_batch* b, int threads, int ns) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  const rs_status s = batch_capture(b, threads, ns, kPartAll, &b->graph);
  if (s != RS_OK) return s;
  b->graph_gam = b->mem[0]->gam;
  b->graph_threads = threads;
  b->graph_streams = ns;
  b->graph_nrun = b->nrun;
  return RS_OK;
}

// replay chunks until every problem has stopped (at most max_replays); when the
// problems still running are half of those the graph covers or fewer, the graph
// is captured again over them only
rs_status batch_run(rs_batch* b, int64_t max_replays) {
  std::vector<int32_t> alive(b->P);
  for (int64_t q = 0; q < max_replays; ++q) {
    BKC(cudaGraphLaunch(b->graph, b->stream));
    BKC(cudaMemcpyAsync(b->fin_h, b->fin, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
    BKC(cudaStreamSynchronize(b->stream));
    if (b->fin_h[2] > 0) {
      b->err = "rs_solve_batch: a bounded device-side wait of the iteration kernel gave up";
      return RS_ETIMEOUT;
    }
    const int run = b->fin_h[0];
    if (run == 0) return RS_OK;
    if (2 * run <= b->nrun) {
      BKC(cudaMemcpy(alive.data(), b->alive, b->P * sizeof(int32_t), cudaMemcpyDeviceToHost));
      rs_status s = batch_set_order(b, alive.data());
      if (s == RS_OK) s = batch_build_graph(b, b->threads, b->nstreams);
      if (s != RS_OK) return s;
    }
  }
  return RS_OK;
}

bool batch_fits(const rs_batch* b, int threads) {
  return (b->mixed() ? rs::batch_cluster_fit<float, true>(b->nrhs, b->tau_max, b->bq_max,
                                                          b->perm_max, b->pld_max, threads)
                     : rs::batch_cluster_fit<double, false>(b->nrhs, b->tau_max, b->bq_max,
                                                            b->perm_max, b->pld_max, threads)) > 0;
}

// The autotuner's cache: one line per batch shape, "<key> <threads> <streams>". The
// key holds everything the choice depends on (problem count and sizes, right-hand
// sides, precision, sketch, chunk, and the GPU's SM count).
std::string batch_tune_key(const rs_batch* b) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  char buf[256];
  std::snprintf(buf, sizeof(buf), "v1:P=%d:nrhs=%d:prec=%d:sketch=%d:chunk=%lld:tau=%lld:bq=%lld:"
                "d=%lld:perm=%lld:pld=%lld:sms=%d", b->P, b->nrhs, b->precision, b->sketch,
                (long long)b->chunk, (long long)b->tau_max, (long long)b->bq_max,
                (long long)b->d_max, (long long)b->perm_max, (long long)b->pld_max, nsm);
  return buf;
}

bool tune_cache_read(const std::string& path, const std::string& key, int* threads, int* streams) {
  std::FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return false;
  char k[256];
  int t = 0, n = 0;
  bool found = false;
  while (std::fscanf(f, "%255s %d %d", k, &t, &n) == 3)
    if (key == k) { *threads = t; *streams = n; found = true; }  // the last line wins
  std::fclose(f);
  return found;
}

// rewrites the file with this key's line replaced (best effort: a failure to write
// leaves the tuning in effect for this batch only)
void tune_cache_write(const std::string& path, const std::string& key, int threads, int streams) {
  std::vector<std::string> keep;
  if (std::FILE* f = std::fopen(path.c_str(), "r")) {
    char k[256];
    int t = 0, n = 0;
    while (std::fscanf(f, "%255s %d %d", k, &t, &n) == 3)
      if (key != k) keep.push_back(std::string(k) + " " + std::to_string(t) + " " + std::to_string(n));
    std::fclose(f);
  }
  keep.push_back(key + " " + std::to_string(threads) + " " + std::to_string(streams));
  const std::string tmp = path + ".tmp";
  std::FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  bool ok = true;
  for (const std::string& l : keep) ok = ok && std::fprintf(f, "%s\n", l.c_str()) > 0;
  ok = (std::fclose(f) == 0) && ok;
  if (ok) std::rename(tmp.c_str(), path.c_str());
  else std::remove(tmp.c_str());
}

// autotuner: one steady-state chunk (tol = 0, no pair stops) per candidate CTA size
// of the iteration kernel and number of phase-1 streams; keeps the fastest. With a
// cache file, a shape tuned before is taken from it (if it still fits) and a new
// choice is written to it.
rs_status batch_tune(rs_batch* b) {
  const std::string key = b->tune_cache.empty() ? std::string() : batch_tune_key(b);
  if (!key.empty()) {
    int t = 0, ns = 0;
    if (tune_cache_read(b->tune_cache, key, &t, &ns) && (t == 128 || t == 256 || t == 512) &&
        ns >= 1 && ns <= kBatchMaxStreams && (ns == 1 || ns <= b->P) && b->bq_max <= 4 * t &&
        batch_fits(b, t)) {
      b->threads = t;
      b->nstreams = ns;
      b->tuned = true;
      b->tune_cached = true;
      return RS_OK;
    }
  }
  const int thr[] = {128, 256, 512};
  const int nss[] = {1, 2, kBatchMaxStreams};
  float best = -1.f;
  int bt = 256, bs = 1;
  rs_status s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BKC(cudaEventCreate(&e0));
  BKC(cudaEventCreate(&e1));
  auto done = [&](rs_status r) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
  };
  for (int ns : nss) {
    if (ns > 1 && ns > b->P) continue;
    for (int t : thr) {
      if (b->bq_max > 4 * t || !batch_fits(b, t)) continue;
      if ((s = batch_reset(b, 0.0, 2 * b->chunk)) != RS_OK) return done(s);
      if ((s = batch_build_graph(b, t, ns)) != RS_OK) return done(s);
      cudaError_t e = cudaGraphLaunch(b->graph, b->stream);  // first replay: uploads the graph
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        b->err = std::string("batch autotuner: ") + cudaGetErrorString(e);
        return done(RS_ECUDA);
      }
      if (best < 0.f || ms < best) { best = ms; bt = t; bs = ns; }
    }
  }
  if (best < 0.f) {
    b->err = "batch autotuner: no launch shape of the iteration kernel fits";
    return done(RS_EUNSUPPORTED);
  }
  b->threads = bt;
  b->nstreams = bs;
  b->tuned = true;
  b->tune_cached = false;
  if (!key.empty()) tune_cache_write(b->tune_cache, key, bt, bs);
  return done(RS_OK);
}

}  // namespace

namespace {

// members, state, B of every right-hand side, device pair arrays
rs_status batch_init(rs_batch* b, const rs_matrix* Xs, const double* const* Ys,
                     int32_t y_on_device, const double* lambdas, int32_t sketch,
                     const int64_t* taus, const rs_mom* mom, uint64_t seed, rs_opts o) {
  const int P = b->P, nrhs = b->nrhs;
  if (o.cuda_stream) {
    b->stream = static_cast<cudaStream_t>(o.cuda_stream);
  } else {
    BKC(cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault));  // as rs_create's own stream
    b->own_stream = true;
  }
  BKC(cudaEventCreate(&b->ev0));
  BKC(cudaEventCreate(&b->ev1));
  b->side.assign(kBatchMaxStreams - 1, nullptr);
  for (cudaStream_t& s : b->side) BKC(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  b->evs.assign(2 * kBatchMaxStreams, nullptr);
  for (cudaEvent_t& e : b->evs) BKC(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  o.cuda_stream = b->stream;
  o.iter_ctas = -1;
  BKC(cudaEventRecord(b->ev0, b->stream));
  // member contexts: A_p, b_p of the first right-hand side, per-slot buffers with M^+.
  // The members share one chunk length: where the memory cap shortened some
  // members' chunks, all are made again with the shortest.
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (rs_ctx* c : b->mem) rs_destroy(c);
    b->mem.assign(P, nullptr);
    for (int p = 0; p < P; ++p) {
      rs_ctx* c = nullptr;
      t_batch_member = true;
      const rs_status s = rs_create(&Xs[p], Ys[p], y_on_device, lambdas[p], RS_PRIMAL, sketch,
                                    taus ? taus[p] : 0, mom, seed + (uint64_t)p, &o, &c);
      t_batch_member = false;
      if (s != RS_OK) {
        b->err = std::string("problem ") + std::to_string(p) + ": " + rs_last_error(nullptr);
        return s;
      }
      b->mem[p] = c;
    }
    int64_t lo = b->mem[0]->chunk, hi = lo;
    for (rs_ctx* c : b->mem) {
      lo = std::min<int64_t>(lo, c->chunk);
      hi = std::max<int64_t>(hi, c->chunk);
    }
    if (lo == hi) break;
    if (attempt == 1) { b->err = "rs_create_batch: members with different chunks"; return RS_EINVAL; }
    o.chunk = lo;
  }
  b->chunk = b->mem[0]->chunk;
  for (rs_ctx* c : b->mem) {
    b->tau_max = std::max<int64_t>(b->tau_max, c->tau);
    b->bq_max = std::max<int64_t>(b->bq_max, c->bq);
    b->d_max = std::max<int64_t>(b->d_max, c->m);
    b->perm_max = std::max<int64_t>(b->perm_max, c->perm_stride);
    b->pld_max = std::max<int64_t>(b->pld_max, c->pld);
  }
  if (b->mixed() && b->d_max > 4096) {
    b->err = "rs_create_batch: RS_MIXED takes problems with d <= 4096";
    return RS_EUNSUPPORTED;
  }
  if (b->bq_max > 4 * 512 || !(batch_fits(b, 512) || batch_fits(b, 256) || batch_fits(b, 128))) {
    b->err = "rs_create_batch: the problems are too large for the batch's iteration kernel";
    return RS_EUNSUPPORTED;
  }
  // per-problem state; B = X^T Y of every right-hand side (FP64)
  b->state.assign(P, nullptr);
  int64_t nmax = 0;
  for (rs_ctx* c : b->mem) nmax = std::max<int64_t>(nmax, c->n);
  double* ytmp = nullptr;
  BKC(cudaMalloc(&ytmp, (size_t)nmax * sizeof(double)));
  rs_status s = RS_OK;
  for (int p = 0; p < P && s == RS_OK; ++p) {
    rs_ctx* c = b->mem[p];
    const size_t v = (size_t)nrhs * c->m;
    cudaError_t e = cudaMalloc(&b->state[p], 48 * v);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->state[p], 0, 48 * v, b->stream);
    double* bp = reinterpret_cast<double*>(b->state[p] + 32 * v);
    for (int r = 0; r < nrhs && e == cudaSuccess; ++r) {
      e = cudaMemcpyAsync(ytmp, Ys[p] + (size_t)r * c->n, (size_t)c->n * sizeof(double),
                          y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) break;
      if (c->xdtype == RS_F32 && c->mixed())
        e = launch_xt_v_pairs(b->stream, static_cast<const float*>(c->X), c->n, c->d, ytmp,
                              bp + (size_t)r * c->m, c->xt_part);
      else if (c->xdtype == RS_F32)
        e = launch_xt_v<float>(b->stream, static_cast<const float*>(c->X), c->n, c->d, ytmp,
                               bp + (size_t)r * c->m, c->xt_part);
      else
        e = launch_xt_v<double>(b->stream, static_cast<const double*>(c->X), c->n, c->d, ytmp,
                                bp + (size_t)r * c->m, c->xt_part);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // ytmp reused
    if (e != cudaSuccess) {
      b->err = std::string("rs_create_batch: B of problem ") + std::to_string(p) + ": " + cudaGetErrorString(e);
      s = (e == cudaErrorMemoryAllocation) ? RS_ENOMEM : RS_ECUDA;
    }
  }
  cudaFree(ytmp);
  if (s != RS_OK) return s;
  const size_t np = (size_t)P * nrhs;
  BKC(cudaMalloc(&b->flag, np * sizeof(int32_t)));
  BKC(cudaMalloc(&b->skip, np * sizeof(int32_t)));
  BKC(cudaMalloc(&b->iters, np * sizeof(int64_t)));
  BKC(cudaMalloc(&b->r0, np * sizeof(double)));
  BKC(cudaMalloc(&b->resid, np * sizeof(double)));
  BKC(cudaMalloc(&b->tol, sizeof(double)));
  BKC(cudaMalloc(&b->fin, 3 * sizeof(int32_t)));
  BKC(cudaMallocHost(&b->fin_h, 3 * sizeof(int32_t)));
  BKC(cudaMalloc(&b->alive, P * sizeof(int32_t)));
  BKC(cudaMalloc(&b->order, P * sizeof(int32_t)));
  BKC(cudaMalloc(&b->err_word, sizeof(int32_t)));
  BKC(cudaMemset(b->err_word, 0, sizeof(int32_t)));
  if (b->mixed()) {
    int64_t n_max = 0;
    for (rs_ctx* c : b->mem) n_max = std::max<int64_t>(n_max, c->n);
    b->xpart.assign(kBatchMaxStreams, nullptr);
    b->xu.assign(kBatchMaxStreams, nullptr);
    const size_t words = (size_t)xtx_two_pass_part(n_max, b->d_max, 4);
    for (double*& x : b->xpart) BKC(cudaMalloc(&x, words * sizeof(double)));
    for (float2*& x : b->xu) BKC(cudaMalloc(&x, (size_t)n_max * 4 * sizeof(float2)));
  }
  if ((s = batch_upload(b)) != RS_OK) return s;
  BKC(cudaEventRecord(b->ev1, b->stream));
  BKC(cudaEventSynchronize(b->ev1));
  float ms = 0.f;
  BKC(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  b->setup_ms = ms;
  return RS_OK;
}

}  // namespace

extern "C" {

rs_status rs_create_batch(int32_t P, const rs_matrix* Xs, const double* const* Ys,
                          int32_t y_on_device, int32_t nrhs, const double* lambdas,
                          int32_t sketch, const int64_t* taus, const rs_mom* mom, uint64_t seed,
                          const rs_opts* opts, rs_batch** out) {
  if (out) *out = nullptr;
  if (P < 1 || !Xs || !Ys || !lambdas || !out) { g_batch_err = "rs_create_batch: null argument or P < 1"; return RS_EINVAL; }
  if (nrhs < 1 || nrhs > 8) { g_batch_err = "rs_create_batch: nrhs must be in [1, 8]"; return RS_EINVAL; }
  if (sketch != RS_SUBSAMPLE && sketch != RS_COUNT && sketch != RS_SUBCOUNT) {
    g_batch_err = "rs_create_batch: the batch takes the subsample, count or subcount sketch";
    return RS_EUNSUPPORTED;
  }
  rs_opts o;
  rs_default_opts(&o);
  if (opts) o = *opts;
  // the batch refreshes at every chunk end: its chunk is the refresh period. A plain
  // FP64 batch keeps 128 slots per problem: its S^T A is FP64, and hundreds of
  // problems hold one chunk each at once
  if (o.chunk <= 0)
    o.chunk = o.precision == RS_MIXED ? (o.refresh_every > 0 ? o.refresh_every : 300) : 128;
  for (int p = 0; p < P; ++p) {
    if (Xs[p].is_csr) { g_batch_err = "rs_create_batch: dense X only"; return RS_EUNSUPPORTED; }
    if (o.precision == RS_MIXED && Xs[p].dtype != RS_F32) { g_batch_err = "rs_create_batch: RS_MIXED takes FP32 X"; return RS_EINVAL; }
    if (!Ys[p]) { g_batch_err = "rs_create_batch: null targets"; return RS_EINVAL; }
  }
  rs_batch* b = new (std::nothrow) rs_batch();
  if (!b) { g_batch_err = "rs_create_batch: out of host memory"; return RS_ENOMEM; }
  DeviceGuard dg(o.device);
  b->P = P;
  b->nrhs = nrhs;
  b->precision = o.precision;
  b->sketch = sketch;
  if (o.tune_cache != nullptr) b->tune_cache = o.tune_cache;
  const rs_status s = batch_init(b, Xs, Ys, y_on_device, lambdas, sketch, taus, mom, seed, o);
  if (s != RS_OK) {
    g_batch_err = b->err;
    batch_free(b);
    delete b;
    return s;
  }
  g_batch_err.clear();
  *out = b;
  return RS_OK;
}

rs_status rs_solve_batch(rs_batch* b, double tol, int64_t max_iters, double* const* W_out,
                         int64_t* iters_out, double* resid_out) {
  if (!b) { g_batch_err = "rs_solve_batch: null batch"; return RS_EINVAL; }
  if (max_iters < 0 || !(tol >= 0.0)) { b->err = "rs_solve_batch: bad tol or max_iters"; return RS_EINVAL; }
  DeviceGuard dg(b->mem[0]->device);
  rs_status s;
  rs_ctx* c0 = b->mem[0];
  if ((s = ensure_schedule(c0, std::max<int64_t>(max_iters, 2 * b->chunk))) != RS_OK) { b->err = c0->err; return s; }
  if ((s = batch_set_order(b, nullptr)) != RS_OK) return s;  // every problem, largest first
  if (!b->tuned) {
    BKC(cudaEventRecord(b->ev0, b->stream));
    if ((s = batch_tune(b)) != RS_OK) return s;
    BKC(cudaEventRecord(b->ev1, b->stream));
    BKC(cudaEventSynchronize(b->ev1));
    float ms = 0.f;
    BKC(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    b->tune_ms = ms;
  }
  if (!b->graph || b->graph_gam != c0->gam || b->graph_threads != b->threads ||
      b->graph_streams != b->nstreams || b->graph_nrun != b->nrun)
    if ((s = batch_build_graph(b, b->threads, b->nstreams)) != RS_OK) return s;
  if ((s = batch_reset(b, tol, max_iters)) != RS_OK) return s;
  BKC(cudaEventRecord(b->ev0, b->stream));
  if (max_iters > 0 && (s = batch_run(b, max_iters + 2)) != RS_OK) return s;
  BKC(cudaEventRecord(b->ev1, b->stream));
  BKC(cudaEventSynchronize(b->ev1));
  float ms = 0.f;
  BKC(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  b->solve_ms = ms;
  const int np = b->P * b->nrhs;
  if (b->mixed())
    BKC(rs::launch_batch_mixed_aux(b->stream, 2, static_cast<const rs::BatchRefM*>(b->refs), np,
                                   batch_pairs(b), b->tol));
  for (int p = 0; p < b->P; ++p) {
    rs_ctx* c = b->mem[p];
    int32_t gen_err = 0;
    BKC(copy_sync(c, &gen_err, c->err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (gen_err) { b->err = "sketch generation: sample threshold search failed"; return RS_ECUDA; }
    if (!W_out || !W_out[p]) continue;
    const size_t v = (size_t)b->nrhs * c->m;
    const unsigned char* src = b->state[p] + (b->mixed() ? 24 * v : 0);
    BKC(cudaMemcpyAsync(W_out[p], src, v * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  std::vector<int32_t> flag(np);
  BKC(cudaMemcpyAsync(flag.data(), b->flag, np * sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
  if (iters_out) BKC(cudaMemcpyAsync(iters_out, b->iters, np * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream));
  if (resid_out) BKC(cudaMemcpyAsync(resid_out, b->resid, np * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BKC(cudaStreamSynchronize(b->stream));
  bool nan = false, open = false;
  for (int32_t f : flag) {
    nan |= (f == 3);
    open |= (f < 2);
  }
  if (nan) { b->err = "rs_solve_batch: NaN or Inf in a residual"; return RS_ENUMERIC; }
  return open ? RS_ENOTCONV : RS_OK;
}

rs_status rs_batch_profile(rs_batch* b, int32_t chunks, double* ms_parts) {
  if (!b || chunks < 1) { g_batch_err = "rs_batch_profile: null batch or chunks < 1"; return RS_EINVAL; }
  DeviceGuard dg(b->mem[0]->device);
  rs_status s;
  rs_ctx* c0 = b->mem[0];
  const int64_t K = (int64_t)chunks * b->chunk;
  if ((s = ensure_schedule(c0, std::max<int64_t>(K, 2 * b->chunk))) != RS_OK) { b->err = c0->err; return s; }
  if ((s = batch_set_order(b, nullptr)) != RS_OK) return s;
  if (!b->tuned && (s = batch_tune(b)) != RS_OK) return s;
  constexpr int NP = 6;
  cudaGraphExec_t g[NP] = {};
  cudaEvent_t ev[NP + 1] = {};
  auto done = [&](rs_status r) {
    for (cudaGraphExec_t x : g) if (x) cudaGraphExecDestroy(x);
    for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
    return r;
  };
  const int parts[NP] = {kPartPhase1, kPartPhase1, kPartPhase1, kPartPhase1, kPartIterate, kPartRefresh};
  const int p1[NP] = {kP1Plan, kP1Rows, kP1Msys, kP1Inv, kP1All, kP1All};
  for (int i = 0; i < NP; ++i)
    if ((s = batch_capture(b, b->threads, b->nstreams, parts[i], &g[i], p1[i])) != RS_OK) return done(s);
  for (cudaEvent_t& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { b->err = "rs_batch_profile: events"; return done(RS_ECUDA); }
  if ((s = batch_reset(b, 0.0, K)) != RS_OK) return done(s);
  double acc[NP] = {};
  for (int q = 0; q < chunks; ++q) {
    cudaError_t e = cudaEventRecord(ev[0], b->stream);
    for (int i = 0; i < NP && e == cudaSuccess; ++i) {
      e = cudaGraphLaunch(g[i], b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[i + 1], b->stream);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[NP]);
    for (int i = 0; i < NP && e == cudaSuccess; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      acc[i] += ms;
    }
    if (e != cudaSuccess) {
      b->err = std::string("rs_batch_profile: ") + cudaGetErrorString(e);
      return done(RS_ECUDA);
    }
  }
  if (ms_parts)
    for (int i = 0; i < NP; ++i) ms_parts[i] = acc[i] / chunks;
  return done(RS_OK);
}

rs_status rs_batch_set_launch(rs_batch* b, int32_t iter_threads, int32_t phase1_streams) {
  if (!b) { g_batch_err = "rs_batch_set_launch: null batch"; return RS_EINVAL; }
  if (iter_threads == 0 && phase1_streams == 0) {
    b->tuned = false;
    return RS_OK;
  }
  if ((iter_threads != 128 && iter_threads != 256 && iter_threads != 512) ||
      (phase1_streams != 1 && phase1_streams != 2 && phase1_streams != kBatchMaxStreams)) {
    b->err = "rs_batch_set_launch: iter_threads in {128, 256, 512}, phase1_streams in {1, 2, 4}";
    return RS_EINVAL;
  }
  DeviceGuard dg(b->mem[0]->device);
  if (b->bq_max > 4 * iter_threads || !batch_fits(b, iter_threads)) {
    b->err = "rs_batch_set_launch: the iteration kernel does not fit with that CTA size";
    return RS_EINVAL;
  }
  b->threads = iter_threads;
  b->nstreams = phase1_streams;
  b->tuned = true;
  return RS_OK;
}

void rs_destroy_batch(rs_batch* b) {
  if (!b) return;
  {
    DeviceGuard dg(b->mem.empty() || !b->mem[0] ? 0 : b->mem[0]->device);
    batch_free(b);
  }
  delete b;
}

const char* rs_batch_last_error(const rs_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}

rs_status rs_batch_info(const rs_batch* b, double* setup_ms, double* solve_ms, double* tune_ms,
                        int32_t* iter_threads, int32_t* phase1_streams) {
  if (!b) return RS_EINVAL;
  if (setup_ms) *setup_ms = b->setup_ms;
  if (solve_ms) *solve_ms = b->solve_ms;
  if (tune_ms) *tune_ms = b->tune_ms;
  if (iter_threads) *iter_threads = b->threads;
  if (phase1_streams) *phase1_streams = b->nstreams;
  return RS_OK;
}

}  // extern "C"

// ===========================================================================
// training the proposal's network (rs_mlp_*): FP32 master weights, Adam moments,
// the bfloat16 copy the proposal reads, gradient work space
// ===========================================================================
struct rs_mlp {
  float *theta = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr;
  uint16_t* wbf = nullptr;
  float *part = nullptr, *loss_part = nullptr;
  double* loss = nullptr;
  int64_t cap_blocks = 0;
  int64_t step = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
};

namespace {
std::string g_mlp_err;

#define MKC(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return (e_ == cudaErrorMemoryAllocation) ? RS_ENOMEM : RS_ECUDA;             \
    }                                                                             \
  } while (0)

void mlp_free(rs_mlp* h) {
  void* ptrs[] = {h->theta, h->mom, h->vel, h->grad, h->wbf, h->part, h->loss_part, h->loss};
  for (void* p : ptrs) if (p) cudaFree(p);
}

rs_status mlp_grad(rs_mlp* h, const float* Z, const float* y, int64_t n) {
  const int64_t nb = mlp_grad_blocks(n);
  if (nb > h->cap_blocks) {
    if (h->part) cudaFree(h->part);
    if (h->loss_part) cudaFree(h->loss_part);
    h->part = nullptr;
    h->loss_part = nullptr;
    MKC(cudaMalloc(&h->part, (size_t)nb * kMlpParams * sizeof(float)));
    MKC(cudaMalloc(&h->loss_part, (size_t)nb * sizeof(float)));
    h->cap_blocks = nb;
  }
  MKC(launch_mlp_grad(h->stream, h->theta, Z, y, n, h->part, h->loss_part, h->grad, h->loss));
  return RS_OK;
}
}  // namespace

extern "C" {

rs_status rs_mlp_create(const float* theta0, int32_t device, void* stream, rs_mlp** out) {
  if (out) *out = nullptr;
  if (!theta0 || !out) { g_mlp_err = "rs_mlp_create: null argument"; return RS_EINVAL; }
  rs_mlp* h = new (std::nothrow) rs_mlp();
  if (!h) { g_mlp_err = "rs_mlp_create: out of host memory"; return RS_ENOMEM; }
  DeviceGuard dg(device);
  h->device = device;
  h->stream = static_cast<cudaStream_t>(stream);
  auto fail = [&](rs_status s) {
    g_mlp_err = h->err;
    mlp_free(h);
    delete h;
    return s;
  };
  const size_t pb = kMlpParams * sizeof(float);
  if (cudaMalloc(&h->theta, pb) != cudaSuccess || cudaMalloc(&h->mom, pb) != cudaSuccess ||
      cudaMalloc(&h->vel, pb) != cudaSuccess || cudaMalloc(&h->grad, pb) != cudaSuccess ||
      cudaMalloc(&h->wbf, kMlpParams * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&h->loss, sizeof(double)) != cudaSuccess) {
    h->err = "rs_mlp_create: device allocation";
    return fail(RS_ENOMEM);
  }
  if (cudaMemcpyAsync(h->theta, theta0, pb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->mom, 0, pb, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->vel, 0, pb, h->stream) != cudaSuccess ||
      launch_f32_to_bf16(h->stream, h->theta, kMlpParams, h->wbf) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->err = "rs_mlp_create: upload";
    return fail(RS_ECUDA);
  }
  *out = h;
  return RS_OK;
}

rs_status rs_mlp_grad(rs_mlp* h, const float* Z, const float* y, int64_t n, float* grad_out,
                      double* loss_out) {
  if (!h || !Z || !y || n < 1) { g_mlp_err = "rs_mlp_grad: bad arguments"; return RS_EINVAL; }
  DeviceGuard dg(h->device);
  rs_status s = mlp_grad(h, Z, y, n);
  if (s != RS_OK) return s;
  if (grad_out) MKC(cudaMemcpyAsync(grad_out, h->grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  if (loss_out) MKC(cudaMemcpyAsync(loss_out, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  MKC(cudaStreamSynchronize(h->stream));
  return RS_OK;
}

rs_status rs_mlp_step(rs_mlp* h, const float* Z, const float* y, int64_t n, double lr,
                      double* loss_out) {
  if (!h || !Z || !y || n < 1 || !(lr > 0.0)) { g_mlp_err = "rs_mlp_step: bad arguments"; return RS_EINVAL; }
  DeviceGuard dg(h->device);
  rs_status s = mlp_grad(h, Z, y, n);
  if (s != RS_OK) return s;
  h->step += 1;
  MKC(launch_mlp_adam(h->stream, h->theta, h->mom, h->vel, h->grad, h->step, (float)lr, 0.9f,
                      0.999f, 1e-8f, h->wbf));
  if (loss_out) {
    MKC(cudaMemcpyAsync(loss_out, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MKC(cudaStreamSynchronize(h->stream));
  }
  return RS_OK;
}

rs_status rs_mlp_scores(rs_mlp* h, const float* Z, int64_t n, float* s_out) {
  if (!h || !Z || !s_out || n < 0) { g_mlp_err = "rs_mlp_scores: bad arguments"; return RS_EINVAL; }
  DeviceGuard dg(h->device);
  MKC(launch_mlp_forward(h->stream, h->wbf, Z, n, s_out));
  return RS_OK;
}

rs_status rs_mlp_get(rs_mlp* h, float* theta_out, uint16_t* bf16_out) {
  if (!h) { g_mlp_err = "rs_mlp_get: null handle"; return RS_EINVAL; }
  DeviceGuard dg(h->device);
  if (theta_out) MKC(cudaMemcpyAsync(theta_out, h->theta, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  if (bf16_out) MKC(cudaMemcpyAsync(bf16_out, h->wbf, kMlpParams * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->stream));
  MKC(cudaStreamSynchronize(h->stream));
  return RS_OK;
}

void rs_mlp_destroy(rs_mlp* h) {
  if (!h) return;
  {
    DeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    mlp_free(h);
  }
  delete h;
}

const char* rs_mlp_last_error(const rs_mlp* h) { return h ? h->err.c_str() : g_mlp_err.c_str(); }

}  // extern "C"
