// State kernels of the batched solve (many problems, several right-hand sides each):
// initial state, the FP64 refresh of mixed precision and the end-of-chunk
// bookkeeping. The iterations themselves run in the cluster kernel of
// rs_batch_cluster.cu.
//
// Mixed precision holds the iterate and the residual as float pairs (hi + lo, about
// 48 significant bits) with FP32 increments Delta_k = x_{k+1} - x_k:
//   Delta_w = beta Delta_w - gamma S delta,   w += Delta_w,
//   Delta_r = beta Delta_r - gamma A S delta, r += Delta_r,
// which is the momentum step of eq. (53) (x_{k+1} = x_k + beta (x_k - x_{k-1}) - ...)
// in FP32 arithmetic only. A right-hand side whose recursive residual meets the
// tolerance waits ("pending") for the FP64 refresh at the end of the chunk, which
// replaces r by the true residual of w (Delta_r kept) and either confirms the pair
// or resumes it.
#include "rs_kernels.cuh"

namespace rs {

// w in FP64 from its float pair (for the FP64 refresh and the output), block per pair
__global__ void k_batch_wd(const BatchRefM* __restrict__ refs, BatchPairs pairs, int all) {
  const BatchRefM f = refs[blockIdx.x];
  if (!all && pairs.flag[f.pair] >= 2) return;
  for (int64_t i = threadIdx.x; i < f.d; i += blockDim.x)
    f.wd[i] = (double)f.w2[i].x + (double)f.w2[i].y;
}

// FP64 refresh, mixed: r = v + lambda w - b replaces the float pair r (Delta_r kept)
__global__ void __launch_bounds__(256) k_batch_refresh_mixed(const BatchRefM* __restrict__ refs,
                                                            BatchPairs pairs,
                                                            const double* __restrict__ tolp) {
  const double tol = *tolp;
  const BatchRefM f = refs[blockIdx.x];
  const int pi = f.pair;
  if (pairs.flag[pi] >= 2) return;
  __shared__ double s_red[32];
  double sq = 0.0;
  for (int64_t i = threadIdx.x; i < f.d; i += blockDim.x) {
    const double rt = f.v[i] + f.lambda * f.wd[i] - f.b[i];
    const float hi = (float)rt;
    f.r2[i] = make_float2(hi, (float)(rt - (double)hi));
    sq += rt * rt;
  }
  sq = block_sum(sq, s_red);
  if (threadIdx.x == 0) {
    const double rel = sqrt(sq) / pairs.r0[pi];
    pairs.resid[pi] = rel;
    if (!isfinite(rel)) pairs.flag[pi] = 3;
    else if (pairs.flag[pi] == 1) pairs.flag[pi] = (rel <= tol) ? 2 : 0;
    pairs.skip[pi] = pairs.flag[pi] >= 2;
  }
}

// mixed state of every pair: w = Delta_w = Delta_r = 0, r = -b; r0 = ||b||
__global__ void __launch_bounds__(256) k_batch_init_mixed(const BatchRefM* __restrict__ refs,
                                                         BatchPairs pairs) {
  const BatchRefM f = refs[blockIdx.x];
  __shared__ double s_red[32];
  double sq = 0.0;
  for (int64_t i = threadIdx.x; i < f.d; i += blockDim.x) {
    const double bi = f.b[i];
    const float hi = (float)(-bi);
    f.r2[i] = make_float2(hi, (float)(-bi - (double)hi));
    f.w2[i] = make_float2(0.f, 0.f);
    f.dw[i] = 0.f;
    f.dr[i] = 0.f;
    f.wd[i] = 0.0;
    sq += bi * bi;
  }
  sq = block_sum(sq, s_red);
  if (threadIdx.x == 0) {
    const double nb = sqrt(sq);
    pairs.r0[f.pair] = nb > 0.0 ? nb : 1.0;
    pairs.flag[f.pair] = nb > 0.0 ? 0 : 2;
    pairs.skip[f.pair] = nb > 0.0 ? 0 : 1;
    pairs.resid[f.pair] = 0.0;
    pairs.iters[f.pair] = 0;
  }
}

// plain state of every pair: w = w_prev = 0, r = r_prev = -b; r0 = ||b|| (block per pair)
__global__ void __launch_bounds__(256) k_batch_init(const BatchRef* __restrict__ refs,
                                                   BatchPairs pairs) {
  const BatchRef f = refs[blockIdx.x];
  __shared__ double s_red[32];
  double sq = 0.0;
  for (int64_t i = threadIdx.x; i < f.d; i += blockDim.x) {
    const double bi = f.b[i];
    f.w[i] = 0.0;
    f.wp[i] = 0.0;
    f.r[i] = -bi;
    f.rp[i] = -bi;
    sq += bi * bi;
  }
  sq = block_sum(sq, s_red);
  if (threadIdx.x == 0) {
    const double nb = sqrt(sq);
    pairs.r0[f.pair] = nb > 0.0 ? nb : 1.0;
    pairs.flag[f.pair] = nb > 0.0 ? 0 : 2;  // b = 0: w = 0 is the solution
    pairs.skip[f.pair] = nb > 0.0 ? 0 : 1;
    pairs.resid[f.pair] = 0.0;
    pairs.iters[f.pair] = 0;
  }
}

cudaError_t launch_batch_mixed_aux(cudaStream_t st, int what, const BatchRefM* refs, int npairs,
                                   BatchPairs pairs, const double* tol) {
  if (what == 0) k_batch_init_mixed<<<npairs, 256, 0, st>>>(refs, pairs);
  else if (what == 1) k_batch_wd<<<npairs, 256, 0, st>>>(refs, pairs, 0);
  else if (what == 2) k_batch_wd<<<npairs, 256, 0, st>>>(refs, pairs, 1);
  else k_batch_refresh_mixed<<<npairs, 256, 0, st>>>(refs, pairs, tol);
  return cudaGetLastError();
}

// end of a chunk: a problem whose right-hand sides have all finished stops (no
// phase 1 in later chunks); alive[p] = 1 while problem p runs; out[0] = problems
// still running, out[1] = failed pairs, out[2] = problems whose iteration kernel
// gave up a bounded wait
__global__ void k_batch_finish(Ctrl* const* __restrict__ ctrls, int P, int nrhs,
                               BatchPairs pairs, int32_t* __restrict__ alive,
                               int32_t* __restrict__ out) {
  __shared__ int s_run, s_fail, s_tmo;
  if (threadIdx.x == 0) { s_run = 0; s_fail = 0; s_tmo = 0; }
  __syncthreads();
  int run = 0, fail = 0, tmo = 0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    int done = 1;
    for (int q = 0; q < nrhs; ++q) {
      const int f = pairs.flag[p * nrhs + q];
      done &= (f >= 2);
      fail += (f == 3);
    }
    Ctrl* c = ctrls[p];
    if (done) c->stop = 1;
    tmo += (c->status == kStatusTimeout);
    alive[p] = !c->stop;
    run += !c->stop;
  }
  atomicAdd(&s_run, run);
  atomicAdd(&s_fail, fail);
  atomicAdd(&s_tmo, tmo);
  __syncthreads();
  if (threadIdx.x == 0) { out[0] = s_run; out[1] = s_fail; out[2] = s_tmo; }
}

cudaError_t launch_batch_finish(cudaStream_t st, Ctrl* const* ctrls, int P, int nrhs,
                                BatchPairs pairs, int32_t* alive, int32_t* out) {
  k_batch_finish<<<1, 256, 0, st>>>(ctrls, P, nrhs, pairs, alive, out);
  return cudaGetLastError();
}

cudaError_t launch_batch_init(cudaStream_t st, const BatchRef* refs, int npairs, BatchPairs pairs) {
  k_batch_init<<<npairs, 256, 0, st>>>(refs, pairs);
  return cudaGetLastError();
}

}  // namespace rs
