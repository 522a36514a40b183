// Many independent ridge problems, several right-hand sides each, in one
// persistent launch per chunk (Algorithm 2, eq. (53), for every problem at once).
//
// Problem p has its own A_p, sketch sequence (seed + p), S^T A and M^+ per slot
// (formed by phase 1 of its member context); its nrhs right-hand sides share them:
// one read of the slot's S^T A per iteration serves all of them ("one
// factorisation shared by the right-hand sides"). CTA p runs the chunk's
// iterations of problem p: r_S and delta = M^+ r_S for every active right-hand
// side, then (A S delta)_i = sum_j (S^T A)[j, i] delta_j for the nrhs of them in
// one pass, the momentum step, the norms and the per-right-hand-side stopping test.
// A right-hand side that meets the tolerance stops; in mixed precision it waits
// ("pending") for the FP64 refresh at the end of the chunk, which either confirms
// it or resumes it.
#include "rs_kernels.cuh"

namespace rs {

namespace {
constexpr int kBMaxRhs = 8;
}

template <typename T, typename TF>
__global__ void k_batch_iterate(const BatchProb<T, TF>* __restrict__ probs, int nrhs,
                                BatchPairs pairs, const double* __restrict__ gam,
                                const double* __restrict__ bet, int64_t chunk,
                                const double* __restrict__ tolp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchProb<T, TF> pr = probs[blockIdx.x];
  Ctrl* ctrl = pr.ctrl;
  if (halted(ctrl)) return;
  const int64_t k0 = ctrl->k0, kstart = ctrl->k;
  const int64_t kend = min(k0 + chunk, ctrl->max_iters);
  const int64_t d = pr.d, tau = pr.tau;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  TF* rsf = reinterpret_cast<TF*>(smem_raw);                       // nrhs x tau
  T* dT = reinterpret_cast<T*>(rsf + (size_t)nrhs * tau);          // nrhs x tau
  double* dD = reinterpret_cast<double*>(
      smem_raw + (((size_t)nrhs * tau * (sizeof(TF) + sizeof(T)) + 15) / 16) * 16);  // nrhs x tau
  double* sred = dD + (size_t)nrhs * tau;                          // 32 x nrhs
  __shared__ int s_act[kBMaxRhs];
  __shared__ int s_any;
  const int pbase = blockIdx.x * nrhs;
  const double tol = *tolp;
  int64_t k = kstart;
  for (; k < kend; ++k) {
    if (tid < nrhs) s_act[tid] = (pairs.flag[pbase + tid] == 0);
    __syncthreads();
    if (tid == 0) {
      int a = 0;
      for (int q = 0; q < nrhs; ++q) a |= s_act[q];
      s_any = a;
    }
    __syncthreads();
    if (!s_any) break;
    const int64_t slot = k - k0;
    const int32_t* perm = pr.perm + slot * pr.perm_stride;
    const int32_t* boff = pr.boff + slot * pr.boff_stride;
    const int32_t* inv = pr.inv + slot * pr.inv_slot;
    const TF* P = pr.P + slot * pr.p_slot;
    const T* SA = pr.SA + slot * pr.sa_slot;
    // r_S = S^T r for every active right-hand side
    for (int64_t e = tid; e < (int64_t)nrhs * tau; e += blockDim.x) {
      const int q = (int)(e / tau);
      const int64_t j = e - (int64_t)q * tau;
      double acc = 0.0;
      if (s_act[q]) {
        const double* r = pr.r + (int64_t)q * d;
        for (int32_t t = boff[j]; t < boff[j + 1]; ++t) {
          const int32_t en = perm[t];
          const double v = r[entry_row(en)];
          acc += entry_neg(en) ? -v : v;
        }
      }
      rsf[e] = (TF)acc;
    }
    __syncthreads();
    // delta = M^+ r_S: warp per row j of P, all right-hand sides at once
    for (int64_t j = wid; j < tau; j += nw) {
      TF acc[kBMaxRhs];
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) acc[q] = TF(0);
      for (int64_t l = lane; l < tau; l += 32) {
        const TF pv = P[j * pr.pld + l];
#pragma unroll
        for (int q = 0; q < kBMaxRhs; ++q)
          if (q < nrhs) acc[q] += pv * rsf[(int64_t)q * tau + l];
      }
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) {
        if (q >= nrhs) break;
        const TF v = warp_sum(acc[q]);
        if (lane == 0) {
          dD[(int64_t)q * tau + j] = (double)v;
          dT[(int64_t)q * tau + j] = (T)v;
        }
      }
    }
    __syncthreads();
    // rows i: A S delta for every right-hand side from one read of S^T A, update
    const double g = gam[k], b = bet[k];
    double sq[kBMaxRhs];
#pragma unroll
    for (int q = 0; q < kBMaxRhs; ++q) sq[q] = 0.0;
    for (int64_t i = tid; i < d; i += blockDim.x) {
      T acc[kBMaxRhs];
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) acc[q] = T(0);
      for (int64_t j = 0; j < tau; ++j) {
        const T sa = SA[j * pr.ld + i];
#pragma unroll
        for (int q = 0; q < kBMaxRhs; ++q)
          if (q < nrhs) acc[q] += sa * dT[(int64_t)q * tau + j];
      }
      const int32_t en = inv[i];
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) {
        if (q >= nrhs || !s_act[q]) continue;
        const double sd = (en == kNotSketched) ? 0.0
                          : (entry_neg(en) ? -dD[(int64_t)q * tau + (en & 0x7FFFFFFF)]
                                           : dD[(int64_t)q * tau + (en & 0x7FFFFFFF)]);
        double* w = pr.w + (int64_t)q * d;
        double* wp = pr.wp + (int64_t)q * d;
        double* r = pr.r + (int64_t)q * d;
        double* rp = pr.rp + (int64_t)q * d;
        const double wi = w[i], wpi = wp[i], ri = r[i], rpi = rp[i];
        const double rn = (1.0 + b) * ri - b * rpi - g * (double)acc[q];
        wp[i] = wi;
        w[i] = (1.0 + b) * wi - b * wpi - g * sd;
        rp[i] = ri;
        r[i] = rn;
        sq[q] += rn * rn;
      }
    }
    // norms (fixed order) and the stopping test of each active right-hand side
#pragma unroll
    for (int q = 0; q < kBMaxRhs; ++q) {
      if (q >= nrhs) break;
      const double v = warp_sum(sq[q]);
      if (lane == 0) sred[wid * nrhs + q] = v;
    }
    __syncthreads();
    if (tid < nrhs && s_act[tid]) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += sred[w * nrhs + tid];
      const int pi = pbase + tid;
      const double rel = sqrt(t) / pairs.r0[pi];
      pairs.resid[pi] = rel;
      pairs.iters[pi] += 1;
      if (!isfinite(rel)) pairs.flag[pi] = 3;
      else if (rel <= tol) pairs.flag[pi] = 2;
    }
    __syncthreads();
  }
  if (tid == 0) {
    ctrl->k = k;
    int done = 1;  // every right-hand side finished (converged or failed)
    for (int q = 0; q < nrhs; ++q) done &= (pairs.flag[pbase + q] >= 2);
    if (done || k >= ctrl->max_iters) ctrl->stop = 1;
    __threadfence();
  }
}

// Mixed precision: the iterate and the residual are held as float pairs (hi + lo,
// about 48 significant bits) with FP32 increments Delta_k = x_{k+1} - x_k:
//   Delta_w = beta Delta_w - gamma S delta,   w += Delta_w,
//   Delta_r = beta Delta_r - gamma A S delta, r += Delta_r,
// which is the momentum step of eq. (53) (x_{k+1} = x_k + beta (x_k - x_{k-1}) - ...)
// without FP64 arithmetic (scarce on this GPU: one CTA updates a whole problem).
// The FP64 refresh replaces r by the true residual of w and keeps Delta_r.
__device__ __forceinline__ void df_add(float2& x, float d) {
  const float s = x.x + d;
  const float bb = s - x.x;
  const float err = (x.x - (s - bb)) + (d - bb);
  const float lo = x.y + err;
  const float hi = s + lo;
  x = make_float2(hi, lo - (hi - s));
}

__global__ void k_batch_iterate_mixed(const BatchProbM* __restrict__ probs, int nrhs,
                                      BatchPairs pairs, const double* __restrict__ gam,
                                      const double* __restrict__ bet, int64_t chunk,
                                      const double* __restrict__ tolp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchProbM pr = probs[blockIdx.x];
  Ctrl* ctrl = pr.ctrl;
  if (halted(ctrl)) return;
  const int64_t k0 = ctrl->k0, kstart = ctrl->k;
  const int64_t kend = min(k0 + chunk, ctrl->max_iters);
  const int64_t d = pr.d, tau = pr.tau;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  float* rsf = reinterpret_cast<float*>(smem_raw);     // nrhs x tau
  float* dl = rsf + (size_t)nrhs * tau;                // nrhs x tau
  float* sred = dl + (size_t)nrhs * tau;               // 32 x nrhs
  __shared__ int s_act[kBMaxRhs];
  __shared__ int s_any;
  const int pbase = blockIdx.x * nrhs;
  const float tol = (float)*tolp;
  int64_t k = kstart;
  for (; k < kend; ++k) {
    if (tid < nrhs) s_act[tid] = (pairs.flag[pbase + tid] == 0);
    __syncthreads();
    if (tid == 0) {
      int a = 0;
      for (int q = 0; q < nrhs; ++q) a |= s_act[q];
      s_any = a;
    }
    __syncthreads();
    if (!s_any) break;
    const int64_t slot = k - k0;
    const int32_t* perm = pr.perm + slot * pr.perm_stride;
    const int32_t* boff = pr.boff + slot * pr.boff_stride;
    const int32_t* inv = pr.inv + slot * pr.inv_slot;
    const float* P = pr.P + slot * pr.p_slot;
    const float* SA = pr.SA + slot * pr.sa_slot;
    for (int64_t e = tid; e < (int64_t)nrhs * tau; e += blockDim.x) {
      const int q = (int)(e / tau);
      const int64_t j = e - (int64_t)q * tau;
      float acc = 0.f;
      if (s_act[q]) {
        const float2* r = pr.r + (int64_t)q * d;
        for (int32_t t = boff[j]; t < boff[j + 1]; ++t) {
          const int32_t en = perm[t];
          const float v = r[entry_row(en)].x;
          acc += entry_neg(en) ? -v : v;
        }
      }
      rsf[e] = acc;
    }
    __syncthreads();
    for (int64_t j = wid; j < tau; j += nw) {
      float acc[kBMaxRhs];
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) acc[q] = 0.f;
      for (int64_t l = lane; l < tau; l += 32) {
        const float pv = P[j * pr.pld + l];
#pragma unroll
        for (int q = 0; q < kBMaxRhs; ++q)
          if (q < nrhs) acc[q] += pv * rsf[(int64_t)q * tau + l];
      }
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) {
        if (q >= nrhs) break;
        const float v = warp_sum(acc[q]);
        if (lane == 0) dl[(int64_t)q * tau + j] = v;
      }
    }
    __syncthreads();
    const float g = (float)gam[k], b = (float)bet[k];
    float sq[kBMaxRhs];
#pragma unroll
    for (int q = 0; q < kBMaxRhs; ++q) sq[q] = 0.f;
    for (int64_t i = tid; i < d; i += blockDim.x) {
      float acc[kBMaxRhs];
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) acc[q] = 0.f;
      int64_t j = 0;
      for (; j + 2 <= tau; j += 2) {  // two rows of S^T A in flight
        const float s0 = SA[j * pr.ld + i], s1 = SA[(j + 1) * pr.ld + i];
#pragma unroll
        for (int q = 0; q < kBMaxRhs; ++q)
          if (q < nrhs) acc[q] += s0 * dl[(int64_t)q * tau + j] + s1 * dl[(int64_t)q * tau + j + 1];
      }
      for (; j < tau; ++j) {
        const float s0 = SA[j * pr.ld + i];
#pragma unroll
        for (int q = 0; q < kBMaxRhs; ++q)
          if (q < nrhs) acc[q] += s0 * dl[(int64_t)q * tau + j];
      }
      const int32_t en = inv[i];
#pragma unroll
      for (int q = 0; q < kBMaxRhs; ++q) {
        if (q >= nrhs || !s_act[q]) continue;
        const float sd = (en == kNotSketched) ? 0.f
                         : (entry_neg(en) ? -dl[(int64_t)q * tau + (en & 0x7FFFFFFF)]
                                          : dl[(int64_t)q * tau + (en & 0x7FFFFFFF)]);
        const int64_t o = (int64_t)q * d + i;
        const float dw = b * pr.dw[o] - g * sd;
        const float dr = b * pr.dr[o] - g * acc[q];
        pr.dw[o] = dw;
        pr.dr[o] = dr;
        float2 w = pr.w[o], r = pr.r[o];
        df_add(w, dw);
        df_add(r, dr);
        pr.w[o] = w;
        pr.r[o] = r;
        sq[q] += r.x * r.x;
      }
    }
#pragma unroll
    for (int q = 0; q < kBMaxRhs; ++q) {
      if (q >= nrhs) break;
      const float v = warp_sum(sq[q]);
      if (lane == 0) sred[wid * nrhs + q] = v;
    }
    __syncthreads();
    if (tid < nrhs && s_act[tid]) {
      float t = 0.f;
      for (int w = 0; w < nw; ++w) t += sred[w * nrhs + tid];
      const int pi = pbase + tid;
      const float rel = sqrtf(t) / (float)pairs.r0[pi];
      pairs.resid[pi] = rel;
      pairs.iters[pi] += 1;
      if (!isfinite(rel)) pairs.flag[pi] = 3;
      else if (rel <= tol) pairs.flag[pi] = 1;
    }
    __syncthreads();
  }
  if (tid == 0) {
    ctrl->k = k;
    int done = 1;
    for (int q = 0; q < nrhs; ++q) done &= (pairs.flag[pbase + q] >= 2);
    if (done || k >= ctrl->max_iters) ctrl->stop = 1;
    __threadfence();
  }
}

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

cudaError_t launch_batch_iterate_mixed(cudaStream_t st, const BatchProbM* probs, int P, int nrhs,
                                       BatchPairs pairs, const double* gam, const double* bet,
                                       int64_t chunk, const double* tol, int64_t tau_max,
                                       int threads) {
  if (nrhs < 1 || nrhs > kBMaxRhs) return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * nrhs * tau_max * 4 + 32 * (size_t)nrhs * 4;
  cudaError_t e = cudaFuncSetAttribute(k_batch_iterate_mixed,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_batch_iterate_mixed<<<P, threads, smem, st>>>(probs, nrhs, pairs, gam, bet, chunk, tol);
  return cudaGetLastError();
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
// phase 1 in later chunks); out[0] = problems still running, out[1] = failed pairs
__global__ void k_batch_finish(Ctrl* const* __restrict__ ctrls, int P, int nrhs,
                               BatchPairs pairs, int32_t* __restrict__ out) {
  __shared__ int s_run, s_fail;
  if (threadIdx.x == 0) { s_run = 0; s_fail = 0; }
  __syncthreads();
  int run = 0, fail = 0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    int done = 1;
    for (int q = 0; q < nrhs; ++q) {
      const int f = pairs.flag[p * nrhs + q];
      done &= (f >= 2);
      fail += (f == 3);
    }
    Ctrl* c = ctrls[p];
    if (done) c->stop = 1;
    run += !c->stop;
  }
  atomicAdd(&s_run, run);
  atomicAdd(&s_fail, fail);
  __syncthreads();
  if (threadIdx.x == 0) { out[0] = s_run; out[1] = s_fail; }
}

cudaError_t launch_batch_finish(cudaStream_t st, Ctrl* const* ctrls, int P, int nrhs,
                                BatchPairs pairs, int32_t* out) {
  k_batch_finish<<<1, 256, 0, st>>>(ctrls, P, nrhs, pairs, out);
  return cudaGetLastError();
}

size_t batch_iterate_smem(int64_t tau_max, int nrhs) {
  return (size_t)nrhs * tau_max * 24 + 32 * (size_t)nrhs * 8;
}

cudaError_t launch_batch_iterate(cudaStream_t st, const BatchProb<double, double>* probs, int P,
                                 int nrhs, BatchPairs pairs, const double* gam, const double* bet,
                                 int64_t chunk, const double* tol, int64_t tau_max, int threads) {
  if (nrhs < 1 || nrhs > kBMaxRhs) return cudaErrorInvalidValue;
  const size_t smem = batch_iterate_smem(tau_max, nrhs);
  cudaError_t e = cudaFuncSetAttribute(k_batch_iterate<double, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_batch_iterate<double, double><<<P, threads, smem, st>>>(probs, nrhs, pairs, gam, bet, chunk, tol);
  return cudaGetLastError();
}

cudaError_t launch_batch_init(cudaStream_t st, const BatchRef* refs, int npairs, BatchPairs pairs) {
  k_batch_init<<<npairs, 256, 0, st>>>(refs, pairs);
  return cudaGetLastError();
}

}  // namespace rs
