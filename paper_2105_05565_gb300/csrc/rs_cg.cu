// Conjugate Gradients on the ridge system A w = b (Hestenes and Stiefel, 1952), the
// competitor of the paper's Experiment 3 (Section 8.3), on the same A (dense, formed
// by the library) or through X (matrix-free, A v = X^T (X v) + lambda v).
//
// With r = A w - b (the sign of the sketch-and-project loop):
//   p = -r + beta p;  v = A p;  alpha = (r . r) / (p . v);  w += alpha p;  r += alpha v;
//   beta = (r_new . r_new) / (r . r).
// One iteration is three launches: k_cg_dir, the product (k_cg_matvec for dense A,
// with p . v fused; matrix-free: the CSR and CSC products, then k_cg_lam_dot), and
// k_cg_update (with r . r fused, the stop test and the history). Reductions end in
// the last block (ticket in CgScal) in a fixed order. Every kernel returns at once
// when the control block says stop or pending; in mixed precision an FP64 refresh
// of r through X (the one of the sketch-and-project path) follows every refresh
// period and decides convergence, and k_cg_rr re-forms r . r after it and restarts
// the directions (iterative refinement with an inner CG on the FP32 A).
#include <algorithm>

#include "rs_kernels.cuh"

namespace rs {

namespace {

// last block of a grid-wide reduction: true in every thread of the block that
// arrives last (after its partial is stored)
__device__ __forceinline__ bool last_block(uint32_t* ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  return s_last != 0;
}

__device__ __forceinline__ double sum_parts(const double* part, int n, double* s_red) {
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v += *((volatile const double*)&part[q]);
  return block_sum(v, s_red);
}

// exact float-pair product and sum (Knuth two-sum), as in the FP64-accurate
// products of the refresh
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

}  // namespace

// p = -r + beta p; with p2 != nullptr also p as float pairs (hi, lo) for the product
// with the FP32 A (the split once here keeps FP64 out of the product's inner loop)
__global__ void k_cg_dir(const Ctrl* __restrict__ ctrl, const CgScal* __restrict__ cs, int64_t m,
                         const double* __restrict__ r, double* __restrict__ p,
                         float2* __restrict__ p2) {
  if (halted(ctrl)) return;
  const double be = cs->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = -r[i] + be * p[i];
    p[i] = pi;
    if (p2 != nullptr) {
      const float h = (float)pi;
      p2[i] = make_float2(h, (float)(pi - (double)h));
    }
  }
}

// v = A p for rows [16 b, 16 b + 16) (two rows per warp), p . v of the block's rows;
// TA = double: FP64 products; TA = float: the FP32 entries times p as a float pair
// (hi + lo), summed exactly in float pairs
template <typename TA>
__global__ void __launch_bounds__(256) k_cg_matvec(const Ctrl* __restrict__ ctrl,
                                                   const TA* __restrict__ A, int64_t lda,
                                                   int64_t m, const double* __restrict__ p,
                                                   const float2* __restrict__ p2,
                                                   double* __restrict__ v, CgScal* __restrict__ cs,
                                                   double* __restrict__ part) {
  __shared__ double s_red[32];
  if (halted(ctrl)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 16 + wid * 2;
  double pv = 0.0;
  if (i0 < m) {
    const bool two = i0 + 1 < m;
    const TA* a0 = A + i0 * lda;
    const TA* a1 = A + (two ? i0 + 1 : i0) * lda;
    double d0, d1;
    if constexpr (sizeof(TA) == 8) {
      double s0 = 0.0, s1 = 0.0;
      for (int64_t j = lane; j < m; j += 32) {
        const double pj = p[j];
        s0 = fma(a0[j], pj, s0);
        s1 = fma(a1[j], pj, s1);
      }
      d0 = warp_sum(s0);
      d1 = warp_sum(s1);
    } else {
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      for (int64_t j = lane; j < m; j += 32) {
        const float2 pj = p2[j];
        const float ph = pj.x, pl = pj.y;
        const float x0 = a0[j], x1 = a1[j];
        float q = __fmul_rn(x0, ph), qe = __fmaf_rn(x0, ph, -q), s, e;
        two_sum_f(h0, q, s, e);
        h0 = s;
        l0 = __fmaf_rn(x0, pl, __fadd_rn(l0, __fadd_rn(e, qe)));
        q = __fmul_rn(x1, ph);
        qe = __fmaf_rn(x1, ph, -q);
        two_sum_f(h1, q, s, e);
        h1 = s;
        l1 = __fmaf_rn(x1, pl, __fadd_rn(l1, __fadd_rn(e, qe)));
      }
      d0 = warp_sum((double)h0 + (double)l0);
      d1 = warp_sum((double)h1 + (double)l1);
    }
    if (lane == 0) {
      v[i0] = d0;
      pv = p[i0] * d0;
      if (two) {
        v[i0 + 1] = d1;
        pv += p[i0 + 1] * d1;
      }
    }
  }
  pv = block_sum(pv, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = pv;
  if (!last_block(&cs->ticket)) return;
  const double tot = sum_parts(part, gridDim.x, s_red);
  if (threadIdx.x == 0) {
    cs->pv = tot;
    cs->ticket = 0u;
    __threadfence();
  }
}

// matrix-free: v += lambda p (v = X^T (X p) from the sparse products), p . v
__global__ void __launch_bounds__(256) k_cg_lam_dot(const Ctrl* __restrict__ ctrl, int64_t m,
                                                    double lambda, const double* __restrict__ p,
                                                    double* __restrict__ v,
                                                    CgScal* __restrict__ cs,
                                                    double* __restrict__ part) {
  __shared__ double s_red[32];
  if (halted(ctrl)) return;
  double pv = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = v[i] + lambda * p[i];
    v[i] = vi;
    pv += p[i] * vi;
  }
  pv = block_sum(pv, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = pv;
  if (!last_block(&cs->ticket)) return;
  const double tot = sum_parts(part, gridDim.x, s_red);
  if (threadIdx.x == 0) {
    cs->pv = tot;
    cs->ticket = 0u;
    __threadfence();
  }
}

// w += alpha p, r += alpha v, r . r; the last block: beta, the history, the stop test
__global__ void __launch_bounds__(256) k_cg_update(Ctrl* __restrict__ ctrl, CgScal* __restrict__ cs,
                                                   int64_t m, const double* __restrict__ p,
                                                   const double* __restrict__ v,
                                                   double* __restrict__ w, double* __restrict__ r,
                                                   double* __restrict__ part,
                                                   double* __restrict__ hist, int mixed) {
  __shared__ double s_red[32];
  if (halted(ctrl)) return;
  const double alpha = cs->rr / cs->pv;
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    w[i] += alpha * p[i];
    const double ri = r[i] + alpha * v[i];
    r[i] = ri;
    rr += ri * ri;
  }
  rr = block_sum(rr, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = rr;
  if (!last_block(&cs->ticket)) return;
  const double tot = sum_parts(part, gridDim.x, s_red);
  if (threadIdx.x == 0) {
    const int64_t k = ctrl->k + 1;
    const double rel = sqrt(tot) / ctrl->r0;
    hist[k] = rel;
    cs->beta = tot / cs->rr;
    cs->rr = tot;
    ctrl->k = k;
    if (!isfinite(rel)) {
      ctrl->status = kStatusNumeric;
      ctrl->stop = 1;
    } else if (!ctrl->no_stop && rel <= ctrl->tol) {
      if (mixed) ctrl->pending = 1;  // confirmed or not by the FP64 refresh
      else ctrl->stop = 1;
    }
    if (k >= ctrl->max_iters) ctrl->stop = 1;
    cs->ticket = 0u;
    __threadfence();
  }
}

// r . r at the start of a solve, and after a refresh replaced r by the FP64 true
// residual: CG then restarts from it (beta = 0, p = -r), iterative refinement with an
// inner CG on the FP32 operator (continuing the old directions with the replaced
// residual loses conjugacy when the FP32 A differs much from the exact one), one block
__global__ void __launch_bounds__(1024) k_cg_rr(const Ctrl* __restrict__ ctrl, CgScal* __restrict__ cs,
                                                int64_t m, const double* __restrict__ r, int init) {
  __shared__ double s_red[32];
  if (!init && stopped(ctrl)) return;
  double rr = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) rr += r[i] * r[i];
  rr = block_sum(rr, s_red);
  if (threadIdx.x == 0) {
    cs->rr = rr;
    cs->beta = 0.0;
    if (init) {
      cs->pv = 0.0;
      cs->ticket = 0u;
    }
  }
}

int cg_blocks(int64_t m) { return (int)std::min<int64_t>((m + 255) / 256, 2 * 152); }
int cg_matvec_blocks(int64_t m) { return (int)((m + 15) / 16); }

cudaError_t launch_cg_dir(cudaStream_t st, const Ctrl* ctrl, const CgScal* cs, int64_t m,
                          const double* r, double* p, float2* p2) {
  k_cg_dir<<<cg_blocks(m), 256, 0, st>>>(ctrl, cs, m, r, p, p2);
  return cudaGetLastError();
}

template <typename TA>
cudaError_t launch_cg_matvec(cudaStream_t st, const Ctrl* ctrl, const TA* A, int64_t lda, int64_t m,
                             const double* p, const float2* p2, double* v, CgScal* cs,
                             double* part) {
  if (sizeof(TA) == 4 && p2 == nullptr) return cudaErrorInvalidValue;
  k_cg_matvec<TA><<<cg_matvec_blocks(m), 256, 0, st>>>(ctrl, A, lda, m, p, p2, v, cs, part);
  return cudaGetLastError();
}
template cudaError_t launch_cg_matvec<float>(cudaStream_t, const Ctrl*, const float*, int64_t,
                                             int64_t, const double*, const float2*, double*,
                                             CgScal*, double*);
template cudaError_t launch_cg_matvec<double>(cudaStream_t, const Ctrl*, const double*, int64_t,
                                              int64_t, const double*, const float2*, double*,
                                              CgScal*, double*);

cudaError_t launch_cg_lam_dot(cudaStream_t st, const Ctrl* ctrl, int64_t m, double lambda,
                              const double* p, double* v, CgScal* cs, double* part) {
  k_cg_lam_dot<<<cg_blocks(m), 256, 0, st>>>(ctrl, m, lambda, p, v, cs, part);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(cudaStream_t st, Ctrl* ctrl, CgScal* cs, int64_t m, const double* p,
                             const double* v, double* w, double* r, double* part, double* hist,
                             int mixed) {
  k_cg_update<<<cg_blocks(m), 256, 0, st>>>(ctrl, cs, m, p, v, w, r, part, hist, mixed);
  return cudaGetLastError();
}

cudaError_t launch_cg_rr(cudaStream_t st, const Ctrl* ctrl, CgScal* cs, int64_t m, const double* r,
                         int init) {
  k_cg_rr<<<1, 1024, 0, st>>>(ctrl, cs, m, r, init);
  return cudaGetLastError();
}

}  // namespace rs
