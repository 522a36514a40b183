// Iterate and residual update of Algorithm 2 (Section 6.3) with the residual
// recursion of eq. (53):
//   w^{k+1} = (1 + beta_k) w^k - beta_k w^{k-1} - gamma_k (S delta)
//   r^{k+1} = (1 + beta_k) r^k - beta_k r^{k-1} - gamma_k (A S delta)
// with (A S delta)_i = sum_j (S^T A)[j, i] delta_j (A symmetric), fused with the
// squared norm of r^{k+1}, the history entry and the stopping test.
#include <map>
#include <mutex>
#include <utility>

#include "rs_kernels.cuh"

namespace rs {

constexpr int kUpdCols = 32;   // elements i per block
constexpr int kUpdWarps = 16;  // warps splitting the tau rows (4 row loads in flight each)

int update_blocks(int64_t m) { return ceil_div(m, kUpdCols); }

template <typename T> struct AccT { using type = double; };
template <> struct AccT<float> { using type = float; };

template <typename T>
__global__ void __launch_bounds__(512) k_update(Ctrl* __restrict__ ctrl, PlanView plan,
                                                RowsView<T> rows, int64_t m, int64_t tau,
                                                UpdateArgs a) {
  using TA = typename AccT<T>::type;
  if (halted(ctrl)) return;
  __shared__ TA red[kUpdWarps][kUpdCols + 1];
  __shared__ TA ured[kUpdWarps][kUpdCols + 1];
  __shared__ double s_part[kUpdWarps];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t k = ctrl->k;
  const int64_t i = (int64_t)blockIdx.x * kUpdCols + lane;
  const int64_t slot = k - ctrl->k0;
  const int32_t* perm = plan.perm ? plan.perm + slot * plan.perm_stride : nullptr;
  const T* SA = rows.SA ? rows.SA + slot * rows.sa_slot : nullptr;
  const T* ST = rows.ST ? rows.ST + slot * rows.st_slot : nullptr;

  TA acc = TA(0), uacc = TA(0);
  if (i < m) {
    auto rowp = [&](int64_t j) -> const T* {
      return SA ? SA + j * rows.ldsa : rows.A + (int64_t)entry_row(perm[j]) * rows.lda;
    };
    if (ST)  // Gaussian: (S delta)_i = sum_j ST[j, i] delta_j
      for (int64_t j = w; j < tau; j += kUpdWarps) uacc += (TA)ST[j * rows.lda + i] * (TA)a.delta[j];
    int64_t j = w;
    // four independent row loads in flight per warp; the sum keeps the j order
    for (; j + 3 * kUpdWarps < tau; j += 4 * kUpdWarps) {
      const T v0 = rowp(j)[i], v1 = rowp(j + kUpdWarps)[i];
      const T v2 = rowp(j + 2 * kUpdWarps)[i], v3 = rowp(j + 3 * kUpdWarps)[i];
      acc += (TA)v0 * (TA)a.delta[j];
      acc += (TA)v1 * (TA)a.delta[j + kUpdWarps];
      acc += (TA)v2 * (TA)a.delta[j + 2 * kUpdWarps];
      acc += (TA)v3 * (TA)a.delta[j + 3 * kUpdWarps];
    }
    for (; j < tau; j += kUpdWarps) acc += (TA)rowp(j)[i] * (TA)a.delta[j];
  }
  red[w][lane] = acc;
  ured[w][lane] = uacc;
  __syncthreads();
  if (w == 0) {
    double sq = 0.0;
    if (i < m) {
      TA s = TA(0);
#pragma unroll
      for (int q = 0; q < kUpdWarps; ++q) s += red[q][lane];
      const double g = a.gam[k], b = a.bet[k];
      double ui;
      if (ST) {
        TA us = TA(0);
#pragma unroll
        for (int q = 0; q < kUpdWarps; ++q) us += ured[q][lane];
        ui = (double)us;
      } else {
        ui = a.u[i];
        a.u[i] = 0.0;
      }
      const double wi = a.w[i], wpi = a.wp[i], ri = a.r[i], rpi = a.rp[i];
      const double wn = (1.0 + b) * wi - b * wpi - g * ui;
      const double rn = (1.0 + b) * ri - b * rpi - g * (double)s;
      a.wp[i] = wi; a.w[i] = wn;
      a.rp[i] = ri; a.r[i] = rn;
      sq = rn * rn;
    }
    sq = warp_sum(sq);
    if (lane == 0) a.partials[blockIdx.x] = sq;
  }
  // last block to finish sums the partials in block order (deterministic)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double part = 0.0;
  for (int64_t b = threadIdx.x; b < gridDim.x; b += blockDim.x)
    part += *((volatile double*)&a.partials[b]);
  part = warp_sum(part);
  if (lane == 0) s_part[w] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < kUpdWarps; ++q) tot += s_part[q];
    const double rel = sqrt(tot) / ctrl->r0;
    a.hist[k + 1] = rel;
    const int64_t kn = k + 1;
    ctrl->k = kn;
    ctrl->ticket = 0u;
    if (!isfinite(rel)) {
      ctrl->status = 4;  // RS_ENUMERIC
      ctrl->stop = 1;
    } else if (!ctrl->no_stop && rel <= ctrl->tol) {
      if (a.mixed) ctrl->pending = 1; else ctrl->stop = 1;
    }
    if (kn >= ctrl->max_iters) ctrl->stop = 1;
    __threadfence();
  }
}

template <typename T>
cudaError_t launch_update(cudaStream_t st, Ctrl* ctrl, PlanView plan, RowsView<T> rows, int64_t m,
                          int64_t tau, UpdateArgs a) {
  k_update<T><<<update_blocks(m), 32 * kUpdWarps, 0, st>>>(ctrl, plan, rows, m, tau, a);
  return cudaGetLastError();
}

__global__ void k_init_state(int64_t m, const double* __restrict__ b, double* __restrict__ w,
                             double* __restrict__ wp, double* __restrict__ r,
                             double* __restrict__ rp, double* __restrict__ u) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    w[i] = 0.0; wp[i] = 0.0; u[i] = 0.0;
    r[i] = -b[i]; rp[i] = -b[i];
  }
}

cudaError_t launch_init_state(cudaStream_t st, int64_t m, const double* b, double* w, double* wp,
                              double* r, double* rp, double* u) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 1024));
  k_init_state<<<blocks, 256, 0, st>>>(m, b, w, wp, r, rp, u);
  return cudaGetLastError();
}

// The maximum dynamic shared memory of a kernel is a per-function attribute: a launcher
// that set it to its own launch's size would lower it for other launches of the same
// function already captured in a CUDA graph (the batch captures one launch per
// problem, of uneven sizes). Raised only, per function and device.
cudaError_t set_smem_max(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[std::make_pair(func, dev)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

__global__ void k_cast_f64_f32(const double* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

cudaError_t launch_cast_f64_f32(cudaStream_t st, const double* in, int64_t n, float* out) {
  const int64_t b = (n + 255) / 256;
  k_cast_f64_f32<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(in, n, out);
  return cudaGetLastError();
}

// out = s * in (the mean of the iterates from their running sum)
__global__ void k_scale(const double* __restrict__ in, double s, int64_t m, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = s * in[i];
}

cudaError_t launch_scale(cudaStream_t st, const double* in, double s, int64_t m, double* out) {
  k_scale<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(in, s, m, out);
  return cudaGetLastError();
}

// start of a chunk: k0 = k. With predict = 2 (plain persistent path, whose FP64
// recursive residual is exact up to rounding and tested every iteration) it also
// sets the convergence forecast: kcap ends the chunk where the decay rate of the
// relative residual since the previous chunk's start reaches tol, with a margin, so
// that phase 1 forms no slot past it. (The mixed path sets kcap after each FP64
// refresh instead.)
__global__ void k_chunk_begin(Ctrl* ctrl, const double* __restrict__ hist) {
  const int64_t k = ctrl->k;
  if (ctrl->predict == 2 && hist != nullptr && !ctrl->stop) {
    const double rel = (k == 0) ? 1.0 : hist[k];
    int64_t cap = 0;
    if (ctrl->pk >= 0 && k > ctrl->pk && rel > ctrl->tol && ctrl->prel > rel && rel > 0.0) {
      const double rate = log(rel / ctrl->prel) / (double)(k - ctrl->pk);  // < 0
      const double left = log(ctrl->tol / rel) / rate;                      // > 0
      if (left < 1e9) cap = k + (int64_t)ceil(1.25 * left) + 8;
    }
    ctrl->kcap = cap;
    ctrl->pk = k;
    ctrl->prel = rel;
  }
  ctrl->k0 = k;
}

cudaError_t launch_chunk_begin(cudaStream_t st, Ctrl* ctrl, const double* hist) {
  k_chunk_begin<<<1, 1, 0, st>>>(ctrl, hist);
  return cudaGetLastError();
}

template cudaError_t launch_update<float>(cudaStream_t, Ctrl*, PlanView, RowsView<float>, int64_t,
                                          int64_t, UpdateArgs);
template cudaError_t launch_update<double>(cudaStream_t, Ctrl*, PlanView, RowsView<double>,
                                           int64_t, int64_t, UpdateArgs);

}  // namespace rs
