// Forming the linear system of eq. (4) (A = X^T X + lambda I, b = X^T y for the
// primal eq. (2); A = X X^T + lambda I, b = y for the dual eq. (3)) and evaluating
// the true residual A v - b through X in FP64 without forming A.
#include <algorithm>
#include <mutex>
#include <string>

#include "ridgesketch.h"
#include "rs_gemm.cuh"
#include "rs_kernels.cuh"

namespace rs {

template <typename TI, typename TO>
cudaError_t launch_form_A(cudaStream_t st, const TI* X, int64_t n, int64_t d, int dual,
                          double lambda, TO* A, int64_t lda) {
  using TA = TO;  // FP64 output accumulates in FP64, FP32 output in FP32
  cudaError_t e;
  int64_t m;
  if (!dual) {  // A[i, j] = sum_k X[k, i] X[k, j]
    m = d;
    e = gemm_strided<TI, TA, TO>(st, d, d, n, X, 1, d, X, d, 1, A, lda, lambda, 1);
  } else {      // A[i, j] = sum_k X[i, k] X[j, k]
    m = n;
    e = gemm_strided<TI, TA, TO>(st, n, n, d, X, d, 1, X, 1, d, A, lda, lambda, 1);
  }
  if (e != cudaSuccess) return e;
  dim3 g((unsigned)((m + 31) / 32), (unsigned)((m + 31) / 32));
  k_mirror_lower<TO><<<g, dim3(32, 32), 0, st>>>(A, m, lda);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mirror_lower(cudaStream_t st, T* A, int64_t m, int64_t lda) {
  dim3 g((unsigned)((m + 31) / 32), (unsigned)((m + 31) / 32));
  k_mirror_lower<T><<<g, dim3(32, 32), 0, st>>>(A, m, lda);
  return cudaGetLastError();
}
template cudaError_t launch_mirror_lower<float>(cudaStream_t, float*, int64_t, int64_t);
template cudaError_t launch_mirror_lower<double>(cudaStream_t, double*, int64_t, int64_t);

// ---- X^T v: column sums of X weighted by v, chunked over rows, FP64 ----
constexpr int64_t kXtRows = 256;

// (n more for the float pairs of v of launch_xt_v_pairs)
size_t xt_part_elems(int64_t n, int64_t d) {
  return (size_t)((n + kXtRows - 1) / kXtRows) * d + (size_t)n;
}

template <typename TI>
__global__ void __launch_bounds__(256) k_xt_v_part(const TI* __restrict__ X, int64_t n, int64_t d,
                                                   const double* __restrict__ v,
                                                   double* __restrict__ part,
                                                   const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (j >= d) return;
  const int64_t i0 = c * kXtRows, i1 = min(n, i0 + kXtRows);
  double acc = 0.0;
  for (int64_t i = i0; i < i1; ++i) acc += (double)X[i * d + j] * v[i];
  part[c * d + j] = acc;
}

// out[j] = sum over c of part[c * d + j], in a fixed order: a block takes 32 columns,
// warp q sums the parts c = q, q + 8, q + 16, ... in order, and the eight warps' sums
// are added in q order
constexpr int kSumWarps = 8;
__global__ void __launch_bounds__(32 * kSumWarps) k_sum_parts(const double* __restrict__ part,
                                                              int64_t nchunk, int64_t d,
                                                              double* __restrict__ out,
                                                              const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  __shared__ double s[kSumWarps][32];
  const int lx = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lx;
  double acc = 0.0;
  if (j < d)
    for (int64_t c = q; c < nchunk; c += kSumWarps) acc += part[c * d + j];
  s[q][lx] = acc;
  __syncthreads();
  if (q == 0 && j < d) {
    double t = s[0][lx];
#pragma unroll
    for (int k = 1; k < kSumWarps; ++k) t += s[k][lx];
    out[j] = t;
  }
}
void launch_sum_parts(cudaStream_t st, const double* part, int64_t nchunk, int64_t d, double* out,
                      const int32_t* stop) {
  k_sum_parts<<<(unsigned)((d + 31) / 32), 32 * kSumWarps, 0, st>>>(part, nchunk, d, out, stop);
}

template <typename TI>
cudaError_t launch_xt_v(cudaStream_t st, const TI* X, int64_t n, int64_t d, const double* v,
                        double* out, double* part, const int32_t* stop) {
  const int64_t nchunk = (n + kXtRows - 1) / kXtRows;
  dim3 g((unsigned)((d + 255) / 256), (unsigned)nchunk);
  k_xt_v_part<TI><<<g, 256, 0, st>>>(X, n, d, v, part, stop);
  launch_sum_parts(st, part, nchunk, d, out, stop);
  return cudaGetLastError();
}

// ---- X v: one warp per row, FP64 ----
template <typename TI>
__global__ void __launch_bounds__(256) k_x_v(const TI* __restrict__ X, int64_t n, int64_t d,
                                             const double* __restrict__ v,
                                             double* __restrict__ out,
                                             const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  double acc = 0.0;
  for (int64_t j = lane; j < d; j += 32) acc += (double)X[i * d + j] * v[j];
  acc = warp_sum(acc);
  if (lane == 0) out[i] = acc;
}

template <typename TI>
cudaError_t launch_x_v(cudaStream_t st, const TI* X, int64_t n, int64_t d, const double* v,
                       double* out, const int32_t* stop) {
  k_x_v<TI><<<(unsigned)((n + 7) / 8), 256, 0, st>>>(X, n, d, v, out, stop);
  return cudaGetLastError();
}

// ---- A v = X^T (X v) in one pass over FP32 X, FP64-accurate through float pairs ----
// X holds exact FP32 data; v is FP64. Products x * v_hi are split exactly with a fused
// multiply-add (x * v = p + e, e = fma(x, v_hi, -p)), sums are carried as unevaluated
// float pairs with the error-free two-sum (Knuth); v_lo = fp32(v - v_hi) adds its small
// product directly. Each block takes a range of rows, two at a time: for every row i
// it forms u_i = x_i . v (block reduction of pairs), then adds u_i x_i to its
// per-column pairs; per-block column sums go to `part` (blocks x d) and are added in
// block order. Inside a warp the two row dots are reduced by a reduce-scatter: the
// first exchange leaves each half-warp one row, so later exchanges carry one pair
// instead of two (the same pairing tree, so the same sums). Two blocks of 128
// registers per thread share an SM. X is read with evict-first loads, as float4 when
// its rows are 16-byte aligned, so that its stream does not push A (read again by
// the next chunk's phase 1) out of L2.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  ah = __fadd_rn(s, e);
  al = __fsub_rn(e, __fsub_rn(ah, s));
}

// column of the c-th value of thread tid: strided singly, or four consecutive (V4)
template <int NT, bool V4>
__device__ __forceinline__ int64_t df_col(int tid, int c) {
  if constexpr (V4) return 4 * ((int64_t)tid + (int64_t)NT * (c >> 2)) + (c & 3);
  else return tid + (int64_t)NT * c;
}

template <int NC, bool V4, int NT = 256>
__global__ void __launch_bounds__(NT, 2) k_xtx_v_df(const float* __restrict__ X, int64_t n, int64_t d,
                                                     const double* __restrict__ v,
                                                     double* __restrict__ part,
                                                     const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  constexpr int R = 2;  // rows per step
  constexpr int NW = NT / 32;
  __shared__ float s_h[NW][R], s_l[NW][R];
  __shared__ float u_h[R], u_l[R];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned full = 0xffffffffu;
  float vh[NC], vl[NC], ah[NC], al[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t col = df_col<NT, V4>(tid, c);
    const double vv = col < d ? v[col] : 0.0;
    vh[c] = (float)vv;
    vl[c] = (float)(vv - (double)vh[c]);
    ah[c] = 0.f;
    al[c] = 0.f;
  }
  const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * rows_per, i1 = min(n, i0 + rows_per);
  for (int64_t ib = i0; ib < i1; ib += R) {
    float x[R][NC];
    float dh[R], dl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      dh[r] = 0.f;
      dl[r] = 0.f;
      const int64_t i = ib + r;
      if constexpr (V4) {
#pragma unroll
        for (int g = 0; g < NC / 4; ++g) {
          const int64_t col = df_col<NT, true>(tid, 4 * g);
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i < i1 && col < d) q = __ldcs(reinterpret_cast<const float4*>(X + i * d + col));
          x[r][4 * g] = q.x;
          x[r][4 * g + 1] = q.y;
          x[r][4 * g + 2] = q.z;
          x[r][4 * g + 3] = q.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int64_t col = df_col<NT, false>(tid, c);
          x[r][c] = (i < i1 && col < d) ? __ldcs(X + i * d + col) : 0.f;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float p = __fmul_rn(x[r][c], vh[c]);
        const float e = __fmaf_rn(x[r][c], vh[c], -p);
        float s, er;
        two_sum(dh[r], p, s, er);
        dh[r] = s;
        dl[r] = __fmaf_rn(x[r][c], vl[c], __fadd_rn(dl[r], __fadd_rn(er, e)));
      }
    // warp reduction of the two row dots: after the exchange across half-warps, lanes
    // 0-15 carry row 0 and lanes 16-31 row 1
    {
      const bool up = (lane & 16) != 0;
      float kh = up ? dh[1] : dh[0], kl = up ? dl[1] : dl[0];
      const float oh = __shfl_xor_sync(full, up ? dh[0] : dh[1], 16);
      const float ol = __shfl_xor_sync(full, up ? dl[0] : dl[1], 16);
      df_add(kh, kl, oh, ol);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const float ph = __shfl_xor_sync(full, kh, o);
        const float pl = __shfl_xor_sync(full, kl, o);
        df_add(kh, kl, ph, pl);
      }
      if ((lane & 15) == 0) {
        s_h[wid][lane >> 4] = kh;
        s_l[wid][lane >> 4] = kl;
      }
    }
    __syncthreads();
    if (tid < R) {
      float h = s_h[0][tid], l = s_l[0][tid];
      for (int q = 1; q < NW; ++q) df_add(h, l, s_h[q][tid], s_l[q][tid]);
      u_h[tid] = h;
      u_l[tid] = l;
    }
    __syncthreads();
    // column pairs += u_i x_i. No barrier after this: the next step writes s_h before
    // its first barrier, which follows every thread's reads of u_h here, and u_h only
    // after that barrier.
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float uh = u_h[r], ul = u_l[r];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float p = __fmul_rn(x[r][c], uh);
        const float e = __fmaf_rn(x[r][c], uh, -p);
        float s, er;
        two_sum(ah[c], p, s, er);
        ah[c] = s;
        al[c] = __fmaf_rn(x[r][c], ul, __fadd_rn(al[c], __fadd_rn(er, e)));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t col = df_col<NT, V4>(tid, c);
    if (col < d) part[blockIdx.x * d + col] = (double)ah[c] + (double)al[c];
  }
}

// the kernel for d <= 4096: float4 loads when every row of X starts on 16 bytes
cudaError_t launch_xtx_df_kernel(cudaStream_t st, int G, const float* X, int64_t n, int64_t d,
                                 const double* v, double* part, const int32_t* stop) {
  const bool v4 = (d % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  if (d <= 1024) {
    if (v4) k_xtx_v_df<4, true><<<G, 256, 0, st>>>(X, n, d, v, part, stop);
    else k_xtx_v_df<4, false><<<G, 256, 0, st>>>(X, n, d, v, part, stop);
  } else if (d <= 2048) {
    if (v4) k_xtx_v_df<8, true><<<G, 256, 0, st>>>(X, n, d, v, part, stop);
    else k_xtx_v_df<8, false><<<G, 256, 0, st>>>(X, n, d, v, part, stop);
  } else if (d <= 4096) {
    if (v4) k_xtx_v_df<16, true><<<G, 256, 0, st>>>(X, n, d, v, part, stop);
    else k_xtx_v_df<16, false><<<G, 256, 0, st>>>(X, n, d, v, part, stop);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int xtx_df_blocks() { return 2 * 152; }  // two per SM

cudaError_t launch_xtx_v_df(cudaStream_t st, const float* X, int64_t n, int64_t d, const double* v,
                            double* out, double* part, const int32_t* stop) {
  const int G = xtx_df_blocks();
  const cudaError_t e = launch_xtx_df_kernel(st, G, X, n, d, v, part, stop);
  if (e != cudaSuccess) return e;
  launch_sum_parts(st, part, G, d, out, stop);
  return cudaGetLastError();
}

// ---- X^T X V for up to four vectors in one pass over FP32 X (same arithmetic) ----
// The vectors' float pairs sit in shared memory (nv x d); every row of X is loaded
// once and serves all nv row dots and all nv column updates. The kernel returns at
// once when every vector is flagged in `skip`.
template <int NC, int R>
__global__ void __launch_bounds__(512, 1) k_xtx_multi_df(const float* __restrict__ X, int64_t n,
                                                         int64_t d, int nv,
                                                         const double* __restrict__ V,
                                                         double* __restrict__ part,
                                                         const int32_t* __restrict__ skip) {
  constexpr int NVM = 4, NWM = 16;
  if (skip != nullptr) {
    int all = 1;
    for (int q = 0; q < nv; ++q) all &= (skip[q] != 0);
    if (all) return;
  }
  extern __shared__ float2 sv[];  // nv x d: (hi, lo) of the vectors
  __shared__ float s_h[NWM][R][NVM], s_l[NWM][R][NVM];
  __shared__ float u_h[R][NVM], u_l[R][NVM];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int NT = blockDim.x;
  for (int64_t e = tid; e < (int64_t)nv * d; e += NT) {
    const double vv = V[e];
    const float h = (float)vv;
    sv[e] = make_float2(h, (float)(vv - (double)h));
  }
  __syncthreads();
  float ah[NVM][NC], al[NVM][NC];
#pragma unroll
  for (int q = 0; q < NVM; ++q)
#pragma unroll
    for (int c = 0; c < NC; ++c) { ah[q][c] = 0.f; al[q][c] = 0.f; }
  const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * rows_per, i1 = min(n, i0 + rows_per);
  for (int64_t ib = i0; ib < i1; ib += R) {
    float x[R][NC];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int64_t col = tid + (int64_t)NT * c;
        x[r][c] = (ib + r < i1 && col < d) ? __ldg(X + (ib + r) * d + col) : 0.f;
      }
    float dh[R][NVM], dlo[R][NVM];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int q = 0; q < NVM; ++q) { dh[r][q] = 0.f; dlo[r][q] = 0.f; }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t col = tid + (int64_t)NT * c;
      if (col >= d) break;
#pragma unroll
      for (int q = 0; q < NVM; ++q) {
        if (q >= nv) break;
        const float2 v = sv[(int64_t)q * d + col];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float p = __fmul_rn(x[r][c], v.x);
          const float e = __fmaf_rn(x[r][c], v.x, -p);
          float s, er;
          two_sum(dh[r][q], p, s, er);
          dh[r][q] = s;
          dlo[r][q] = __fmaf_rn(x[r][c], v.y, __fadd_rn(dlo[r][q], __fadd_rn(er, e)));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int q = 0; q < NVM; ++q) {
        if (q >= nv) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, dh[r][q], o);
          const float ol = __shfl_xor_sync(0xffffffffu, dlo[r][q], o);
          df_add(dh[r][q], dlo[r][q], oh, ol);
        }
        if (lane == 0) { s_h[wid][r][q] = dh[r][q]; s_l[wid][r][q] = dlo[r][q]; }
      }
    __syncthreads();
    if (tid < R * NVM) {
      const int r = tid / NVM, q = tid % NVM;
      if (q < nv) {
        float h = s_h[0][r][q], l = s_l[0][r][q];
        for (int w = 1; w < nw; ++w) df_add(h, l, s_h[w][r][q], s_l[w][r][q]);
        u_h[r][q] = h;
        u_l[r][q] = l;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int q = 0; q < NVM; ++q) {
        if (q >= nv) break;
        const float uh = u_h[r][q], ul = u_l[r][q];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float p = __fmul_rn(x[r][c], uh);
          const float e = __fmaf_rn(x[r][c], uh, -p);
          float s, er;
          two_sum(ah[q][c], p, s, er);
          ah[q][c] = s;
          al[q][c] = __fmaf_rn(x[r][c], ul, __fadd_rn(al[q][c], __fadd_rn(er, e)));
        }
      }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NVM; ++q) {
    if (q >= nv) break;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t col = tid + (int64_t)NT * c;
      if (col < d) part[((int64_t)blockIdx.x * nv + q) * d + col] = (double)ah[q][c] + (double)al[q][c];
    }
  }
}

// out[q] = sum over blocks of part[block][q] in block order
__global__ void k_sum_parts_multi(const double* __restrict__ part, int nblk, int nv, int64_t d,
                                  double* __restrict__ out, const int32_t* __restrict__ skip) {
  const int q = blockIdx.y;
  if (skip != nullptr && skip[q]) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[((int64_t)b * nv + q) * d + j];
  out[(int64_t)q * d + j] = acc;
}

int xtx_multi_blocks() { return 152; }

cudaError_t launch_xtx_multi_df(cudaStream_t st, const float* X, int64_t n, int64_t d, int nv,
                                const double* V, double* out, double* part, const int32_t* skip) {
  if (nv < 1 || nv > 4 || d > 4096) return cudaErrorInvalidValue;
  const int G = xtx_multi_blocks();
  const size_t smem = (size_t)nv * d * sizeof(float2);
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kern) {
    e = set_smem_max((const void*)kern, (size_t)((int)smem));
    if (e == cudaSuccess) kern<<<G, 512, smem, st>>>(X, n, d, nv, V, part, skip);
  };
  if (d <= 1024) go(k_xtx_multi_df<2, 2>);
  else if (d <= 2048) go(k_xtx_multi_df<4, 2>);
  else go(k_xtx_multi_df<8, 1>);
  if (e != cudaSuccess) return e;
  k_sum_parts_multi<<<dim3((unsigned)((d + 255) / 256), (unsigned)nv), 256, 0, st>>>(part, G, nv, d,
                                                                                      out, skip);
  return cudaGetLastError();
}

// ---- X^T X W for up to four vectors in two passes (same float-pair arithmetic) ----
// Pass 1: U = X W, a warp per row of X (lanes over the columns, the vectors' float
// pairs in shared memory), the row dots reduced across the warp as float pairs; no
// block-wide synchronisation. Pass 2: V = X^T U, a thread per column over a range
// of rows (the range's U in shared memory), per-range sums added in range order.
template <int NV>
__global__ void __launch_bounds__(1024) k_xw_df(const float* __restrict__ X, int64_t n, int64_t d,
                                               int nv, const double* __restrict__ W,
                                               float2* __restrict__ U,
                                               const int32_t* __restrict__ skip) {
  if (skip != nullptr) {
    int all = 1;
    for (int q = 0; q < nv; ++q) all &= (skip[q] != 0);
    if (all) return;
  }
  extern __shared__ float2 sw[];  // d x NV: (hi, lo) of the vectors, column-major in q
  for (int64_t e = threadIdx.x; e < d * NV; e += blockDim.x) {
    const int64_t c = e / NV;
    const int q = (int)(e - c * NV);
    const double v = q < nv ? W[(int64_t)q * d + c] : 0.0;
    const float h = (float)v;
    sw[e] = make_float2(h, (float)(v - (double)h));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwg = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wg; i < n; i += nwg) {
    float dh[NV], dlo[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) { dh[q] = 0.f; dlo[q] = 0.f; }
    const float* xr = X + i * d;
    for (int64_t c0 = lane; c0 < d; c0 += 128) {  // four columns in flight per lane
      float xs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xs[u] = (c0 + 32 * u < d) ? __ldg(xr + c0 + 32 * u) : 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t c = c0 + 32 * u;
        if (c >= d) break;
        const float x = xs[u];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const float2 v = sw[c * NV + q];
          const float p = __fmul_rn(x, v.x);
          const float e = __fmaf_rn(x, v.x, -p);
          float s, er;
          two_sum(dh[q], p, s, er);
          dh[q] = s;
          dlo[q] = __fmaf_rn(x, v.y, __fadd_rn(dlo[q], __fadd_rn(er, e)));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, dh[q], o);
        const float ol = __shfl_xor_sync(0xffffffffu, dlo[q], o);
        df_add(dh[q], dlo[q], oh, ol);
      }
    }
    if (lane < NV) {
      float h = dh[0], l = dlo[0];
#pragma unroll
      for (int q = 1; q < NV; ++q)
        if (lane == q) { h = dh[q]; l = dlo[q]; }
      U[i * NV + lane] = make_float2(h, l);
    }
  }
}

constexpr int kXtuCols = 256;  // columns per block of pass 2
constexpr int kXtuRows = 512;  // rows per block of pass 2

template <int NV>
__global__ void __launch_bounds__(kXtuCols) k_xtu_df(const float* __restrict__ X, int64_t n,
                                                     int64_t d, int nv,
                                                     const float2* __restrict__ U,
                                                     double* __restrict__ part,
                                                     const int32_t* __restrict__ skip,
                                                     int64_t rb0 = 0) {
  if (skip != nullptr) {
    int all = 1;
    for (int q = 0; q < nv; ++q) all &= (skip[q] != 0);
    if (all) return;
  }
  __shared__ float2 su[kXtuRows * NV];
  const int64_t rb = rb0 + blockIdx.y;  // row block
  const int64_t r0 = rb * kXtuRows;
  const int64_t r1 = min(n, r0 + kXtuRows);
  for (int64_t e = threadIdx.x; e < (r1 - r0) * NV; e += blockDim.x) su[e] = U[r0 * NV + e];
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * kXtuCols + threadIdx.x;
  if (c >= d) return;
  float ah[NV], al[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) { ah[q] = 0.f; al[q] = 0.f; }
  for (int64_t i = r0; i < r1; ++i) {
    const float x = __ldg(X + i * d + c);
    const float2* u = su + (i - r0) * NV;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const float2 uq = u[q];
      const float p = __fmul_rn(x, uq.x);
      const float e = __fmaf_rn(x, uq.x, -p);
      float s, er;
      two_sum(ah[q], p, s, er);
      ah[q] = s;
      al[q] = __fmaf_rn(x, uq.y, __fadd_rn(al[q], __fadd_rn(er, e)));
    }
  }
#pragma unroll
  for (int q = 0; q < NV; ++q)
    if (q < nv) part[(rb * nv + q) * d + c] = (double)ah[q] + (double)al[q];
}

// U[i] = (hi, lo) float pair of v[i]
__global__ void k_split_pairs(const double* __restrict__ v, int64_t n, float2* __restrict__ U,
                              const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = v[i];
  const float h = (float)x;
  U[i] = make_float2(h, (float)(x - (double)h));
}

// X^T v for FP32 X in float-pair arithmetic (the FP64 pipe is too narrow on this GPU
// for one FP64 FMA per entry of X): v split into float pairs, then the column sums
// of pass 2 of the two-pass product, then the FP64 sum of the row blocks' sums.
// in three steps for row ranges: split v, the column sums of the 512-row blocks of
// rows [r0, r1) (r0 a multiple of 512), the sum of all blocks
cudaError_t xt_pairs_split(cudaStream_t st, const double* v, int64_t n, int64_t d, double* part,
                           const int32_t* stop) {
  const int64_t nblk = (n + kXtuRows - 1) / kXtuRows;
  float2* U = reinterpret_cast<float2*>(part + nblk * d);  // after the row blocks' sums
  k_split_pairs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, n, U, stop);
  return cudaGetLastError();
}
cudaError_t xt_pairs_rows(cudaStream_t st, const float* X, int64_t n, int64_t d, double* part,
                          int64_t r0, int64_t r1, const int32_t* stop) {
  if (r0 % kXtuRows != 0 || r1 <= r0) return cudaErrorInvalidValue;
  const int64_t nblk = (n + kXtuRows - 1) / kXtuRows;
  const float2* U = reinterpret_cast<const float2*>(part + nblk * d);
  const int64_t b0 = r0 / kXtuRows, b1 = (std::min(r1, n) + kXtuRows - 1) / kXtuRows;
  const dim3 g2((unsigned)((d + kXtuCols - 1) / kXtuCols), (unsigned)(b1 - b0));
  k_xtu_df<1><<<g2, kXtuCols, 0, st>>>(X, n, d, 1, U, part, stop, b0);
  return cudaGetLastError();
}
cudaError_t xt_pairs_sum(cudaStream_t st, int64_t n, int64_t d, double* part, double* out,
                         const int32_t* stop) {
  const int64_t nblk = (n + kXtuRows - 1) / kXtuRows;
  launch_sum_parts(st, part, nblk, d, out, stop);
  return cudaGetLastError();
}

cudaError_t launch_xt_v_pairs(cudaStream_t st, const float* X, int64_t n, int64_t d,
                              const double* v, double* out, double* part, const int32_t* stop) {
  cudaError_t e = xt_pairs_split(st, v, n, d, part, stop);
  if (e == cudaSuccess) e = xt_pairs_rows(st, X, n, d, part, 0, n, stop);
  if (e == cudaSuccess) e = xt_pairs_sum(st, n, d, part, out, stop);
  return e;
}

int64_t xtx_two_pass_part(int64_t n, int64_t d, int nv) {
  return ((n + kXtuRows - 1) / kXtuRows) * nv * d;
}

cudaError_t launch_xtx_two_pass(cudaStream_t st, const float* X, int64_t n, int64_t d, int nv,
                                const double* W, double* out, float2* U, double* part,
                                const int32_t* skip) {
  if (nv < 1 || nv > 4) return cudaErrorInvalidValue;
  const int NV = nv <= 1 ? 1 : (nv <= 2 ? 2 : 4);
  const size_t smem = (size_t)d * NV * sizeof(float2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const unsigned g1 = (unsigned)std::min<int64_t>((n + 31) / 32, 152);
  const dim3 g2((unsigned)((d + kXtuCols - 1) / kXtuCols), (unsigned)((n + kXtuRows - 1) / kXtuRows));
  cudaError_t e = cudaSuccess;
  auto go = [&](auto k1, auto k2) {
    e = set_smem_max((const void*)k1, (size_t)((int)smem));
    if (e != cudaSuccess) return;
    k1<<<g1, 1024, smem, st>>>(X, n, d, nv, W, U, skip);
    k2<<<g2, kXtuCols, 0, st>>>(X, n, d, nv, U, part, skip, (int64_t)0);
  };
  if (NV == 1) go(k_xw_df<1>, k_xtu_df<1>);
  else if (NV == 2) go(k_xw_df<2>, k_xtu_df<2>);
  else go(k_xw_df<4>, k_xtu_df<4>);
  if (e != cudaSuccess) return e;
  k_sum_parts_multi<<<dim3((unsigned)((d + 255) / 256), (unsigned)nv), 256, 0, st>>>(
      part, (int)g2.y, nv, d, out, skip);
  return cudaGetLastError();
}

// ---- kernel ridge (Section 2.2) ----
// K_ij = exp(-||p_i - p_j||^2 / (2 sigma^2)) (eq. (Gausskernel)) in FP64 from the
// differences of the points (no norm expansion): 32 x 32 output tiles, the two row
// blocks of points staged in shared memory in chunks of 32 features
template <typename TP>
__global__ void __launch_bounds__(256) k_rbf_f64(const TP* __restrict__ P, int64_t n, int64_t d,
                                                 double inv2s2, double* __restrict__ K,
                                                 int64_t ldK) {
  __shared__ double si[32][33], sj[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k0 = 0; k0 < d; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int64_t k = k0 + tx;
      si[r][tx] = (i0 + r < n && k < d) ? (double)P[(i0 + r) * d + k] : 0.0;
      sj[r][tx] = (j0 + r < n && k < d) ? (double)P[(j0 + r) * d + k] : 0.0;
    }
    __syncthreads();
    const int kn = (int)((d - k0) < 32 ? (d - k0) : 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      for (int k = 0; k < kn; ++k) {
        const double df = si[r][k] - sj[tx][k];
        acc[q] = fma(df, df, acc[q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < n && j < n) K[i * ldK + j] = (i == j) ? 1.0 : exp(-acc[q] * inv2s2);
  }
}

template <typename TP>
cudaError_t launch_rbf_f64(cudaStream_t st, const TP* P, int64_t n, int64_t d, double sigma,
                           double* K, int64_t ldK) {
  const dim3 g((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  k_rbf_f64<TP><<<g, 256, 0, st>>>(P, n, d, 1.0 / (2.0 * sigma * sigma), K, ldK);
  return cudaGetLastError();
}
template cudaError_t launch_rbf_f64<double>(cudaStream_t, const double*, int64_t, int64_t, double,
                                            double*, int64_t);
template cudaError_t launch_rbf_f64<float>(cudaStream_t, const float*, int64_t, int64_t, double,
                                           double*, int64_t);

// A += lambda (K - I): from K^T K + lambda I to K^T (K + lambda I) (eq. (kernelridge));
// the diagonal of the Gaussian kernel is 1, so only the off-diagonal entries change
template <typename T>
__global__ void k_add_offdiag(T* __restrict__ A, int64_t lda, const T* __restrict__ K, int64_t ldK,
                              int64_t n, double lambda) {
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && j < n && i != j) A[i * lda + j] = (T)((double)A[i * lda + j] + lambda * (double)K[i * ldK + j]);
}

template <typename T>
cudaError_t launch_add_offdiag(cudaStream_t st, T* A, int64_t lda, const T* K, int64_t ldK,
                               int64_t n, double lambda) {
  k_add_offdiag<T><<<dim3((unsigned)((n + 255) / 256), (unsigned)n), 256, 0, st>>>(A, lda, K, ldK,
                                                                                    n, lambda);
  return cudaGetLastError();
}
template cudaError_t launch_add_offdiag<float>(cudaStream_t, float*, int64_t, const float*, int64_t,
                                               int64_t, double);
template cudaError_t launch_add_offdiag<double>(cudaStream_t, double*, int64_t, const double*,
                                                int64_t, int64_t, double);

// ---- variant of the one-pass X^T X v that allocates nothing (rs_gram_apply_noalloc) ----
// The per-block column sums live in a fixed device array of this file instead of a
// buffer the caller or the library allocates: kNoAllocBlocks x kNoAllocMaxD doubles
// (2 MiB), held by every GPU that loads the library until the process exits.
constexpr int kNoAllocBlocks = 64;
constexpr int64_t kNoAllocMaxD = 4096;
static __device__ __align__(256) double g_noalloc_part[kNoAllocBlocks * kNoAllocMaxD];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};  // device address of g_noalloc_part, per device ordinal
}  // namespace

}  // namespace rs

extern "C" rs_status rs_gram_apply_noalloc(const float* X, int64_t n, int64_t d, const double* v,
                                           double* out, void* stream) {
  using namespace rs;
  if (X == nullptr || v == nullptr || out == nullptr) {
    set_global_error_msg("rs_gram_apply_noalloc: null pointer");
    return RS_EINVAL;
  }
  if (n < 1 || d < 1 || d > kNoAllocMaxD) {
    set_global_error_msg("rs_gram_apply_noalloc: need n >= 1 and 1 <= d <= 4096");
    return RS_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_global_error_msg("rs_gram_apply_noalloc: no usable current device");
    return RS_ECUDA;
  }
  void* part = nullptr;
  {
    // set-up on the first call on this device: the host-side name of the array is
    // not a device address, so ask the runtime for it (with this device current)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
      if (e != cudaSuccess || p == nullptr) {
        set_global_error_msg((std::string("rs_gram_apply_noalloc: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e)).c_str());
        return RS_ECUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    part = g_noalloc_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* pp = static_cast<double*>(part);
  // every block writes all d of its column sums, so nothing needs clearing first
  cudaError_t e = launch_xtx_df_kernel(st, kNoAllocBlocks, X, n, d, v, pp, nullptr);
  if (e == cudaSuccess) {
    launch_sum_parts(st, pp, kNoAllocBlocks, d, out, nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_global_error_msg((std::string("rs_gram_apply_noalloc: ") + cudaGetErrorString(e)).c_str());
    return RS_ECUDA;
  }
  return RS_OK;
}

namespace rs {

// ---- true residual r = v + lambda x - b ----
// mode 1: replace the recursive residual pair (r, r_prev) by (r_true, r_true - (r - r_prev))
//         and decide convergence on ||r_true|| / ||r^0||; mode 0: only *rel_out.
__global__ void __launch_bounds__(256) k_refresh_finish(Ctrl* __restrict__ ctrl, int mode, int64_t m,
                                                        const double* __restrict__ v,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ b, double lambda,
                                                        double* __restrict__ r,
                                                        double* __restrict__ rp,
                                                        double* __restrict__ partials,
                                                        double* __restrict__ hist,
                                                        double* __restrict__ rel_out) {
  __shared__ double s_red[32];
  __shared__ int s_last;
  if (mode == 1 && (*(volatile int32_t*)&ctrl->stop)) return;
  double sq = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double rt = v[i] + lambda * x[i] - b[i];
    if (mode == 1) {
      const double diff = r[i] - rp[i];
      r[i] = rt;
      rp[i] = rt - diff;
    }
    sq += rt * rt;
  }
  sq = block_sum(sq, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = sq;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double part = 0.0;
  for (int64_t q = threadIdx.x; q < gridDim.x; q += blockDim.x) part += *((volatile double*)&partials[q]);
  part = block_sum(part, s_red);
  if (threadIdx.x == 0) {
    ctrl->ticket = 0u;
    const double rel = sqrt(part) / ctrl->r0;
    if (mode == 1) {
      const int64_t k = ctrl->k;
      hist[k] = rel;
      ctrl->checked_k = k;
      if (!isfinite(rel)) {
        ctrl->status = 4;
        ctrl->stop = 1;
      } else if (rel <= ctrl->tol) {
        ctrl->stop = 1;
      }
      ctrl->pending = 0;
      if (k >= ctrl->max_iters) ctrl->stop = 1;
      if (ctrl->predict) {
        // forecast: the decay rate of the FP64 residual since the previous refresh
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
    } else {
      *rel_out = rel;
    }
    __threadfence();
  }
}

cudaError_t launch_refresh_finish(cudaStream_t st, Ctrl* ctrl, int mode, int64_t m, const double* v,
                                  const double* x, const double* b, double lambda, double* r,
                                  double* rp, double* partials, double* hist, double* rel_out) {
  int blocks = (int)std::min<int64_t>((m + 255) / 256, 152);
  if (blocks < 1) blocks = 1;
  k_refresh_finish<<<blocks, 256, 0, st>>>(ctrl, mode, m, v, x, b, lambda, r, rp, partials, hist,
                                           rel_out);
  return cudaGetLastError();
}

#define RS_INST(TI)                                                                            \
  template cudaError_t launch_xt_v<TI>(cudaStream_t, const TI*, int64_t, int64_t, const double*, \
                                       double*, double*, const int32_t*);                      \
  template cudaError_t launch_x_v<TI>(cudaStream_t, const TI*, int64_t, int64_t, const double*,  \
                                      double*, const int32_t*);                                              \
  template cudaError_t launch_form_A<TI, double>(cudaStream_t, const TI*, int64_t, int64_t, int, \
                                                 double, double*, int64_t);                    \
  template cudaError_t launch_form_A<TI, float>(cudaStream_t, const TI*, int64_t, int64_t, int,  \
                                                double, float*, int64_t);
RS_INST(float)
RS_INST(double)
#undef RS_INST

}  // namespace rs
