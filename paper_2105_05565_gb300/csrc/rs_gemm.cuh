// Tiled SIMT matrix product used where tensor cores do not apply (FP64) or the
// operand is small:  C[i*ldc + j] = sum_k P(i,k) Q(k,j)  (+ diag on i == j)
// with P(i,k) = P[i*p0 + k*p1], Q(k,j) = Q[k*q0 + j*q1] (any strides), so one
// kernel serves X^T X, X X^T, S^T A and (S^T A) S.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_common.cuh"

namespace rs {

template <typename TI, typename TA, typename TO>
__global__ void __launch_bounds__(256)
k_gemm_strided(int64_t M, int64_t N, int64_t K, const TI* P, int64_t p0, int64_t p1,
               const TI* Q, int64_t q0, int64_t q1, TO* C, int64_t ldc,
               double diag, int lower_only, const Ctrl* __restrict__ ctrl, int64_t bP,
               int64_t bQ, int64_t bC) {
  constexpr int BM = 64, BN = 64, BK = 16;
  // batched use (blockIdx.z = slot of a chunk): skip slots the solve will not reach
  if (ctrl != nullptr && (int64_t)blockIdx.z >= active_slots(ctrl, 0, gridDim.z)) return;
  P += (int64_t)blockIdx.z * bP;
  Q += (int64_t)blockIdx.z * bQ;
  C += (int64_t)blockIdx.z * bC;
  __shared__ TA sP[BK][BM + 4];
  __shared__ TA sQ[BK][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  if (lower_only && j0 > i0 + BM - 1) return;  // tile strictly above the diagonal
  TA c[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) c[x][y] = TA(0);
  const bool p_kfast = (p1 == 1);
  const bool q_jfast = (q1 == 1);
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int e = tid + 256 * s;
      int ii, kk;
      if (p_kfast) { kk = e & 15; ii = e >> 4; } else { ii = e & 63; kk = e >> 6; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      sP[kk][ii] = (gi < M && gk < K) ? (TA)P[gi * p0 + gk * p1] : TA(0);
      int jj;
      if (q_jfast) { jj = e & 63; kk = e >> 6; } else { kk = e & 15; jj = e >> 4; }
      const int64_t gj = j0 + jj, gk2 = k0 + kk;
      sQ[kk][jj] = (gj < N && gk2 < K) ? (TA)Q[gk2 * q0 + gj * q1] : TA(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = sP[kk][ty * 4 + x];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = sQ[kk][tx * 4 + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) c[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t gi = i0 + ty * 4 + x;
    if (gi >= M) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t gj = j0 + tx * 4 + y;
      if (gj >= N) continue;
      double v = (double)c[x][y];
      if (gi == gj) v += diag;
      C[gi * ldc + gj] = (TO)v;
    }
  }
}

// Mirror the lower triangle of a square matrix onto the upper one.
template <typename T>
__global__ void k_mirror_lower(T* __restrict__ C, int64_t n, int64_t ldc) {
  const int64_t i = blockIdx.y * 32 + threadIdx.y;
  const int64_t j = blockIdx.x * 32 + threadIdx.x;
  if (i < n && j < n && j > i) C[i * ldc + j] = C[j * ldc + i];
}

template <typename TI, typename TA, typename TO>
inline cudaError_t gemm_strided(cudaStream_t st, int64_t M, int64_t N, int64_t K, const TI* P,
                                int64_t p0, int64_t p1, const TI* Q, int64_t q0, int64_t q1, TO* C,
                                int64_t ldc, double diag, int lower_only = 0,
                                const Ctrl* ctrl = nullptr, int nbatch = 1, int64_t bP = 0,
                                int64_t bQ = 0, int64_t bC = 0) {
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)nbatch);
  k_gemm_strided<TI, TA, TO><<<grid, 256, 0, st>>>(M, N, K, P, p0, p1, Q, q0, q1, C, ldc, diag,
                                                  lower_only, ctrl, bP, bQ, bC);
  return cudaGetLastError();
}

}  // namespace rs
