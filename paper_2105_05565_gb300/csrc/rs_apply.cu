// Applying the sketch (Section 4): the tau sketched rows S^T A (A is symmetric, so
// S^T A = (A S)^T), the sketched system M = S^T A S and the sketched residual
// r_S = S^T r of eq. (14).
#include "rs_gemm.cuh"
#include "rs_kernels.cuh"

namespace rs {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ void vadd(float4& a, const float4& b, bool neg) {
  if (neg) { a.x -= b.x; a.y -= b.y; a.z -= b.z; a.w -= b.w; }
  else { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }
}
__device__ __forceinline__ void vadd(double2& a, const double2& b, bool neg) {
  if (neg) { a.x -= b.x; a.y -= b.y; } else { a.x += b.x; a.y += b.y; }
}

__device__ __forceinline__ int64_t slot_of(const Ctrl* c, int force) {
  return force ? 0 : (c->k - c->k0);
}

// ---------------------------------------------------------------------------
// Count / SubCount (Section 4.2): SA[j, :] = sum over bucket j of sign * A[row, :].
// One warp per (bucket, column slab of 32 vectors); rows summed in bucket order
// (ascending row for Count, sample order for SubCount): deterministic.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sa_rows(const Ctrl* __restrict__ ctrl, int force,
                                                 PlanView plan, const T* __restrict__ A, int64_t lda,
                                                 int64_t m, int64_t tau, T* __restrict__ SA,
                                                 int64_t ldsa) {
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  if (!force && halted(ctrl)) return;
  const int64_t slot = slot_of(ctrl, force);
  const int32_t* perm = plan.perm + slot * plan.perm_stride;
  const int32_t* boff = plan.boff + slot * plan.boff_stride;
  const int lane = threadIdx.x & 31;
  const int64_t nslab = (m + 32 * VN - 1) / (32 * VN);
  const int64_t units = tau * nslab;
  const int64_t gw = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * 8;
  for (int64_t u = gw; u < units; u += nw) {
    const int64_t j = u / nslab;
    const int64_t c = (u - j * nslab) * 32 * VN + lane * VN;
    V acc;
    if constexpr (VN == 4) acc = make_float4(0.f, 0.f, 0.f, 0.f); else acc = make_double2(0.0, 0.0);
    const int32_t t1 = boff[j + 1];
    int32_t t = boff[j];
    for (; t + 4 <= t1; t += 4) {
      const int32_t e0 = perm[t], e1 = perm[t + 1], e2 = perm[t + 2], e3 = perm[t + 3];
      const V v0 = __ldg(reinterpret_cast<const V*>(A + (int64_t)entry_row(e0) * lda + c));
      const V v1 = __ldg(reinterpret_cast<const V*>(A + (int64_t)entry_row(e1) * lda + c));
      const V v2 = __ldg(reinterpret_cast<const V*>(A + (int64_t)entry_row(e2) * lda + c));
      const V v3 = __ldg(reinterpret_cast<const V*>(A + (int64_t)entry_row(e3) * lda + c));
      vadd(acc, v0, entry_neg(e0));
      vadd(acc, v1, entry_neg(e1));
      vadd(acc, v2, entry_neg(e2));
      vadd(acc, v3, entry_neg(e3));
    }
    for (; t < t1; ++t) {
      const int32_t e = perm[t];
      vadd(acc, __ldg(reinterpret_cast<const V*>(A + (int64_t)entry_row(e) * lda + c)), entry_neg(e));
    }
    if (c < ldsa) *reinterpret_cast<V*>(SA + j * ldsa + c) = acc;
  }
}

template <typename T>
cudaError_t launch_sa_rows(cudaStream_t st, const Ctrl* ctrl, int force, PlanView plan, const T* A,
                           int64_t lda, int64_t m, int64_t tau, T* SA, int64_t ldsa) {
  constexpr int VN = Vec<T>::n;
  const int64_t units = tau * ((m + 32 * VN - 1) / (32 * VN));
  int blocks = (int)std::min<int64_t>((units + 7) / 8, 152 * 16);
  if (blocks < 1) blocks = 1;
  k_sa_rows<T><<<blocks, 256, 0, st>>>(ctrl, force, plan, A, lda, m, tau, SA, ldsa);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bucket-row sketches: M[j, l] = sum over bucket l of sign * row_j[row],
// r_S[l] = sum over bucket l of sign * r[row]. Block j < tau builds row j of M;
// block tau builds r_S. row_j is A[C_j, :] (subsample) or SA[j, :].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_msys_rows(const Ctrl* __restrict__ ctrl, int force,
                                                   PlanView plan, RowsView<T> rows, int64_t m,
                                                   int64_t tau, const double* __restrict__ r,
                                                   double* __restrict__ M, double* __restrict__ rS) {
  if (!force && halted(ctrl)) return;
  const int64_t slot = slot_of(ctrl, force);
  const int32_t* perm = plan.perm + slot * plan.perm_stride;
  const int32_t* boff = plan.boff + slot * plan.boff_stride;
  const int64_t j = blockIdx.x;
  if (j < tau) {
    const T* rowj = rows.SA ? rows.SA + j * rows.ldsa
                            : rows.A + (int64_t)entry_row(perm[boff[j]]) * rows.lda;
    for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) {
      T acc = T(0);
      const int32_t t1 = boff[l + 1];
      for (int32_t t = boff[l]; t < t1; ++t) {
        const int32_t e = perm[t];
        const T v = rowj[entry_row(e)];
        acc += entry_neg(e) ? -v : v;
      }
      M[j * tau + l] = (double)acc;
    }
  } else {
    for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) {
      double acc = 0.0;
      const int32_t t1 = boff[l + 1];
      for (int32_t t = boff[l]; t < t1; ++t) {
        const int32_t e = perm[t];
        const double v = r[entry_row(e)];
        acc += entry_neg(e) ? -v : v;
      }
      rS[l] = acc;
    }
  }
}

template <typename T>
cudaError_t launch_msys_rows(cudaStream_t st, const Ctrl* ctrl, int force, PlanView plan,
                             RowsView<T> rows, int64_t m, int64_t tau, const double* r, double* M,
                             double* rS) {
  k_msys_rows<T><<<(unsigned)(tau + 1), 256, 0, st>>>(ctrl, force, plan, rows, m, tau, r, M, rS);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gaussian sketch (Section 4.1): dense products with the m x tau matrix S.
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_gauss_sa(cudaStream_t st, const Ctrl* ctrl, int force, const T* S, const T* A,
                            int64_t lda, int64_t m, int64_t tau, T* SA, int64_t ldsa) {
  // SA[j, c] = sum_i S[i, j] A[i, c]
  return gemm_strided<T, T, T>(st, tau, m, m, S, 1, tau, A, lda, 1, SA, ldsa, 0.0, 0,
                               force ? nullptr : ctrl);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gauss_rs(const Ctrl* __restrict__ ctrl, int force,
                                                  const T* __restrict__ S, int64_t m, int64_t tau,
                                                  const double* __restrict__ r,
                                                  double* __restrict__ rS) {
  if (!force && halted(ctrl)) return;
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (j < tau)
    for (int64_t i = w; i < m; i += 8) acc += (double)S[i * tau + j] * r[i];
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && j < tau) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[q][lane];
    rS[j] = s;
  }
}

template <typename T>
cudaError_t launch_gauss_msys(cudaStream_t st, const Ctrl* ctrl, int force, const T* S,
                              const T* SA, int64_t ldsa, int64_t m, int64_t tau, const double* r,
                              double* M, double* rS) {
  // M[j, l] = sum_c SA[j, c] S[c, l]
  cudaError_t e = gemm_strided<T, T, double>(st, tau, tau, m, SA, ldsa, 1, S, tau, 1, M, tau, 0.0,
                                             0, force ? nullptr : ctrl);
  if (e != cudaSuccess) return e;
  k_gauss_rs<T><<<(unsigned)((tau + 31) / 32), 256, 0, st>>>(ctrl, force, S, m, tau, r, rS);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_gauss_u(const Ctrl* __restrict__ ctrl, int force,
                                                 const T* __restrict__ S, int64_t m, int64_t tau,
                                                 const double* __restrict__ delta,
                                                 double* __restrict__ u) {
  if (!force && halted(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= m) return;
  double acc = 0.0;
  for (int64_t j = lane; j < tau; j += 32) acc += (double)S[i * tau + j] * delta[j];
  acc = warp_sum(acc);
  if (lane == 0) u[i] = acc;
}

template <typename T>
cudaError_t launch_gauss_u(cudaStream_t st, const Ctrl* ctrl, int force, const T* S, int64_t m,
                           int64_t tau, const double* delta, double* u) {
  k_gauss_u<T><<<(unsigned)((m + 7) / 8), 256, 0, st>>>(ctrl, force, S, m, tau, delta, u);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SRHT (Section 4.3): S = (tau m')^{-1/2} D H_{m'}[0:m, C]. Products with S are
// fast Walsh-Hadamard transforms (Sylvester order, eq. (18)) of length m' in
// shared memory.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void fwht_smem(T* buf, int64_t n) {
  for (int64_t h = 1; h < n; h <<= 1) {
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
      const int64_t i = (t / h) * 2 * h + (t % h);
      const T a = buf[i], b = buf[i + h];
      buf[i] = a + b;
      buf[i + h] = a - b;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double row_sign(uint64_t key, int64_t i) {
  return draw_neg(draw_k(key, 1, (uint64_t)i)) ? -1.0 : 1.0;
}

// SA[j, c] = scale * (H (D A[:, c]))[C_j]; A symmetric so column c is row c.
template <typename T>
__global__ void __launch_bounds__(1024) k_srht_sa(const Ctrl* __restrict__ ctrl, int force,
                                                  int64_t k_arg, uint64_t seed, PlanView plan,
                                                  const T* __restrict__ A, int64_t lda, int64_t m,
                                                  int64_t mp, int64_t tau, T* __restrict__ SA,
                                                  int64_t ldsa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  if (!force && halted(ctrl)) return;
  const int64_t k = force ? k_arg : ctrl->k;
  const uint64_t key = iter_key(seed, k);
  const int32_t* C = plan.perm + slot_of(ctrl, force) * plan.perm_stride;
  const int64_t c = blockIdx.x;
  for (int64_t i = threadIdx.x; i < mp; i += blockDim.x)
    buf[i] = i < m ? (T)(row_sign(key, i) * (double)A[c * lda + i]) : T(0);
  fwht_smem(buf, mp);
  const T scale = (T)(1.0 / sqrt((double)tau * (double)mp));
  for (int64_t j = threadIdx.x; j < tau; j += blockDim.x) SA[j * ldsa + c] = scale * buf[entry_row(C[j])];
}

template <typename T>
__global__ void __launch_bounds__(1024) k_srht_msys(const Ctrl* __restrict__ ctrl, int force,
                                                    int64_t k_arg, uint64_t seed, PlanView plan,
                                                    const T* __restrict__ SA, int64_t ldsa,
                                                    int64_t m, int64_t mp, int64_t tau,
                                                    const double* __restrict__ r,
                                                    double* __restrict__ M, double* __restrict__ rS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* buf = reinterpret_cast<double*>(smem_raw);
  if (!force && halted(ctrl)) return;
  const int64_t k = force ? k_arg : ctrl->k;
  const uint64_t key = iter_key(seed, k);
  const int32_t* C = plan.perm + slot_of(ctrl, force) * plan.perm_stride;
  const int64_t j = blockIdx.x;
  for (int64_t i = threadIdx.x; i < mp; i += blockDim.x) {
    double v = 0.0;
    if (i < m) v = row_sign(key, i) * (j < tau ? (double)SA[j * ldsa + i] : r[i]);
    buf[i] = v;
  }
  fwht_smem(buf, mp);
  const double scale = 1.0 / sqrt((double)tau * (double)mp);
  for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) {
    const double v = scale * buf[entry_row(C[l])];
    if (j < tau) M[j * tau + l] = v; else rS[l] = v;
  }
}

__global__ void __launch_bounds__(1024) k_srht_u(const Ctrl* __restrict__ ctrl, int force,
                                                 int64_t k_arg, uint64_t seed, PlanView plan,
                                                 int64_t m, int64_t mp, int64_t tau,
                                                 const double* __restrict__ delta,
                                                 double* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* buf = reinterpret_cast<double*>(smem_raw);
  if (!force && halted(ctrl)) return;
  const int64_t k = force ? k_arg : ctrl->k;
  const uint64_t key = iter_key(seed, k);
  const int32_t* C = plan.perm + slot_of(ctrl, force) * plan.perm_stride;
  for (int64_t i = threadIdx.x; i < mp; i += blockDim.x) buf[i] = 0.0;
  __syncthreads();
  for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) buf[entry_row(C[l])] = delta[l];
  fwht_smem(buf, mp);
  const double scale = 1.0 / sqrt((double)tau * (double)mp);
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) u[i] = scale * row_sign(key, i) * buf[i];
}

// largest padded length whose FP64 transform buffer fits in shared memory
int64_t srht_max_pad(int elem_bytes) { (void)elem_bytes; return 16384; }

template <typename T>
cudaError_t launch_srht_sa(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                           uint64_t seed, PlanView C, const T* A, int64_t lda, int64_t m,
                           int64_t mp, int64_t tau, T* SA, int64_t ldsa) {
  const size_t smem = (size_t)mp * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_srht_sa<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_srht_sa<T><<<(unsigned)m, 1024, smem, st>>>(ctrl, force, k_arg, seed, C, A, lda, m, mp, tau,
                                                SA, ldsa);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_srht_msys(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                             uint64_t seed, PlanView C, const T* SA, int64_t ldsa, int64_t m,
                             int64_t mp, int64_t tau, const double* r, double* M, double* rS) {
  const size_t smem = (size_t)mp * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_srht_msys<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_srht_msys<T><<<(unsigned)(tau + 1), 1024, smem, st>>>(ctrl, force, k_arg, seed, C, SA, ldsa, m,
                                                          mp, tau, r, M, rS);
  return cudaGetLastError();
}

cudaError_t launch_srht_u(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                          uint64_t seed, PlanView C, int64_t m, int64_t mp, int64_t tau,
                          const double* delta, double* u) {
  const size_t smem = (size_t)mp * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_srht_u, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_srht_u<<<1, 1024, smem, st>>>(ctrl, force, k_arg, seed, C, m, mp, tau, delta, u);
  return cudaGetLastError();
}

#define RS_INST(T)                                                                              \
  template cudaError_t launch_sa_rows<T>(cudaStream_t, const Ctrl*, int, PlanView, const T*,     \
                                         int64_t, int64_t, int64_t, T*, int64_t);               \
  template cudaError_t launch_msys_rows<T>(cudaStream_t, const Ctrl*, int, PlanView, RowsView<T>, \
                                           int64_t, int64_t, const double*, double*, double*);   \
  template cudaError_t launch_gauss_sa<T>(cudaStream_t, const Ctrl*, int, const T*, const T*,    \
                                          int64_t, int64_t, int64_t, T*, int64_t);              \
  template cudaError_t launch_gauss_msys<T>(cudaStream_t, const Ctrl*, int, const T*, const T*,  \
                                            int64_t, int64_t, int64_t, const double*, double*,  \
                                            double*);                                            \
  template cudaError_t launch_gauss_u<T>(cudaStream_t, const Ctrl*, int, const T*, int64_t,      \
                                         int64_t, const double*, double*);                       \
  template cudaError_t launch_srht_sa<T>(cudaStream_t, const Ctrl*, int, int64_t, uint64_t,      \
                                         PlanView, const T*, int64_t, int64_t, int64_t,    \
                                         int64_t, T*, int64_t);                                  \
  template cudaError_t launch_srht_msys<T>(cudaStream_t, const Ctrl*, int, int64_t, uint64_t,    \
                                           PlanView, const T*, int64_t, int64_t, int64_t,  \
                                           int64_t, const double*, double*, double*);
RS_INST(float)
RS_INST(double)
#undef RS_INST

}  // namespace rs
