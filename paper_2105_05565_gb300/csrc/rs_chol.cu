// Small SPD solve of eq. (14): delta = (S^T A S)^dagger r_S.
//
// Cholesky factorisation M = L L^T (right-looking, column by column) with a pivot
// rule for the least-norm case: when the pivot of column j is at most
// tau * eps * max_i M_ii, index j is dropped (column j of L set to e_j, delta_j = 0)
// and the remaining indices solve the reduced system. When A is positive definite
// null(S^T A S) = null(S), so every solution gives the same S delta and A S delta:
// the iterates equal those of the pseudo-inverse.
//
// The factor is held packed (lower triangle, row-major) in shared memory when it
// fits, otherwise in a global scratch buffer. One CTA of 1024 threads.
#include "rs_kernels.cuh"

namespace rs {

__host__ __device__ __forceinline__ int64_t pk(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

constexpr size_t kCholSmemLimit = 200 * 1024;

template <typename T>
size_t chol_smem_bytes(int64_t tau) {
  return (size_t)pk(tau, 0) * sizeof(T) + (size_t)tau * sizeof(double) + (size_t)tau + 64;
}

template <typename T>
size_t chol_scratch_elems(int64_t tau) { return (size_t)pk(tau, 0); }

template <typename T>
__global__ void __launch_bounds__(1024) k_chol_solve(const Ctrl* __restrict__ ctrl, int force,
                                                     const double* __restrict__ M,
                                                     const double* __restrict__ rS, int64_t tau,
                                                     T* __restrict__ gscratch, int use_smem,
                                                     double* __restrict__ delta, PlanView plan,
                                                     double* __restrict__ u,
                                                     int32_t* __restrict__ ndropped) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!force && halted(ctrl)) return;
  double* y = reinterpret_cast<double*>(smem_raw);
  unsigned char* dropped = smem_raw + tau * sizeof(double);
  T* a = use_smem ? reinterpret_cast<T*>(smem_raw + ((tau * sizeof(double) + tau + 15) / 16) * 16)
                  : gscratch;
  __shared__ double s_red[32];
  __shared__ T s_piv;
  __shared__ int s_drop;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;

  double dmax = 0.0;
  for (int64_t i = tid; i < tau; i += blockDim.x) {
    y[i] = rS[i];
    dropped[i] = 0;
    dmax = fmax(dmax, M[i * tau + i]);
  }
  for (int64_t i = wid; i < tau; i += nw)
    for (int64_t j = lane; j <= i; j += 32) a[pk(i, j)] = (T)M[i * tau + j];
  // block max of the diagonal
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) s_red[wid] = dmax;
  __syncthreads();
  if (wid == 0) {
    double v = lane < nw ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const T thr = (T)((double)tau * Eps<T>::v * s_red[0]);
  int drops = 0;

  for (int64_t k = 0; k < tau; ++k) {
    if (tid == 0) {
      const T d = a[pk(k, k)];
      const int dr = !(d > thr);
      s_drop = dr;
      s_piv = dr ? T(1) : (T)sqrt((double)d);
      a[pk(k, k)] = s_piv;
      dropped[k] = (unsigned char)dr;
      drops += dr;
    }
    __syncthreads();
    const T inv = s_drop ? T(0) : T(1) / s_piv;
    for (int64_t i = k + 1 + tid; i < tau; i += blockDim.x) a[pk(i, k)] *= inv;
    __syncthreads();
    for (int64_t i = k + 1 + wid; i < tau; i += nw) {
      const T lik = a[pk(i, k)];
      if (lik != T(0)) {
        T* rowi = a + pk(i, 0);
        for (int64_t j = k + 1 + lane; j <= i; j += 32) rowi[j] -= lik * a[pk(j, k)];
      }
    }
    __syncthreads();
  }
  // forward substitution L y = r_S (dropped: y_k = 0)
  for (int64_t k = 0; k < tau; ++k) {
    if (tid == 0) y[k] = dropped[k] ? 0.0 : y[k] / (double)a[pk(k, k)];
    __syncthreads();
    const double yk = y[k];
    for (int64_t i = k + 1 + tid; i < tau; i += blockDim.x) y[i] -= (double)a[pk(i, k)] * yk;
    __syncthreads();
  }
  // back substitution L^T delta = y
  for (int64_t k = tau - 1; k >= 0; --k) {
    if (tid == 0) y[k] = dropped[k] ? 0.0 : y[k] / (double)a[pk(k, k)];
    __syncthreads();
    const double dk = y[k];
    const T* rowk = a + pk(k, 0);
    for (int64_t j = tid; j < k; j += blockDim.x) y[j] -= (double)rowk[j] * dk;
    __syncthreads();
  }
  for (int64_t i = tid; i < tau; i += blockDim.x) delta[i] = y[i];
  if (tid == 0 && ndropped != nullptr && drops > 0) atomicAdd(ndropped, drops);
  // u = S delta for the bucket-row sketches: u[row] = sign * delta_bucket
  if (plan.perm != nullptr) {
    const int64_t slot = force ? 0 : (ctrl->k - ctrl->k0);
    const int32_t* perm = plan.perm + slot * plan.perm_stride;
    const int32_t* boff = plan.boff + slot * plan.boff_stride;
    for (int64_t l = wid; l < tau; l += nw) {
      const double dl = y[l];
      const int32_t t1 = boff[l + 1];
      for (int32_t t = boff[l] + lane; t < t1; t += 32) {
        const int32_t e = perm[t];
        u[entry_row(e)] = entry_neg(e) ? -dl : dl;
      }
    }
  }
}

template <typename T>
cudaError_t launch_chol_solve(cudaStream_t st, const Ctrl* ctrl, int force, const double* M,
                              const double* rS, int64_t tau, T* gscratch, double* delta,
                              PlanView plan, double* u, int32_t* ndropped) {
  const size_t need = chol_smem_bytes<T>(tau);
  const int use_smem = need <= kCholSmemLimit;
  const size_t smem = use_smem ? need : (size_t)tau * sizeof(double) + tau + 64;
  cudaError_t e = cudaFuncSetAttribute(k_chol_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_chol_solve<T><<<1, 1024, smem, st>>>(ctrl, force, M, rS, tau, gscratch, use_smem, delta, plan,
                                         u, ndropped);
  return cudaGetLastError();
}

template size_t chol_scratch_elems<float>(int64_t);
template size_t chol_scratch_elems<double>(int64_t);
template cudaError_t launch_chol_solve<float>(cudaStream_t, const Ctrl*, int, const double*,
                                              const double*, int64_t, float*, double*, PlanView,
                                              double*, int32_t*);
template cudaError_t launch_chol_solve<double>(cudaStream_t, const Ctrl*, int, const double*,
                                               const double*, int64_t, double*, double*, PlanView,
                                               double*, int32_t*);

}  // namespace rs
