// The small SPD system of eq. (14): delta = (S^T A S)^dagger r_S.
//
// Phase 1 (k_factor_inv, batched over the slots of a chunk, one CTA per slot):
// Cholesky factorisation M = L L^T, right-looking, with the pivot rule of the
// least-norm case: a pivot at most tau * eps * max_i M_ii drops its index j (row
// and column j of L become e_j). The triangular factor is then inverted in place
// (right-looking triangular solve against the identity) and the dropped rows and
// columns of L^{-1} are zeroed, so that
//     delta = L^{-T} (L^{-1} r_S)
// is the solution of the reduced system with delta_j = 0 at dropped indices.
// When A is positive definite null(S^T A S) = null(S): every solution gives the
// same S delta and A S delta as the pseudo-inverse.
//
// Phase 2 (k_delta, once per iteration, a thread-block cluster): r_S = S^T r,
// y = L^{-1} r_S, delta = L^{-T} y and u = S delta. The tau^3 work of every
// iteration sits in phase 1, off the sequential chain of iterations.
#include <cooperative_groups.h>

#include "rs_kernels.cuh"

namespace rs {

__host__ __device__ __forceinline__ int64_t pk(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

template <typename T>
size_t factor_smem_bytes(int64_t tau) {
  return (size_t)pk(tau, 0) * sizeof(T) + (size_t)tau + 64;
}
size_t factor_ws_elems(int64_t tau) { return (size_t)pk(tau, 0); }

// ---------------------------------------------------------------------------
// phase 1: factor and invert, one CTA (1024 threads) per slot
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) k_factor_inv(const Ctrl* __restrict__ ctrl, int force,
                                                     int nslots, const double* __restrict__ M,
                                                     int64_t m_slot, int64_t tau,
                                                     T* __restrict__ Linv, int64_t l_slot,
                                                     T* __restrict__ ws, int use_smem,
                                                     int32_t* __restrict__ ndropped) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t s = blockIdx.x;
  if (s >= active_slots(ctrl, force, nslots)) return;
  unsigned char* dropped = smem_raw;
  T* a = use_smem ? reinterpret_cast<T*>(smem_raw + ((tau + 15) / 16) * 16) : ws + s * pk(tau, 0);
  const double* Ms = M + s * m_slot;
  T* out = Linv + s * l_slot;
  __shared__ double s_red[32];
  __shared__ T s_piv;
  __shared__ int s_drop;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;

  double dmax = 0.0;
  for (int64_t i = tid; i < tau; i += blockDim.x) {
    dropped[i] = 0;
    dmax = fmax(dmax, Ms[i * tau + i]);
  }
  for (int64_t i = wid; i < tau; i += nw)
    for (int64_t j = lane; j <= i; j += 32) a[pk(i, j)] = (T)Ms[i * tau + j];
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

  // Cholesky, column by column
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
    const int dr = s_drop;
    const T inv = dr ? T(0) : T(1) / s_piv;
    for (int64_t i = k + 1 + tid; i < tau; i += blockDim.x) a[pk(i, k)] *= inv;
    if (dr)
      for (int64_t j = tid; j < k; j += blockDim.x) a[pk(k, j)] = T(0);
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
  // in-place inverse: solve L X = I right-looking; row k of X replaces row k of L
  // once every update from rows above has been applied
  for (int64_t k = 0; k < tau; ++k) {
    const T inv = T(1) / a[pk(k, k)];
    for (int64_t c = tid; c < k; c += blockDim.x) a[pk(k, c)] *= inv;
    __syncthreads();
    if (tid == 0) a[pk(k, k)] = inv;
    __syncthreads();
    const T* xk = a + pk(k, 0);
    for (int64_t i = k + 1 + wid; i < tau; i += nw) {
      T* rowi = a + pk(i, 0);
      const T lik = rowi[k];
      __syncwarp();
      if (lik != T(0)) {
        for (int64_t c = lane; c <= k; c += 32) {
          if (c == k) rowi[k] = -lik * xk[k];
          else rowi[c] -= lik * xk[c];
        }
      }
    }
    __syncthreads();
  }
  // zero dropped rows and columns, write L^{-1} (tau x tau, zero above the diagonal)
  for (int64_t i = wid; i < tau; i += nw) {
    const bool di = dropped[i];
    for (int64_t j = lane; j < tau; j += 32) {
      T v = T(0);
      if (j <= i && !di && !dropped[j]) v = a[pk(i, j)];
      out[i * tau + j] = v;
    }
  }
  if (tid == 0 && ndropped != nullptr && drops > 0) atomicAdd(ndropped, drops);
}

template <typename T>
cudaError_t launch_factor_inv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              const double* M, int64_t m_slot, int64_t tau, T* Linv, int64_t l_slot,
                              T* ws, int32_t* ndropped) {
  const size_t need = factor_smem_bytes<T>(tau);
  const int use_smem = need <= 200 * 1024;
  const size_t smem = use_smem ? need : (size_t)tau + 64;
  cudaError_t e = cudaFuncSetAttribute(k_factor_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_factor_inv<T><<<nslots, 1024, smem, st>>>(ctrl, force, nslots, M, m_slot, tau, Linv, l_slot, ws,
                                              use_smem, ndropped);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// phase 2: r_S, delta = L^{-T} L^{-1} r_S, u = S delta on a cluster of CS CTAs.
// CTA q owns the index range [q*chunk, (q+1)*chunk) of r_S, y and delta.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_delta(const Ctrl* __restrict__ ctrl, int force,
                                               int64_t k_arg, DeltaArgs<T> g) {
  namespace cg = cooperative_groups;
  using TA = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  // ctrl is read once; no writer runs during this kernel: every CTA exits together
  if (!force && halted(ctrl)) return;
  const int64_t tau = g.tau, m = g.m;
  const int64_t k = force ? k_arg : ctrl->k;
  const int64_t slot = force ? 0 : (ctrl->k - ctrl->k0);
  const int64_t chunk = (tau + CS - 1) / CS;
  const int64_t lo = rank * chunk, hi = lo + chunk < tau ? lo + chunk : tau;
  TA* rsv = reinterpret_cast<TA*>(smem_raw);
  TA* yv = rsv + tau;
  TA* dl = yv + tau;
  TA* red = dl + tau;  // 256 partials
  double* fb = reinterpret_cast<double*>(smem_raw + (((3 * tau + 256) * sizeof(TA) + 15) / 16) * 16);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const T* Li = g.Linv + slot * g.l_slot;
  const int32_t* perm = g.plan.perm ? g.plan.perm + slot * g.plan.perm_stride : nullptr;
  const int32_t* boff = g.plan.boff ? g.plan.boff + slot * g.plan.boff_stride : nullptr;
  const double scale = g.kind == 2 ? 1.0 / sqrt((double)tau * (double)g.mp) : 1.0;
  const uint64_t key = iter_key(g.seed, k);

  // 1. r_S for the own range (SRHT: CTA 0 computes all of it)
  if (g.kind == 0) {
    for (int64_t l = lo + wid; l < hi; l += 8) {
      double acc = 0.0;
      const int32_t t1 = boff[l + 1];
      for (int32_t t = boff[l] + lane; t < t1; t += 32) {
        const int32_t e = perm[t];
        const double v = g.r[entry_row(e)];
        acc += entry_neg(e) ? -v : v;
      }
      acc = warp_sum(acc);
      if (lane == 0) rsv[l] = (TA)acc;
    }
  } else if (g.kind == 1) {
    const T* STs = g.ST + slot * g.st_slot;
    for (int64_t l = lo + wid; l < hi; l += 8) {
      double acc = 0.0;
      for (int64_t i = lane; i < m; i += 32) acc += (double)STs[l * g.ld + i] * g.r[i];
      acc = warp_sum(acc);
      if (lane == 0) rsv[l] = (TA)acc;
    }
  } else if (rank == 0) {
    for (int64_t i = tid; i < g.mp; i += blockDim.x)
      fb[i] = i < m ? (draw_neg(draw_k(key, 1, (uint64_t)i)) ? -g.r[i] : g.r[i]) : 0.0;
    fwht_smem(fb, g.mp);
    for (int64_t l = tid; l < tau; l += blockDim.x) rsv[l] = (TA)(scale * fb[entry_row(perm[l])]);
  }
  cluster.sync();
  for (int64_t l = tid; l < tau; l += blockDim.x) {
    const int own = g.kind == 2 ? 0 : (int)(l / chunk);
    if (own != rank) rsv[l] = cluster.map_shared_rank(rsv, own)[l];
  }
  __syncthreads();
  if (rank == 0 && g.rS_out != nullptr)
    for (int64_t l = tid; l < tau; l += blockDim.x) g.rS_out[l] = (double)rsv[l];
  // 2. y = L^{-1} r_S on the own rows (one warp per row)
  for (int64_t i = lo + wid; i < hi; i += 8) {
    TA acc = TA(0);
    const T* row = Li + i * tau;
    for (int64_t j = lane; j <= i; j += 32) acc += (TA)row[j] * rsv[j];
    acc = warp_sum(acc);
    if (lane == 0) yv[i] = acc;
  }
  cluster.sync();
  for (int64_t i = tid; i < tau; i += blockDim.x) {
    const int own = (int)(i / chunk);
    if (own != rank) yv[i] = cluster.map_shared_rank(yv, own)[i];
  }
  __syncthreads();
  // 3. delta = L^{-T} y on the own columns: thread = (column, part of the rows)
  const int64_t ncol = hi - lo;
  if (ncol > 0) {
    int64_t parts = 256 / ncol;
    if (parts < 1) parts = 1;
    for (int64_t c0 = 0; c0 < ncol; c0 += 256) {
      const int64_t cl = c0 + tid % (ncol < 256 ? ncol : 256);
      const int64_t part = tid / (ncol < 256 ? ncol : 256);
      TA acc = TA(0);
      if (cl < ncol && part < parts) {
        const int64_t j = lo + cl;
        for (int64_t i = j + part; i < tau; i += parts) acc += (TA)Li[i * tau + j] * yv[i];
      }
      red[tid] = acc;
      __syncthreads();
      const int64_t nc = (ncol - c0) < 256 ? (ncol - c0) : 256;
      for (int64_t q = tid; q < nc; q += blockDim.x) {
        TA s = TA(0);
        const int64_t width = ncol < 256 ? ncol : 256;
        for (int64_t p = 0; p < parts; ++p) s += red[p * width + q];
        dl[lo + c0 + q] = s;
        g.delta_out[lo + c0 + q] = (double)s;
      }
      __syncthreads();
    }
  }
  // 4. u = S delta
  if (g.kind == 0) {
    for (int64_t l = lo + wid; l < hi; l += 8) {
      const double d = (double)dl[l];
      const int32_t t1 = boff[l + 1];
      for (int32_t t = boff[l] + lane; t < t1; t += 32) {
        const int32_t e = perm[t];
        g.u[entry_row(e)] = entry_neg(e) ? -d : d;
      }
    }
  } else if (g.kind == 2) {
    cluster.sync();
    if (rank == 0) {
      for (int64_t l = tid; l < tau; l += blockDim.x) {
        const int own = (int)(l / chunk);
        if (own != 0) dl[l] = cluster.map_shared_rank(dl, own)[l];
      }
      for (int64_t i = tid; i < g.mp; i += blockDim.x) fb[i] = 0.0;
      __syncthreads();
      for (int64_t l = tid; l < tau; l += blockDim.x) fb[entry_row(perm[l])] = (double)dl[l];
      fwht_smem(fb, g.mp);
      for (int64_t i = tid; i < m; i += blockDim.x)
        g.u[i] = scale * (draw_neg(draw_k(key, 1, (uint64_t)i)) ? -fb[i] : fb[i]);
    }
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

template <typename T>
int delta_cluster_size(int64_t tau) {
  const int64_t per = sizeof(T) == 8 ? 16 : 64;  // indices per CTA
  int cs = 1;
  const int csmax = sizeof(T) == 8 ? 16 : 8;
  while (cs < csmax && (int64_t)cs * per < tau) cs <<= 1;
  return cs;
}

template <typename T>
cudaError_t launch_delta(cudaStream_t st, const Ctrl* ctrl, int force, int64_t k_arg,
                         DeltaArgs<T> g) {
  static thread_local int64_t last_tau = -1, last_mp = -1;
  static thread_local int cs = 1;
  size_t smem = (((3 * g.tau + 256) * sizeof(T) + 15) / 16) * 16;
  if (g.kind == 2) smem += (size_t)g.mp * sizeof(double);
  auto kern = k_delta<T>;
  if (last_tau != g.tau || last_mp != g.mp) {
    last_tau = g.tau;
    last_mp = g.mp;
    cs = delta_cluster_size<T>(g.tau);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    while (cs > 1 && (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1)) {
      cudaGetLastError();
      cs >>= 1;
      cfg.gridDim = dim3((unsigned)cs);
      attr[0].val.clusterDim.x = (unsigned)cs;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cs);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, ctrl, force, k_arg, g);
}

#define RS_INST(T)                                                                             \
  template cudaError_t launch_factor_inv<T>(cudaStream_t, const Ctrl*, int, int, const double*, \
                                            int64_t, int64_t, T*, int64_t, T*, int32_t*);       \
  template cudaError_t launch_delta<T>(cudaStream_t, const Ctrl*, int, int64_t, DeltaArgs<T>);
RS_INST(float)
RS_INST(double)
#undef RS_INST

}  // namespace rs
