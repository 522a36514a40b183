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
#include <cooperative_groups.h>

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

// ---------------------------------------------------------------------------
// Cluster version: the factor is spread over a thread-block cluster of CS CTAs
// (distributed shared memory). Row blocks of NB rows are dealt cyclically
// (block rb lives in CTA rb % CS). Right-looking blocked Cholesky, one panel of
// NB columns at a time:
//   A  owner of the diagonal block factors it (one warp) and solves its part of
//      L y = r_S (the forward substitution rides along with the factorisation);
//   B  every CTA copies L_pp, solves its rows of the panel (L_ip = M_ip L_pp^-T)
//      and updates its part of y;
//   C  every CTA gathers the panel column and updates its trailing rows.
// Back substitution L^T delta = y panel by panel from the last: every CTA sums
// its rows' contributions, the owner of the panel reduces them and solves.
// The trailing updates, which hold nearly all tau^3/3 flops, are spread over
// the CS SMs of the cluster; this matters most in FP64, which runs at 2 FMA per
// clock per SM on this GPU.
// ---------------------------------------------------------------------------
template <typename T, int NB>
struct CholLayout {
  int64_t P, tp, slots, ldr;
  size_t off_rows, off_y, off_diag, off_pan, off_delta, off_part, off_z, off_yp, off_drop, total;
  __host__ __device__ CholLayout(int64_t tau, int cs) {
    P = (tau + NB - 1) / NB;
    tp = P * NB;
    slots = (P + cs - 1) / cs;
    ldr = tp;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 15) / 16 * 16; return r; };
    off_rows = take((size_t)slots * NB * ldr * sizeof(T));
    off_y = take((size_t)slots * NB * sizeof(T));
    off_diag = take((size_t)NB * (NB + 1) * sizeof(T));
    off_pan = take((size_t)tp * (NB + 1) * sizeof(T));
    off_delta = take((size_t)tp * sizeof(T));
    off_part = take((size_t)NB * sizeof(T));
    off_z = take((size_t)NB * sizeof(T));
    off_yp = take((size_t)NB * sizeof(T));
    off_drop = take((size_t)tp);
    total = o;
  }
};

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_chol_cluster(const Ctrl* __restrict__ ctrl, int force,
                                                      const double* __restrict__ M,
                                                      const double* __restrict__ rS, int64_t tau,
                                                      double* __restrict__ delta_out, PlanView plan,
                                                      double* __restrict__ u,
                                                      int32_t* __restrict__ ndropped) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  // every CTA of the cluster takes the same early exit: ctrl is read once here
  // and nobody writes it while this kernel runs
  if (!force && halted(ctrl)) return;
  const CholLayout<T, NB> L(tau, CS);
  T* rows = reinterpret_cast<T*>(smem_raw + L.off_rows);
  T* yv = reinterpret_cast<T*>(smem_raw + L.off_y);
  T* diag = reinterpret_cast<T*>(smem_raw + L.off_diag);
  T* pan = reinterpret_cast<T*>(smem_raw + L.off_pan);
  T* dl = reinterpret_cast<T*>(smem_raw + L.off_delta);
  T* part = reinterpret_cast<T*>(smem_raw + L.off_part);
  T* zb = reinterpret_cast<T*>(smem_raw + L.off_z);
  T* yp = reinterpret_cast<T*>(smem_raw + L.off_yp);
  unsigned char* dropped = smem_raw + L.off_drop;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t P = L.P, tp = L.tp, ldr = L.ldr;
  const int nown = (int)((P - rank + CS - 1) / CS);  // row blocks owned by this CTA
  __shared__ double s_red[8];

  // pivot threshold tau * eps * max_i M_ii (every CTA reads the whole diagonal)
  double dmax = 0.0;
  for (int64_t i = tid; i < tau; i += blockDim.x) dmax = fmax(dmax, M[i * tau + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) s_red[wid] = dmax;
  __syncthreads();
  if (tid == 0) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v = fmax(v, s_red[q]);
    s_red[0] = v;
  }
  __syncthreads();
  const T thr = (T)((double)tau * Eps<T>::v * s_red[0]);

  // load own row blocks (lower part up to the block's last column), padded with I
  for (int ls = 0; ls < nown; ++ls) {
    const int64_t rb = rank + (int64_t)ls * CS;
    const int64_t cend = (rb + 1) * NB;
    for (int64_t e = tid; e < (int64_t)NB * cend; e += blockDim.x) {
      const int64_t i = e / cend, c = e - i * cend;
      const int64_t R = rb * NB + i;
      double v = (R < tau && c < tau) ? M[R * tau + c] : (R == c ? 1.0 : 0.0);
      rows[(ls * NB + i) * ldr + c] = (T)v;
    }
    for (int i = tid; i < NB; i += blockDim.x) {
      const int64_t R = rb * NB + i;
      yv[ls * NB + i] = R < tau ? (T)rS[R] : T(0);
    }
  }
  for (int64_t i = tid; i < tp; i += blockDim.x) { dropped[i] = 0; dl[i] = T(0); }
  cluster.sync();

  for (int64_t p = 0; p < P; ++p) {
    const int owner = (int)(p % CS);
    const int64_t c0 = p * NB;
    if (rank == owner && wid == 0) {  // A: factor the diagonal block, forward-solve y_p
      T* blk = rows + ((p / CS) * NB) * ldr + c0;  // blk[i * ldr + j] = row c0+i, col c0+j
      T* yb = yv + (p / CS) * NB;
      for (int kk = 0; kk < NB; ++kk) {
        const T d = blk[kk * ldr + kk];
        const bool dr = !(d > thr);
        const T piv = dr ? T(1) : (T)sqrt((double)d);
        __syncwarp();
        if (lane == 0) { blk[kk * ldr + kk] = piv; dropped[c0 + kk] = dr; }
        for (int i = kk + 1 + lane; i < NB; i += 32) blk[i * ldr + kk] = dr ? T(0) : blk[i * ldr + kk] / piv;
        __syncwarp();
        for (int i = kk + 1 + lane; i < NB; i += 32) {
          const T lik = blk[i * ldr + kk];
          for (int j = kk + 1; j <= i; ++j) blk[i * ldr + j] -= lik * blk[j * ldr + kk];
        }
        __syncwarp();
      }
      for (int kk = 0; kk < NB; ++kk) {
        if (lane == 0) yb[kk] = dropped[c0 + kk] ? T(0) : yb[kk] / blk[kk * ldr + kk];
        __syncwarp();
        for (int i = kk + 1 + lane; i < NB; i += 32) yb[i] -= blk[i * ldr + kk] * yb[kk];
        __syncwarp();
      }
    }
    cluster.sync();  // #1: L_pp, y_p final in the owner
    {
      const T* oblk = cluster.map_shared_rank(rows, owner) + ((p / CS) * NB) * ldr + c0;
      const T* oy = cluster.map_shared_rank(yv, owner) + (p / CS) * NB;
      const unsigned char* odr = cluster.map_shared_rank(dropped, owner);
      for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e - i * NB;
        diag[i * (NB + 1) + j] = (j <= i) ? oblk[i * ldr + j] : T(0);
      }
      for (int i = tid; i < NB; i += blockDim.x) {
        yp[i] = oy[i];
        dropped[c0 + i] = odr[c0 + i];
      }
    }
    __syncthreads();
    // B: panel rows of own blocks below p, and the y update
    for (int r = tid; r < nown * NB; r += blockDim.x) {
      const int ls = r / NB, i = r - ls * NB;
      const int64_t rb = rank + (int64_t)ls * CS;
      if (rb <= p) continue;
      T* row = rows + (ls * NB + i) * ldr + c0;
      T x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        T s = row[j];
#pragma unroll
        for (int l = 0; l < j; ++l) s -= x[l] * diag[j * (NB + 1) + l];
        x[j] = dropped[c0 + j] ? T(0) : s / diag[j * (NB + 1) + j];
      }
      T acc = yv[ls * NB + i];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        row[j] = x[j];
        acc -= x[j] * yp[j];
      }
      yv[ls * NB + i] = acc;
    }
    cluster.sync();  // #2: the whole panel column is final
    if (p + 1 < P) {
      // C: gather the panel column of rows below the panel, then the trailing update
      const int64_t q0 = p + 1;
      const int64_t nq = P - q0;
      for (int64_t e = tid; e < nq * NB * NB; e += blockDim.x) {
        const int64_t qi = e / (NB * NB), rem = e - qi * NB * NB;
        const int i = (int)(rem / NB), l = (int)(rem - (rem / NB) * NB);
        const int64_t q = q0 + qi;
        const T* src = cluster.map_shared_rank(rows, (int)(q % CS));
        pan[(qi * NB + i) * (NB + 1) + l] = src[((q / CS) * NB + i) * ldr + c0 + l];
      }
      __syncthreads();
      const int64_t cs0 = q0 * NB;  // first trailing column
      for (int ls = 0; ls < nown; ++ls) {
        const int64_t rb = rank + (int64_t)ls * CS;
        if (rb <= p) continue;
        for (int i = 0; i < NB; ++i) {
          const int64_t R = rb * NB + i;
          T* row = rows + (ls * NB + i) * ldr;
          T lr[NB];
#pragma unroll
          for (int l = 0; l < NB; ++l) lr[l] = row[c0 + l];
          for (int64_t c = cs0 + tid; c <= R; c += blockDim.x) {
            const T* pc = pan + (c - cs0) * (NB + 1);
            T s = row[c];
#pragma unroll
            for (int l = 0; l < NB; ++l) s -= lr[l] * pc[l];
            row[c] = s;
          }
        }
      }
      __syncthreads();
    }
  }

  // back substitution L^T delta = y
  for (int64_t p = P - 1; p >= 0; --p) {
    const int owner = (int)(p % CS);
    const int64_t c0 = p * NB;
    for (int l = tid; l < NB; l += blockDim.x) {
      T s = T(0);
      for (int ls = 0; ls < nown; ++ls) {
        const int64_t rb = rank + (int64_t)ls * CS;
        if (rb <= p) continue;
        for (int i = 0; i < NB; ++i) s += rows[(ls * NB + i) * ldr + c0 + l] * dl[rb * NB + i];
      }
      part[l] = s;
    }
    cluster.sync();  // #3: partial sums ready
    if (rank == owner && wid == 0) {
      const T* blk = rows + ((p / CS) * NB) * ldr + c0;
      const T* yb = yv + (p / CS) * NB;
      for (int l = lane; l < NB; l += 32) {
        T s = yb[l];
        for (int q = 0; q < CS; ++q) s -= cluster.map_shared_rank(part, q)[l];
        zb[l] = s;
      }
      __syncwarp();
      for (int kk = NB - 1; kk >= 0; --kk) {
        if (lane == 0) {
          const T v = dropped[c0 + kk] ? T(0) : zb[kk] / blk[kk * ldr + kk];
          dl[c0 + kk] = v;
          zb[kk] = v;
        }
        __syncwarp();
        const T dk = zb[kk];
        for (int j = lane; j < kk; j += 32) zb[j] -= blk[kk * ldr + j] * dk;
        __syncwarp();
      }
    }
    cluster.sync();  // #4: delta_p final in the owner
    if (rank != owner) {
      const T* od = cluster.map_shared_rank(dl, owner);
      for (int i = tid; i < NB; i += blockDim.x) dl[c0 + i] = od[c0 + i];
    }
    __syncthreads();
  }

  if (rank == 0)
    for (int64_t i = tid; i < tau; i += blockDim.x) delta_out[i] = (double)dl[i];
  if (tid == 0 && ndropped != nullptr) {
    int cnt = 0;
    for (int ls = 0; ls < nown; ++ls)
      for (int i = 0; i < NB; ++i) {
        const int64_t R = (rank + (int64_t)ls * CS) * NB + i;
        if (R < tau && dropped[R]) ++cnt;
      }
    if (cnt) atomicAdd(ndropped, cnt);
  }
  if (plan.perm != nullptr) {  // u = S delta for the bucket-row sketches
    const int64_t slot = force ? 0 : (ctrl->k - ctrl->k0);
    const int32_t* perm = plan.perm + slot * plan.perm_stride;
    const int32_t* boff = plan.boff + slot * plan.boff_stride;
    for (int64_t l = rank * (int64_t)(blockDim.x >> 5) + wid; l < tau;
         l += (int64_t)CS * (blockDim.x >> 5)) {
      const double d = (double)dl[l];
      const int32_t t1 = boff[l + 1];
      for (int32_t t = boff[l] + lane; t < t1; t += 32) {
        const int32_t e = perm[t];
        u[entry_row(e)] = entry_neg(e) ? -d : d;
      }
    }
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// cluster size and shared memory of the cluster kernel for tau; cs = 0 if it
// cannot be used (the single-CTA kernel then runs)
template <typename T, int NB>
int chol_cluster_cs(int64_t tau, size_t* smem_out) {
  const int64_t P = (tau + NB - 1) / NB;
  const int csmax = (sizeof(T) == 8) ? 16 : 8;
  for (int cs = 1; cs <= csmax; cs <<= 1) {
    const int want = (int)std::min<int64_t>(P, csmax);
    if (cs < want && cs < csmax) continue;
    const CholLayout<T, NB> L(tau, cs);
    if (L.total <= 220 * 1024) {
      *smem_out = L.total;
      return cs;
    }
  }
  return 0;
}

template <typename T, int NB>
cudaError_t launch_chol_cluster(cudaStream_t st, int cs, size_t smem, const Ctrl* ctrl, int force,
                                const double* M, const double* rS, int64_t tau, double* delta,
                                PlanView plan, double* u, int32_t* ndropped) {
  auto kern = k_chol_cluster<T, NB>;
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
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, ctrl, force, M, rS, tau, delta, plan, u, ndropped);
}

// cluster kernel usable for (T, tau)? records the choice per instantiation
template <typename T>
struct ClusterChoice {
  int64_t tau = -1;
  int cs = 0;
  size_t smem = 0;
};

template <typename T>
cudaError_t launch_chol_solve(cudaStream_t st, const Ctrl* ctrl, int force, const double* M,
                              const double* rS, int64_t tau, T* gscratch, double* delta,
                              PlanView plan, double* u, int32_t* ndropped) {
  static thread_local ClusterChoice<T> ch;
  constexpr int NB = sizeof(T) == 8 ? 16 : 32;
  if (ch.tau != tau) {
    ch.tau = tau;
    ch.cs = chol_cluster_cs<T, NB>(tau, &ch.smem);
    if (ch.cs > 0) {  // can a cluster of this size be scheduled?
      auto kern = k_chol_cluster<T, NB>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ch.smem);
      if (ch.cs > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)ch.cs);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = ch.smem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)ch.cs;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        ch.cs = 0;
      }
    }
  }
  if (ch.cs > 0)
    return launch_chol_cluster<T, NB>(st, ch.cs, ch.smem, ctrl, force, M, rS, tau, delta, plan, u,
                                      ndropped);
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
