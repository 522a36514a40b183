// Phase 2 of a chunk, fused: every iteration of Algorithm 2 (Section 6.3) of the
// chunk runs inside one launch of a thread-block cluster of CS CTAs.
//
// Per iteration k (slot s = k - k0 prepared by phase 1):
//   r_S     = S_s^T r                         every CTA, from the global r
//   y       = L_s^{-1} r_S                    own rows of L^{-1} (tau / CS of them)
//   part_q  = (own rows of L^{-1})^T y_own    partial of delta = L^{-T} y
//   -- cluster barrier --
//   delta   = sum_q part_q                    every CTA, through distributed shared memory
//   (A S delta)_i, (S delta)_i, w_i, r_i      own slice of i (m / CS of them), eq. (53)
//   ||r||^2 partial
//   -- cluster barrier --
//   ||r^{k+1}|| and the stopping test         every CTA, same order, same decision
// Two cluster barriers per iteration; no kernel boundary and no host involvement
// inside a chunk. Partial buffers are safe to reuse: a CTA rewrites them only after
// the next barrier, which every CTA reaches after its reads.
#include <cooperative_groups.h>

#include "rs_kernels.cuh"

namespace rs {

template <typename T> struct V2;
template <> struct V2<float> { using type = float4; static constexpr int n = 4; };
template <> struct V2<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ void vfma(double (&acc)[4], const float4& v, double d) {
  acc[0] += (double)v.x * d; acc[1] += (double)v.y * d; acc[2] += (double)v.z * d; acc[3] += (double)v.w * d;
}
__device__ __forceinline__ void vfma(float (&acc)[4], const float4& v, float d) {
  acc[0] += v.x * d; acc[1] += v.y * d; acc[2] += v.z * d; acc[3] += v.w * d;
}
__device__ __forceinline__ void vfma(double (&acc)[2], const double2& v, double d) {
  acc[0] += v.x * d; acc[1] += v.y * d;
}


__global__ void k_inv_reset(const Ctrl* __restrict__ ctrl, int force, int nslots, int64_t m,
                            int32_t* __restrict__ inv, int64_t inv_slot) {
  const int64_t s = blockIdx.y;
  if (s >= active_slots(ctrl, force, nslots)) return;
  int32_t* iv = inv + s * inv_slot;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    iv[i] = kNotSketched;
}

__global__ void k_inv_fill(const Ctrl* __restrict__ ctrl, int force, int nslots, PlanView plan,
                           int64_t tau, int32_t* __restrict__ inv, int64_t inv_slot) {
  const int64_t s = blockIdx.y;
  if (s >= active_slots(ctrl, force, nslots)) return;
  const int32_t* perm = plan.perm + s * plan.perm_stride;
  const int32_t* boff = plan.boff + s * plan.boff_stride;
  int32_t* iv = inv + s * inv_slot;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < tau;
       b += (int64_t)gridDim.x * blockDim.x)
    for (int32_t t = boff[b]; t < boff[b + 1]; ++t) {
      const int32_t e = perm[t];
      iv[entry_row(e)] = (int32_t)((uint32_t)b | ((uint32_t)e & 0x80000000u));
    }
}

cudaError_t launch_inv_map(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, PlanView plan,
                           int64_t m, int64_t tau, int all_rows, int32_t* inv, int64_t inv_slot) {
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 64));
  if (!all_rows) k_inv_reset<<<dim3(gx, nslots), 256, 0, st>>>(ctrl, force, nslots, m, inv, inv_slot);
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tau + 255) / 256, 16));
  k_inv_fill<<<dim3(gb, nslots), 256, 0, st>>>(ctrl, force, nslots, plan, tau, inv, inv_slot);
  return cudaGetLastError();
}

template <typename T, typename TF>
__global__ void __launch_bounds__(256) k_iterate(Ctrl* __restrict__ ctrl, IterArgs<T, TF> g) {
  namespace cg = cooperative_groups;
  using TV = typename V2<T>::type;
  constexpr int VN = V2<T>::n;
  using TA = T;  // accumulation type of A S delta and S delta
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  // ctrl is read once; nothing else writes it while this kernel runs, so every CTA
  // of the cluster takes the same branches
  if (halted(ctrl)) return;
  const int64_t tau = g.tau, m = g.m;
  const int64_t k0 = ctrl->k0;
  int64_t k = ctrl->k;
  const int64_t kend = min(k0 + g.sub_end, ctrl->max_iters);
  const double tol = ctrl->tol, r0 = ctrl->r0;
  const int no_stop = ctrl->no_stop;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  const int64_t rper = (tau + CS - 1) / CS;            // rows of L^{-1} per CTA
  const int64_t lo = min(tau, rank * rper), hi = min(tau, lo + rper);
  const int64_t iper = ((m + CS - 1) / CS + VN - 1) / VN * VN;  // slice of i per CTA
  const int64_t ilo = min(m, rank * iper), ihi = min(m, ilo + iper);

  TF* rsf = reinterpret_cast<TF*>(smem_raw);            // tau
  TF* yv = rsf + tau;                                   // rper
  TF* part = yv + rper;                                 // tau
  double* dfull = reinterpret_cast<double*>(smem_raw + (((2 * tau + rper) * sizeof(TF) + 15) / 16) * 16);
  double* nrm = dfull + tau;                            // 1 (+ pad)
  TA* red = reinterpret_cast<TA*>(nrm + 2);             // 2 * 256 * VN
  double* stg_r = reinterpret_cast<double*>(red + 2 * 256 * VN);   // m (g.stage)
  int32_t* stg_p = reinterpret_cast<int32_t*>(stg_r + (g.stage ? m : 0));  // plan
  __shared__ double s_w[8];

  int outcome = 0;  // 0 chunk done, 1 converged, 2 numeric failure
  while (k < kend) {
    const int64_t slot = k - k0;
    const int32_t* perm = g.plan.perm ? g.plan.perm + slot * g.plan.perm_stride : nullptr;
    const int32_t* boff = g.plan.boff ? g.plan.boff + slot * g.plan.boff_stride : nullptr;
    const TF* Li = g.Linv + slot * g.l_slot;
    const T* ST = g.ST ? g.ST + slot * g.sa_slot : nullptr;
    // r_S = S^T r (every CTA, all tau entries). r and the slot's plan are first
    // copied to shared memory with coalesced loads; the gathers then hit shared memory.
    if (g.kind == 0) {
      if (g.stage) {
        double* sr = stg_r;
        int32_t* sp = stg_p;
        int32_t* sb = stg_p + g.plan.perm_stride;
#pragma unroll 8
        for (int64_t i = tid; i < m; i += blockDim.x) sr[i] = g.r[i];
#pragma unroll 8
        for (int64_t t = tid; t < g.plan.perm_stride; t += blockDim.x) sp[t] = perm[t];
        for (int64_t t = tid; t <= tau; t += blockDim.x) sb[t] = boff[t];
        __syncthreads();
        for (int64_t l = tid; l < tau; l += blockDim.x) {
          double acc = 0.0;
          const int32_t t1 = sb[l + 1];
          for (int32_t t = sb[l]; t < t1; ++t) {
            const int32_t e = sp[t];
            const double v = sr[entry_row(e)];
            acc = sadd(acc, v, entry_neg(e));
          }
          rsf[l] = (TF)acc;
        }
      } else {
        for (int64_t l = tid; l < tau; l += blockDim.x) {
          double acc = 0.0;
          const int32_t t1 = boff[l + 1];
          for (int32_t t = boff[l]; t < t1; ++t) {
            const int32_t e = perm[t];
            const double v = g.r[entry_row(e)];
            acc = sadd(acc, v, entry_neg(e));
          }
          rsf[l] = (TF)acc;
        }
      }
    } else {
      for (int64_t l = wid; l < tau; l += 8) {
        double acc = 0.0;
#pragma unroll 8
        for (int64_t i = lane; i < m; i += 32) acc += (double)ST[l * g.lda + i] * g.r[i];
        acc = warp_sum(acc);
        if (lane == 0) rsf[l] = (TF)acc;
      }
    }
    __syncthreads();
    // y = L^{-1} r_S on the own rows (one warp per row)
    for (int64_t i = lo + wid; i < hi; i += 8) {
      TF acc = TF(0);
      const TF* row = Li + i * tau;
#pragma unroll 8
      for (int64_t j = lane; j <= i; j += 32) acc += __ldg(row + j) * rsf[j];
      acc = warp_sum(acc);
      if (lane == 0) yv[i - lo] = acc;
    }
    __syncthreads();
    // partial of delta = L^{-T} y from the own rows
    for (int64_t j = tid; j < tau; j += blockDim.x) {
      TF acc = TF(0);
#pragma unroll 8
      for (int64_t i = (j > lo ? j : lo); i < hi; ++i) acc += __ldg(Li + i * tau + j) * yv[i - lo];
      part[j] = acc;
    }
    cluster.sync();
    // delta (every CTA, same summation order)
    for (int64_t j = tid; j < tau; j += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < CS; ++q) acc += (double)cluster.map_shared_rank(part, q)[j];
      dfull[j] = acc;
      if (rank == 0) {
        g.delta_out[j] = acc;
        if (g.rS_out) g.rS_out[j] = (double)rsf[j];
      }
    }
    __syncthreads();
    // own slice of i: (A S delta)_i from the sketched rows, (S delta)_i, update
    const int64_t nvec = (ihi - ilo + VN - 1) / VN;
    const int64_t vlanes = nvec < 64 ? (nvec > 0 ? nvec : 1) : 64;
    const int64_t jparts = blockDim.x / vlanes;
    double sq = 0.0;
    for (int64_t v0 = 0; v0 < nvec; v0 += vlanes) {
      const int64_t vi = v0 + tid % vlanes;
      const int64_t jp = tid / vlanes;
      TA acc[VN], uacc[VN];
#pragma unroll
      for (int q = 0; q < VN; ++q) { acc[q] = TA(0); uacc[q] = TA(0); }
      if (vi < nvec && jp < jparts) {
        const int64_t i = ilo + vi * VN;
        constexpr int UNR = 8;  // row loads in flight per thread
        for (int64_t j0 = jp; j0 < tau; j0 += UNR * jparts) {
          TV v[UNR];
#pragma unroll
          for (int q = 0; q < UNR; ++q) {
            const int64_t j = j0 + q * jparts;
            if (j < tau) {
              const T* rowj = (g.SA != nullptr) ? g.SA + slot * g.sa_slot + j * g.lda
                                                : g.A + (int64_t)entry_row(perm[j]) * g.lda;
              v[q] = __ldg(reinterpret_cast<const TV*>(rowj + i));
            }
          }
#pragma unroll
          for (int q = 0; q < UNR; ++q) {
            const int64_t j = j0 + q * jparts;
            if (j < tau) vfma(acc, v[q], (TA)dfull[j]);
          }
          if (ST) {
#pragma unroll
            for (int q = 0; q < UNR; ++q) {
              const int64_t j = j0 + q * jparts;
              if (j < tau) v[q] = __ldg(reinterpret_cast<const TV*>(ST + j * g.lda + i));
            }
#pragma unroll
            for (int q = 0; q < UNR; ++q) {
              const int64_t j = j0 + q * jparts;
              if (j < tau) vfma(uacc, v[q], (TA)dfull[j]);
            }
          }
        }
      }
      // reduce the row parts (fixed order)
#pragma unroll
      for (int q = 0; q < VN; ++q) red[(tid) * VN + q] = acc[q];
      __syncthreads();
      if (tid < vlanes && v0 + tid < nvec) {
        const int64_t i0 = ilo + (v0 + tid) * VN;
        TA s[VN];
#pragma unroll
        for (int q = 0; q < VN; ++q) s[q] = TA(0);
        for (int64_t p = 0; p < jparts; ++p)
#pragma unroll
          for (int q = 0; q < VN; ++q) s[q] += red[(p * vlanes + tid) * VN + q];
        const double gk = g.gam[k], bk = g.bet[k];
#pragma unroll
        for (int q = 0; q < VN; ++q) {
          const int64_t i = i0 + q;
          if (i >= m) continue;
          double ui;
          if (ST) {
            ui = 0.0;  // filled below from uacc parts
          } else {
            const int32_t e = g.inv[slot * g.inv_slot + i];
            ui = (e == kNotSketched) ? 0.0 : (entry_neg(e) ? -dfull[e & 0x7FFFFFFF] : dfull[e & 0x7FFFFFFF]);
          }
          red[(tid) * VN + q] = s[q];  // keep A S delta for the Gaussian pass below
          if (!ST) {
            const double wi = g.w[i], wpi = g.wp[i], ri = g.r[i], rpi = g.rp[i];
            const double wn = (1.0 + bk) * wi - bk * wpi - gk * ui;
            const double rn = (1.0 + bk) * ri - bk * rpi - gk * (double)s[q];
            g.wp[i] = wi; g.w[i] = wn;
            g.rp[i] = ri; g.r[i] = rn;
            sq += rn * rn;
          }
        }
      }
      if (ST) {  // Gaussian: S delta from the second set of partial sums
        __syncthreads();
        TA* ured = red + blockDim.x * VN;
#pragma unroll
        for (int q = 0; q < VN; ++q) ured[tid * VN + q] = uacc[q];
        __syncthreads();
        if (tid < vlanes && v0 + tid < nvec) {
          const int64_t i0 = ilo + (v0 + tid) * VN;
          const double gk = g.gam[k], bk = g.bet[k];
#pragma unroll
          for (int q = 0; q < VN; ++q) {
            const int64_t i = i0 + q;
            if (i >= m) continue;
            TA us = TA(0);
            for (int64_t p = 0; p < jparts; ++p) us += ured[(p * vlanes + tid) * VN + q];
            const double asd = (double)red[tid * VN + q];
            const double wi = g.w[i], wpi = g.wp[i], ri = g.r[i], rpi = g.rp[i];
            const double wn = (1.0 + bk) * wi - bk * wpi - gk * (double)us;
            const double rn = (1.0 + bk) * ri - bk * rpi - gk * asd;
            g.wp[i] = wi; g.w[i] = wn;
            g.rp[i] = ri; g.r[i] = rn;
            sq += rn * rn;
          }
        }
      }
      __syncthreads();
    }
    // ||r^{k+1}||^2: CTA partial, then the cluster total in every CTA
    sq = warp_sum(sq);
    if (lane == 0) s_w[wid] = sq;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_w[q];
      nrm[0] = t;
    }
    cluster.sync();
    double tot = 0.0;
    for (int q = 0; q < CS; ++q) tot += cluster.map_shared_rank(nrm, q)[0];
    const double rel = sqrt(tot) / r0;
    if (rank == 0 && tid == 0) g.hist[k + 1] = rel;
    ++k;
    if (!isfinite(rel)) { outcome = 2; break; }
    if (!no_stop && rel <= tol) { outcome = 1; break; }
  }
  if (rank == 0 && tid == 0) {
    ctrl->k = k;
    if (outcome == 2) { ctrl->status = 4; ctrl->stop = 1; }
    if (outcome == 1) { if (g.mixed) ctrl->pending = 1; else ctrl->stop = 1; }
    if (k >= ctrl->max_iters) ctrl->stop = 1;
    __threadfence();
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

template <typename T, typename TF>
size_t iterate_smem(int64_t tau, int cs, int64_t stage_bytes) {
  const int64_t rper = (tau + cs - 1) / cs;
  return (((2 * tau + rper) * sizeof(TF) + 15) / 16) * 16 + (tau + 2) * sizeof(double) +
         2 * 256 * V2<T>::n * sizeof(T) + stage_bytes + 64;
}

template <typename T, typename TF>
cudaError_t launch_iterate(cudaStream_t st, Ctrl* ctrl, IterArgs<T, TF> g) {
  static thread_local int64_t last_tau = -1, last_stage = -1;
  static thread_local int cs = 16;
  auto kern = k_iterate<T, TF>;
  // stage r and the plan in shared memory when they fit next to the other buffers
  const int64_t stage_bytes = (g.kind == 0) ? g.m * 8 + (g.plan.perm_stride + g.tau + 1) * 4 : 0;
  g.stage = (g.kind == 0 && stage_bytes <= 160 * 1024) ? 1 : 0;
  const int64_t sb = g.stage ? stage_bytes : 0;
  if (last_tau != g.tau || last_stage != sb) {
    last_tau = g.tau;
    last_stage = sb;
    cs = 16;
    for (;;) {
      const size_t smem = iterate_smem<T, TF>(g.tau, cs, sb);
      set_smem_max((const void*)kern, (size_t)((int)smem));
      if (cs > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
      if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl >= 1) break;
      cudaGetLastError();
      if (cs == 1) break;
      cs >>= 1;
    }
  }
  const size_t smem = iterate_smem<T, TF>(g.tau, cs, sb);
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
  return cudaLaunchKernelEx(&cfg, kern, ctrl, g);
}

template cudaError_t launch_iterate<float, float>(cudaStream_t, Ctrl*, IterArgs<float, float>);
template cudaError_t launch_iterate<float, double>(cudaStream_t, Ctrl*, IterArgs<float, double>);
template cudaError_t launch_iterate<double, double>(cudaStream_t, Ctrl*, IterArgs<double, double>);

}  // namespace rs
