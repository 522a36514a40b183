// Iterations of many problems at once: one thread-block cluster of kBatchCluster
// CTAs per problem, all right-hand sides of the problem in the same pass
// (Algorithm 2 with the momentum step of eq. (53), for A_p W = B_p column by column).
//
// CTA c of problem p owns the rows [c bq, (c + 1) bq) of w and r and the buckets
// (rows of S^T A, entries of r_S and delta) [c jpc, (c + 1) jpc). One iteration:
//   r_S pieces   warp per own bucket: sum of the signed residual entries of the
//                bucket (global r, fixed lane order), every right-hand side at once;
//                the bucket's plan entries come from shared memory, copied there
//                in bulk during the previous iteration;
//   exchange 1   cluster barrier; every CTA reads the pieces of the others from
//                distributed shared memory (full r_S) and the per-CTA squared norms
//                of r from the previous update (stopping test, identical in every
//                CTA);
//   delta pieces warp per own bucket: the bucket's row of M^+ (in shared memory,
//                copied in bulk ahead) times r_S;
//   exchange 2   cluster barrier; full delta from the pieces;
//   update       own rows: (A S delta)_i = sum_j (S^T A)[j, i] delta_j from the CTA's
//                contiguous slice of S^T A, streamed through a ring of bulk copies
//                that runs ahead into the next iterations; the momentum step, new r
//                written to global memory, the squared norms of the new r;
//   barrier 3    the new r visible to every CTA of the cluster.
// All sums run in a fixed order, so results do not depend on timing. Every wait on a
// copy is bounded; a CTA whose wait gives up raises a flag that the next exchange
// carries to every CTA of the cluster, so that all leave the loop together.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "rs_kernels.cuh"
#include "rs_ptx.cuh"

namespace rs {

namespace {
// two stages of large pieces: one bulk copy stream per CTA gains from larger pieces,
// not from more of them in flight
constexpr int kStages = 2;
// row pairs per thread (bq <= 2 * row_pairs * threads): two up to four right-hand
// sides, one beyond (register budget)
__host__ __device__ constexpr int row_pairs(int nr) { return nr <= 4 ? 2 : 1; }
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ float ld_dsmem(uint32_t addr, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double ld_dsmem(uint32_t addr, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

__device__ bool wait_full(uint64_t* bar, uint32_t parity) {
  if (ptx::mbar_test(bar, parity)) return true;
  const uint64_t t0 = ptx::now_ns();
  while (!ptx::mbar_test(bar, parity))
    if (ptx::now_ns() - t0 > kWaitNs) return false;
  return true;
}

// x += d for an unevaluated float pair x = hi + lo (two-sum, renormalised)
__device__ __forceinline__ void pair_add(float2& x, float d) {
  const float s = __fadd_rn(x.x, d);
  const float bb = __fsub_rn(s, x.x);
  const float err = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float lo = __fadd_rn(x.y, err);
  const float hi = __fadd_rn(s, lo);
  x = make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

// NR consecutive values from 16-byte aligned shared memory (vector loads)
template <typename T, int NR>
__device__ __forceinline__ void ld_vec(const T* p, T (&v)[NR]) {
  constexpr int bytes = (int)sizeof(T) * NR;
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) {
      const float4 x = reinterpret_cast<const float4*>(p)[i];
      memcpy(&v[i * 16 / (int)sizeof(T)], &x, 16);
    }
  } else if constexpr (bytes == 8) {
    const float2 x = *reinterpret_cast<const float2*>(p);
    memcpy(&v[0], &x, 8);
  } else {
#pragma unroll
    for (int i = 0; i < NR; ++i) v[i] = p[i];
  }
}

struct ClSmem {  // byte offsets of the dynamic shared memory, capacities in elements
  uint32_t ring, bars, xr, xn, xd, rsf, dl, red, pperm, pboff, pP, total;
  uint32_t cap_perm, cap_boff, cap_P;
};

template <typename T, int NR>
__host__ __device__ ClSmem cl_smem(uint32_t stage_bytes, int64_t tau_max, int64_t perm_max,
                                   int64_t pld_max) {
  const uint32_t jpc = (uint32_t)((tau_max + kBatchCluster - 1) / kBatchCluster);
  const uint32_t es = (uint32_t)sizeof(T);
  auto al = [](uint32_t v) { return (v + 15u) / 16u * 16u; };
  ClSmem s;
  // plan window of the own buckets: about perm_max / kBatchCluster entries; a CTA
  // whose window is larger reads its plan from global memory instead
  s.cap_perm = (uint32_t)std::min<int64_t>((perm_max + 3) / 4 * 4,
                                           (2 * ((perm_max + kBatchCluster - 1) / kBatchCluster) + 64 + 3) / 4 * 4);
  s.cap_boff = (jpc + 8u + 3u) / 4u * 4u;
  s.cap_P = jpc * (uint32_t)pld_max;
  s.ring = 0;
  s.bars = s.ring + kStages * stage_bytes;
  s.xr = al(s.bars + (kStages + 2) * 8);
  s.xn = al(s.xr + 2 * jpc * NR * es);
  s.xd = al(s.xn + 2 * (NR + 1) * es);
  s.rsf = al(s.xd + 2 * jpc * NR * es);
  s.dl = al(s.rsf + (uint32_t)tau_max * NR * es);
  s.red = al(s.dl + (uint32_t)tau_max * NR * es);
  s.pperm = al(s.red + 32 * NR * es);
  s.pboff = al(s.pperm + 2 * s.cap_perm * 4);
  s.pP = al(s.pboff + 2 * s.cap_boff * 4);
  s.total = al(s.pP + 2 * s.cap_P * es);
  return s;
}
}  // namespace

template <typename T, bool kMixed, int NR>
__global__ void __launch_bounds__(512, 1)
    k_batch_cluster(const BatchProbC<T>* __restrict__ probs, const int32_t* __restrict__ order,
                    int nrhs, BatchPairs pairs, const double* __restrict__ gam,
                    const double* __restrict__ bet, int64_t chunk, const double* __restrict__ tolp,
                    uint32_t stage_bytes, int64_t tau_max, int64_t perm_max, int64_t pld_max,
                    int32_t* err_word) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  constexpr int RPn = row_pairs(NR);
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t rank = cluster_rank();
  const int pidx = order[blockIdx.x / kBatchCluster];
  const BatchProbC<T>& pr = probs[pidx];
  Ctrl* ctrl = pr.ctrl;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int NT = blockDim.x;
  const ClSmem L = cl_smem<T, NR>(stage_bytes, tau_max, perm_max, pld_max);
  unsigned char* ring = smem + L.ring;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);  // kStages ring + 2 aux
  T* xr = reinterpret_cast<T*>(smem + L.xr);
  T* xn = reinterpret_cast<T*>(smem + L.xn);
  T* xd = reinterpret_cast<T*>(smem + L.xd);
  T* rsf = reinterpret_cast<T*>(smem + L.rsf);
  T* dl = reinterpret_cast<T*>(smem + L.dl);
  T* red = reinterpret_cast<T*>(smem + L.red);
  int32_t* pperm = reinterpret_cast<int32_t*>(smem + L.pperm);
  int32_t* pboff = reinterpret_cast<int32_t*>(smem + L.pboff);
  T* pP = reinterpret_cast<T*>(smem + L.pP);
  __shared__ int s_act[NR];
  __shared__ int s_go, s_err;
  __shared__ int32_t s_a0[2], s_b0[2];  // window starts of the plan pieces per buffer
  __shared__ int s_gperm[2];            // 1: the plan window did not fit, read it from global
  __shared__ int64_t s_k0, s_k, s_kend;

  // the problem's control block and pair flags, read by every CTA before any of
  // them changes them (barrier below)
  if (tid == 0) {
    s_k0 = ctrl->k0;
    s_k = ctrl->k;
    s_kend = lmin(s_k0 + chunk, ctrl->max_iters);
    s_go = !halted(ctrl);
    s_err = 0;
    for (int s = 0; s < kStages + 2; ++s) ptx::mbar_init(bars + s, 1);
    ptx::fence_mbar_init();
  }
  const int pbase = pidx * nrhs;
  if (tid < NR) s_act[tid] = (tid < nrhs) && (pairs.flag[pbase + tid] == 0);
  __syncthreads();
  ptx::cluster_sync_all();
  if (!s_go) return;  // the same in every CTA of the cluster
  const int64_t k0 = s_k0, kstart = s_k, kend = s_kend;
  const int64_t d = pr.d, tau = pr.tau, bq = pr.bq;
  const int64_t i0 = (int64_t)rank * bq;
  const int nrow = (int)lmax(0, lmin(d, i0 + bq) - i0);
  const int64_t jpc = (tau + kBatchCluster - 1) / kBatchCluster;
  const int64_t jpc_max = (tau_max + kBatchCluster - 1) / kBatchCluster;
  const int64_t jb0 = (int64_t)rank * jpc;
  const int64_t jb1 = lmin(tau, jb0 + jpc);
  const bool has_aux = jb1 > jb0;
  const int64_t bqs = (bq + 3) / 4 * 4;
  // ring of S^T A pieces: J rows of the CTA's tau x bqs slice per stage
  const int64_t J = lmax(1, lmin(tau, stage_bytes / (bqs * (int64_t)sizeof(T))));
  const int64_t npc = (tau + J - 1) / J;
  const int64_t total = (nrow > 0) ? (kend - kstart) * npc : 0;
  int64_t iss = 0, use = 0;
  auto issue = [&](int64_t g) {
    const int64_t slot = (kstart - k0) + g / npc;
    const int64_t j0 = (g % npc) * J;
    const int64_t rows = lmin(J, tau - j0);
    const T* src = pr.SA + slot * pr.sa_slot + (int64_t)rank * tau * bqs + j0 * bqs;
    const uint32_t bytes = (uint32_t)(rows * bqs * (int64_t)sizeof(T));
    uint64_t* bar = bars + (g % kStages);
    ptx::mbar_arrive_expect_tx(bar, bytes);
    ptx::bulk_g2s(ring + (g % kStages) * stage_bytes, src, bytes, bar);
  };
  // plan piece (the own buckets' entries and offsets) and the own rows of M^+ of a
  // slot, into buffer slot & 1; t0, t1 = the slot's boff[jb0], boff[jb1]
  int aux_iss[2] = {0, 0}, aux_use[2] = {0, 0};
  auto issue_aux = [&](int64_t slot, int32_t t0, int32_t t1) {
    const int b = (int)(slot & 1);
    const int32_t a0 = t0 & ~3, a1 = (t1 + 3) & ~3;
    const int32_t b0 = (int32_t)(jb0 & ~3), b1 = (int32_t)((jb1 + 1 + 3) & ~3);
    const uint32_t pbytes = (uint32_t)(a1 - a0) * 4u;
    const uint32_t bbytes = (uint32_t)(b1 - b0) * 4u;
    const uint32_t Pbytes = (uint32_t)((jb1 - jb0) * pr.pld * (int64_t)sizeof(T));
    const bool fits = (uint32_t)(a1 - a0) <= L.cap_perm;
    s_a0[b] = a0;
    s_b0[b] = b0;
    s_gperm[b] = !fits;
    uint64_t* bar = bars + kStages + b;
    ptx::mbar_arrive_expect_tx(bar, (fits ? pbytes : 0u) + bbytes + Pbytes);
    if (fits && pbytes > 0)
      ptx::bulk_g2s(pperm + b * L.cap_perm, pr.perm + slot * pr.perm_stride + a0, pbytes, bar);
    ptx::bulk_g2s(pboff + b * L.cap_boff, pr.boff + slot * pr.boff_stride + b0, bbytes, bar);
    ptx::bulk_g2s(pP + b * L.cap_P, pr.P + slot * pr.p_slot + jb0 * pr.pld, Pbytes, bar);
  };
  if (tid == 0) {
    for (; iss < lmin(total, kStages); ++iss) issue(iss);
    if (has_aux && kstart < kend) {
      const int32_t* bo = pr.boff + (kstart - k0) * pr.boff_stride;
      issue_aux(kstart - k0, bo[jb0], bo[jb1]);
    }
  }
  if (has_aux && kstart < kend) aux_iss[(kstart - k0) & 1]++;
  const T tol = (T)*tolp;
  int par = 0;
  int64_t k = kstart;
  bool broke = false;
  for (; k < kend; ++k) {
    const int64_t slot = k - k0;
    const int buf = (int)(slot & 1);
    // boff values of the next slot for its plan copy (consumed after the delta step)
    int32_t nt0 = 0, nt1 = 0;
    const bool pre = has_aux && k + 1 < kend;
    if (pre && tid == 0) {
      const int32_t* bo = pr.boff + (slot + 1) * pr.boff_stride;
      nt0 = bo[jb0];
      nt1 = bo[jb1];
    }
    if (has_aux) {
      if (!wait_full(bars + kStages + buf, (uint32_t)(aux_use[buf] & 1))) s_err = 1;
      aux_use[buf]++;
    }
    // (1) r_S pieces of the own buckets
    {
      const int32_t* bo = pboff + buf * L.cap_boff - s_b0[buf];
      const int32_t* pe = s_gperm[buf] ? pr.perm + slot * pr.perm_stride
                                        : pperm + buf * L.cap_perm - s_a0[buf];
      for (int64_t j = jb0 + wid; j < jb1; j += nw) {
        T acc[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = T(0);
        const int32_t t1 = bo[j + 1];
        for (int32_t t = bo[j] + lane; t < t1; t += 32) {
          const int32_t en = pe[t];
          const int64_t row = entry_row(en);
          const bool neg = entry_neg(en);
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            if (q < nrhs) {
              T v;
              if constexpr (kMixed) v = pr.r2[(int64_t)q * d + row].x;
              else v = pr.r[(int64_t)q * d + row];
              acc[q] = sadd(acc[q], v, neg);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const T v = warp_sum(acc[q]);
          if (lane == 0) xr[(par * jpc_max + (j - jb0)) * NR + q] = v;
        }
      }
    }
    if (tid == 0) xn[par * (NR + 1) + NR] = s_err ? T(1) : T(0);
    __syncthreads();
    ptx::cluster_sync_all();  // exchange 1
    // (2) stopping test on the current r (norms from the previous update), full r_S
    if (k > kstart && tid < nrhs && s_act[tid]) {
      T n2 = T(0);
      for (int c = 0; c < kBatchCluster; ++c)
        n2 += ld_dsmem(ptx::map_rank(xn + par * (NR + 1) + tid, c), T(0));
      const int pi = pbase + tid;
      const T rel = sqrt(n2) / (T)pairs.r0[pi];
      if (!isfinite(rel) || rel <= tol) s_act[tid] = 0;
      if (rank == 0) {
        pairs.resid[pi] = (double)rel;
        if (!isfinite(rel)) pairs.flag[pi] = 3;
        else if (rel <= tol) pairs.flag[pi] = kMixed ? 1 : 2;
      }
    }
    if (tid == 32) {
      int e = 0;
      for (int c = 0; c < kBatchCluster; ++c)
        e |= ld_dsmem(ptx::map_rank(xn + par * (NR + 1) + NR, c), T(0)) != T(0);
      s_go = !e;
    }
    for (int64_t e = tid; e < tau * NR; e += NT) {
      const int64_t j = e / NR;
      const int q = (int)(e - j * NR);
      const int64_t own = j / jpc;
      rsf[e] = ld_dsmem(ptx::map_rank(xr + (par * jpc_max + (j - own * jpc)) * NR + q, (uint32_t)own), T(0));
    }
    __syncthreads();
    int any = 0;
#pragma unroll
    for (int q = 0; q < NR; ++q) any |= s_act[q];
    if (!any || !s_go) {  // uniform over the cluster
      broke = true;
      break;
    }
    // (3) delta pieces of the own buckets: row j of M^+ times r_S
    {
      const T* Pb = pP + buf * L.cap_P;
      for (int64_t j = jb0 + wid; j < jb1; j += nw) {
        T acc[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = T(0);
        const T* prow = Pb + (j - jb0) * pr.pld;
        for (int64_t l = lane; l < tau; l += 32) {
          const T pv = prow[l];
          T rv[NR];
          ld_vec<T, NR>(rsf + l * NR, rv);
#pragma unroll
          for (int q = 0; q < NR; ++q) acc[q] += pv * rv[q];
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const T v = warp_sum(acc[q]);
          if (lane == 0) xd[(par * jpc_max + (j - jb0)) * NR + q] = v;
        }
      }
    }
    // the next slot's plan piece and M^+ rows into the other buffer (last read in
    // the previous iteration)
    if (pre) {
      if (tid == 0) issue_aux(slot + 1, nt0, nt1);
      aux_iss[(slot + 1) & 1]++;
    }
    __syncthreads();
    ptx::cluster_sync_all();  // exchange 2
    for (int64_t e = tid; e < tau * NR; e += NT) {
      const int64_t j = e / NR;
      const int q = (int)(e - j * NR);
      const int64_t own = j / jpc;
      dl[e] = ld_dsmem(ptx::map_rank(xd + (par * jpc_max + (j - own * jpc)) * NR + q, (uint32_t)own), T(0));
    }
    __syncthreads();
    // (4) update of the own rows
    T sq[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) sq[q] = T(0);
    if (nrow > 0) {
      const int32_t* inv = pr.inv + slot * pr.inv_slot + i0;
      int32_t en[RPn][2];
#pragma unroll
      for (int u = 0; u < RPn; ++u) {
        const int il = 2 * (tid + u * NT);
        en[u][0] = il < nrow ? inv[il] : kNotSketched;
        en[u][1] = il + 1 < nrow ? inv[il + 1] : kNotSketched;
      }
      T acc[RPn][2][NR];
#pragma unroll
      for (int u = 0; u < RPn; ++u)
#pragma unroll
        for (int q = 0; q < NR; ++q) { acc[u][0][q] = T(0); acc[u][1][q] = T(0); }
      for (int64_t pc = 0; pc < npc; ++pc, ++use) {
        const int st = (int)(use % kStages);
        if (!wait_full(bars + st, (uint32_t)((use / kStages) & 1))) s_err = 1;
        const T* piece = reinterpret_cast<const T*>(ring + st * stage_bytes);
        const int64_t j0 = pc * J;
        const int64_t rows = lmin(J, tau - j0);
        for (int64_t jj = 0; jj < rows; ++jj) {
          T dq[NR];
          ld_vec<T, NR>(dl + (j0 + jj) * NR, dq);
#pragma unroll
          for (int u = 0; u < RPn; ++u) {
            const int il = 2 * (tid + u * NT);
            if (il < nrow) {
              const T2 sa = *reinterpret_cast<const T2*>(piece + jj * bqs + il);
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                acc[u][0][q] += sa.x * dq[q];
                acc[u][1][q] += sa.y * dq[q];
              }
            }
          }
        }
        __syncthreads();  // stage consumed
        if (tid == 0 && iss < total) issue(iss++);
      }
      const T g = (T)gam[k], b = (T)bet[k];
#pragma unroll
      for (int u = 0; u < RPn; ++u) {
        const int il0 = 2 * (tid + u * NT);
        if (il0 >= nrow) continue;
        // the pair of rows: all state loads first, then the updates and stores
        // (two rows at a time up to four right-hand sides, else one)
        constexpr int HB = NR <= 4 ? 2 : 1;
#pragma unroll
        for (int h0 = 0; h0 < 2; h0 += HB) {
        if constexpr (kMixed) {
          float dw[2][NR], dr[2][NR];
          float2 w2[2][NR], r2[2][NR];
#pragma unroll
          for (int h = h0; h < h0 + HB; ++h)
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              if (q < nrhs && il0 + h < nrow) {
                const int64_t o = (int64_t)q * d + i0 + il0 + h;
                dw[h][q] = pr.dw[o]; dr[h][q] = pr.dr[o]; w2[h][q] = pr.w2[o]; r2[h][q] = pr.r2[o];
              }
            }
#pragma unroll
          for (int h = h0; h < h0 + HB; ++h) {
            const int32_t e = en[u][h];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              if (q >= nrhs || il0 + h >= nrow || !s_act[q]) continue;
              const float sd = (e == kNotSketched) ? 0.f
                               : (entry_neg(e) ? -dl[entry_row(e) * NR + q] : dl[entry_row(e) * NR + q]);
              const int64_t o = (int64_t)q * d + i0 + il0 + h;
              const float ndw = b * dw[h][q] - g * sd;
              const float ndr = b * dr[h][q] - g * acc[u][h][q];
              pair_add(w2[h][q], ndw);
              pair_add(r2[h][q], ndr);
              pr.dw[o] = ndw;
              pr.dr[o] = ndr;
              pr.w2[o] = w2[h][q];
              pr.r2[o] = r2[h][q];
              sq[q] += r2[h][q].x * r2[h][q].x;
            }
          }
        } else {
          T w[2][NR], wp[2][NR], r[2][NR], rp[2][NR];
#pragma unroll
          for (int h = h0; h < h0 + HB; ++h)
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              if (q < nrhs && il0 + h < nrow) {
                const int64_t o = (int64_t)q * d + i0 + il0 + h;
                w[h][q] = pr.w[o]; wp[h][q] = pr.wp[o]; r[h][q] = pr.r[o]; rp[h][q] = pr.rp[o];
              }
            }
#pragma unroll
          for (int h = h0; h < h0 + HB; ++h) {
            const int32_t e = en[u][h];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              if (q >= nrhs || il0 + h >= nrow || !s_act[q]) continue;
              const T sd = (e == kNotSketched) ? T(0)
                           : (entry_neg(e) ? -dl[entry_row(e) * NR + q] : dl[entry_row(e) * NR + q]);
              const int64_t o = (int64_t)q * d + i0 + il0 + h;
              const T rn = (T(1) + b) * r[h][q] - b * rp[h][q] - g * acc[u][h][q];
              pr.wp[o] = w[h][q];
              pr.w[o] = (T(1) + b) * w[h][q] - b * wp[h][q] - g * sd;
              pr.rp[o] = r[h][q];
              pr.r[o] = rn;
              sq[q] += rn * rn;
            }
          }
        }
        }
      }
    }
    // squared norms of the new r over the own rows (fixed order) for the next test
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const T v = warp_sum(sq[q]);
      if (lane == 0) red[wid * NR + q] = v;
    }
    __syncthreads();
    if (tid < NR) {
      T t = T(0);
      for (int w = 0; w < nw; ++w) t += red[w * NR + tid];
      xn[(par ^ 1) * (NR + 1) + tid] = t;
      if (rank == 0 && tid < nrhs && s_act[tid]) pairs.iters[pbase + tid] += 1;
    }
    __syncthreads();
    ptx::cluster_sync_all();  // barrier 3: the new r visible in the cluster
    par ^= 1;
  }
  if (!broke && k > kstart) {
    // stopping test on the r of the last iteration of the chunk
    if (tid == 0) xn[par * (NR + 1) + NR] = s_err ? T(1) : T(0);
    __syncthreads();
    ptx::cluster_sync_all();
    if (tid < nrhs && s_act[tid]) {
      T n2 = T(0);
      for (int c = 0; c < kBatchCluster; ++c)
        n2 += ld_dsmem(ptx::map_rank(xn + par * (NR + 1) + tid, c), T(0));
      const int pi = pbase + tid;
      const T rel = sqrt(n2) / (T)pairs.r0[pi];
      if (rank == 0) {
        pairs.resid[pi] = (double)rel;
        if (!isfinite(rel)) pairs.flag[pi] = 3;
        else if (rel <= tol) pairs.flag[pi] = kMixed ? 1 : 2;
      }
    }
    if (tid == 32) {
      int e = 0;
      for (int c = 0; c < kBatchCluster; ++c)
        e |= ld_dsmem(ptx::map_rank(xn + par * (NR + 1) + NR, c), T(0)) != T(0);
      if (e) s_go = 0;
    }
  }
  // copies still in flight (issued ahead of a left loop) land before exit
  if (tid == 0) {
    for (; use < iss; ++use) wait_full(bars + (use % kStages), (uint32_t)((use / kStages) & 1));
    for (int b = 0; b < 2; ++b)
      for (; aux_use[b] < aux_iss[b]; ++aux_use[b]) wait_full(bars + kStages + b, (uint32_t)(aux_use[b] & 1));
  }
  __syncthreads();
  ptx::cluster_sync_all();  // no CTA leaves while another reads its shared memory
  if (rank == 0 && tid == 0) {
    ctrl->k = k;
    if (!s_go || s_err) {
      ctrl->status = kStatusTimeout;
      ctrl->stop = 1;
      atomicExch(err_word, 1);
    }
    int done = 1;
    for (int q = 0; q < nrhs; ++q) done &= (pairs.flag[pbase + q] >= 2);
    if (done || k >= ctrl->max_iters) ctrl->stop = 1;
    __threadfence();
  }
}

namespace {

// shared memory of a launch: the ring stage is sized so that two CTAs fit on an SM
// where they can, never below one row of the widest slice
template <typename T, int NR>
ClSmem cl_plan(int64_t tau_max, int64_t bq_max, int64_t perm_max, int64_t pld_max,
               uint32_t* stage_out) {
  const uint32_t row = (uint32_t)((bq_max + 3) / 4 * 4 * (int64_t)sizeof(T));
  const uint32_t row128 = (row + 127u) / 128u * 128u;
  const ClSmem base = cl_smem<T, NR>(0, tau_max, perm_max, pld_max);
  const uint32_t half = 113u * 1024u;
  const uint32_t full = 227u * 1024u;
  uint32_t stage = 65536u;
  if (base.total < half) stage = std::min<uint32_t>(stage, (half - base.total) / kStages / 128u * 128u);
  else if (base.total < full) stage = std::min<uint32_t>(stage, (full - base.total) / kStages / 128u * 128u);
  stage = std::max<uint32_t>(stage, row128);
  *stage_out = stage;
  return cl_smem<T, NR>(stage, tau_max, perm_max, pld_max);
}

template <typename T, bool kMixed, int NR>
cudaError_t launch_nr(cudaStream_t st, const BatchProbC<T>* probs, const int32_t* order, int nprob,
                      int nrhs, BatchPairs pairs, const double* gam, const double* bet,
                      int64_t chunk, const double* tol, int64_t tau_max, int64_t bq_max,
                      int64_t perm_max, int64_t pld_max, int threads, int32_t* err_word,
                      int* fit_out) {
  uint32_t stage = 0;
  const ClSmem L = cl_plan<T, NR>(tau_max, bq_max, perm_max, pld_max, &stage);
  if (L.total > 227u * 1024u) return cudaErrorInvalidValue;
  auto kern = k_batch_cluster<T, kMixed, NR>;
  cudaError_t e = set_smem_max((const void*)kern, (size_t)((int)L.total));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(std::max(nprob, 1) * kBatchCluster));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = L.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBatchCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (fit_out != nullptr) {  // occupancy query only
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
    *fit_out = (e == cudaSuccess) ? ncl : 0;
    return e;
  }
  if (nprob <= 0) return cudaSuccess;
  return cudaLaunchKernelEx(&cfg, kern, probs, order, nrhs, pairs, gam, bet, chunk, tol, stage,
                            tau_max, perm_max, pld_max, err_word);
}

template <typename T, bool kMixed>
cudaError_t dispatch(cudaStream_t st, const BatchProbC<T>* probs, const int32_t* order, int nprob,
                     int nrhs, BatchPairs pairs, const double* gam, const double* bet,
                     int64_t chunk, const double* tol, int64_t tau_max, int64_t bq_max,
                     int64_t perm_max, int64_t pld_max, int threads, int32_t* err_word,
                     int* fit_out) {
  if (nrhs < 1 || nrhs > 8 || threads % 32 != 0 || threads > 512 || threads < 64)
    return cudaErrorInvalidValue;
  if (bq_max > (int64_t)2 * row_pairs(nrhs <= 4 ? 4 : 8) * threads) return cudaErrorInvalidValue;
#define RS_NR(N)                                                                                 \
  return launch_nr<T, kMixed, N>(st, probs, order, nprob, nrhs, pairs, gam, bet, chunk, tol,     \
                                 tau_max, bq_max, perm_max, pld_max, threads, err_word, fit_out)
  if (nrhs <= 1) RS_NR(1);
  if (nrhs <= 2) RS_NR(2);
  if (nrhs <= 4) RS_NR(4);
  RS_NR(8);
#undef RS_NR
}

}  // namespace

template <typename T, bool kMixed>
cudaError_t launch_batch_cluster(cudaStream_t st, const BatchProbC<T>* probs, const int32_t* order,
                                 int nprob, int nrhs, BatchPairs pairs, const double* gam,
                                 const double* bet, int64_t chunk, const double* tol,
                                 int64_t tau_max, int64_t bq_max, int64_t perm_max, int64_t pld_max,
                                 int threads, int32_t* err_word) {
  return dispatch<T, kMixed>(st, probs, order, nprob, nrhs, pairs, gam, bet, chunk, tol, tau_max,
                             bq_max, perm_max, pld_max, threads, err_word, nullptr);
}

// clusters of the kernel that fit on the GPU at once (0: the launch cannot run)
template <typename T, bool kMixed>
int batch_cluster_fit(int nrhs, int64_t tau_max, int64_t bq_max, int64_t perm_max, int64_t pld_max,
                      int threads) {
  int ncl = 0;
  BatchPairs none{};
  if (dispatch<T, kMixed>(nullptr, nullptr, nullptr, 0, nrhs, none, nullptr, nullptr, 0, nullptr,
                          tau_max, bq_max, perm_max, pld_max, threads, nullptr, &ncl) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl;
}

#define RS_BCL_INST(T, MX)                                                                        \
  template cudaError_t launch_batch_cluster<T, MX>(                                               \
      cudaStream_t, const BatchProbC<T>*, const int32_t*, int, int, BatchPairs, const double*,   \
      const double*, int64_t, const double*, int64_t, int64_t, int64_t, int64_t, int, int32_t*); \
  template int batch_cluster_fit<T, MX>(int, int64_t, int64_t, int64_t, int64_t, int);
RS_BCL_INST(float, true)
RS_BCL_INST(double, false)
#undef RS_BCL_INST

}  // namespace rs
