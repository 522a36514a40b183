// Applying the sketch (Section 4), for a whole chunk of iterations at once.
//
// S_k^T A and M_k = S_k^T A S_k do not depend on the iterate (only r_S = S_k^T r
// does), so they are formed for every iteration ("slot") of a chunk in batched,
// throughput-bound launches before the chunk's iterations run. A is symmetric,
// so S^T A = (A S)^T and the tau sketched rows are row combinations of A.
#include "rs_gemm.cuh"
#include "rs_kernels.cuh"

namespace rs {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

// a += sign * b as one fused multiply-add by +-1 per element: the product is exact, so
// the result is the correctly rounded a + b or a - b. A branch on the sign is
// predicated both ways and issues both adds, which halves the rate of the FP64 sums.
__device__ __forceinline__ void vadd(float4& a, const float4& b, bool neg) {
  const float sg = neg ? -1.f : 1.f;
  a.x = fmaf(b.x, sg, a.x);
  a.y = fmaf(b.y, sg, a.y);
  a.z = fmaf(b.z, sg, a.z);
  a.w = fmaf(b.w, sg, a.w);
}
__device__ __forceinline__ void vadd(double2& a, const double2& b, bool neg) {
  const double sg = neg ? -1.0 : 1.0;
  a.x = fma(b.x, sg, a.x);
  a.y = fma(b.y, sg, a.y);
}

// offset of entry (j, i) of a slot's S^T A: row-major with row stride ld (bq = 0),
// or blocked by slices of bq rows of the iterate: the tau x round_up(bq, 4) block
// of slice i / bq is contiguous (the persistent iteration kernel copies one block
// per CTA and iteration)
__host__ __device__ __forceinline__ int64_t sa_off(int64_t j, int64_t i, int64_t ld, int64_t bq,
                                                   int64_t tau) {
  if (bq == 0) return j * ld + i;
  const int64_t bqs = (bq + 3) / 4 * 4;
  const int64_t c = i / bq;
  return c * tau * bqs + j * bqs + (i - c * bq);
}

// ---------------------------------------------------------------------------
// Count / SubCount (Section 4.2): SA_s[j, :] = sum over bucket j of sign * A[row, :]
// for every slot s of the chunk. One warp per (slot, bucket, column slab of 32
// vectors); rows summed in bucket order (ascending row for Count, sample order
// for SubCount): deterministic. A (FP32, 67 MB at m = 4096) stays in L2 across
// the slots.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sa_batched(const Ctrl* __restrict__ ctrl, int force,
                                                    int nslots, PlanView plan,
                                                    const T* __restrict__ A, int64_t lda,
                                                    int64_t m, int64_t tau, T* __restrict__ SA,
                                                    int64_t ldsa, int64_t sa_slot, int64_t bq) {
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int lane = threadIdx.x & 31;
  const int64_t nslab = (m + 32 * VN - 1) / (32 * VN);
  const int64_t per_slot = tau * nslab;
  const int64_t units = nact * per_slot;
  const int64_t gw = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * 8;
  for (int64_t u = gw; u < units; u += nw) {
    const int64_t s = u / per_slot;
    const int64_t rem = u - s * per_slot;
    const int64_t j = rem / nslab;
    const int64_t c = (rem - j * nslab) * 32 * VN + lane * VN;
    const int32_t* perm = plan.perm + s * plan.perm_stride;
    const int32_t* boff = plan.boff + s * plan.boff_stride;
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
    if (bq == 0 ? c < ldsa : c < m)
      *reinterpret_cast<V*>(SA + s * sa_slot + sa_off(j, c, ldsa, bq, tau)) = acc;
  }
}

template <typename T>
cudaError_t launch_sa_batched(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              PlanView plan, const T* A, int64_t lda, int64_t m, int64_t tau, T* SA,
                              int64_t ldsa, int64_t sa_slot, int64_t bq) {
  constexpr int VN = Vec<T>::n;
  const int64_t units = (int64_t)nslots * tau * ((m + 32 * VN - 1) / (32 * VN));
  int blocks = (int)std::min<int64_t>((units + 7) / 8, 152 * 8);
  if (blocks < 1) blocks = 1;
  if (bq % 4 != 0) return cudaErrorInvalidValue;  // a vector never straddles two blocks
  k_sa_batched<T><<<blocks, 256, 0, st>>>(ctrl, force, nslots, plan, A, lda, m, tau, SA, ldsa,
                                          sa_slot, bq);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// M_s = S_s^T A S_s (FP64 out, tau x tau per slot) for the bucket-row sketches:
// M[j, l] = sum over bucket l of sign * row_j[row], row_j = A[C_j, :] (subsample)
// or SA_s[j, :]. One block per (slot, j); the plan and row j are staged in shared
// memory with coalesced loads when they fit.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_msys_batched(const Ctrl* __restrict__ ctrl, int force,
                                                      int nslots, PlanView plan, RowsView<T> rows,
                                                      int64_t m, int64_t tau, int64_t nperm,
                                                      int staged, double* __restrict__ M,
                                                      int64_t m_slot, float* __restrict__ Mf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t s = blockIdx.x / tau;
  const int64_t j = blockIdx.x - s * tau;
  if (s >= nact) return;
  const int32_t* perm = plan.perm + s * plan.perm_stride;
  const int32_t* boff = plan.boff + s * plan.boff_stride;
  double* Ms = M + s * m_slot;
  if (rows.SA == nullptr) {  // subsample: M[j, l] = A[C_j, C_l]
    const T* rowj = rows.A + (int64_t)entry_row(perm[j]) * rows.lda;
    for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) {
      Ms[j * tau + l] = (double)rowj[entry_row(perm[l])];
      if (Mf != nullptr) Mf[s * tau * tau + j * tau + l] = (float)rowj[entry_row(perm[l])];
    }
    return;
  }
  const T* Ss = rows.SA + s * rows.sa_slot;
  const int32_t* sp = perm;
  const int32_t* sb = boff;
  const T* sr = Ss + j * rows.ldsa;  // row j when row-major
  if (staged) {
    int32_t* sperm = reinterpret_cast<int32_t*>(smem_raw);
    int32_t* sboff = sperm + nperm;
    T* srow = reinterpret_cast<T*>(smem_raw + ((size_t)(nperm + tau + 1) * 4 + 15) / 16 * 16);
    for (int64_t t = threadIdx.x; t < nperm; t += blockDim.x) sperm[t] = perm[t];
    for (int64_t t = threadIdx.x; t <= tau; t += blockDim.x) sboff[t] = boff[t];
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x)
      srow[t] = Ss[sa_off(j, t, rows.ldsa, rows.bq, tau)];
    __syncthreads();
    sp = sperm; sb = sboff; sr = srow;
  }
  const bool flat = staged || rows.bq == 0;
  for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) {
    T acc = T(0);
    const int32_t t1 = sb[l + 1];
    for (int32_t t = sb[l]; t < t1; ++t) {
      const int32_t e = sp[t];
      const T v = flat ? sr[entry_row(e)] : Ss[sa_off(j, entry_row(e), rows.ldsa, rows.bq, tau)];
      acc = sadd(acc, v, entry_neg(e));
    }
    Ms[j * tau + l] = (double)acc;
    if (Mf != nullptr) Mf[s * tau * tau + j * tau + l] = (float)acc;
  }
}

template <typename T>
cudaError_t launch_msys_batched(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                                PlanView plan, RowsView<T> rows, int64_t m, int64_t tau,
                                double* M, int64_t m_slot, float* Mf) {
  const int64_t nperm = plan.perm_stride;
  size_t smem = 0;
  int staged = 0;
  if (rows.SA != nullptr) {
    smem = ((size_t)(nperm + tau + 1) * 4 + 15) / 16 * 16 + (size_t)m * sizeof(T);
    staged = smem <= 200 * 1024;
    if (!staged) smem = 0;
  }
  if (smem > 0) {
    cudaError_t e = set_smem_max((const void*)k_msys_batched<T>, (size_t)((int)smem));
    if (e != cudaSuccess) return e;
  }
  k_msys_batched<T><<<(unsigned)(nslots * tau), 512, smem, st>>>(ctrl, force, nslots, plan, rows, m,
                                                                  tau, nperm, staged, M, m_slot, Mf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S^T A and M = S^T A S of the bucket-row sketches in one pass: a block owns kJB
// buckets j of one slot; it stages the slot's plan, forms the rows SA_s[j, :] (sum
// over bucket j of sign * A[row, :], rows in bucket order) in shared memory, writes
// them out, and then M_s[j, l] = sum over bucket l of sign * SA_s[j, row] from
// shared memory, so S^T A is not read back.
// ---------------------------------------------------------------------------
// one bucket per block, two vectors of each of two rows in flight per thread, four
// 256-thread blocks per SM (64 registers): the reads of A come from L2, and more
// resident warps hide their latency better than more loads per thread (FP32: 2.87
// against 3.26 ms per 600 slots at m = 4096 for two buckets per block, four vectors
// and two blocks per SM; FP64 runs at the FP64 add rate either way)
constexpr int kJB = 1;  // buckets per block

template <typename T>
size_t sa_msys_smem(int64_t m, int64_t tau, int64_t nperm) {
  return ((size_t)(nperm + tau + 1) * 4 + 15) / 16 * 16 + (size_t)kJB * round_up(m, 4) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_sa_msys(const Ctrl* __restrict__ ctrl, int force, int nslots,
                                                 PlanView plan, const T* __restrict__ A, int64_t lda,
                                                 int64_t m, int64_t tau, int64_t nperm,
                                                 T* __restrict__ SA, int64_t ldsa, int64_t sa_slot,
                                                 int64_t bq, double* __restrict__ M, int64_t m_slot,
                                                 float* __restrict__ Mf) {
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t nj = (tau + kJB - 1) / kJB;
  const int64_t s = blockIdx.x / nj;
  const int64_t jb = (blockIdx.x - s * nj) * kJB;
  if (s >= nact) return;
  const int tid = threadIdx.x;
  int32_t* sperm = reinterpret_cast<int32_t*>(smem_raw);
  int32_t* sboff = sperm + nperm;
  const int64_t mr = round_up(m, 4);
  T* srow = reinterpret_cast<T*>(smem_raw + ((size_t)(nperm + tau + 1) * 4 + 15) / 16 * 16);
  const int32_t* perm = plan.perm + s * plan.perm_stride;
  const int32_t* boff = plan.boff + s * plan.boff_stride;
  for (int64_t t = tid; t < nperm; t += blockDim.x) sperm[t] = perm[t];
  for (int64_t t = tid; t <= tau; t += blockDim.x) sboff[t] = boff[t];
  __syncthreads();
  const int nrow = (int)(jb + kJB <= tau ? kJB : tau - jb);
  T* SAs = SA + s * sa_slot;
  // rows SA[j, :], j = jb .. jb + nrow - 1: each thread kVU vectors of VN columns at
  // once (kVU x 2 row loads in flight), rows summed in bucket order
  const int64_t nvec = (m + VN - 1) / VN;
  constexpr int kVU = 2;
  for (int r = 0; r < nrow; ++r) {
    const int64_t j = jb + r;
    const int32_t t0 = sboff[j], t1 = sboff[j + 1];
    for (int64_t v0 = tid; v0 < nvec; v0 += (int64_t)blockDim.x * kVU) {
      V acc[kVU];
#pragma unroll
      for (int u = 0; u < kVU; ++u) {
        if constexpr (VN == 4) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f); else acc[u] = make_double2(0.0, 0.0);
      }
      int32_t t = t0;
      for (; t + 2 <= t1; t += 2) {
        const int32_t ea = sperm[t], eb = sperm[t + 1];
        const T* ra = A + (int64_t)entry_row(ea) * lda;
        const T* rb = A + (int64_t)entry_row(eb) * lda;
        V va[kVU], vb[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
          const int64_t v = v0 + (int64_t)u * blockDim.x;
          if (v < nvec) {
            va[u] = __ldg(reinterpret_cast<const V*>(ra + v * VN));
            vb[u] = __ldg(reinterpret_cast<const V*>(rb + v * VN));
          }
        }
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
          if (v0 + (int64_t)u * blockDim.x < nvec) {
            vadd(acc[u], va[u], entry_neg(ea));
            vadd(acc[u], vb[u], entry_neg(eb));
          }
        }
      }
      if (t < t1) {
        const int32_t e = sperm[t];
        const T* ra = A + (int64_t)entry_row(e) * lda;
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
          const int64_t v = v0 + (int64_t)u * blockDim.x;
          if (v < nvec) vadd(acc[u], __ldg(reinterpret_cast<const V*>(ra + v * VN)), entry_neg(e));
        }
      }
#pragma unroll
      for (int u = 0; u < kVU; ++u) {
        const int64_t v = v0 + (int64_t)u * blockDim.x;
        if (v >= nvec) continue;
        const int64_t c = v * VN;
        *reinterpret_cast<V*>(srow + r * mr + c) = acc[u];
        // S^T A streams out marked evict-first, so that A stays in L2 for the other
        // slots (read back by the iterations a chunk later, from DRAM in any case)
        if (bq == 0 ? c < ldsa : c < m)
          __stcs(reinterpret_cast<V*>(SAs + sa_off(j, c, ldsa, bq, tau)), acc[u]);
      }
    }
  }
  __syncthreads();
  // M[j, l] for the block's rows, bucket l traversed once for all of them
  double* Ms = M + s * m_slot;
  for (int64_t l = tid; l < tau; l += blockDim.x) {
    T acc[kJB];
#pragma unroll
    for (int r = 0; r < kJB; ++r) acc[r] = T(0);
    const int32_t t1 = sboff[l + 1];
    for (int32_t t = sboff[l]; t < t1; ++t) {
      const int32_t e = sperm[t];
      const int64_t i = entry_row(e);
      const bool ng = entry_neg(e);
#pragma unroll
      for (int r = 0; r < kJB; ++r) {
        const T v = srow[r * mr + i];
        acc[r] = sadd(acc[r], v, ng);
      }
    }
    if (Mf != nullptr)
      for (int r = 0; r < nrow; ++r) Mf[s * m_slot + (jb + r) * tau + l] = (float)acc[r];
    else
      for (int r = 0; r < nrow; ++r) Ms[(jb + r) * tau + l] = (double)acc[r];
  }
}

// false when the block's buffers do not fit shared memory (two-kernel path)
template <typename T>
bool sa_msys_fits(int64_t m, int64_t tau, int64_t nperm) {
  // the problems this path takes: the plan and the rows of two buckets fit 200 KB (a
  // fixed rule, independent of the block's shape, so that larger m keep the paths
  // that share reads of A between slots in L2)
  return ((size_t)(nperm + tau + 1) * 4 + 15) / 16 * 16 + (size_t)2 * round_up(m, 4) * sizeof(T) <=
         200 * 1024;
}

template <typename T>
cudaError_t launch_sa_msys(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, PlanView plan,
                           const T* A, int64_t lda, int64_t m, int64_t tau, T* SA, int64_t ldsa,
                           int64_t sa_slot, int64_t bq, double* M, int64_t m_slot, float* Mf) {
  const int64_t nperm = plan.perm_stride;
  const size_t smem = sa_msys_smem<T>(m, tau, nperm);
  if (smem > 200 * 1024 || bq % 4 != 0) return cudaErrorInvalidValue;
  cudaError_t e = set_smem_max((const void*)k_sa_msys<T>, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  const int64_t nj = (tau + kJB - 1) / kJB;
  k_sa_msys<T><<<(unsigned)(nslots * nj), 256, smem, st>>>(ctrl, force, nslots, plan, A, lda, m, tau,
                                                           nperm, SA, ldsa, sa_slot, bq, M, m_slot,
                                                           Mf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gaussian sketch (Section 4.1): S_s stored transposed, ST_s (tau x ld), so that
// S^T A and S delta read rows. SA_s = ST_s A and M_s = SA_s ST_s^T as batched
// matrix products (blockIdx.z = slot).
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_gauss_system(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                                const T* ST, int64_t st_slot, const T* A, int64_t lda, int64_t m,
                                int64_t tau, T* SA, int64_t ldsa, int64_t sa_slot, double* M,
                                int64_t m_slot) {
  const Ctrl* c = force ? nullptr : ctrl;
  // SA[j, c] = sum_i ST[j, i] A[i, c]
  cudaError_t e = gemm_strided<T, T, T>(st, tau, m, m, ST, lda, 1, A, lda, 1, SA, ldsa, 0.0, 0, c,
                                        nslots, st_slot, 0, sa_slot);
  if (e != cudaSuccess) return e;
  // M[j, l] = sum_c SA[j, c] ST[l, c]
  return gemm_strided<T, T, double>(st, tau, tau, m, SA, ldsa, 1, ST, 1, lda, M, tau, 0.0, 0, c,
                                    nslots, sa_slot, st_slot, m_slot);
}

// M = S^T A S of every slot from S^T A formed elsewhere (the tensor-core product)
template <typename T>
cudaError_t launch_gauss_msys(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              const T* ST, int64_t st_slot, int64_t m, int64_t tau, const T* SA,
                              int64_t ldsa, int64_t sa_slot, double* M, int64_t m_slot,
                              int64_t lda) {
  const Ctrl* c = force ? nullptr : ctrl;
  // M[j, l] = sum_c SA[j, c] ST[l, c]
  return gemm_strided<T, T, double>(st, tau, tau, m, SA, ldsa, 1, ST, 1, lda, M, tau, 0.0, 0, c,
                                    nslots, sa_slot, st_slot, m_slot);
}

// ---------------------------------------------------------------------------
// SRHT (Section 4.3): S = (tau m')^{-1/2} D H_{m'}[0:m, C]. Products with S are
// fast Walsh-Hadamard transforms (Sylvester order, eq. (18)) of length m' in
// shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double row_sign(uint64_t key, int64_t i) {
  return draw_neg(draw_k(key, 1, (uint64_t)i)) ? -1.0 : 1.0;
}

// SA_s[j, c] = scale * (H (D A[:, c]))[C_j]; A symmetric so column c is row c.
// grid (m, slots)
template <typename T>
__global__ void __launch_bounds__(1024) k_srht_sa(const Ctrl* __restrict__ ctrl, int force,
                                                  int nslots, int64_t k0_arg, uint64_t seed,
                                                  PlanView plan, const T* __restrict__ A,
                                                  int64_t lda, int64_t m, int64_t mp, int64_t tau,
                                                  T* __restrict__ SA, int64_t ldsa,
                                                  int64_t sa_slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t s = blockIdx.y;
  if (s >= nact) return;
  const int64_t k = (force ? k0_arg : ctrl->k0) + s;
  const uint64_t key = iter_key(seed, k);
  const int32_t* C = plan.perm + s * plan.perm_stride;
  const int64_t c = blockIdx.x;
  for (int64_t i = threadIdx.x; i < mp; i += blockDim.x)
    buf[i] = i < m ? (T)(row_sign(key, i) * (double)A[c * lda + i]) : T(0);
  fwht_smem(buf, mp);
  const T scale = (T)(1.0 / sqrt((double)tau * (double)mp));
  T* SAs = SA + s * sa_slot;
  for (int64_t j = threadIdx.x; j < tau; j += blockDim.x) SAs[j * ldsa + c] = scale * buf[entry_row(C[j])];
}

// M_s[j, :] = scale * (H (D SA_s[j, :]))[C]; grid (tau, slots)
template <typename T>
__global__ void __launch_bounds__(1024) k_srht_msys(const Ctrl* __restrict__ ctrl, int force,
                                                    int nslots, int64_t k0_arg, uint64_t seed,
                                                    PlanView plan, const T* __restrict__ SA,
                                                    int64_t ldsa, int64_t sa_slot, int64_t m,
                                                    int64_t mp, int64_t tau, double* __restrict__ M,
                                                    int64_t m_slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* buf = reinterpret_cast<double*>(smem_raw);
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t s = blockIdx.y;
  if (s >= nact) return;
  const int64_t k = (force ? k0_arg : ctrl->k0) + s;
  const uint64_t key = iter_key(seed, k);
  const int32_t* C = plan.perm + s * plan.perm_stride;
  const int64_t j = blockIdx.x;
  const T* row = SA + s * sa_slot + j * ldsa;
  for (int64_t i = threadIdx.x; i < mp; i += blockDim.x)
    buf[i] = i < m ? row_sign(key, i) * (double)row[i] : 0.0;
  fwht_smem(buf, mp);
  const double scale = 1.0 / sqrt((double)tau * (double)mp);
  double* Ms = M + s * m_slot;
  for (int64_t l = threadIdx.x; l < tau; l += blockDim.x) Ms[j * tau + l] = scale * buf[entry_row(C[l])];
}

int64_t srht_max_pad() { return 16384; }

template <typename T>
cudaError_t launch_srht_system(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                               int64_t k0_arg, uint64_t seed, PlanView plan, const T* A,
                               int64_t lda, int64_t m, int64_t mp, int64_t tau, T* SA, int64_t ldsa,
                               int64_t sa_slot, double* M, int64_t m_slot) {
  size_t smem = (size_t)mp * sizeof(T);
  cudaError_t e = set_smem_max((const void*)k_srht_sa<T>, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_srht_sa<T><<<dim3((unsigned)m, (unsigned)nslots), 1024, smem, st>>>(
      ctrl, force, nslots, k0_arg, seed, plan, A, lda, m, mp, tau, SA, ldsa, sa_slot);
  smem = (size_t)mp * sizeof(double);
  e = set_smem_max((const void*)k_srht_msys<T>, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_srht_msys<T><<<dim3((unsigned)tau, (unsigned)nslots), 1024, smem, st>>>(
      ctrl, force, nslots, k0_arg, seed, plan, SA, ldsa, sa_slot, m, mp, tau, M, m_slot);
  return cudaGetLastError();
}

#define RS_INST(T)                                                                                \
  template bool sa_msys_fits<T>(int64_t, int64_t, int64_t);                                        \
  template cudaError_t launch_sa_msys<T>(cudaStream_t, const Ctrl*, int, int, PlanView, const T*,  \
                                         int64_t, int64_t, int64_t, T*, int64_t, int64_t, int64_t, \
                                         double*, int64_t, float*);                                \
  template cudaError_t launch_sa_batched<T>(cudaStream_t, const Ctrl*, int, int, PlanView,         \
                                            const T*, int64_t, int64_t, int64_t, T*, int64_t,      \
                                            int64_t, int64_t);                                     \
  template cudaError_t launch_msys_batched<T>(cudaStream_t, const Ctrl*, int, int, PlanView,       \
                                              RowsView<T>, int64_t, int64_t, double*, int64_t,     \
                                              float*);                                             \
  template cudaError_t launch_gauss_msys<T>(cudaStream_t, const Ctrl*, int, int, const T*,        \
                                           int64_t, int64_t, int64_t, const T*, int64_t, int64_t,   \
                                           double*, int64_t, int64_t);                              \
  template cudaError_t launch_gauss_system<T>(cudaStream_t, const Ctrl*, int, int, const T*,       \
                                              int64_t, const T*, int64_t, int64_t, int64_t, T*,    \
                                              int64_t, int64_t, double*, int64_t);                 \
  template cudaError_t launch_srht_system<T>(cudaStream_t, const Ctrl*, int, int, int64_t,         \
                                             uint64_t, PlanView, const T*, int64_t, int64_t,       \
                                             int64_t, int64_t, T*, int64_t, int64_t, double*,      \
                                             int64_t);
RS_INST(float)
RS_INST(double)
#undef RS_INST

}  // namespace rs
