// Matrix-free primal ridge on a sparse X (CSR): A = X^T X + lambda I is never formed
// (eq. (2)); A V = X^T (X V) + lambda V. Sketches with bucket rows (subsample,
// subcount, count) over the d columns of X.
//
// Setup: CSC of X by a stable counting sort (deterministic order: rows ascending in
// every column), b = X^T y by column gathers.
//
// Phase 1, per slot of a chunk: the rows of X that meet the slot's sampled columns
// are compacted (count, batched prefix sum, fill, all in row order) into XS, the
// n x tau sketched design restricted to those rows, as compact rows of
// (bucket, sigma * x) entries; then M = (XS)^T (XS) + lambda S^T S, with
// S^T S = diag(bucket sizes), from the rows' outer products.
//
// Phase 2, per iteration: delta = M^+ S^T r; v = (XS) delta on the compact rows;
// u = X^T v by column gathers over the CSC (a column longer than kPiece entries is
// split into pieces summed in order by the update); then A S delta = u + lambda
// S delta and the momentum step of eq. (53) on w and r, the norm and the
// stopping test (last-block reduction).
#include <cuda_bf16.h>

#include "rs_kernels.cuh"

namespace rs {

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// ---------------------------------------------------------------------------
// CSC of X. The nnz range is cut into nb contiguous parts, one warp per part in
// order; a part's per-column counts (pass 1) and cursors (pass 2) live in row b
// of the nb x d table. Lanes of one step with the same column are ranked by lane
// order (match_any), so every column lists its rows in ascending order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t row_of(const int64_t* __restrict__ rowptr, int64_t n, int64_t e) {
  int64_t lo = 0, hi = n;  // rowptr[lo] <= e < rowptr[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_csc_count(const int32_t* __restrict__ colidx, int64_t nnz, int nb, int64_t d,
                            int32_t* __restrict__ table) {
  const int b = blockIdx.x, lane = threadIdx.x;
  const int64_t per = (nnz + nb - 1) / nb;
  const int64_t e0 = min(nnz, b * per), e1 = min(nnz, e0 + per);
  int32_t* tb = table + (int64_t)b * d;
  for (int64_t e = e0; e < e1; e += 32) {
    const int64_t ee = e + lane;
    const int32_t c = ee < e1 ? colidx[ee] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(same) - 1;
    if (c >= 0 && lane == leader) tb[c] += __popc(same);
    __syncwarp();
  }
}

// colptr[c + 1] = total count of column c; table[b][c] = count of part b
__global__ void k_csc_totals(const int32_t* __restrict__ table, int nb, int64_t d,
                             int64_t* __restrict__ colcnt) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= d) return;
  int64_t t = 0;
  for (int b = 0; b < nb; ++b) t += table[(int64_t)b * d + c];
  colcnt[c] = t;
}

// exclusive scan of n int64 values in one block (setup-sized inputs), out[n] = total
__global__ void __launch_bounds__(1024) k_scan_one(const int64_t* __restrict__ in, int64_t n,
                                                   int64_t* __restrict__ out) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + 1023) / 1024;
  const int64_t i0 = min(n, t * per), i1 = min(n, i0 + per);
  int64_t s = 0;
  for (int64_t i = i0; i < i1; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the parts
    const int64_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = t > 0 ? part[t - 1] : 0;
  for (int64_t i = i0; i < i1; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == 1023) out[n] = part[1023];
}

// table[b][c] <- colptr[c] + sum_{b' < b} count[b'][c]: the first slot of part b in column c
__global__ void k_csc_cursors(int32_t* __restrict__ table, int nb, int64_t d,
                              const int64_t* __restrict__ colptr) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= d) return;
  int64_t run = colptr[c];
  for (int b = 0; b < nb; ++b) {
    const int32_t cnt = table[(int64_t)b * d + c];
    table[(int64_t)b * d + c] = (int32_t)(run - colptr[c]);  // offset within the column
    run += cnt;
  }
}

template <typename VT>
__global__ void k_csc_fill(const int64_t* __restrict__ rowptr, int64_t n,
                           const int32_t* __restrict__ colidx, const VT* __restrict__ val,
                           int64_t nnz, int nb, int64_t d, int32_t* __restrict__ table,
                           const int64_t* __restrict__ colptr, int32_t* __restrict__ rowidx,
                           VT* __restrict__ cval) {
  const int b = blockIdx.x, lane = threadIdx.x;
  const int64_t per = (nnz + nb - 1) / nb;
  const int64_t e0 = min(nnz, b * per), e1 = min(nnz, e0 + per);
  int32_t* tb = table + (int64_t)b * d;
  for (int64_t e = e0; e < e1; e += 32) {
    const int64_t ee = e + lane;
    const int32_t c = ee < e1 ? colidx[ee] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(same) - 1;
    int32_t base = 0;
    if (c >= 0 && lane == leader) base = tb[c];
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c >= 0) {
      const int rank = __popc(same & ((1u << lane) - 1u));
      const int64_t pos = colptr[c] + base + rank;
      rowidx[pos] = (int32_t)row_of(rowptr, n, ee);
      cval[pos] = val[ee];
      if (lane == leader) tb[c] = base + __popc(same);
    }
    __syncwarp();
  }
}

template <typename VT>
cudaError_t build_csc(cudaStream_t st, const int64_t* rowptr, int64_t n, const int32_t* colidx,
                      const VT* val, int64_t nnz, int64_t d, int32_t* table, int nb,
                      int64_t* colcnt, int64_t* colptr, int32_t* rowidx, VT* cval) {
  cudaError_t e = cudaMemsetAsync(table, 0, (size_t)nb * d * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_csc_count<<<nb, 32, 0, st>>>(colidx, nnz, nb, d, table);
  const unsigned gd = (unsigned)((d + 255) / 256);
  k_csc_totals<<<gd, 256, 0, st>>>(table, nb, d, colcnt);
  k_scan_one<<<1, 1024, 0, st>>>(colcnt, d, colptr);
  k_csc_cursors<<<gd, 256, 0, st>>>(table, nb, d, colptr);
  k_csc_fill<VT><<<nb, 32, 0, st>>>(rowptr, n, colidx, val, nnz, nb, d, table, colptr, rowidx, cval);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Products with X and X^T
// ---------------------------------------------------------------------------
// z[r] = sum_e val[e] * x[col[e]] over row r, FP64 (one thread per row, row order)
template <typename VT>
__global__ void k_csr_spmv_d(const int64_t* __restrict__ rowptr, int64_t n,
                             const int32_t* __restrict__ colidx, const VT* __restrict__ val,
                             const double* __restrict__ x, double* __restrict__ z,
                             const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) acc += to_d(val[e]) * x[colidx[e]];
    z[r] = acc;
  }
}

// Column gathers of X^T v as pieces: piece i covers the entries
// [pstart[i], min(pstart[i] + kPiece, colptr[pcol[i] + 1])) of column pcol[i] and
// writes pu[i]; column c owns the pieces [cpiece[c], cpiece[c + 1]). One warp per
// piece, lanes strided, fixed reduction order.
template <typename VT, typename AT>
__global__ void __launch_bounds__(256) k_csc_pieces(const int64_t* __restrict__ colptr,
                                                    const int32_t* __restrict__ rowidx,
                                                    const VT* __restrict__ cval,
                                                    const int32_t* __restrict__ pcol,
                                                    const int64_t* __restrict__ pstart,
                                                    int64_t npieces, const AT* __restrict__ v,
                                                    AT* __restrict__ pu,
                                                    const int32_t* __restrict__ stop,
                                                    const Ctrl* __restrict__ ctrl) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  if (ctrl != nullptr && halted(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = w; i < npieces; i += nw) {
    const int64_t e0 = pstart[i];
    const int64_t e1 = min(e0 + (int64_t)kPiece, colptr[pcol[i] + 1]);
    AT acc = AT(0);
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      AT x;
      if constexpr (sizeof(AT) == 8) x = to_d(cval[e]); else x = to_f(cval[e]);
      acc += x * v[rowidx[e]];
    }
    acc = warp_sum(acc);
    if (lane == 0) pu[i] = acc;
  }
}

// out[c] = sum of column c's pieces in order (+ lambda * add[c] when add != nullptr)
__global__ void k_pieces_sum(const int32_t* __restrict__ cpiece, int64_t d,
                             const double* __restrict__ pu, double* __restrict__ out,
                             const int32_t* __restrict__ stop) {
  if (stop != nullptr && *(volatile const int32_t*)stop) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d;
       c += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t i = cpiece[c]; i < cpiece[c + 1]; ++i) s += pu[i];
    out[c] = s;
  }
}

template <typename VT>
cudaError_t sparse_xtv_d(cudaStream_t st, const SparseX<VT>& X, const double* v, double* out,
                         double* pu, const int32_t* stop) {
  const int64_t blocks = std::min<int64_t>((X.npieces + 7) / 8, 152 * 16);
  k_csc_pieces<VT, double><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
      X.colptr, X.rowidx, X.cval, X.pcol, X.pstart, X.npieces, v, pu, stop, nullptr);
  k_pieces_sum<<<(unsigned)std::min<int64_t>((X.d + 255) / 256, 1024), 256, 0, st>>>(
      X.cpiece, X.d, pu, out, stop);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t sparse_xv_d(cudaStream_t st, const SparseX<VT>& X, const double* x, double* z,
                        const int32_t* stop) {
  const int64_t blocks = std::min<int64_t>((X.n + 255) / 256, 152 * 8);
  k_csr_spmv_d<VT><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
      X.rowptr, X.n, X.colidx, X.val, x, z, stop);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Phase 1: XS on the rows that meet the sampled columns, then M
// ---------------------------------------------------------------------------
constexpr int kMfRows = 4;                        // rows per thread
constexpr int kMfBlock = 1024 * kMfRows;          // rows per block

__device__ __forceinline__ int mf_row_count(const MfArgs& a, const int32_t* __restrict__ inv,
                                            int64_t r) {
  int c = 0;
  if (r < a.n)
    for (int64_t e = a.rowptr[r]; e < a.rowptr[r + 1]; ++e) c += inv[a.colidx[e]] != kNotSketched;
  return c;
}

// per (row block, slot): entries and non-empty rows of the block
__global__ void __launch_bounds__(1024) k_mf_count(const Ctrl* __restrict__ ctrl, int force,
                                                   int nslots, MfArgs a) {
  const int64_t s = blockIdx.y;
  if (s >= active_slots(ctrl, force, nslots)) return;
  const int32_t* inv = a.inv + s * a.inv_slot;
  int ce = 0, cr = 0;
#pragma unroll
  for (int q = 0; q < kMfRows; ++q) {
    const int64_t r = (int64_t)blockIdx.x * kMfBlock + q * 1024 + threadIdx.x;
    const int c = mf_row_count(a, inv, r);
    ce += c;
    cr += c > 0;
  }
  __shared__ int s_e[32], s_r[32];
  ce = warp_sum(ce);
  cr = warp_sum(cr);
  if ((threadIdx.x & 31) == 0) { s_e[threadIdx.x >> 5] = ce; s_r[threadIdx.x >> 5] = cr; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int te = 0, tr = 0;
    for (int w = 0; w < 32; ++w) { te += s_e[w]; tr += s_r[w]; }
    a.bsum[(s * a.nrb + blockIdx.x) * 2] = te;
    a.bsum[(s * a.nrb + blockIdx.x) * 2 + 1] = tr;
  }
}

// per slot: exclusive scan of the block counts; totals; cptr[R] = E
__global__ void __launch_bounds__(1024) k_mf_bscan(const Ctrl* __restrict__ ctrl, int force,
                                                   int nslots, MfArgs a) {
  const int64_t s = blockIdx.x;
  if (s >= active_slots(ctrl, force, nslots)) return;
  if (threadIdx.x != 0) return;  // nrb is small (n / 4096)
  int32_t* bs = a.bsum + s * a.nrb * 2;
  int32_t* bo = a.boffs + s * a.nrb * 2;
  int te = 0, tr = 0;
  for (int64_t b = 0; b < a.nrb; ++b) {
    bo[b * 2] = te;
    bo[b * 2 + 1] = tr;
    te += bs[b * 2];
    tr += bs[b * 2 + 1];
  }
  a.tot[s * 2] = te;
  a.tot[s * 2 + 1] = tr;
  a.cptr[s * (a.rcap + 1) + tr] = te;
}

// per (row block, slot): block-local scan of the rows' counts and the compact rows
template <typename VT, typename AT>
__global__ void __launch_bounds__(1024) k_mf_fill(const Ctrl* __restrict__ ctrl, int force,
                                                  int nslots, MfArgs a, const VT* __restrict__ val,
                                                  AT* __restrict__ eval) {
  const int64_t s = blockIdx.y;
  if (s >= active_slots(ctrl, force, nslots)) return;
  const int32_t* inv = a.inv + s * a.inv_slot;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  int cnt[kMfRows];
  int ce = 0, cr = 0;
#pragma unroll
  for (int q = 0; q < kMfRows; ++q) {  // thread t owns rows t*4 .. t*4 + 3 of the block
    const int64_t r = (int64_t)blockIdx.x * kMfBlock + t * kMfRows + q;
    cnt[q] = mf_row_count(a, inv, r);
    ce += cnt[q];
    cr += cnt[q] > 0;
  }
  // exclusive scan of (ce, cr) over the block's threads
  __shared__ int s_e[32], s_r[32];
  int ie = ce, ir = cr;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ve = __shfl_up_sync(0xffffffffu, ie, o), vr = __shfl_up_sync(0xffffffffu, ir, o);
    if (lane >= o) { ie += ve; ir += vr; }
  }
  if (lane == 31) { s_e[wid] = ie; s_r[wid] = ir; }
  __syncthreads();
  if (wid == 0) {
    int ve = s_e[lane], vr = s_r[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ue = __shfl_up_sync(0xffffffffu, ve, o), ur = __shfl_up_sync(0xffffffffu, vr, o);
      if (lane >= o) { ve += ue; vr += ur; }
    }
    s_e[lane] = ve;
    s_r[lane] = vr;
  }
  __syncthreads();
  const int32_t* bo = a.boffs + (s * a.nrb + blockIdx.x) * 2;
  int eo = bo[0] + (wid > 0 ? s_e[wid - 1] : 0) + ie - ce;
  int ro = bo[1] + (wid > 0 ? s_r[wid - 1] : 0) + ir - cr;
  int32_t* crow = a.crow + s * a.rcap;
  int32_t* cptr = a.cptr + s * (a.rcap + 1);
  int32_t* eb = a.ebuck + s * a.ecap;
  AT* ev = eval + s * a.ecap;
#pragma unroll
  for (int q = 0; q < kMfRows; ++q) {
    if (cnt[q] == 0) continue;
    const int64_t r = (int64_t)blockIdx.x * kMfBlock + t * kMfRows + q;
    crow[ro] = (int32_t)r;
    cptr[ro] = eo;
    for (int64_t e = a.rowptr[r]; e < a.rowptr[r + 1]; ++e) {
      const int32_t iv = inv[a.colidx[e]];
      if (iv == kNotSketched) continue;
      eb[eo] = iv & 0x7FFFFFFF;
      AT x;
      if constexpr (sizeof(AT) == 8) x = to_d(val[e]); else x = to_f(val[e]);
      ev[eo] = entry_neg(iv) ? -x : x;
      ++eo;
    }
    ++ro;
  }
}

// M = (XS)^T (XS) + lambda S^T S for every active slot (M zeroed before)
template <typename AT>
__global__ void k_mf_gram(const Ctrl* __restrict__ ctrl, int force, int nslots, MfArgs a,
                          const AT* __restrict__ eval, PlanView plan, double* __restrict__ M,
                          int64_t m_slot) {
  const int64_t s = blockIdx.y;
  if (s >= active_slots(ctrl, force, nslots)) return;
  const int32_t R = a.tot[s * 2 + 1];
  const int32_t* cptr = a.cptr + s * (a.rcap + 1);
  const int32_t* eb = a.ebuck + s * a.ecap;
  const AT* ev = eval + s * a.ecap;
  double* Ms = M + s * m_slot;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < R;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e0 = cptr[t], e1 = cptr[t + 1];
    for (int32_t i = e0; i < e1; ++i) {
      const int32_t bi = eb[i];
      const double xi = (double)ev[i];
      atomicAdd(&Ms[(int64_t)bi * a.tau + bi], xi * xi);
      for (int32_t j = i + 1; j < e1; ++j) {
        const double v = xi * (double)ev[j];
        const int32_t bj = eb[j];
        atomicAdd(&Ms[(int64_t)bi * a.tau + bj], v);
        atomicAdd(&Ms[(int64_t)bj * a.tau + bi], v);
      }
    }
  }
  if (blockIdx.x == 0) {
    const int32_t* boff = plan.boff + s * plan.boff_stride;
    for (int64_t j = threadIdx.x; j < a.tau; j += blockDim.x)
      atomicAdd(&Ms[j * a.tau + j], a.lambda * (double)(boff[j + 1] - boff[j]));
  }
}

// ---------------------------------------------------------------------------
// Phase 2, one iteration
// ---------------------------------------------------------------------------
// delta = P S^T r (P = M^+, tau x pld); r_S is formed in every block from the plan
template <typename TF>
__global__ void __launch_bounds__(256) k_mf_delta(Ctrl* __restrict__ ctrl, PlanView plan,
                                                  const double* __restrict__ r,
                                                  const TF* __restrict__ P, int64_t pld,
                                                  int64_t p_slot, int64_t tau,
                                                  double* __restrict__ delta,
                                                  double* __restrict__ rS_out) {
  if (halted(ctrl)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TF* rs = reinterpret_cast<TF*>(smem_raw);
  const int64_t slot = ctrl->k - ctrl->k0;
  const int32_t* perm = plan.perm + slot * plan.perm_stride;
  const int32_t* boff = plan.boff + slot * plan.boff_stride;
  for (int64_t j = threadIdx.x; j < tau; j += blockDim.x) {
    double acc = 0.0;
    for (int32_t t = boff[j]; t < boff[j + 1]; ++t) {
      const int32_t e = perm[t];
      const double v = r[entry_row(e)];
      acc = sadd(acc, v, entry_neg(e));
    }
    rs[j] = (TF)acc;
    if (blockIdx.x == 0 && rS_out != nullptr) rS_out[j] = acc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const TF* Ps = P + slot * p_slot;
  for (int64_t j = blockIdx.x * 8 + (threadIdx.x >> 5); j < tau; j += (int64_t)gridDim.x * 8) {
    TF acc = TF(0);
    for (int64_t l = lane; l < tau; l += 32) acc += Ps[j * pld + l] * rs[l];
    acc = warp_sum(acc);
    if (lane == 0) delta[j] = (double)acc;
  }
}

// v[row_t] = sum over the compact row t of (sigma x)_e delta[bucket_e]
template <typename AT>
__global__ void k_mf_v(const Ctrl* __restrict__ ctrl, MfArgs a, const AT* __restrict__ eval,
                       const double* __restrict__ delta, AT* __restrict__ v) {
  if (halted(ctrl)) return;
  const int64_t s = ctrl->k - ctrl->k0;
  const int32_t R = a.tot[s * 2 + 1];
  const int32_t* crow = a.crow + s * a.rcap;
  const int32_t* cptr = a.cptr + s * (a.rcap + 1);
  const int32_t* eb = a.ebuck + s * a.ecap;
  const AT* ev = eval + s * a.ecap;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < R;
       t += (int64_t)gridDim.x * blockDim.x) {
    AT acc = AT(0);
    for (int32_t e = cptr[t]; e < cptr[t + 1]; ++e) acc += ev[e] * (AT)delta[eb[e]];
    v[crow[t]] = acc;
  }
}

// A S delta = X^T v + lambda S delta (X^T v from the column pieces, in order), the
// momentum step of eq. (53) on w and r, ||r^{k+1}||^2 and the stopping test by the
// last block; v is cleared on the slot's rows for the next iteration
template <typename AT>
__global__ void __launch_bounds__(256) k_mf_update(Ctrl* __restrict__ ctrl, MfArgs a,
                                                   const int32_t* __restrict__ cpiece,
                                                   const AT* __restrict__ pu,
                                                   AT* __restrict__ v, UpdateArgs u) {
  if (halted(ctrl)) return;
  const int64_t k = ctrl->k;
  const int64_t s = k - ctrl->k0;
  const int32_t* inv = a.inv + s * a.inv_slot;
  const double g = u.gam[k], b = u.bet[k];
  double sq = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.d;
       c += (int64_t)gridDim.x * blockDim.x) {
    AT xs = AT(0);
    for (int32_t i = cpiece[c]; i < cpiece[c + 1]; ++i) xs += pu[i];
    const int32_t e = inv[c];
    const double sd = (e == kNotSketched) ? 0.0
                      : (entry_neg(e) ? -u.delta[e & 0x7FFFFFFF] : u.delta[e & 0x7FFFFFFF]);
    const double asd = (double)xs + a.lambda * sd;
    const double wi = u.w[c], wpi = u.wp[c], ri = u.r[c], rpi = u.rp[c];
    const double rn = (1.0 + b) * ri - b * rpi - g * asd;
    u.wp[c] = wi;
    u.w[c] = (1.0 + b) * wi - b * wpi - g * sd;
    u.rp[c] = ri;
    u.r[c] = rn;
    sq += rn * rn;
  }
  {
    const int32_t R = a.tot[s * 2 + 1];
    const int32_t* crow = a.crow + s * a.rcap;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < R;
         t += (int64_t)gridDim.x * blockDim.x)
      v[crow[t]] = AT(0);
  }
  __shared__ double s_part[8];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  sq = warp_sum(sq);
  if (lane == 0) s_part[w] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += s_part[q];
    u.partials[blockIdx.x] = t;
  }
  // last block to finish sums the partials in block order (deterministic)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int64_t q = 0; q < gridDim.x; ++q) tot += *((volatile double*)&u.partials[q]);
    const double rel = sqrt(tot) / ctrl->r0;
    u.hist[k + 1] = rel;
    const int64_t kn = k + 1;
    ctrl->k = kn;
    ctrl->ticket = 0u;
    if (!isfinite(rel)) {
      ctrl->status = 4;  // RS_ENUMERIC
      ctrl->stop = 1;
    } else if (!ctrl->no_stop && rel <= ctrl->tol) {
      if (u.mixed) ctrl->pending = 1; else ctrl->stop = 1;
    }
    if (kn >= ctrl->max_iters) ctrl->stop = 1;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int64_t mf_row_blocks(int64_t n) { return (n + kMfBlock - 1) / kMfBlock; }

// *err = 1 unless rowptr[0] = 0, rowptr is non-decreasing, rowptr[n] = nnz and every
// column index lies in [0, d) (every read below stays inside the given arrays)
__global__ void k_csr_check(const int64_t* __restrict__ rowptr, int64_t n,
                            const int32_t* __restrict__ colidx, int64_t nnz, int64_t d,
                            int32_t* __restrict__ err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  if (t == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) atomicExch(err, 1);
  for (int64_t r = t; r < n; r += nt)
    if (rowptr[r + 1] < rowptr[r]) atomicExch(err, 1);
  for (int64_t e = t; e < nnz; e += nt)
    if (colidx[e] < 0 || (int64_t)colidx[e] >= d) atomicExch(err, 1);
}

cudaError_t launch_csr_check(cudaStream_t st, const int64_t* rowptr, int64_t n,
                             const int32_t* colidx, int64_t nnz, int64_t d, int32_t* err) {
  k_csr_check<<<304, 256, 0, st>>>(rowptr, n, colidx, nnz, d, err);
  return cudaGetLastError();
}

template <typename VT, typename AT>
cudaError_t launch_mf_phase1(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, MfArgs a,
                             const VT* val, AT* eval, PlanView plan, double* M, int64_t m_slot) {
  cudaError_t e = cudaMemsetAsync(M, 0, (size_t)nslots * m_slot * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)a.nrb, (unsigned)nslots);
  k_mf_count<<<grid, 1024, 0, st>>>(ctrl, force, nslots, a);
  k_mf_bscan<<<nslots, 32, 0, st>>>(ctrl, force, nslots, a);
  k_mf_fill<VT, AT><<<grid, 1024, 0, st>>>(ctrl, force, nslots, a, val, eval);
  const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.rcap + 255) / 256, 64));
  k_mf_gram<AT><<<dim3(gg, (unsigned)nslots), 256, 0, st>>>(ctrl, force, nslots, a, eval, plan, M,
                                                           m_slot);
  return cudaGetLastError();
}

template <typename VT, typename AT>
cudaError_t launch_mf_iteration(cudaStream_t st, Ctrl* ctrl, MfArgs a, const SparseX<VT>& X,
                                const AT* eval, PlanView plan, const AT* P, int64_t pld,
                                int64_t p_slot, AT* v, AT* pu, UpdateArgs u, double* rS_out) {
  const size_t smem = (size_t)a.tau * sizeof(AT);
  const unsigned gdel = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.tau + 7) / 8, 152));
  k_mf_delta<AT><<<gdel, 256, smem, st>>>(ctrl, plan, u.r, P, pld, p_slot, a.tau,
                                          const_cast<double*>(u.delta), rS_out);
  const unsigned gv = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.rcap + 255) / 256, 152 * 8));
  k_mf_v<AT><<<gv, 256, 0, st>>>(ctrl, a, eval, u.delta, v);
  const int64_t bp = std::min<int64_t>((X.npieces + 7) / 8, 152 * 16);
  k_csc_pieces<VT, AT><<<(unsigned)std::max<int64_t>(bp, 1), 256, 0, st>>>(
      X.colptr, X.rowidx, X.cval, X.pcol, X.pstart, X.npieces, v, pu, nullptr, ctrl);
  const unsigned gu = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.d + 255) / 256, 256));
  k_mf_update<AT><<<gu, 256, 0, st>>>(ctrl, a, X.cpiece, pu, v, u);
  return cudaGetLastError();
}

#define RS_SPARSE_INST(VT)                                                                    \
  template cudaError_t build_csc<VT>(cudaStream_t, const int64_t*, int64_t, const int32_t*,  \
                                     const VT*, int64_t, int64_t, int32_t*, int, int64_t*,    \
                                     int64_t*, int32_t*, VT*);                                \
  template cudaError_t sparse_xtv_d<VT>(cudaStream_t, const SparseX<VT>&, const double*,     \
                                        double*, double*, const int32_t*);                   \
  template cudaError_t sparse_xv_d<VT>(cudaStream_t, const SparseX<VT>&, const double*,      \
                                       double*, const int32_t*);                             \
  template cudaError_t launch_mf_phase1<VT, float>(cudaStream_t, const Ctrl*, int, int, MfArgs, \
                                                   const VT*, float*, PlanView, double*, int64_t); \
  template cudaError_t launch_mf_phase1<VT, double>(cudaStream_t, const Ctrl*, int, int, MfArgs, \
                                                    const VT*, double*, PlanView, double*,       \
                                                    int64_t);                                    \
  template cudaError_t launch_mf_iteration<VT, float>(cudaStream_t, Ctrl*, MfArgs,              \
                                                      const SparseX<VT>&, const float*,         \
                                                      PlanView, const float*, int64_t, int64_t, \
                                                      float*, float*, UpdateArgs, double*);     \
  template cudaError_t launch_mf_iteration<VT, double>(cudaStream_t, Ctrl*, MfArgs,             \
                                                       const SparseX<VT>&, const double*,       \
                                                       PlanView, const double*, int64_t,        \
                                                       int64_t, double*, double*, UpdateArgs,   \
                                                       double*);
RS_SPARSE_INST(float)
RS_SPARSE_INST(double)
RS_SPARSE_INST(__nv_bfloat16)
#undef RS_SPARSE_INST

}  // namespace rs
