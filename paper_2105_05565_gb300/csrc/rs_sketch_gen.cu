// Sketch generation (Section 4): ordered samples, count buckets, signs, Gaussian
// entries. The draws follow the counter-based definition in rs_common.cuh, so a
// sketch depends only on (seed, k) and can be generated ahead of the iteration
// that uses it: one launch fills a chunk of consecutive iterations ("slots").
#include "rs_kernels.cuh"

namespace rs {

// ---------------------------------------------------------------------------
// Ordered sample without replacement of `cnt` lanes of [0, n): the lanes with the
// smallest keys draw(key, 0, i), by increasing (key, i). One CTA per slot.
//   mode 0: subsample  -> perm[p] = C_p,               boff[j] = j
//   mode 1: subcount   -> perm[p] = C_p | sign(p),     boff[j] = j * kk
//   mode 2: srht       -> perm[p] = C_p (C_p < n = m'), no boff
// Shared memory: cap * (8 + 4) bytes, cap a power of two >= 2 cnt + 64.
// ---------------------------------------------------------------------------
__global__ void k_gen_sample(const Ctrl* __restrict__ ctrl, int64_t k0_arg, uint64_t seed,
                             int64_t n, int64_t cnt, int32_t cap, int mode, int64_t kk,
                             int64_t tau, int32_t* __restrict__ perm, int64_t perm_stride,
                             int32_t* __restrict__ boff, int64_t boff_stride,
                             int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem_raw);
  int32_t* sidx = reinterpret_cast<int32_t*>(skey + cap);
  __shared__ unsigned long long s_count;
  __shared__ int32_t s_ok;
  __shared__ uint64_t s_T;

  const int64_t k0 = k0_arg >= 0 ? k0_arg : ctrl->k;
  const int64_t k = k0 + blockIdx.x;
  if (k0_arg < 0 && (stopped(ctrl) || k >= ctrl->max_iters)) return;
  const uint64_t key = iter_key(seed, k);
  int32_t* out = perm + (int64_t)blockIdx.x * perm_stride;

  // threshold search: find T with cnt <= #{key_i < T} <= cap
  double c_lo = 0.0, c_hi = -1.0;
  double c_try = (double)cnt + 4.0 * sqrt((double)cnt) + 32.0;
  uint64_t T = ~0ull;
  bool take_all = (n <= cap);
  int it = 0;
  for (; !take_all && it < 80; ++it) {
    const double frac = c_try / (double)n;
    T = frac >= 1.0 ? ~0ull : (uint64_t)(frac * 18446744073709551616.0);
    if (threadIdx.x == 0) s_count = 0ull;
    __syncthreads();
    unsigned long long local = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) local += (draw_k(key, 0, i) < T);
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_count, local);
    __syncthreads();
    const unsigned long long c = s_count;
    __syncthreads();
    if (c >= (unsigned long long)cnt && c <= (unsigned long long)cap) break;
    if (c < (unsigned long long)cnt) {
      c_lo = c_try;
      c_try = (c_hi < 0.0) ? 2.0 * c_try : 0.5 * (c_lo + c_hi);
    } else {
      c_hi = c_try;
      c_try = 0.5 * (c_lo + c_hi);
    }
  }
  if (!take_all && it >= 80) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  if (take_all) T = ~0ull;
  // collect (key, lane) pairs below T; with take_all every lane (keys equal to
  // ~0ull are kept as well since the comparison is skipped)
  if (threadIdx.x == 0) s_count = 0ull;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t kv = draw_k(key, 0, i);
    if (take_all || kv < T) {
      const unsigned long long pos = atomicAdd(&s_count, 1ull);
      skey[pos] = kv;
      sidx[pos] = (int32_t)i;
    }
  }
  __syncthreads();
  const int32_t have = (int32_t)s_count;
  int32_t len = 1;
  while (len < have) len <<= 1;
  for (int32_t i = have + threadIdx.x; i < len; i += blockDim.x) {
    skey[i] = ~0ull;
    sidx[i] = 0x7FFFFFFF;
  }
  __syncthreads();
  // bitonic sort of (key, lane) ascending
  for (int32_t size = 2; size <= len; size <<= 1) {
    for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int32_t t = threadIdx.x; t < (len >> 1); t += blockDim.x) {
        const int32_t lo = 2 * t - (t & (stride - 1));
        const int32_t hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const uint64_t ka = skey[lo], kb = skey[hi];
        const int32_t ia = sidx[lo], ib = sidx[hi];
        const bool gt = (ka > kb) || (ka == kb && ia > ib);
        if (gt == up) {
          skey[lo] = kb; skey[hi] = ka;
          sidx[lo] = ib; sidx[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
  for (int64_t p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int32_t row = sidx[p];
    bool neg = false;
    if (mode == 1) neg = draw_neg(draw_k(key, 1, (uint64_t)p));
    out[p] = pack_entry(row, neg);
  }
  if (boff != nullptr) {
    int32_t* bo = boff + (int64_t)blockIdx.x * boff_stride;
    for (int64_t j = threadIdx.x; j <= tau; j += blockDim.x)
      bo[j] = (int32_t)(mode == 1 ? j * kk : j);
  }
  (void)s_ok; (void)s_T;
}

// ---------------------------------------------------------------------------
// Count sketch (Section 4.2): every row i in [m] has bucket h(i) and sign from
// draw(key, 1, i). Output per slot: perm = rows sorted by (bucket, row) with the
// sign in bit 31, boff[b] = start of bucket b (boff[tau] = m). Stable counting
// sort in one CTA (1024 threads). Shared memory: (2 tau + 32 tau/2) ints.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_gen_count(const Ctrl* __restrict__ ctrl, int64_t k0_arg,
                                                    uint64_t seed, int64_t m, int64_t tau,
                                                    int32_t* __restrict__ perm, int64_t perm_stride,
                                                    int32_t* __restrict__ boff, int64_t boff_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t* cntb = reinterpret_cast<int32_t*>(smem_raw);         // tau
  int32_t* run = cntb + tau;                                     // tau
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(run + tau);      // 32 * tau
  __shared__ int32_t s_part[1024];

  const int64_t k0 = k0_arg >= 0 ? k0_arg : ctrl->k;
  const int64_t k = k0 + blockIdx.x;
  if (k0_arg < 0 && (stopped(ctrl) || k >= ctrl->max_iters)) return;
  const uint64_t key = iter_key(seed, k);
  int32_t* out = perm + (int64_t)blockIdx.x * perm_stride;
  int32_t* bo = boff + (int64_t)blockIdx.x * boff_stride;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (int64_t b = tid; b < tau; b += blockDim.x) cntb[b] = 0;
  for (int64_t t = tid; t < 32 * tau; t += blockDim.x) wcnt[t] = 0;
  __syncthreads();
  for (int64_t i = tid; i < m; i += blockDim.x) atomicAdd(&cntb[draw_bucket(draw_k(key, 1, i), tau)], 1);
  __syncthreads();
  // exclusive scan of cntb -> run (block-wide: each thread owns a contiguous range)
  const int64_t per = (tau + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = tid * per, b1 = (b0 + per < tau) ? b0 + per : tau;
  int32_t loc = 0;
  for (int64_t b = b0; b < b1; ++b) loc += cntb[b];
  s_part[tid] = loc;
  __syncthreads();
  if (wid == 0) {  // scan of 1024 partial sums by one warp (32 per lane)
    int32_t acc = 0;
    for (int j = 0; j < 32; ++j) acc += s_part[lane * 32 + j];
    int32_t incl = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int32_t base = incl - acc;
    for (int j = 0; j < 32; ++j) {
      const int32_t v = s_part[lane * 32 + j];
      s_part[lane * 32 + j] = base;
      base += v;
    }
  }
  __syncthreads();
  int32_t acc = s_part[tid];
  for (int64_t b = b0; b < b1; ++b) {
    run[b] = acc;
    bo[b] = acc;
    acc += cntb[b];
  }
  if (tid == 0) bo[tau] = (int32_t)m;
  __syncthreads();
  // stable placement, 1024 rows per round
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int64_t c0 = 0; c0 < m; c0 += blockDim.x) {
    const int64_t i = c0 + tid;
    const bool valid = i < m;
    uint64_t d = valid ? draw_k(key, 1, i) : 0ull;
    const int32_t b = valid ? draw_bucket(d, tau) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int intra = __popc(peers & lt_mask);
    if (valid && intra == 0) wcnt[wid * tau + b] = (uint16_t)__popc(peers);
    __syncthreads();
    if (valid) {
      int32_t pos = run[b] + intra;
      for (int w = 0; w < wid; ++w) pos += wcnt[w * tau + b];
      out[pos] = pack_entry((int32_t)i, draw_neg(d));
    }
    __syncthreads();
    for (int64_t bb = tid; bb < tau; bb += blockDim.x) {
      int32_t s = 0;
      for (int w = 0; w < 32; ++w) {
        s += wcnt[w * tau + bb];
        wcnt[w * tau + bb] = 0;
      }
      run[bb] += s;
    }
    __syncthreads();
  }
}

// Gaussian sketch entries (Box-Muller on draws of streams 2, 3), stored
// transposed per slot: ST_s[j * ld + i] = S_k[i, j] with lane i * tau + j, k = k0 + s.
template <typename T>
__global__ void k_gen_gauss(const Ctrl* __restrict__ ctrl, int force, int nslots, int64_t k0_arg,
                            uint64_t seed, int64_t m, int64_t tau, T* __restrict__ ST, int64_t ld,
                            int64_t st_slot) {
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t s = blockIdx.y;
  if (s >= nact) return;
  const int64_t k = (force ? k0_arg : ctrl->k0) + s;
  const uint64_t key = iter_key(seed, k);
  const int64_t total = m * tau;
  T* out = ST + s * st_slot;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < total;
       l += (int64_t)gridDim.x * blockDim.x) {
    const double u1 = ((double)(draw_k(key, 2, l) >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(draw_k(key, 3, l) >> 11) * 0x1.0p-53;
    const int64_t i = l / tau, j = l - i * tau;
    out[j * ld + i] = (T)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int sample_cap(int64_t n, int64_t cnt) {
  int64_t want = 2 * cnt + 64;
  if (n < want) want = n;
  int64_t cap = 64;
  while (cap < want) cap <<= 1;
  return (int)cap;
}

cudaError_t launch_gen_sample(cudaStream_t st, const Ctrl* ctrl, int64_t k0_arg, int nslots,
                              uint64_t seed, int64_t n, int64_t cnt, int mode, int64_t kk,
                              int64_t tau, int32_t* perm, int64_t perm_stride, int32_t* boff,
                              int64_t boff_stride, int32_t* err) {
  const int cap = sample_cap(n, cnt);
  const size_t smem = (size_t)cap * 12;
  cudaError_t e = set_smem_max((const void*)k_gen_sample, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_gen_sample<<<nslots, 1024, smem, st>>>(ctrl, k0_arg, seed, n, cnt, cap, mode, kk, tau, perm,
                                           perm_stride, boff, boff_stride, err);
  return cudaGetLastError();
}

cudaError_t launch_gen_count(cudaStream_t st, const Ctrl* ctrl, int64_t k0_arg, int nslots,
                             uint64_t seed, int64_t m, int64_t tau, int32_t* perm,
                             int64_t perm_stride, int32_t* boff, int64_t boff_stride) {
  const size_t smem = (size_t)tau * 8 + (size_t)tau * 32 * 2;
  cudaError_t e = set_smem_max((const void*)k_gen_count, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_gen_count<<<nslots, 1024, smem, st>>>(ctrl, k0_arg, seed, m, tau, perm, perm_stride, boff,
                                          boff_stride);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gen_gauss(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                             int64_t k0_arg, uint64_t seed, int64_t m, int64_t tau, T* ST,
                             int64_t ld, int64_t st_slot) {
  const int64_t total = m * tau;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  k_gen_gauss<T><<<dim3(blocks, nslots), 256, 0, st>>>(ctrl, force, nslots, k0_arg, seed, m, tau,
                                                        ST, ld, st_slot);
  return cudaGetLastError();
}
template cudaError_t launch_gen_gauss<double>(cudaStream_t, const Ctrl*, int, int, int64_t, uint64_t,
                                              int64_t, int64_t, double*, int64_t, int64_t);
template cudaError_t launch_gen_gauss<float>(cudaStream_t, const Ctrl*, int, int, int64_t, uint64_t,
                                             int64_t, int64_t, float*, int64_t, int64_t);

}  // namespace rs
