// Shared device helpers of the ridge sketch-and-project library (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rs {

// ---------------------------------------------------------------------------
// Counter-based draws. Written from the SplitMix64 definition (Steele, Lea &
// Flood, OOPSLA 2014): output function mix64 and increment GAMMA.
//   key(seed, k)        = mix64(seed + (k+1) GAMMA)
//   draw(seed, k, s, i) = mix64(key(seed, k) + (1 + i + s 2^40) GAMMA)
// Streams: 0 sample keys, 1 sign + bucket, 2/3 Gaussian uniforms, 4 proposal.
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t iter_key(uint64_t seed, int64_t k) {
  return mix64(seed + (uint64_t)(k + 1) * kGamma);
}
__host__ __device__ __forceinline__ uint64_t draw_k(uint64_t key, uint32_t stream, uint64_t lane) {
  return mix64(key + (1ull + lane + ((uint64_t)stream << 40)) * kGamma);
}
// bucket in [0, tau): multiply-shift of the low 32 bits; sign from bit 63
__host__ __device__ __forceinline__ int32_t draw_bucket(uint64_t d, int64_t tau) {
  return (int32_t)(((d & 0xFFFFFFFFull) * (uint64_t)tau) >> 32);
}
__host__ __device__ __forceinline__ bool draw_neg(uint64_t d) { return (d >> 63) != 0; }

// packed sketch entry: row index in the low 31 bits, sign (1 = negative) in bit 31
__host__ __device__ __forceinline__ int32_t pack_entry(int32_t row, bool neg) {
  return (int32_t)((uint32_t)row | (neg ? 0x80000000u : 0u));
}
__host__ __device__ __forceinline__ int32_t entry_row(int32_t e) { return e & 0x7FFFFFFF; }
__host__ __device__ __forceinline__ bool entry_neg(int32_t e) { return e < 0; }
// acc + (neg ? -v : v) as one fused multiply-add by +-1: the product is exact, so the
// result is the correctly rounded sum or difference. A branch on the sign is
// predicated both ways and issues both adds.
template <typename T>
__device__ __forceinline__ T sadd(T acc, T v, bool neg) {
  return fma(v, neg ? T(-1) : T(1), acc);
}

// inverse map of a sketch plan: inv[i] = bucket | sign bit for rows in the sketch,
// kNotSketched otherwise
constexpr int32_t kNotSketched = 0x7FFFFFFF;

// ---------------------------------------------------------------------------
// Device control block of one context: iteration counter, stop flags, norms.
// ---------------------------------------------------------------------------
// device-side status codes of Ctrl::status (the values of RS_ENUMERIC, RS_ETIMEOUT)
constexpr int32_t kStatusNumeric = 4;
constexpr int32_t kStatusTimeout = 5;

struct Ctrl {
  int64_t k;          // next iteration index
  int64_t k0;         // first iteration of the current chunk
  int64_t max_iters;  // iteration cap of the current solve
  int32_t stop;       // 1: finished (converged, cap reached or error)
  int32_t pending;    // 1 (mixed): recursive residual <= tol, awaiting the FP64 check
  int32_t status;     // rs_status of the device side
  uint32_t ticket;    // last-block-done counter of reductions
  int32_t no_stop;    // 1: ignore tol (rs_step)
  int32_t pad;
  double r0;          // ||r^0|| = ||b||
  double tol;
  int64_t checked_k;  // last k whose FP64 true residual (a refresh) is hist[k]; -1: none
  // convergence forecast of the persistent paths: kcap > 0 ends the next chunk at the
  // iteration where the FP64 residual's decay reaches tol (with a margin), so that
  // phase 1 forms no slot past it. predict = 1 (mixed): set after each FP64 refresh,
  // from the decay since the previous one; predict = 2 (plain): set at each chunk's
  // start, from the decay of the recursive residual since the previous chunk's start.
  // pk, prel: iteration and relative residual of that previous point
  int64_t kcap;
  int64_t pk;
  double prel;
  int32_t predict;
  int32_t pad2;
};

__device__ __forceinline__ bool halted(const Ctrl* c) {
  return (*(volatile const int32_t*)&c->stop) | (*(volatile const int32_t*)&c->pending);
}

__device__ __forceinline__ bool stopped(const Ctrl* c) {
  return *(volatile const int32_t*)&c->stop;
}

// number of slots of the current chunk that run: all of them for a forced (probe)
// launch, none once the solve has stopped, else those below max_iters. Phase 1
// does not depend on the iterate, so a pending FP64 check (which may resume the
// solve) does not stop it: it may run beside that check.
__device__ __forceinline__ int64_t active_slots(const Ctrl* c, int force, int nslots) {
  if (force) return nslots;
  if (stopped(c)) return 0;
  int64_t left = c->max_iters - c->k0;
  if (c->kcap > 0 && c->kcap - c->k0 < left) left = c->kcap - c->k0;
  return left < 0 ? 0 : (left < nslots ? left : (int64_t)nslots);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed tree over warps); result valid in every thread.
template <typename T>
__device__ T block_sum(T v, T* sh /* >= 32 entries */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// In-place fast Walsh-Hadamard transform of length n (a power of two) in shared
// memory, Sylvester order (entry (i, c) of H is (-1)^popcount(i & c)). Called by
// every thread of the block.
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

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int ceil_div(int64_t x, int64_t a) { return (int)((x + a - 1) / a); }

}  // namespace rs
