// Learned sketch proposal: per-coordinate features, the 4 -> 64 -> 64 -> 1 scoring
// network (bfloat16 weights and activations, FP32 accumulation), the eps-mixed
// softmax proposal and Gumbel-top-tau selection of the subsample sketch's rows;
// the network's gradient and Adam for training it on solver trajectories.
//
// The proposal is evaluated once per chunk, from the residual and the visit ages
// at the chunk's first iteration k0; iteration k0 + t of the chunk draws its own
// sample with the Gumbel noise of stream 4 of the counter-based generator:
//   z_j   = standardised (ln A_jj, ln(1 + |r_j| / rms(r)), ln ||A[:, j]||, ln(1 + age_j))
//   s_j   = w3 . relu(W2 relu(W1 z_j + b1) + b2) + b3
//   p_j   = (1 - eps) softmax(s)_j + eps / m
//   key_j = ln p_j - ln(-ln u_j),  u_j = (hi32(draw(seed, k, 4, j)) + 1/2) 2^-32
//   C_k   = the tau largest keys (ties: smaller index), rows in increasing order.
// Sorting the keys descending and keeping the first tau is a draw of tau rows
// without replacement from p (Gumbel-top-k).
#include <algorithm>

#include "rs_kernels.cuh"

namespace rs {

namespace {
constexpr int kH = 64;
constexpr int kNF = 4;
constexpr int kOffB1 = kH * kNF;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");

__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
// round to the nearest bfloat16 (ties to even) and back to FP32
__device__ __forceinline__ float round_bf16(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t r = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  return __uint_as_float(r);
}
__device__ __forceinline__ uint16_t to_bf16(float x) {
  return (uint16_t)(__float_as_uint(round_bf16(x)) >> 16);
}

// network weights in shared memory: all of them as FP32 (bfloat16 values), and W2
// again as bfloat16 bits, row-major W2[o][i], the B operand of the tensor-core layer
struct MlpSmem {
  float p[kMlpParams + 3];
  __align__(16) uint16_t w2h[kH * kH];
};

__device__ __forceinline__ void load_weights_bf16(MlpSmem& s, const uint16_t* w) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) s.p[i] = bf16_to_f(w[i]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) s.w2h[i] = w[kOffW2 + i];
}

// D (16 x 8, FP32) += A (16 x 16, bfloat16, row-major) B (16 x 8, bfloat16, column-major)
// on the tensor cores (warp-wide mma). Fragments, with g = lane / 4 and t = lane % 4:
// A: a[0] = (row g, cols 2t, 2t+1), a[1] = (row g+8, same), a[2] = (row g, cols 2t+8,
// 2t+9), a[3] = (row g+8, same); B: b[0] = (rows 2t, 2t+1, col g), b[1] = (rows 2t+8,
// 2t+9, col g); D: d[0..1] = (row g, cols 2t, 2t+1), d[2..3] = (row g+8, same). In a
// packed register the lower-indexed element sits in the low 16 bits.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)to_bf16(lo) | ((uint32_t)to_bf16(hi) << 16);
}
__device__ __forceinline__ uint32_t ld_b32(const uint16_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// layer 1 of the two rows (g, g + 8) of a warp's 16-row tile, as the A fragments of
// layer 2: h1 = bfloat16(relu(W1 z + b1)), fragment kc covers h1 columns 16 kc..16 kc+15
__device__ __forceinline__ void mlp_layer1_frag(const float* w, const float zg[kNF],
                                                const float zg8[kNF], uint32_t (&afr)[4][4]) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int o0 = 16 * kc + 8 * half + 2 * t;
      float h[2][2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int o = o0 + q;
        float a0 = w[kOffB1 + o], a1 = a0;
#pragma unroll
        for (int f = 0; f < kNF; ++f) {
          a0 = fmaf(w[o * kNF + f], zg[f], a0);
          a1 = fmaf(w[o * kNF + f], zg8[f], a1);
        }
        h[0][q] = fmaxf(a0, 0.f);
        h[1][q] = fmaxf(a1, 0.f);
      }
      afr[kc][2 * half] = pack_bf16(h[0][0], h[0][1]);
      afr[kc][2 * half + 1] = pack_bf16(h[1][0], h[1][1]);
    }
}

// scores of the warp's 16 rows: lane (g, t) returns those of rows g and g + 8 (the four
// lanes of a group agree). Layer 2 on the tensor cores (bfloat16 operands, FP32
// accumulation); h2 rounded to bfloat16; the output layer in FP32.
__device__ __forceinline__ void mlp_forward_warp(const MlpSmem& s, const float zg[kNF],
                                                 const float zg8[kNF], float& out_g,
                                                 float& out_g8) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t afr[4][4];
  mlp_layer1_frag(s.p, zg, zg8, afr);
  float og = 0.f, og8 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int o0 = 8 * nt + 2 * t;
    float c[4] = {s.p[kOffB2 + o0], s.p[kOffB2 + o0 + 1], s.p[kOffB2 + o0], s.p[kOffB2 + o0 + 1]};
    const uint16_t* wrow = s.w2h + (8 * nt + g) * kH;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const uint32_t b[2] = {ld_b32(wrow + 16 * kc + 2 * t), ld_b32(wrow + 16 * kc + 2 * t + 8)};
      mma_bf16(c, afr[kc], b);
    }
    const float w0 = s.p[kOffW3 + o0], w1 = s.p[kOffW3 + o0 + 1];
    og = fmaf(w0, round_bf16(fmaxf(c[0], 0.f)), fmaf(w1, round_bf16(fmaxf(c[1], 0.f)), og));
    og8 = fmaf(w0, round_bf16(fmaxf(c[2], 0.f)), fmaf(w1, round_bf16(fmaxf(c[3], 0.f)), og8));
  }
  og += __shfl_xor_sync(0xffffffffu, og, 1);
  og += __shfl_xor_sync(0xffffffffu, og, 2);
  og8 += __shfl_xor_sync(0xffffffffu, og8, 1);
  og8 += __shfl_xor_sync(0xffffffffu, og8, 2);
  out_g = og + s.p[kOffB3];
  out_g8 = og8 + s.p[kOffB3];
}

}  // namespace

// ---- static features: standardised ln A_jj and ln ||A[:, j]|| (A symmetric) ----
template <typename T>
__global__ void __launch_bounds__(256) k_lp_rownorm(const T* __restrict__ A, int64_t lda, int64_t m,
                                                    float* __restrict__ raw) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= m) return;
  double sq = 0.0;
  for (int64_t c = lane; c < m; c += 32) {
    const double v = (double)A[row * lda + c];
    sq += v * v;
  }
  sq = warp_sum(sq);
  if (lane == 0) {
    raw[row] = (float)log((double)A[row * lda + row]);
    raw[m + row] = (float)(0.5 * log(sq));
  }
}

// z = (x - mean) / (std + 1e-6) of `count` arrays of length m (one block each)
__global__ void __launch_bounds__(1024) k_lp_standardise(const float* __restrict__ raw, int64_t m,
                                                         float* __restrict__ z) {
  __shared__ double sh[32];
  const float* x = raw + (int64_t)blockIdx.x * m;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) s += x[j];
  const double mean = block_sum(s, sh) / (double)m;
  __syncthreads();
  double v = 0.0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    const double dd = x[j] - mean;
    v += dd * dd;
  }
  const double sd = sqrt(block_sum(v, sh) / (double)m);
  const double inv = 1.0 / (sd + 1e-6);
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x)
    z[(int64_t)blockIdx.x * m + j] = (float)((x[j] - mean) * inv);
}

template <typename T>
cudaError_t launch_lp_static(cudaStream_t st, const T* A, int64_t lda, int64_t m, float* raw,
                             float* zstat) {
  k_lp_rownorm<T><<<(unsigned)((m * 32 + 255) / 256), 256, 0, st>>>(A, lda, m, raw);
  k_lp_standardise<<<2, 1024, 0, st>>>(raw, m, zstat);
  return cudaGetLastError();
}

// ---- training data from a solver trajectory (rs_collect) ----
// Before iteration k: e2 = ||w_k - w*||_A^2 = (w_k - w*) . r_k (r_k = A w_k - b) and
// ||r_k||; the collection stops (ctrl->stop) once e2 <= 0 or ||r_k|| <= tol ||r_0||.
// One block; FP64 sums in a fixed order.
__global__ void __launch_bounds__(1024) k_collect_pre(Ctrl* __restrict__ ctrl,
                                                      const double* __restrict__ w,
                                                      const double* __restrict__ wstar,
                                                      const double* __restrict__ r, int64_t m,
                                                      double tol, double* __restrict__ e2_out) {
  __shared__ double s_red[32];
  if (stopped(ctrl)) return;
  double e2 = 0.0, n2 = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    e2 += (w[i] - wstar[i]) * r[i];
    n2 += r[i] * r[i];
  }
  e2 = block_sum(e2, s_red);
  n2 = block_sum(n2, s_red);
  if (threadIdx.x == 0) {
    *e2_out = e2;
    if (!(e2 > 0.0) || sqrt(n2) <= tol * ctrl->r0) ctrl->stop = 1;
    __threadfence();
  }
}

// The rows drawn at iteration k (bucket p of the slot-0 plan holds one row for the
// subsample sketch) with their chunk-start features and the targets
//   y_p = (1/2) ln(m max(a_p, 0) / e2 + 1e-3),   a_p = (r_C)_p delta_p,
// where r_C . delta is the exact decrease of ||w - w*||_A^2 of the step without
// momentum (the projection identity of Section 3). Appended at *count (one block).
__global__ void k_collect_rows(const Ctrl* __restrict__ ctrl, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ boff, int64_t tau,
                               const float* __restrict__ feat, const double* __restrict__ rS,
                               const double* __restrict__ delta, const double* __restrict__ e2p,
                               int64_t m, int64_t cap, float* __restrict__ Z,
                               float* __restrict__ y, int64_t* __restrict__ count) {
  if (stopped(ctrl)) return;
  const int64_t base = *count;
  const double e2 = *e2p;
  for (int64_t p = threadIdx.x; p < tau; p += blockDim.x) {
    if (base + p >= cap) continue;
    const int64_t row = entry_row(perm[boff[p]]);
#pragma unroll
    for (int f = 0; f < kNF; ++f) Z[(base + p) * kNF + f] = feat[row * kNF + f];
    const double a = rS[p] * delta[p];
    y[base + p] = (float)(0.5 * log((double)m * fmax(a, 0.0) / e2 + 1e-3));
  }
  __syncthreads();
  if (threadIdx.x == 0) *count = base + tau < cap ? base + tau : cap;
}

cudaError_t launch_collect_pre(cudaStream_t st, Ctrl* ctrl, const double* w, const double* wstar,
                               const double* r, int64_t m, double tol, double* e2_out) {
  k_collect_pre<<<1, 1024, 0, st>>>(ctrl, w, wstar, r, m, tol, e2_out);
  return cudaGetLastError();
}

cudaError_t launch_collect_rows(cudaStream_t st, const Ctrl* ctrl, const int32_t* perm,
                                const int32_t* boff, int64_t tau, const float* feat,
                                const double* rS, const double* delta, const double* e2,
                                int64_t m, int64_t cap, float* Z, float* y, int64_t* count) {
  k_collect_rows<<<1, 256, 0, st>>>(ctrl, perm, boff, tau, feat, rS, delta, e2, m, cap, Z, y,
                                    count);
  return cudaGetLastError();
}

// ---- importance sampling (Section 7): fixed scores s_j = ln A_jj, so that the
// proposal with eps = 0 is p_j = exp(s_j) / sum_l exp(s_l) = A_jj / trace(A) ----
template <typename T>
__global__ void k_lp_diag_score(const T* __restrict__ A, int64_t lda, int64_t m,
                                float* __restrict__ score) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) score[j] = (float)log((double)A[j * lda + j]);
}

template <typename T>
cudaError_t launch_lp_diag_score(cudaStream_t st, const T* A, int64_t lda, int64_t m,
                                 float* score) {
  k_lp_diag_score<T><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(A, lda, m, score);
  return cudaGetLastError();
}
template cudaError_t launch_lp_diag_score<float>(cudaStream_t, const float*, int64_t, int64_t,
                                                 float*);
template cudaError_t launch_lp_diag_score<double>(cudaStream_t, const double*, int64_t, int64_t,
                                                  float*);

// ---- per chunk: the dynamic features and their statistics (one block) ----
// dyn: x1_j = ln(1 + |r_j| / rms(r)) and x3_j = ln(1 + age_j), age_j = k0 - last_j,
// in FP32 (2 m floats); stats: 1 / rms(r), mean and 1 / (std + 1e-6) of x1 and x3
// (sums in FP64)
__global__ void __launch_bounds__(1024) k_lp_stats(const Ctrl* __restrict__ ctrl, int64_t k0_arg,
                                                   const double* __restrict__ r, int64_t m,
                                                   const int32_t* __restrict__ last,
                                                   float* __restrict__ dyn,
                                                   double* __restrict__ stats) {
  __shared__ double sh[32];
  const int64_t k0 = k0_arg >= 0 ? k0_arg : ctrl->k0;
  double q = 0.0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) q += r[j] * r[j];
  const double rms = sqrt(block_sum(q, sh) / (double)m);
  __syncthreads();
  const float ir = rms > 0.0 ? (float)(1.0 / rms) : 0.f;
  double s1 = 0.0, s3 = 0.0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    const float x1 = log1pf(fabsf((float)r[j]) * ir);
    const float x3 = log1pf((float)(k0 - last[j]));
    dyn[j] = x1;
    dyn[m + j] = x3;
    s1 += x1;
    s3 += x3;
  }
  const double m1 = block_sum(s1, sh) / (double)m;
  __syncthreads();
  const double m3 = block_sum(s3, sh) / (double)m;
  __syncthreads();
  double v1 = 0.0, v3 = 0.0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    const double a = (double)dyn[j] - m1;
    const double b = (double)dyn[m + j] - m3;
    v1 += a * a;
    v3 += b * b;
  }
  const double sd1 = sqrt(block_sum(v1, sh) / (double)m);
  __syncthreads();
  const double sd3 = sqrt(block_sum(v3, sh) / (double)m);
  if (threadIdx.x == 0) {
    stats[0] = ir;
    stats[1] = m1;
    stats[2] = 1.0 / (sd1 + 1e-6);
    stats[3] = m3;
    stats[4] = 1.0 / (sd3 + 1e-6);
  }
}

__device__ __forceinline__ void lp_feature_row(const float* zstat, const double* stats,
                                               const float* dyn, int64_t m, int64_t j,
                                               float z[kNF]) {
  z[0] = zstat[j];
  z[1] = (float)(((double)dyn[j] - stats[1]) * stats[2]);
  z[2] = zstat[m + j];
  z[3] = (float)(((double)dyn[m + j] - stats[3]) * stats[4]);
}

// ---- per chunk: scores s_j (uniform proposal: s = 0) ----
constexpr int kScoreRows = 128;  // rows of a 256-thread block: 8 warp tiles of 16

__global__ void __launch_bounds__(256) k_lp_score(const uint16_t* __restrict__ w, const float* zstat,
                                                  const double* stats, const float* __restrict__ dyn,
                                                  int64_t m, float* __restrict__ score,
                                                  float* feat_out) {
  __shared__ __align__(16) MlpSmem s;
  if (w != nullptr) load_weights_bf16(s, w);
  __syncthreads();
  // warp tiles of 16 rows: lane (g, t) holds rows g and g + 8 of its warp's tile
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t j0 = (int64_t)blockIdx.x * kScoreRows + (threadIdx.x >> 5) * 16;
  if (j0 >= m) return;  // whole warp (the tile's first row is past m)
  const int64_t jg = j0 + g, jg8 = jg + 8;
  float zg[kNF] = {0.f, 0.f, 0.f, 0.f}, zg8[kNF] = {0.f, 0.f, 0.f, 0.f};
  if (jg < m) lp_feature_row(zstat, stats, dyn, m, jg, zg);
  if (jg8 < m) lp_feature_row(zstat, stats, dyn, m, jg8, zg8);
  if (feat_out != nullptr && t == 0) {
#pragma unroll
    for (int i = 0; i < kNF; ++i) {
      if (jg < m) feat_out[jg * kNF + i] = zg[i];
      if (jg8 < m) feat_out[jg8 * kNF + i] = zg8[i];
    }
  }
  float sg = 0.f, sg8 = 0.f;
  if (w != nullptr) mlp_forward_warp(s, zg, zg8, sg, sg8);
  if (t == 0) {
    if (jg < m) score[jg] = sg;
    if (jg8 < m) score[jg8] = sg8;
  }
}

// ---- per slot: proposal, Gumbel keys, top tau (one block per slot) ----
// keys and row indices sorted in shared memory (bitonic, descending by key, ties by
// ascending row); the first tau rows are then sorted ascending into the plan
__global__ void __launch_bounds__(1024) k_lp_select(const Ctrl* __restrict__ ctrl, int force,
                                                    int nslots, int64_t k0_arg, uint64_t seed,
                                                    const float* __restrict__ score, int64_t m,
                                                    int64_t tau, float eps, int64_t npow2,
                                                    int32_t* __restrict__ perm, int64_t perm_stride,
                                                    int32_t* __restrict__ boff, int64_t boff_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* key = reinterpret_cast<float*>(smem_raw);
  int32_t* idx = reinterpret_cast<int32_t*>(key + npow2);
  __shared__ float s_red[32];
  __shared__ float s_bc[2];
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t t = blockIdx.x;
  if (t >= nact) return;
  const int64_t k = (k0_arg >= 0 ? k0_arg : ctrl->k0) + t;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  // softmax normaliser: max and sum of exp(s - max)
  float mx = -INFINITY;
  for (int64_t j = tid; j < m; j += blockDim.x) mx = fmaxf(mx, score[j]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[wid] = mx;
  __syncthreads();
  if (tid == 0) {
    float v = s_red[0];
    for (int i = 1; i < nw; ++i) v = fmaxf(v, s_red[i]);
    s_bc[0] = v;
  }
  __syncthreads();
  mx = s_bc[0];
  float se = 0.f;
  for (int64_t j = tid; j < m; j += blockDim.x) se += expf(score[j] - mx);
  se = warp_sum(se);
  __syncthreads();
  if (lane == 0) s_red[wid] = se;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
    for (int i = 0; i < nw; ++i) v += s_red[i];
    s_bc[1] = v;
  }
  __syncthreads();
  const float c1 = (1.f - eps) / s_bc[1], c0 = eps / (float)m;
  const uint64_t kk = iter_key(seed, k);
  for (int64_t j = tid; j < npow2; j += blockDim.x) {
    if (j < m) {
      const float lp = logf(c1 * expf(score[j] - mx) + c0);
      const uint32_t hi = (uint32_t)(draw_k(kk, 4, (uint64_t)j) >> 32);
      const float u = ((float)hi + 0.5f) * 2.3283064365386963e-10f;
      key[j] = lp - logf(-logf(u));
      idx[j] = (int32_t)j;
    } else {
      key[j] = -INFINITY;
      idx[j] = 0x7FFFFFFF;
    }
  }
  __syncthreads();
  // bitonic sort: "a before b" when key_a > key_b or (equal and idx_a < idx_b)
  for (int64_t size = 2; size <= npow2; size <<= 1) {
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t i = tid; i < npow2 / 2; i += blockDim.x) {
        const int64_t lo = 2 * i - (i & (stride - 1));
        const int64_t hi2 = lo + stride;
        const bool desc = ((lo & size) == 0);
        const float ka = key[lo], kb = key[hi2];
        const int32_t ia = idx[lo], ib = idx[hi2];
        const bool a_first = (ka > kb) || (ka == kb && ia < ib);
        if (a_first != desc) {
          key[lo] = kb; key[hi2] = ka;
          idx[lo] = ib; idx[hi2] = ia;
        }
      }
      __syncthreads();
    }
  }
  // the tau selected rows in increasing order (bitonic on tau padded to a power of two)
  int64_t tp = 1;
  while (tp < tau) tp <<= 1;
  int32_t* sel = reinterpret_cast<int32_t*>(key);  // keys no longer needed
  for (int64_t i = tid; i < tp; i += blockDim.x) sel[i] = i < tau ? idx[i] : 0x7FFFFFFF;
  __syncthreads();
  for (int64_t size = 2; size <= tp; size <<= 1) {
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t i = tid; i < tp / 2; i += blockDim.x) {
        const int64_t lo = 2 * i - (i & (stride - 1));
        const int64_t hi2 = lo + stride;
        const bool asc = ((lo & size) == 0);
        const int32_t a = sel[lo], b = sel[hi2];
        if ((a > b) == asc) { sel[lo] = b; sel[hi2] = a; }
      }
      __syncthreads();
    }
  }
  int32_t* ps = perm + t * perm_stride;
  int32_t* bs = boff + t * boff_stride;
  for (int64_t p = tid; p < tau; p += blockDim.x) ps[p] = sel[p];
  for (int64_t p = tid; p <= tau; p += blockDim.x) bs[p] = (int32_t)p;
}

// ---- after the plans: last visit of every drawn row ----
__global__ void k_lp_age(const Ctrl* __restrict__ ctrl, int force, int nslots, int64_t k0_arg,
                         const int32_t* __restrict__ perm, int64_t perm_stride, int64_t tau,
                         int32_t* __restrict__ last) {
  const int64_t nact = active_slots(ctrl, force, nslots);
  const int64_t k0 = k0_arg >= 0 ? k0_arg : ctrl->k0;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nact * tau) return;
  const int64_t t = e / tau, p = e - t * tau;
  atomicMax(last + entry_row(perm[t * perm_stride + p]), (int32_t)(k0 + t));
}

cudaError_t launch_lp_plans(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, int64_t k0_arg,
                            uint64_t seed, const uint16_t* w, float eps, const float* zstat,
                            float* dyn, double* stats, const double* r, int32_t* last, int64_t m,
                            int64_t tau, float* score, int32_t* perm, int64_t perm_stride,
                            int32_t* boff, int64_t boff_stride, bool update_age,
                            bool fixed_score) {
  int64_t npow2 = 1;
  while (npow2 < m) npow2 <<= 1;
  const size_t smem = (size_t)npow2 * 8;
  if (smem > 200 * 1024 || tau > m) return cudaErrorInvalidValue;
  if (!fixed_score) {  // the network's scores of this chunk's features
    k_lp_stats<<<1, 1024, 0, st>>>(ctrl, k0_arg, r, m, last, dyn, stats);
    k_lp_score<<<(unsigned)((m + kScoreRows - 1) / kScoreRows), 256, 0, st>>>(w, zstat, stats, dyn, m, score,
                                                            nullptr);
  }
  cudaError_t e = set_smem_max((const void*)k_lp_select, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_lp_select<<<(unsigned)nslots, 1024, smem, st>>>(ctrl, force, nslots, k0_arg, seed, score, m, tau,
                                                    eps, npow2, perm, perm_stride, boff, boff_stride);
  if (update_age)
    k_lp_age<<<(unsigned)((nslots * tau + 255) / 256), 256, 0, st>>>(ctrl, force, nslots, k0_arg,
                                                                      perm, perm_stride, tau, last);
  return cudaGetLastError();
}

cudaError_t launch_lp_features(cudaStream_t st, const Ctrl* ctrl, int64_t k0, const float* zstat,
                               float* dyn, double* stats, const double* r, const int32_t* last,
                               int64_t m, float* score, float* feat_out) {
  k_lp_stats<<<1, 1024, 0, st>>>(ctrl, k0, r, m, last, dyn, stats);
  k_lp_score<<<(unsigned)((m + kScoreRows - 1) / kScoreRows), 256, 0, st>>>(nullptr, zstat, stats, dyn, m, score,
                                                          feat_out);
  return cudaGetLastError();
}

// ---- network scores of given feature rows (inference / parity) ----
__global__ void __launch_bounds__(256) k_mlp_forward(const uint16_t* __restrict__ w,
                                                     const float* __restrict__ Z, int64_t n,
                                                     float* __restrict__ s_out) {
  __shared__ __align__(16) MlpSmem s;
  load_weights_bf16(s, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t i0 = (int64_t)blockIdx.x * kScoreRows + (threadIdx.x >> 5) * 16;
  if (i0 >= n) return;
  const int64_t ig = i0 + g, ig8 = ig + 8;
  float zg[kNF], zg8[kNF];
#pragma unroll
  for (int f = 0; f < kNF; ++f) {
    zg[f] = ig < n ? Z[ig * kNF + f] : 0.f;
    zg8[f] = ig8 < n ? Z[ig8 * kNF + f] : 0.f;
  }
  float sg, sg8;
  mlp_forward_warp(s, zg, zg8, sg, sg8);
  if (t == 0) {
    if (ig < n) s_out[ig] = sg;
    if (ig8 < n) s_out[ig8] = sg8;
  }
}

cudaError_t launch_mlp_forward(cudaStream_t st, const uint16_t* w, const float* Z, int64_t n,
                               float* s_out) {
  if (n <= 0) return cudaSuccess;
  k_mlp_forward<<<(unsigned)((n + kScoreRows - 1) / kScoreRows), 256, 0, st>>>(w, Z, n, s_out);
  return cudaGetLastError();
}

// ---- training: gradient of the mean loss (s - y)^2 / 2 over n rows ----
// A block takes kGB rows, a warp tile of 16 rows per warp. The forward as in the
// scores (layer 2 on the tensor cores: bfloat16 operands, FP32 accumulation;
// bfloat16-rounded activations); the backward: dL/da2 = ds w3 [a2 > 0], rounded to
// bfloat16 for the two 64 x 64 contractions, dL/dh1 = dL/da2 W2 (the C fragments of
// dL/da2 are the A fragments of that product) and the block's W2 gradient
// sum_r dL/da2[r, o] h1[r, i] (tensor cores over the rows, from transposed bfloat16
// copies in shared memory); the other parameters' gradients as FP32 sums over the
// block's rows in row order. Per-block sums go to part (blocks x kMlpParams) and are
// added in block order. The roundings pass gradients straight through.
namespace {
constexpr int kGB = 128;  // rows per block
constexpr int kGT = 256;  // threads per block: 8 warp tiles of 16 rows

struct GradSmem {
  float w[kMlpParams + 3];              // bfloat16-rounded weights as FP32
  __align__(16) uint16_t w2h[kH * kH];  // W2[o][i] as bfloat16 bits
  __align__(16) uint16_t w2th[kH * kH]; // W2^T[i][o]
  __align__(16) uint16_t d2t[kH][kGB];  // dL/da2 transposed [o][r], bfloat16
  __align__(16) uint16_t h1t[kH][kGB];  // h1 transposed [i][r], bfloat16
  float z[kNF][kGB];
  float h2[kH][kGB];
  float d2[kH][kGB];   // dL/da2 in FP32 (b2)
  float d1[kH][kGB];   // dL/da1 (W1, b1)
  float ds[kGB];
  float loss[kGB];
};

__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }
}  // namespace

__global__ void __launch_bounds__(kGT, 1) k_mlp_grad(const float* __restrict__ theta,
                                                     const float* __restrict__ Z,
                                                     const float* __restrict__ y, int64_t n,
                                                     float* __restrict__ part,
                                                     float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GradSmem& s = *reinterpret_cast<GradSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, g = lane >> 2, t = lane & 3;
  for (int i = tid; i < kMlpParams; i += kGT) s.w[i] = round_bf16(theta[i]);
  for (int i = tid; i < kH * kH; i += kGT) {
    const uint16_t h = to_bf16(theta[kOffW2 + i]);
    s.w2h[i] = h;
    s.w2th[(i % kH) * kH + i / kH] = h;
  }
  const int64_t base = (int64_t)blockIdx.x * kGB;
  const int rg = wid * 16 + g, rg8 = rg + 8;  // block-local rows of this lane
  const bool live_g = base + rg < n, live_g8 = base + rg8 < n;
  float zg[kNF], zg8[kNF];
#pragma unroll
  for (int f = 0; f < kNF; ++f) {
    zg[f] = live_g ? Z[(base + rg) * kNF + f] : 0.f;
    zg8[f] = live_g8 ? Z[(base + rg8) * kNF + f] : 0.f;
    if (t == 0) {
      s.z[f][rg] = zg[f];
      s.z[f][rg8] = zg8[f];
    }
  }
  __syncthreads();
  // forward: layer 1 as A fragments (also kept transposed for the W2 gradient)
  uint32_t afr[4][4];
  mlp_layer1_frag(s.w, zg, zg8, afr);
#pragma unroll
  for (int kc = 0; kc < 4; ++kc)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int o0 = 16 * kc + 8 * half + 2 * t;
      const uint32_t a = afr[kc][2 * half], b = afr[kc][2 * half + 1];
      s.h1t[o0][rg] = (uint16_t)(a & 0xFFFFu);
      s.h1t[o0 + 1][rg] = (uint16_t)(a >> 16);
      s.h1t[o0][rg8] = (uint16_t)(b & 0xFFFFu);
      s.h1t[o0 + 1][rg8] = (uint16_t)(b >> 16);
    }
  // layer 2 on the tensor cores
  float c2[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int o0 = 8 * nt + 2 * t;
    c2[nt][0] = s.w[kOffB2 + o0];
    c2[nt][1] = s.w[kOffB2 + o0 + 1];
    c2[nt][2] = c2[nt][0];
    c2[nt][3] = c2[nt][1];
    const uint16_t* wrow = s.w2h + (8 * nt + g) * kH;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const uint32_t b[2] = {ld_b32(wrow + 16 * kc + 2 * t), ld_b32(wrow + 16 * kc + 2 * t + 8)};
      mma_bf16(c2[nt], afr[kc], b);
    }
  }
  // output layer, loss, ds
  float og = 0.f, og8 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int o0 = 8 * nt + 2 * t;
    const float h[4] = {round_bf16(fmaxf(c2[nt][0], 0.f)), round_bf16(fmaxf(c2[nt][1], 0.f)),
                        round_bf16(fmaxf(c2[nt][2], 0.f)), round_bf16(fmaxf(c2[nt][3], 0.f))};
    s.h2[o0][rg] = h[0];
    s.h2[o0 + 1][rg] = h[1];
    s.h2[o0][rg8] = h[2];
    s.h2[o0 + 1][rg8] = h[3];
    og = fmaf(s.w[kOffW3 + o0], h[0], fmaf(s.w[kOffW3 + o0 + 1], h[1], og));
    og8 = fmaf(s.w[kOffW3 + o0], h[2], fmaf(s.w[kOffW3 + o0 + 1], h[3], og8));
  }
  og += __shfl_xor_sync(0xffffffffu, og, 1);
  og += __shfl_xor_sync(0xffffffffu, og, 2);
  og8 += __shfl_xor_sync(0xffffffffu, og8, 1);
  og8 += __shfl_xor_sync(0xffffffffu, og8, 2);
  const float err_g = live_g ? og + s.w[kOffB3] - y[base + rg] : 0.f;
  const float err_g8 = live_g8 ? og8 + s.w[kOffB3] - y[base + rg8] : 0.f;
  const float ds_g = err_g / (float)n, ds_g8 = err_g8 / (float)n;
  if (t == 0) {
    s.ds[rg] = ds_g;
    s.ds[rg8] = ds_g8;
    s.loss[rg] = 0.5f * err_g * err_g;
    s.loss[rg8] = 0.5f * err_g8 * err_g8;
  }
  // dL/da2 = ds w3 [a2 > 0]: FP32 for b2, bfloat16 for the products (A fragments)
  uint32_t dA[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int o0 = 8 * nt + 2 * t;
    const float w0 = s.w[kOffW3 + o0], w1 = s.w[kOffW3 + o0 + 1];
    const float d[4] = {c2[nt][0] > 0.f ? ds_g * w0 : 0.f, c2[nt][1] > 0.f ? ds_g * w1 : 0.f,
                        c2[nt][2] > 0.f ? ds_g8 * w0 : 0.f, c2[nt][3] > 0.f ? ds_g8 * w1 : 0.f};
    s.d2[o0][rg] = d[0];
    s.d2[o0 + 1][rg] = d[1];
    s.d2[o0][rg8] = d[2];
    s.d2[o0 + 1][rg8] = d[3];
    const uint32_t pg = pack_bf16(d[0], d[1]), pg8 = pack_bf16(d[2], d[3]);
    s.d2t[o0][rg] = (uint16_t)(pg & 0xFFFFu);
    s.d2t[o0 + 1][rg] = (uint16_t)(pg >> 16);
    s.d2t[o0][rg8] = (uint16_t)(pg8 & 0xFFFFu);
    s.d2t[o0 + 1][rg8] = (uint16_t)(pg8 >> 16);
    dA[nt >> 1][2 * (nt & 1)] = pg;
    dA[nt >> 1][2 * (nt & 1) + 1] = pg8;
  }
  // dL/dh1 = dL/da2 W2 (tensor cores), dL/da1 = dL/dh1 [h1 > 0]
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const uint16_t* wrow = s.w2th + (8 * nt + g) * kH;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const uint32_t b[2] = {ld_b32(wrow + 16 * kc + 2 * t), ld_b32(wrow + 16 * kc + 2 * t + 8)};
      mma_bf16(acc, dA[kc], b);
    }
    const int i0 = 8 * nt + 2 * t;
    const uint32_t hg = afr[nt >> 1][2 * (nt & 1)], hg8 = afr[nt >> 1][2 * (nt & 1) + 1];
    s.d1[i0][rg] = bf_lo(hg) > 0.f ? acc[0] : 0.f;
    s.d1[i0 + 1][rg] = bf_hi(hg) > 0.f ? acc[1] : 0.f;
    s.d1[i0][rg8] = bf_lo(hg8) > 0.f ? acc[2] : 0.f;
    s.d1[i0 + 1][rg8] = bf_hi(hg8) > 0.f ? acc[3] : 0.f;
  }
  __syncthreads();
  float* pb = part + (int64_t)blockIdx.x * kMlpParams;
  // W2 gradient: sum over the block's rows of dL/da2[r, o] h1[r, i] on the tensor cores;
  // warp w: o tile 16 (w / 2) .. + 15, i tiles 4 (w % 2) .. + 3 of 8
  {
    const int mt = wid >> 1, nt0 = (wid & 1) * 4;
    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
#pragma unroll
    for (int kc = 0; kc < kGB / 16; ++kc) {
      const int r0 = 16 * kc + 2 * t;
      const uint32_t a[4] = {ld_b32(&s.d2t[16 * mt + g][r0]), ld_b32(&s.d2t[16 * mt + g + 8][r0]),
                             ld_b32(&s.d2t[16 * mt + g][r0 + 8]),
                             ld_b32(&s.d2t[16 * mt + g + 8][r0 + 8])};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ii = 8 * (nt0 + q) + g;
        const uint32_t b[2] = {ld_b32(&s.h1t[ii][r0]), ld_b32(&s.h1t[ii][r0 + 8])};
        mma_bf16(acc[q], a, b);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i0 = 8 * (nt0 + q) + 2 * t, o = 16 * mt + g;
      pb[kOffW2 + o * kH + i0] = acc[q][0];
      pb[kOffW2 + o * kH + i0 + 1] = acc[q][1];
      pb[kOffW2 + (o + 8) * kH + i0] = acc[q][2];
      pb[kOffW2 + (o + 8) * kH + i0 + 1] = acc[q][3];
    }
  }
  // the other parameters' gradients (sums over the block's rows in row order)
  for (int e = tid; e < kMlpParams; e += kGT) {
    if (e >= kOffW2 && e < kOffB2) continue;  // W2: above
    float acc = 0.f;
    if (e < kOffB1) {                      // W1[o][i]
      const int o = e / kNF, i = e % kNF;
      for (int r = 0; r < kGB; ++r) acc = fmaf(s.d1[o][r], s.z[i][r], acc);
    } else if (e < kOffW2) {               // b1[o]
      const int o = e - kOffB1;
      for (int r = 0; r < kGB; ++r) acc += s.d1[o][r];
    } else if (e < kOffW3) {               // b2[o]
      const int o = e - kOffB2;
      for (int r = 0; r < kGB; ++r) acc += s.d2[o][r];
    } else if (e < kOffB3) {               // w3[o]
      const int o = e - kOffW3;
      for (int r = 0; r < kGB; ++r) acc = fmaf(s.ds[r], s.h2[o][r], acc);
    } else {                               // b3
      for (int r = 0; r < kGB; ++r) acc += s.ds[r];
    }
    pb[e] = acc;
  }
  if (tid == 0) {
    float l = 0.f;
    for (int r = 0; r < kGB; ++r) l += s.loss[r];
    loss_part[blockIdx.x] = l;
  }
}

// grad = sum of the block parts in block order; loss = their row-loss sums / n
__global__ void k_mlp_sum(const float* __restrict__ part, const float* __restrict__ loss_part,
                          int nblk, int64_t n, float* __restrict__ grad, double* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kMlpParams) {
    float acc = 0.f;
    for (int b = 0; b < nblk; ++b) acc += part[(int64_t)b * kMlpParams + e];
    grad[e] = acc;
  }
  if (e == 0 && loss != nullptr) {
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += loss_part[b];
    *loss = l / (double)n;
  }
}

int mlp_grad_blocks(int64_t n) { return (int)((n + kGB - 1) / kGB); }

cudaError_t launch_mlp_grad(cudaStream_t st, const float* theta, const float* Z, const float* y,
                            int64_t n, float* part, float* loss_part, float* grad, double* loss) {
  if (n <= 0) return cudaErrorInvalidValue;
  const int nblk = mlp_grad_blocks(n);
  const size_t smem = sizeof(GradSmem);
  cudaError_t e = set_smem_max((const void*)k_mlp_grad, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_mlp_grad<<<nblk, kGT, smem, st>>>(theta, Z, y, n, part, loss_part);
  k_mlp_sum<<<(kMlpParams + 255) / 256, 256, 0, st>>>(part, loss_part, nblk, n, grad, loss);
  return cudaGetLastError();
}

// ---- Adam (Kingma and Ba, 2015) on the FP32 master weights; bfloat16 copy ----
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ mom,
                           float* __restrict__ vel, const float* __restrict__ grad, float lr,
                           float b1, float b2, float eps, float c1, float c2,
                           uint16_t* __restrict__ w_bf16) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kMlpParams) return;
  const float g = grad[e];
  const float m = b1 * mom[e] + (1.f - b1) * g;
  const float v = b2 * vel[e] + (1.f - b2) * g * g;
  mom[e] = m;
  vel[e] = v;
  const float t = theta[e] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  theta[e] = t;
  if (w_bf16 != nullptr) w_bf16[e] = to_bf16(t);
}

cudaError_t launch_mlp_adam(cudaStream_t st, float* theta, float* mom, float* vel, const float* grad,
                            int64_t step, float lr, float b1, float b2, float eps, uint16_t* w_bf16) {
  const float c1 = (float)(1.0 - pow((double)b1, (double)step));
  const float c2 = (float)(1.0 - pow((double)b2, (double)step));
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(theta, mom, vel, grad, lr, b1, b2, eps, c1,
                                                       c2, w_bf16);
  return cudaGetLastError();
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = to_bf16(x[e]);
}

cudaError_t launch_f32_to_bf16(cudaStream_t st, const float* x, int64_t n, uint16_t* out) {
  k_f32_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, out);
  return cudaGetLastError();
}

template cudaError_t launch_lp_static<float>(cudaStream_t, const float*, int64_t, int64_t, float*,
                                             float*);
template cudaError_t launch_lp_static<double>(cudaStream_t, const double*, int64_t, int64_t,
                                              float*, float*);

}  // namespace rs
