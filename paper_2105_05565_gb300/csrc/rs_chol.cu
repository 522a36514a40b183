// The small SPD system of eq. (14): delta = (S^T A S)^dagger r_S.
//
// Phase 1 (k_factor_blk, batched over the slots of a chunk, one CTA per slot):
// blocked Cholesky factorisation M = L L^T, right-looking, with the pivot rule of the
// least-norm case: a pivot at most tau * eps * max_i M_ii drops its index j (row
// and column j of L become e_j). The triangular factor is then inverted in place
// (block row by block row) and the dropped rows and
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

#include "rs_gemm.cuh"
#include <algorithm>

#include "rs_kernels.cuh"

namespace rs {

__host__ __device__ __forceinline__ int64_t pk(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

// ---------------------------------------------------------------------------
// phase 1: blocked factor and inverse, one CTA (512 threads = 16 warps) per slot.
// The lower triangle is held as NB x NB tiles (row stride NB + 1, so that rows of
// a tile fall in distinct shared-memory banks); tile ops run one warp per tile,
// each lane accumulating an 8 x 4 block of the output in registers.
// ---------------------------------------------------------------------------
constexpr int NBK = 32;        // tile size
constexpr int TSK = NBK + 1;   // row stride of a tile
constexpr int TILE = NBK * TSK;

__host__ __device__ __forceinline__ int64_t ntiles_lower(int64_t P) { return P * (P + 1) / 2; }
// tiles of the lower triangle + one temporary tile per row block
__host__ __device__ size_t factor_ws_elems(int64_t tau) {
  const int64_t P = (tau + NBK - 1) / NBK;
  return (size_t)(ntiles_lower(P) + P) * TILE;
}

template <typename T>
__device__ __forceinline__ T* tile_at(T* base, int64_t I, int64_t J) {
  return base + (I * (I + 1) / 2 + J) * TILE;
}

// acc (8 rows x 4 cols of the lane) += SGN * A op(B), op(B) = B^T (TB) or B
template <typename T, bool TB, int SGN>
__device__ __forceinline__ void wtile_mma(T (&acc)[8][4], const T* __restrict__ A,
                                          const T* __restrict__ B, int ly, int lx) {
#pragma unroll 2
  for (int l = 0; l < NBK; ++l) {
    T a[8], b[4];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = A[(ly * 8 + r) * TSK + l];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = TB ? B[(lx * 4 + c) * TSK + l] : B[l * TSK + lx * 4 + c];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (SGN > 0) acc[r][c] += a[r] * b[c];
        else acc[r][c] -= a[r] * b[c];
      }
  }
}
template <typename T>
__device__ __forceinline__ void wtile_zero(T (&acc)[8][4]) {
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
}
template <typename T>
__device__ __forceinline__ void wtile_load(T (&acc)[8][4], const T* C, int ly, int lx) {
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = C[(ly * 8 + r) * TSK + lx * 4 + c];
}
template <typename T>
__device__ __forceinline__ void wtile_store(T* C, const T (&acc)[8][4], int ly, int lx) {
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) C[(ly * 8 + r) * TSK + lx * 4 + c] = acc[r][c];
}

template <typename T>
__global__ void __launch_bounds__(512) k_factor_blk(const Ctrl* __restrict__ ctrl, int force,
                                                     int nslots, const double* __restrict__ M,
                                                     int64_t m_slot, int64_t tau,
                                                     T* __restrict__ Linv, int64_t l_slot,
                                                     T* __restrict__ ws, int use_smem,
                                                     int32_t* __restrict__ ndropped) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t s = blockIdx.x;
  if (s >= active_slots(ctrl, force, nslots)) return;
  const int64_t P = (tau + NBK - 1) / NBK;
  const int64_t tp = P * NBK;
  unsigned char* dropped = smem_raw;  // tp flags (tau <= 4096)
  T* tiles = use_smem ? reinterpret_cast<T*>(smem_raw + 4096)
                      : ws + s * (int64_t)factor_ws_elems(tau);
  T* temps = tiles + ntiles_lower(P) * TILE;
  const double* Ms = M + s * m_slot;
  T* out = Linv + s * l_slot;
  __shared__ double s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int ly = lane >> 3, lx = lane & 7;
  const unsigned full = 0xffffffffu;

  // load the lower triangle into tiles (identity padding), max of the diagonal
  double dmax = 0.0;
  for (int64_t i = tid; i < tau; i += blockDim.x) dmax = fmax(dmax, Ms[i * tau + i]);
  for (int64_t i = tid; i < tp; i += blockDim.x) dropped[i] = 0;
  for (int64_t t = wid; t < ntiles_lower(P) * NBK; t += nw) {  // one tile row per warp step
    const int64_t tile = t / NBK, rr = t - tile * NBK;
    int64_t I = 0;
    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
    const int64_t J = tile - I * (I + 1) / 2;
    const int64_t R = I * NBK + rr, Cc = J * NBK + lane;
    double v = 0.0;
    if (R < tau && Cc < tau) v = Ms[R * tau + Cc];
    else if (R == Cc) v = 1.0;
    tiles[tile * TILE + rr * TSK + lane] = (T)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(full, dmax, o));
  if (lane == 0) s_red[wid] = dmax;
  __syncthreads();
  if (wid == 0) {
    double v = lane < nw ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(full, v, o));
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const T thr = (T)((double)tau * Eps<T>::v * s_red[0]);

  for (int64_t p = 0; p < P; ++p) {
    const int64_t c0 = p * NBK;
    T* D = tile_at(tiles, p, p);
    if (wid == 0) {
      // factor the diagonal tile: lane i holds row i
      T r[NBK];
#pragma unroll
      for (int j = 0; j < NBK; ++j) r[j] = D[lane * TSK + j];
#pragma unroll
      for (int kk = 0; kk < NBK; ++kk) {
        const T d = __shfl_sync(full, r[kk], kk);
        const bool dr = !(d > thr);
        const T piv = dr ? T(1) : (T)sqrt((double)d);
        const T inv = dr ? T(0) : T(1) / piv;
        if (lane == kk) {
          r[kk] = piv;
          if (dr) {
#pragma unroll
            for (int j = 0; j < kk; ++j) r[j] = T(0);
          }
        } else if (lane > kk) {
          r[kk] *= inv;
        }
#pragma unroll
        for (int j = kk + 1; j < NBK; ++j) {
          const T ljk = __shfl_sync(full, r[kk], j);
          if (lane >= j) r[j] -= r[kk] * ljk;
        }
        if (lane == 0) dropped[c0 + kk] = dr;
      }
      // store L_pp, then invert it: lane c holds column c of L_pp^{-1}
#pragma unroll
      for (int j = 0; j < NBK; ++j) D[lane * TSK + j] = (j <= lane) ? r[j] : T(0);
      __syncwarp();
      T x[NBK];
#pragma unroll
      for (int i = 0; i < NBK; ++i) {
        T acc = (i == lane) ? T(1) : T(0);
#pragma unroll
        for (int k = 0; k < i; ++k) acc -= D[i * TSK + k] * x[k];
        x[i] = (i < lane) ? T(0) : acc / D[i * TSK + i];
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < NBK; ++i) D[i * TSK + lane] = x[i];
    }
    __syncthreads();
    // a dropped index q becomes e_q in L: clear its row in the tiles left of the panel
    for (int64_t e = tid; e < p * NBK * NBK; e += blockDim.x) {
      const int64_t J = e / (NBK * NBK), rem = e - J * NBK * NBK;
      const int rr = (int)(rem / NBK), cc = (int)(rem - (rem / NBK) * NBK);
      if (dropped[c0 + rr]) tile_at(tiles, p, J)[rr * TSK + cc] = T(0);
    }
    // panel tiles below: L_Ip = M_Ip L_pp^{-T} (dropped columns stay zero)
    for (int64_t I = p + 1 + wid; I < P; I += nw) {
      T acc[8][4];
      wtile_zero(acc);
      T* C = tile_at(tiles, I, p);
      wtile_mma<T, true, 1>(acc, C, D, ly, lx);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (dropped[c0 + lx * 4 + c])
#pragma unroll
          for (int r = 0; r < 8; ++r) acc[r][c] = T(0);
      __syncwarp();
      wtile_store(C, acc, ly, lx);
    }
    __syncthreads();
    // trailing update M_IJ -= L_Ip L_Jp^T, p < J <= I
    const int64_t q = P - p - 1;
    for (int64_t t = wid; t < q * (q + 1) / 2; t += nw) {
      int64_t a = 0;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int64_t I = p + 1 + a, J = p + 1 + (t - a * (a + 1) / 2);
      T acc[8][4];
      T* C = tile_at(tiles, I, J);
      wtile_load(acc, C, ly, lx);
      wtile_mma<T, true, -1>(acc, tile_at(tiles, I, p), tile_at(tiles, J, p), ly, lx);
      wtile_store(C, acc, ly, lx);
    }
    __syncthreads();
  }
  // inverse of L, row block by row block, in place (diagonal tiles hold L_II^{-1}):
  // X_IJ = -L_II^{-1} sum_{K=J}^{I-1} L_IK X_KJ
  for (int64_t I = 1; I < P; ++I) {
    for (int64_t J = wid; J < I; J += nw) {
      T acc[8][4];
      wtile_zero(acc);
      for (int64_t K = J; K < I; ++K)
        wtile_mma<T, false, 1>(acc, tile_at(tiles, I, K), tile_at(tiles, K, J), ly, lx);
      T* tmp = temps + J * TILE;
      wtile_store(tmp, acc, ly, lx);
      __syncwarp();
      wtile_zero(acc);
      wtile_mma<T, false, -1>(acc, tile_at(tiles, I, I), tmp, ly, lx);
      __syncwarp();
      wtile_store(tmp, acc, ly, lx);
    }
    __syncthreads();
    for (int64_t e = tid; e < I * TILE; e += blockDim.x) {
      const int64_t J = e / TILE, off = e - J * TILE;
      tile_at(tiles, I, J)[off] = temps[J * TILE + off];
    }
    __syncthreads();
  }
  // write L^{-1} with the dropped rows and columns zeroed (tau x tau, zero above)
  for (int64_t i = wid; i < tau; i += nw) {
    const bool di = dropped[i];
    const int64_t I = i / NBK, rr = i - I * NBK;
    for (int64_t j = lane; j < tau; j += 32) {
      T v = T(0);
      if (j <= i && !di && !dropped[j]) {
        const int64_t J = j / NBK;
        v = tile_at(tiles, I, J)[rr * TSK + (j - J * NBK)];
      }
      out[i * tau + j] = v;
    }
  }
  if (tid == 0 && ndropped != nullptr) {
    int cnt = 0;
    for (int64_t i = 0; i < tau; ++i) cnt += dropped[i];
    if (cnt) atomicAdd(ndropped, cnt);
  }
}

template <typename T>
cudaError_t launch_factor_inv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                              const double* M, int64_t m_slot, int64_t tau, T* Linv, int64_t l_slot,
                              T* ws, int32_t* ndropped) {
  const size_t need = factor_ws_elems(tau) * sizeof(T) + 4096;
  const int use_smem = need <= 220 * 1024 && tau <= 4096;
  const size_t smem = use_smem ? need : 4096;
  if (!use_smem && ws == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = set_smem_max((const void*)k_factor_blk<T>, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  k_factor_blk<T><<<nslots, 512, smem, st>>>(ctrl, force, nslots, M, m_slot, tau, Linv, l_slot, ws,
                                              use_smem, ndropped);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// phase 1 for the persistent iteration kernel: P = M^+ = L^{-T} L^{-1} (eq. (14)),
// one CTA of kPotriThreads (four warps) per slot, four CTAs per SM.
//
// FP64 arithmetic runs at about one warp instruction per 64 cycles on each of an
// SM's four schedulers, so the factor is bound by how many schedulers have FP64
// work at every moment, not by memory: the tiles live in global memory (L1/L2), four
// slots share an SM (one warp of each per scheduler) so that one slot's narrow phases
// (a diagonal tile, the last trailing updates) overlap the others' wide ones, and a
// chunk of 600 slots runs in one wave on 152 SMs; every phase is cut into
// 32 x 32 tile tasks:
//   1. Cholesky, right-looking, with the least-norm pivot rule of k_factor_blk;
//      the diagonal tiles end up holding L_II^{-1};
//   2. X = L^{-1} right-looking over all block columns at once: round r first
//      finalises X_{J+r,J} = -X_{J+r,J+r} T_{J+r,J} for every J, then adds
//      L_{I,K} X_{K,J} (K = J + r) to the accumulators T_{I,J} of every I > K;
//      the critical path is 2 (P - 1) tile products instead of P (P + 1) / 2 - 1;
//   3. the dropped rows and columns of X are zeroed, then
//      P_{IJ} = sum_{K >= I} X_{KI}^T X_{KJ} for the lower tiles I >= J only
//      (a sixth of a full tau^3 product), each written with its transpose.
// ---------------------------------------------------------------------------
constexpr int kPotriThreads = 128;

// L (lower tiles incl. the diagonal) + the strictly lower tiles of X
__host__ __device__ size_t potri_ws_elems(int64_t tau) {
  const int64_t P = (tau + NBK - 1) / NBK;
  return (size_t)(ntiles_lower(P) + P * (P - 1) / 2) * TILE;
}
// the tiles stay in shared memory up to this size (tau <= 128 in FP64), else they
// live in a global work space of potri_ws_elems(tau) elements per slot
constexpr size_t kPotriSmemMax = 200 * 1024;
bool potri_needs_ws(int64_t tau, size_t elem) { return potri_ws_elems(tau) * elem > kPotriSmemMax; }

template <typename T>
__device__ __forceinline__ T* xtile_at(T* base, int64_t I, int64_t J) {  // I > J
  return base + ((I - 1) * I / 2 + J) * TILE;
}

// acc (8 x 4 of the lane) += SGN * op(A) op(B); op(A) = A^T (TA), op(B) = B^T (TB)
template <typename T, bool TA, bool TB, int SGN>
__device__ __forceinline__ void wtile_mma_g(T (&acc)[8][4], const T* __restrict__ A,
                                            const T* __restrict__ B, int ly, int lx) {
#pragma unroll 2
  for (int l = 0; l < NBK; ++l) {
    T a[8], b[4];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = TA ? A[l * TSK + ly * 8 + r] : A[(ly * 8 + r) * TSK + l];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = TB ? B[(lx * 4 + c) * TSK + l] : B[l * TSK + lx * 4 + c];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (SGN > 0) acc[r][c] += a[r] * b[c];
        else acc[r][c] -= a[r] * b[c];
      }
  }
}

// ---- tile products of k_potri on a mirrored lane mapping ----
// FP64 runs at one warp-wide DFMA per 64 cycles per scheduler here, so the small
// solve is bound by its count of DFMAs; loads, selects and moves go to other pipes.
// Several of its tile products have a triangular operand, whose zero half a plain
// 32 x 32 product multiplies too. Here lane (ly, lx) owns the rows p, 31 - p for
// p = ly + 4k (k < 4) and the columns b, 31 - b for b = lx, lx + 8: in a product
// whose column c needs the terms l <= c (or l >= c), the pair (b, 31 - b) needs 33
// terms in all, the same in every lane, so the loops below stay uniform across the
// warp and skip the zeros (528 DFMAs per lane instead of 1024). Each output sums its
// terms in ascending l, as the full product does.
__device__ __forceinline__ int prow_of(int ly, int i) {
  const int p = ly + 4 * (i >> 1);
  return (i & 1) ? NBK - 1 - p : p;
}
__device__ __forceinline__ int pcol_of(int lx, int j) {
  const int b = lx + 8 * (j >> 1);
  return (j & 1) ? NBK - 1 - b : b;
}
template <typename T, bool TA>
__device__ __forceinline__ T opa(const T* A, int r, int l) { return TA ? A[l * TSK + r] : A[r * TSK + l]; }
template <typename T, bool TB>
__device__ __forceinline__ T opb(const T* B, int l, int c) { return TB ? B[c * TSK + l] : B[l * TSK + c]; }

template <typename T>
__device__ __forceinline__ void ptile_zero(T (&acc)[8][4]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}
template <typename T>
__device__ __forceinline__ void ptile_load(T (&acc)[8][4], const T* C, int ly, int lx) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = C[prow_of(ly, i) * TSK + pcol_of(lx, j)];
}
template <typename T>
__device__ __forceinline__ void ptile_store(T* C, const T (&acc)[8][4], int ly, int lx) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) C[prow_of(ly, i) * TSK + pcol_of(lx, j)] = acc[i][j];
}

// acc += SGN op(A) op(B), full operands
template <typename T, bool TA, bool TB, int SGN>
__device__ __forceinline__ void ptile_mma(T (&acc)[8][4], const T* __restrict__ A,
                                          const T* __restrict__ B, int ly, int lx) {
#pragma unroll 1  // FP64-pipe bound: ILP comes from the other warps
  for (int l = 0; l < NBK; ++l) {
    T a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = opa<T, TA>(A, prow_of(ly, i), l);
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = opb<T, TB>(B, l, pcol_of(lx, j));
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(SGN > 0 ? a[i] : -a[i], b[j], acc[i][j]);
  }
}

// acc += SGN op(A) op(B) where op(B)[l][c] = 0 for l > c (UP) or for l < c (!UP):
// column c takes the terms l in [0, c] (UP) or [c, 31]
template <typename T, bool TA, bool TB, int SGN, bool UP>
__device__ __forceinline__ void ptile_mma_tri_b(T (&acc)[8][4], const T* __restrict__ A,
                                                const T* __restrict__ B, int ly, int lx) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int b = lx + 8 * q;  // columns b (j = 2q), then 31 - b (j = 2q + 1)
    const int n1 = UP ? b + 1 : NBK - b;  // terms of column b
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = acc[i][2 * q];
    int col = b;
#pragma unroll 1
    for (int t = 0; t < NBK + 1; ++t) {
      if (t == n1) {  // column b done: column 31 - b
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          acc[i][2 * q] = v[i];
          v[i] = acc[i][2 * q + 1];
        }
        col = NBK - 1 - b;
      }
      const int l = UP ? (t < n1 ? t : t - n1) : (t < n1 ? b + t : t - 1);
      const T bv = opb<T, TB>(B, l, col);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const T a = opa<T, TA>(A, prow_of(ly, i), l);
        v[i] = fma(SGN > 0 ? a : -a, bv, v[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][2 * q + 1] = v[i];
  }
}

// acc += SGN op(A) op(B) where op(A)[r][l] = 0 for l > r (LO) or for l < r (!LO):
// row r takes the terms l in [0, r] (LO) or [r, 31]
template <typename T, bool TA, bool TB, int SGN, bool LO>
__device__ __forceinline__ void ptile_mma_tri_a(T (&acc)[8][4], const T* __restrict__ A,
                                                const T* __restrict__ B, int ly, int lx) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int p = ly + 4 * k;  // rows p (i = 2k), then 31 - p (i = 2k + 1)
    const int n1 = LO ? p + 1 : NBK - p;  // terms of row p
    T v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = acc[2 * k][j];
    int row = p;
#pragma unroll 1
    for (int t = 0; t < NBK + 1; ++t) {
      if (t == n1) {  // row p done: row 31 - p
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[2 * k][j] = v[j];
          v[j] = acc[2 * k + 1][j];
        }
        row = NBK - 1 - p;
      }
      const int l = LO ? (t < n1 ? t : t - n1) : (t < n1 ? p + t : t - 1);
      const T a = opa<T, TA>(A, row, l);
      const T as = SGN > 0 ? a : -a;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = fma(as, opb<T, TB>(B, l, pcol_of(lx, j)), v[j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[2 * k + 1][j] = v[j];
  }
}

// Lower-triangle outputs (c <= r) of a diagonal tile, with 18 accumulators per lane:
// for each (k, q), p = ly + 4k and b = lx + 8q, the output (31 - p, b) (always below
// the diagonal) and (p, b) if b <= p, else (31 - p, 31 - b); the outputs (p, 31 - b)
// lie above it. A lane with b = p for two (k, q) (lx = ly or ly + 4) also owns the
// diagonal outputs (31 - p, 31 - p) of those two: 16 regular outputs per lane, two
// more in a quarter of the lanes, 18 DFMAs per term in every lane instead of 32.
// v[2 (2k + q)] is (31 - p, b), v[2 (2k + q) + 1] the second, v[16], v[17] the ties.
__device__ __forceinline__ bool syrk_low(int ly, int lx, int k, int q) {
  return lx + 8 * q <= ly + 4 * k;
}
__device__ __forceinline__ void syrk_pos(int ly, int lx, int v, int& r, int& c, bool& valid) {
  valid = true;
  if (v < 16) {
    const int k = v >> 2, q = (v >> 1) & 1;
    const int p = ly + 4 * k, b = lx + 8 * q;
    if ((v & 1) == 0) { r = NBK - 1 - p; c = b; }
    else if (b <= p) { r = p; c = b; }
    else { r = NBK - 1 - p; c = NBK - 1 - b; }
  } else {
    valid = (lx == ly) || (lx == ly + 4);
    const int kt = (lx == ly ? 0 : 1) + (v == 17 ? 2 : 0);
    r = c = NBK - 1 - (ly + 4 * kt);
  }
}
template <typename T>
__device__ __forceinline__ void syrk_load(T (&v)[18], const T* C, int ly, int lx) {
#pragma unroll
  for (int i = 0; i < 18; ++i) {
    int r, c;
    bool ok;
    syrk_pos(ly, lx, i, r, c, ok);
    v[i] = ok ? C[r * TSK + c] : T(0);
  }
}
template <typename T>
__device__ __forceinline__ void syrk_store(T* C, const T (&v)[18], int ly, int lx) {
#pragma unroll
  for (int i = 0; i < 18; ++i) {
    int r, c;
    bool ok;
    syrk_pos(ly, lx, i, r, c, ok);
    if (ok) C[r * TSK + c] = v[i];
  }
}
// v += SGN op(A) op(B) on the lower-triangle outputs of a diagonal tile
template <typename T, bool TA, bool TB, int SGN>
__device__ __forceinline__ void ptile_syrk_lower(T (&v)[18], const T* __restrict__ A,
                                                 const T* __restrict__ B, int ly, int lx) {
  bool low[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 2; ++q) low[k][q] = syrk_low(ly, lx, k, q);
  const bool t0 = (lx == ly);  // ties at (k, q) = (0, 0), (2, 1); else (1, 0), (3, 1)
#pragma unroll 1
  for (int l = 0; l < NBK; ++l) {
    T a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = opa<T, TA>(A, prow_of(ly, i), l);
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = opb<T, TB>(B, l, pcol_of(lx, j));
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int o = 2 * (2 * k + q);
        const T ra = low[k][q] ? a[2 * k] : a[2 * k + 1];
        const T cb = low[k][q] ? b[2 * q] : b[2 * q + 1];
        v[o] = fma(SGN > 0 ? a[2 * k + 1] : -a[2 * k + 1], b[2 * q], v[o]);
        v[o + 1] = fma(SGN > 0 ? ra : -ra, cb, v[o + 1]);
      }
    const T x16 = t0 ? a[1] : a[3], x17 = t0 ? a[5] : a[7];
    v[16] = fma(SGN > 0 ? x16 : -x16, b[1], v[16]);
    v[17] = fma(SGN > 0 ? x17 : -x17, b[3], v[17]);
  }
}

// Diagonal tile D of the blocked Cholesky by the calling warp: L_DD (an index whose
// pivot is not above thr is dropped: its row becomes e_q, drop[q] = 1), then L_DD^{-1}
// in its place.
template <typename T>
__device__ __forceinline__ void potri_diag(T* D, unsigned char* drop, T thr) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  T r[NBK];
#pragma unroll
  for (int j = 0; j < NBK; ++j) r[j] = D[lane * TSK + j];
#pragma unroll
  for (int kk = 0; kk < NBK; ++kk) {
    const T d = __shfl_sync(full, r[kk], kk);
    const bool dr = !(d > thr);
    const T piv = dr ? T(1) : (T)sqrt((double)d);
    const T inv = dr ? T(0) : T(1) / piv;
    if (lane == kk) {
      r[kk] = piv;
      if (dr) {
#pragma unroll
        for (int j = 0; j < kk; ++j) r[j] = T(0);
      }
    } else if (lane > kk) {
      r[kk] *= inv;
    }
#pragma unroll
    for (int j = kk + 1; j < NBK; ++j) {
      const T ljk = __shfl_sync(full, r[kk], j);
      if (lane >= j) r[j] -= r[kk] * ljk;
    }
    if (lane == 0) drop[kk] = dr;
  }
#pragma unroll
  for (int j = 0; j < NBK; ++j) D[lane * TSK + j] = (j <= lane) ? r[j] : T(0);
  __syncwarp();
  T x[NBK];  // lane c: column c of L_pp^{-1}
#pragma unroll
  for (int i = 0; i < NBK; ++i) {
    T acc = (i == lane) ? T(1) : T(0);
#pragma unroll
    for (int k = 0; k < i; ++k) acc -= D[i * TSK + k] * x[k];
    x[i] = (i < lane) ? T(0) : acc / D[i * TSK + i];
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < NBK; ++i) D[i * TSK + lane] = x[i];
}

// M^+ of one slot, by every thread of the CTA. T: arithmetic and L^{-1}; TP: the
// stored P (FP32 for an FP32 iteration kernel). Ms: the slot's tau x tau M; Ps: its
// P (row stride pld) or null; LinvS: its L^{-1} or null; tiles: potri_ws_elems(tau)
// elements of shared or global memory
template <typename T, typename TP>
__device__ __forceinline__ void potri_slot(const double* __restrict__ Ms, int64_t tau,
                                           T* __restrict__ LinvS, TP* __restrict__ Ps,
                                           int64_t pld, T* __restrict__ tiles,
                                           int32_t* __restrict__ ndropped) {
  __shared__ unsigned char dropped[4096];
  __shared__ double s_red[32];
  const int64_t P = (tau + NBK - 1) / NBK;
  const int64_t tp = P * NBK;
  T* xt = tiles + ntiles_lower(P) * TILE;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int ly = lane >> 3, lx = lane & 7;
  const unsigned full = 0xffffffffu;

  // load the lower triangle into tiles (identity padding), zero the X accumulators,
  // max of the diagonal
  double dmax = 0.0;
  for (int64_t i = tid; i < tau; i += blockDim.x) dmax = fmax(dmax, Ms[i * tau + i]);
  for (int64_t i = tid; i < tp; i += blockDim.x) dropped[i] = 0;
  for (int64_t t = wid; t < ntiles_lower(P) * NBK; t += nw) {  // one tile row per warp step
    const int64_t tile = t / NBK, rr = t - tile * NBK;
    int64_t I = 0;
    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
    const int64_t J = tile - I * (I + 1) / 2;
    const int64_t R = I * NBK + rr, Cc = J * NBK + lane;
    double v = 0.0;
    if (R < tau && Cc < tau) v = Ms[R * tau + Cc];
    else if (R == Cc) v = 1.0;
    tiles[tile * TILE + rr * TSK + lane] = (T)v;
  }
  for (int64_t e = tid; e < P * (P - 1) / 2 * TILE; e += blockDim.x) xt[e] = T(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(full, dmax, o));
  if (lane == 0) s_red[wid] = dmax;
  __syncthreads();
  if (wid == 0) {
    double v = lane < nw ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(full, v, o));
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const T thr = (T)((double)tau * Eps<T>::v * s_red[0]);

  // 1. Cholesky (diagonal tiles become L_II^{-1}, the others L_IJ). With eight or
  // more warps, look-ahead: warp 0 updates the next diagonal tile first in each
  // trailing phase and factors it at once, while the other warps update the other
  // tiles, so the single-warp factorisation overlaps them (same operations in the
  // same order per tile; one block barrier less per step). A slot of tau = 256 in
  // the 512-thread form: 3.25 against 3.37 ms; the rest of its critical path is in
  // the panels, the inverse and the product.
  const bool ahead = nw >= 8;
  // step -1 only factors tile 0; step p forms the panel p, updates the trailing
  // tiles and factors tile p + 1
  for (int64_t p = -1; p < P; ++p) {
    const int64_t c0 = p * NBK;
    if (p >= 0) {
      T* D = tile_at(tiles, p, p);
      // a dropped index q becomes e_q in L: clear its row in the tiles left of the panel
      for (int64_t e = tid; e < p * NBK * NBK; e += blockDim.x) {
        const int64_t J = e / (NBK * NBK), rem = e - J * NBK * NBK;
        const int rr = (int)(rem / NBK), cc = (int)(rem - (rem / NBK) * NBK);
        if (dropped[c0 + rr]) tile_at(tiles, p, J)[rr * TSK + cc] = T(0);
      }
      // panel tiles below: L_Ip = M_Ip L_pp^{-T} (dropped columns stay zero)
      for (int64_t I = p + 1 + wid; I < P; I += nw) {
        T acc[8][4];
        ptile_zero(acc);
        T* C = tile_at(tiles, I, p);
        // C L_pp^{-T}: column c of L_pp^{-T} is zero below row c
        ptile_mma_tri_b<T, false, true, 1, true>(acc, C, D, ly, lx);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (dropped[c0 + pcol_of(lx, c)])
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r][c] = T(0);
        __syncwarp();
        ptile_store(C, acc, ly, lx);
      }
      __syncthreads();
      // trailing update M_IJ -= L_Ip L_Jp^T, p < J <= I. Task 0 is the tile (p+1, p+1);
      // with look-ahead warp 0 takes only it and then factors that tile below, while
      // the other warps share the rest
      const int64_t q = P - p - 1;
      const int64_t ntask = q * (q + 1) / 2;
      const int64_t tstep = !ahead ? nw : (wid == 0 ? ntask + 1 : nw - 1);
      for (int64_t t = wid; t < ntask; t += tstep) {
        int64_t a = 0;
        while ((a + 1) * (a + 2) / 2 <= t) ++a;
        const int64_t I = p + 1 + a, J = p + 1 + (t - a * (a + 1) / 2);
        T* C = tile_at(tiles, I, J);
        if (I == J) {  // only the lower half of a diagonal tile is used
          T v[18];
          syrk_load(v, C, ly, lx);
          ptile_syrk_lower<T, false, true, -1>(v, tile_at(tiles, I, p), tile_at(tiles, I, p), ly, lx);
          syrk_store(C, v, ly, lx);
        } else {
          T acc[8][4];
          ptile_load(acc, C, ly, lx);
          ptile_mma<T, false, true, -1>(acc, tile_at(tiles, I, p), tile_at(tiles, J, p), ly, lx);
          ptile_store(C, acc, ly, lx);
        }
      }
      if (!ahead) __syncthreads();
    }
    if (wid == 0 && p + 1 < P) {
      __syncwarp();
      potri_diag<T>(tile_at(tiles, p + 1, p + 1), dropped + (p + 1) * NBK, thr);
    }
    __syncthreads();
  }
  // 2. X = L^{-1}: the diagonal tiles hold X_II; the strictly lower X_IJ are built in
  // xt, which holds the accumulators T_IJ = sum_{K < I} L_IK X_KJ until finalised
  for (int64_t r = 0; r + 1 < P; ++r) {
    if (r >= 1) {  // X_{J+r,J} = -X_{J+r,J+r} T_{J+r,J}
      for (int64_t J = wid; J + r < P; J += nw) {
        const int64_t I = J + r;
        T* X = xtile_at(xt, I, J);
        T acc[8][4];
        ptile_zero(acc);
        // X_II is lower triangular: row r takes the terms l <= r
        ptile_mma_tri_a<T, false, false, -1, true>(acc, tile_at(tiles, I, I), X, ly, lx);
        __syncwarp();
        ptile_store(X, acc, ly, lx);
      }
      __syncthreads();
    }
    // T_IJ += L_IK X_KJ with K = J + r final, for every I > K (tasks in column order)
    const int64_t ntask = (P - 1 - r) * (P - r) / 2;
    for (int64_t t = wid; t < ntask; t += nw) {
      int64_t J = 0, left = t;
      while (left >= P - 1 - J - r) { left -= P - 1 - J - r; ++J; }
      const int64_t K = J + r, I = K + 1 + left;
      T* X = xtile_at(xt, I, J);
      T acc[8][4];
      ptile_load(acc, X, ly, lx);
      if (r == 0)  // X_JJ is lower triangular: column c takes the terms l >= c
        ptile_mma_tri_b<T, false, false, 1, false>(acc, tile_at(tiles, I, K), tile_at(tiles, J, J),
                                                   ly, lx);
      else
        ptile_mma<T, false, false, 1>(acc, tile_at(tiles, I, K), xtile_at(xt, K, J), ly, lx);
      ptile_store(X, acc, ly, lx);
    }
    __syncthreads();
  }
  if (P >= 2) {  // the last round: X_{P-1,0}
    if (wid == 0) {
      T* X = xtile_at(xt, P - 1, 0);
      T acc[8][4];
      ptile_zero(acc);
      ptile_mma_tri_a<T, false, false, -1, true>(acc, tile_at(tiles, P - 1, P - 1), X, ly, lx);
      __syncwarp();
      ptile_store(X, acc, ly, lx);
    }
    __syncthreads();
  }
  // 3. zero the dropped (and padding) rows and columns of X
  for (int64_t e = tid; e < ntiles_lower(P) * NBK * NBK; e += blockDim.x) {
    const int64_t tile = e / (NBK * NBK), rem = e - tile * (NBK * NBK);
    int64_t I = 0;
    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
    const int64_t J = tile - I * (I + 1) / 2;
    const int rr = (int)(rem / NBK), cc = (int)(rem - (rem / NBK) * NBK);
    const int64_t i = I * NBK + rr, j = J * NBK + cc;
    if (i >= tau || j >= tau || dropped[i] || dropped[j])
      (I == J ? tile_at(tiles, I, I) : xtile_at(xt, I, J))[rr * TSK + cc] = T(0);
  }
  __syncthreads();
  // P_IJ = sum_{K >= I} X_KI^T X_KJ, I >= J; tasks in order of decreasing work
  if (Ps != nullptr) {
    for (int64_t t = wid; t < ntiles_lower(P); t += nw) {
      int64_t I = 0;
      while ((I + 1) * (I + 2) / 2 <= t) ++I;
      const int64_t J = t - I * (I + 1) / 2;
      if (I == J) {  // a diagonal tile of the symmetric P: its lower half, then mirrored
        T v[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) v[i] = T(0);
        for (int64_t K = I; K < P; ++K) {
          const T* XK = (K == I) ? tile_at(tiles, I, I) : xtile_at(xt, K, I);
          ptile_syrk_lower<T, true, false, 1>(v, XK, XK, ly, lx);
        }
#pragma unroll
        for (int e = 0; e < 18; ++e) {
          int r, c;
          bool ok;
          syrk_pos(ly, lx, e, r, c, ok);
          const int64_t i = I * NBK + r, l = I * NBK + c;
          if (ok && i < tau && l < tau) {
            Ps[i * pld + l] = (TP)v[e];
            if (i != l) Ps[l * pld + i] = (TP)v[e];
          }
        }
        continue;
      }
      T acc[8][4];
      ptile_zero(acc);
      // K = I: X_II^T is upper triangular, row r takes the terms l >= r
      ptile_mma_tri_a<T, true, false, 1, false>(acc, tile_at(tiles, I, I), xtile_at(xt, I, J),
                                                ly, lx);
      for (int64_t K = I + 1; K < P; ++K)
        ptile_mma<T, true, false, 1>(acc, xtile_at(xt, K, I), xtile_at(xt, K, J), ly, lx);
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int64_t i = I * NBK + prow_of(ly, r), l = J * NBK + pcol_of(lx, c);
          if (i < tau && l < tau) {
            Ps[i * pld + l] = (TP)acc[r][c];
            Ps[l * pld + i] = (TP)acc[r][c];
          }
        }
    }
  }
  // L^{-1} with the dropped rows and columns zeroed (tau x tau, zero above), if asked
  if (LinvS != nullptr) {
    T* out = LinvS;
    for (int64_t i = wid; i < tau; i += nw) {
      const int64_t I = i / NBK, rr = i - I * NBK;
      for (int64_t j = lane; j < tau; j += 32) {
        T v = T(0);
        if (j <= i) {
          const int64_t J = j / NBK;
          v = (I == J ? tile_at(tiles, I, I) : xtile_at(xt, I, J))[rr * TSK + (j - J * NBK)];
        }
        out[i * tau + j] = v;
      }
    }
  }
  if (tid == 0 && ndropped != nullptr) {
    int cnt = 0;
    for (int64_t i = 0; i < tau; ++i) cnt += dropped[i];
    if (cnt) atomicAdd(ndropped, cnt);
  }
}

// NT threads per slot. A chunk launches both forms; the active slot count (known on
// the device) picks one: above `few` (the SM count), four 128-thread CTAs per SM keep
// the FP64 pipes busy across slots; up to it, one 512-thread CTA per slot gives every
// scheduler four warps of that slot, so that the few slots of a chunk cut short by
// the convergence forecast take a fraction of one slot's single-warp latency.
template <typename T, typename TP, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_potri(
    const Ctrl* __restrict__ ctrl, int force, int nslots, const double* __restrict__ M,
    int64_t m_slot, int64_t tau, T* __restrict__ Linv, int64_t l_slot, TP* __restrict__ Pout,
    int64_t pld, int64_t p_slot, T* __restrict__ ws, int use_smem, int32_t* __restrict__ ndropped,
    int64_t few) {
  extern __shared__ __align__(16) unsigned char potri_smem[];
  const int64_t s = blockIdx.x;
  const int64_t nact = active_slots(ctrl, force, nslots);
  if ((NT == kPotriThreads) == (nact <= few)) return;  // the other form runs this chunk
  if (s >= nact) return;
  T* tiles = use_smem ? reinterpret_cast<T*>(potri_smem) : ws + s * (int64_t)potri_ws_elems(tau);
  potri_slot<T, TP>(M + s * m_slot, tau, Linv != nullptr ? Linv + s * l_slot : nullptr,
                    Pout != nullptr ? Pout + s * p_slot : nullptr, pld, tiles, ndropped);
}

// M^+ of the running problems of a batch in one launch: a grid of at most four CTAs
// per SM walks the (problem, slot) pairs, problem order[t] taking the pairs
// [t chunk, (t + 1) chunk), each CTA in its own tile work space of ws_elems elements
// (the problems come largest first, so the large systems start first)
template <typename T, typename TP>
__global__ void __launch_bounds__(kPotriThreads, 4) k_potri_batch(
    const PotriJob* __restrict__ jobs, const int32_t* __restrict__ order, int nrun, int chunk,
    T* __restrict__ ws, int64_t ws_elems) {
  const int64_t total = (int64_t)nrun * chunk;
  T* tiles = ws + (int64_t)blockIdx.x * ws_elems;
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int t = (int)(g / chunk), s = (int)(g - (int64_t)t * chunk);
    const PotriJob j = jobs[order[t]];
    if (s >= active_slots(j.ctrl, 0, chunk)) continue;  // uniform over the CTA
    potri_slot<T, TP>(j.M + s * j.m_slot, j.tau, nullptr,
                      j.P != nullptr ? static_cast<TP*>(j.P) + s * j.p_slot : nullptr, j.pld,
                      tiles, j.ndropped);
    __syncthreads();  // the tiles (and the drop flags) serve the next slot
  }
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
        acc = sadd(acc, v, entry_neg(e));
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
    cudaError_t e = set_smem_max((const void*)kern, (size_t)((int)smem));
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

// ---------------------------------------------------------------------------
// M^+ in FP32 by symmetric sweeps (Gauss-Jordan elimination without pivoting on a
// symmetric matrix, Goodnight 1979): sweeping index p maps
//   a_pp -> -1 / a_pp,  a_ip -> a_ip / a_pp,  a_il -> a_il - a_ip a_pl / a_pp  (i, l != p)
// and sweeping every index turns M into -M^{-1}. The pivot a_pp at the moment of
// its sweep is the Schur complement pivot of the Cholesky factorisation, so the drop
// rule is the factor's: a pivot at most tau * eps * max_i M_ii is not swept and its
// row and column are zeroed at the end, which gives the inverse of the kept
// principal submatrix, padded with zeros (the same least-norm reading as the
// factor kernel).
//
// Eight indices P are swept at once (a block sweep): with X = A[:, P] and
// Z = A_PP^+ (the 8 x 8 sweep of the diagonal block, drop rule included),
//   A_RR -> A_RR - X_R Z X_R^T,  A_RP -> X_R Z,  A_PP -> -Z,
// i.e. with Y = X Z one rank-8 update A_IJ -= X_I Y_J^T of every other block.
// The sweep runs on the unit-diagonal matrix M' = D^{-1/2} M D^{-1/2} (D = diag M),
// and M^+ = D^{-1/2} M'^+ D^{-1/2}.
//
// One CTA per slot; the lower triangle of 8 x 8 blocks lives in registers, one block
// per thread (tau = 256: 528 blocks, 17 warps; 96 registers keep 5 warps of one
// scheduler within its register file; all register indexing is static). The owner
// of the next diagonal block sweeps it (8 x 8, in registers) as soon as its last
// update is done, overlapping the other blocks' updates; X, Z and Y go through
// shared memory; two barriers per block of eight indices.
// ---------------------------------------------------------------------------
constexpr int kSwB = 8;         // register block edge = indices swept at once
constexpr int kSwMaxTau = 256;

__host__ __device__ inline int sweep_threads(int64_t tau) {
  const int nb = (int)((tau + kSwB - 1) / kSwB);
  return (nb * (nb + 1) / 2 + 31) / 32 * 32;
}

// Sweep of a diagonal 8 x 8 block held in registers (both triangles) by its owner
// thread, with the drop rule (pivot <= thrs[p], the threshold in the scaled matrix):
// a becomes -Z on the kept indices (0 on dropped rows and columns); Z goes to Zo.
__device__ __forceinline__ void diag_sweep(float (&a)[kSwB][kSwB], int Pb, const float* thrs,
                                           unsigned char* dropped, float (*Zo)[kSwB + 1]) {
  unsigned dmask = 0;
#pragma unroll
  for (int kk = 0; kk < kSwB; ++kk) {
    const int p = Pb * kSwB + kk;
    const float d = a[kk][kk];
    if (dropped[p] || !(d > thrs[p])) {
      dmask |= 1u << kk;
      continue;
    }
    const float id = __frcp_rn(d);
#pragma unroll
    for (int r = 0; r < kSwB; ++r)
#pragma unroll
      for (int c = 0; c < kSwB; ++c)
        if (r != kk && c != kk) a[r][c] = fmaf(-a[r][kk] * id, a[kk][c], a[r][c]);
#pragma unroll
    for (int c = 0; c < kSwB; ++c)
      if (c != kk) {
        a[kk][c] *= id;
        a[c][kk] *= id;
      }
    a[kk][kk] = -id;
  }
#pragma unroll
  for (int r = 0; r < kSwB; ++r)
#pragma unroll
    for (int c = 0; c < kSwB; ++c) {
      const bool keep = !((dmask >> r) & 1u) && !((dmask >> c) & 1u);
      a[r][c] = keep ? a[r][c] : 0.f;
      Zo[r][c] = -a[r][c];
    }
#pragma unroll
  for (int kk = 0; kk < kSwB; ++kk)
    if ((dmask >> kk) & 1u) dropped[Pb * kSwB + kk] = 1;
}

__global__ void __maxnreg__(96) k_sweep_inv(const Ctrl* __restrict__ ctrl, int force, int nslots,
                                            const float* __restrict__ M, int64_t m_slot, int tau,
                                            float* __restrict__ P, int64_t pld, int64_t p_slot,
                                            int32_t* __restrict__ ndropped) {
  const int64_t slot = blockIdx.x;
  if (slot >= active_slots(ctrl, force, nslots)) return;
  // X = A[:, P] and Y = X Z column by column, rows padded to 9 per block of 8 so
  // that lanes reading different blocks hit different banks: X[i][kk] at
  // Xs[kk][(i / 8) * 9 + i % 8]
  constexpr int kRow9 = kSwMaxTau / kSwB * (kSwB + 1);
  __shared__ float Xs[kSwB][kRow9];
  __shared__ float Ys[kSwB][kRow9];
  __shared__ float Zs[kSwB][kSwB + 1];      // Z of the current panel
  __shared__ float thrs[kSwMaxTau];         // pivot threshold in the scaled matrix
  __shared__ float sc[kSwMaxTau];           // M_ii^{-1/2}, 0 for an index dropped at the start
  __shared__ unsigned char dropped[kSwMaxTau];
  __shared__ float s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nb = (tau + kSwB - 1) / kSwB;
  const int tp = nb * kSwB;
  const int nblocks = nb * (nb + 1) / 2;
  const bool own = tid < nblocks;
  int I = 0;
  while ((I + 1) * (I + 2) / 2 <= tid) ++I;
  const int J = tid - I * (I + 1) / 2;  // block (I, J), I >= J
  const float* Ms = M + slot * m_slot;
  float dmax = 0.f;
  for (int i = tid; i < tau; i += blockDim.x) dmax = fmaxf(dmax, Ms[(int64_t)i * tau + i]);
  {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0) s_red[wid] = dmax;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < nw; ++w) t = fmaxf(t, s_red[w]);
      s_red[0] = t;
    }
    __syncthreads();
  }
  const float thr = (float)tau * 1.1920928955078125e-07f * s_red[0];
  for (int i = tid; i < tp; i += blockDim.x) {
    const float d = (i < tau) ? Ms[(int64_t)i * tau + i] : 0.f;
    const bool dr = (i >= tau) || !(d > thr);  // padding counts as dropped
    dropped[i] = dr;
    sc[i] = dr ? 0.f : rsqrtf(d);
    thrs[i] = dr ? 0.f : thr / d;
  }
  __syncthreads();
  float a[kSwB][kSwB];
#pragma unroll
  for (int r = 0; r < kSwB; ++r) {
    const int i = I * kSwB + r;
    const float si = (own && i < tau) ? sc[i] : 0.f;
#pragma unroll
    for (int c = 0; c < kSwB; ++c) {
      const int l = J * kSwB + c;
      a[r][c] = (own && i < tau && l < tau) ? Ms[(int64_t)i * tau + l] * si * sc[l] : 0.f;
    }
  }
  if (own && I == 0 && J == 0) diag_sweep(a, 0, thrs, dropped, Zs);

  for (int Pb = 0; Pb < nb; ++Pb) {
    __syncthreads();  // Z of the panel in Zs; X, Y of the previous panel consumed
    // the panel blocks publish X and Y = X Z: (I > Pb, Pb) holds X_I, (Pb, J < Pb)
    // holds X_J^T
    if (own && J == Pb && I > Pb) {
#pragma unroll
      for (int r = 0; r < kSwB; ++r)
#pragma unroll
        for (int kk = 0; kk < kSwB; ++kk) Xs[kk][I * (kSwB + 1) + r] = a[r][kk];
    } else if (own && I == Pb && J < Pb) {
#pragma unroll
      for (int kk = 0; kk < kSwB; ++kk)
#pragma unroll
        for (int c = 0; c < kSwB; ++c) Xs[kk][J * (kSwB + 1) + c] = a[kk][c];
    }
    __syncthreads();
    // Y = X Z by every thread (an entry each: 8 FMAs in the order of kk), instead of
    // 512 FMAs by each panel block's owner
    for (int e = tid; e < nb * kSwB * kSwB; e += blockDim.x) {
      const int blk = e / (kSwB * kSwB);
      if (blk == Pb) continue;
      const int c = (e / kSwB) % kSwB, r = e % kSwB;
      const int col = blk * (kSwB + 1) + r;
      float y = 0.f;
#pragma unroll
      for (int kk = 0; kk < kSwB; ++kk) y = fmaf(Xs[kk][col], Zs[kk][c], y);
      Ys[c][col] = y;
    }
    __syncthreads();
    // A_IJ -= X_I Y_J^T; A_IP = Y_I, A_PJ = Y_J^T; A_PP = -Z already
    if (own) {
      if (I == Pb && J == Pb) {
        // swept by this thread after the previous panel's update
      } else if (J == Pb) {
#pragma unroll
        for (int r = 0; r < kSwB; ++r)
#pragma unroll
          for (int c = 0; c < kSwB; ++c) a[r][c] = Ys[c][I * (kSwB + 1) + r];
      } else if (I == Pb) {
#pragma unroll
        for (int r = 0; r < kSwB; ++r)
#pragma unroll
          for (int c = 0; c < kSwB; ++c) a[r][c] = Ys[r][J * (kSwB + 1) + c];
      } else {
#pragma unroll 1
        for (int kk = 0; kk < kSwB; ++kk) {  // rolled: one rank-1 step of loads live
          float y[kSwB];
#pragma unroll
          for (int c = 0; c < kSwB; ++c) y[c] = Ys[kk][J * (kSwB + 1) + c];
#pragma unroll
          for (int r = 0; r < kSwB; ++r) {
            const float x = Xs[kk][I * (kSwB + 1) + r];
#pragma unroll
            for (int c = 0; c < kSwB; ++c) a[r][c] = fmaf(-x, y[c], a[r][c]);
          }
        }
        // the next panel's diagonal block is final now: sweep it while the other
        // blocks are still being updated (Z is read again only after the barrier)
        if (I == Pb + 1 && J == Pb + 1) diag_sweep(a, Pb + 1, thrs, dropped, Zs);
      }
    }
  }
  __syncthreads();
  // P = -D^{-1/2} (swept M') D^{-1/2} on the kept indices, both triangles
  if (own) {
    float* Ps = P + slot * p_slot;
#pragma unroll
    for (int r = 0; r < kSwB; ++r) {
      const int i = I * kSwB + r;
      const float si = (i < tp && !dropped[i]) ? -sc[i] : 0.f;
#pragma unroll
      for (int c = 0; c < kSwB; ++c) {
        const int l = J * kSwB + c;
        a[r][c] *= (!dropped[l]) ? si * sc[l] : 0.f;
      }
    }
    if ((I + 1) * kSwB <= tau) {  // full blocks: rows of 8 as two float4 stores
#pragma unroll
      for (int r = 0; r < kSwB; ++r) {
        float* row = Ps + (int64_t)(I * kSwB + r) * pld + J * kSwB;
        if (I != J) {
          *reinterpret_cast<float4*>(row) = make_float4(a[r][0], a[r][1], a[r][2], a[r][3]);
          *reinterpret_cast<float4*>(row + 4) = make_float4(a[r][4], a[r][5], a[r][6], a[r][7]);
        } else {
#pragma unroll
          for (int c = 0; c <= r; ++c) row[c] = a[r][c];
        }
      }
      if (I != J) {
#pragma unroll
        for (int c = 0; c < kSwB; ++c) {
          float* row = Ps + (int64_t)(J * kSwB + c) * pld + I * kSwB;
          *reinterpret_cast<float4*>(row) = make_float4(a[0][c], a[1][c], a[2][c], a[3][c]);
          *reinterpret_cast<float4*>(row + 4) = make_float4(a[4][c], a[5][c], a[6][c], a[7][c]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < kSwB; ++r)
#pragma unroll
          for (int c = 0; c < r; ++c) Ps[(int64_t)(J * kSwB + c) * pld + I * kSwB + r] = a[r][c];
      }
    } else {  // the ragged last block row
#pragma unroll
      for (int r = 0; r < kSwB; ++r)
#pragma unroll
        for (int c = 0; c < kSwB; ++c) {
          const int i = I * kSwB + r, l = J * kSwB + c;
          if (i < tau && l < tau && (I != J || c <= r)) {
            Ps[(int64_t)i * pld + l] = a[r][c];
            Ps[(int64_t)l * pld + i] = a[r][c];
          }
        }
    }
  }
  if (tid == 0 && ndropped != nullptr) {
    int cnt = 0;
    for (int i = 0; i < tau; ++i) cnt += dropped[i];
    if (cnt) atomicAdd(ndropped, cnt);
  }
}

cudaError_t launch_sweep_inv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                             const float* M, int64_t m_slot, int64_t tau, float* P, int64_t pld,
                             int64_t p_slot, int32_t* ndropped) {
  if (tau < 1 || tau > kSwMaxTau) return cudaErrorInvalidValue;
  k_sweep_inv<<<nslots, sweep_threads(tau), 0, st>>>(ctrl, force, nslots, M, m_slot, (int)tau, P,
                                                     pld, p_slot, ndropped);
  return cudaGetLastError();
}

template <typename T, typename TP>
cudaError_t launch_potri(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, const double* M,
                         int64_t m_slot, int64_t tau, T* Linv, int64_t l_slot, TP* P, int64_t pld,
                         int64_t p_slot, T* ws, int32_t* ndropped) {
  const int use_smem = potri_needs_ws(tau, sizeof(T)) ? 0 : 1;
  if (tau < 1 || tau > 4096 || (!use_smem && ws == nullptr)) return cudaErrorInvalidValue;
  const size_t smem = use_smem ? potri_ws_elems(tau) * sizeof(T) : 0;
  if (use_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_potri<T, TP, kPotriThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPotriSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_potri<T, TP, 4 * kPotriThreads>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPotriSmemMax);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  k_potri<T, TP, kPotriThreads><<<nslots, kPotriThreads, smem, st>>>(
      ctrl, force, nslots, M, m_slot, tau, Linv, l_slot, P, pld, p_slot, ws, use_smem, ndropped,
      (int64_t)nsm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_potri<T, TP, 4 * kPotriThreads><<<(unsigned)std::min<int64_t>(nslots, nsm),
                                      4 * kPotriThreads, smem, st>>>(
      ctrl, force, nslots, M, m_slot, tau, Linv, l_slot, P, pld, p_slot, ws, use_smem, ndropped,
      (int64_t)nsm);
  return cudaGetLastError();
}
template cudaError_t launch_potri<float, float>(cudaStream_t, const Ctrl*, int, int, const double*,
                                                int64_t, int64_t, float*, int64_t, float*, int64_t,
                                                int64_t, float*, int32_t*);
template cudaError_t launch_potri<double, double>(cudaStream_t, const Ctrl*, int, int,
                                                  const double*, int64_t, int64_t, double*, int64_t,
                                                  double*, int64_t, int64_t, double*, int32_t*);
template cudaError_t launch_potri<double, float>(cudaStream_t, const Ctrl*, int, int,
                                                 const double*, int64_t, int64_t, double*, int64_t,
                                                 float*, int64_t, int64_t, double*, int32_t*);

int potri_batch_ctas() {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return 4 * nsm;
}

template <typename T, typename TP>
cudaError_t launch_potri_batch(cudaStream_t st, const PotriJob* jobs, const int32_t* order,
                               int nrun, int chunk, int64_t tau_max, T* ws) {
  if (nrun <= 0) return cudaSuccess;
  if (tau_max < 1 || tau_max > 4096 || ws == nullptr || chunk < 1) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)nrun * chunk;
  const int grid = (int)std::min<int64_t>(total, potri_batch_ctas());
  k_potri_batch<T, TP><<<grid, kPotriThreads, 0, st>>>(jobs, order, nrun, chunk, ws,
                                                        (int64_t)potri_ws_elems(tau_max));
  return cudaGetLastError();
}
template cudaError_t launch_potri_batch<float, float>(cudaStream_t, const PotriJob*, const int32_t*,
                                                      int, int, int64_t, float*);
template cudaError_t launch_potri_batch<double, double>(cudaStream_t, const PotriJob*,
                                                        const int32_t*, int, int, int64_t, double*);
template cudaError_t launch_potri_batch<double, float>(cudaStream_t, const PotriJob*,
                                                       const int32_t*, int, int, int64_t, double*);

// P_s = L_s^{-T} L_s^{-1}: P(i, j) = sum_k Linv[k, i] Linv[k, j], every slot in one launch
template <typename TF>
cudaError_t launch_pinv(cudaStream_t st, const Ctrl* ctrl, int force, int nslots, const TF* Linv,
                        int64_t l_slot, int64_t tau, TF* P, int64_t pld, int64_t p_slot) {
  return gemm_strided<TF, TF, TF>(st, tau, tau, tau, Linv, 1, tau, Linv, tau, 1, P, pld, 0.0, 0,
                                  force ? nullptr : ctrl, nslots, l_slot, l_slot, p_slot);
}

#define RS_INST(T)                                                                             \
  template cudaError_t launch_pinv<T>(cudaStream_t, const Ctrl*, int, int, const T*, int64_t,  \
                                      int64_t, T*, int64_t, int64_t);                          \
  template cudaError_t launch_factor_inv<T>(cudaStream_t, const Ctrl*, int, int, const double*, \
                                            int64_t, int64_t, T*, int64_t, T*, int32_t*);       \
  template cudaError_t launch_delta<T>(cudaStream_t, const Ctrl*, int, int64_t, DeltaArgs<T>);
RS_INST(float)
RS_INST(double)
#undef RS_INST

}  // namespace rs
