// A = X^T X + lambda I on the 5th-generation tensor cores (mixed form, eq. (2)).
//
// TF32 operands, FP32 accumulation in tensor memory. X is first copied transposed
// (Xt = X^T, d x ldk, K = n contiguous and zero padded) so that both operands of
// C = Xt Xt^T are K-major. The lower triangle is cut into 128 x 256 tiles (128 rows
// ti, 256 columns tj, tj <= ti / 2), one CTA per tile. Consecutive CTAs take the row
// blocks 2a and 2a + 1 of the same column block, so the second read of that B block
// is served from L2. Per 128 x 256 x 32 step a CTA reads 16 KB of A rows and 32 KB
// of B rows (two 128-row boxes) into its own shared memory.
//   warp 0 (one lane)  TMA producer: its A box and both B boxes into a ring of
//                      kStages stages; a stage is refilled once the MMAs that read
//                      it have retired (one arrival on its `empty` barrier);
//   warp 1 (one lane)  MMA issuer: 4 x tcgen05.mma (M 128, N 256, K 8) per stage,
//                      tcgen05.commit frees the stage;
//   warps 0-3          epilogue: tcgen05.ld of the 128 x 256 FP32 accumulator (each
//                      warp its 32 TMEM lanes), + lambda on the diagonal, to global.
// The upper triangle is mirrored afterwards. Every mbarrier wait is bounded; on a
// timeout the CTA records an error, stops issuing, and frees its tensor memory.
#include <cuda.h>

#include <cstring>

#include "rs_kernels.cuh"

namespace rs {

namespace {

constexpr int kBM = 128;                            // rows of a CTA's tile
constexpr int kBN = 256;                            // columns (the pair's B block)
constexpr int kBK = 32;                             // K step: 32 fp32 = one 128-byte row
constexpr int kStages = 4;
constexpr int kABytes = kBM * kBK * 4;              // 16 KB
constexpr int kBHalfBytes = (kBN / 2) * kBK * 4;    // 16 KB, one 128-row box of B
constexpr int kStageBytes = kABytes + 2 * kBHalfBytes;  // 48 KB
constexpr uint32_t kTmemCols = 256;
constexpr uint64_t kWaitNs = 4000000000ull;  // 4 s bound of every wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait on phase `parity`, bounded by kWaitNs of the global timer; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255) {
      const uint64_t t = now_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > kWaitNs) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// UMMA shared-memory descriptor, K-major operand in the 128-byte swizzled layout
// written by TMA: 8-row groups of 128-byte rows, 1024 bytes apart.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, D f32, A/B tf32, both K-major, M = 128, N = 256
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
// arrive once on `bar` when the MMAs issued so far retire
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// ---- epilogue through shared memory and TMA stores ----
constexpr int kOutCols = 32;                        // columns of one output box (128 bytes)
constexpr int kOutBoxBytes = kBM * kOutCols * 4;    // 16 KB

// 32 consecutive accumulator columns of the warp's 32 TMEM lanes (one row per lane)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, const void* src, int x,
                                                  int y) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most N bulk groups of this thread still reading shared memory / still in flight
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
// generic-proxy writes of shared memory visible to the bulk copies that follow
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The first ncb 32-column boxes of the CTA's 128-row accumulator, one after the
// other: TMEM -> registers (op(row, column, bits) gives each stored value) -> a
// 128 x 32 box in the 128-byte swizzled layout of the output tensor map (16-byte
// chunk j of row r at chunk j ^ (r % 8), so that the lanes' stores hit distinct
// banks) -> one TMA store (or reduce-add) of the box at (x0 + 32 cb, y0). Two boxes
// alternate in `stage` (1024-byte aligned, 32 KB free); the store of box cb - 2 must
// have read its buffer before box cb is written there. Every thread of the CTA calls
// this; thread 0 issues and waits for the bulk copies.
template <typename Op>
__device__ __forceinline__ void epilogue_tma(uint32_t tmem, unsigned char* stage,
                                             const CUtensorMap* tout, int x0, int y0, int ncb,
                                             bool reduce, Op op) {
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int rl = wid * 32 + lane;
  for (int cb = 0; cb < ncb; ++cb) {
    unsigned char* buf = stage + (cb & 1) * kOutBoxBytes;
    if (cb >= 2) {
      if (tid == 0) bulk_wait_read<1>();
      __syncthreads();
    }
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(wid * 32) << 16) + (uint32_t)(cb * kOutCols), v);
    float4* row = reinterpret_cast<float4*>(buf + rl * 128);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = cb * kOutCols + 4 * j;
      row[j ^ (rl & 7)] = make_float4(op(rl, c, v[4 * j]), op(rl, c + 1, v[4 * j + 1]),
                                      op(rl, c + 2, v[4 * j + 2]), op(rl, c + 3, v[4 * j + 3]));
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (reduce) tma_reduce_add_2d(tout, buf, x0 + cb * kOutCols, y0);
      else tma_store_2d(tout, buf, x0 + cb * kOutCols, y0);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait<0>();
}
}  // namespace

// K steps [kb0, kb0 + nk); mode 1 (accumulate): add the tiles to A (a later range of
// rows of X); mode 0: store them with lambda on the diagonal; mode 2 (the Gaussian
// kernel of eq. (Gausskernel) on the rows of the operand, C = P P^T): store
// exp(-max(sq_r + sq_c - 2 C_rc, 0) * rbf_scale), rbf_scale = 1 / (2 sigma^2)
// With tma_out, tout maps A (d x d, row stride lda) for the TMA-store epilogue: the
// tile's boxes are written whole, so a diagonal tile also writes (or adds to) its
// part above the diagonal, which the caller's mirror overwrites.
__global__ void __launch_bounds__(128, 1) k_gram_tc(const __grid_constant__ CUtensorMap tmap,
                                                   const __grid_constant__ CUtensorMap tout,
                                                   int64_t d, int64_t kb0, int64_t nk,
                                                   double lambda, int accumulate,
                                                   float* __restrict__ A, int64_t lda,
                                                   int32_t* __restrict__ err,
                                                   const float* __restrict__ sqn,
                                                   float rbf_scale, int tma_out) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled stages
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const uint32_t crank = blockIdx.x & 1;

  // CTAs 2p and 2p + 1: row blocks 2a + crank, column block tj <= a
  const int64_t p = blockIdx.x / 2;
  int64_t a = 0;
  while ((a + 1) * (a + 2) / 2 <= p) ++a;
  const int64_t tj = p - a * (a + 1) / 2;
  const int row0 = (int)((2 * a + (int64_t)crank) * kBM), col0 = (int)(tj * kBN);
  if (row0 >= d) return;  // the odd row block past the last one (uniform over the CTA)

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);  // released by the commit of the MMAs that read it
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to TMA
  }
  if (wid == 0) {  // tensor memory for the 128 x 256 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (wid == 0 && lane == 0) {
    // producer: the A box and the two 128-row boxes of the B block
    int64_t kb = 0;
    for (; kb < nk; ++kb) {
      const int s = (int)(kb % kStages);
      const uint32_t ph = (uint32_t)((kb / kStages) & 1);
      if (!mbar_wait(&empty_bar[s], ph ^ 1)) { s_abort = 1; atomicExch(err, 1); break; }
      if (*(volatile int*)&s_abort) break;
      unsigned char* st = base + s * kStageBytes;
      mbar_arrive_expect_tx(&full_bar[s], kStageBytes);  // A + both boxes of B
      const int kx = (int)((kb0 + kb) * kBK);
      tma_load_2d(st, &tmap, &full_bar[s], kx, row0);
      tma_load_2d(st + kABytes, &tmap, &full_bar[s], kx, col0);
      tma_load_2d(st + kABytes + kBHalfBytes, &tmap, &full_bar[s], kx, col0 + kBN / 2);
    }
  } else if (wid == 1 && lane == 0) {
    // MMA issuer
    for (int64_t kb = 0; kb < nk; ++kb) {
      const int s = (int)(kb % kStages);
      const uint32_t ph = (uint32_t)((kb / kStages) & 1);
      if (!mbar_wait(&full_bar[s], ph)) { s_abort = 1; atomicExch(err, 1); break; }
      if (*(volatile int*)&s_abort) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + s * kStageBytes);
      const uint32_t sb = sa + kABytes;
#pragma unroll
      for (int ks = 0; ks < kBK / 8; ++ks)  // K = 8 tf32 = 32 bytes per MMA
        mma_tf32(tmem, umma_desc_sw128(sa + ks * 32), umma_desc_sw128(sb + ks * 32),
                 (kb > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);  // the stage is free once these MMAs retire
    }
    mma_commit(&done_bar);  // arrives once every MMA issued above has retired
  }
  __syncwarp();
  // epilogue: all 128 threads, warp w reads TMEM lanes 32w..32w+31
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0));
  if (!ok && lane == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && !*(volatile int*)&s_abort && tma_out) {
    // boxes not entirely above the tile's last row, nor past column d
    const int64_t lim = min((int64_t)row0 + kBM - col0, d - col0);
    const int64_t nbox = (lim + kOutCols - 1) / kOutCols;
    const int ncb = (int)(nbox < kBN / kOutCols ? nbox : kBN / kOutCols);
    const int mode = accumulate;
    epilogue_tma(tmem, base, &tout, col0, row0, ncb, mode == 1,
                 [&](int rl, int c, uint32_t bits) -> float {
                   const int64_t r = row0 + rl, cidx = col0 + c;
                   float f = __uint_as_float(bits);
                   if (mode == 2) {
                     if (r >= d || cidx >= d) return 0.f;  // clipped by the store
                     const float d2 = fmaxf(sqn[r] + sqn[cidx] - 2.f * f, 0.f);
                     return (cidx == r) ? 1.f : expf(-d2 * rbf_scale);
                   }
                   if (mode == 0 && cidx == r) f = (float)((double)f + lambda);
                   return f;
                 });
  } else if (ok && !*(volatile int*)&s_abort) {
    const int64_t r = row0 + wid * 32 + lane;
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      if (col0 + c0 > row0 + kBM - 1) break;  // above every row of the tile (uniform)
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(wid * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < d) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int64_t cidx = col0 + c0 + q;
          if (cidx < d && cidx <= r) {
            float f = __uint_as_float(v[q]);
            if (accumulate == 2) {
              const float d2 = fmaxf(sqn[r] + sqn[cidx] - 2.f * f, 0.f);
              f = (cidx == r) ? 1.f : expf(-d2 * rbf_scale);
            } else if (accumulate) {
              f += A[r * lda + cidx];
            } else if (cidx == r) {
              f = (float)((double)f + lambda);
            }
            A[r * lda + cidx] = f;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// C = P Q^T for K-major P (Mr x K, map ta) and Q (N x K, map tb), FP32 out, on the same
// pipeline as k_gram_tc (128 x 256 tiles, one CTA each, 4 stages of TMA loads, TF32
// MMAs into tensor memory). Used for S^T A of the Gaussian sketch: P = the chunk's S^T
// blocks stacked (rows slot * tau + j), Q = A (symmetric, so A^T = A). Row blocks of
// slots past the active ones (convergence forecast, iteration cap) are skipped.
// With tma_out, tc maps C (Mr x N, row stride ldc) for the TMA-store epilogue; a tile
// that reaches past the active rows writes its rows past them too (rows of slots that
// no iteration reads).
__global__ void __launch_bounds__(128, 1) k_gemm_tc_nt(const __grid_constant__ CUtensorMap ta,
                                                      const __grid_constant__ CUtensorMap tb,
                                                      const __grid_constant__ CUtensorMap tc,
                                                      int64_t Mr, int64_t N, int64_t nk,
                                                      float* __restrict__ C, int64_t ldc,
                                                      const Ctrl* __restrict__ ctrl, int force,
                                                      int nslots, int64_t rows_per_slot,
                                                      int32_t* __restrict__ err, int tma_out) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t rows_live = (ctrl != nullptr || force)
                                ? active_slots(ctrl, force, nslots) * rows_per_slot
                                : Mr;
  const int64_t rmax = rows_live < Mr ? rows_live : Mr;
  const int row0 = (int)((int64_t)blockIdx.y * kBM), col0 = (int)((int64_t)blockIdx.x * kBN);
  if (row0 >= rmax) return;  // uniform over the CTA
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], 1);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  if (wid == 0 && lane == 0) {  // producer
    for (int64_t kb = 0; kb < nk; ++kb) {
      const int q = (int)(kb % kStages);
      const uint32_t ph = (uint32_t)((kb / kStages) & 1);
      if (!mbar_wait(&empty_bar[q], ph ^ 1)) { s_abort = 1; atomicExch(err, 1); break; }
      if (*(volatile int*)&s_abort) break;
      unsigned char* stg = base + q * kStageBytes;
      mbar_arrive_expect_tx(&full_bar[q], kStageBytes);
      const int kx = (int)(kb * kBK);
      tma_load_2d(stg, &ta, &full_bar[q], kx, row0);
      tma_load_2d(stg + kABytes, &tb, &full_bar[q], kx, col0);
      tma_load_2d(stg + kABytes + kBHalfBytes, &tb, &full_bar[q], kx, col0 + kBN / 2);
    }
  } else if (wid == 1 && lane == 0) {  // MMA issuer
    for (int64_t kb = 0; kb < nk; ++kb) {
      const int q = (int)(kb % kStages);
      const uint32_t ph = (uint32_t)((kb / kStages) & 1);
      if (!mbar_wait(&full_bar[q], ph)) { s_abort = 1; atomicExch(err, 1); break; }
      if (*(volatile int*)&s_abort) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + q * kStageBytes);
      const uint32_t sb = sa + kABytes;
#pragma unroll
      for (int ks = 0; ks < kBK / 8; ++ks)
        mma_tf32(tmem, umma_desc_sw128(sa + ks * 32), umma_desc_sw128(sb + ks * 32),
                 (kb > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&empty_bar[q]);
    }
    mma_commit(&done_bar);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0));
  if (!ok && lane == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && !*(volatile int*)&s_abort && tma_out) {
    const int64_t lim = N - col0;
    const int64_t nbox = (lim + kOutCols - 1) / kOutCols;
    const int ncb = (int)(nbox < kBN / kOutCols ? nbox : kBN / kOutCols);
    epilogue_tma(tmem, base, &tc, col0, row0, ncb, false,
                 [](int, int, uint32_t bits) -> float { return __uint_as_float(bits); });
  } else if (ok && !*(volatile int*)&s_abort) {
    const int64_t r = row0 + wid * 32 + lane;
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      if (col0 + c0 >= N) break;  // uniform
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(wid * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < rmax) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int64_t cidx = col0 + c0 + q;
          if (cidx < N) C[r * ldc + cidx] = __uint_as_float(v[q]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// Xt[i * ldk + k] = X[k * d + i] (zero for k >= n): 32 x 32 tiles through shared memory;
// with Xcopy != nullptr the tile is also stored to Xcopy (same layout as X), so that a
// copy of X and its transpose come from one read of X
__global__ void k_transpose_pad(const float* __restrict__ X, int64_t n, int64_t d,
                                float* __restrict__ Xt, int64_t ldk, int64_t k_base,
                                float* __restrict__ Xcopy) {
  __shared__ float tile[32][33];
  const int64_t k0 = k_base + (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = k0 + r, i = i0 + threadIdx.x;
    const float v = (k < n && i < d) ? X[k * d + i] : 0.f;
    tile[r][threadIdx.x] = v;
    if (Xcopy != nullptr && k < n && i < d) Xcopy[k * d + i] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, k = k0 + threadIdx.x;
    if (i < d && k < ldk) Xt[i * ldk + k] = tile[threadIdx.x][r];
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

size_t gram_tc_ws_floats(int64_t n, int64_t d) { return (size_t)d * (size_t)round_up(n, 32); }

// tensor map of an FP32 output (rows x cols, row stride ld floats) in 128-row x 32-column
// boxes, 128-byte swizzled, for the TMA-store epilogue; false (the kernel then stores
// directly) when the base or the row stride is not 16-byte aligned
static bool out_map(EncodeTiledFn enc, CUtensorMap* map, float* base, int64_t rows, int64_t cols,
                    int64_t ld) {
  std::memset(map, 0, sizeof(*map));
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 4) % 16 != 0 || rows <= 0 || cols <= 0)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kOutCols, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the rows [r0, r1) of X (r0 a multiple of 32; r1 too, or r1 = n): their part of
// X^T X into the lower triangle of A (d x lda; the caller mirrors), stored with lambda
// on the diagonal for r0 = 0, else added to A
cudaError_t launch_gram_tc_rows(cudaStream_t st, const float* X, int64_t n, int64_t d,
                                double lambda, float* A, int64_t lda, float* Xt_ws, int32_t* err,
                                int64_t r0, int64_t r1, float* Xcopy) {
  const int64_t ldk = round_up(n, 32);
  const int64_t k1 = (r1 >= n) ? ldk : r1;  // the last range takes the zero padding
  if (r0 % 32 != 0 || k1 % 32 != 0 || r0 >= k1) return cudaErrorInvalidValue;
  dim3 tb(32, 8), tg((unsigned)((k1 - r0) / 32), (unsigned)((d + 31) / 32));
  k_transpose_pad<<<tg, tb, 0, st>>>(X, n, d, Xt_ws, ldk, r0, Xcopy);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)d};
  const cuuint64_t strides[1] = {(cuuint64_t)ldk * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};  // also one half of B
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Xt_ws, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  CUtensorMap omap;
  const int tma_out = out_map(enc, &omap, A, d, d, lda) ? 1 : 0;
  const int64_t T = (d + kBM - 1) / kBM;  // row blocks
  const int64_t Tp = (T + 1) / 2;         // row-block pairs
  const int64_t pairs = Tp * (Tp + 1) / 2;  // (pair, column block) with tj <= pair
  const size_t smem = (size_t)kStages * kStageBytes + 1024;
  e = set_smem_max((const void*)k_gram_tc, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_gram_tc, map, omap, d, r0 / kBK, (k1 - r0) / kBK, lambda,
                            r0 > 0 ? 1 : 0, A, lda, err, (const float*)nullptr, 0.f, tma_out);
}

// the rows of P (n x d) zero-padded to ldk = round_up(d, 32) columns (the K-major
// operand of C = P P^T), and their squared norms in FP32 (summed in FP64)
__global__ void k_pad_rows(const float* __restrict__ P, int64_t n, int64_t d, int64_t ldk,
                           float* __restrict__ out, float* __restrict__ sqn) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t k = lane; k < ldk; k += 32) {
    const float v = k < d ? P[i * d + k] : 0.f;
    out[i * ldk + k] = v;
    s += (double)v * (double)v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) sqn[i] = (float)s;
}

size_t rbf_tc_ws_floats(int64_t n, int64_t d) { return (size_t)n * round_up(d, 32) + (size_t)n; }

// K = exp(-||p_i - p_j||^2 / (2 sigma^2)) of the rows of P (n x d, FP32, device), the
// lower triangle on the tensor cores (TF32 products, FP32 accumulation in tensor
// memory, the kernel's exponential in the epilogue), into K (n x ldK); the caller
// mirrors the upper triangle. ws: rbf_tc_ws_floats(n, d) floats.
cudaError_t launch_rbf_tc(cudaStream_t st, const float* P, int64_t n, int64_t d, double sigma,
                          float* K, int64_t ldK, float* ws, int32_t* err) {
  const int64_t ldk = round_up(d, 32);
  float* Pp = ws;
  float* sqn = ws + (size_t)n * ldk;
  k_pad_rows<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(P, n, d, ldk, Pp, sqn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ldk * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Pp, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  CUtensorMap omap;
  const int tma_out = out_map(enc, &omap, K, n, n, ldK) ? 1 : 0;
  const int64_t T = (n + kBM - 1) / kBM;
  const int64_t Tp = (T + 1) / 2;
  const int64_t pairs = Tp * (Tp + 1) / 2;
  const size_t smem = (size_t)kStages * kStageBytes + 1024;
  e = set_smem_max((const void*)k_gram_tc, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  const float scale = (float)(1.0 / (2.0 * sigma * sigma));
  return cudaLaunchKernelEx(&cfg, k_gram_tc, map, omap, n, (int64_t)0, ldk / kBK, 0.0, 2, K, ldK,
                            err, (const float*)sqn, scale, tma_out);
}

// S^T A of every slot of a chunk for the Gaussian sketch on the tensor cores:
// SA[s tau + j, c] = sum_i ST[s tau + j, i] A[c, i] (A symmetric). ST and SA hold the
// slots' tau x ld blocks back to back (row stride ld, zero beyond column m); lda and ld
// multiples of 4 (16-byte row strides for the tensor maps)
cudaError_t launch_gauss_sa_tc(cudaStream_t st, const Ctrl* ctrl, int force, int nslots,
                               const float* ST, int64_t ld, int64_t m, int64_t tau,
                               const float* A, int64_t lda, float* SA, int32_t* err) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (ld % 32 != 0 || lda % 4 != 0) return cudaErrorInvalidValue;
  const int64_t rows = (int64_t)nslots * tau;
  CUtensorMap ma, mb;
  const cuuint64_t da[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  const cuuint64_t sta[1] = {(cuuint64_t)ld * 4};
  const cuuint64_t db[2] = {(cuuint64_t)ld, (cuuint64_t)m};
  const cuuint64_t stb[1] = {(cuuint64_t)lda * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ST), da, sta, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  r = enc(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), db, stb, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  CUtensorMap mc;
  const int tma_out = out_map(enc, &mc, SA, rows, m, ld) ? 1 : 0;
  const size_t smem = (size_t)kStages * kStageBytes + 1024;
  cudaError_t e = set_smem_max((const void*)k_gemm_tc_nt, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((m + kBN - 1) / kBN), (unsigned)((rows + kBM - 1) / kBM));
  k_gemm_tc_nt<<<grid, 128, smem, st>>>(ma, mb, mc, rows, m, ld / kBK, SA, ld, ctrl, force, nslots,
                                         tau, err, tma_out);
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(cudaStream_t st, const float* X, int64_t n, int64_t d, double lambda,
                           float* A, int64_t lda, float* Xt_ws, int32_t* err, float* Xcopy) {
  return launch_gram_tc_rows(st, X, n, d, lambda, A, lda, Xt_ws, err, 0, n, Xcopy);
}

}  // namespace rs
