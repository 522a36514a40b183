// Phase 2 of a chunk on the whole GPU: every iteration of Algorithm 2 (Section 6.3,
// update of eq. (53)) of the chunk runs inside one launch of nblk CTAs (clusters of
// kWideCluster), for the bucket-row sketches (subsample, count, subcount).
//
// CTA c owns the rows [c q, (c + 1) q) of w, w_prev, r, r_prev and keeps them in
// shared memory for the whole launch. With P_k = M_k^+ formed in phase 1 and the
// sketch written as S_k = sum_i sigma_i e_i e_{b_i}^T,
//   delta_k = P_k S_k^T r_k = sum_c sum_{i in c, sketched} sigma_i r_i P_k[b_i, :],
// so every CTA contributes a partial of delta_k from its own rows alone. One
// all-reduce per iteration (tau partial entries plus the partial ||r_k||^2) gives
// every CTA the same delta_k and ||r_k||; each then updates its own rows:
//   (A S_k delta_k)_i = sum_j (S_k^T A)[j, i] delta_j   from its block of S_k^T A,
//   (S_k delta_k)_i   = sigma_i delta_{b_i},
//   w_i, r_i          by the momentum step (1 + beta) x - beta x_prev - gamma (...).
// Phase 1 writes S_k^T A blocked by CTA (the tau x q block of CTA c is contiguous),
// so one bulk copy per iteration stages it in shared memory; the rows P_k[b_i, :]
// and the slot's inverse map are bulk-copied too, all one or two iterations ahead
// and issued after the CTA has published its partials, so that they overlap the
// all-reduce.
//
// All-reduce, deterministic, in two stages. CTA rank r of a cluster owns the entries
// [r E, (r + 1) E) of the tau + 1. (1) Inside the cluster: every CTA stores its
// partials of those entries into rank r's shared memory with st.async (the bytes
// complete on r's gather mbarrier), and r adds them over the 16 CTAs in rank order.
// (2) Across clusters: r publishes its cluster sums to global memory as
// self-validating words (payload and exchange tag in one 8-byte word), reads the
// sums of every cluster, re-reading the words whose tag is not current yet, and adds
// them in cluster order (one cluster: no global memory at all). (3) r stores the
// totals into the shared memory of every CTA of its cluster with st.async. Each
// global word is thus read by one CTA per cluster instead of every CTA polling the
// partials of every other one. Every wait is bounded (global timer); a CTA that
// gives up raises the abort word, which ends the others' waits.
//
// Precision of the mixed form (T = TF = float): FP64 instructions take 64 cycles
// (add, FMA) to about 100 (conversions) on this GPU, and every one of them on the
// path from one all-reduce to the next adds to the iteration's latency. So w,
// w_prev, r, r_prev are float pairs (hi + lo) in shared memory, each update adds
// an FP32 increment to them exactly (error-free sums), the all-reduced delta
// arrives as float pairs, and ||r_k||^2 / ||r_0||^2 is summed in FP32 for the
// stopping test (a convergence it signals is confirmed by the FP64 refresh). FP64
// arithmetic remains only at the launch's start and end.
#include "rs_kernels.cuh"
#include "rs_ptx.cuh"

namespace rs {

namespace {

constexpr int kWThreads = 256;
constexpr int kWWarps = kWThreads / 32;
constexpr int kIssueWarp = kWWarps - 1;        // issues the bulk copies
constexpr int kRowsPerLane = 2;                 // rows of a lane in the A S delta product
// waits at the end of a launch for copies already in flight into this CTA's shared
// memory: they land within microseconds, so this bound is generous and independent
// of the caller's limit on the other waits
constexpr uint64_t kDrainNs = 2000000000ull;

// clusters of one launch at most (the stage-2 sums of the all-reduce)
constexpr int kMaxClusters = 16;

struct WideLayout {
  int64_t qs, E;
  size_t sa, pb, iv, mine, tot, dT, red, gat, st, coef, prow, pinv, hn2, bars, gb, sum, total;
};

__host__ __device__ inline size_t wl_take(size_t& o, size_t bytes) {
  const size_t at = o;
  o += (bytes + 127) / 128 * 128;
  return at;
}

// shared-memory layout of one CTA (host and device agree on it)
__host__ __device__ inline WideLayout wide_layout(int64_t q, int64_t tau, int64_t pld, int se,
                                                  int sf, int64_t chunk, int nsab) {
  WideLayout L;
  L.qs = (q + 3) / 4 * 4;
  L.E = (tau + 1 + kWideCluster - 1) / kWideCluster;  // all-reduce entries per cluster rank
  size_t o = 0;
  L.sa = wl_take(o, (size_t)nsab * tau * L.qs * se);  // S^T A block, 1 or 2 buffers
  L.pb = wl_take(o, (size_t)L.qs * pld * sf);       // rows of P for the own rows
  L.iv = wl_take(o, (size_t)3 * L.qs * 4);          // inverse map slices, 3 slots
  L.mine = wl_take(o, (size_t)tau * 8);             // own partials of delta
  L.tot = wl_take(o, (size_t)(tau + 1) * 8);        // all-reduced totals
  L.dT = wl_take(o, (size_t)tau * se);              // delta in the product type
  const int64_t rw = kWWarps * L.qs > kMaxClusters * L.E ? kWWarps * L.qs : kMaxClusters * L.E;
  L.red = wl_take(o, (size_t)rw * 8);               // cross-warp / cross-cluster partial sums
  L.gat = wl_take(o, (size_t)2 * kWideCluster * L.E * 8);  // cluster's partials of own entries
  L.st = wl_take(o, (size_t)4 * L.qs * 8);          // r, r_prev, w, w_prev
  L.coef = wl_take(o, (size_t)L.qs * 8);            // sigma_i r_i of the staged rows
  L.prow = wl_take(o, (size_t)L.qs * 4);            // staged row -> own row | sign
  L.pinv = wl_take(o, (size_t)L.qs * 4);            // own row -> staged row, or -1
  L.hn2 = wl_take(o, (size_t)(chunk + 1) * 8);      // ||r_k||^2 of the tested iterations
  L.bars = wl_take(o, 8 * 8);                       // mbarriers
  L.gb = wl_take(o, (size_t)2 * chunk * 8);         // gamma_k, beta_k of the chunk
  L.sum = wl_take(o, (size_t)L.qs * 8);             // running sums of the own w rows
  L.total = o;
  return L;
}

// bounded wait on an mbarrier phase (wait_ns of the global timer); false on timeout
// or (abort_word != nullptr) when another CTA has raised the abort word
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, const int32_t* abort_word,
                         uint64_t wait_ns) {
  if (ptx::mbar_test(bar, parity)) return true;
  const uint64_t t0 = ptx::now_ns();
  for (uint32_t it = 1;; ++it) {
    if (ptx::mbar_test(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (abort_word != nullptr && ptx::ld_relaxed_s32(abort_word) != 0) return false;
      if (ptx::now_ns() - t0 > wait_ns) return false;
    }
  }
}

struct Xch {
  uint64_t* part;   // 2 (parity) x nclu x 2 ne words: the clusters' sums
  int32_t* abort_word;
  uint64_t wait_ns;  // bound of every wait
  int nclu, clu;     // clusters of the launch, this CTA's cluster
  uint32_t crank;
  int64_t tau, ne, E;
  void* mine;       // PT[tau]: own partials of delta
  const void* mine_nrm;  // own partial of ||r||^2 (float for PT = float, else double)
  double* tot;      // ne all-reduced totals (delta, then ||r||^2)
  void* red;        // per-cluster sums of the own entries
  void* gat;        // PT[2][kWideCluster][E]: the cluster's partials of the own entries
  uint64_t* xbar;   // the totals have arrived
  uint64_t* gbar;   // the cluster's partials of the own entries have arrived
};

// The clusters' sums travel as self-validating words: a 32-bit payload and the
// exchange's 32-bit tag in one 8-byte word (single-copy atomic), so a reader that
// sees the tag has the payload and no separate flag, fence or release is needed.
// Tags increase from exchange to exchange and from launch to launch and the buffer
// alternates by parity, so a stale word never carries the current tag. Two words
// per entry: PT = float, the sum as a float pair (hi, lo); PT = double, the low and
// high halves of the sum.
__device__ __forceinline__ uint64_t ll_word(uint32_t payload, uint32_t tag) {
  return (uint64_t)payload | ((uint64_t)tag << 32);
}

// error-free sum of two floats (Knuth): s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float t = s - a;
  e = (a - (s - t)) + (b - t);
}

// entries of the all-reduce owned by cluster rank crank
__device__ __forceinline__ int64_t xch_own(int64_t ne, int64_t E, uint32_t crank) {
  const int64_t e0 = (int64_t)crank * E;
  return e0 < ne ? (ne - e0 < E ? ne - e0 : E) : 0;
}

// arm the gather mbarrier for the next exchange: the bytes of the own entries from
// every CTA of the cluster. It is armed before the launch's first exchange and right
// after each wait on it, so always before a peer can store into it: a peer sends
// exchange n + 1 only once it has the totals of exchange n, which include this
// CTA's, stored after this CTA's wait.
template <typename PT>
__device__ __forceinline__ void arm_gather(uint64_t* gbar, int64_t ne, int64_t E, uint32_t crank) {
  ptx::mbar_arrive_expect_tx(gbar, (uint32_t)(xch_own(ne, E, crank) * kWideCluster * sizeof(PT)));
}

// All-reduce of the partials over every CTA into `tot`, first half: store every
// partial into the gather buffer of the cluster rank that owns its entry. `n` counts
// this launch's exchanges. No block barrier is needed for the exchange: thread t
// stores the partials mine[t + 256 u] it wrote itself, thread 0 the norm it summed
// itself, and every thread read `tot` of the previous exchange before the block
// barrier that precedes the partials. The totals' mbarrier was armed for this exchange at the end
// of the previous one (or before the first), so before any total can arrive: a total
// needs every CTA's partials, sent after the next block barrier.
template <typename PT>
__device__ void xch_begin(const Xch& x, uint32_t tag, uint32_t n) {
  const int tid = threadIdx.x;
  const PT* mine = static_cast<const PT*>(x.mine);
  PT* gat = static_cast<PT*>(x.gat) + (size_t)(n & 1) * kWideCluster * x.E + x.crank * x.E;
  auto send = [&](int64_t e, PT v) {
    const uint32_t rk = (uint32_t)(e / x.E);
    const uint32_t dst = ptx::map_rank(gat + (e - (int64_t)rk * x.E), rk);
    if constexpr (sizeof(PT) == 4) ptx::st_async_b32(dst, __float_as_uint(v), ptx::map_rank(x.gbar, rk));
    else ptx::st_async_f64(dst, v, ptx::map_rank(x.gbar, rk));
  };
  for (int64_t e = tid; e < x.tau; e += kWThreads) send(e, mine[e]);
  if (tid == 0) send(x.tau, *static_cast<const PT*>(x.mine_nrm));
}

// second half, by the thread that owns each entry of this cluster rank: wait for
// the cluster's partials of the entry and add them in rank order; with more than
// one cluster, publish the sum, read every cluster's sum of the entry (re-reading
// words whose tag is not current yet) and add them in cluster order (PT = float:
// float pairs throughout, so the sums are as accurate as in FP64 without FP64
// arithmetic); store the total into the `tot` of every CTA of the cluster (PT =
// float: a normalised float pair (hi, lo) in each 8-byte entry). Then every thread
// waits for the cluster's totals; one block barrier at the end agrees on failure
// (abort or timeout anywhere), after which the call returns false everywhere.
template <typename PT>
__device__ bool xch_end(const Xch& x, uint32_t tag, uint32_t n) {
  constexpr bool F = sizeof(PT) == 4;
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)x.crank * x.E;
  const int64_t nown = xch_own(x.ne, x.E, x.crank);
  bool ok = true;
  if (tid < nown) {
    ok = wait_bar(x.gbar, n & 1, x.abort_word, x.wait_ns);
    // phase n is complete for this thread; the peers' stores of exchange n + 1 come
    // only after the totals of exchange n, which wait for every owner thread here
    if (ok && tid == 0) arm_gather<PT>(x.gbar, x.ne, x.E, x.crank);
    float S = 0.f, C = 0.f;  // PT = float
    double acc = 0.0;        // PT = double
    if (ok) {
      const PT* gat = static_cast<const PT*>(x.gat) + (size_t)(n & 1) * kWideCluster * x.E + tid;
#pragma unroll
      for (int c = 0; c < kWideCluster; ++c) {
        if constexpr (F) {
          float t, err;
          two_sum(S, gat[c * x.E], t, err);
          S = t;
          C += err;
        } else {
          acc += gat[c * x.E];
        }
      }
    }
    if (ok && x.nclu > 1) {
      uint64_t* pb = x.part + (size_t)(n & 1) * x.nclu * 2 * x.ne;
      {
        uint32_t lo, hi;
        if constexpr (F) {
          lo = __float_as_uint(S);
          hi = __float_as_uint(C);
        } else {
          const uint64_t b = (uint64_t)__double_as_longlong(acc);
          lo = (uint32_t)b;
          hi = (uint32_t)(b >> 32);
        }
        uint64_t* w = pb + ((size_t)x.clu * x.ne + e0 + tid) * 2;
        ptx::st_relaxed_u64(w, ll_word(lo, tag));
        ptx::st_relaxed_u64(w + 1, ll_word(hi, tag));
      }
      // every cluster's words of this entry, all loads of a pass in flight at once
      uint64_t a[kMaxClusters], b[kMaxClusters];
      uint32_t pend = (x.nclu >= 32) ? 0xffffffffu : ((1u << x.nclu) - 1u);
      const uint64_t t0 = ptx::now_ns();
      for (uint32_t pass = 0; pend != 0; ++pass) {
#pragma unroll
        for (int g = 0; g < kMaxClusters; ++g) {
          if (pend & (1u << g)) {
            const uint64_t* w = pb + ((size_t)g * x.ne + e0 + tid) * 2;
            a[g] = ptx::ld_relaxed_u64(w);
            b[g] = ptx::ld_relaxed_u64(w + 1);
          }
        }
#pragma unroll
        for (int g = 0; g < kMaxClusters; ++g)
          if ((pend & (1u << g)) && (uint32_t)(a[g] >> 32) == tag && (uint32_t)(b[g] >> 32) == tag)
            pend &= ~(1u << g);
        if (pend != 0 && (pass & 15) == 15 &&
            (ptx::ld_relaxed_s32(x.abort_word) != 0 || ptx::now_ns() - t0 > x.wait_ns)) {
          ok = false;
          break;
        }
      }
      if (ok) {
        S = 0.f;
        C = 0.f;
        acc = 0.0;
#pragma unroll
        for (int g = 0; g < kMaxClusters; ++g) {
          if (g >= x.nclu) break;
          if constexpr (F) {
            float t, err;
            two_sum(S, __uint_as_float((uint32_t)a[g]), t, err);
            S = t;
            C += err + __uint_as_float((uint32_t)b[g]);
          } else {
            acc += __longlong_as_double((long long)((a[g] & 0xFFFFFFFFull) | (b[g] << 32)));
          }
        }
      }
    }
    if (ok) {
      const int64_t e = e0 + tid;
      if constexpr (F) {
        float hi, lo;
        two_sum(S, C, hi, lo);
        const uint64_t v = (uint64_t)__float_as_uint(hi) | ((uint64_t)__float_as_uint(lo) << 32);
#pragma unroll
        for (uint32_t rk = 0; rk < (uint32_t)kWideCluster; ++rk)
          ptx::st_async_b64(ptx::map_rank(x.tot + e, rk), v, ptx::map_rank(x.xbar, rk));
      } else {
#pragma unroll
        for (uint32_t rk = 0; rk < (uint32_t)kWideCluster; ++rk)
          ptx::st_async_f64(ptx::map_rank(x.tot + e, rk), acc, ptx::map_rank(x.xbar, rk));
      }
    } else {
      atomicExch(x.abort_word, 1);
    }
  } else if (tid == 0) {
    arm_gather<PT>(x.gbar, x.ne, x.E, x.crank);  // no own entries: zero bytes
  }
  ok = ok && wait_bar(x.xbar, n & 1, x.abort_word, x.wait_ns);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(x.abort_word, 1);
    return false;
  }
  if (tid == 0) ptx::mbar_arrive_expect_tx(x.xbar, (uint32_t)(x.ne * 8));  // exchange n + 1
  return true;
}

// float pair (hi, lo) of a double, and back
__device__ __forceinline__ float2 split2(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ double join2(float2 a) { return (double)a.x + (double)a.y; }

// a + b for a float pair a and a float b, error-free up to the final rounding of lo
__device__ __forceinline__ float2 add_pf(float2 a, float b) {
  float s, e;
  two_sum(a.x, b, s, e);
  e += a.y;
  float h, l;
  two_sum(s, e, h, l);
  return make_float2(h, l);
}

}  // namespace

template <typename T, typename TF>
__global__ void __launch_bounds__(kWThreads, 1) k_iterate_wide(Ctrl* __restrict__ ctrl,
                                                              WideArgs<T, TF> g) {
  extern __shared__ __align__(128) unsigned char smem[];
  // ctrl is read once; no CTA writes it before every CTA has passed its first
  // exchange, so all CTAs take the same branches
  if (halted(ctrl)) return;
  const int64_t k0 = ctrl->k0, kstart = ctrl->k;
  // this launch's part of the chunk ends at k0 + sub_end (an FP64 refresh may follow)
  int64_t kend = min(k0 + g.sub_end, ctrl->max_iters);
  if (ctrl->kcap > 0 && ctrl->kcap < kend) kend = ctrl->kcap;  // convergence forecast
  if (kstart >= kend) return;
  const double tol = ctrl->tol, r0 = ctrl->r0;
  const double thr2 = (tol * r0) * (tol * r0);
  const double thr2_lo = thr2 * (1.0 - 1e-9), thr2_hi = thr2 * (1.0 + 1e-9);
  // float-pair state (mixed form): norms relative to ||r_0||, thresholds in FP32
  constexpr bool kFP = sizeof(T) == 4 && sizeof(TF) == 4;
  const float inv_r0f = r0 > 0.0 ? (float)(1.0 / r0) : 0.f;
  const float thr2f = (float)(tol * tol);
  const int no_stop = ctrl->no_stop;
  const uint64_t tag0 = (*g.epoch) << 24;
  // Algorithm 3 coefficients in FP32 (mixed form): alpha, (1 - beta)(1 - alpha), gamma
  const float aaf = (float)g.acc_a, cvf = (float)((1.0 - g.acc_b) * (1.0 - g.acc_a)),
              agf = (float)g.acc_g;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int cta = blockIdx.x;
  uint32_t crank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
  const int64_t tau = g.tau, m = g.m;
  const int nsab = g.nsab;
  const WideLayout L =
      wide_layout(g.q, tau, g.pld, (int)sizeof(T), (int)sizeof(TF), g.chunk, nsab);
  const int64_t qs = L.qs;
  const int64_t ilo = (int64_t)cta * g.q;
  const int64_t qc = ilo < m ? (m - ilo < g.q ? m - ilo : g.q) : 0;  // own rows
  const int64_t qcp = (qc + 3) / 4 * 4;                                // copied width
  const bool has_rows = qc > 0;

  T* sab = reinterpret_cast<T*>(smem + L.sa);
  TF* pbuf = reinterpret_cast<TF*>(smem + L.pb);
  int32_t* ivb = reinterpret_cast<int32_t*>(smem + L.iv);
  TF* mine = reinterpret_cast<TF*>(smem + L.mine);
  double* tot = reinterpret_cast<double*>(smem + L.tot);
  T* dT = reinterpret_cast<T*>(smem + L.dT);
  T* red = reinterpret_cast<T*>(smem + L.red);
  TF* coef = reinterpret_cast<TF*>(smem + L.coef);
  double* sr = reinterpret_cast<double*>(smem + L.st);
  double* srp = sr + qs;
  double* sw = srp + qs;
  double* swp = sw + qs;
  // the same buffers as float pairs (kFP)
  float2* fr = reinterpret_cast<float2*>(sr);
  float2* frp = fr + qs;
  float2* fw = frp + qs;
  float2* fwp = fw + qs;
  const float2* tot2 = reinterpret_cast<const float2*>(tot);
  int32_t* prow = reinterpret_cast<int32_t*>(smem + L.prow);
  int32_t* pinv = reinterpret_cast<int32_t*>(smem + L.pinv);
  double* hn2 = reinterpret_cast<double*>(smem + L.hn2);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* sa_full = bars;        // 2
  uint64_t* iv_full = bars + 2;    // 3
  uint64_t* p_full = bars + 5;     // 1
  uint64_t* xbar = bars + 6;       // 1
  uint64_t* gbar = bars + 7;       // 1
  double* ssum = reinterpret_cast<double*>(smem + L.sum);  // sum of w^0..w^k (averaging)
  double* sgam = reinterpret_cast<double*>(smem + L.gb);
  double* sbet = sgam + g.chunk;
  float* sgamf = reinterpret_cast<float*>(sgam);  // kFP: gamma_k, beta_k in FP32
  float* sbetf = sgamf + g.chunk;
  float2* hn2f = reinterpret_cast<float2*>(hn2);  // kFP: ||r_k||^2 / ||r_0||^2 as float pairs
  __shared__ int s_nrows;
  __shared__ double s_red[32];
  __shared__ double s_nrm;  // own partial of ||r||^2
  __shared__ float s_redf[32];
  __shared__ float s_nrmf;  // kFP: own partial of ||r||^2 / ||r_0||^2

  if (tid == 0) {
    for (int b = 0; b < 8; ++b) ptx::mbar_init(bars + b, 1);
    // the first exchange: the cluster's partials of the own entries, the totals
    arm_gather<TF>(bars + 7, tau + 1, L.E, crank);
    ptx::mbar_arrive_expect_tx(bars + 6, (uint32_t)((tau + 1) * 8));
    ptx::fence_mbar_init();
  }
  for (int64_t k = kstart + tid; k < kend; k += kWThreads) {
    if constexpr (kFP) {
      sgamf[k - k0] = (float)g.gam[k];
      sbetf[k - k0] = (float)g.bet[k];
    } else {
      sgam[k - k0] = g.gam[k];
      sbet[k - k0] = g.bet[k];
    }
  }
  for (int64_t i = tid; i < qc; i += kWThreads) {
    ssum[i] = g.wsum != nullptr ? g.wsum[ilo + i] : 0.0;
    if constexpr (kFP) {
      fr[i] = split2(g.r[ilo + i]);
      frp[i] = split2(g.rp[ilo + i]);
      fw[i] = split2(g.w[ilo + i]);
      fwp[i] = split2(g.wp[ilo + i]);
    } else {
      sr[i] = g.r[ilo + i];
      srp[i] = g.rp[ilo + i];
      sw[i] = g.w[ilo + i];
      swp[i] = g.wp[ilo + i];
    }
  }
  __syncthreads();
  ptx::cluster_sync_all();  // peers' mbarriers are initialised before any remote store

  Xch x;
  x.part = g.part; x.abort_word = g.abort_word; x.wait_ns = g.wait_ns;
  x.nclu = g.nblk / kWideCluster; x.clu = cta / kWideCluster; x.crank = crank;
  x.tau = tau; x.ne = tau + 1; x.E = L.E;
  x.mine = mine; x.tot = tot; x.red = red; x.gat = smem + L.gat; x.xbar = xbar; x.gbar = gbar;
  if constexpr (kFP) x.mine_nrm = &s_nrmf; else x.mine_nrm = &s_nrm;

  // copy bookkeeping, identical in every thread: issued / consumed phases per buffer
  uint32_t sa_iss[2] = {0, 0}, sa_use[2] = {0, 0};
  uint32_t iv_iss[3] = {0, 0, 0}, iv_use[3] = {0, 0, 0};
  uint32_t p_iss = 0, p_use = 0;
  bool ok = true;

  auto slot_of = [&](int64_t k) { return k - k0; };
  // (issue warp) inverse-map slice of slot s
  auto issue_iv = [&](int64_t s) {
    const int b = (int)(s % 3);
    if (wid == kIssueWarp && lane == 0) {
      ptx::mbar_arrive_expect_tx(iv_full + b, (uint32_t)(qcp * 4));
      ptx::bulk_g2s(ivb + b * qs, g.inv + s * g.inv_slot + ilo, (uint32_t)(qcp * 4), iv_full + b);
    }
    iv_iss[b]++;
  };
  // (every thread) the inverse map of slot s is in place
  auto wait_iv = [&](int64_t s) -> bool {
    const int b = (int)(s % 3);
    const bool r = wait_bar(iv_full + b, iv_use[b] & 1, g.abort_word, g.wait_ns);
    iv_use[b]++;
    return !__syncthreads_or(!r);
  };
  // (issue warp) the CTA's tau x qs block of S^T A of slot s: one bulk copy
  auto issue_sa = [&](int64_t s) {
    const int b = (int)(s % nsab);
    if (wid == kIssueWarp && lane == 0) {
      const uint32_t bytes = (uint32_t)(tau * qs * sizeof(T));
      ptx::mbar_arrive_expect_tx(sa_full + b, bytes);
      ptx::bulk_g2s(sab + (size_t)b * tau * qs, g.rows + s * g.sa_slot + (int64_t)cta * tau * qs,
                    bytes, sa_full + b);
    }
    sa_iss[b]++;
  };
  // (issue warp) rows P_s[b_i, :] for the sketched own rows; the inverse map of s
  // must be in place (waited by the issue warp itself: `iv_ready`)
  auto issue_p = [&](int64_t s, bool iv_ready) {
    if (wid == kIssueWarp) {
      const int bi = (int)(s % 3);
      bool okw = iv_ready || wait_bar(iv_full + bi, iv_use[bi] & 1, g.abort_word, g.wait_ns);
      if (!okw) {
        if (lane == 0) atomicExch(g.abort_word, 1);
      }
      const int32_t* iv = ivb + bi * qs;
      int nrows = 0;
      for (int64_t i0 = 0; i0 < qc; i0 += 32) {
        const int64_t i = i0 + lane;
        const int32_t e = (okw && i < qc) ? iv[i] : kNotSketched;
        const bool sk = (e != kNotSketched);
        const unsigned bal = __ballot_sync(0xffffffffu, sk);
        const int t = nrows + __popc(bal & ((1u << lane) - 1u));
        if (sk) prow[t] = (int32_t)((uint32_t)i | ((uint32_t)e & 0x80000000u));
        if (i < qc) pinv[i] = sk ? t : -1;
        nrows += __popc(bal);
      }
      __syncwarp();
      const uint32_t rb = (uint32_t)(g.pld * sizeof(TF));
      if (lane == 0) {
        s_nrows = nrows;
        ptx::mbar_arrive_expect_tx(p_full, rb * (uint32_t)nrows);
      }
      __syncwarp();
      const TF* Ps = g.P + s * g.p_slot;
      for (int t = lane; t < nrows; t += 32) {
        const int32_t e = iv[prow[t] & 0x7FFFFFFF];
        ptx::bulk_g2s(pbuf + (size_t)t * g.pld, Ps + (int64_t)(e & 0x7FFFFFFF) * g.pld, rb, p_full);
      }
    }
    p_iss++;
  };
  // own partials of delta_k (with_delta) and of ||r_k||^2: the squares are summed
  // per warp into s_red by whoever last wrote the rows (the update, or `fresh`)
  auto partial = [&](bool with_delta, bool fresh) -> bool {
    const bool use_p = with_delta && has_rows;
    if (fresh) {
      if constexpr (kFP) {
        float sq = 0.f;
        for (int64_t i = tid; i < qc; i += kWThreads) {
          const float v = fr[i].x * inv_r0f;
          sq = fmaf(v, v, sq);
        }
        if (wid * 32 < qc) sq = warp_sum(sq);
        if (lane == 0) s_redf[wid] = sq;
      } else {
        double sq = 0.0;
        for (int64_t i = tid; i < qc; i += kWThreads) sq += sr[i] * sr[i];
        if (wid * 32 < qc) sq = warp_sum(sq);
        if (lane == 0) s_red[wid] = sq;
      }
    }
    if (use_p) {
      const bool r = wait_bar(p_full, p_use & 1, g.abort_word, g.wait_ns);
      p_use++;
      if (__syncthreads_or(!r)) return false;
    } else {
      __syncthreads();
    }
    // sigma_i r_i of the staged rows, once each in the partial's precision (FP64
    // arithmetic is scarce on this GPU: nothing of it in the loop below)
    const int nrows = use_p ? s_nrows : 0;
    if (fresh) {  // else the row update has written them
      for (int t = tid; t < nrows; t += kWThreads) {
        const int32_t pr = prow[t];
        // r_S of r (Algorithm 2) or of r_z = r_w - alpha (r_w - r_v) (Algorithm 3)
        if constexpr (kFP) {
          float v = fr[pr & 0x7FFFFFFF].x;
          if (g.accel) v -= aaf * (v - frp[pr & 0x7FFFFFFF].x);
          coef[t] = pr < 0 ? -v : v;
        } else {
          double v = sr[pr & 0x7FFFFFFF];
          if (g.accel) v = g.acc_a * srp[pr & 0x7FFFFFFF] + (1.0 - g.acc_a) * v;
          coef[t] = (TF)(pr < 0 ? -v : v);
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      if constexpr (kFP) {
        float t = 0.f;
        if (has_rows)
          for (int w = 0; w < kWWarps; ++w) t += s_redf[w];
        s_nrmf = t;
      } else {
        double t = 0.0;
        if (has_rows)
          for (int w = 0; w < kWWarps; ++w) t += s_red[w];
        s_nrm = t;
      }
    }
    // four independent chains over the staged rows, added in a fixed order
    const int64_t pld = g.pld;
    for (int64_t j = tid; j < tau; j += kWThreads) {
      const TF* pj = pbuf + j;
      TF a0 = TF(0), a1 = TF(0), a2 = TF(0), a3 = TF(0);
      int t = 0;
      for (; t + 4 <= nrows; t += 4) {
        a0 += coef[t] * pj[(int64_t)t * pld];
        a1 += coef[t + 1] * pj[(int64_t)(t + 1) * pld];
        a2 += coef[t + 2] * pj[(int64_t)(t + 2) * pld];
        a3 += coef[t + 3] * pj[(int64_t)(t + 3) * pld];
      }
      for (; t < nrows; ++t) a0 += coef[t] * pj[(int64_t)t * pld];
      mine[j] = (a0 + a1) + (a2 + a3);
    }
    return true;
  };

  int64_t k = kstart;
  uint32_t nx = 0;   // exchanges so far
  int outcome = 0;   // 0 chunk done, 1 converged, 2 numeric failure, 3 timed out
  if (has_rows) {
    const int64_t s0 = slot_of(k);
    issue_iv(s0);
    if (k + 1 < kend) issue_iv(s0 + 1);
    issue_sa(s0);
    ok = wait_iv(s0);
    if (ok) issue_p(s0, true);
  }
  if (g.stall_ns > 0 && cta == 0) {
    // fault injection (tests of the bounded waits): this CTA publishes its first
    // partials stall_ns late, so that the other CTAs' waits for them run out
    const uint64_t t0 = ptx::now_ns();
    while (ptx::now_ns() - t0 < (uint64_t)g.stall_ns) {
    }
  }
  if (ok) ok = partial(true, true);
  while (ok) {
    const uint32_t tag = (uint32_t)(tag0 + nx + 1);
    xch_begin<TF>(x, tag, nx);
    // prefetch, after the partials are out: S^T A and P rows of the next slot,
    // the inverse map of the one after. The P rows, their row maps and count replace
    // the ones the partials just read: the issue warp waits on named barrier 1 until
    // every other warp has passed it (after its partials), the others do not wait
    if (has_rows && k + 1 < kend) {
      if (wid == kIssueWarp) ptx::named_bar_sync(1, kWThreads);
      else ptx::named_bar_arrive(1, kWThreads);
      const int64_t s1 = slot_of(k + 1);
      if (nsab == 2) issue_sa(s1);  // one buffer: issued once iteration k has read it
      issue_p(s1, false);
      if (k + 2 < kend) issue_iv(s1 + 1);
    }
    ok = xch_end<TF>(x, tag, nx);
    ++nx;
    if (!ok) break;
    // stopping test on ||r_k|| (k = kstart was tested before this launch): every
    // thread takes the same decision from the same total (thread 0 records the
    // norm); FP64 square root and division only within 1e-9 of the boundary
    int dec = 0;
    if (k > kstart) {
      if constexpr (kFP) {
        // relative ||r_k||^2 in FP32; the FP64 refresh confirms a convergence
        const float2 n2 = tot2[tau];
        if (tid == 0) hn2f[k - k0] = n2;
        const float nf = n2.x + n2.y;
        if (!isfinite(nf)) dec = 2;
        else if (!no_stop && nf <= thr2f) dec = 1;
      } else {
        const double n2 = tot[tau];
        if (tid == 0) hn2[k - k0] = n2;
        if (!isfinite(n2)) {
          dec = 2;
        } else if (!no_stop) {
          if (n2 <= thr2_lo) dec = 1;
          else if (n2 <= thr2_hi) dec = (sqrt(n2) / r0 <= tol) ? 1 : 0;
        }
      }
    }
    if (k >= kend) {
      __syncthreads();
      outcome = dec;
      break;
    }
    // iteration k on the own rows; delta in the product's type, each warp converting
    // the entries of its own columns of the product below (no block barrier)
    const int64_t s = slot_of(k);
    const int64_t jc = (tau + kWWarps - 1) / kWWarps;
    const int64_t j0 = wid * jc, j1 = (j0 + jc < tau) ? j0 + jc : tau;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      if constexpr (kFP) dT[j] = tot2[j].x + tot2[j].y;
      else dT[j] = (T)tot[j];
    }
    __syncwarp();
    const int b = (int)(s % nsab);
    bool r = true;
    if (has_rows) {
      r = (k == kstart) || wait_bar(iv_full + (s % 3), iv_use[s % 3] & 1, g.abort_word, g.wait_ns);
      if (k > kstart) iv_use[s % 3]++;
      r = r && wait_bar(sa_full + b, sa_use[b] & 1, g.abort_word, g.wait_ns);
      sa_use[b]++;
    }
    if (dec != 0) {  // uniform: stop, unless a wait gave up somewhere
      if (__syncthreads_or(!r)) ok = false;
      else outcome = dec;
      break;
    }
    if (has_rows) {
      // (A S delta)_i: warp w takes the columns [w jc, (w + 1) jc), lane the rows
      // lane + 32 u, kRowsPerLane at a time; a failed wait is agreed on at the block
      // barrier after the product (the product only reads this CTA's shared memory)
      const T* sb = sab + (size_t)b * tau * qs;
      for (int64_t i0 = 0; i0 < qc; i0 += 32 * kRowsPerLane) {
        T acc[kRowsPerLane][4];  // 4 independent chains over j
#pragma unroll
        for (int u = 0; u < kRowsPerLane; ++u)
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) acc[u][q4] = T(0);
        int64_t j = j0;
        for (; j + 4 <= j1; j += 4) {
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const T d = dT[j + q4];
#pragma unroll
            for (int u = 0; u < kRowsPerLane; ++u) {
              const int64_t i = i0 + lane + 32 * u;
              if (i < qs) acc[u][q4] += sb[(j + q4) * qs + i] * d;
            }
          }
        }
        for (; j < j1; ++j) {
          const T d = dT[j];
#pragma unroll
          for (int u = 0; u < kRowsPerLane; ++u) {
            const int64_t i = i0 + lane + 32 * u;
            if (i < qs) acc[u][0] += sb[j * qs + i] * d;
          }
        }
#pragma unroll
        for (int u = 0; u < kRowsPerLane; ++u) {
          const int64_t i = i0 + lane + 32 * u;
          if (i < qs) red[wid * qs + i] = (acc[u][0] + acc[u][1]) + (acc[u][2] + acc[u][3]);
        }
      }
      if (__syncthreads_or(!r)) { ok = false; break; }
      if (nsab == 1 && k + 1 < kend) issue_sa(s + 1);
      const int32_t* iv = ivb + (s % 3) * qs;
      if constexpr (kFP) {
        // x_{k+1} = x_k + beta (x_k - x_{k-1}) - gamma (...): the increment in FP32,
        // added to the float pair exactly
        const float gk = sgamf[k - k0], bk = sbetf[k - k0];
        float sq = 0.f;
        for (int64_t i = tid; i < qc; i += kWThreads) {
          float asum = 0.f;
#pragma unroll
          for (int w = 0; w < kWWarps; ++w) asum += red[w * qs + i];
          const int32_t e = iv[i];
          float ui = 0.f;
          if (e != kNotSketched) {
            const float2 dv = tot2[e & 0x7FFFFFFF];
            ui = entry_neg(e) ? -(dv.x + dv.y) : (dv.x + dv.y);
          }
          const float2 ri = fr[i], rpi = frp[i], wi = fw[i], wpi = fwp[i];
          const float dr = (ri.x - rpi.x) + (ri.y - rpi.y);
          const float dw = (wi.x - wpi.x) + (wi.y - wpi.y);
          float2 rn, wn;
          float cz;  // r_S coefficient of the next iteration (hi part)
          if (g.accel) {
            // Algorithm 3 as increments: with z = w - alpha (w - v),
            // w+ = z - S delta, v+ = v + (1 - beta)(1 - alpha)(w - v) - gamma S delta,
            // and the same for r_w, r_v with A S delta
            const float2 rvn = add_pf(rpi, fmaf(cvf, dr, -agf * (float)asum));
            rn = add_pf(ri, fmaf(-aaf, dr, -(float)asum));
            wn = add_pf(wi, fmaf(-aaf, dw, -ui));
            fwp[i] = add_pf(wpi, fmaf(cvf, dw, -agf * ui));
            frp[i] = rvn;
            cz = rn.x - aaf * (rn.x - rvn.x);
          } else {
            rn = add_pf(ri, fmaf(bk, dr, -gk * (float)asum));
            wn = add_pf(wi, fmaf(bk, dw, -gk * ui));
            frp[i] = ri;
            fwp[i] = wi;
            cz = rn.x;
          }
          fr[i] = rn;
          fw[i] = wn;
          if (g.wsum != nullptr) ssum[i] += (double)wn.x + (double)wn.y;
          const int32_t t = pinv[i];  // staged row of slot k + 1
          if (t >= 0) coef[t] = prow[t] < 0 ? -cz : cz;
          const float v = rn.x * inv_r0f;
          sq = fmaf(v, v, sq);
        }
        if (wid * 32 < qc) sq = warp_sum(sq);
        if (lane == 0) s_redf[wid] = sq;
      } else {
        const double gk = sgam[k - k0], bk = sbet[k - k0];
        double sq = 0.0;
        for (int64_t i = tid; i < qc; i += kWThreads) {
          T asum = T(0);
#pragma unroll
          for (int w = 0; w < kWWarps; ++w) asum += red[w * qs + i];
          const double asd = (double)asum;
          const int32_t e = iv[i];
          const double ui = (e == kNotSketched) ? 0.0
                            : (entry_neg(e) ? -tot[e & 0x7FFFFFFF] : tot[e & 0x7FFFFFFF]);
          const double ri = sr[i], rpi = srp[i], wi = sw[i], wpi = swp[i];
          double rn, wn, cz;
          if (g.accel) {  // Algorithm 3: (w, v, r_w, r_v) in (w, w_prev, r, r_prev)
            const double z = g.acc_a * wpi + (1.0 - g.acc_a) * wi;
            const double rz = g.acc_a * rpi + (1.0 - g.acc_a) * ri;
            rn = rz - asd;
            wn = z - ui;
            const double rvn = g.acc_b * rpi + (1.0 - g.acc_b) * rz - g.acc_g * asd;
            srp[i] = rvn;
            swp[i] = g.acc_b * wpi + (1.0 - g.acc_b) * z - g.acc_g * ui;
            cz = g.acc_a * rvn + (1.0 - g.acc_a) * rn;
          } else {
            rn = (1.0 + bk) * ri - bk * rpi - gk * asd;
            wn = (1.0 + bk) * wi - bk * wpi - gk * ui;
            srp[i] = ri;
            swp[i] = wi;
            cz = rn;
          }
          sr[i] = rn;
          const int32_t t = pinv[i];  // staged row of slot k + 1
          if (t >= 0) coef[t] = (TF)(prow[t] < 0 ? -cz : cz);
          sw[i] = wn;
          if (g.wsum != nullptr) ssum[i] += wn;
          sq += rn * rn;
        }
        if (wid * 32 < qc) sq = warp_sum(sq);
        if (lane == 0) s_red[wid] = sq;
      }
    }
    if (cta == 0 && k + 1 == kend) {
      for (int64_t j = tid; j < tau; j += kWThreads) {
        if constexpr (kFP) g.delta_out[j] = join2(tot2[j]);
        else g.delta_out[j] = tot[j];
      }
    }
    ++k;
    ok = partial(k < kend, false);
  }
  if (!ok) {
    outcome = 3;
    // let the peers' stores of the last exchange land (bounded)
    if (nx > 0) {
      wait_bar(gbar, (nx - 1) & 1, nullptr, kDrainNs);
      wait_bar(xbar, (nx - 1) & 1, nullptr, kDrainNs);
    }
  }
  // no bulk copy may still be writing this CTA's shared memory when it exits
  if (has_rows) {
    for (int b = 0; b < nsab; ++b)
      for (; sa_use[b] < sa_iss[b]; ++sa_use[b]) wait_bar(sa_full + b, sa_use[b] & 1, nullptr, kDrainNs);
    for (int b = 0; b < 3; ++b)
      for (; iv_use[b] < iv_iss[b]; ++iv_use[b]) wait_bar(iv_full + b, iv_use[b] & 1, nullptr, kDrainNs);
    for (; p_use < p_iss; ++p_use) wait_bar(p_full, p_use & 1, nullptr, kDrainNs);
  }
  __syncthreads();
  for (int64_t i = tid; i < qc; i += kWThreads) {
    if (g.wsum != nullptr) g.wsum[ilo + i] = ssum[i];
    if constexpr (kFP) {
      g.r[ilo + i] = join2(fr[i]);
      g.rp[ilo + i] = join2(frp[i]);
      g.w[ilo + i] = join2(fw[i]);
      g.wp[ilo + i] = join2(fwp[i]);
    } else {
      g.r[ilo + i] = sr[i];
      g.rp[ilo + i] = srp[i];
      g.w[ilo + i] = sw[i];
      g.wp[ilo + i] = swp[i];
    }
  }
  // relative residuals of the tested iterations (kstart was tested before)
  if (cta == 0) {
    const int64_t klast = (outcome == 3) ? kstart : k;
    for (int64_t kk = kstart + 1 + tid; kk <= klast; kk += kWThreads) {
      if constexpr (kFP) g.hist[kk] = sqrt(join2(hn2f[kk - k0]));
      else g.hist[kk] = sqrt(hn2[kk - k0]) / r0;
    }
  }
  if (cta == 0 && tid == 0) {
    ctrl->k = k;
    if (outcome == 3) { ctrl->status = kStatusTimeout; ctrl->stop = 1; }
    if (outcome == 2) { ctrl->status = kStatusNumeric; ctrl->stop = 1; }
    if (outcome == 1) { if (g.mixed) ctrl->pending = 1; else ctrl->stop = 1; }
    if (k >= ctrl->max_iters) ctrl->stop = 1;
    *g.epoch = (tag0 >> 24) + 1;
    __threadfence();
  }
  // no CTA leaves while a peer may still store into its shared memory
  ptx::cluster_sync_all();
}

template <typename T, typename TF>
bool wide_plan(int64_t m, int64_t tau, int max_ctas, int64_t chunk, WidePlan* out) {
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (nsm <= 0 || optin <= 0) return false;
  const int64_t pld = (tau + 3) / 4 * 4;
  int nsab = 2;
  auto smem_of = [&](int64_t q) {
    return wide_layout(q, tau, pld, (int)sizeof(T), (int)sizeof(TF), chunk, nsab).total;
  };
  auto kern = k_iterate_wide<T, TF>;
  int64_t cap_ctas = (int64_t)nsm / kWideCluster * kWideCluster;
  if (max_ctas > 0)
    cap_ctas = std::min<int64_t>(cap_ctas, std::max(kWideCluster, max_ctas / kWideCluster * kWideCluster));
  int64_t q = std::max<int64_t>(4, round_up((m + cap_ctas - 1) / cap_ctas, 4));
  for (;;) {
    if (smem_of(q) > (size_t)optin) nsab = 1;  // S^T A single buffered
    const size_t smem = smem_of(q);
    // the staged block must fit one bulk copy's transaction count as well
    if (smem > (size_t)optin || (size_t)tau * round_up(q, 4) * sizeof(T) >= (1u << 20)) return false;
    if (kWideCluster > 8 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (set_smem_max((const void*)kern, (size_t)((int)smem)) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const int64_t nblk = round_up((m + q - 1) / q, kWideCluster);
    if (nblk > (int64_t)kMaxClusters * kWideCluster) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblk);
    cfg.blockDim = dim3(kWThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kWideCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (ncl <= 0) return false;
    if ((int64_t)ncl * kWideCluster >= nblk) {
      out->nblk = (int)nblk;
      out->q = q;
      out->smem = smem;
      out->nsab = nsab;
      return true;
    }
    // fewer clusters are resident than the slices need: widen the slices
    q = std::max<int64_t>(q + 4, round_up((m + (int64_t)ncl * kWideCluster - 1) /
                                              ((int64_t)ncl * kWideCluster), 4));
  }
}

template <typename T, typename TF>
cudaError_t launch_iterate_wide(cudaStream_t st, Ctrl* ctrl, const WideArgs<T, TF>& g, size_t smem) {
  auto kern = k_iterate_wide<T, TF>;
  cudaError_t e = set_smem_max((const void*)kern, (size_t)((int)smem));
  if (e != cudaSuccess) return e;
  if (kWideCluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.nblk);
  cfg.blockDim = dim3(kWThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kWideCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, ctrl, g);
}

#define RS_WIDE_INST(T, TF)                                                                     \
  template bool wide_plan<T, TF>(int64_t, int64_t, int, int64_t, WidePlan*);                   \
  template cudaError_t launch_iterate_wide<T, TF>(cudaStream_t, Ctrl*, const WideArgs<T, TF>&, \
                                                  size_t);
RS_WIDE_INST(float, float)
RS_WIDE_INST(float, double)
RS_WIDE_INST(double, double)
#undef RS_WIDE_INST

}  // namespace rs
