// k_rank.cu -- per-generation ranking with binary64 rescoring.
//
// Exact top-k from a binary32 pre-ranking (guard band):
//   every circuit's binary64 fitness F lies in [F_lo, F_hi], derived from its
//   binary32 fitness and a bound eps_d on the error of d = (N - |tr|)/N
//   (F = 1 - sqrt(d) - penalty).  Let tau be the k-th largest F_lo.  At least k
//   circuits have F >= tau, so any circuit with F_hi < tau is outside the
//   top-k; the candidates {F_hi >= tau} are rescored in binary64 (k_rescore in
//   k_circuit.cu) and sorted by (F desc, cost asc, index asc).  Binary64
//   searches use the degenerate band F_lo = F_hi = F.
// The selection is a radix select over the top 24 bits of the F_lo keys (two
// 4096-bin histogram passes).  Up to kSelClusterFrom circuits per search it
// runs on one 1024-thread CTA per search; above, on a thread-block cluster of
// kSelCta CTAs per search: each CTA histograms a contiguous slice of the
// population, the cluster combines the histograms through distributed shared
// memory (CTA r sums bins [512 r, 512 r + 512) over all CTAs) and every CTA
// finds the threshold from the combined counts (the cluster's barriers cost
// more than they save on small populations).  A later launch sorts the
// candidates (bitonic, in chunks of up to 2048 so any number fits in shared
// memory).
#include <cooperative_groups.h>

#include "qe_dev.cuh"
#include "qe_host.h"

namespace cg = cooperative_groups;

namespace qe {

// one CTA per search (populations up to kSelClusterFrom circuits)
constexpr int kRankThreads = 1024;
constexpr size_t kSelectSmem = (4096 + 2 * 4096) * sizeof(uint32_t);
constexpr int kKeyCache = 4096;  // circuits whose keys the selection keeps in shared memory
// a cluster per search (larger populations)
constexpr uint32_t kSelClusterFrom = 16384;
constexpr int kSelCta = 8;                    // CTAs per search (one cluster)
constexpr int kSelThreads = 256;
constexpr int kSelSlice = 4096 / kSelCta;     // histogram bins each CTA combines
constexpr int kSelCache = 2048;  // circuits per CTA whose keys stay in shared memory
constexpr int kSortThreads = 256;
constexpr int kSortN = 2048;

__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// binary64 fitness interval of circuit c as a pair of float keys (binary32
// arithmetic only; the slop covers its rounding)
__device__ __forceinline__ void bounds(const DevProblem &p, const RankJob &jb, uint32_t c,
                                       float F, uint32_t &klo, uint32_t &khi) {
  if (!(F == F)) {
    klo = khi = 1u;  // NaN ranks last
    return;
  }
  if (p.prec == 0) {
    const double D = ((const double *)jb.fit)[c];
    klo = fkey(__double2float_rd(D));
    khi = fkey(__double2float_ru(D));
    return;
  }
  float lo, hi;
  guard_band(p, F, jb.meta[c], lo, hi);
  klo = fkey(lo);
  khi = fkey(hi);
}

// suffix scan of the 4096-bin histogram: finds the bin where the count taken
// from the top first reaches rem; every thread owns 4 consecutive bins
__device__ __forceinline__ void find_bin(const uint32_t *hist, uint32_t rem, uint32_t *s_wsum,
                                         uint32_t *s_bin, uint32_t *s_rem) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // thread t owns bins 4095-4t .. 4092-4t (descending)
  uint32_t h[4], loc = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = hist[4095 - 4 * tid - q];
    loc += h[q];
  }
  uint32_t v = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) s_wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = s_wsum[lane], x = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    s_wsum[32 + lane] = x - w;  // exclusive prefix of the warp totals
  }
  __syncthreads();
  uint32_t run = s_wsum[32 + wid] + v - loc;  // count above this thread's first bin
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (run < rem && run + h[q] >= rem) {
      *s_bin = 4095 - 4 * tid - q;
      *s_rem = rem - run;
    }
    run += h[q];
  }
  __syncthreads();
}

// Combine the cluster's histograms and find the bin where the count taken from
// the top first reaches rem: this CTA sums its slice of bins over every CTA
// into tot (block_rank r: bins [kSelSlice r, kSelSlice (r + 1))), then, after
// a cluster barrier (no histogram is read after it), every CTA locates the
// slice from the slice totals and the bin inside it from that slice's counts.
// Returns the bin (0..4095) in *s_bin and the count still wanted inside it in
// *s_rem.  The caller keeps tot unchanged until the next cluster barrier.
__device__ __forceinline__ void cluster_find_bin(cg::cluster_group &cl, const uint32_t *hist,
                                                 uint32_t *tot, uint32_t *s_stot,
                                                 uint32_t *s_wsum, uint32_t rem,
                                                 uint32_t *s_bin, uint32_t *s_rem) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t r = cl.block_rank();
  uint32_t part = 0;
  for (int i = tid; i < kSelSlice; i += kSelThreads) {
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < kSelCta; ++q) v += cl.map_shared_rank(hist, q)[r * kSelSlice + i];
    tot[i] = v;
    part += v;
  }
  part = __reduce_add_sync(kFull, part);
  if (lane == 0) s_wsum[wid] = part;
  __syncthreads();
  if (tid == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) t += s_wsum[w];
    s_stot[kSelCta] = t;  // this CTA's slice total, read by the others
  }
  cl.sync();
  if (tid < kSelCta) s_stot[tid] = cl.map_shared_rank(s_stot, tid)[kSelCta];
  __syncthreads();
  // the slice: from the highest (CTA kSelCta - 1) down
  int sl = 0;
  uint32_t above = 0;
  for (int q = kSelCta - 1; q >= 0; --q) {
    if (above + s_stot[q] >= rem || q == 0) {
      sl = q;
      break;
    }
    above += s_stot[q];
  }
  const uint32_t want = rem - above;
  // the bin inside it: thread t owns bins kSelSlice-1-2t and kSelSlice-2-2t
  const uint32_t *ts = cl.map_shared_rank(tot, sl);
  uint32_t h[2], loc = 0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    h[q] = ts[kSelSlice - 1 - 2 * tid - q];
    loc += h[q];
  }
  uint32_t v = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += u;
  }
  __syncthreads();  // s_wsum is free again
  if (lane == 31) s_wsum[wid] = v;
  __syncthreads();
  uint32_t run = v - loc;
  for (int w = 0; w < wid; ++w) run += s_wsum[w];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (run < want && run + h[q] >= want) {
      *s_bin = (uint32_t)(sl * kSelSlice + kSelSlice - 1 - 2 * tid - q);
      *s_rem = want - run;
    }
    run += h[q];
  }
  __syncthreads();
}

// a pipelined job ranks generation gen - 1 from buffer (gen - 1) & 1
__device__ __forceinline__ RankJob resolve(RankJob jb, const DevProblem &p, uint32_t gen) {
  if (jb.pipelined) {
    const size_t b = (gen - 1u) & 1u;
    jb.fit = (const char *)jb.fit + b * p.P * (p.prec == 0 ? 8 : 4);
    jb.meta += b * p.P;
    jb.gsrc += b * p.P * p.L;
    if (jb.asrc) jb.asrc += b * p.P * p.L;
  }
  return jb;
}

__global__ void __launch_bounds__(kRankThreads) k_rank_select(const DevProblem *__restrict__ probs,
                                                              const RankJob *__restrict__ jobs,
                                                              RankJob single, DevGlobal g) {
  wait_predecessor();  // in the batch graph: the evaluations' fitness and costs
  RankJob jb = jobs ? jobs[blockIdx.x] : single;
  const DevProblem &p = probs[jb.prob];
  if (jb.pipelined) {
    // the chain of generation gen - 1 runs once: skip when there is none or
    // when it was already ranked (drained); every block takes the same decision
    const uint32_t gen = *g.gen;
    const bool active = gen > 0 && *g.ranked < gen;
    if (threadIdx.x == 0) *g.rank_active = active ? 1u : 0u;
    if (!active) return;
    jb = resolve(jb, p, gen);
  }
  const uint32_t n = jb.n;
  const uint32_t k = p.k < n ? p.k : n;
  extern __shared__ uint32_t dyn_smem[];
  uint32_t *hist = dyn_smem;                // 4096 bins
  uint32_t *s_lo = dyn_smem + 4096;         // kKeyCache low keys
  uint32_t *s_hi = s_lo + kKeyCache;        // kKeyCache high keys
  __shared__ uint32_t s_wsum[64];
  __shared__ uint32_t s_bin, s_rem, s_cnt, s_base;
  __shared__ double s_sum[kRankThreads / 32];
  __shared__ unsigned long long s_work[kRankThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool cached = n <= (uint32_t)kKeyCache;
  for (int b = tid; b < 4096; b += kRankThreads) hist[b] = 0;
  __syncthreads();

  // pass 1: one read of every fitness: keys (cached in shared memory), the
  // histogram of the top 12 bits of the low keys, the mean and the work.
  // Histogram updates are aggregated per warp (__match_any_sync): fitness
  // values are often discrete, and many lanes hit the same bin.
  // Mean fitness: binary64 searches sum in binary64; binary32 searches sum in
  // binary32 within each warp and in binary64 across warps, so that their
  // selection issues almost no binary64 instruction (GB300's binary64 pipe is
  // thin, and this kernel runs on one SM per search).
  double sum = 0.0;
  float sum32 = 0.f;
  unsigned long long work = 0;
  for (uint32_t c0 = 0; c0 < n; c0 += kRankThreads) {
    const uint32_t c = c0 + tid;
    uint32_t bin = 4096u;
    if (c < n) {
      float F;
      if (p.prec == 0) {
        const double Fw = ((const double *)jb.fit)[c];
        F = (float)Fw;
        sum += Fw;
      } else {
        F = ((const float *)jb.fit)[c];
        sum32 += F;
      }
      const uint32_t meta = jb.meta[c];
      work += meta >> 8;
      uint32_t lo, hi;
      bounds(p, jb, c, F, lo, hi);
      if (cached) {
        s_lo[c] = lo;
        s_hi[c] = hi;
      }
      bin = lo >> 20;
    }
    const uint32_t peers = __match_any_sync(kFull, bin);
    if (bin < 4096u && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
  }
  if (jb.update_record) {
    if (p.prec == 0) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum32 += __shfl_xor_sync(kFull, sum32, o);
      sum = (double)sum32;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) work += __shfl_xor_sync(kFull, work, o);
    if (lane == 0) {
      s_sum[wid] = sum;
      s_work[wid] = work;
    }
  }
  __syncthreads();
  if (jb.update_record && wid == 0) {
    double t = s_sum[lane];
    unsigned long long wt = s_work[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(kFull, t, o);
      wt += __shfl_xor_sync(kFull, wt, o);
    }
    if (lane == 0) {
      p.rec->mean_fitness = n ? t / (double)n : 0.0;
      p.rec->useful_flops = wt;
    }
  }

  // tau = the k-th largest low key with its last 8 bits cleared (top 12 bits,
  // then the next 12), so tau <= the exact k-th largest and at least k circuits
  // have F_lo >= tau (a lower tau only adds candidates)
  find_bin(hist, k, s_wsum, &s_bin, &s_rem);
  const uint32_t b1 = s_bin, rem = s_rem;
  for (int b = tid; b < 4096; b += kRankThreads) hist[b] = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < n; c0 += kRankThreads) {
    const uint32_t c = c0 + tid;
    uint32_t bin = 4096u;
    if (c < n) {
      uint32_t lo, hi;
      if (cached) lo = s_lo[c];
      else {
        const float F = p.prec == 0 ? (float)((const double *)jb.fit)[c] : ((const float *)jb.fit)[c];
        bounds(p, jb, c, F, lo, hi);
      }
      if ((lo >> 20) == b1) bin = (lo >> 8) & 4095u;
    }
    const uint32_t peers = __match_any_sync(kFull, bin);
    if (bin < 4096u && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
  }
  __syncthreads();
  find_bin(hist, rem, s_wsum, &s_bin, &s_rem);
  const uint32_t tau = (b1 << 20) | (s_bin << 8);

  // candidates: F_hi >= tau
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < n; c0 += kRankThreads) {
    const uint32_t c = c0 + tid;
    bool take = false;
    if (c < n) {
      uint32_t lo, hi;
      if (cached) hi = s_hi[c];
      else {
        const float F = p.prec == 0 ? (float)((const double *)jb.fit)[c] : ((const float *)jb.fit)[c];
        bounds(p, jb, c, F, lo, hi);
      }
      take = hi >= tau;
    }
    const uint32_t bal = __ballot_sync(kFull, take);
    uint32_t wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(&s_cnt, __popc(bal));
    wbase = __shfl_sync(kFull, wbase, 0);
    if (take) {
      const uint32_t slot = wbase + __popc(bal & ((1u << lane) - 1));
      p.cand[slot] = c;
      // binary64 searches: the final value; binary32 searches: the binary32
      // value, which the rescoring checks against the guard band and replaces
      p.cand_f[slot] = p.prec == 0 ? ((const double *)jb.fit)[c]
                                   : (double)((const float *)jb.fit)[c];
    }
  }
  __syncthreads();
  const uint32_t M = s_cnt;
  if (tid == 0) {
    *p.cand_n = M;
    s_base = (p.prec == 0) ? 0u : atomicAdd(g.rescore_n, M);
  }
  __syncthreads();
  if (p.prec != 0)
    for (uint32_t s = tid; s < M; s += kRankThreads) g.rescore_list[s_base + s] = (jb.prob << 20) | s;
}

__global__ void __cluster_dims__(kSelCta, 1, 1) __launch_bounds__(kSelThreads)
    k_rank_select_cl(const DevProblem *__restrict__ probs, const RankJob *__restrict__ jobs,
                  RankJob single, DevGlobal g) {
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t rank = cl.block_rank();
  RankJob jb = jobs ? jobs[blockIdx.x / kSelCta] : single;
  const DevProblem &p = probs[jb.prob];
  if (jb.pipelined) {
    // the chain of generation gen - 1 runs once: skip when there is none or
    // when it was already ranked (drained); every CTA takes the same decision,
    // before any cluster barrier
    const uint32_t gen = *g.gen;
    const bool active = gen > 0 && *g.ranked < gen;
    if (threadIdx.x == 0 && blockIdx.x == 0) *g.rank_active = active ? 1u : 0u;
    if (!active) return;
    jb = resolve(jb, p, gen);
  }
  const uint32_t n = jb.n;
  const uint32_t k = p.k < n ? p.k : n;
  // this CTA's circuits [c_lo, c_hi)
  const uint32_t chunk = (n + kSelCta - 1) / kSelCta;
  const uint32_t c_lo = rank * chunk < n ? rank * chunk : n;
  const uint32_t c_hi = c_lo + chunk < n ? c_lo + chunk : n;
  const bool cached = chunk <= (uint32_t)kSelCache;
  __shared__ uint32_t hist[4096];
  __shared__ uint32_t s_lo[kSelCache], s_hi[kSelCache];
  __shared__ uint32_t tot[kSelSlice];
  __shared__ uint32_t s_stot[kSelCta + 1];
  __shared__ uint32_t s_wsum[32];
  __shared__ uint32_t s_bin, s_rem, s_cnt, s_base;
  __shared__ double s_sum[kSelThreads / 32], s_part[kSelCta];
  __shared__ unsigned long long s_work[kSelThreads / 32], s_pwork[kSelCta];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int b = tid; b < 4096; b += kSelThreads) hist[b] = 0;
  if (tid == 0) s_cnt = 0;
  __syncthreads();

  // pass 1: one read of every fitness: keys (cached in shared memory), the
  // histogram of the top 12 bits of the low keys, the mean and the work.
  // Histogram updates are aggregated per warp (__match_any_sync): fitness
  // values are often discrete, and many lanes hit the same bin.
  // Mean fitness: binary64 searches sum in binary64; binary32 searches sum in
  // binary32 within each warp and in binary64 across warps, so that their
  // selection issues almost no binary64 instruction (GB300's binary64 pipe is
  // thin).
  double sum = 0.0;
  float sum32 = 0.f;
  unsigned long long work = 0;
  for (uint32_t c0 = c_lo; c0 < c_hi; c0 += kSelThreads) {
    const uint32_t c = c0 + tid;
    uint32_t bin = 4096u;
    if (c < c_hi) {
      float F;
      if (p.prec == 0) {
        const double Fw = ((const double *)jb.fit)[c];
        F = (float)Fw;
        sum += Fw;
      } else {
        F = ((const float *)jb.fit)[c];
        sum32 += F;
      }
      const uint32_t meta = jb.meta[c];
      work += meta >> 8;
      uint32_t lo, hi;
      bounds(p, jb, c, F, lo, hi);
      if (cached) {
        s_lo[c - c_lo] = lo;
        s_hi[c - c_lo] = hi;
      }
      bin = lo >> 20;
    }
    const uint32_t peers = __match_any_sync(kFull, bin);
    if (bin < 4096u && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
  }
  if (jb.update_record) {
    if (p.prec == 0) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum32 += __shfl_xor_sync(kFull, sum32, o);
      sum = (double)sum32;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) work += __shfl_xor_sync(kFull, work, o);
    if (lane == 0) {
      s_sum[wid] = sum;
      s_work[wid] = work;
    }
  }
  cl.sync();  // every CTA's histogram is final; the leader's counter is zero

  // tau = the k-th largest low key with its last 8 bits cleared (top 12 bits,
  // then the next 12), so tau <= the exact k-th largest and at least k circuits
  // have F_lo >= tau (a lower tau only adds candidates)
  cluster_find_bin(cl, hist, tot, s_stot, s_wsum, k, &s_bin, &s_rem);
  const uint32_t b1 = s_bin, rem = s_rem;
  for (int b = tid; b < 4096; b += kSelThreads) hist[b] = 0;
  __syncthreads();
  for (uint32_t c0 = c_lo; c0 < c_hi; c0 += kSelThreads) {
    const uint32_t c = c0 + tid;
    uint32_t bin = 4096u;
    if (c < c_hi) {
      uint32_t lo, hi;
      if (cached) lo = s_lo[c - c_lo];
      else {
        const float F = p.prec == 0 ? (float)((const double *)jb.fit)[c] : ((const float *)jb.fit)[c];
        bounds(p, jb, c, F, lo, hi);
      }
      if ((lo >> 20) == b1) bin = (lo >> 8) & 4095u;
    }
    const uint32_t peers = __match_any_sync(kFull, bin);
    if (bin < 4096u && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
  }
  // every CTA has read the slice counts of the first search (their owner may
  // now overwrite them) and every fine histogram is final
  cl.sync();
  cluster_find_bin(cl, hist, tot, s_stot, s_wsum, rem, &s_bin, &s_rem);
  const uint32_t tau = (b1 << 20) | (s_bin << 8);

  // candidates: F_hi >= tau, slots from the leader's counter
  uint32_t *cnt0 = cl.map_shared_rank(&s_cnt, 0);
  for (uint32_t c0 = c_lo; c0 < c_hi; c0 += kSelThreads) {
    const uint32_t c = c0 + tid;
    bool take = false;
    if (c < c_hi) {
      uint32_t lo, hi;
      if (cached) hi = s_hi[c - c_lo];
      else {
        const float F = p.prec == 0 ? (float)((const double *)jb.fit)[c] : ((const float *)jb.fit)[c];
        bounds(p, jb, c, F, lo, hi);
      }
      take = hi >= tau;
    }
    const uint32_t bal = __ballot_sync(kFull, take);
    uint32_t wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(cnt0, __popc(bal));
    wbase = __shfl_sync(kFull, wbase, 0);
    if (take) {
      const uint32_t slot = wbase + __popc(bal & ((1u << lane) - 1));
      p.cand[slot] = c;
      // binary64 searches: the final value; binary32 searches: the binary32
      // value, which the rescoring checks against the guard band and replaces
      p.cand_f[slot] = p.prec == 0 ? ((const double *)jb.fit)[c]
                                   : (double)((const float *)jb.fit)[c];
    }
  }
  // this CTA's share of the mean and the work, to the leader
  if (jb.update_record && wid == 0) {
    double t = lane < kSelThreads / 32 ? s_sum[lane] : 0.0;
    unsigned long long wt = lane < kSelThreads / 32 ? s_work[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(kFull, t, o);
      wt += __shfl_xor_sync(kFull, wt, o);
    }
    if (lane == 0) {
      cl.map_shared_rank(s_part, 0)[rank] = t;
      cl.map_shared_rank(s_pwork, 0)[rank] = wt;
    }
  }
  cl.sync();  // every candidate is counted and written; the shares delivered
  if (rank != 0) return;
  const uint32_t M = s_cnt;
  if (tid == 0) {
    *p.cand_n = M;
    s_base = (p.prec == 0) ? 0u : atomicAdd(g.rescore_n, M);
    if (jb.update_record) {
      double t = 0.0;
      unsigned long long wt = 0;
      for (int q = 0; q < kSelCta; ++q) {
        t += s_part[q];
        wt += s_pwork[q];
      }
      p.rec->mean_fitness = n ? t / (double)n : 0.0;
      p.rec->useful_flops = wt;
    }
  }
  __syncthreads();
  if (p.prec != 0)
    for (uint32_t s = tid; s < M; s += kSelThreads) g.rescore_list[s_base + s] = (jb.prob << 20) | s;
}

__device__ __forceinline__ bool key_less(unsigned long long ah, unsigned long long al,
                                         unsigned long long bh, unsigned long long bl) {
  return ah < bh || (ah == bh && al < bl);
}

// Best-so-far record and report fields of a ranked generation (one warp):
// lane 0 decides, the warp copies the gates of an improvement.
__device__ __forceinline__ void record_best(const DevProblem &p, const RankJob &jb, const DevGlobal &g,
                                            uint32_t gen, unsigned long long kh0,
                                            unsigned long long kl0, uint32_t kept, int lane) {
  const unsigned long long kMaxKey = ~0ull;
  Best *rec = p.rec;
  const bool valid = kept > 0 && kh0 < kMaxKey - 1;
  const double F = valid ? dkey_inv(~kh0) : 0.0;
  const uint32_t c = (uint32_t)(kl0 & 0xffffffffu);
  const uint32_t cost = (uint32_t)(kl0 >> 32);
  int improve = 0;
  if (lane == 0) {
    rec->generation = gen + 1;
    rec->error_word |= *g.err;
    if (jb.pipelined) *g.ranked = gen + 1;
    if (valid) {
      rec->gen_best_fitness = F;
      if (F > rec->best_fitness || (F == rec->best_fitness && cost < rec->best_cost)) {
        rec->best_fitness = F;
        rec->best_cost = cost;
        rec->best_gen = gen;
        rec->best_len = p.L;
        improve = 1;
      }
    }
  }
  improve = __shfl_sync(kFull, improve, 0);
  if (improve) {
    const uint8_t *gs = jb.gsrc + (size_t)c * p.L;
    for (uint32_t t = lane; t < 64; t += 32) rec->best_gates[t] = t < p.L ? gs[t] : 0;
    if (p.ising && jb.asrc) {
      const float2 *as = jb.asrc + (size_t)c * p.L;
      for (uint32_t t = lane; t < 64; t += 32)
        rec->best_amps[t] = t < p.L ? as[t] : make_float2(0.f, 0.f);
    }
  }
}

// compare-exchange of two 128-bit keys held as (hi, lo) pairs
__device__ __forceinline__ void keep_side(unsigned long long &h, unsigned long long &l,
                                          unsigned long long ph, unsigned long long pl,
                                          bool keep_min) {
  const bool pless = key_less(ph, pl, h, l);
  if (keep_min == pless) {
    h = ph;
    l = pl;
  }
}

// err_out != NULL: block 0 also writes the error word there (the batch path,
// whose jobs' top-k lists are written in place) and clears the rescoring
// queue for the next ranking on the same scratch
__global__ void __launch_bounds__(kSortThreads) k_rank_sort(const DevProblem *__restrict__ probs,
                                                            const RankJob *__restrict__ jobs,
                                                            RankJob single, DevGlobal g,
                                                            Ranked *err_out) {
  wait_predecessor();  // the candidates and their binary64 fitness
  if (err_out && blockIdx.x == 0 && threadIdx.x == 0) {
    Ranked e{};
    e.circuit = *g.err;  // every kernel that sets it has completed
    *err_out = e;
    *g.rescore_n = 0;
  }
  RankJob jb = jobs ? jobs[blockIdx.x] : single;
  const DevProblem &p = probs[jb.prob];
  uint32_t gen = 0;
  if (jb.pipelined) {
    if (!*g.rank_active) return;
    gen = *g.gen - 1u;  // the generation being ranked
    jb = resolve(jb, p, gen + 1u);
  } else if (jb.update_record) {
    gen = *g.gen;
  }
  const uint32_t n = jb.n;
  const uint32_t k = p.k < n ? p.k : n;
  const uint32_t M = *p.cand_n;
  __shared__ unsigned long long kh[kSortN], kl[kSortN];
  const int tid = threadIdx.x;
  const unsigned long long kMaxKey = ~0ull;
  if (M <= 64) {
    // one warp: 64 keys, two per lane (index lane and lane + 32), bitonic by
    // shuffles; no block barriers
    if (tid >= 32) return;
    const int lane = tid;
    unsigned long long h[2], l[2];
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const uint32_t i = lane + 32 * sl;
      h[sl] = kMaxKey;
      l[sl] = kMaxKey;
      if (i < M) {
        const uint32_t c = p.cand[i];
        const double F = p.cand_f[i];
        h[sl] = (F == F) ? ~dkey(F) : kMaxKey - 1;
        l[sl] = ((unsigned long long)(jb.meta[c] & 0xffu) << 32) | c;
      }
    }
#pragma unroll
    for (uint32_t size = 2; size <= 64; size <<= 1) {
#pragma unroll
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        if (stride == 32) {  // partner is the lane's other key
          const bool asc = true;
          const unsigned long long h0 = h[0], l0 = l[0];
          keep_side(h[0], l[0], h[1], l[1], asc);
          keep_side(h[1], l[1], h0, l0, !asc);
        } else {
#pragma unroll
          for (int sl = 0; sl < 2; ++sl) {
            const uint32_t i = lane + 32 * sl;
            const unsigned long long ph = __shfl_xor_sync(kFull, h[sl], stride);
            const unsigned long long pl = __shfl_xor_sync(kFull, l[sl], stride);
            const bool asc = (i & size) == 0, lower = (i & stride) == 0;
            keep_side(h[sl], l[sl], ph, pl, lower == asc);
          }
        }
      }
    }
    const uint32_t kept = M < k ? M : k;
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const uint32_t i = lane + 32 * sl;
      if (i < kept) {
        Ranked rr;
        rr.circuit = (uint32_t)(l[sl] & 0xffffffffu);
        rr.cost = (uint32_t)(l[sl] >> 32);
        rr.fitness = (h[sl] >= kMaxKey - 1) ? __longlong_as_double(0x7ff8000000000000ll)
                                           : dkey_inv(~h[sl]);
        p.topk_out[i] = rr;
      }
    }
    if (jb.update_record) {
      const unsigned long long h0 = __shfl_sync(kFull, h[0], 0), l0 = __shfl_sync(kFull, l[0], 0);
      record_best(p, jb, g, gen, h0, l0, kept, lane);
    }
    return;
  }
  uint32_t kept = 0, next = 0;
  // ascending order of (~dkey(F), cost << 32 | c) == (F desc, cost asc, c asc);
  // each round sorts the kept top-k plus the next candidates with a bitonic
  // network sized to the next power of two of their count
  do {
    const uint32_t added = (M - next) < (uint32_t)(kSortN - kept) ? (M - next) : (kSortN - kept);
    uint32_t S = 2;
    while (S < kept + added) S <<= 1;
    for (uint32_t s = kept + tid; s < S; s += kSortThreads) {
      const uint32_t src = next + (s - kept);
      if (s < kept + added) {
        const uint32_t c = p.cand[src];
        const double F = p.cand_f[src];
        const uint32_t cost = jb.meta[c] & 0xffu;
        kh[s] = (F == F) ? ~dkey(F) : kMaxKey - 1;
        kl[s] = ((unsigned long long)cost << 32) | c;
      } else {
        kh[s] = kMaxKey;
        kl[s] = kMaxKey;
      }
    }
    next += added;
    __syncthreads();
    for (uint32_t size = 2; size <= S; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = tid; i < S; i += kSortThreads) {
          const uint32_t jx = i ^ stride;
          if (jx > i) {
            const bool asc = (i & size) == 0;
            const bool lt = key_less(kh[jx], kl[jx], kh[i], kl[i]);
            if (lt == asc) {
              unsigned long long t = kh[i];
              kh[i] = kh[jx];
              kh[jx] = t;
              t = kl[i];
              kl[i] = kl[jx];
              kl[jx] = t;
            }
          }
        }
        __syncthreads();
      }
    }
    const uint32_t have = kept + added;
    kept = have < k ? have : k;
    __syncthreads();
  } while (next < M);

  for (uint32_t s = tid; s < kept; s += kSortThreads) {
    Ranked r;
    r.circuit = (uint32_t)(kl[s] & 0xffffffffu);
    r.cost = (uint32_t)(kl[s] >> 32);
    r.fitness = (kh[s] >= kMaxKey - 1) ? __longlong_as_double(0x7ff8000000000000ll)
                                      : dkey_inv(~kh[s]);
    p.topk_out[s] = r;
  }
  if (jb.update_record && tid < 32) record_best(p, jb, g, gen, kh[0], kl[0], kept, tid);
}

// top-k lists of a batch of ranked jobs, back to back, and the error word
__global__ void __launch_bounds__(128) k_gather_topk(const DevProblem *__restrict__ probs,
                                                     const RankJob *__restrict__ jobs,
                                                     const uint32_t *__restrict__ koff,
                                                     uint32_t n_jobs, Ranked *out, DevGlobal g) {
  wait_predecessor();  // the sorted lists
  for (uint32_t m = blockIdx.x; m < n_jobs; m += gridDim.x) {
    const RankJob jb = jobs[m];
    const DevProblem &p = probs[jb.prob];
    const uint32_t k = p.k < jb.n ? p.k : jb.n;
    for (uint32_t s = threadIdx.x; s < k; s += blockDim.x) out[koff[m] + s] = p.topk_out[s];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ranked e{};
    e.circuit = *g.err;
    out[koff[n_jobs]] = e;
  }
}

__global__ void k_finish(DevGlobal g) {
  wait_predecessor();  // the ranking and the update read the counter
  *g.gen += 1;
  *g.rescore_n = 0;
}

__global__ void k_reset_counter(DevGlobal g) { *g.rescore_n = 0; }

// ------------------------------------------------------------ batch copies
// The batched host call's copies between page-locked host memory (through its
// device mapping) and the slot's device staging, done by the GPU's threads so
// that the call's graph holds kernels only.

// bytes [0, n) from src to dst, grid-stride, in 16-, 4- or 1-byte words as the
// addresses and the length allow
__device__ __forceinline__ void copy_span(char *dst, const char *src, size_t n, size_t t0,
                                          size_t nt) {
  if ((((uintptr_t)dst | (uintptr_t)src | n) & 15u) == 0) {
    for (size_t i = t0; i < n / 16; i += nt)
      reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
  } else if ((((uintptr_t)dst | (uintptr_t)src | n) & 3u) == 0) {
    for (size_t i = t0; i < n / 4; i += nt)
      reinterpret_cast<uint32_t *>(dst)[i] = reinterpret_cast<const uint32_t *>(src)[i];
  } else {
    for (size_t i = t0; i < n; i += nt) dst[i] = src[i];
  }
}

__global__ void __launch_bounds__(256) k_copy_in(char *dst, const char *src, size_t n) {
  copy_span(dst, src, n, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
            (size_t)gridDim.x * blockDim.x);
}

// The call's outputs to the host: the fitness (fit_n bytes) and the top-k
// lists (list_n bytes); then the last block to finish writes the error word
// to its host slot, after every block's writes are visible system-wide (a
// system fence before each block's arrival on the counter, which the last
// block resets for the slot's next call).  The host polls that word.
__global__ void __launch_bounds__(256) k_copy_out(char *h_fit, const char *d_fit, size_t fit_n,
                                                  char *h_list, const char *d_list,
                                                  size_t list_n, uint32_t *h_errw,
                                                  const uint32_t *d_errw, uint32_t *count) {
  wait_predecessor();  // the sort's lists and error word
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nt = (size_t)gridDim.x * blockDim.x;
  if (fit_n) copy_span(h_fit, d_fit, fit_n, t0, nt);
  if (list_n) copy_span(h_list, d_list, list_n, t0, nt);
  __threadfence_system();
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *count = 0;
    __threadfence_system();
    *(volatile uint32_t *)h_errw = *(volatile const uint32_t *)d_errw;
  }
}

cudaError_t launch_copy_in(void *dst, const void *src, size_t n, uint32_t num_sms,
                           cudaStream_t st) {
  if (!n) return cudaSuccess;
  uint64_t blocks = (n / 16 + 255) / 256;
  if (blocks > (uint64_t)num_sms * 4) blocks = (uint64_t)num_sms * 4;
  if (!blocks) blocks = 1;
  k_copy_in<<<(uint32_t)blocks, 256, 0, st>>>((char *)dst, (const char *)src, n);
  return cudaGetLastError();
}

cudaError_t launch_copy_out(void *h_fit, const void *d_fit, size_t fit_n, void *h_list,
                            const void *d_list, size_t list_n, uint32_t *h_errw,
                            const uint32_t *d_errw, uint32_t *count, uint32_t num_sms,
                            cudaStream_t st) {
  const size_t n = fit_n > list_n ? fit_n : list_n;
  uint64_t blocks = (n / 16 + 255) / 256;
  if (blocks > (uint64_t)num_sms * 4) blocks = (uint64_t)num_sms * 4;
  if (!blocks) blocks = 1;
  k_copy_out<<<(uint32_t)blocks, 256, 0, st>>>((char *)h_fit, (const char *)d_fit, fit_n,
                                               (char *)h_list, (const char *)d_list, list_n,
                                               h_errw, d_errw, count);
  return cudaGetLastError();
}

cudaError_t launch_rank_select(const DevProblem *probs, const RankJob *jobs, uint32_t n_jobs,
                               const RankJob &single, const DevGlobal &g, cudaStream_t st,
                               uint32_t max_n) {
  if (!n_jobs) return cudaSuccess;
  if (max_n < kSelClusterFrom)
    k_rank_select<<<n_jobs, kRankThreads, kSelectSmem, st>>>(probs, jobs, single, g);
  else
    k_rank_select_cl<<<n_jobs * kSelCta, kSelThreads, 0, st>>>(probs, jobs, single, g);
  return cudaGetLastError();
}

cudaError_t launch_rank_sort(const DevProblem *probs, const RankJob *jobs, uint32_t n_jobs,
                             const RankJob &single, const DevGlobal &g, cudaStream_t st,
                             Ranked *err_out) {
  if (!n_jobs) return cudaSuccess;
  k_rank_sort<<<n_jobs, kSortThreads, 0, st>>>(probs, jobs, single, g, err_out);
  return cudaGetLastError();
}

bool is_select_kernel(const void *f) {
  return f == (const void *)k_rank_select || f == (const void *)k_rank_select_cl;
}
bool batch_kernel_waits(const void *f) {
  return f == (const void *)k_rank_select || f == (const void *)k_copy_out;
}
bool rank_kernel_waits(const void *f) {
  return f == (const void *)k_rank_sort || f == (const void *)k_finish ||
         f == (const void *)k_gather_topk;
}

cudaError_t rank_init() {
  return cudaFuncSetAttribute(k_rank_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSelectSmem);
}

// 1024-thread CTAs of a selection launch, in quarters of an SM's threads
uint32_t select_quarters(uint32_t n_jobs, uint32_t max_n) {
  return max_n < kSelClusterFrom ? 2 * n_jobs : n_jobs * kSelCta / 2;
}

cudaError_t launch_finish(const DevGlobal &g, cudaStream_t st) {
  k_finish<<<1, 1, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_gather_topk(const DevProblem *probs, const RankJob *jobs, const uint32_t *koff,
                               uint32_t n_jobs, Ranked *out, const DevGlobal &g, cudaStream_t st) {
  const uint32_t blocks = n_jobs ? (n_jobs < 1024 ? n_jobs : 1024) : 1;
  k_gather_topk<<<blocks, 128, 0, st>>>(probs, jobs, koff, n_jobs, out, g);
  return cudaGetLastError();
}

cudaError_t launch_reset_counter(const DevGlobal &g, cudaStream_t st) {
  k_reset_counter<<<1, 1, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace qe
