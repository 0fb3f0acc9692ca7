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
// One CTA per search does the selection (4-pass radix select of the k-th
// largest F_lo key) and, in a second launch, the sort (bitonic, in chunks of
// 2048 so any number of candidates fits in shared memory).
#include "qe_dev.cuh"
#include "qe_host.h"

namespace qe {

constexpr int kRankThreads = 1024;
constexpr int kSortN = 2048;

__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// binary64 fitness interval of circuit c as a pair of float keys
__device__ __forceinline__ void bounds(const DevProblem &p, const RankJob &jb, uint32_t c,
                                       uint32_t &klo, uint32_t &khi) {
  if (p.prec == 0) {
    const double F = ((const double *)jb.fit)[c];
    if (!(F == F)) {
      klo = khi = 1u;  // NaN ranks last
      return;
    }
    klo = fkey(__double2float_rd(F));
    khi = fkey(__double2float_ru(F));
    return;
  }
  const float F = ((const float *)jb.fit)[c];
  if (!(F == F)) {
    klo = khi = 1u;
    return;
  }
  float pen = 0.f;
  if (p.cost_weight != 0.0) {
    const uint32_t cost = jb.meta[c] & 0xffu;
    pen = (float)(p.cost_weight * ((double)cost / (double)p.L));
  }
  const float f = F + pen;
  const float t = 1.f - f;
  const float d = t * t;
  const float dl = fmaxf(0.f, d - p.eps_d), dh = d + p.eps_d;
  const float fhi = 1.f - sqrtf(dl), flo = 1.f - sqrtf(dh);
  const float slop = 2e-6f;
  klo = fkey(flo - pen - slop);
  khi = fkey(fhi - pen + slop);
}

__global__ void __launch_bounds__(kRankThreads) k_rank_select(const DevProblem *__restrict__ probs,
                                                              const RankJob *__restrict__ jobs,
                                                              RankJob single, DevGlobal g) {
  const RankJob jb = jobs ? jobs[blockIdx.x] : single;
  const DevProblem &p = probs[jb.prob];
  const uint32_t n = jb.n;
  const uint32_t k = p.k < n ? p.k : n;
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_bin, s_rem, s_cnt, s_base;
  __shared__ float s_sum[kRankThreads / 32];
  __shared__ unsigned long long s_work[kRankThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  // mean fitness and useful work (report fields)
  if (jb.update_record) {
    float sum = 0.f;
    unsigned long long work = 0;
    for (uint32_t c = tid; c < n; c += kRankThreads) {
      sum += p.prec == 0 ? (float)((const double *)jb.fit)[c] : ((const float *)jb.fit)[c];
      work += jb.meta[c] >> 8;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sum += __shfl_xor_sync(kFull, sum, o);
      work += __shfl_xor_sync(kFull, work, o);
    }
    if (lane == 0) {
      s_sum[wid] = sum;
      s_work[wid] = work;
    }
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      unsigned long long wt = 0;
      for (int w = 0; w < kRankThreads / 32; ++w) {
        tot += (double)s_sum[w];
        wt += s_work[w];
      }
      p.rec->mean_fitness = n ? tot / (double)n : 0.0;
      p.rec->useful_flops = wt;
    }
  }

  // radix select: tau = k-th largest low key
  uint32_t prefix = 0, mask = 0;
  if (tid == 0) s_rem = k;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += kRankThreads) hist[b] = 0;
    __syncthreads();
    for (uint32_t c = tid; c < n; c += kRankThreads) {
      uint32_t lo, hi;
      bounds(p, jb, c, lo, hi);
      if ((lo & mask) == prefix) atomicAdd(&hist[(lo >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t rem = s_rem, b = 255;
      for (;; --b) {
        const uint32_t h = hist[b];
        if (h >= rem || b == 0) break;
        rem -= h;
      }
      s_bin = b;
      s_rem = rem;
    }
    __syncthreads();
    prefix |= s_bin << shift;
    mask |= 255u << shift;
  }
  const uint32_t tau = prefix;

  // candidates: F_hi >= tau
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < n; c0 += kRankThreads) {
    const uint32_t c = c0 + tid;
    bool take = false;
    if (c < n) {
      uint32_t lo, hi;
      bounds(p, jb, c, lo, hi);
      take = hi >= tau;
    }
    const uint32_t bal = __ballot_sync(kFull, take);
    uint32_t wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(&s_cnt, __popc(bal));
    wbase = __shfl_sync(kFull, wbase, 0);
    if (take) {
      const uint32_t slot = wbase + __popc(bal & ((1u << lane) - 1));
      p.cand[slot] = c;
      if (p.prec == 0) p.cand_f[slot] = ((const double *)jb.fit)[c];
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

__device__ __forceinline__ bool key_less(unsigned long long ah, unsigned long long al,
                                         unsigned long long bh, unsigned long long bl) {
  return ah < bh || (ah == bh && al < bl);
}

__global__ void __launch_bounds__(kRankThreads) k_rank_sort(const DevProblem *__restrict__ probs,
                                                            const RankJob *__restrict__ jobs,
                                                            RankJob single, DevGlobal g) {
  const RankJob jb = jobs ? jobs[blockIdx.x] : single;
  const DevProblem &p = probs[jb.prob];
  const uint32_t n = jb.n;
  const uint32_t k = p.k < n ? p.k : n;
  const uint32_t M = *p.cand_n;
  __shared__ unsigned long long kh[kSortN], kl[kSortN];
  const int tid = threadIdx.x;
  const unsigned long long kMaxKey = ~0ull;
  uint32_t kept = 0, next = 0;
  // ascending order of (~dkey(F), cost << 32 | c) == (F desc, cost asc, c asc)
  do {
    for (uint32_t s = tid; s < (uint32_t)kSortN; s += kRankThreads) {
      if (s >= kept) {
        const uint32_t src = next + (s - kept);
        if (src < M) {
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
    }
    const uint32_t added = (M - next) < (uint32_t)(kSortN - kept) ? (M - next) : (kSortN - kept);
    next += added;
    __syncthreads();
    for (uint32_t size = 2; size <= (uint32_t)kSortN; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = tid; i < (uint32_t)kSortN; i += kRankThreads) {
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

  for (uint32_t s = tid; s < kept; s += kRankThreads) {
    Ranked r;
    r.circuit = (uint32_t)(kl[s] & 0xffffffffu);
    r.cost = (uint32_t)(kl[s] >> 32);
    r.fitness = (kh[s] >= kMaxKey - 1) ? __longlong_as_double(0x7ff8000000000000ll)
                                      : dkey_inv(~kh[s]);
    p.topk_out[s] = r;
  }
  if (tid == 0 && jb.update_record) {
    Best *rec = p.rec;
    const uint32_t gen = *g.gen;
    rec->generation = gen + 1;
    rec->error_word |= *g.err;
    if (kept > 0 && kh[0] < kMaxKey - 1) {
      const double F = dkey_inv(~kh[0]);
      const uint32_t c = (uint32_t)(kl[0] & 0xffffffffu);
      const uint32_t cost = (uint32_t)(kl[0] >> 32);
      rec->gen_best_fitness = F;
      if (F > rec->best_fitness || (F == rec->best_fitness && cost < rec->best_cost)) {
        rec->best_fitness = F;
        rec->best_cost = cost;
        rec->best_gen = gen;
        rec->best_len = p.L;
        const uint8_t *gs = jb.gsrc + (size_t)c * p.L;
        for (uint32_t t = 0; t < 64; ++t) rec->best_gates[t] = t < p.L ? gs[t] : 0;
      }
    }
  }
}

__global__ void k_finish(DevGlobal g) {
  *g.gen += 1;
  *g.rescore_n = 0;
}

__global__ void k_reset_counter(DevGlobal g) { *g.rescore_n = 0; }

cudaError_t launch_rank_select(const DevProblem *probs, const RankJob *jobs, uint32_t n_jobs,
                               const RankJob &single, const DevGlobal &g, cudaStream_t st) {
  if (!n_jobs) return cudaSuccess;
  k_rank_select<<<n_jobs, kRankThreads, 0, st>>>(probs, jobs, single, g);
  return cudaGetLastError();
}

cudaError_t launch_rank_sort(const DevProblem *probs, const RankJob *jobs, uint32_t n_jobs,
                             const RankJob &single, const DevGlobal &g, cudaStream_t st) {
  if (!n_jobs) return cudaSuccess;
  k_rank_sort<<<n_jobs, kRankThreads, 0, st>>>(probs, jobs, single, g);
  return cudaGetLastError();
}

cudaError_t launch_finish(const DevGlobal &g, cudaStream_t st) {
  k_finish<<<1, 1, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_reset_counter(const DevGlobal &g, cudaStream_t st) {
  k_reset_counter<<<1, 1, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace qe
