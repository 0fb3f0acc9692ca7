// k_ga.cu -- the classical GA of the paper's comparison (Sec. V-B) on the same
// evaluation path: integer gate-string genomes, stochastic universal sampling,
// one-point crossover, per-gene mutation, elitism.  On the Ising library the
// genes are (gate, angle) pairs bred as the paper's comparator does (Sec. V-B):
// angles start on the 2 pi / Q lattice, crossover takes two points, and a gene
// not drawn fresh may have its angle turned by a multiple of range / Q.
//
// Per generation g (genome in gate_idx buffer g & 1, already evaluated into
// fit/meta buffer g & 1 by the circuit kernel without sampling):
//   k_ga_tiles one CTA per tile of 1024 circuits: SUS weights
//              floor(clamp(F,0,1) 2^32), their inclusive prefix sums within the
//              tile (integers, so exact in any order), the tile's total and its
//              elite = best by (F desc, cost asc, index asc) in the working
//              precision;
//   k_ga_top   one CTA per search: the tiles' offsets (exclusive scan of their
//              totals), the total W and the search's elite;
//   k_ga_parents one thread per circuit c: SUS pointers are s + m floor(W/P),
//              and child m's parent is the first c with cum[c] > pointer, so c
//              writes its own children's parent index (the m whose pointer
//              lies in [cum[c-1], cum[c])) -- no search per child;
//   k_ga_next  one warp per pair of children: parents from that table,
//              one-point crossover at 1 + below(u, L-1) (Ising: genes in
//              [min, max) of two such points swapped), per-gene mutation,
//              child 0 = the elite; written to gate_idx buffer (g+1) & 1
//              (Ising angles: amps buffer (g+1) & 1).
// Philox streams as the oracle: (0, 0, g) for the SUS offset, (pair, 1, g) for
// the cut, (child, 2 + t, g) for gene t's mutation, all with stream 4; the
// initial genome draws (c, t, 0) with stream 5.
#include "qe_dev.cuh"
#include "qe_host.h"

namespace qe {

constexpr int kGaThreads = 1024;

__device__ __forceinline__ uint32_t find_ga(const uint32_t *prefix, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double ga_fitness(const DevProblem &p, uint32_t par, uint32_t c) {
  return p.prec == 0 ? p.fit64[(size_t)par * p.P + c] : (double)p.fit32[(size_t)par * p.P + c];
}

// SUS weight: max(F, 0) clamped to 1 as a 32-bit fixed-point integer
__device__ __forceinline__ unsigned long long sus_weight(double F) {
  if (!(F > 0.0)) return 0ull;
  const double x = F < 1.0 ? F : 1.0;
  return (unsigned long long)floor(__dmul_rn(x, 4294967296.0));
}

// a before b in the ranking key (F desc, cost asc, index asc); NaN last
__device__ __forceinline__ bool ga_better(double Fa, uint32_t ca, uint32_t ia, double Fb,
                                          uint32_t cb, uint32_t ib) {
  const bool na = !(Fa == Fa), nb = !(Fb == Fb);
  if (na != nb) return nb;
  if (!na && Fa != Fb) return Fa > Fb;
  if (ca != cb) return ca < cb;
  return ia < ib;
}

// keep the better of (F, cost, idx) and lane l ^ o's candidate
__device__ __forceinline__ void elite_shfl(double &F, uint32_t &cost, uint32_t &idx, int o) {
  const double oF = __shfl_xor_sync(kFull, F, o);
  const uint32_t oc = __shfl_xor_sync(kFull, cost, o), oi = __shfl_xor_sync(kFull, idx, o);
  if (oi != 0xffffffffu && (idx == 0xffffffffu || ga_better(oF, oc, oi, F, cost, idx))) {
    F = oF;
    cost = oc;
    idx = oi;
  }
}

// The tile of 1024 circuits of GA search ids[q] that block b covers, from the
// searches' tile prefix sums
__device__ __forceinline__ void ga_tile_of(const uint32_t *tprefix, uint32_t n_ga, uint32_t b,
                                           uint32_t &q, uint32_t &t) {
  q = find_ga(tprefix, n_ga, b);
  t = b - __ldg(tprefix + q);
}

// one tile: weights, their prefix sums within the tile, the tile's total and elite
__global__ void __launch_bounds__(kGaThreads) k_ga_tiles(const DevProblem *__restrict__ probs,
                                                         const uint32_t *__restrict__ ids,
                                                         const uint32_t *__restrict__ tprefix,
                                                         uint32_t n_ga, DevGlobal g) {
  uint32_t q, t;
  ga_tile_of(tprefix, n_ga, blockIdx.x, q, t);
  const DevProblem &p = probs[ids[q]];
  const uint32_t par = *g.gen & 1u;
  const uint32_t P = p.P, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t c = t * kGaThreads + tid;
  __shared__ unsigned long long s_sum[kGaThreads / 32], s_tot;
  __shared__ double s_F[kGaThreads / 32];
  __shared__ uint32_t s_cost[kGaThreads / 32], s_idx[kGaThreads / 32];
  double bF = 0.0;
  uint32_t bcost = 0xffffffffu, bidx = 0xffffffffu;
  unsigned long long w = 0;
  if (c < P) {
    bF = ga_fitness(p, par, c);
    w = sus_weight(bF);
    bcost = p.meta[(size_t)par * P + c] & 0xffu;
    bidx = c;
  }
  unsigned long long v = w;  // warp inclusive scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(kFull, v, o);
    if (lane >= (uint32_t)o) v += u;
  }
  if (lane == 31) s_sum[wid] = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) elite_shfl(bF, bcost, bidx, o);
  if (lane == 0) {
    s_F[wid] = bF;
    s_cost[wid] = bcost;
    s_idx[wid] = bidx;
  }
  __syncthreads();
  if (wid == 0) {
    const unsigned long long x0 = s_sum[lane];
    unsigned long long x = x0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, x, o);
      if (lane >= (uint32_t)o) x += u;
    }
    s_sum[lane] = x - x0;  // exclusive prefix of the warp totals
    if (lane == 31) s_tot = x;
    double F = s_F[lane];
    uint32_t cost = s_cost[lane], idx = s_idx[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) elite_shfl(F, cost, idx, o);
    if (lane == 0) {
      s_F[0] = F;
      s_cost[0] = cost;
      s_idx[0] = idx;
    }
  }
  __syncthreads();
  if (c < P) p.ga_cum[c] = s_sum[wid] + v;
  if (tid == 0) {
    GaTile tl;
    tl.sum = s_tot;
    tl.F = s_F[0];
    tl.cost = s_cost[0];
    tl.idx = s_idx[0];
    p.ga_tiles[t] = tl;
  }
}

// one search: the tiles' offsets (in place of their totals), W and the elite
__global__ void __launch_bounds__(kGaThreads) k_ga_top(const DevProblem *__restrict__ probs,
                                                       const uint32_t *__restrict__ ids) {
  const DevProblem &p = probs[ids[blockIdx.x]];
  const uint32_t nt = (p.P + kGaThreads - 1) / kGaThreads;  // <= 1024 (P <= 2^20)
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ unsigned long long s_sum[kGaThreads / 32], s_tot;
  __shared__ double s_F[kGaThreads / 32];
  __shared__ uint32_t s_cost[kGaThreads / 32], s_idx[kGaThreads / 32];
  unsigned long long w = 0;
  double bF = 0.0;
  uint32_t bcost = 0xffffffffu, bidx = 0xffffffffu;
  if (tid < nt) {
    const GaTile tl = p.ga_tiles[tid];
    w = tl.sum;
    bF = tl.F;
    bcost = tl.cost;
    bidx = tl.idx;
  }
  unsigned long long v = w;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(kFull, v, o);
    if (lane >= (uint32_t)o) v += u;
  }
  if (lane == 31) s_sum[wid] = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) elite_shfl(bF, bcost, bidx, o);
  if (lane == 0) {
    s_F[wid] = bF;
    s_cost[wid] = bcost;
    s_idx[wid] = bidx;
  }
  __syncthreads();
  if (wid == 0) {
    const unsigned long long x0 = s_sum[lane];
    unsigned long long x = x0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, x, o);
      if (lane >= (uint32_t)o) x += u;
    }
    s_sum[lane] = x - x0;
    if (lane == 31) s_tot = x;
    double F = s_F[lane];
    uint32_t cost = s_cost[lane], idx = s_idx[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) elite_shfl(F, cost, idx, o);
    if (lane == 0) p.ga_info[1] = idx;  // elite
  }
  __syncthreads();
  if (tid < nt) p.ga_tiles[tid].sum = s_sum[wid] + v - w;  // tiles before this one
  if (tid == 0) p.ga_info[0] = s_tot;                       // W
}

// one circuit c: the children whose SUS pointer s + m D lies in
// [cum[c-1], cum[c]) get parent c (D = floor(W/P); no table when D = 0)
__global__ void __launch_bounds__(kGaThreads) k_ga_parents(const DevProblem *__restrict__ probs,
                                                           const uint32_t *__restrict__ ids,
                                                           const uint32_t *__restrict__ tprefix,
                                                           uint32_t n_ga, DevGlobal g) {
  uint32_t q, t;
  ga_tile_of(tprefix, n_ga, blockIdx.x, q, t);
  const DevProblem &p = probs[ids[q]];
  const uint32_t P = p.P;
  const uint32_t c = t * kGaThreads + threadIdx.x;
  if (c >= P) return;
  const unsigned long long W = p.ga_info[0];
  const unsigned long long D = W / P;
  if (D == 0) return;
  const uint32_t gen = *g.gen;
  const uint4 u = draw(p, 0, 0, gen, kStGa);
  const unsigned long long r64 = ((unsigned long long)u.y << 32) | u.x;
  const unsigned long long s0 = __umul64hi(r64, D);
  const unsigned long long incl = p.ga_cum[c] + p.ga_tiles[t].sum;
  unsigned long long excl = 0;
  if (c > 0) {
    const uint32_t tp = (c - 1) / kGaThreads;
    excl = p.ga_cum[c - 1] + p.ga_tiles[tp].sum;
  }
  // children m with s0 + m D < x
  auto below_ptr = [&](unsigned long long x) -> unsigned long long {
    return x <= s0 ? 0ull : (x - s0 + D - 1) / D;
  };
  unsigned long long m = below_ptr(excl), m_end = below_ptr(incl);
  if (m_end > P) m_end = P;
  for (; m < m_end; ++m) p.ga_parent[m] = c;
}

// Per-gene mutation: word x decides a fresh gene (gate from y; Ising: its
// angle from z on the 2 pi / Q lattice); for an Ising gene kept, word w decides
// a turn of its angle by +-m range / Q (m from z, the sign from y's low bit),
// rotated in binary32 in the order of the encoding's qubit mutation
__device__ __forceinline__ void ga_mutate(const DevProblem &p, const DevGlobal &g, const uint4 v,
                                          bool ising, uint8_t &gene, float2 &amp) {
  if ((unsigned long long)v.x < p.ga_T) {
    gene = (uint8_t)below(v.y, p.G);
    if (ising) amp = g.ph_tab[below(v.z, kQ)];
  } else if (ising && (unsigned long long)v.w < p.ga_T) {
    const float2 cs = p.qubit_tab[below(v.z, kQ + 1)];
    const float c = cs.x, s = (v.y & 1u) ? -cs.y : cs.y;
    const float b0 = amp.x, b1 = amp.y;
    amp.x = __fadd_rn(__fadd_rn(0.f, __fmul_rn(c, b0)), __fmul_rn(-s, b1));
    amp.y = __fadd_rn(__fadd_rn(0.f, __fmul_rn(s, b0)), __fmul_rn(c, b1));
  }
}

// first c in [0, P) with cum[c] > ptr (P - 1 if none)
__global__ void __launch_bounds__(256) k_ga_next(const DevProblem *__restrict__ probs,
                                                 const uint32_t *__restrict__ ids,
                                                 const uint32_t *__restrict__ prefix,
                                                 uint32_t n_ga, uint32_t total_pairs, DevGlobal g) {
  const uint32_t gen = *g.gen;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total_pairs; w += nw) {
    const uint32_t q = find_ga(prefix, n_ga, w);
    const DevProblem &p = probs[ids[q]];
    const uint32_t pair = w - prefix[q];
    const uint32_t P = p.P, L = p.L;
    const uint8_t *src = p.gate_idx + (size_t)(gen & 1u) * P * L;
    uint8_t *dst = p.gate_idx + (size_t)((gen + 1u) & 1u) * P * L;
    // Ising genes also carry angles, bred with them
    const bool ising = p.ising != 0;
    const float2 *asrc = ising ? p.amps + (size_t)(gen & 1u) * P * L : nullptr;
    float2 *adst = ising ? p.amps + (size_t)((gen + 1u) & 1u) * P * L : nullptr;
    const uint32_t m0 = 2 * pair, m1 = m0 + 1;
    const unsigned long long W = p.ga_info[0];
    const uint32_t elite = (uint32_t)p.ga_info[1];
    const unsigned long long D = W / P;
    uint32_t a = m0, b = m1 < P ? m1 : m0;
    if (D > 0) {  // SUS parents, from the table k_ga_parents wrote
      a = p.ga_parent[m0];
      if (m1 < P) b = p.ga_parent[m1];
    }
    // gene t of child m0 comes from parent b for t in [lo, hi), else from a
    uint32_t lo = L, hi = L;
    if (m1 < P && L > 1) {
      const uint4 v = draw(p, pair, 1, gen, kStGa);
      const uint32_t x = 1 + below(v.x, L - 1);
      if (ising) {  // two points
        const uint32_t y = 1 + below(v.y, L - 1);
        lo = x < y ? x : y;
        hi = x < y ? y : x;
      } else {  // one point: the tail from x on
        lo = x;
      }
    }
    for (uint32_t t = lane; t < L; t += 32) {
      const bool sw = t >= lo && t < hi;
      const size_t ea = (size_t)(sw ? b : a) * L + t, eb = (size_t)(sw ? a : b) * L + t;
      // child m0
      uint8_t x = src[ea];
      float2 ax = ising ? asrc[ea] : make_float2(0.f, 0.f);
      if (m0 == 0) {
        x = src[(size_t)elite * L + t];
        if (ising) ax = asrc[(size_t)elite * L + t];
      } else {
        ga_mutate(p, g, draw(p, m0, 2 + t, gen, kStGa), ising, x, ax);
      }
      dst[(size_t)m0 * L + t] = x;
      if (ising) adst[(size_t)m0 * L + t] = ax;
      if (m1 < P) {
        uint8_t y = src[eb];
        float2 ay = ising ? asrc[eb] : make_float2(0.f, 0.f);
        ga_mutate(p, g, draw(p, m1, 2 + t, gen, kStGa), ising, y, ay);
        dst[(size_t)m1 * L + t] = y;
        if (ising) adst[(size_t)m1 * L + t] = ay;
      }
    }
  }
}

// initial genome: gene (c, t) = below(u.x, G) with Philox (c, t, 0, stream 5);
// an Ising gene's angle from u.y on the 2 pi / Q lattice
__global__ void __launch_bounds__(256) k_ga_init(const DevProblem *__restrict__ probs,
                                                 uint32_t prob, DevGlobal g) {
  const DevProblem &p = probs[prob];
  const size_t n = (size_t)p.P * p.L;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const uint32_t c = (uint32_t)(e / p.L), t = (uint32_t)(e % p.L);
    const uint4 u = draw(p, c, t, 0, kStGaInit);
    p.gate_idx[e] = (uint8_t)below(u.x, p.G);
    if (p.ising) p.amps[e] = g.ph_tab[below(u.y, kQ)];
  }
}

cudaError_t launch_ga_init(const DevProblem *probs, uint32_t prob, uint32_t P, uint32_t L,
                           const DevGlobal &g, cudaStream_t st) {
  uint64_t blocks = ((uint64_t)P * L + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (!blocks) blocks = 1;
  k_ga_init<<<(uint32_t)blocks, 256, 0, st>>>(probs, prob, g);
  return cudaGetLastError();
}

cudaError_t launch_ga_prep(const DevProblem *probs, const uint32_t *ids, const uint32_t *tprefix,
                           uint32_t n_ga, uint32_t n_tiles, const DevGlobal &g, cudaStream_t st) {
  if (!n_ga || !n_tiles) return cudaSuccess;
  k_ga_tiles<<<n_tiles, kGaThreads, 0, st>>>(probs, ids, tprefix, n_ga, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ga_top<<<n_ga, kGaThreads, 0, st>>>(probs, ids);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ga_parents<<<n_tiles, kGaThreads, 0, st>>>(probs, ids, tprefix, n_ga, g);
  return cudaGetLastError();
}

cudaError_t launch_ga_next(const LaunchCfg &lc, const DevProblem *probs, const uint32_t *ids,
                           const uint32_t *prefix, uint32_t n_ga, uint32_t total_pairs,
                           const DevGlobal &g, cudaStream_t st) {
  if (!n_ga || !total_pairs) return cudaSuccess;
  uint64_t blocks = ((uint64_t)total_pairs + 7) / 8;
  const uint64_t cap = (uint64_t)lc.num_sms * 8;
  if (blocks > cap) blocks = cap;
  k_ga_next<<<(uint32_t)blocks, 256, 0, st>>>(probs, ids, prefix, n_ga, total_pairs, g);
  return cudaGetLastError();
}

}  // namespace qe
