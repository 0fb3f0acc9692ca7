// qe_dev.cuh -- device-side data layout and primitives of the QEQEA engine.
//
// One search's state lives in a single device arena (see capi.cu):
//   segs       : S segments x 64 B = {cur, best}, each 32 B
//                {q0re,q0im,q1re,q1im,q2re,q2im,b0,b1} as 2 float4, so elitism
//                touches one 64-B line whichever record it keeps
//   fk         : S x {best_f (binary32 bits), sfkey} -- the segment's best
//                fitness and this generation's segment fitness as an
//                order-preserving key (0 = untouched, reset by the update),
//                side by side so both arrive in one DRAM burst
//   gate_idx   : 2 x P*L uint8 (the generation's circuits, double-buffered by
//                generation parity so a generation's ranking can overlap the
//                next generation; a GA search keeps its genome here),
//                seg_id: P*L uint32 (QEQEA only)
//   mut_list   : 2 x P individual ids, mut_cnt: 2 counters (QEQEA only)
//   amps       : 2 x P*L float2 slot angles as qubit amplitudes (Ising only)
//   ga_cum     : P uint64 SUS prefix sums within tiles of 1024, ga_tiles: the
//                tiles' offsets and elites, ga_parent: P SUS parents (GA only)
//   fit32/fit64: 2 x P (working-precision fitness), meta: 2 x P (cost | work << 8)
// where S = R*P*L and seg = r*L*P + i*L + t (Eq. (10)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qe {

constexpr int kQ = 4096;            // mutation magnitude quantisation
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint8_t kOpIdentity = 0xff;
constexpr uint8_t kOpNeg = 0x80;    // sign bit of the op byte: sigma = -1 (CV^dag, T^dag)
// Ising ops (no sign bit): kOpIsingRot + 3w + k = R_{x,y,z} on wire w (k = 0, 1, 2),
// kOpIsingJ + q = the interaction template on wire pair q (lexicographic i < j)
constexpr uint8_t kOpIsingRot = 64, kOpIsingJ = 80;
// 1/sqrt(2) rounded to binary64 and to binary32
constexpr double kH64 = 0x1.6a09e667f3bcdp-1;
constexpr float kH32 = 0x1.6a09e6p-1f;

// Philox4x32-10 counter words: (a, b, gen, run << 4 | stream)
enum Stream : uint32_t {
  kStSample = 0,
  kStMutDecide = 1,
  kStMutSeg = 2,
  kStShot = 3,  // repeated qutrit measurements
  kStGa = 4,
  kStGaInit = 5
};

// encodings (mirror QE_ENC_*)
constexpr uint32_t kEncQeqea = 0u, kEncGa = 1u;

// device error word bits (mirrors QE_ERRW_*)
constexpr uint32_t kErrBadGate = 1u, kErrNonFinite = 2u, kErrGuardBand = 4u;

struct Ranked {
  uint32_t circuit, cost;
  double fitness;
};

// best-so-far record and the per-generation report fields of one search
struct Best {
  uint32_t generation, best_gen;
  double best_fitness, gen_best_fitness, mean_fitness;
  unsigned long long useful_flops;
  uint32_t best_cost, best_len, error_word, reserved;
  uint8_t best_gates[64];
  float2 best_amps[64];  // Ising: the best circuit's slot angles
};

// one scan tile of a GA search's SUS weights: the sum of its weights (after
// the tile scan: the sum of all earlier tiles' weights) and its elite
struct GaTile {
  unsigned long long sum;
  double F;
  uint32_t cost, idx;
};

struct DevProblem {
  uint32_t n, N, L, P, R, G, LP;
  uint32_t lib, prec, fit_kind, enc, topk, k;  // k = max(topk, 1)
  uint32_t run, has_qubit, base;                // base = 1 if I is library index 0
  uint32_t measure_qubit;  // the qubit decides "gate present" (identity in the library)
  uint32_t ising;          // the Ising library: every slot carries an angle
  uint32_t shots;          // qutrit measurements per slot (1 = one; majority otherwise)
  uint32_t dense;          // the target is the dense unitary tgt32/tgt64, not perm
  uint32_t prefetch;       // the circuit kernel prefetches the update's lines into L2
  uint32_t key0, key1;
  float eps_d;        // bound on |d32 - d64|, d = (N - |tr|)/N, for the binary32 path
  float pen_per_gate; // cost_weight / L in binary32 (ranking bounds only)
  double p_mut, cost_weight, ga_rate;
  // an individual mutates when its Philox word u < mut_T, i.e. when
  // (u + 1/2) 2^-32 < p_mut (mut_T = ceil(p_mut 2^32 - 1/2), clamped to [0, 2^32])
  unsigned long long mut_T;
  // GA: a gene mutates when its Philox word u < ga_T (same rule with ga_rate)
  unsigned long long ga_T;
  uint64_t nseg;
  uint8_t perm[32];
  uint8_t gop[80];    // library index -> op byte (see k_circuit.cu), kOpIdentity for I
  // state and per-generation buffers
  float4 *segs;  // 4 float4 per segment: cur (2), best (2)
  uint32_t *fk;  // 2 words per segment: best_f bits, sfkey
  uint8_t *gate_idx;
  uint32_t *seg_id;
  float *fit32;
  double *fit64;
  uint32_t *meta;
  // ranking scratch
  uint32_t *cand;
  double *cand_f;
  uint32_t *cand_n;
  Ranked *topk_out;
  Best *rec;
  // mutation table: cos/sin of m * mutation_range / Q, m = 0..Q
  float2 *qubit_tab;
  // dense target T[i][j] at i * N + j, in binary32 and binary64 (dense != 0)
  float2 *tgt32;
  double2 *tgt64;
  // Ising: each slot's qubit amplitudes (b0, b1) as sampled (its angle), 2 x P*L,
  // double-buffered by generation parity like gate_idx
  float2 *amps;
  // individuals that mutate this generation, listed by the circuit kernel:
  // 2 x P entries and 2 counters, by generation parity (the circuit kernel of
  // generation g appends to half g & 1 and clears the counter of the other)
  uint32_t *mut_list;
  uint32_t *mut_cnt;
  // GA buffers: SUS prefix sums of the weights within each scan tile, the
  // tiles (offsets and elites), {W, elite}, and each child's SUS parent
  unsigned long long *ga_cum;
  GaTile *ga_tiles;
  unsigned long long *ga_info;
  uint32_t *ga_parent;
};

// context-wide device pointers
struct DevGlobal {
  float2 *th_tab;     // cos/sin of m * (pi/2) / Q
  float2 *ph_tab;     // cos/sin of m * (2 pi) / Q
  uint32_t *gen;      // generation counter (graph replays read it)
  uint32_t *err;      // error word
  uint32_t *rescore_list;  // (problem << 20 | slot) pairs to rescore in binary64
  uint32_t *rescore_n;
  uint32_t *ranked;       // generations whose ranking is done (pipelined ranking)
  uint32_t *rank_active;  // 1 while a pipelined ranking chain has work to do
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds; each round multiplies counter
// words 0 and 2 by the two round multipliers and xors the high halves into the
// other words with the key, which is bumped by the two Weyl constants.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 draw(const DevProblem &p, uint32_t a, uint32_t b, uint32_t gen,
                                      uint32_t stream) {
  return philox(make_uint4(a, b, gen, (p.run << 4) | stream), p.key0, p.key1);
}

// integer in [0, m)
__device__ __forceinline__ uint32_t below(uint32_t u, uint32_t m) { return __umulhi(u, m); }
// real in (0,1), binary64: (u + 1/2) 2^-32 (exact)
__device__ __forceinline__ double unit64(uint32_t u) {
  return __dmul_rn(__dadd_rn((double)u, 0.5), 0x1p-32);
}
// real in (0,1), binary32: ((u >> 9) + 1/2) 2^-23 (exact)
__device__ __forceinline__ float unit32(uint32_t u) {
  return __fmul_rn(__fadd_rn(__uint2float_rn(u >> 9), 0.5f), 0x1p-23f);
}

// order-preserving map of a non-NaN float to uint32 (never 0)
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// order-preserving map of a non-NaN double to uint64
__device__ __forceinline__ unsigned long long dkey(double f) {
  unsigned long long b = (unsigned long long)__double_as_longlong(f);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// The ranking's guard band: the interval [lo, hi] that must hold the binary64
// fitness of a circuit whose binary32 fitness is F and whose gate cost is
// cost, given |d32 - d64| <= eps_d with d = (1 - f)^2 = ((N - |tr|)/N) and
// f = F + cost_weight * cost / L (binary32 arithmetic; the slop covers the
// rounding of these few operations).  The selection keeps every circuit whose
// hi reaches the k-th largest lo; the rescoring checks each candidate's
// binary64 fitness against the same interval.
__device__ __forceinline__ void guard_band(const DevProblem &p, float F, uint32_t cost, float &lo,
                                           float &hi) {
  const float pen = p.pen_per_gate * (float)(cost & 0xffu);
  const float f = F + pen;
  const float t = 1.f - f;
  const float d = t * t;
  const float dl = fmaxf(0.f, d - p.eps_d), dh = d + p.eps_d;
  const float fhi = 1.f - sqrtf(dl), flo = 1.f - sqrtf(dh);
  const float slop = 2e-6f;
  lo = flo - pen - slop;
  hi = fhi - pen + slop;
}

// ---------------------------------------------------------------- state access
__device__ __forceinline__ float4 *cur_of(const DevProblem &p, uint32_t seg) {
  return p.segs + 4 * (size_t)seg;
}
__device__ __forceinline__ float4 *best_of(const DevProblem &p, uint32_t seg) {
  return p.segs + 4 * (size_t)seg + 2;
}
__device__ __forceinline__ float *bestf_of(const DevProblem &p, uint32_t seg) {
  return reinterpret_cast<float *>(p.fk + 2 * (size_t)seg);
}
__device__ __forceinline__ uint32_t *key_of(const DevProblem &p, uint32_t seg) {
  return p.fk + 2 * (size_t)seg + 1;
}

// ---------------------------------------------------------------- dependent launch
// A kernel behind a programmatic graph edge may be launched before the kernel
// it depends on has finished (the launch overlaps that kernel's last blocks);
// it waits here, before reading anything that kernel writes, until the
// kernel has completed and its writes are visible.  Launched any other way it
// returns at once.
__device__ __forceinline__ void wait_predecessor() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------- 32-B records
// A segment's cur or best record is 32 B and 32-B aligned: each is moved as
// one 256-bit access (sm_100 and later), half the load/store instructions of
// two float4 moves, which matters where the update is bound by the number of
// scattered memory requests in flight.
__device__ __forceinline__ void ld_rec(const float4 *p, float4 &a, float4 &b) {
  asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z),
                 "=f"(b.w)
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st_rec(float4 *p, const float4 a, const float4 b) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y),
               "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
               : "memory");
}

// ---------------------------------------------------------------- lane layout
// A warp holds one circuit's N x N unitary (WB = 0) or its 2^-WB share of the
// columns (2^WB warps per circuit, warp w holding columns w 2^CB .. (w + 1)
// 2^CB - 1; columns evolve independently, so the split changes no value):
// lane = (row group g, column j), the column's low CB bits in the low lane
// bits, g in the next RBL lane bits; each lane keeps ROWS rows of its column in
// registers: row i = (g << RBR) | r.  The top RBL row bits live in lane bits,
// the low RBR row bits in register indices.  Lanes beyond USED are shadows
// that compute but never write.
template <int NQ, int WB = 0>
struct Lay {
  static constexpr int N = 1 << NQ;
  static constexpr int CB = NQ - WB;  // column bits in the lane index
  static constexpr int RBL = (NQ < 5 - CB) ? NQ : 5 - CB;
  static constexpr int RBR = NQ - RBL;
  static constexpr int ROWS = 1 << RBR;
  static constexpr int USED = 1 << (CB + RBL);  // lanes that hold data
};

}  // namespace qe
