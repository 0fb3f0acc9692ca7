// k_update.cu -- segment fitness, elitism and adaptive mutation (Sec. IV-E1,
// IV-F), and the initial state (Sec. IV-B).
//
// Two kernels, which may run concurrently, split the update of every search:
//  role A (k_update_elite), one thread per (circuit, slot): if the segment's
//    individual is not mutated this generation, the first thread to take the
//    segment's fitness key (a 64-bit atomicAnd that clears it) applies
//    elitism to it; from 2^20 slots k_update_elite4 does the same with four
//    lanes per slot, each moving a quarter of the segment's 64-B line;
//  role B, for each segment of an individual that mutates: elitism where the
//    segment was used, then mutation.  Inside the generation graph
//    (k_update_mutate_list) one thread per segment of the individuals the
//    circuit kernel listed; for qe_update or contexts with many searches
//    (k_update_mutate) one warp per (32 individuals, region).
// A segment belongs to exactly one role, so no segment is touched twice.
// All mutation arithmetic is binary32 with _rn intrinsics in the order the
// oracle fixes (no contraction), so the state stays bit-identical to it; the
// SU(3) operator of Eq. (12) is evaluated per segment in that order (su3).
#include "qe_dev.cuh"
#include "qe_host.h"

namespace qe {

// contexts with at most this many QEQEA searches use the listed mutation role;
// every block of that kernel walks the searches one after another
constexpr uint32_t kListMaxSearches = 64;
// role A runs four lanes per slot (k_update_elite4) from this many slots of
// all searches together
#ifndef QE_QUAD_MIN_SLOTS
#define QE_QUAD_MIN_SLOTS (1u << 20)
#endif
constexpr uint64_t kQuadMinSlots = QE_QUAD_MIN_SLOTS;

struct fc {
  float re, im;
};
__device__ __forceinline__ fc fmulc(fc a, fc b) {
  return {__fsub_rn(__fmul_rn(a.re, b.re), __fmul_rn(a.im, b.im)),
          __fadd_rn(__fmul_rn(a.re, b.im), __fmul_rn(a.im, b.re))};
}
__device__ __forceinline__ fc faddc(fc a, fc b) {
  return {__fadd_rn(a.re, b.re), __fadd_rn(a.im, b.im)};
}
__device__ __forceinline__ fc fsubc(fc a, fc b) {
  return {__fsub_rn(a.re, b.re), __fsub_rn(a.im, b.im)};
}
__device__ __forceinline__ fc fscale(fc a, float s) { return {__fmul_rn(a.re, s), __fmul_rn(a.im, s)}; }
__device__ __forceinline__ fc fneg(fc a) { return {-a.re, -a.im}; }

// Eq. (12) in binary32 with parameter j (0..2: theta_1..3, 3..7: phi_1..5) at
// cos/sin (c, s) and every other parameter zero (cos 1, sin 0): phase factors
// e^{i(+-a +-b ...)} are products of the single-parameter phases taken left
// to right, real factors applied left to right, every operation rounded on
// its own -- the evaluation order of the oracle, so each entry is the
// oracle's bit for bit.  (Evaluated per segment: a table of every (j, level)
// pair would cost 72 scattered bytes per mutated segment.)
__device__ __forceinline__ void su3(uint32_t j, float c, float s, fc (&U)[9]) {
  float cv[8], sv[8];
#pragma unroll
  for (uint32_t k = 0; k < 8; ++k) {
    cv[k] = k == j ? c : 1.f;
    sv[k] = k == j ? s : 0.f;
  }
  const float c1 = cv[0], c2 = cv[1], c3 = cv[2], s1 = sv[0], s2 = sv[1], s3 = sv[2];
  auto ep = [&](int k) { return fc{cv[2 + k], sv[2 + k]}; };
  auto em = [&](int k) { return fc{cv[2 + k], -sv[2 + k]}; };
  U[0] = fscale(fscale(ep(1), c1), c2);
  U[1] = fscale(ep(3), s1);
  U[2] = fscale(fscale(ep(4), c1), s2);
  U[3] = fsubc(fscale(fscale(fmulc(em(4), em(5)), s2), s3),
               fscale(fscale(fscale(fmulc(fmulc(ep(1), ep(2)), em(3)), s1), c2), c3));
  U[4] = fscale(fscale(ep(2), c1), c3);
  U[5] = fsubc(fneg(fscale(fscale(fmulc(em(1), em(5)), c2), s3)),
               fscale(fscale(fscale(fmulc(fmulc(ep(2), em(3)), ep(4)), s1), s2), c3));
  U[6] = fsubc(fneg(fscale(fscale(fmulc(em(2), em(4)), s2), c3)),
               fscale(fscale(fscale(fmulc(fmulc(ep(1), em(3)), ep(5)), s1), c2), s3));
  U[7] = fscale(fscale(ep(5), c1), s3);
  U[8] = fsubc(fscale(fscale(fmulc(em(1), em(2)), c2), c3),
               fscale(fscale(fscale(fmulc(fmulc(em(3), ep(4)), ep(5)), s1), s2), s3));
}

__device__ __forceinline__ bool mutates(const DevProblem &p, uint32_t i, uint32_t gen) {
  const uint4 v = draw(p, i, 0, gen, kStMutDecide);
  return (unsigned long long)v.x < p.mut_T;
}

// Elitism (Sec. IV-E1): keep the state as the new best if the segment's
// fitness this generation beats its best so far, otherwise revert to the best.
// The caller has loaded the segment's best fitness and its 64-B line holding
// both records; the record kept is returned in c0/c1.
__device__ __forceinline__ void elitism(const DevProblem &p, uint32_t seg, float sf, float bf,
                                        float4 &c0, float4 &c1, const float4 b0,
                                        const float4 b1) {
  if (sf > bf) {
    st_rec(best_of(p, seg), c0, c1);
    *bestf_of(p, seg) = sf;
  } else {
    c0 = b0;
    c1 = b1;
    st_rec(cur_of(p, seg), b0, b1);
  }
}

// Adaptive mutation of one segment (Sec. IV-F) with e = 1 - clamp(best_f).
__device__ __forceinline__ void mutate(const DevProblem &p, const DevGlobal &g, uint32_t seg,
                                       uint32_t gen, float bf, float4 a, float4 b) {
  const uint4 w = draw(p, seg, 0, gen, kStMutSeg);
  const float fcl = bf < 0.f ? 0.f : (bf > 1.f ? 1.f : bf);
  float e = __fsub_rn(1.f, fcl);
  if (!(e == e)) e = 1.f;  // a NaN best fitness (set by the caller) mutates fully
  float4 *cp = cur_of(p, seg);
  if (p.has_qubit && w.x < 0x80000000u) {
    // qubit: rotation by +-(1 - f) * mutationRange, quantised to range/Q
    const uint32_t m = (uint32_t)floorf(__fmul_rn(e, (float)kQ));
    const float2 cs = p.qubit_tab[m];
    const float c = cs.x, s = (w.y & 1u) ? -cs.y : cs.y;
    const float b0 = b.z, b1 = b.w;
    b.z = __fadd_rn(__fadd_rn(0.f, __fmul_rn(c, b0)), __fmul_rn(-s, b1));
    b.w = __fadd_rn(__fadd_rn(0.f, __fmul_rn(s, b0)), __fmul_rn(c, b1));
    cp[1] = b;
    return;
  }
  // qutrit: one Eq. (12) parameter set to a draw from its domain times (1 - f)
  const uint32_t j = below(w.y, 8);
  const uint32_t m = (uint32_t)floorf(__fmul_rn(__fmul_rn(unit32(w.z), e), (float)kQ));
  const float2 cs = __ldg((j < 3 ? g.th_tab : g.ph_tab) + m);
  fc U[9];
  su3(j, cs.x, cs.y, U);
  const fc q[3] = {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}};
  fc o[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    fc acc = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k) acc = faddc(acc, fmulc(U[3 * r + k], q[k]));
    o[r] = acc;
  }
  a = make_float4(o[0].re, o[0].im, o[1].re, o[1].im);
  b.x = o[2].re;
  b.y = o[2].im;
  st_rec(cp, a, b);
}

__device__ __forceinline__ uint32_t find_q(const uint32_t *prefix, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// role A: elitism of used segments whose individual does not mutate
__global__ void __launch_bounds__(256, 8) k_update_elite(const DevProblem *__restrict__ probs,
                                                         const uint32_t *__restrict__ group,
                                                         const uint32_t *__restrict__ prefA,
                                                         uint32_t n_group, uint32_t totalA,
                                                         const uint32_t *d_gen, uint32_t gen_arg,
                                                         const uint32_t *seg_override) {
  wait_predecessor();  // the circuit kernel's ids, keys and lists
  const uint32_t gen = d_gen ? *d_gen : gen_arg;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < totalA;
       e += gridDim.x * blockDim.x) {
    const uint32_t q = find_q(prefA, n_group, e);
    const DevProblem &p = probs[group[q]];
    const uint32_t local = e - prefA[q];
    const uint32_t seg = seg_override ? seg_override[local] : p.seg_id[local];
    if (seg >= p.nseg) continue;  // caller-provided ids are checked
    const uint32_t i = (seg % p.LP) / p.L;
    if (mutates(p, i, gen)) continue;
    // best fitness and fitness key in one 64-bit atomic that clears the key
    // (low word: best_f bits, high word: key); one slot per segment sees it set
    const unsigned long long pr =
        atomicAnd(reinterpret_cast<unsigned long long *>(p.fk + 2 * (size_t)seg), 0xffffffffull);
    const float bf = __uint_as_float((uint32_t)pr);
    const uint32_t key = (uint32_t)(pr >> 32);
    if (!key) continue;
    // only the record that is copied is read: cur when it becomes the best,
    // else best, which replaces cur
    const float sf = fkey_inv(key);
    float4 *line = cur_of(p, seg);
    float4 r0, r1;
    if (sf > bf) {
      ld_rec(line, r0, r1);
      st_rec(best_of(p, seg), r0, r1);
      *bestf_of(p, seg) = sf;
    } else {
      ld_rec(line + 2, r0, r1);
      st_rec(line, r0, r1);
    }
  }
}

// Role A with four lanes per slot, for large populations, where role A is
// bound by the number of scattered requests in flight rather than by their
// latency: lane 0 of a quad takes the {best_f, key} word first; then the two
// lanes holding the record that is copied read its 16-B halves (lanes 0, 1:
// cur; lanes 2, 3: best, the quarters of the segment's 64-B line) and elitism
// copies it through one shuffle: best <- cur on lanes 2, 3 (from lanes 0, 1),
// cur <- best on lanes 0, 1 (from lanes 2, 3).  Each request covers whole
// sectors, and the record that is not copied is never read.
__global__ void __launch_bounds__(256, 8) k_update_elite4(const DevProblem *__restrict__ probs,
                                                          const uint32_t *__restrict__ group,
                                                          const uint32_t *__restrict__ prefA,
                                                          uint32_t n_group, uint32_t totalA,
                                                          const uint32_t *d_gen, uint32_t gen_arg,
                                                          const uint32_t *seg_override) {
  wait_predecessor();  // the circuit kernel's ids, keys and lists
  const uint32_t gen = d_gen ? *d_gen : gen_arg;
  const int lane = threadIdx.x & 31, q4 = lane & 3, qbase = lane & ~3;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  // the trip count is the same for every lane of a warp (shuffles below)
  for (uint32_t base = w0 * 8u; base < totalA; base += nw * 8u) {
    const uint32_t e = base + (uint32_t)(lane >> 2);
    const DevProblem *pp = probs;
    uint32_t seg = 0;
    bool act = e < totalA;
    if (act) {
      const uint32_t q = find_q(prefA, n_group, e);
      pp = probs + group[q];
      const uint32_t local = e - prefA[q];
      seg = seg_override ? seg_override[local] : pp->seg_id[local];
      act = seg < pp->nseg;  // caller-provided ids are checked
      if (act) act = !mutates(*pp, (seg % pp->LP) / pp->L, gen);
    }
    unsigned long long pr = 0;
    // best fitness and fitness key in one 64-bit atomic that clears the key
    if (act && q4 == 0)
      pr = atomicAnd(reinterpret_cast<unsigned long long *>(pp->fk + 2 * (size_t)seg),
                     0xffffffffull);
    pr = __shfl_sync(kFull, pr, qbase);
    const uint32_t key = (uint32_t)(pr >> 32);
    const float sf = fkey_inv(key), bf = __uint_as_float((uint32_t)pr);
    const bool up = sf > bf;  // cur becomes the best: lanes 0, 1 read, 2, 3 write
    // only the record that is copied is read (lanes 0, 1 hold cur's quarters,
    // lanes 2, 3 best's)
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 *line = act && key ? cur_of(*pp, seg) : nullptr;
    if (line && (up ? q4 < 2 : q4 >= 2)) v = line[q4];
    float4 o;
    o.x = __shfl_xor_sync(kFull, v.x, 2);
    o.y = __shfl_xor_sync(kFull, v.y, 2);
    o.z = __shfl_xor_sync(kFull, v.z, 2);
    o.w = __shfl_xor_sync(kFull, v.w, 2);
    if (line) {
      if (up) {
        if (q4 >= 2) line[q4] = o;
        if (q4 == 0) *bestf_of(*pp, seg) = sf;
      } else if (q4 < 2) {
        line[q4] = o;
      }
    }
  }
}

// one segment of a mutating individual: elitism if it was used this
// generation (its fitness key is set), then mutation
__device__ __forceinline__ void mutate_segment(const DevProblem &p, const DevGlobal &g,
                                               uint32_t seg, uint32_t gen) {
  const uint2 fkv = *reinterpret_cast<const uint2 *>(p.fk + 2 * (size_t)seg);
  const uint32_t key = fkv.y;
  float bf = __uint_as_float(fkv.x);
  const float4 *line = cur_of(p, seg);
  float4 c0, c1;
  ld_rec(line, c0, c1);
  if (key) {
    float4 b0, b1;
    ld_rec(line + 2, b0, b1);
    *key_of(p, seg) = 0u;
    const float sf = fkey_inv(key);
    elitism(p, seg, sf, bf, c0, c1, b0, b1);
    if (sf > bf) bf = sf;
  }
  mutate(p, g, seg, gen, bf, c0, c1);
}

// role B, inside the generation graph: the segments of the individuals the
// circuit kernel listed, one thread per segment (the list has no order; each
// segment is independent), searches one after another
__global__ void __launch_bounds__(256) k_update_mutate_list(const DevProblem *__restrict__ probs,
                                                            const uint32_t *__restrict__ group,
                                                            uint32_t n_group,
                                                            const uint32_t *d_gen, DevGlobal g) {
  wait_predecessor();  // the circuit kernel's ids, keys and lists
  const uint32_t gen = *d_gen, par = gen & 1u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t q = 0; q < n_group; ++q) {
    const DevProblem &p = probs[group[q]];
    const uint32_t RL = p.R * p.L;
    const uint32_t total = p.mut_cnt[par] * RL;
    const uint32_t *list = p.mut_list + (size_t)par * p.P;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
      const uint32_t e = x / RL, rem = x - e * RL;
      const uint32_t r = rem / p.L, t = rem - r * p.L;
      mutate_segment(p, g, r * p.LP + list[e] * p.L + t, gen);
    }
  }
}

// role B for qe_update (no circuit kernel has listed the individuals): one
// warp per (32 individuals, region), the decision drawn here
__global__ void __launch_bounds__(256) k_update_mutate(const DevProblem *__restrict__ probs,
                                                       const uint32_t *__restrict__ group,
                                                       const uint32_t *__restrict__ prefB,
                                                       uint32_t n_group, uint32_t totalB,
                                                       const uint32_t *d_gen, uint32_t gen_arg,
                                                       DevGlobal g) {
  wait_predecessor();  // the circuit kernel's ids, keys and lists
  const uint32_t gen = d_gen ? *d_gen : gen_arg;
  const int lane = threadIdx.x & 31;
  const uint32_t nwB = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < totalB; w += nwB) {
    const uint32_t q = find_q(prefB, n_group, w);
    const DevProblem &p = probs[group[q]];
    const uint32_t local = w - prefB[q];
    const uint32_t groups = (p.P + 31) / 32;
    const uint32_t r = local / groups;
    const uint32_t i0 = (local - r * groups) * 32;
    const uint32_t i = i0 + lane;
    const bool mine = i < p.P && mutates(p, i, gen);
    const uint32_t bal = __ballot_sync(kFull, mine);
    const uint32_t items = __popc(bal) * p.L;
    for (uint32_t x = lane; x < items; x += 32) {
      const uint32_t b = x / p.L, t = x - b * p.L;
      const uint32_t ii = i0 + __fns(bal, 0, (int)b + 1);
      mutate_segment(p, g, r * p.LP + ii * p.L + t, gen);
    }
  }
}

// segment fitness of caller-provided circuits (qe_update): max over circuits
__global__ void __launch_bounds__(256) k_scatter(const DevProblem *__restrict__ probs,
                                                 uint32_t prob, const uint32_t *__restrict__ seg_id,
                                                 const double *__restrict__ fitness, uint32_t *err) {
  const DevProblem &p = probs[prob];
  const size_t n = (size_t)p.P * p.L;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const double F = fitness[e / p.L];
    const float f = (float)F;
    const uint32_t seg = seg_id[e];
    if (seg >= p.nseg) {
      atomicOr(err, kErrBadGate);
      continue;
    }
    if (f == f) atomicMax(key_of(p, seg), fkey(f));
  }
}

// uniform initial encoding (Sec. IV-B): qutrit amplitudes 1/sqrt(3), qubit
// amplitudes 1/sqrt(2), best = cur, best fitness -1, no segment fitness yet
__global__ void __launch_bounds__(256) k_init_state(const DevProblem *__restrict__ probs,
                                                    uint32_t prob, float a, float b) {
  const DevProblem &p = probs[prob];
  for (size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.nseg;
       s += (size_t)gridDim.x * blockDim.x) {
    const float4 v0 = make_float4(a, 0.f, a, 0.f), v1 = make_float4(a, 0.f, b, b);
    float4 *line = p.segs + 4 * s;
    line[0] = v0;
    line[1] = v1;
    line[2] = v0;
    line[3] = v1;
    reinterpret_cast<uint2 *>(p.fk)[s] = make_uint2(__float_as_uint(-1.f), 0u);
  }
}

bool is_update_kernel(const void *f) {
  return f == (const void *)k_update_elite || f == (const void *)k_update_elite4 ||
         f == (const void *)k_update_mutate ||
         f == (const void *)k_update_mutate_list;
}

cudaError_t launch_init_state(const DevProblem *probs, uint32_t prob, uint64_t nseg,
                              cudaStream_t st) {
  uint64_t blocks = (nseg + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (!blocks) blocks = 1;
  const float a = (float)(1.0 / sqrt(3.0));
  const float b = (float)kH64;
  k_init_state<<<(uint32_t)blocks, 256, 0, st>>>(probs, prob, a, b);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const DevProblem *probs, uint32_t prob, uint32_t P, uint32_t L,
                           const uint32_t *seg_id, const double *fitness, uint32_t *err,
                           cudaStream_t st) {
  uint64_t blocks = ((uint64_t)P * L + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (!blocks) blocks = 1;
  k_scatter<<<(uint32_t)blocks, 256, 0, st>>>(probs, prob, seg_id, fitness, err);
  return cudaGetLastError();
}

cudaError_t launch_update(const LaunchCfg &lc, const DevProblem *probs, const uint32_t *group,
                          const uint32_t *prefA, const uint32_t *prefB, uint32_t n_group,
                          uint32_t totalA, uint32_t totalB, const uint32_t *d_gen, uint32_t gen,
                          const uint32_t *seg_override, const DevGlobal &g, cudaStream_t stA,
                          cudaStream_t stB) {
  const bool quad = (uint64_t)totalA >= kQuadMinSlots;
  uint64_t bA = ((uint64_t)totalA * (quad ? 4 : 1) + 255) / 256;
  const uint64_t capA = (uint64_t)lc.num_sms * 8;
  if (bA > capA) bA = capA;
  if (!bA) bA = 1;
  uint64_t bB = ((uint64_t)totalB + 7) / 8;
  const uint64_t capB = (uint64_t)lc.num_sms * 8;
  if (bB > capB) bB = capB;
  if (!bB) bB = 1;
  if (quad)
    k_update_elite4<<<(uint32_t)bA, 256, 0, stA>>>(probs, group, prefA, n_group, totalA, d_gen,
                                                   gen, seg_override);
  else
    k_update_elite<<<(uint32_t)bA, 256, 0, stA>>>(probs, group, prefA, n_group, totalA, d_gen,
                                                  gen, seg_override);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (d_gen && n_group <= kListMaxSearches) {
    // generation graph: the circuit kernel listed the mutating individuals
    k_update_mutate_list<<<lc.num_sms * 8, 256, 0, stB>>>(probs, group, n_group, d_gen, g);
  } else {
    k_update_mutate<<<(uint32_t)bB, 256, 0, stB>>>(probs, group, prefB, n_group, totalB, d_gen,
                                                   gen, g);
  }
  return cudaGetLastError();
}

}  // namespace qe
