// k_update.cu -- segment fitness, elitism and adaptive mutation (Sec. IV-E1,
// IV-F), and the initial state (Sec. IV-B).
//
// One launch does both update roles for every search of a group:
//  role A, one thread per (circuit, slot): if the segment's individual is not
//    mutated this generation, the first thread to take the segment's fitness
//    key (atomicExch to 0) applies elitism to it;
//  role B, one warp per 32 individuals: for each individual that mutates, the
//    warp walks all R*L of its segments, applies elitism where the segment was
//    used, then mutates it.
// A segment belongs to exactly one role, so no segment is touched twice.
// All mutation arithmetic is binary32 with _rn intrinsics in the order the
// oracle fixes (no contraction), so the state stays bit-identical to it.
#include "qe_dev.cuh"
#include "qe_host.h"

namespace qe {

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

// Eq. (12) in binary32; cv/sv index 0..2 = theta1..3, 3..7 = phi1..5.
// Phase factors e^{i(+-a +-b ...)} are products of the single-parameter
// phases taken left to right, real factors are applied left to right.
__device__ __forceinline__ void su3_f32(const float (&cv)[8], const float (&sv)[8], fc (&U)[9]) {
  const float c1 = cv[0], c2 = cv[1], c3 = cv[2], s1 = sv[0], s2 = sv[1], s3 = sv[2];
#define EP(k) (fc{cv[2 + (k)], sv[2 + (k)]})
#define EM(k) (fc{cv[2 + (k)], -sv[2 + (k)]})
  U[0] = fscale(fscale(EP(1), c1), c2);
  U[1] = fscale(EP(3), s1);
  U[2] = fscale(fscale(EP(4), c1), s2);
  U[3] = fsubc(fscale(fscale(fmulc(EM(4), EM(5)), s2), s3),
               fscale(fscale(fscale(fmulc(fmulc(EP(1), EP(2)), EM(3)), s1), c2), c3));
  U[4] = fscale(fscale(EP(2), c1), c3);
  U[5] = fsubc(fneg(fscale(fscale(fmulc(EM(1), EM(5)), c2), s3)),
               fscale(fscale(fscale(fmulc(fmulc(EP(2), EM(3)), EP(4)), s1), s2), c3));
  U[6] = fsubc(fneg(fscale(fscale(fmulc(EM(2), EM(4)), s2), c3)),
               fscale(fscale(fscale(fmulc(fmulc(EP(1), EM(3)), EP(5)), s1), c2), s3));
  U[7] = fscale(fscale(EP(5), c1), s3);
  U[8] = fsubc(fscale(fscale(fmulc(EM(1), EM(2)), c2), c3),
               fscale(fscale(fscale(fmulc(fmulc(EM(3), EP(4)), EP(5)), s1), s2), s3));
#undef EP
#undef EM
}

__device__ __forceinline__ bool mutates(const DevProblem &p, uint32_t i, uint32_t gen) {
  const uint4 v = draw(p, i, 0, gen, kStMutDecide);
  return (unsigned long long)v.x < p.mut_T;
}

// Elitism (Sec. IV-E1): keep the state as the new best if the segment's
// fitness this generation beats its best so far, otherwise revert to the best.
__device__ __forceinline__ void elitism(const DevProblem &p, uint32_t seg, float sf) {
  const size_t s2 = 2 * (size_t)seg;
  if (sf > p.best_f[seg]) {
    p.best[s2] = p.cur[s2];
    p.best[s2 + 1] = p.cur[s2 + 1];
    p.best_f[seg] = sf;
  } else {
    p.cur[s2] = p.best[s2];
    p.cur[s2 + 1] = p.best[s2 + 1];
  }
}

// Adaptive mutation of one segment (Sec. IV-F) with e = 1 - clamp(best_f).
__device__ __forceinline__ void mutate(const DevProblem &p, const DevGlobal &g, uint32_t seg,
                                       uint32_t gen) {
  const uint4 w = draw(p, seg, 0, gen, kStMutSeg);
  const float bf = p.best_f[seg];
  const float fcl = bf < 0.f ? 0.f : (bf > 1.f ? 1.f : bf);
  float e = __fsub_rn(1.f, fcl);
  if (!(e == e)) e = 1.f;  // a NaN best fitness (set by the caller) mutates fully
  const size_t s2 = 2 * (size_t)seg;
  if (p.has_qubit && w.x < 0x80000000u) {
    // qubit: rotation by +-(1 - f) * mutationRange, quantised to range/Q
    const uint32_t m = (uint32_t)floorf(__fmul_rn(e, (float)kQ));
    const float2 cs = p.qubit_tab[m];
    const float c = cs.x, s = (w.y & 1u) ? -cs.y : cs.y;
    float4 b = p.cur[s2 + 1];
    const float b0 = b.z, b1 = b.w;
    b.z = __fadd_rn(__fadd_rn(0.f, __fmul_rn(c, b0)), __fmul_rn(-s, b1));
    b.w = __fadd_rn(__fadd_rn(0.f, __fmul_rn(s, b0)), __fmul_rn(c, b1));
    p.cur[s2 + 1] = b;
    return;
  }
  // qutrit: one Eq. (12) parameter set to a draw from its domain times (1 - f)
  const uint32_t j = below(w.y, 8);
  const uint32_t m = (uint32_t)floorf(__fmul_rn(__fmul_rn(unit32(w.z), e), (float)kQ));
  const float2 cs = (j < 3) ? g.th_tab[m] : g.ph_tab[m];
  float cv[8], sv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    cv[k] = ((uint32_t)k == j) ? cs.x : 1.f;
    sv[k] = ((uint32_t)k == j) ? cs.y : 0.f;
  }
  fc U[9];
  su3_f32(cv, sv, U);
  float4 a = p.cur[s2], b = p.cur[s2 + 1];
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
  p.cur[s2] = a;
  p.cur[s2 + 1] = b;
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

__global__ void __launch_bounds__(256) k_update(const DevProblem *__restrict__ probs,
                                                const uint32_t *__restrict__ group,
                                                const uint32_t *__restrict__ prefA,
                                                const uint32_t *__restrict__ prefB,
                                                uint32_t n_group, uint32_t totalA,
                                                uint32_t totalB, uint32_t blocksA,
                                                const uint32_t *d_gen, uint32_t gen_arg,
                                                const uint32_t *seg_override, DevGlobal g) {
  const uint32_t gen = d_gen ? *d_gen : gen_arg;
  if (blockIdx.x < blocksA) {
    // role A: elitism of segments whose individual does not mutate
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < totalA;
         e += blocksA * blockDim.x) {
      const uint32_t q = find_q(prefA, n_group, e);
      const DevProblem &p = probs[group[q]];
      const uint32_t local = e - prefA[q];
      const uint32_t seg = seg_override ? seg_override[local] : p.seg_id[local];
      if (seg >= p.nseg) continue;  // caller-provided ids are checked
      const uint32_t i = (seg % p.LP) / p.L;
      if (mutates(p, i, gen)) continue;
      const uint32_t key = atomicExch(p.sfkey + seg, 0u);
      if (key) elitism(p, seg, fkey_inv(key));
    }
    return;
  }
  // role B: individuals that mutate
  const int lane = threadIdx.x & 31;
  const uint32_t nwB = ((gridDim.x - blocksA) * blockDim.x) >> 5;
  for (uint32_t w = (((blockIdx.x - blocksA) * blockDim.x) + threadIdx.x) >> 5; w < totalB;
       w += nwB) {
    const uint32_t q = find_q(prefB, n_group, w);
    const DevProblem &p = probs[group[q]];
    const uint32_t i0 = (w - prefB[q]) * 32;
    const uint32_t i = i0 + lane;
    const bool mine = i < p.P && mutates(p, i, gen);
    uint32_t bal = __ballot_sync(kFull, mine);
    const uint32_t RL = p.R * p.L;
    while (bal) {
      const int b = __ffs(bal) - 1;
      bal &= bal - 1;
      const uint32_t ii = i0 + b;
      for (uint32_t s = lane; s < RL; s += 32) {
        const uint32_t r = s / p.L, t = s - r * p.L;
        const uint32_t seg = r * p.LP + ii * p.L + t;
        const uint32_t key = p.sfkey[seg];
        if (key) {
          p.sfkey[seg] = 0;
          elitism(p, seg, fkey_inv(key));
        }
        mutate(p, g, seg, gen);
      }
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
    if (f == f) atomicMax(p.sfkey + seg, fkey(f));
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
    p.cur[2 * s] = v0;
    p.cur[2 * s + 1] = v1;
    p.best[2 * s] = v0;
    p.best[2 * s + 1] = v1;
    p.best_f[s] = -1.f;
    p.sfkey[s] = 0u;
  }
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
                          const uint32_t *seg_override, const DevGlobal &g, cudaStream_t st) {
  uint64_t bA = ((uint64_t)totalA + 255) / 256;
  uint64_t capA = (uint64_t)lc.num_sms * 8;
  if (bA > capA) bA = capA;
  if (!bA) bA = 1;
  uint64_t bB = ((uint64_t)totalB + 7) / 8;
  uint64_t capB = (uint64_t)lc.num_sms * 8;
  if (bB > capB) bB = capB;
  if (!bB) bB = 1;
  k_update<<<(uint32_t)(bA + bB), 256, 0, st>>>(probs, group, prefA, prefB, n_group, totalA,
                                                totalB, (uint32_t)bA, d_gen, gen, seg_override,
                                                g);
  return cudaGetLastError();
}

}  // namespace qe
