// noalloc.cu -- qe_eval_rank_static: evaluation plus binary64-rescored ranking
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while the CUDA caching
// allocator of a host framework owns the device memory, plugins loaded into a
// process whose memory budget is fixed up front, and real-time loops that must
// not block in the allocator.  For them this entry point needs no context and
// allocates nothing: the ranking's scratch (candidate list, rescored values,
// rescore queue, gate costs, the search descriptor and two counters) lives in
// one file-scope device array, g_qe_static_scratch, sized for at most
// kStaticMaxCircuits circuits per call.  Every GPU that loads this library
// holds that array (about 1.25 MiB) until the process exits.
//
// Host code never passes the array's name to a kernel (on the host that name
// is only a stand-in, not a device address); the first call on each device
// looks up the device address with cudaGetSymbolAddress and caches it.  Under
// lazy module loading (CUDA_MODULE_LOADING=LAZY, the default since CUDA 12.2)
// that first call is also what loads this file's module, and the driver then
// allocates the array and the code; calls after it allocate nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/qe.h"
#include "qe_dev.cuh"
#include "qe_host.h"

namespace {

constexpr uint32_t kStaticMaxCircuits = 65536;
// byte layout of the scratch array
constexpr size_t kOffProb = 0;                                   // DevProblem (368 B)
constexpr size_t kOffCount = 1024;                               // 4 x uint32 counters
constexpr size_t kOffMeta = 2048;                                // gate cost per circuit
constexpr size_t kOffCand = kOffMeta + 4 * (size_t)kStaticMaxCircuits;
constexpr size_t kOffCandF = kOffCand + 4 * (size_t)kStaticMaxCircuits;
constexpr size_t kOffQueue = kOffCandF + 8 * (size_t)kStaticMaxCircuits;
constexpr size_t kStaticBytes = kOffQueue + 4 * (size_t)kStaticMaxCircuits;
static_assert(sizeof(qe::DevProblem) <= kOffCount - kOffProb, "descriptor slot too small");

static __device__ __align__(256) unsigned char g_qe_static_scratch[kStaticBytes];

// writes the search descriptor into the scratch array and clears the counters
// that must start at zero (rescore queue length, error word)
__global__ void k_static_setup(qe::DevProblem p) {
  *reinterpret_cast<qe::DevProblem *>(g_qe_static_scratch + kOffProb) = p;
  uint32_t *cnt = reinterpret_cast<uint32_t *>(g_qe_static_scratch + kOffCount);
  cnt[0] = 0u;
  cnt[1] = 0u;
  cnt[2] = 0u;
  cnt[3] = 0u;
}

struct DeviceSlot {
  bool ready = false;
  unsigned char *base = nullptr;  // device address of g_qe_static_scratch
  qe::LaunchCfg lc;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;

qe_status say(char *msg, size_t len, qe_status st, const char *text) {
  if (msg && len) snprintf(msg, len, "%s", text);
  return st;
}

uint32_t regions_of(uint32_t n, uint32_t lib) {
  uint32_t r = 0;
  if (lib & QE_LIB_NCV) r += n * (n - 1);
  if (lib & QE_LIB_HT) r += n;
  return r;
}

// library index -> op byte, in the library order of include/qe.h
void ops_of(uint32_t n, uint32_t lib, uint8_t *gop) {
  uint32_t g = 0;
  if (lib & QE_LIB_IDENTITY) gop[g++] = qe::kOpIdentity;
  if (lib & QE_LIB_NCV)
    for (uint32_t c = 0; c < n; ++c)
      for (uint32_t t = 0; t < n; ++t) {
        if (t == c) continue;
        const uint32_t pair = c * (n - 1) + (t > c ? t - 1 : t);
        gop[g++] = (uint8_t)(2 * pair);
        gop[g++] = (uint8_t)(2 * pair + 1);
        gop[g++] = (uint8_t)((2 * pair + 1) | qe::kOpNeg);
      }
  if (lib & QE_LIB_HT)
    for (uint32_t w = 0; w < n; ++w) {
      const uint32_t base = 2 * n * (n - 1) + 2 * w;
      gop[g++] = (uint8_t)base;
      gop[g++] = (uint8_t)(base + 1);
      gop[g++] = (uint8_t)((base + 1) | qe::kOpNeg);
    }
}

}  // namespace

extern "C" qe_status qe_eval_rank_static(const qe_problem *prob, const uint8_t *d_gate_idx,
                                         uint32_t n_circuits, void *d_fitness, qe_ranked *d_topk,
                                         void *cuda_stream, char *h_msg, size_t msg_len) {
  if (h_msg && msg_len) h_msg[0] = '\0';
  if (!prob) return say(h_msg, msg_len, QE_EINVAL, "null problem");
  const qe_problem &q = *prob;
  if (q.n_qubits < 1 || q.n_qubits > QE_MAX_QUBITS || q.circuit_len < 1 ||
      q.circuit_len > QE_MAX_LEN || q.population < 1 || q.population > QE_MAX_POP ||
      (q.library & ~(QE_LIB_NCV | QE_LIB_HT | QE_LIB_IDENTITY)) ||
      regions_of(q.n_qubits, q.library) == 0 || q.fitness_kind > QE_FIT_PROB ||
      q.topk > QE_MAX_TOPK || !std::isfinite(q.cost_weight))
    return say(h_msg, msg_len, QE_EINVAL, "invalid problem description");
  if (q.precision != QE_PREC_FP32 && q.precision != QE_PREC_FP64)
    return say(h_msg, msg_len, QE_EUNSUPPORTED, "precision must be QE_PREC_FP32 or QE_PREC_FP64");
  const uint32_t N = 1u << q.n_qubits;
  bool seen[32] = {false};
  for (uint32_t j = 0; j < N; ++j) {
    const uint32_t v = q.target_perm[j];
    if (v >= N || seen[v]) return say(h_msg, msg_len, QE_EINVAL, "target_perm is not a permutation");
    seen[v] = true;
  }
  if (n_circuits > kStaticMaxCircuits) {
    char b[160];
    snprintf(b, sizeof b, "n_circuits = %u exceeds the static scratch limit of %u circuits",
             n_circuits, kStaticMaxCircuits);
    return say(h_msg, msg_len, QE_EINVAL, b);
  }
  if (n_circuits == 0) return QE_OK;
  if (!d_gate_idx || !d_fitness) return say(h_msg, msg_len, QE_EINVAL, "null device buffer");

  // once per device: the device address of the scratch array and launch shapes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return say(h_msg, msg_len, QE_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return say(h_msg, msg_len, QE_EUNSUPPORTED, "device index");
  DeviceSlot slot;
  {
    std::lock_guard<std::mutex> lk(g_slots_mu);
    DeviceSlot &s = g_slots[dev];
    if (!s.ready) {
      cudaDeviceProp prop;
      e = cudaGetDeviceProperties(&prop, dev);
      if (e != cudaSuccess) return say(h_msg, msg_len, QE_ECUDA, cudaGetErrorString(e));
      if (!(prop.major == 10 && prop.minor == 3))
        return say(h_msg, msg_len, QE_EUNSUPPORTED, "this library is built for sm_103a only");
      void *addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_qe_static_scratch);
      if (e != cudaSuccess || !addr)
        return say(h_msg, msg_len, QE_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
      s.lc.num_sms = (uint32_t)prop.multiProcessorCount;
      e = qe::query_circuit_occupancy(s.lc);
      if (e == cudaSuccess) e = qe::rank_init();
      if (e != cudaSuccess) return say(h_msg, msg_len, QE_ECUDA, cudaGetErrorString(e));
      s.base = (unsigned char *)addr;
      s.ready = true;
    }
    slot = s;
  }

  // descriptor: buffers point into the scratch array or at the caller's outputs
  qe::DevProblem d;
  memset(&d, 0, sizeof d);
  d.n = q.n_qubits;
  d.N = N;
  d.L = q.circuit_len;
  d.P = n_circuits;
  d.R = regions_of(d.n, q.library);
  d.G = ((q.library & QE_LIB_IDENTITY) ? 1u : 0u) + 3u * d.R;
  d.LP = d.L * d.P;
  d.lib = q.library;
  d.prec = q.precision;
  d.fit_kind = q.fitness_kind;
  d.topk = q.topk;
  d.k = q.topk ? q.topk : 1;
  d.cost_weight = q.cost_weight;
  d.eps_d = (float)((double)d.L * 8e-7 + 2e-6);
  d.pen_per_gate = (float)(q.cost_weight / (double)d.L);
  for (uint32_t j = 0; j < 32; ++j) d.perm[j] = j < N ? q.target_perm[j] : 0;
  memset(d.gop, qe::kOpIdentity, sizeof d.gop);
  ops_of(d.n, q.library, d.gop);
  unsigned char *b = slot.base;
  d.meta = (uint32_t *)(b + kOffMeta);
  d.cand = (uint32_t *)(b + kOffCand);
  d.cand_f = (double *)(b + kOffCandF);
  d.cand_n = (uint32_t *)(b + kOffCount) + 3;
  d.topk_out = (qe::Ranked *)d_topk;
  if (q.precision == QE_PREC_FP64) d.fit64 = (double *)d_fitness;
  else d.fit32 = (float *)d_fitness;
  qe::DevGlobal g{};
  g.rescore_n = (uint32_t *)(b + kOffCount) + 0;
  g.err = (uint32_t *)(b + kOffCount) + 1;
  g.gen = (uint32_t *)(b + kOffCount) + 2;
  g.rescore_list = (uint32_t *)(b + kOffQueue);
  const qe::DevProblem *probs = (const qe::DevProblem *)(b + kOffProb);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool canon = q.precision == QE_PREC_FP64;
  k_static_setup<<<1, 1, 0, st>>>(d);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = qe::launch_eval(slot.lc, d.n, probs, 0, canon, d_gate_idx, nullptr, n_circuits,
                        d_fitness, d.meta, nullptr, g, st);
  if (d_topk) {
    qe::RankJob j{};
    j.prob = 0;
    j.n = n_circuits;
    j.fit = d_fitness;
    j.meta = d.meta;
    j.gsrc = d_gate_idx;
    j.update_record = 0;
    if (e == cudaSuccess) e = qe::launch_rank_select(probs, nullptr, 1, j, g, st, n_circuits);
    if (e == cudaSuccess && !canon)
      e = qe::launch_rescore(slot.lc, d.n, false, probs, d_gate_idx, nullptr, false, g, st);
    if (e == cudaSuccess) e = qe::launch_rank_sort(probs, nullptr, 1, j, g, st);
  }
  if (e != cudaSuccess) return say(h_msg, msg_len, QE_ECUDA, cudaGetErrorString(e));
  return QE_OK;
}
