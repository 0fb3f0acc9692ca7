// capi.cu -- the C ABI of include/qe.h: context, validation, device arena,
// host-built tables, CUDA-graph capture of one generation, and the calls.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <unistd.h>

#include "../../include/qe.h"
#include "qe_dev.cuh"
#include "qe_host.h"

using namespace qe;

namespace {

thread_local std::string g_init_error;

// the update's lines per generation that the circuit kernel may prefetch into
// L2 (half of GB300's 129 MB L2)
constexpr double kPrefetchBudget = 64.0 * 1024 * 1024;

struct Group {
  bool canon = false;
  bool ising = false;  // the Ising library (slots carry angles)
  uint32_t n = 0;  // qubit count of every search in the group
  std::vector<uint32_t> ids;
  uint32_t *d_ids = nullptr, *d_prefix = nullptr;
  uint32_t total = 0;
};

}  // namespace

// How a generation graph is launched; results do not depend on it.
struct Plan {
  bool select_first = true;  // launch-completion edge: ranking selection -> circuits
  uint32_t grid_mode = 0;    // circuit kernels: 0 resident blocks, 1 one block less per SM,
                             // 2 one warp per circuit in a single launch wave
  bool concurrent = false;   // circuit kernels of different widths on parallel streams
};

constexpr int kBatchSlots = (int)QE_BATCH_SLOTS;  // qe_eval_host_batch_async calls in flight

// One slot of the batched host evaluation: device staging (grown on demand:
// the items' gates, fitness and costs, and the slot's own ranking scratch),
// pinned host staging of the top-k lists, the graphs of the last layout (key:
// ranking flag, item count, the items' problems and circuit counts): one
// graph of the evaluations and the ranking, run on the slot's stream -- and
// the call in flight.

// the staging's error-word slot while a call's graph has not yet copied the
// word there (no error word has every bit set)
constexpr uint32_t kErrwPending = 0xffffffffu;

struct BatchSlot {
  void *d = nullptr;
  size_t d_bytes = 0;
  void *h = nullptr;
  void *hd = nullptr;  // the staging's device mapping
  size_t h_bytes = 0;
  std::vector<uint32_t> key;
  std::vector<unsigned char> meta;  // host copy of the jobs, offsets and gate table
  cudaGraph_t eg = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_done = nullptr;
  size_t err_off = 0;  // the slot's error word in its staging
  uint32_t desc_version = 0;  // the context's descriptors the slot's copies were made from
  // the call in flight (ticket: also the slot's last call, for reuse order);
  // flag: the call's graph ends with the copy of its error word, which the
  // wait polls in the staging instead of synchronising on ev_done
  bool busy = false;
  bool flag = false;
  uint64_t ticket = 0;
  qe_ranked *h_topk = nullptr;
  size_t k_total = 0;
};

struct qe_ctx {
  int device = 0;
  cudaStream_t user = nullptr;
  cudaStream_t cap = nullptr, side = nullptr, side2 = nullptr;
  std::vector<cudaStream_t> gstreams;  // extra streams for concurrent circuit kernels
  std::vector<cudaEvent_t> gjoin;
  cudaEvent_t gfork = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr, ev_fork2 = nullptr;
  std::vector<qe_problem> probs;
  std::vector<DevProblem> hp;
  DevProblem *d_probs = nullptr;
  DevGlobal g{};
  LaunchCfg lc;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<Group> groups;  // circuit launches, one per (arithmetic, qubit count)
  // widths with binary32 searches: bit 0 discrete libraries, bit 1 Ising
  uint8_t rescore_nq[QE_MAX_QUBITS + 1] = {0};
  uint32_t max_P = 0;    // the largest population
  // all QEQEA searches (update launch)
  uint32_t n_upd = 0, upd_totalA = 0, upd_totalB = 0;
  uint32_t *d_upd_ids = nullptr, *d_upd_prefA = nullptr, *d_upd_prefB = nullptr;
  // all GA searches (breeding launches): ids and prefix sums of ceil(P/2) pairs
  uint32_t n_ga = 0, ga_pairs = 0, ga_tiles = 0;
  uint32_t *d_ga_ids = nullptr, *d_ga_prefix = nullptr, *d_ga_tprefix = nullptr;
  // QEQEA searches measuring each qutrit K > 1 times (k_presample): ids and
  // prefix sums of P*L slots
  uint32_t n_shot = 0;
  uint32_t *d_shot_ids = nullptr;
  unsigned long long *d_shot_prefix = nullptr, shot_total = 0;
  // per-search single arrays for qe_update: {id}, {0, P*L}, {0, ceil(P/32)*R}
  uint32_t *d_single = nullptr;
  RankJob *d_jobs = nullptr;
  uint32_t n_jobs = 0;
  Best *d_recs = nullptr;
  Best *h_recs = nullptr;  // pinned
  uint8_t *d_stage_gates = nullptr;
  void *d_stage_fit = nullptr;
  // qe_eval_host_batch(_async): kBatchSlots slots, each call's copies,
  // evaluations and ranking on its slot's stream and scratch, so that calls
  // in flight overlap
  BatchSlot bslot[kBatchSlots];
  std::vector<char> b_seen;     // the batch call's argument check
  std::vector<uint32_t> b_key;  // the batch call's graph key
  uint64_t next_ticket = 1;
  // bumped whenever a search's descriptor changes after qe_init (qe_set_target):
  // a batch slot whose copies are older recaptures its layout
  uint32_t desc_version = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // launch plan of the generation graph (qe_autotune picks it by timing)
  Plan plan;
  bool tuned = false;
  std::string plan_text;
  cudaGraph_t dgraph = nullptr;      // ranking of the last generation alone (drain)
  cudaGraphExec_t dexec = nullptr;
  bool pending_rank = false;         // the last generation is not ranked yet
  bool has_last = false;             // a generation ran since qe_init / qe_load
  std::vector<std::vector<double>> targets;  // dense targets (empty: the permutation)
  // stage timing: events recorded inside the generation graph
  bool timing = false;
  bool timing_serial = false;  // every kernel of the generation on one stream
  cudaEvent_t tev[8] = {nullptr};
  uint32_t gen = 0;
  bool poisoned = false;
  std::string err;
};

namespace {

qe_status fail(qe_ctx *ctx, qe_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  else g_init_error = msg;
  return st;
}

qe_status cuda_fail(qe_ctx *ctx, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (ctx) ctx->poisoned = true;
  return fail(ctx, QE_ECUDA, m);
}

#define QE_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

uint32_t regions(uint32_t n, uint32_t lib) {
  if (lib == QE_LIB_ISING) return n + n * (n - 1) / 2;
  uint32_t r = 0;
  if (lib & QE_LIB_NCV) r += n * (n - 1);
  if (lib & QE_LIB_HT) r += n;
  return r;
}

uint32_t gates(uint32_t n, uint32_t lib) {
  if (lib == QE_LIB_ISING) return 3u * n + n * (n - 1) / 2;
  return ((lib & QE_LIB_IDENTITY) ? 1u : 0u) + 3u * regions(n, lib);
}

// op byte of every library index (see k_circuit.cu for the op numbering)
void build_ops(uint32_t n, uint32_t lib, uint8_t *gop) {
  uint32_t g = 0;
  if (lib == QE_LIB_ISING) {
    for (uint32_t w = 0; w < n; ++w)
      for (uint32_t k = 0; k < 3; ++k) gop[g++] = (uint8_t)(kOpIsingRot + 3 * w + k);
    for (uint32_t q = 0; q < n * (n - 1) / 2; ++q) gop[g++] = (uint8_t)(kOpIsingJ + q);
    return;
  }
  if (lib & QE_LIB_IDENTITY) gop[g++] = kOpIdentity;
  if (lib & QE_LIB_NCV)
    for (uint32_t c = 0; c < n; ++c)
      for (uint32_t t = 0; t < n; ++t) {
        if (t == c) continue;
        const uint32_t tt = t > c ? t - 1 : t;
        const uint32_t pair = c * (n - 1) + tt;
        gop[g++] = (uint8_t)(2 * pair);               // CNOT
        gop[g++] = (uint8_t)(2 * pair + 1);           // CV
        gop[g++] = (uint8_t)((2 * pair + 1) | kOpNeg);  // CV^dag
      }
  if (lib & QE_LIB_HT)
    for (uint32_t w = 0; w < n; ++w) {
      const uint32_t base = 2 * n * (n - 1) + 2 * w;
      gop[g++] = (uint8_t)base;                  // H
      gop[g++] = (uint8_t)(base + 1);            // T
      gop[g++] = (uint8_t)((base + 1) | kOpNeg);  // T^dag
    }
}

qe_status validate(const qe_problem &p, uint32_t idx) {
  char b[256];
  auto bad = [&](const char *what) {
    snprintf(b, sizeof b, "problem %u: %s", idx, what);
    return fail(nullptr, QE_EINVAL, b);
  };
  if (p.n_qubits < 1 || p.n_qubits > QE_MAX_QUBITS) return bad("n_qubits must be 1..5");
  if (p.circuit_len < 1 || p.circuit_len > QE_MAX_LEN) return bad("circuit_len must be 1..64");
  if (p.population < 1 || p.population > QE_MAX_POP) return bad("population must be 1..2^20");
  if (p.library & ~(QE_LIB_NCV | QE_LIB_HT | QE_LIB_IDENTITY | QE_LIB_ISING))
    return bad("unknown library bits");
  if ((p.library & QE_LIB_ISING) && p.library != QE_LIB_ISING)
    return bad("QE_LIB_ISING is used alone");
  const uint32_t R = regions(p.n_qubits, p.library);
  if (R == 0) return bad("library has no gates for this n_qubits");
  if (p.encoding > QE_ENC_GA) return bad("unknown encoding");
  if (p.precision > QE_PREC_SPLIT_TC) return bad("unknown precision");
  if (p.fitness_kind > QE_FIT_PROB) return bad("unknown fitness_kind");
  if (p.topk > QE_MAX_TOPK || p.topk > p.population) return bad("topk must be <= min(P, 1024)");
  if (!(p.p_mutation >= 0.0 && p.p_mutation <= 1.0)) return bad("p_mutation must be in [0,1]");
  if (!(std::isfinite(p.mutation_range) && p.mutation_range >= 0.0))
    return bad("mutation_range must be finite and >= 0");
  if (!(p.ga_mutation_rate >= 0.0 && p.ga_mutation_rate <= 1.0))
    return bad("ga_mutation_rate must be in [0,1]");
  if (p.shots > QE_MAX_SHOTS) return bad("shots must be in [0, 64]");
  if (p.reserved != 0) return bad("reserved must be 0");
  if (!std::isfinite(p.cost_weight)) return bad("cost_weight must be finite");
  const uint64_t S = (uint64_t)R * p.circuit_len * p.population;
  if (S >= (1ull << 32)) return bad("regions * L * P must be < 2^32");
  const uint32_t N = 1u << p.n_qubits;
  bool seen[32] = {false};
  for (uint32_t j = 0; j < N; ++j) {
    const uint32_t v = p.target_perm[j];
    if (v >= N || seen[v]) return bad("target_perm is not a permutation of 0..2^n-1");
    seen[v] = true;
  }
  if (p.precision == QE_PREC_SPLIT_TC) {
    snprintf(b, sizeof b,
             "problem %u: QE_PREC_SPLIT_TC is not provided (gates are applied in registers; "
             "use QE_PREC_FP32)", idx);
    return fail(nullptr, QE_EUNSUPPORTED, b);
  }
  return QE_OK;
}

// device arena: bump allocation with 256-byte alignment
struct Arena {
  size_t off = 0;
  std::vector<std::pair<void **, size_t>> req;
  template <typename T>
  void take(T **p, size_t bytes) {
    req.push_back({(void **)p, off});
    off += (bytes + 255) & ~(size_t)255;
  }
  void bind(char *base) {
    for (auto &r : req) *r.first = base + r.second;
  }
};

// bound on |d32 - d64| of the binary32 composition after L gates: every gate
// application perturbs each unit column by at most a few ulps of binary32, so
// the error of every column grows by <= ~4 * 2^-24 * sqrt(2) per gate, |tr|
// changes by at most N times the column error, d = (N - |tr|)/N by at most
// the column error; the probability form doubles it.  Generous by a factor 2.
float eps_d_for(uint32_t L) { return (float)((double)L * 8e-7 + 2e-6); }
// with a dense target the binary32 score itself sums N products per column
// (each column's terms bounded by 1 in sum): |tr| moves by at most ~N^2 ulps
// more, d by ~N ulps; (N + 8) * 2^-23 is generous
float eps_d_dense(uint32_t L, uint32_t N) {
  return eps_d_for(L) + (float)((double)(N + 8) * 0x1p-23);
}

// a dense target: finite, and unitary to 1e-6 in every entry of T^dag T
bool target_ok(const double *T, uint32_t N) {
  for (uint32_t e = 0; e < 2 * N * N; ++e)
    if (!std::isfinite(T[e])) return false;
  for (uint32_t k = 0; k < N; ++k)
    for (uint32_t l = 0; l < N; ++l) {
      double re = 0.0, im = 0.0;  // (T^dag T)_kl
      for (uint32_t i = 0; i < N; ++i) {
        const double ar = T[2 * (i * N + k)], ai = T[2 * (i * N + k) + 1];
        const double br = T[2 * (i * N + l)], bi = T[2 * (i * N + l) + 1];
        re += ar * br + ai * bi;
        im += ar * bi - ai * br;
      }
      if (std::fabs(re - (k == l ? 1.0 : 0.0)) > 1e-6 || std::fabs(im) > 1e-6) return false;
    }
  return true;
}

unsigned long long threshold(double p) {
  // number of u in [0, 2^32) with (u + 1/2) 2^-32 < p
  const double X = p * 4294967296.0;
  if (X <= 0.5) return 0ull;
  const double y = std::ceil(X - 0.5);
  if (y >= 4294967296.0) return 4294967296ull;
  return (unsigned long long)y;
}

qe_status check_ctx(qe_ctx *ctx, uint32_t prob) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  if (prob >= ctx->probs.size()) return fail(ctx, QE_EINVAL, "problem index out of range");
  return QE_OK;
}

// Node priorities: the ranking chain (a latency chain on a few SMs) first,
// then the circuit kernels, the update last.
qe_status set_priorities(qe_ctx *ctx, cudaGraph_t graph) {
  int lo_pri = 0, hi_pri = 0;
  QE_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
  size_t nn = 0;
  QE_CUDA(ctx, cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  QE_CUDA(ctx, cudaGraphGetNodes(graph, nodes.data(), &nn));
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    QE_CUDA(ctx, cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    QE_CUDA(ctx, cudaGraphKernelNodeGetParams(nd, &kp));
    cudaKernelNodeAttrValue v;
    memset(&v, 0, sizeof v);
    // greatest priority: ranking; then the circuit kernels; least: the update
    const int mid_pri = (lo_pri + hi_pri) / 2;
    v.priority = is_update_kernel(kp.func) ? lo_pri : (is_circuit_kernel(kp.func) ? mid_pri : hi_pri);
    QE_CUDA(ctx, cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v));
  }
  return QE_OK;
}

// Let the first circuit kernel(s) of a generation start only once every block of
// the previous generation's selection kernel is resident (a launch-completion
// edge: the circuit kernel does not wait for the selection to finish).  Without
// it the circuit kernel's persistent grid fills every SM first and the ranking
// chain, the longer of the two concurrent paths, starts only as its blocks
// retire.  Skipped when the selection has more blocks than the GPU holds at
// once (many searches), where waiting for all of them to start would delay the
// circuits instead.
qe_status add_select_first_edge(qe_ctx *ctx, cudaGraph_t graph) {
  // see above (two 1024-thread selection CTAs fit an SM)
  if (select_quarters(ctx->n_jobs, ctx->max_P) > 4u * ctx->lc.num_sms) return QE_OK;
  size_t nn = 0;
  QE_CUDA(ctx, cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  QE_CUDA(ctx, cudaGraphGetNodes(graph, nodes.data(), &nn));
  auto circuit_node = [&](cudaGraphNode_t nd, bool &yes) -> qe_status {
    cudaGraphNodeType ty;
    QE_CUDA(ctx, cudaGraphNodeGetType(nd, &ty));
    yes = false;
    if (ty != cudaGraphNodeTypeKernel) return QE_OK;
    cudaKernelNodeParams kp;
    QE_CUDA(ctx, cudaGraphKernelNodeGetParams(nd, &kp));
    yes = is_circuit_kernel(kp.func);
    return QE_OK;
  };
  cudaGraphNode_t sel = nullptr;
  std::vector<cudaGraphNode_t> firsts;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    QE_CUDA(ctx, cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    QE_CUDA(ctx, cudaGraphKernelNodeGetParams(nd, &kp));
    if (is_select_kernel(kp.func)) sel = nd;
    if (!is_circuit_kernel(kp.func)) continue;
    // a group launched first: no circuit kernel before it
    size_t nd_deps = 0;
    QE_CUDA(ctx, cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &nd_deps));
    std::vector<cudaGraphNode_t> deps(nd_deps);
    if (nd_deps) QE_CUDA(ctx, cudaGraphNodeGetDependencies(nd, deps.data(), nullptr, &nd_deps));
    bool after_circuit = false;
    for (auto dp : deps) {
      bool yes = false;
      qe_status st = circuit_node(dp, yes);
      if (st != QE_OK) return st;
      after_circuit = after_circuit || yes;
    }
    if (!after_circuit) firsts.push_back(nd);
  }
  if (!sel) return QE_OK;
  cudaGraphEdgeData ed;
  memset(&ed, 0, sizeof ed);
  ed.from_port = cudaGraphKernelNodePortLaunchCompletion;
  ed.type = cudaGraphDependencyTypeProgrammatic;
  for (auto f : firsts) QE_CUDA(ctx, cudaGraphAddDependencies(graph, &sel, &f, &ed, 1));
  return QE_OK;
}

// Programmatic dependent launch: every plain edge from a kernel node to a kernel
// that begins by waiting for its predecessor (the update roles, the binary64
// rescoring, the ranking sort, the top-k gather, the generation counter's
// finish) becomes a programmatic edge, so that the kernel
// is launched while its predecessor's last blocks still run instead of after
// the predecessor has completed; it then waits on the device for that
// completion before reading what the predecessor wrote.
// batch: the batched host call's graph, whose evaluation, one-CTA selection
// and copy out also wait for their predecessors
qe_status add_pdl_edges(qe_ctx *ctx, cudaGraph_t graph, bool batch) {
  size_t nn = 0;
  QE_CUDA(ctx, cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  QE_CUDA(ctx, cudaGraphGetNodes(graph, nodes.data(), &nn));
  auto kernel_of = [&](cudaGraphNode_t nd, const void **f) -> qe_status {
    cudaGraphNodeType ty;
    QE_CUDA(ctx, cudaGraphNodeGetType(nd, &ty));
    *f = nullptr;
    if (ty != cudaGraphNodeTypeKernel) return QE_OK;
    cudaKernelNodeParams kp;
    QE_CUDA(ctx, cudaGraphKernelNodeGetParams(nd, &kp));
    *f = kp.func;
    return QE_OK;
  };
  cudaGraphEdgeData prog;
  memset(&prog, 0, sizeof prog);
  prog.from_port = cudaGraphKernelNodePortProgrammatic;
  prog.type = cudaGraphDependencyTypeProgrammatic;
  for (auto nd : nodes) {
    const void *f = nullptr;
    qe_status st = kernel_of(nd, &f);
    if (st != QE_OK) return st;
    if (!f || !(is_update_kernel(f) || is_rescore_kernel(f) || rank_kernel_waits(f) ||
                (batch && (is_eval_jobs_kernel(f) || batch_kernel_waits(f)))))
      continue;
    size_t nd_deps = 0;
    QE_CUDA(ctx, cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &nd_deps));
    if (!nd_deps) continue;
    std::vector<cudaGraphNode_t> deps(nd_deps);
    std::vector<cudaGraphEdgeData> eds(nd_deps);
    QE_CUDA(ctx, cudaGraphNodeGetDependencies(nd, deps.data(), eds.data(), &nd_deps));
    for (size_t k = 0; k < nd_deps; ++k) {
      const void *pf = nullptr;
      st = kernel_of(deps[k], &pf);
      if (st != QE_OK) return st;
      if (!pf || eds[k].type != cudaGraphDependencyTypeDefault || eds[k].from_port != 0) continue;
      QE_CUDA(ctx, cudaGraphRemoveDependencies(graph, &deps[k], &nd, &eds[k], 1));
      QE_CUDA(ctx, cudaGraphAddDependencies(graph, &deps[k], &nd, &prog, 1));
    }
  }
  return QE_OK;
}

// the ranking chain of generation *gen - 1 (select -> binary64 rescoring -> sort)
cudaError_t enqueue_rank_chain(qe_ctx *ctx, cudaStream_t cs) {
  RankJob none{};
  cudaError_t e =
      launch_rank_select(ctx->d_probs, ctx->d_jobs, ctx->n_jobs, none, ctx->g, cs, ctx->max_P);
  for (uint32_t nq = 1; nq <= QE_MAX_QUBITS; ++nq)
    for (int is = 0; is < 2; ++is)
      if (e == cudaSuccess && ((ctx->rescore_nq[nq] >> is) & 1))
        e = launch_rescore(ctx->lc, nq, is == 1, ctx->d_probs, nullptr, nullptr, true, ctx->g, cs);
  if (e == cudaSuccess)
    e = launch_rank_sort(ctx->d_probs, ctx->d_jobs, ctx->n_jobs, none, ctx->g, cs);
  return e;
}

// One generation, software-pipelined: generation g's circuit kernels and
// update run on side streams while the main stream ranks generation g - 1
// (its circuits and fitness sit in the other half of the double buffers).
// Stage events (when timing): 0 start; 1 after the circuit kernels; 2 after
// the selection, 3 after the rescoring, 4 after the sort (ranking of g - 1);
// 5 before and 6 after the update; 7 end of the generation.  Serialised
// stage timing puts every kernel on the capture stream in the order circuits,
// update, ranking, so that each interval is its stage's own duration.
qe_status build_gen_graph(qe_ctx *ctx, const Plan &plan, cudaGraph_t *out_graph,
                          cudaGraphExec_t *out_exec) {
  cudaStream_t cs = ctx->cap;
  const bool serial = ctx->timing && ctx->timing_serial;
  cudaStream_t side = serial ? cs : ctx->side, side2 = serial ? cs : ctx->side2;
  LaunchCfg lc = ctx->lc;
  lc.grid_mode = plan.grid_mode;
  QE_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  auto mark = [&](int k, cudaStream_t st) {
    if (e == cudaSuccess && ctx->timing)
      e = cudaEventRecordWithFlags(ctx->tev[k], st, cudaEventRecordExternal);
  };
  mark(0, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ctx->ev_fork, 0);
  // generation g: K-shot measurements, circuits, then the two update roles
  if (e == cudaSuccess && ctx->n_shot)
    e = launch_presample(lc, ctx->d_probs, ctx->d_shot_ids, ctx->d_shot_prefix, ctx->n_shot,
                         ctx->shot_total, ctx->g, side);
  const bool conc = plan.concurrent && ctx->groups.size() > 1 && !serial;
  if (conc && e == cudaSuccess) e = cudaEventRecord(ctx->gfork, side);
  for (size_t k = 0; k < ctx->groups.size(); ++k) {
    const Group &gr = ctx->groups[k];
    cudaStream_t gs = (conc && k > 0) ? ctx->gstreams[k - 1] : side;
    if (conc && k > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(gs, ctx->gfork, 0);
    // the circuit kernel with the K-shot and dense-target paths only for a
    // group that has a search using one of them
    bool ext = false;
    for (uint32_t id : gr.ids) ext = ext || ctx->hp[id].shots > 1 || ctx->hp[id].dense;
    if (e == cudaSuccess)
      e = launch_step(lc, gr.n, ctx->d_probs, gr.d_ids, gr.d_prefix,
                      (uint32_t)gr.ids.size(), gr.total, gr.canon, gr.ising, ext, ctx->g, gs);
    if (conc && k > 0 && e == cudaSuccess) e = cudaEventRecord(ctx->gjoin[k - 1], gs);
  }
  for (size_t k = 1; conc && k < ctx->groups.size(); ++k)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ctx->gjoin[k - 1], 0);
  mark(1, side);
  if (e == cudaSuccess && ctx->n_ga)
    e = launch_ga_prep(ctx->d_probs, ctx->d_ga_ids, ctx->d_ga_tprefix, ctx->n_ga, ctx->ga_tiles,
                       ctx->g, side);
  mark(5, side);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork2, side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side2, ctx->ev_fork2, 0);
  if (e == cudaSuccess && ctx->n_upd)
    e = launch_update(ctx->lc, ctx->d_probs, ctx->d_upd_ids, ctx->d_upd_prefA, ctx->d_upd_prefB,
                      ctx->n_upd, ctx->upd_totalA, ctx->upd_totalB, ctx->g.gen, 0, nullptr, ctx->g,
                      side, side2);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join2, side2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ctx->ev_join2, 0);
  mark(6, side);
  // generation g - 1: ranking
  if (e == cudaSuccess)
    e = launch_rank_select(ctx->d_probs, ctx->d_jobs, ctx->n_jobs, RankJob{}, ctx->g, cs,
                           ctx->max_P);
  mark(2, cs);
  for (uint32_t nq = 1; nq <= QE_MAX_QUBITS; ++nq)
    for (int is = 0; is < 2; ++is)
      if (e == cudaSuccess && ((ctx->rescore_nq[nq] >> is) & 1))
        e = launch_rescore(ctx->lc, nq, is == 1, ctx->d_probs, nullptr, nullptr, true, ctx->g, cs);
  mark(3, cs);
  if (e == cudaSuccess) e = launch_rank_sort(ctx->d_probs, ctx->d_jobs, ctx->n_jobs, RankJob{}, ctx->g, cs);
  mark(4, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->ev_join, 0);
  // GA breeding of generation g + 1 overwrites the buffer generation g - 1's
  // ranking has just read
  if (e == cudaSuccess && ctx->n_ga)
    e = launch_ga_next(ctx->lc, ctx->d_probs, ctx->d_ga_ids, ctx->d_ga_prefix, ctx->n_ga,
                       ctx->ga_pairs, ctx->g, cs);
  if (e == cudaSuccess) e = launch_finish(ctx->g, cs);
  mark(7, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "capturing the generation graph");
  }
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
  qe_status st = set_priorities(ctx, graph);
  if (st == QE_OK) st = add_pdl_edges(ctx, graph, false);
  if (st == QE_OK && plan.select_first && !serial) st = add_select_first_edge(ctx, graph);
  if (st != QE_OK) {
    cudaGraphDestroy(graph);
    return st;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "cudaGraphInstantiateWithFlags");
  }
  *out_graph = graph;
  *out_exec = exec;
  return QE_OK;
}

std::string plan_string(const Plan &p) {
  static const char *modes[3] = {"resident blocks", "resident blocks - 1 per SM",
                                 "one warp per circuit"};
  return std::string("selection before circuits: ") + (p.select_first ? "yes" : "no") +
         "; circuit grid: " + modes[p.grid_mode < 3 ? p.grid_mode : 0] +
         (p.concurrent ? "; widths on parallel streams" : "");
}

qe_status build_graph(qe_ctx *ctx) {
  qe_status st = build_gen_graph(ctx, ctx->plan, &ctx->graph, &ctx->gexec);
  if (st != QE_OK) return st;
  if (ctx->plan_text.empty()) ctx->plan_text = plan_string(ctx->plan) + " (default)";
  if (ctx->dexec) return QE_OK;
  // drain graph: the ranking chain alone, then a clean rescore queue
  cudaStream_t cs = ctx->cap;
  QE_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_rank_chain(ctx, cs);
  if (e == cudaSuccess) e = launch_reset_counter(ctx->g, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "capturing the ranking graph");
  }
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
  ctx->dgraph = graph;
  qe_status pst = add_pdl_edges(ctx, graph, false);
  if (pst != QE_OK) return pst;
  QE_CUDA(ctx, cudaGraphInstantiate(&ctx->dexec, graph, 0));
  return QE_OK;
}

// rank the last generation now if its ranking is still pending
qe_status drain(qe_ctx *ctx) {
  if (!ctx->pending_rank || !ctx->dexec) return QE_OK;
  QE_CUDA(ctx, cudaGraphLaunch(ctx->dexec, ctx->user));
  ctx->pending_rank = false;
  return QE_OK;
}

}  // namespace

extern "C" {

qe_status qe_library_info(uint32_t n_qubits, uint32_t library, uint32_t *n_gates,
                          uint32_t *n_regions) {
  if (n_qubits < 1 || n_qubits > QE_MAX_QUBITS) return QE_EINVAL;
  if (library & ~(QE_LIB_NCV | QE_LIB_HT | QE_LIB_IDENTITY | QE_LIB_ISING)) return QE_EINVAL;
  if ((library & QE_LIB_ISING) && library != QE_LIB_ISING) return QE_EINVAL;
  if (n_gates) *n_gates = gates(n_qubits, library);
  if (n_regions) *n_regions = regions(n_qubits, library);
  return QE_OK;
}

const char *qe_last_error(const qe_ctx *ctx) {
  if (!ctx) return g_init_error.c_str();
  return ctx->err.c_str();
}

void qe_destroy(qe_ctx *ctx) {
  if (!ctx) return;
  for (BatchSlot &b : ctx->bslot) {
    if (b.st) cudaStreamSynchronize(b.st);
    if (b.ex) cudaGraphExecDestroy(b.ex);
    if (b.eg) cudaGraphDestroy(b.eg);
    if (b.d) cudaFree(b.d);
    if (b.h) cudaFreeHost(b.h);
    if (b.ev_done) cudaEventDestroy(b.ev_done);
    if (b.st) cudaStreamDestroy(b.st);
  }
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->dexec) cudaGraphExecDestroy(ctx->dexec);
  if (ctx->dgraph) cudaGraphDestroy(ctx->dgraph);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (auto &ev : ctx->tev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->side2) cudaStreamDestroy(ctx->side2);
  if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
  if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
  if (ctx->gfork) cudaEventDestroy(ctx->gfork);
  for (auto v : ctx->gjoin) cudaEventDestroy(v);
  for (auto st : ctx->gstreams) cudaStreamDestroy(st);
  if (ctx->h_recs) cudaFreeHost(ctx->h_recs);
  if (ctx->arena) cudaFree(ctx->arena);
  delete ctx;
}

qe_status qe_init(qe_ctx **out, const qe_problem *probs, uint32_t n_probs, void *cuda_stream) {
  g_init_error.clear();
  if (!out || !probs) return fail(nullptr, QE_EINVAL, "null argument");
  if (n_probs < 1 || n_probs > QE_MAX_PROBLEMS) return fail(nullptr, QE_EINVAL, "n_probs must be 1..4096");
  for (uint32_t i = 0; i < n_probs; ++i) {
    qe_status st = validate(probs[i], i);
    if (st != QE_OK) return st;
  }
  if (std::getenv("QE_FAULT_ALLOC"))
    return fail(nullptr, QE_ENOMEM, "device allocation refused (QE_FAULT_ALLOC)");

  qe_ctx *ctx = new qe_ctx();
  ctx->user = (cudaStream_t)cuda_stream;
  ctx->probs.assign(probs, probs + n_probs);
  auto bail = [&](qe_status st) {
    g_init_error = ctx->err;
    qe_destroy(ctx);
    return st;
  };
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaGetDevice"));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, ctx->device);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaGetDeviceProperties"));
  if (!(prop.major == 10 && prop.minor == 3))
    return bail(fail(ctx, QE_EUNSUPPORTED,
                     std::string("this library is built for sm_103a only; device is ") +
                         prop.name));
  ctx->lc.num_sms = (uint32_t)prop.multiProcessorCount;
  e = query_circuit_occupancy(ctx->lc);
  if (e == cudaSuccess) e = rank_init();
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "occupancy query"));

  // ---- arena layout
  Arena ar;
  ctx->hp.resize(n_probs);
  ctx->targets.assign(n_probs, std::vector<double>());
  size_t total_P = 0, max_PL = 0, max_P = 0;
  for (uint32_t i = 0; i < n_probs; ++i) {
    const qe_problem &q = probs[i];
    DevProblem &d = ctx->hp[i];
    memset(&d, 0, sizeof d);
    d.n = q.n_qubits;
    d.N = 1u << d.n;
    d.L = q.circuit_len;
    d.P = q.population;
    d.R = regions(d.n, q.library);
    d.G = gates(d.n, q.library);
    d.LP = d.L * d.P;
    d.lib = q.library;
    d.prec = q.precision;
    d.fit_kind = q.fitness_kind;
    d.enc = q.encoding;
    d.topk = q.topk;
    d.k = q.topk ? q.topk : 1;
    d.run = i;
    // the qubit exists with the identity (gate present, measured) and in the
    // Ising library (the angle, not measured); either may be mutated
    d.has_qubit = (q.library & (QE_LIB_IDENTITY | QE_LIB_ISING)) ? 1u : 0u;
    d.measure_qubit = (q.library & QE_LIB_IDENTITY) ? 1u : 0u;
    d.ising = q.library == QE_LIB_ISING ? 1u : 0u;
    d.shots = (q.encoding == QE_ENC_QEQEA && q.shots > 1) ? q.shots : 1u;
    d.base = d.measure_qubit;
    d.key0 = (uint32_t)q.seed;
    d.key1 = (uint32_t)(q.seed >> 32);
    d.eps_d = eps_d_for(d.L);
    d.pen_per_gate = (float)(q.cost_weight / (double)d.L);
    d.p_mut = q.p_mutation;
    d.cost_weight = q.cost_weight;
    d.ga_rate = q.ga_mutation_rate;
    d.mut_T = threshold(q.p_mutation);
    d.ga_T = threshold(q.ga_mutation_rate);
    d.nseg = (uint64_t)d.R * d.L * d.P;
    for (uint32_t j = 0; j < 32; ++j) d.perm[j] = j < d.N ? q.target_perm[j] : 0;
    memset(d.gop, kOpIdentity, sizeof d.gop);
    build_ops(d.n, q.library, d.gop);
    const size_t P = d.P, PL = (size_t)d.P * d.L;
    if (q.encoding == QE_ENC_QEQEA) {
      ar.take(&d.segs, d.nseg * 64);
      ar.take(&d.fk, d.nseg * 8);
      ar.take(&d.seg_id, PL * 4);
      ar.take(&d.qubit_tab, (kQ + 1) * sizeof(float2));
      ar.take(&d.mut_list, 2 * P * 4);
      ar.take(&d.mut_cnt, 2 * 4);
    } else {
      ar.take(&d.ga_cum, P * 8);
      ar.take(&d.ga_tiles, ((P + 1023) / 1024) * sizeof(GaTile));
      ar.take(&d.ga_info, 16);
      ar.take(&d.ga_parent, P * 4);
      // the Ising GA turns genes' angles with the same table as the qubit mutation
      if (d.ising) ar.take(&d.qubit_tab, (kQ + 1) * sizeof(float2));
    }
    // Ising: the slots' angles (QEQEA: as sampled; GA: the genomes' angles)
    if (d.ising) ar.take(&d.amps, 2 * PL * sizeof(float2));
    // generation buffers, two of each (generation parity)
    ar.take(&d.gate_idx, 2 * PL);
    if (q.precision == QE_PREC_FP64) ar.take(&d.fit64, 2 * P * 8);
    else ar.take(&d.fit32, 2 * P * 4);
    ar.take(&d.meta, 2 * P * 4);
    ar.take(&d.cand, P * 4);
    ar.take(&d.cand_f, P * 8);
    ar.take(&d.cand_n, 4);
    ar.take(&d.topk_out, d.k * sizeof(Ranked));
    if (q.fitness_kind == QE_FIT_TRACE) {  // room for a dense target (qe_set_target)
      ar.take(&d.tgt32, (size_t)d.N * d.N * sizeof(float2));
      ar.take(&d.tgt64, (size_t)d.N * d.N * sizeof(double2));
    }
    total_P += P;
    if (PL > max_PL) max_PL = PL;
    if (P > max_P) max_P = P;
    if (P > ctx->max_P) ctx->max_P = (uint32_t)P;
  }
  // the update's lines of one generation, all searches together: the used
  // segments' 64-B records and the mutating individuals' records and fitness
  // words; the circuit kernel prefetches them into L2 only when they fit in
  // half of it (otherwise they are evicted before the update reads them)
  {
    double upd_bytes = 0.0;
    for (uint32_t i = 0; i < n_probs; ++i) {
      const DevProblem &d = ctx->hp[i];
      if (d.enc != QE_ENC_QEQEA) continue;
      const double PL = (double)d.P * d.L;
      upd_bytes += PL * 64.0 + d.p_mut * PL * d.R * 72.0;
    }
    const uint32_t pf = upd_bytes <= kPrefetchBudget ? 1u : 0u;
    for (uint32_t i = 0; i < n_probs; ++i) ctx->hp[i].prefetch = pf;
  }
  ar.take(&ctx->d_recs, n_probs * sizeof(Best));
  ar.take(&ctx->d_probs, n_probs * sizeof(DevProblem));
  ar.take(&ctx->g.th_tab, (kQ + 1) * sizeof(float2));
  ar.take(&ctx->g.ph_tab, (kQ + 1) * sizeof(float2));
  ar.take(&ctx->g.gen, 4);
  ar.take(&ctx->g.err, 4);
  ar.take(&ctx->g.rescore_n, 4);
  ar.take(&ctx->g.ranked, 4);
  ar.take(&ctx->g.rank_active, 4);
  ar.take(&ctx->g.rescore_list, total_P * 4);
  ar.take(&ctx->d_jobs, n_probs * sizeof(RankJob));
  ar.take(&ctx->d_single, n_probs * 5 * 4);
  ar.take(&ctx->d_stage_gates, max_PL);
  ar.take(&ctx->d_stage_fit, max_P * 8);
  // groups: searches by (arithmetic, library kind, qubit count), widest first
  std::vector<uint32_t> upd, ga, shot;
  for (int k = 0; k < 2; ++k)
    for (int is = 0; is < 2; ++is)
      for (uint32_t nq = QE_MAX_QUBITS; nq >= 1; --nq) {
        Group gr;
        gr.canon = k == 1;
        gr.ising = is == 1;
        gr.n = nq;
        for (uint32_t i = 0; i < n_probs; ++i) {
          if (probs[i].n_qubits != nq) continue;
          if ((probs[i].precision == QE_PREC_FP64) != gr.canon) continue;
          if ((probs[i].library == QE_LIB_ISING) != gr.ising) continue;
          gr.ids.push_back(i);
        }
        if (!gr.ids.empty()) ctx->groups.push_back(gr);
      }
  for (uint32_t i = 0; i < n_probs; ++i) {
    if (probs[i].encoding == QE_ENC_QEQEA) upd.push_back(i);
    else ga.push_back(i);
    if (probs[i].encoding == QE_ENC_QEQEA && probs[i].shots > 1) shot.push_back(i);
    if (probs[i].precision != QE_PREC_FP64)
      ctx->rescore_nq[probs[i].n_qubits] |= probs[i].library == QE_LIB_ISING ? 2 : 1;
  }
  for (auto &gr : ctx->groups) {
    ar.take(&gr.d_ids, gr.ids.size() * 4);
    ar.take(&gr.d_prefix, (gr.ids.size() + 1) * 4);
  }
  ctx->n_upd = (uint32_t)upd.size();
  ar.take(&ctx->d_upd_ids, (upd.size() + 1) * 4);
  ar.take(&ctx->d_upd_prefA, (upd.size() + 1) * 4);
  ar.take(&ctx->d_upd_prefB, (upd.size() + 1) * 4);
  ctx->n_ga = (uint32_t)ga.size();
  ar.take(&ctx->d_ga_ids, (ga.size() + 1) * 4);
  ar.take(&ctx->d_ga_prefix, (ga.size() + 1) * 4);
  ar.take(&ctx->d_ga_tprefix, (ga.size() + 1) * 4);
  ctx->n_shot = (uint32_t)shot.size();
  ar.take(&ctx->d_shot_ids, (shot.size() + 1) * 4);
  ar.take(&ctx->d_shot_prefix, (shot.size() + 1) * 8);

  size_t free_b = 0, total_b = 0;
  e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaMemGetInfo"));
  if (ar.off + (64u << 20) > free_b) {
    char b[160];
    snprintf(b, sizeof b, "needs %.3f GB of device memory, %.3f GB free", ar.off / 1e9,
             free_b / 1e9);
    return bail(fail(ctx, QE_ENOMEM, b));
  }
  e = cudaMalloc(&ctx->arena, ar.off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(ctx, QE_ENOMEM, "cudaMalloc of the state arena failed"));
  }
  ctx->arena_bytes = ar.off;
  ar.bind((char *)ctx->arena);

  // ---- host-side tables and descriptors
  std::vector<float2> tab(kQ + 1);
  auto trig = [&](double step, float2 *dst, cudaStream_t st) -> cudaError_t {
    for (int m = 0; m <= kQ; ++m) {
      const double ang = (double)m * step;
      tab[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    cudaError_t r = cudaMemcpyAsync(dst, tab.data(), tab.size() * sizeof(float2),
                                    cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    return r;
  };
  const double pi = 3.14159265358979323846;
  cudaStream_t us = ctx->user;
  if ((e = trig((pi / 2.0) / (double)kQ, ctx->g.th_tab, us)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "uploading tables"));
  if ((e = trig((2.0 * pi) / (double)kQ, ctx->g.ph_tab, us)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "uploading tables"));
  std::vector<Best> recs(n_probs);
  std::vector<RankJob> jobs(n_probs);
  std::vector<uint32_t> single(n_probs * 5);
  for (uint32_t i = 0; i < n_probs; ++i) {
    DevProblem &d = ctx->hp[i];
    d.rec = ctx->d_recs + i;
    if (d.qubit_tab && (e = trig(probs[i].mutation_range / (double)kQ, d.qubit_tab, us)) != cudaSuccess)
      return bail(cuda_fail(ctx, e, "uploading tables"));
    Best &b = recs[i];
    memset(&b, 0, sizeof b);
    b.best_fitness = -HUGE_VAL;
    b.gen_best_fitness = -HUGE_VAL;
    b.best_cost = 0xffffffffu;
    RankJob &j = jobs[i];
    j.prob = i;
    j.n = d.P;
    j.fit = d.prec == QE_PREC_FP64 ? (const void *)d.fit64 : (const void *)d.fit32;
    j.meta = d.meta;
    j.gsrc = d.gate_idx;
    j.asrc = d.amps;
    j.update_record = 1;
    j.pipelined = 1;
    single[5 * i + 0] = i;
    single[5 * i + 1] = 0;
    single[5 * i + 2] = d.P * d.L;
    single[5 * i + 3] = 0;
    single[5 * i + 4] = ((d.P + 31) / 32) * d.R;
  }
  ctx->n_jobs = n_probs;
  std::vector<uint32_t> host_u32;
  auto put = [&](uint32_t *dst, const std::vector<uint32_t> &v) -> cudaError_t {
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice, us);
  };
  e = cudaMemcpyAsync(ctx->d_probs, ctx->hp.data(), n_probs * sizeof(DevProblem),
                      cudaMemcpyHostToDevice, us);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->d_recs, recs.data(), n_probs * sizeof(Best), cudaMemcpyHostToDevice, us);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->d_jobs, jobs.data(), n_probs * sizeof(RankJob), cudaMemcpyHostToDevice, us);
  if (e == cudaSuccess) e = put(ctx->d_single, single);
  for (auto &gr : ctx->groups) {
    std::vector<uint32_t> pre(gr.ids.size() + 1, 0);
    for (size_t k = 0; k < gr.ids.size(); ++k) pre[k + 1] = pre[k] + ctx->hp[gr.ids[k]].P;
    gr.total = pre.back();
    if (e == cudaSuccess) e = put(gr.d_ids, gr.ids);
    if (e == cudaSuccess) e = put(gr.d_prefix, pre);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
  }
  {
    std::vector<uint32_t> pa(upd.size() + 1, 0), pb(upd.size() + 1, 0);
    for (size_t k = 0; k < upd.size(); ++k) {
      pa[k + 1] = pa[k] + ctx->hp[upd[k]].P * ctx->hp[upd[k]].L;
      pb[k + 1] = pb[k] + ((ctx->hp[upd[k]].P + 31) / 32) * ctx->hp[upd[k]].R;
    }
    ctx->upd_totalA = pa.back();
    ctx->upd_totalB = pb.back();
    if (e == cudaSuccess) e = put(ctx->d_upd_ids, upd);
    if (e == cudaSuccess) e = put(ctx->d_upd_prefA, pa);
    if (e == cudaSuccess) e = put(ctx->d_upd_prefB, pb);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
  }
  {
    std::vector<uint32_t> pg(ga.size() + 1, 0), pt(ga.size() + 1, 0);
    for (size_t k = 0; k < ga.size(); ++k) {
      pg[k + 1] = pg[k] + (ctx->hp[ga[k]].P + 1) / 2;
      pt[k + 1] = pt[k] + (ctx->hp[ga[k]].P + 1023) / 1024;
    }
    ctx->ga_pairs = pg.back();
    ctx->ga_tiles = pt.back();
    if (e == cudaSuccess) e = put(ctx->d_ga_ids, ga);
    if (e == cudaSuccess) e = put(ctx->d_ga_prefix, pg);
    if (e == cudaSuccess) e = put(ctx->d_ga_tprefix, pt);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
  }
  {
    std::vector<unsigned long long> ps(shot.size() + 1, 0);
    for (size_t k = 0; k < shot.size(); ++k)
      ps[k + 1] = ps[k] + (unsigned long long)ctx->hp[shot[k]].P * ctx->hp[shot[k]].L;
    ctx->shot_total = ps.back();
    if (e == cudaSuccess) e = put(ctx->d_shot_ids, shot);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->d_shot_prefix, ps.data(), ps.size() * 8, cudaMemcpyHostToDevice, us);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->g.gen, 0, 4, us);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->g.err, 0, 4, us);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->g.rescore_n, 0, 4, us);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->g.ranked, 0, 4, us);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->g.rank_active, 0, 4, us);
  for (uint32_t i = 0; i < n_probs && e == cudaSuccess; ++i) {
    const DevProblem &d = ctx->hp[i];
    if (d.enc == QE_ENC_QEQEA) {
      e = launch_init_state(ctx->d_probs, i, d.nseg, us);
      if (e == cudaSuccess) e = cudaMemsetAsync(d.mut_cnt, 0, 2 * 4, us);
    }
    else e = launch_ga_init(ctx->d_probs, i, d.P, d.L, ctx->g, us);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(us);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "initialising the state"));
  e = cudaMallocHost(&ctx->h_recs, n_probs * sizeof(Best));
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaMallocHost"));
  e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->gfork, cudaEventDisableTiming);
  for (size_t k = 1; k < ctx->groups.size() && e == cudaSuccess; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t v = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) ctx->gstreams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
    if (e == cudaSuccess) ctx->gjoin.push_back(v);
  }
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "creating streams"));
  *out = ctx;
  return QE_OK;
}

qe_status qe_sample(qe_ctx *ctx, uint32_t prob, uint32_t gen, uint8_t *d_gate_idx,
                    uint32_t *d_seg_id) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (d.enc != QE_ENC_QEQEA) return fail(ctx, QE_ESTATE, "qe_sample needs a QEQEA search");
  if (!d_gate_idx || !d_seg_id) return fail(ctx, QE_EINVAL, "null output buffer");
  QE_CUDA(ctx, launch_sample(ctx->lc, ctx->d_probs, prob, d.P, d.L, gen, d_gate_idx, d_seg_id,
                             ctx->user));
  return QE_OK;
}

// the message of a nonzero device error word (the first bit set, in QE_ERRW_* order)
static const char *errw_text(uint32_t errw) {
  if (errw & kErrBadGate) return "invalid gate index in the circuits";
  if (errw & kErrNonFinite) return "non-finite fitness";
  return "a binary64 fitness lay outside the guard band of its binary32 value (the top-k may "
         "be inexact)";
}

static qe_status rank_single(qe_ctx *ctx, uint32_t prob, uint32_t n, const void *fit,
                             const uint32_t *meta, const uint8_t *gsrc, const float2 *asrc,
                             qe_ranked *h_topk) {
  const DevProblem &d = ctx->hp[prob];
  RankJob j{};
  j.prob = prob;
  j.n = n;
  j.fit = fit;
  j.meta = meta;
  j.gsrc = gsrc;
  j.asrc = asrc;
  j.update_record = 0;
  cudaStream_t us = ctx->user;
  QE_CUDA(ctx, launch_reset_counter(ctx->g, us));
  QE_CUDA(ctx, launch_rank_select(ctx->d_probs, nullptr, 1, j, ctx->g, us, n));
  if (d.prec != QE_PREC_FP64)
    QE_CUDA(ctx, launch_rescore(ctx->lc, d.n, d.ising != 0, ctx->d_probs, gsrc, asrc, false,
                                ctx->g, us));
  QE_CUDA(ctx, launch_rank_sort(ctx->d_probs, nullptr, 1, j, ctx->g, us));
  QE_CUDA(ctx, launch_reset_counter(ctx->g, us));
  const uint32_t k = d.k < n ? d.k : n;
  std::vector<Ranked> tmp(k);
  uint32_t errw = 0;
  if (k) QE_CUDA(ctx, cudaMemcpyAsync(tmp.data(), d.topk_out, k * sizeof(Ranked),
                                      cudaMemcpyDeviceToHost, us));
  QE_CUDA(ctx, cudaMemcpyAsync(&errw, ctx->g.err, 4, cudaMemcpyDeviceToHost, us));
  QE_CUDA(ctx, cudaStreamSynchronize(us));
  for (uint32_t s = 0; s < k; ++s) {
    h_topk[s].circuit = tmp[s].circuit;
    h_topk[s].cost = tmp[s].cost;
    h_topk[s].fitness = tmp[s].fitness;
  }
  if (errw) {
    QE_CUDA(ctx, cudaMemsetAsync(ctx->g.err, 0, 4, us));
    QE_CUDA(ctx, cudaStreamSynchronize(us));
    return fail(ctx, QE_ENUMERIC, errw_text(errw));
  }
  return QE_OK;
}

static qe_status eval_impl(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx,
                           const float2 *d_amps, uint32_t n_circuits, void *d_fitness,
                           uint32_t *d_cost, qe_ranked *h_topk) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (!d_fitness || (n_circuits && !d_gate_idx)) return fail(ctx, QE_EINVAL, "null buffer");
  if (d.ising && n_circuits && !d_amps)
    return fail(ctx, QE_EINVAL, "Ising circuits need their angles (qe_eval_amp)");
  if (n_circuits > (1u << 24)) return fail(ctx, QE_EINVAL, "n_circuits must be <= 2^24");
  if (h_topk && n_circuits > d.P)
    return fail(ctx, QE_EINVAL, "ranking needs n_circuits <= population");
  if (h_topk) {
    st = drain(ctx);  // the ranking scratch and d.meta may still hold a pending ranking
    if (st != QE_OK) return st;
  }
  uint32_t *cost = d_cost ? d_cost : (h_topk ? d.meta : nullptr);
  const float2 *amps = d.ising ? d_amps : nullptr;
  QE_CUDA(ctx, launch_eval(ctx->lc, d.n, ctx->d_probs, prob, d.prec == QE_PREC_FP64, d_gate_idx,
                           amps, n_circuits, d_fitness, cost, nullptr, ctx->g, ctx->user));
  if (!h_topk || n_circuits == 0) return QE_OK;
  return rank_single(ctx, prob, n_circuits, d_fitness, cost, d_gate_idx, amps, h_topk);
}

qe_status qe_eval(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, uint32_t n_circuits,
                  void *d_fitness, uint32_t *d_cost, qe_ranked *h_topk) {
  return eval_impl(ctx, prob, d_gate_idx, nullptr, n_circuits, d_fitness, d_cost, h_topk);
}

qe_status qe_eval_amp(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, const float *d_amps,
                      uint32_t n_circuits, void *d_fitness, uint32_t *d_cost, qe_ranked *h_topk) {
  return eval_impl(ctx, prob, d_gate_idx, (const float2 *)d_amps, n_circuits, d_fitness, d_cost,
                   h_topk);
}

qe_status qe_rank(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, const float *d_amps,
                  const void *d_fitness, const uint32_t *d_cost, uint32_t n_circuits,
                  qe_ranked *h_topk) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (!h_topk) return fail(ctx, QE_EINVAL, "null h_topk");
  if (n_circuits == 0) return QE_OK;
  if (!d_gate_idx || !d_fitness || !d_cost) return fail(ctx, QE_EINVAL, "null buffer");
  if (d.ising && !d_amps) return fail(ctx, QE_EINVAL, "Ising circuits need their angles");
  if (n_circuits > d.P) return fail(ctx, QE_EINVAL, "ranking needs n_circuits <= population");
  st = drain(ctx);  // the ranking scratch may still hold a pending ranking
  if (st != QE_OK) return st;
  return rank_single(ctx, prob, n_circuits, d_fitness, d_cost, d_gate_idx,
                     d.ising ? (const float2 *)d_amps : nullptr, h_topk);
}

qe_status qe_eval_host(qe_ctx *ctx, uint32_t prob, const uint8_t *h_gate_idx,
                       uint32_t n_circuits, void *h_fitness, qe_ranked *h_topk) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (!h_fitness || (n_circuits && !h_gate_idx)) return fail(ctx, QE_EINVAL, "null buffer");
  if (n_circuits > d.P) return fail(ctx, QE_EINVAL, "n_circuits must be <= population");
  if (d.ising) return fail(ctx, QE_EINVAL, "Ising circuits need their angles (qe_eval_amp)");
  const size_t fb = d.prec == QE_PREC_FP64 ? 8 : 4;
  cudaStream_t us = ctx->user;
  st = drain(ctx);
  if (st != QE_OK) return st;
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->d_stage_gates, h_gate_idx, (size_t)n_circuits * d.L,
                               cudaMemcpyHostToDevice, us));
  QE_CUDA(ctx, launch_eval(ctx->lc, d.n, ctx->d_probs, prob, d.prec == QE_PREC_FP64,
                           ctx->d_stage_gates, nullptr, n_circuits, ctx->d_stage_fit, d.meta,
                           nullptr, ctx->g, us));
  if (h_topk && n_circuits) {
    st = rank_single(ctx, prob, n_circuits, ctx->d_stage_fit, d.meta, ctx->d_stage_gates, nullptr,
                     h_topk);
    if (st != QE_OK && st != QE_ENUMERIC) return st;
  }
  QE_CUDA(ctx, cudaMemcpyAsync(h_fitness, ctx->d_stage_fit, n_circuits * fb,
                               cudaMemcpyDeviceToHost, us));
  QE_CUDA(ctx, cudaStreamSynchronize(us));
  return st;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device staging of one batch slot (256-B aligned sections): the error word,
// the items' gates, fitness and cost words back to back, the top-k lists of
// all items plus the error word after them (the call's output), the slot's
// ranking scratch, and what is uploaded once per layout: the ranking jobs,
// their top-k offsets, the per-job gate table the binary64 rescoring reads
// and the jobs' search descriptors.
struct BatchLayout {
  size_t err = 0, gates = 0, fit = 0, cost = 0, topk = 0;
  // the slot's own ranking scratch: candidates, their fitness and counts, the
  // binary64 rescoring queue and its length, the generation words the
  // ranking kernels may read
  size_t cand = 0, cand_f = 0, cand_n = 0, rq = 0, words = 0;
  // uploaded once per layout: jobs, top-k offsets, gate table, the jobs'
  // search descriptors pointing at the slot's scratch, the evaluation jobs
  size_t jobs = 0, koff = 0, gtab = 0, probs = 0, ejobs = 0, total = 0;
};

static BatchLayout batch_layout(size_t gate_bytes, size_t n_total, size_t fb, size_t k_total,
                                size_t n_items) {
  BatchLayout b;
  size_t o = 0;
  b.err = o;  // the slot's device error word
  o += 256;
  b.gates = o;
  o += align256(gate_bytes ? gate_bytes : 1);
  b.fit = o;
  o += align256((n_total ? n_total : 1) * fb);
  b.cost = o;
  o += align256((n_total ? n_total : 1) * 4);
  b.topk = o;
  o += align256((k_total + 1) * sizeof(Ranked));
  b.cand = o;
  o += align256((n_total ? n_total : 1) * 4);
  b.cand_f = o;
  o += align256((n_total ? n_total : 1) * 8);
  b.cand_n = o;
  o += align256(n_items * 4);
  b.rq = o;
  o += align256((n_total ? n_total : 1) * 4);
  b.words = o;  // rescore_n, gen, ranked, rank_active, the copy-out counter
  o += 256;
  b.jobs = o;
  o += align256(n_items * sizeof(RankJob));
  b.koff = o;
  o += align256((n_items + 1) * 4);
  b.gtab = o;
  o += align256(n_items * sizeof(void *));
  b.probs = o;
  o += align256(n_items * sizeof(DevProblem));
  b.ejobs = o;
  o += align256(n_items * sizeof(EvalJob));
  b.total = o;
  return b;
}

// the device address of page-locked host memory, or NULL for other memory
// (the batch graph's copy kernels reach the caller's buffers through it)
static void *host_mapping(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Enqueue one batched host evaluation in a free slot, all on the slot's
// stream: the copy of the gates, the evaluations, the ranking (on the slot's
// own scratch: the jobs' search descriptors are slot copies whose candidate
// lists, counts and top-k lists live in the slot's staging, with the slot's
// own rescoring queue and error word) and the fitness and top-k copies back,
// the copies inside the slot's graph when the caller's buffers are
// page-locked.  Calls in different slots share no device memory, so their
// rankings, latency chains on a few SMs each, run concurrently.
static qe_status batch_submit(qe_ctx *ctx, uint32_t n_items, const uint32_t *h_probs,
                              const uint32_t *h_n_circuits, const uint8_t *h_gate_idx,
                              void *h_fitness, qe_ranked *h_topk, uint64_t *ticket) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  const uint32_t np = (uint32_t)ctx->probs.size();
  if (!h_probs || !h_n_circuits) return fail(ctx, QE_EINVAL, "null item array");
  if (n_items < 1 || n_items > np) return fail(ctx, QE_EINVAL, "n_items must be 1..n_probs");
  std::vector<char> &seen = ctx->b_seen;  // reused: no allocation per call
  seen.assign(np, 0);
  uint32_t prec = 0;
  size_t gate_bytes = 0, n_total = 0, k_total = 0;
  for (uint32_t m = 0; m < n_items; ++m) {
    const uint32_t q = h_probs[m];
    if (q >= np) return fail(ctx, QE_EINVAL, "problem index out of range");
    if (seen[q]) return fail(ctx, QE_EINVAL, "a problem appears twice in the batch");
    seen[q] = 1;
    const DevProblem &d = ctx->hp[q];
    if (d.ising) return fail(ctx, QE_EINVAL, "Ising circuits need their angles (qe_eval_amp)");
    if (h_n_circuits[m] > d.P) return fail(ctx, QE_EINVAL, "n_circuits must be <= population");
    const uint32_t pr = d.prec == QE_PREC_FP64 ? 0u : 1u;
    if (m == 0) prec = pr;
    else if (pr != prec)
      return fail(ctx, QE_EINVAL, "the batch mixes binary32 and binary64 searches");
    gate_bytes += (size_t)h_n_circuits[m] * d.L;
    n_total += h_n_circuits[m];
    k_total += d.k < h_n_circuits[m] ? d.k : h_n_circuits[m];
  }
  if ((gate_bytes && !h_gate_idx) || (n_total && !h_fitness))
    return fail(ctx, QE_EINVAL, "null buffer");
  const size_t fb = prec == 0 ? 8 : 4;
  const bool rank = h_topk != nullptr;
  // page-locked caller buffers are copied by kernels of the call's graph
  // through their device mappings (one launch per call); other memory by
  // copies around the graph.  Checked every call: a graph is only reused for
  // the same mappings.
  void *dg = gate_bytes ? host_mapping(h_gate_idx) : nullptr;
  void *df = n_total ? host_mapping(h_fitness) : nullptr;
  bool fold = (!gate_bytes || dg) && (!n_total || df);
  std::vector<uint32_t> &key = ctx->b_key;
  key.clear();
  key.push_back(rank ? 1u : 0u);
  key.push_back(n_items);
  for (uint32_t m = 0; m < n_items; ++m) {
    key.push_back(h_probs[m]);
    key.push_back(h_n_circuits[m]);
  }
  key.push_back(fold ? 1u : 0u);
  if (fold) {
    const uint64_t pg = (uint64_t)(uintptr_t)dg, pf = (uint64_t)(uintptr_t)df;
    key.push_back((uint32_t)pg);
    key.push_back((uint32_t)(pg >> 32));
    key.push_back((uint32_t)pf);
    key.push_back((uint32_t)(pf >> 32));
  }
  // a free slot whose graph was made for this call; else an unused one; else
  // the free slot used longest ago (callers that cycle through a ring of
  // buffer sets keep one graph per set)
  BatchSlot *slot = nullptr, *spare = nullptr;
  for (BatchSlot &b : ctx->bslot) {
    if (b.busy) continue;
    if (b.ex && b.key == key && b.desc_version == ctx->desc_version) {
      slot = &b;
      break;
    }
    if (!spare || (spare->ex && (!b.ex || b.ticket < spare->ticket))) spare = &b;
  }
  if (!slot) slot = spare;
  if (!slot) return fail(ctx, QE_ESTATE, "every batch slot has a call in flight: wait for one first");
  BatchSlot &b = *slot;
  if (!b.st) {
    QE_CUDA(ctx, cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking));
    QE_CUDA(ctx, cudaEventCreateWithFlags(&b.ev_done, cudaEventDisableTiming));
  }
  // pinned host staging: the top-k lists and, after them, the error word
  // (the gathered lists end with it; without a ranking it is copied alone)
  const size_t kt = rank ? k_total : 0;
  const size_t hb = (kt + 1) * sizeof(Ranked);
  bool new_h = false;
  if (hb > b.h_bytes) {
    QE_CUDA(ctx, cudaStreamSynchronize(b.st));
    if (b.h) cudaFreeHost(b.h);
    b.h = nullptr;
    b.hd = nullptr;
    b.h_bytes = 0;
    QE_CUDA(ctx, cudaHostAlloc(&b.h, hb, cudaHostAllocMapped));
    b.h_bytes = hb;
    if (cudaHostGetDevicePointer(&b.hd, b.h, 0) != cudaSuccess) {
      cudaGetLastError();
      b.hd = nullptr;
    }
    new_h = true;  // a graph that copies into the old staging is stale
  }
  if (fold && !b.hd) {
    // no device mapping of the staging: copies around the graph after all
    fold = false;
    const size_t at = 2 + 2 * (size_t)n_items;
    key.resize(at + 1);
    key[at] = 0u;
  }

  const BatchLayout lay = batch_layout(gate_bytes, n_total, fb, k_total, n_items);
  const bool regrow = lay.total > b.d_bytes;
  if (regrow || new_h || key != b.key || !b.ex || b.desc_version != ctx->desc_version) {
    if (b.ex) cudaGraphExecDestroy(b.ex);
    if (b.eg) cudaGraphDestroy(b.eg);
    b.ex = nullptr;
    b.eg = nullptr;
    b.key.clear();
    if (regrow) {
      QE_CUDA(ctx, cudaStreamSynchronize(b.st));
      if (b.d) cudaFree(b.d);
      b.d = nullptr;
      b.d_bytes = 0;
      QE_CUDA(ctx, cudaMalloc(&b.d, lay.total));
      b.d_bytes = lay.total;
      QE_CUDA(ctx, cudaMemsetAsync((char *)b.d + lay.err, 0, 4, b.st));
    }
    // the rescoring queue's length and the generation words: a new layout
    // puts them where the last one kept other data; from here on each
    // ranking's sort leaves the length at zero for the next call
    QE_CUDA(ctx, cudaMemsetAsync((char *)b.d + lay.words, 0, 256, b.st));
    b.err_off = lay.err;
    char *base = (char *)b.d;
    // this slot's copy of the context's device pointers, with its own error
    // word, rescoring queue and generation words
    DevGlobal gs = ctx->g;
    gs.err = (uint32_t *)(base + lay.err);
    gs.rescore_list = (uint32_t *)(base + lay.rq);
    gs.rescore_n = (uint32_t *)(base + lay.words);
    gs.gen = gs.rescore_n + 1;
    gs.ranked = gs.rescore_n + 2;
    gs.rank_active = gs.rescore_n + 3;
    // jobs, top-k offsets and the gate table, uploaded once per layout
    b.meta.assign(lay.total - lay.jobs, 0);
    RankJob *hj = (RankJob *)b.meta.data();
    uint32_t *hk = (uint32_t *)(b.meta.data() + (lay.koff - lay.jobs));
    const uint8_t **hg = (const uint8_t **)(b.meta.data() + (lay.gtab - lay.jobs));
    DevProblem *hd = (DevProblem *)(b.meta.data() + (lay.probs - lay.jobs));
    std::vector<uint32_t> items;  // items with circuits (ranked)
    size_t go = 0, fo = 0, ko = 0;
    std::vector<size_t> goff(n_items), foff(n_items);
    for (uint32_t m = 0; m < n_items; ++m) {
      const DevProblem &d = ctx->hp[h_probs[m]];
      const uint32_t n = h_n_circuits[m];
      goff[m] = go;
      foff[m] = fo;
      if (n) {
        // job x ranks its search through the slot's descriptor x
        const uint32_t x = (uint32_t)items.size();
        DevProblem &dp = hd[x];
        dp = d;
        dp.cand = (uint32_t *)(base + lay.cand) + fo;
        dp.cand_f = (double *)(base + lay.cand_f) + fo;
        dp.cand_n = (uint32_t *)(base + lay.cand_n) + x;
        // the sort writes the job's list straight into the call's output
        dp.topk_out = (Ranked *)(base + lay.topk) + ko;
        dp.rec = nullptr;  // no job of a batch updates a record
        hg[x] = (const uint8_t *)(base + lay.gates + go);
        RankJob &j = hj[x];
        j.prob = x;
        j.n = n;
        j.fit = base + lay.fit + fo * fb;
        j.meta = (const uint32_t *)(base + lay.cost) + fo;
        j.gsrc = (const uint8_t *)(base + lay.gates + go);
        j.asrc = nullptr;
        j.update_record = 0;
        j.pipelined = 0;
        hk[items.size()] = (uint32_t)ko;
        ko += d.k < n ? d.k : n;
        items.push_back(m);
      }
      go += (size_t)n * d.L;
      fo += n;
    }
    const uint32_t n_jobs = (uint32_t)items.size();
    hk[n_jobs] = (uint32_t)ko;
    // the evaluation jobs grouped by width: one launch per width present, its
    // jobs' circuits numbered consecutively
    EvalJob *he = (EvalJob *)(b.meta.data() + (lay.ejobs - lay.jobs));
    uint32_t w_first[QE_MAX_QUBITS + 1] = {0}, w_jobs[QE_MAX_QUBITS + 1] = {0};
    uint32_t w_total[QE_MAX_QUBITS + 1] = {0};
    uint32_t ne = 0;
    for (uint32_t nq = 1; nq <= QE_MAX_QUBITS; ++nq) {
      w_first[nq] = ne;
      for (uint32_t x = 0; x < n_jobs; ++x) {
        const uint32_t m = items[x];
        if (ctx->hp[h_probs[m]].n != nq) continue;
        EvalJob &ej = he[ne++];
        ej.prob = x;
        ej.first = w_total[nq];
        ej.n = h_n_circuits[m];
        ej.pad = 0;
        ej.gates = (const uint8_t *)(base + lay.gates + goff[m]);
        ej.fit = base + lay.fit + foff[m] * fb;
        ej.cost = (uint32_t *)(base + lay.cost) + foff[m];
        w_total[nq] += h_n_circuits[m];
        ++w_jobs[nq];
      }
    }
    QE_CUDA(ctx, cudaMemcpyAsync(base + lay.jobs, b.meta.data(), b.meta.size(),
                                 cudaMemcpyHostToDevice, b.st));
    // the evaluations: one launch per width, on up to three captured streams
    // when there are several widths (one width: a single chain)
    const DevProblem *sprobs = (const DevProblem *)(base + lay.probs);
    const EvalJob *dej = (const EvalJob *)(base + lay.ejobs);
    uint32_t n_widths = 0;
    for (uint32_t nq = 1; nq <= QE_MAX_QUBITS; ++nq) n_widths += w_jobs[nq] ? 1u : 0u;
    cudaStream_t cs = ctx->cap;
    cudaStream_t lanes[3] = {cs, ctx->side, ctx->side2};
    QE_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (fold && gate_bytes)  // the circuits in, ahead of every evaluation
      e = launch_copy_in(base + lay.gates, dg, gate_bytes, ctx->lc.num_sms, cs);
    const bool forked = n_widths > 1;
    if (forked) {
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, cs);
      for (int l = 1; l < 3 && e == cudaSuccess; ++l)
        e = cudaStreamWaitEvent(lanes[l], ctx->ev_fork, 0);
    }
    for (uint32_t nq = 1, wi = 0; nq <= QE_MAX_QUBITS && e == cudaSuccess; ++nq) {
      if (!w_jobs[nq]) continue;
      e = launch_eval_jobs(ctx->lc, nq, prec == 0, sprobs, dej + w_first[nq], w_jobs[nq],
                           w_total[nq], gs, lanes[forked ? wi % 3 : 0]);
      ++wi;
    }
    if (forked) {
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->side);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join2, ctx->side2);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->ev_join, 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->ev_join2, 0);
    }
    // then, in the same graph, the ranking of every item with circuits: the
    // jobs' descriptors send each sorted list straight to its place in the
    // gathered output, and the sort writes the error word after them and
    // clears the slot's rescoring queue (zero when the slot is allocated)
    if (rank && e == cudaSuccess) {
      const RankJob *dj = (const RankJob *)(base + lay.jobs);
      Ranked *gathered = (Ranked *)(base + lay.topk);
      if (n_jobs) {
        uint32_t max_n = 0;
        for (uint32_t x = 0; x < n_jobs; ++x)
          max_n = h_n_circuits[items[x]] > max_n ? h_n_circuits[items[x]] : max_n;
        e = launch_rank_select(sprobs, dj, n_jobs, RankJob{}, gs, cs, max_n);
        if (prec != 0) {
          uint32_t widths = 0;
          for (uint32_t x = 0; x < n_jobs; ++x) widths |= 1u << ctx->hp[h_probs[items[x]]].n;
          for (uint32_t nq = 1; nq <= QE_MAX_QUBITS; ++nq)
            if (e == cudaSuccess && ((widths >> nq) & 1))
              e = launch_rescore(ctx->lc, nq, false, sprobs, nullptr, nullptr, false, gs, cs,
                                 (const uint8_t *const *)(base + lay.gtab),
                                 (uint32_t)(4 * k_total));
        }
        if (e == cudaSuccess)
          e = launch_rank_sort(sprobs, dj, n_jobs, RankJob{}, gs, cs, gathered + k_total);
      } else {
        // nothing to rank: the error word alone
        e = launch_gather_topk(sprobs, dj, (const uint32_t *)(base + lay.koff), 0, gathered, gs,
                               cs);
      }
    }
    if (fold && e == cudaSuccess) {
      // the fitness and the lists out after the sort, and then, once all of
      // them are visible to the host, the error word: the wait polls for it
      // in the staging.  (Copy-engine nodes for these copies measured ~0.8 us
      // of host launch time each against ~0.2 us for a kernel node.)
      e = launch_copy_out(df, base + lay.fit, n_total * fb, b.hd, base + lay.topk,
                          rank ? kt * sizeof(Ranked) : 0,
                          (uint32_t *)((char *)b.hd + kt * sizeof(Ranked)),
                          (const uint32_t *)(base + (rank ? lay.topk + kt * sizeof(Ranked)
                                                          : lay.err)),
                          (uint32_t *)(base + lay.words) + 4, ctx->lc.num_sms, cs);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e, "capturing the batch graph");
    }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    b.eg = graph;
    qe_status pst = add_pdl_edges(ctx, graph, true);
    if (pst != QE_OK) return pst;
    QE_CUDA(ctx, cudaGraphInstantiate(&b.ex, graph, 0));
    b.key = key;
    b.desc_version = ctx->desc_version;
  }
  char *base = (char *)b.d;
  if (fold) {
    // the slot is idle: nothing of its last call writes the staging any more
    ((volatile uint32_t *)((char *)b.h + kt * sizeof(Ranked)))[0] = kErrwPending;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    QE_CUDA(ctx, cudaGraphLaunch(b.ex, b.st));
  } else {
    if (gate_bytes)
      QE_CUDA(ctx, cudaMemcpyAsync(base + lay.gates, h_gate_idx, gate_bytes,
                                   cudaMemcpyHostToDevice, b.st));
    QE_CUDA(ctx, cudaGraphLaunch(b.ex, b.st));
    if (n_total)
      QE_CUDA(ctx, cudaMemcpyAsync(h_fitness, base + lay.fit, n_total * fb,
                                   cudaMemcpyDeviceToHost, b.st));
    if (rank) QE_CUDA(ctx, cudaMemcpyAsync(b.h, base + lay.topk, hb, cudaMemcpyDeviceToHost, b.st));
    else QE_CUDA(ctx, cudaMemcpyAsync(b.h, base + lay.err, 4, cudaMemcpyDeviceToHost, b.st));
    QE_CUDA(ctx, cudaEventRecord(b.ev_done, b.st));
  }
  b.busy = true;
  b.flag = fold;
  b.ticket = ctx->next_ticket++;
  b.h_topk = h_topk;
  b.k_total = kt;
  if (ticket) *ticket = b.ticket;
  return QE_OK;
}

// Wait for a slot's call and hand out its top-k lists and error status.
static qe_status batch_complete(qe_ctx *ctx, BatchSlot &b) {
  b.busy = false;
  if (b.flag) {
    // poll the error word's slot for up to 2 ms, then block on the stream (a
    // long call, or a failed one whose copies never ran: the stream's error)
    const volatile uint32_t *w =
        (const volatile uint32_t *)((const char *)b.h + b.k_total * sizeof(Ranked));
    bool seen = false;
    const auto t0 = std::chrono::steady_clock::now();
    for (uint32_t i = 0; !seen; ++i) {
      seen = *w != kErrwPending;
      if (!seen && (i & 255u) == 255u &&
          std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(2))
        break;
    }
    if (seen) std::atomic_thread_fence(std::memory_order_acquire);
    else QE_CUDA(ctx, cudaStreamSynchronize(b.st));
  } else {
    QE_CUDA(ctx, cudaEventSynchronize(b.ev_done));
  }
  const Ranked *r = (const Ranked *)b.h;
  for (size_t s = 0; s < b.k_total; ++s) {
    b.h_topk[s].circuit = r[s].circuit;
    b.h_topk[s].cost = r[s].cost;
    b.h_topk[s].fitness = r[s].fitness;
  }
  const uint32_t errw = r[b.k_total].circuit;
  if (errw) {
    QE_CUDA(ctx, cudaMemsetAsync((char *)b.d + b.err_off, 0, 4, b.st));
    QE_CUDA(ctx, cudaStreamSynchronize(b.st));
    return fail(ctx, QE_ENUMERIC, errw_text(errw));
  }
  return QE_OK;
}

qe_status qe_eval_host_batch(qe_ctx *ctx, uint32_t n_items, const uint32_t *h_probs,
                             const uint32_t *h_n_circuits, const uint8_t *h_gate_idx,
                             void *h_fitness, qe_ranked *h_topk) {
  uint64_t t = 0;
  qe_status st = batch_submit(ctx, n_items, h_probs, h_n_circuits, h_gate_idx, h_fitness, h_topk,
                              &t);
  if (st != QE_OK) return st;
  return qe_eval_host_batch_wait(ctx, t);
}

qe_status qe_eval_host_batch_async(qe_ctx *ctx, uint32_t n_items, const uint32_t *h_probs,
                                   const uint32_t *h_n_circuits, const uint8_t *h_gate_idx,
                                   void *h_fitness, qe_ranked *h_topk, uint64_t *ticket) {
  if (!ticket) return fail(ctx, QE_EINVAL, "null ticket");
  return batch_submit(ctx, n_items, h_probs, h_n_circuits, h_gate_idx, h_fitness, h_topk,
                      ticket);
}

qe_status qe_eval_host_batch_wait(qe_ctx *ctx, uint64_t ticket) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  for (BatchSlot &b : ctx->bslot)
    if (b.busy && b.ticket == ticket) return batch_complete(ctx, b);
  return fail(ctx, QE_EINVAL, "no batched call in flight with this ticket");
}

static qe_status compose_impl(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx,
                              const float2 *d_amps, uint32_t n_circuits, void *d_unitary) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (!d_unitary || (n_circuits && !d_gate_idx)) return fail(ctx, QE_EINVAL, "null buffer");
  if (n_circuits > (1u << 20)) return fail(ctx, QE_EINVAL, "n_circuits must be <= 2^20");
  if (d.ising && n_circuits && !d_amps)
    return fail(ctx, QE_EINVAL, "Ising circuits need their angles (qe_compose_amp)");
  QE_CUDA(ctx, launch_eval(ctx->lc, d.n, ctx->d_probs, prob, d.prec == QE_PREC_FP64, d_gate_idx,
                           d.ising ? d_amps : nullptr, n_circuits, nullptr, nullptr, d_unitary,
                           ctx->g, ctx->user));
  return QE_OK;
}

qe_status qe_compose(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, uint32_t n_circuits,
                     void *d_unitary) {
  return compose_impl(ctx, prob, d_gate_idx, nullptr, n_circuits, d_unitary);
}

qe_status qe_compose_amp(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx,
                         const float *d_amps, uint32_t n_circuits, void *d_unitary) {
  return compose_impl(ctx, prob, d_gate_idx, (const float2 *)d_amps, n_circuits, d_unitary);
}

qe_status qe_update(qe_ctx *ctx, uint32_t prob, uint32_t gen, const uint32_t *d_seg_id,
                    const double *d_fitness) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (d.enc != QE_ENC_QEQEA) return fail(ctx, QE_ESTATE, "qe_update needs a QEQEA search");
  if (!d_seg_id || !d_fitness) return fail(ctx, QE_EINVAL, "null buffer");
  cudaStream_t us = ctx->user;
  QE_CUDA(ctx, launch_scatter(ctx->d_probs, prob, d.P, d.L, d_seg_id, d_fitness, ctx->g.err, us));
  const uint32_t *s = ctx->d_single + 5 * prob;
  QE_CUDA(ctx, launch_update(ctx->lc, ctx->d_probs, s, s + 1, s + 3, 1, d.P * d.L,
                             ((d.P + 31) / 32) * d.R, nullptr, gen, d_seg_id, ctx->g, us, us));
  return QE_OK;
}

qe_status qe_step(qe_ctx *ctx, uint32_t n_gen, qe_report *h_reports) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  if (!ctx->gexec) {
    qe_status st = build_graph(ctx);
    if (st != QE_OK) return st;
  }
  for (uint32_t k = 0; k < n_gen; ++k) QE_CUDA(ctx, cudaGraphLaunch(ctx->gexec, ctx->user));
  ctx->gen += n_gen;
  if (n_gen) ctx->pending_rank = ctx->has_last = true;
  if (!h_reports) return QE_OK;  // enqueued only; the last generation ranks later
  {
    qe_status st = drain(ctx);
    if (st != QE_OK) return st;
  }
  const uint32_t np = (uint32_t)ctx->probs.size();
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->h_recs, ctx->d_recs, np * sizeof(Best), cudaMemcpyDeviceToHost,
                               ctx->user));
  QE_CUDA(ctx, cudaStreamSynchronize(ctx->user));
  uint32_t errw = 0;
  for (uint32_t i = 0; i < np; ++i) {
    const Best &b = ctx->h_recs[i];
    errw |= b.error_word;
    qe_report &r = h_reports[i];
    r.generation = b.generation;
    r.best_gen = b.best_gen;
    r.best_fitness = b.best_fitness;
    r.gen_best_fitness = b.gen_best_fitness;
    r.mean_fitness = b.mean_fitness;
    r.useful_flops = b.useful_flops;
    r.best_cost = b.best_cost;
    r.best_len = b.best_len;
    r.error_word = b.error_word;
    r.reserved = 0;
    memcpy(r.best_gates, b.best_gates, 64);
    memcpy(r.best_amps, b.best_amps, sizeof r.best_amps);
  }
  if (errw) return fail(ctx, QE_ENUMERIC, errw_text(errw));
  return QE_OK;
}

qe_status qe_autotune(qe_ctx *ctx, uint32_t gens_per_plan, float *h_ms, uint32_t *n_plans) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  if (ctx->timing) return fail(ctx, QE_ESTATE, "qe_autotune needs stage timing off");
  if (gens_per_plan < 1 || gens_per_plan > 64)
    return fail(ctx, QE_EINVAL, "gens_per_plan must be 1..64");
  if (!ctx->gexec) {
    qe_status st = build_graph(ctx);  // also the drain graph
    if (st != QE_OK) return st;
  }
  // candidate plans: with and without the selection-first edge, three grids
  // (the middle one only where some circuit kernel keeps several blocks per SM)
  bool several = false;
  for (auto &gr : ctx->groups)
    several = several || (gr.canon ? ctx->lc.step64[gr.n] : ctx->lc.step32[gr.n]) > 1;
  std::vector<Plan> cands;
  const int n_conc = ctx->groups.size() > 1 ? 2 : 1;
  for (int cc = 0; cc < n_conc; ++cc)
    for (int sf = 1; sf >= 0; --sf)
      for (uint32_t gm = 0; gm < 3; ++gm) {
        if (gm == 1 && !several) continue;
        Plan p;
        p.select_first = sf == 1;
        p.grid_mode = gm;
        p.concurrent = cc == 1;
        cands.push_back(p);
      }
  const size_t C = cands.size();
  std::vector<cudaGraph_t> graphs(C, nullptr);
  std::vector<cudaGraphExec_t> execs(C, nullptr);
  std::vector<cudaEvent_t> ev(2 * C, nullptr);
  auto cleanup = [&](size_t keep) {
    for (size_t i = 0; i < C; ++i) {
      if (i == keep) continue;
      if (execs[i]) cudaGraphExecDestroy(execs[i]);
      if (graphs[i]) cudaGraphDestroy(graphs[i]);
    }
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  };
  qe_status st = QE_OK;
  cudaError_t e = cudaSuccess;
  uint32_t launched = 0;
  // every candidate runs real generations: one to settle, then gens_per_plan timed
  for (size_t i = 0; i < C && st == QE_OK && e == cudaSuccess; ++i) {
    st = build_gen_graph(ctx, cands[i], &graphs[i], &execs[i]);
    if (st != QE_OK) break;
    e = cudaEventCreate(&ev[2 * i]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[2 * i + 1]);
    if (e == cudaSuccess) e = cudaGraphLaunch(execs[i], ctx->user);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i], ctx->user);
    for (uint32_t k = 0; k < gens_per_plan && e == cudaSuccess; ++k)
      e = cudaGraphLaunch(execs[i], ctx->user);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], ctx->user);
    if (e == cudaSuccess) launched += 1 + gens_per_plan;
  }
  if (e == cudaSuccess && st == QE_OK) e = cudaStreamSynchronize(ctx->user);
  ctx->gen += launched;
  if (launched) ctx->pending_rank = ctx->has_last = true;
  if (st != QE_OK || e != cudaSuccess) {
    cleanup(C);
    return st != QE_OK ? st : cuda_fail(ctx, e, "autotuning the generation graph");
  }
  std::vector<float> ms(C, 0.f);
  size_t best = 0;
  for (size_t i = 0; i < C; ++i) {
    e = cudaEventElapsedTime(&ms[i], ev[2 * i], ev[2 * i + 1]);
    if (e != cudaSuccess) {
      cleanup(C);
      return cuda_fail(ctx, e, "cudaEventElapsedTime");
    }
    ms[i] /= (float)gens_per_plan;
    if (ms[i] < ms[best]) best = i;
  }
  cleanup(best);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph = graphs[best];
  ctx->gexec = execs[best];
  ctx->plan = cands[best];
  ctx->tuned = true;
  char b[96];
  snprintf(b, sizeof b, " (autotuned: %.4f ms per generation; %zu plans tried)", ms[best], C);
  ctx->plan_text = plan_string(ctx->plan) + b;
  if (n_plans) {
    const uint32_t cap = *n_plans;
    if (h_ms)
      for (size_t i = 0; i < C && i < cap; ++i) h_ms[i] = ms[i];
    *n_plans = (uint32_t)C;
  }
  return QE_OK;
}

qe_status qe_launch_plan(const qe_ctx *ctx, char *h_buf, size_t len) {
  if (!ctx || !h_buf || !len) return QE_EINVAL;
  const std::string t = ctx->plan_text.empty() ? plan_string(ctx->plan) + " (default)"
                                               : ctx->plan_text;
  snprintf(h_buf, len, "%s", t.c_str());
  return QE_OK;
}

qe_status qe_stage_timing(qe_ctx *ctx, int enable) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  if (enable < 0 || enable > 2) return fail(ctx, QE_EINVAL, "stage timing mode must be 0, 1 or 2");
  const bool want = enable != 0, serial = enable == 2;
  if (want == ctx->timing && (!want || serial == ctx->timing_serial)) return QE_OK;
  QE_CUDA(ctx, cudaStreamSynchronize(ctx->user));
  if (want && !ctx->tev[0])
    for (auto &ev : ctx->tev) QE_CUDA(ctx, cudaEventCreate(&ev));
  qe_status dst = drain(ctx);
  if (dst != QE_OK) return dst;
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  if (ctx->graph) {
    cudaGraphDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (ctx->dexec) {
    cudaGraphExecDestroy(ctx->dexec);
    ctx->dexec = nullptr;
  }
  if (ctx->dgraph) {
    cudaGraphDestroy(ctx->dgraph);
    ctx->dgraph = nullptr;
  }
  ctx->timing = want;
  ctx->timing_serial = want && serial;
  return QE_OK;
}

qe_status qe_stage_times(qe_ctx *ctx, float *ms) {
  if (!ctx || !ms) return fail(ctx, QE_EINVAL, "null argument");
  if (!ctx->timing || !ctx->gexec) return fail(ctx, QE_ESTATE, "stage timing is not enabled");
  QE_CUDA(ctx, cudaStreamSynchronize(ctx->user));
  // serialised: the selection starts after the update, not with the generation
  const int sel0 = ctx->timing_serial ? 6 : 0;
  const int pairs[6][2] = {{0, 1}, {sel0, 2}, {2, 3}, {3, 4}, {5, 6}, {0, 7}};
  for (int k = 0; k < 6; ++k)
    QE_CUDA(ctx, cudaEventElapsedTime(&ms[k], ctx->tev[pairs[k][0]], ctx->tev[pairs[k][1]]));
  return QE_OK;
}

qe_status qe_generation(const qe_ctx *ctx, uint32_t *gen) {
  if (!ctx || !gen) return QE_EINVAL;
  *gen = ctx->gen;
  return QE_OK;
}

qe_status qe_last_generation(qe_ctx *ctx, uint32_t prob, uint8_t *h_gate_idx, uint32_t *h_seg_id,
                             double *h_fitness, qe_ranked *h_topk) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  if (!ctx->has_last) return fail(ctx, QE_ESTATE, "no generation has run since qe_init or qe_load");
  const DevProblem &d = ctx->hp[prob];
  cudaStream_t us = ctx->user;
  st = drain(ctx);
  if (st != QE_OK) return st;
  const size_t PL = (size_t)d.P * d.L;
  const size_t b = (ctx->gen - 1) & 1u;  // buffer of the last generation
  std::vector<float> f32;
  std::vector<Ranked> tk;
  if (h_gate_idx)
    QE_CUDA(ctx, cudaMemcpyAsync(h_gate_idx, d.gate_idx + b * PL, PL, cudaMemcpyDeviceToHost, us));
  if (h_seg_id && d.seg_id)
    QE_CUDA(ctx, cudaMemcpyAsync(h_seg_id, d.seg_id, PL * 4, cudaMemcpyDeviceToHost, us));
  if (h_fitness) {
    if (d.prec == QE_PREC_FP64) {
      QE_CUDA(ctx, cudaMemcpyAsync(h_fitness, d.fit64 + b * d.P, (size_t)d.P * 8,
                                   cudaMemcpyDeviceToHost, us));
    } else {
      f32.resize(d.P);
      QE_CUDA(ctx, cudaMemcpyAsync(f32.data(), d.fit32 + b * d.P, (size_t)d.P * 4,
                                   cudaMemcpyDeviceToHost, us));
    }
  }
  if (h_topk) {
    tk.resize(d.k);
    QE_CUDA(ctx, cudaMemcpyAsync(tk.data(), d.topk_out, d.k * sizeof(Ranked),
                                 cudaMemcpyDeviceToHost, us));
  }
  QE_CUDA(ctx, cudaStreamSynchronize(us));
  if (h_fitness && !f32.empty())
    for (uint32_t c = 0; c < d.P; ++c) h_fitness[c] = (double)f32[c];
  if (h_topk)
    for (uint32_t s = 0; s < d.k; ++s) {
      h_topk[s].circuit = tk[s].circuit;
      h_topk[s].cost = tk[s].cost;
      h_topk[s].fitness = tk[s].fitness;
    }
  return QE_OK;
}

qe_status qe_state_bytes(const qe_ctx *ctx, uint32_t prob, size_t *bytes) {
  if (!ctx || !bytes || prob >= ctx->probs.size()) return QE_EINVAL;
  const DevProblem &d = ctx->hp[prob];
  if (d.enc == QE_ENC_QEQEA) *bytes = (size_t)d.nseg * (32 + 32 + 4);
  else *bytes = (size_t)d.P * d.L * (d.ising ? 1 + 8 : 1);  // genes (+ Ising angles)
  return QE_OK;
}

static qe_status state_copy(qe_ctx *ctx, uint32_t prob, void *h, size_t bytes, bool out) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  size_t need = 0;
  qe_state_bytes(ctx, prob, &need);
  if (!h || bytes != need) return fail(ctx, QE_EINVAL, "state buffer must be qe_state_bytes long");
  const DevProblem &d = ctx->hp[prob];
  cudaStream_t us = ctx->user;
  const cudaMemcpyKind kd = out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
  char *hb = (char *)h;
  if (d.enc == QE_ENC_QEQEA) {
    // the caller's layout is cur[S][8], best[S][8], best_f[S]; on the device
    // cur and best share a 64-B line and best_f sits beside the fitness key
    const size_t S = d.nseg;
    char *sg = (char *)d.segs, *fk = (char *)d.fk;
    struct Part {
      char *dev;
      size_t dpitch, width, host_off;
    } parts[3] = {{sg, 64, 32, 0}, {sg + 32, 64, 32, S * 32}, {fk, 8, 4, S * 64}};
    for (const Part &pt : parts) {
      if (out)
        QE_CUDA(ctx, cudaMemcpy2DAsync(hb + pt.host_off, pt.width, pt.dev, pt.dpitch, pt.width, S,
                                       kd, us));
      else
        QE_CUDA(ctx, cudaMemcpy2DAsync(pt.dev, pt.dpitch, hb + pt.host_off, pt.width, pt.width, S,
                                       kd, us));
    }
  } else {
    // the genome the next generation evaluates: the genes, then (Ising) their
    // angles as qubit amplitudes, two floats a gene
    const size_t PL = (size_t)d.P * d.L;
    uint8_t *genome = d.gate_idx + (size_t)(ctx->gen & 1u) * PL;
    if (!out)
      for (size_t e = 0; e < PL; ++e)
        if (((const uint8_t *)hb)[e] >= d.G)
          return fail(ctx, QE_EINVAL, "genome holds a gate index outside the library");
    if (out) QE_CUDA(ctx, cudaMemcpyAsync(hb, genome, PL, kd, us));
    else QE_CUDA(ctx, cudaMemcpyAsync(genome, hb, PL, kd, us));
    if (d.ising) {
      float2 *am = d.amps + (size_t)(ctx->gen & 1u) * PL;
      if (out) QE_CUDA(ctx, cudaMemcpyAsync(hb + PL, am, PL * sizeof(float2), kd, us));
      else QE_CUDA(ctx, cudaMemcpyAsync(am, hb + PL, PL * sizeof(float2), kd, us));
    }
  }
  QE_CUDA(ctx, cudaStreamSynchronize(us));
  return QE_OK;
}

qe_status qe_get_state(qe_ctx *ctx, uint32_t prob, void *h_buf, size_t bytes) {
  return state_copy(ctx, prob, h_buf, bytes, true);
}

qe_status qe_set_state(qe_ctx *ctx, uint32_t prob, const void *h_buf, size_t bytes) {
  return state_copy(ctx, prob, const_cast<void *>(h_buf), bytes, false);
}

}  // extern "C"

// Install (T != NULL, checked already) or clear search prob's dense target:
// both binary32 and binary64 copies, the flag and the ranking bound in the
// device descriptor.  Synchronises.
static qe_status put_target(qe_ctx *ctx, uint32_t prob, const double *T) {
  DevProblem &d = ctx->hp[prob];
  cudaStream_t us = ctx->user;
  // batch calls in flight read the target: let them finish first
  for (BatchSlot &b : ctx->bslot)
    if (b.busy) QE_CUDA(ctx, cudaStreamSynchronize(b.st));
  ++ctx->desc_version;
  const uint32_t NN = d.N * d.N;
  std::vector<double> &keep = ctx->targets[prob];
  if (T) {
    keep.assign(T, T + 2 * NN);
    std::vector<float2> t32(NN);
    std::vector<double2> t64(NN);
    for (uint32_t e = 0; e < NN; ++e) {
      t32[e] = make_float2((float)T[2 * e], (float)T[2 * e + 1]);
      t64[e] = make_double2(T[2 * e], T[2 * e + 1]);
    }
    QE_CUDA(ctx, cudaMemcpyAsync(d.tgt32, t32.data(), NN * sizeof(float2), cudaMemcpyHostToDevice, us));
    QE_CUDA(ctx, cudaMemcpyAsync(d.tgt64, t64.data(), NN * sizeof(double2), cudaMemcpyHostToDevice, us));
  } else {
    keep.clear();
  }
  if ((d.dense != 0) != (T != nullptr)) {
    // the search's group may need the other circuit kernel: recapture the
    // generation graph at the next qe_step (the launch plan is kept)
    QE_CUDA(ctx, cudaStreamSynchronize(us));
    if (ctx->gexec) {
      cudaGraphExecDestroy(ctx->gexec);
      ctx->gexec = nullptr;
    }
    if (ctx->graph) {
      cudaGraphDestroy(ctx->graph);
      ctx->graph = nullptr;
    }
  }
  d.dense = T ? 1u : 0u;
  d.eps_d = T ? eps_d_dense(d.L, d.N) : eps_d_for(d.L);
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->d_probs + prob, &d, sizeof(DevProblem), cudaMemcpyHostToDevice, us));
  QE_CUDA(ctx, cudaStreamSynchronize(us));
  return QE_OK;
}

extern "C" qe_status qe_set_target(qe_ctx *ctx, uint32_t prob, const double *h_target) {
  qe_status st = check_ctx(ctx, prob);
  if (st != QE_OK) return st;
  const DevProblem &d = ctx->hp[prob];
  if (h_target && d.fit_kind != QE_FIT_TRACE)
    return fail(ctx, QE_EUNSUPPORTED, "a dense target takes the trace fitness of Eq. (11)");
  if (h_target && !target_ok(h_target, d.N))
    return fail(ctx, QE_EINVAL, "target is not a finite unitary (T^dag T = I to 1e-6)");
  if ((st = drain(ctx)) != QE_OK) return st;  // rank a pending generation on its own target
  return put_target(ctx, prob, h_target);
}

// ------------------------------------------------------------ checkpoints
// File: CkptHeader, then the payload {qe_problem[n], qe_report[n], and per
// search a uint64 byte count and its state in the qe_get_state layout, then a
// uint64 byte count and its dense target (none: the permutation)}, all
// little-endian as the host writes them; the header carries the payload's
// FNV-1a 64-bit hash.  Philox draws are keyed by (seed, generation, ...), so
// the encoding state, the best-so-far records and the generation counter are
// the whole state of a run: a loaded context continues it bit for bit.
namespace {

struct CkptHeader {
  char magic[8];  // "QECKPT1"
  uint32_t version, n_probs, gen, problem_bytes, report_bytes, reserved;
  uint64_t payload_bytes, hash;
};
static_assert(sizeof(CkptHeader) == 48, "checkpoint header layout");
const char kCkptMagic[8] = {'Q', 'E', 'C', 'K', 'P', 'T', '1', 0};
constexpr uint32_t kCkptVersion = 1;

uint64_t fnv1a64(const char *b, size_t n) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= (uint8_t)b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Reads and checks a whole checkpoint file: magic, version, struct sizes,
// payload length and hash.  On success the payload starts with the problems.
qe_status read_ckpt(qe_ctx *ctx, const char *path, CkptHeader &hd, std::vector<char> &pay) {
  if (!path) return fail(ctx, QE_EINVAL, "null path");
  FILE *f = fopen(path, "rb");
  if (!f) return fail(ctx, QE_EIO, std::string("cannot open ") + path);
  bool ok = fread(&hd, sizeof hd, 1, f) == 1;
  if (ok && (memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion ||
             hd.problem_bytes != sizeof(qe_problem) || hd.report_bytes != sizeof(qe_report) ||
             hd.n_probs == 0 || hd.payload_bytes > ((uint64_t)1 << 40))) {
    fclose(f);
    return fail(ctx, QE_EINVAL, "not a checkpoint of this format version");
  }
  if (ok) {
    pay.resize(hd.payload_bytes);
    ok = hd.payload_bytes == 0 || fread(pay.data(), 1, pay.size(), f) == pay.size();
    char extra;
    ok = ok && fread(&extra, 1, 1, f) == 0;  // nothing after the payload
  }
  fclose(f);
  if (!ok || fnv1a64(pay.data(), pay.size()) != hd.hash)
    return fail(ctx, QE_EINVAL, "checkpoint is truncated or corrupted");
  if (pay.size() < (uint64_t)hd.n_probs * (sizeof(qe_problem) + sizeof(qe_report)))
    return fail(ctx, QE_EINVAL, "checkpoint is truncated or corrupted");
  return QE_OK;
}

void report_of(const Best &b, qe_report &r) {
  memset(&r, 0, sizeof r);
  r.generation = b.generation;
  r.best_gen = b.best_gen;
  r.best_fitness = b.best_fitness;
  r.gen_best_fitness = b.gen_best_fitness;
  r.mean_fitness = b.mean_fitness;
  r.useful_flops = b.useful_flops;
  r.best_cost = b.best_cost;
  r.best_len = b.best_len;
  r.error_word = b.error_word;
  memcpy(r.best_gates, b.best_gates, 64);
  memcpy(r.best_amps, b.best_amps, sizeof r.best_amps);
}

void best_of(const qe_report &r, Best &b) {
  memset(&b, 0, sizeof b);
  b.generation = r.generation;
  b.best_gen = r.best_gen;
  b.best_fitness = r.best_fitness;
  b.gen_best_fitness = r.gen_best_fitness;
  b.mean_fitness = r.mean_fitness;
  b.useful_flops = r.useful_flops;
  b.best_cost = r.best_cost;
  b.best_len = r.best_len;
  b.error_word = r.error_word;
  memcpy(b.best_gates, r.best_gates, 64);
  memcpy(b.best_amps, r.best_amps, sizeof b.best_amps);
}

}  // namespace

extern "C" {

qe_status qe_save(qe_ctx *ctx, const char *path) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  if (!path) return fail(ctx, QE_EINVAL, "null path");
  qe_status st = drain(ctx);  // the last generation's record
  if (st != QE_OK) return st;
  const uint32_t np = (uint32_t)ctx->probs.size();
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->h_recs, ctx->d_recs, np * sizeof(Best), cudaMemcpyDeviceToHost,
                               ctx->user));
  QE_CUDA(ctx, cudaStreamSynchronize(ctx->user));
  std::vector<char> pay(np * (sizeof(qe_problem) + sizeof(qe_report)));
  memcpy(pay.data(), ctx->probs.data(), np * sizeof(qe_problem));
  for (uint32_t i = 0; i < np; ++i) {
    qe_report r;
    report_of(ctx->h_recs[i], r);
    memcpy(pay.data() + np * sizeof(qe_problem) + i * sizeof(qe_report), &r, sizeof r);
  }
  for (uint32_t i = 0; i < np; ++i) {
    size_t nb = 0;
    qe_state_bytes(ctx, i, &nb);
    const size_t at = pay.size();
    pay.resize(at + 8 + nb);
    const uint64_t nb64 = nb;
    memcpy(pay.data() + at, &nb64, 8);
    if ((st = state_copy(ctx, i, pay.data() + at + 8, nb, true)) != QE_OK) return st;
    const std::vector<double> &T = ctx->targets[i];
    const uint64_t tb = T.size() * sizeof(double);
    pay.resize(pay.size() + 8 + tb);
    memcpy(pay.data() + at + 8 + nb, &tb, 8);
    if (tb) memcpy(pay.data() + at + 16 + nb, T.data(), tb);
  }
  CkptHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.n_probs = np;
  hd.gen = ctx->gen;
  hd.problem_bytes = sizeof(qe_problem);
  hd.report_bytes = sizeof(qe_report);
  hd.payload_bytes = pay.size();
  hd.hash = fnv1a64(pay.data(), pay.size());
  // write beside the target, then rename over it: a crash leaves the old file
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(ctx, QE_EIO, "cannot create " + tmp);
  bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 && fwrite(pay.data(), 1, pay.size(), f) == pay.size();
  ok = fflush(f) == 0 && ok;
  ok = fsync(fileno(f)) == 0 && ok;
  ok = fclose(f) == 0 && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return fail(ctx, QE_EIO, std::string("cannot write ") + path);
  }
  return QE_OK;
}

qe_status qe_load(qe_ctx *ctx, const char *path) {
  if (!ctx) return fail(nullptr, QE_EINVAL, "null context");
  if (ctx->poisoned) return fail(ctx, QE_ESTATE, "context is poisoned by an earlier CUDA error");
  CkptHeader hd;
  std::vector<char> pay;
  qe_status st = read_ckpt(ctx, path, hd, pay);
  if (st != QE_OK) return st;
  const uint32_t np = (uint32_t)ctx->probs.size();
  if (hd.n_probs != np ||
      memcmp(pay.data(), ctx->probs.data(), np * sizeof(qe_problem)) != 0)
    return fail(ctx, QE_EINVAL, "checkpoint holds other searches than this context");
  // check everything before changing anything
  const char *reps = pay.data() + np * sizeof(qe_problem);
  std::vector<size_t> off(np), toff(np, 0);
  size_t at = np * (sizeof(qe_problem) + sizeof(qe_report));
  for (uint32_t i = 0; i < np; ++i) {
    qe_report r;
    memcpy(&r, reps + i * sizeof(qe_report), sizeof r);
    if (r.generation != hd.gen)
      return fail(ctx, QE_EINVAL, "checkpoint record and generation counter disagree");
    size_t nb = 0;
    qe_state_bytes(ctx, i, &nb);
    uint64_t nb64 = 0;
    if (at + 8 > pay.size()) return fail(ctx, QE_EINVAL, "checkpoint is truncated or corrupted");
    memcpy(&nb64, pay.data() + at, 8);
    if (nb64 != nb || at + 8 + nb > pay.size())
      return fail(ctx, QE_EINVAL, "checkpoint state has the wrong size");
    off[i] = at + 8;
    const DevProblem &d = ctx->hp[i];
    if (d.enc == QE_ENC_GA) {
      const uint8_t *g = (const uint8_t *)pay.data() + off[i];
      for (size_t e = 0; e < (size_t)d.P * d.L; ++e)
        if (g[e] >= d.G) return fail(ctx, QE_EINVAL, "checkpoint genome holds an invalid gene");
    }
    at += 8 + nb;
    uint64_t tb = 0;
    if (at + 8 > pay.size()) return fail(ctx, QE_EINVAL, "checkpoint is truncated or corrupted");
    memcpy(&tb, pay.data() + at, 8);
    const uint64_t want = (uint64_t)d.N * d.N * 16;
    if ((tb != 0 && tb != want) || at + 8 + tb > pay.size())
      return fail(ctx, QE_EINVAL, "checkpoint target has the wrong size");
    if (tb) {
      std::vector<double> T(tb / 8);
      memcpy(T.data(), pay.data() + at + 8, tb);
      if (d.fit_kind != QE_FIT_TRACE || !target_ok(T.data(), d.N))
        return fail(ctx, QE_EINVAL, "checkpoint target is not a unitary for the trace fitness");
      toff[i] = at + 8;
    }
    at += 8 + tb;
  }
  if (at != pay.size()) return fail(ctx, QE_EINVAL, "checkpoint is truncated or corrupted");
  // the loaded generation is ranked already: the next generation graph skips
  // the pipelined ranking of generation gen - 1
  cudaStream_t us = ctx->user;
  ctx->gen = hd.gen;
  ctx->pending_rank = ctx->has_last = false;
  for (uint32_t i = 0; i < np; ++i) {
    qe_report r;
    memcpy(&r, reps + i * sizeof(qe_report), sizeof r);
    best_of(r, ctx->h_recs[i]);
    size_t nb = 0;
    qe_state_bytes(ctx, i, &nb);
    if ((st = state_copy(ctx, i, pay.data() + off[i], nb, false)) != QE_OK) return st;
    std::vector<double> T;
    if (toff[i]) {
      T.resize((size_t)2 * ctx->hp[i].N * ctx->hp[i].N);
      memcpy(T.data(), pay.data() + toff[i], T.size() * 8);
    }
    if ((st = put_target(ctx, i, toff[i] ? T.data() : nullptr)) != QE_OK) return st;
    const DevProblem &d = ctx->hp[i];
    if (d.mut_cnt) QE_CUDA(ctx, cudaMemsetAsync(d.mut_cnt, 0, 2 * 4, us));
  }
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->d_recs, ctx->h_recs, np * sizeof(Best), cudaMemcpyHostToDevice,
                               us));
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->g.gen, &hd.gen, 4, cudaMemcpyHostToDevice, us));
  QE_CUDA(ctx, cudaMemcpyAsync(ctx->g.ranked, &hd.gen, 4, cudaMemcpyHostToDevice, us));
  QE_CUDA(ctx, cudaMemsetAsync(ctx->g.rescore_n, 0, 4, us));
  QE_CUDA(ctx, cudaMemsetAsync(ctx->g.rank_active, 0, 4, us));
  QE_CUDA(ctx, cudaStreamSynchronize(us));
  return QE_OK;
}

qe_status qe_checkpoint_info(const char *path, qe_problem *h_probs, uint32_t capacity,
                             uint32_t *n_probs, uint32_t *gen) {
  CkptHeader hd;
  std::vector<char> pay;
  qe_status st = read_ckpt(nullptr, path, hd, pay);
  if (st != QE_OK) return st;
  if (n_probs) *n_probs = hd.n_probs;
  if (gen) *gen = hd.gen;
  if (h_probs && capacity >= hd.n_probs)
    memcpy(h_probs, pay.data(), hd.n_probs * sizeof(qe_problem));
  return QE_OK;
}

}  // extern "C"
