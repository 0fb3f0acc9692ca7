// qe_host.h -- internal launch interface between the C ABI (capi.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qe_dev.cuh"

namespace qe {

struct LaunchCfg {
  uint32_t num_sms = 1;
  // resident 256-thread blocks per SM of the circuit kernels, by qubit count
  uint32_t step32[6] = {1, 1, 1, 1, 1, 1};
  uint32_t step64[6] = {1, 1, 1, 1, 1, 1};
  // generation circuit kernels: 0 = resident blocks, 1 = one block less per SM
  // (room for a concurrent ranking chain), 2 = one warp per circuit, one wave
  uint32_t grid_mode = 0;
};

// persistent grid: at most the resident blocks of the whole GPU, fewer if
// there are fewer warps of work (wpb warps per block)
inline uint32_t grid_for(const LaunchCfg &lc, uint64_t warps, uint32_t per_sm, uint32_t wpb = 8) {
  uint64_t need = (warps + wpb - 1) / wpb;
  uint64_t cap = (uint64_t)lc.num_sms * per_sm;
  if (need > cap) need = cap;
  return need ? (uint32_t)need : 1u;
}

// one ranking job: search `prob` over n circuits whose working-precision
// fitness is at fit (float or double by the search's precision) and whose
// cost|work words are at meta; gates at gsrc (rescoring); update_record says
// whether the best-so-far record and report fields are written.
// pipelined: the buffers are the search's double-buffered generation buffers
// and the job ranks generation *gen - 1 (buffer (gen-1) & 1); the chain is
// skipped when that generation is already ranked (or gen == 0).
// one search's caller circuits in a batched evaluation launch: circuits
// [first, first + n) of the launch are this job's, gate strings at gates,
// fitness (float or double by the launch's precision) and costs out
struct EvalJob {
  uint32_t prob;   // descriptor index
  uint32_t first;  // circuits of the launch before this job's
  uint32_t n;
  uint32_t pad;
  const uint8_t *gates;
  void *fit;
  uint32_t *cost;
};

struct RankJob {
  uint32_t prob;
  uint32_t n;
  const void *fit;
  const uint32_t *meta;
  const uint8_t *gsrc;
  const float2 *asrc;  // Ising: the circuits' slot angles (NULL otherwise)
  uint32_t update_record;
  uint32_t pipelined;
};

// k_circuit.cu
cudaError_t query_circuit_occupancy(LaunchCfg &lc);
bool is_circuit_kernel(const void *f);  // a generation circuit kernel (graph node priorities)
bool is_rescore_kernel(const void *f);  // binary64 rescoring (waits for its predecessor)
bool is_eval_jobs_kernel(const void *f);  // the batch evaluation (waits for its predecessor)
// all searches of a launch have n qubits
cudaError_t launch_step(const LaunchCfg &lc, uint32_t n, const DevProblem *probs,
                        const uint32_t *group, const uint32_t *prefix, uint32_t n_group,
                        uint32_t total, bool canon, bool ising, bool ext, const DevGlobal &g,
                        cudaStream_t st);
cudaError_t launch_presample(const LaunchCfg &lc, const DevProblem *probs, const uint32_t *ids,
                             const unsigned long long *prefix, uint32_t n_ids,
                             unsigned long long total, const DevGlobal &g, cudaStream_t st);
cudaError_t launch_sample(const LaunchCfg &lc, const DevProblem *probs, uint32_t prob, uint32_t P,
                          uint32_t L, uint32_t gen, uint8_t *gate_idx, uint32_t *seg_id,
                          cudaStream_t st);
// amps: the slots' angles as qubit amplitudes (Ising searches), else NULL
cudaError_t launch_eval(const LaunchCfg &lc, uint32_t nq, const DevProblem *probs, uint32_t prob,
                        bool canon, const uint8_t *gates, const float2 *amps, uint32_t n,
                        void *fit, uint32_t *cost, void *S, const DevGlobal &g,
                        cudaStream_t st);
// the batched evaluation: n_jobs jobs of width nq (ascending first), total
// circuits, one launch
cudaError_t launch_eval_jobs(const LaunchCfg &lc, uint32_t nq, bool canon,
                             const DevProblem *probs, const EvalJob *jobs, uint32_t n_jobs,
                             uint32_t total, const DevGlobal &g, cudaStream_t st);
// gsrc == NULL: each candidate's search's own generation buffer; pipelined:
// that buffer is the one of generation *gen - 1, and nothing runs unless the
// chain is active.  gtab != NULL (device array indexed by problem): each
// candidate's gates come from gtab[its problem] instead.
// expect != 0: the grid is sized for that many candidates (at most the
// resident grid); 0: the resident grid
cudaError_t launch_rescore(const LaunchCfg &lc, uint32_t nq, bool ising, const DevProblem *probs,
                           const uint8_t *gsrc, const float2 *asrc, bool pipelined,
                           const DevGlobal &g, cudaStream_t st,
                           const uint8_t *const *gtab = nullptr, uint32_t expect = 0);

// k_update.cu
bool is_update_kernel(const void *f);  // an update kernel (graph node priorities)
cudaError_t launch_init_state(const DevProblem *probs, uint32_t prob, uint64_t nseg,
                              cudaStream_t st);
cudaError_t launch_scatter(const DevProblem *probs, uint32_t prob, uint32_t P, uint32_t L,
                           const uint32_t *seg_id, const double *fitness, uint32_t *err,
                           cudaStream_t st);
// elitism + mutation for the searches group[0..n_group); prefA: P*L prefix,
// prefB: ceil(P/32) prefix; gen read from *d_gen when d_gen != NULL
// role A (elitism) on stA, role B (mutation) on stB; the two may run concurrently
cudaError_t launch_update(const LaunchCfg &lc, const DevProblem *probs, const uint32_t *group,
                          const uint32_t *prefA, const uint32_t *prefB, uint32_t n_group,
                          uint32_t totalA, uint32_t totalB, const uint32_t *d_gen, uint32_t gen,
                          const uint32_t *seg_override, const DevGlobal &g, cudaStream_t stA,
                          cudaStream_t stB);

// k_rank.cu
cudaError_t rank_init();  // once per device before the first ranking launch
// jobs == NULL: one job given by value in `single`
bool is_select_kernel(const void *f);  // the ranking's selection kernel (graph edges)
// kernels that wait for their predecessor in the batch graph only (the
// one-CTA selection, the copy out)
bool batch_kernel_waits(const void *f);
// threads of a selection launch over n_jobs searches of at most max_n
// circuits, in units of 512 (a quarter of an SM's 2048)
uint32_t select_quarters(uint32_t n_jobs, uint32_t max_n);
bool rank_kernel_waits(const void *f);  // sort, top-k gather, finish: wait for their predecessor
// max_n: the most circuits of any job (picks one CTA or a cluster per search)
cudaError_t launch_rank_select(const DevProblem *probs, const RankJob *jobs, uint32_t n_jobs,
                               const RankJob &single, const DevGlobal &g, cudaStream_t st,
                               uint32_t max_n);
// err_out != NULL: also write the error word there and clear the rescoring queue
cudaError_t launch_rank_sort(const DevProblem *probs, const RankJob *jobs, uint32_t n_jobs,
                             const RankJob &single, const DevGlobal &g, cudaStream_t st,
                             Ranked *err_out = nullptr);
cudaError_t launch_finish(const DevGlobal &g, cudaStream_t st);
// the top-k lists of n_jobs ranked jobs back to back (job m's from out[koff[m]],
// koff has n_jobs + 1 entries), then the device error word in the entry
// out[koff[n_jobs]]
cudaError_t launch_gather_topk(const DevProblem *probs, const RankJob *jobs, const uint32_t *koff,
                               uint32_t n_jobs, Ranked *out, const DevGlobal &g, cudaStream_t st);

// GA (k_ga.cu): initial genome of one search into gate_idx buffer 0; per
// generation the SUS prefix sums and elite of the searches in ids, then the
// next genome (one warp per pair of children; prefix = pair-count prefix sums)
cudaError_t launch_ga_init(const DevProblem *probs, uint32_t prob, uint32_t P, uint32_t L,
                           const DevGlobal &g, cudaStream_t st);
// tprefix: the searches' prefix sums of ceil(P / 1024) scan tiles, n_tiles their total
cudaError_t launch_ga_prep(const DevProblem *probs, const uint32_t *ids, const uint32_t *tprefix,
                           uint32_t n_ga, uint32_t n_tiles, const DevGlobal &g, cudaStream_t st);
cudaError_t launch_ga_next(const LaunchCfg &lc, const DevProblem *probs, const uint32_t *ids,
                           const uint32_t *prefix, uint32_t n_ga, uint32_t total_pairs,
                           const DevGlobal &g, cudaStream_t st);
cudaError_t launch_reset_counter(const DevGlobal &g, cudaStream_t st);
// the batched host call's copies through the device mappings of page-locked
// host memory: n bytes in; the fitness and lists out, then the error word
// (written last, after a system fence, by the last block; count: a zeroed
// device word the kernel leaves zero)
cudaError_t launch_copy_in(void *dst, const void *src, size_t n, uint32_t num_sms,
                           cudaStream_t st);
cudaError_t launch_copy_out(void *h_fit, const void *d_fit, size_t fit_n, void *h_list,
                            const void *d_list, size_t list_n, uint32_t *h_errw,
                            const uint32_t *d_errw, uint32_t *count, uint32_t num_sms,
                            cudaStream_t st);

}  // namespace qe
