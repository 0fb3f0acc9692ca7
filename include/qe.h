/*
 * qe.h -- C ABI of the GB300-native batched fitness engine for the Quantum
 * Encoded Quantum Evolutionary Algorithm (QEQEA) of Krylov & Lukac,
 * arXiv:1809.11134, and of the classical GA that shares its evaluation.
 *
 * One search ("problem") evolves circuits of circuit_len gates on n_qubits
 * wires toward a permutation target.  Every generation the engine
 *   1. measures the qubit/qutrit encoding into population circuits
 *      (Sec. IV-D, segment index of Eq. (10)),
 *   2. composes each circuit's 2^n x 2^n unitary (Sec. IV-C) and scores it with
 *      Eq. (11) (minus an optional gate-cost penalty),
 *   3. ranks the circuits, rescoring the best ones in binary64,
 *   4. applies segment fitness, elitism and adaptive mutation (Sec. IV-E1, IV-F,
 *      Eq. (12)).
 * All four steps run as sm_103a CUDA kernels on one GPU; there is no CPU
 * fallback.  Many independent searches of uneven shape share every launch.
 *
 * Conventions used throughout:
 *   - wire w is bit (n-1-w) of a basis index (wire 0 = most significant bit);
 *   - S = G_{L-1} ... G_1 G_0 (slot 0 acts first);
 *   - gate library order: [I if QE_LIB_IDENTITY]; if QE_LIB_NCV, for control
 *     c = 0..n-1, for target t = 0..n-1, t != c: CNOT, CV, CV^dag on (c -> t);
 *     if QE_LIB_HT, for wire w = 0..n-1: H, T, T^dag.  V = (1/2)[[1+i,1-i],[1-i,1+i]];
 *   - regions (Sec. IV-B): one per ordered wire pair (its qutrit picks
 *     CNOT/CV/CV^dag), then one per wire (its qutrit picks H/T/T^dag); with
 *     QE_LIB_IDENTITY every segment's qubit decides "gate present" vs I;
 *   - segment index (Eq. (10)): seg = region*L*P + individual*L + slot.
 *
 * Memory: d_* arguments are caller-owned DEVICE pointers, h_* arguments are
 * caller-owned HOST pointers; the library never frees either.  All search
 * state is library-owned device memory, allocated once in qe_init.
 * Streams: every call is ordered on the stream passed to qe_init; calls that
 * return host data (qe_step, qe_eval/qe_eval_host with h_topk, qe_get_state,
 * qe_last_generation) synchronise that stream.
 * Errors: every call returns a qe_status and never aborts, traps or prints.
 * QE_EINVAL leaves all state unchanged.  After QE_ECUDA or QE_ETIMEOUT the
 * context is poisoned and every call except qe_last_error / qe_destroy
 * returns QE_ESTATE.  qe_last_error gives the context's last message.
 * Thread safety: a context may be used by one host thread at a time.
 */
#ifndef QE_H
#define QE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qe_ctx qe_ctx;

typedef enum {
  QE_OK = 0,
  QE_EINVAL = 1,       /* invalid argument; nothing changed */
  QE_ENOMEM = 2,       /* device memory exhausted (qe_init) */
  QE_ECUDA = 3,        /* a CUDA call failed; context poisoned */
  QE_ETIMEOUT = 4,     /* a bounded device wait expired; context poisoned */
  QE_ENUMERIC = 5,     /* device saw an invalid gate index or a non-finite fitness */
  QE_ESTATE = 6,       /* context poisoned, or call invalid for this problem */
  QE_EUNSUPPORTED = 7, /* valid request not implemented by this build / device */
  QE_EIO = 8           /* a checkpoint file could not be opened, read or written */
} qe_status;

/* gate library bits */
#define QE_LIB_NCV 1u
#define QE_LIB_HT 2u
#define QE_LIB_IDENTITY 4u
/* The paper's own library (Sec. III Eqs. (3)-(5), Sec. IV-A), used alone:
 * regions = the n wires (the qutrit picks the rotation axis x/y/z on that
 * wire), then the n(n-1)/2 wire pairs i < j in lexicographic order (an
 * interaction template J_ij).  Library index 3w + k is R_{x,y,z} on wire w,
 * 3n + q is J on pair q: G = 3n + n(n-1)/2.  A slot's angle theta is the angle
 * of the sampled segment's qubit amplitudes (b0, b1) = (cos theta,
 * sin theta), theta in [0, 2 pi) (the qubit is not measured), and the gates
 * use cos(theta/2) = sgn(b1) sqrt((1 + b0)/2), sin(theta/2) = sqrt((1 - b0)/2)
 * (sgn(b1) = -1 iff b1 < 0); J(theta) = exp(-i theta/2 Z_i Z_j).  The qubit
 * mutation turns theta by +-(1 - f) mutationRange (Sec. IV-F).  Under
 * QE_ENC_GA the genes are (gate, angle) pairs bred as the paper's comparator
 * (Sec. V-B): see qe_step.  Circuits given by the caller carry their angles as
 * such amplitude pairs (qe_eval_amp, qe_compose_amp). */
#define QE_LIB_ISING 8u

/* arithmetic of the composition */
#define QE_PREC_FP64 0u     /* binary64, fixed operation order: bit-identical to the oracle */
#define QE_PREC_FP32 1u     /* binary32 in registers, binary64 rescoring of the top-k */
/* hi/lo split products on tensor cores: reserved, QE_EUNSUPPORTED.  A gate
 * here updates O(N^2) amplitudes in registers; as a dense product on tensor
 * cores it would be O(N^3) work with three split products per gate, whose
 * ceiling at full tensor throughput is at or below the register form's
 * measured rate, with a larger rounding error. */
#define QE_PREC_SPLIT_TC 2u

/* fitness kind (Sec. IV-E) */
#define QE_FIT_TRACE 0u /* Eq. (11): 1 - sqrt((N - |tr(S^dag T)|)/N) */
#define QE_FIT_PROB 1u  /* 1 - sqrt((N - sum_j |S_{perm[j] j}|^2)/N): Table 2 -> Table 3 reading */

/* encoding */
#define QE_ENC_QEQEA 0u /* qubit/qutrit encoding, Sec. IV */
#define QE_ENC_GA 1u    /* classical GA on integer gate strings (Sec. V-B comparison) */

#define QE_MAX_QUBITS 5u
#define QE_MAX_SHOTS 64u
#define QE_MAX_LEN 64u
#define QE_MAX_POP (1u << 20)
#define QE_MAX_TOPK 1024u
#define QE_MAX_PROBLEMS 4096u

/* device error word bits (qe_report.error_word) */
#define QE_ERRW_BAD_GATE 1u    /* a gate index >= the library size was evaluated */
#define QE_ERRW_NONFINITE 2u   /* a fitness value was NaN or infinite */
/* a binary32 search's rescored binary64 fitness lay outside the interval that
 * its binary32 fitness and the bound eps_d = 8e-7 L + 2e-6 on the error of
 * d = (N - |tr|)/N imply, so the top-k may be inexact; every rescored
 * candidate is checked */
#define QE_ERRW_GUARD_BAND 4u

/* calls of qe_eval_host_batch_async that can be in flight at once */
#define QE_BATCH_SLOTS 16u

/* One search.  sizeOfIndividual = circuit_len, sizeOfPopulation = population,
 * numberOfWires = n_qubits (Sec. IV-B). */
typedef struct {
  uint32_t n_qubits;      /* 1..5 */
  uint32_t circuit_len;   /* L: 1..64 */
  uint32_t population;    /* P: 1..2^20; regions*L*P must be < 2^32 */
  uint32_t library;       /* QE_LIB_* bits; at least one region must exist */
  uint32_t encoding;      /* QE_ENC_* */
  uint32_t precision;     /* QE_PREC_* */
  uint32_t fitness_kind;  /* QE_FIT_* */
  uint32_t topk;          /* circuits rescored in binary64 and ranked per generation; 0..min(P,1024) */
  uint64_t seed;          /* Philox4x32-10 key (low word, high word) */
  double p_mutation;      /* probabilityOfMutation per individual per generation, [0,1] */
  double mutation_range;  /* mutationRange in radians, finite, >= 0 */
  double ga_mutation_rate;/* GA: per-gene replacement probability, [0,1] */
  double cost_weight;     /* lambda: F = f - lambda * cost / L; cost = non-identity gates */
  uint8_t target_perm[32];/* T|j> = |target_perm[j]>, a permutation of 0..2^n-1 */
  uint32_t shots;         /* K: measurements of a slot's qutrit, 0..QE_MAX_SHOTS; K > 1 keeps
                             the most frequent outcome, the lowest on a tie (Sec. IV-A1:
                             the qutrit is measured repeatedly to approximate its state);
                             0 and 1 measure once.  QEQEA only (the GA ignores it).  Shot j
                             compares word j mod 4 of Philox (c, t + 64 floor(j/4), gen,
                             run << 4 | 3) with the outcome CDF in binary32. */
  uint32_t reserved;      /* 0 */
} qe_problem;

/* one ranked circuit: index in the population, gate cost, binary64 fitness */
typedef struct {
  uint32_t circuit;
  uint32_t cost;
  double fitness;
} qe_ranked;

/* per-search report after qe_step */
typedef struct {
  uint32_t generation;      /* generations completed */
  uint32_t best_gen;        /* generation in which best_fitness was found */
  double best_fitness;      /* best binary64 F seen so far */
  double gen_best_fitness;  /* best binary64 F of the last generation */
  double mean_fitness;      /* mean F (working precision) of the last generation */
  uint64_t useful_flops;    /* real operations of the last generation's compositions */
  uint32_t best_cost;
  uint32_t best_len;
  uint32_t error_word;      /* QE_ERRW_* bits seen so far */
  uint32_t reserved;
  uint8_t best_gates[64];   /* gate indices of the best circuit, best_len of them */
  float best_amps[128];     /* Ising: its slots' angles as qubit amplitudes (b0, b1) per
                               slot; zero for the other libraries */
} qe_report;

/* Library geometry without a context: number of gate types and of regions
 * (Sec. IV-B) for n_qubits and library bits.  QE_EINVAL on bad arguments. */
qe_status qe_library_info(uint32_t n_qubits, uint32_t library, uint32_t *n_gates,
                          uint32_t *n_regions);

/* Create a context holding n_probs independent searches on the current CUDA
 * device; cuda_stream (a cudaStream_t, NULL = legacy default stream) orders
 * every later call.  Validates every problem before touching the GPU
 * (QE_EINVAL), allocates all state in one device arena (QE_ENOMEM when
 * cudaMemGetInfo says it cannot fit), initialises the encoding to uniform
 * amplitudes (qutrit 1/sqrt(3) each, qubit 1/sqrt(2) each, best fitness -1)
 * and sets the generation counter to 0.  *out is set only on QE_OK. */
qe_status qe_init(qe_ctx **out, const qe_problem *probs, uint32_t n_probs, void *cuda_stream);

/* Circuit construction by measurement (Sec. IV-D, Eq. (10)) for search prob at
 * generation gen: writes d_gate_idx[c*L + t] (uint8 library index) and
 * d_seg_id[c*L + t] (uint32 segment index) for c < P, t < L.  A pure function
 * of (encoding state, seed, gen, prob).  QEQEA searches only. */
qe_status qe_sample(qe_ctx *ctx, uint32_t prob, uint32_t gen, uint8_t *d_gate_idx,
                    uint32_t *d_seg_id);

/* Fitness of n_circuits circuits d_gate_idx[c*L + t] of search prob
 * (Sec. IV-C composition, Eq. (11) score, minus lambda*cost/L).  d_fitness is
 * float[n] for QE_PREC_FP32/SPLIT_TC and double[n] for QE_PREC_FP64; d_cost
 * (uint32[n], may be NULL) receives the gate costs.  If h_topk is not NULL the
 * best min(topk, n) circuits (topk from the problem, at least 1) are rescored
 * in binary64 and written to h_topk sorted by (fitness desc, cost asc, index
 * asc); this needs n_circuits <= P and synchronises.  Invalid gate indices
 * give NaN fitness and QE_ENUMERIC (when h_topk is given) or the error bit. */
qe_status qe_eval(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, uint32_t n_circuits,
                  void *d_fitness, uint32_t *d_cost, qe_ranked *h_topk);

/* Ranking of given fitness values (the selection and binary64 rescoring of
 * the top-k; Sec. IV-E ranks circuits by Eq. (11)): n_circuits circuits
 * d_gate_idx[c*L + t] of search prob with their working-precision fitness
 * d_fitness (float[n] for binary32 searches, double[n] for binary64) and gate
 * costs d_cost (uint32[n], as qe_eval writes them), e.g. evaluated on several
 * devices and gathered; d_amps: the Ising library's slot angles (float2 per
 * slot, as qe_eval_amp), NULL otherwise.  The best min(topk, n) circuits
 * (topk at least 1) are rescored in binary64 from their gates and written to
 * h_topk sorted by (fitness desc, cost asc, index asc).  A binary32 search
 * keeps every circuit whose binary64 fitness can reach the k-th best given
 * the bound on its binary32 error, and checks every rescored candidate
 * against that bound: a candidate outside it (a fitness that is not the
 * binary32 value of its circuit, or a composition error above the bound)
 * makes the call return QE_ENUMERIC (error word bit QE_ERRW_GUARD_BAND; the
 * message says so), as do invalid gates and non-finite fitness.
 * n_circuits <= P; synchronises; a pending generation's ranking is finished
 * first. */
qe_status qe_rank(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, const float *d_amps,
                  const void *d_fitness, const uint32_t *d_cost, uint32_t n_circuits,
                  qe_ranked *h_topk);

/* qe_eval on HOST buffers: copies h_gate_idx to the device, evaluates, copies
 * the fitness (float or double by precision) back to h_fitness and fills
 * h_topk if not NULL.  n_circuits <= P.  Synchronises.  Pinned host memory
 * makes the copies asynchronous with respect to other host work. */
qe_status qe_eval_host(qe_ctx *ctx, uint32_t prob, const uint8_t *h_gate_idx,
                       uint32_t n_circuits, void *h_fitness, qe_ranked *h_topk);

/* qe_eval_host for several searches in one call (Sec. IV-C composition,
 * Eq. (11) score minus lambda*cost/L, as qe_eval).  Item m evaluates
 * h_n_circuits[m] (<= P of that search) circuits of search h_probs[m]; the
 * items' problems are distinct and either all binary64 or all binary32
 * searches (QE_EINVAL otherwise), and none uses QE_LIB_ISING.  Host buffers,
 * items back to back in item order:
 *   h_gate_idx  uint8, item m's n_m * L_m gate indices (row-major c*L + t);
 *   h_fitness   float (binary32 searches) or double (binary64), n_m per item;
 *   h_topk      NULL, or k_m = min(max(topk_m, 1), n_m) entries per item: its
 *               best circuits rescored in binary64 and sorted by (fitness
 *               desc, cost asc, index asc), circuit indices local to the item.
 * One host->device copy, one graph launch (the evaluations on three streams,
 * then one ranking of every item) and the device->host copies, then one
 * synchronisation.  The graph is captured on the first call with a given item
 * layout (problems, counts, ranking or not) and replayed while the layout
 * repeats; the first call, and any call needing more staging than before,
 * allocates device staging (and pinned host staging for the top-k lists) that
 * the context keeps until qe_destroy.  Pinned host buffers make the copies
 * asynchronous with respect to other host work.  Invalid gate indices give
 * NaN fitness and QE_ENUMERIC (the fitness is still written).  The call runs
 * on a stream and scratch memory of its own (not ordered after other work on
 * the context's stream, and touching no state of the context's searches: it
 * can run beside qe_step).  qe_set_target waits for batch calls in flight
 * before it changes a target, and later calls use the new one.  Equivalent to
 * qe_eval_host_batch_async followed by qe_eval_host_batch_wait; QE_ESTATE if
 * every slot has a call in flight. */
qe_status qe_eval_host_batch(qe_ctx *ctx, uint32_t n_items, const uint32_t *h_probs,
                             const uint32_t *h_n_circuits, const uint8_t *h_gate_idx,
                             void *h_fitness, qe_ranked *h_topk);

/* qe_eval_host_batch without the synchronisation: enqueues the call and
 * returns a ticket (*ticket, nonzero) for qe_eval_host_batch_wait.  The
 * context has QE_BATCH_SLOTS staging slots, each with its own stream, device
 * scratch (candidates, rescoring queue, error word) and graphs, so that many
 * calls can be in flight and run concurrently: copies, evaluations and
 * rankings of different calls overlap.  Until its wait returns, a call still
 * reads h_gate_idx and writes h_fitness and h_topk: the caller keeps them
 * alive and untouched, and gives calls in flight distinct buffers.  h_probs
 * and h_n_circuits are read before return.  Arguments are checked as by
 * qe_eval_host_batch; QE_ESTATE when every slot has a call in flight,
 * QE_EINVAL for a NULL ticket.  Each slot's graphs follow the layout of its
 * last call, so repeating fixed layouts replays captured graphs.  When
 * h_gate_idx and h_fitness are page-locked (cudaHostAlloc, cudaHostRegister;
 * checked on every call) kernels of the slot's graph copy them through their
 * device mappings and a call is one graph launch; such a graph is replayed
 * only for the same mappings, and a call goes to a free slot whose graph
 * matches it when there is one.  Other host memory is copied by separate
 * asynchronous copies around the graph. */
qe_status qe_eval_host_batch_async(qe_ctx *ctx, uint32_t n_items, const uint32_t *h_probs,
                                   const uint32_t *h_n_circuits, const uint8_t *h_gate_idx,
                                   void *h_fitness, qe_ranked *h_topk, uint64_t *ticket);

/* Waits for the call with this ticket (for page-locked buffers by polling
 * the call's staged error word for up to 2 ms, then by blocking on its
 * slot's stream), fills its h_topk and frees its slot;
 * QE_ENUMERIC as qe_eval_host_batch; QE_EINVAL for a ticket that is not in
 * flight (never issued, or already waited for).  Calls may be waited for in
 * any order. */
qe_status qe_eval_host_batch_wait(qe_ctx *ctx, uint64_t ticket);

/* The composed unitaries themselves: d_unitary receives n_circuits row-major
 * N x N complex matrices, (re, im) interleaved, float for QE_PREC_FP32 and
 * SPLIT_TC, double for QE_PREC_FP64 (same arithmetic as qe_eval). */
qe_status qe_compose(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, uint32_t n_circuits,
                     void *d_unitary);

/* qe_eval / qe_compose for the Ising library: d_amps[2*(c*L + t) + {0,1}] are
 * the qubit amplitudes (b0, b1) = (cos theta, sin theta) that give slot t of
 * circuit c its angle (see QE_LIB_ISING); float, caller-owned DEVICE memory.
 * For the other libraries d_amps is ignored.  qe_eval, qe_eval_host and
 * qe_compose return QE_EINVAL for an Ising search. */
qe_status qe_eval_amp(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx, const float *d_amps,
                      uint32_t n_circuits, void *d_fitness, uint32_t *d_cost, qe_ranked *h_topk);
qe_status qe_compose_amp(qe_ctx *ctx, uint32_t prob, const uint8_t *d_gate_idx,
                         const float *d_amps, uint32_t n_circuits, void *d_unitary);

/* Segment fitness, elitism and adaptive mutation (Sec. IV-E1, IV-F) of search
 * prob at generation gen, given the d_seg_id[P*L] of that generation's
 * circuits and their d_fitness[P] (double).  A pure function of (state, seed,
 * gen, seg_id, fitness).  QEQEA searches only. */
qe_status qe_update(qe_ctx *ctx, uint32_t prob, uint32_t gen, const uint32_t *d_seg_id,
                    const double *d_fitness);

/* Run n_gen whole generations of every search (sample -> compose/score ->
 * rank with binary64 rescoring -> update, or the GA's eval -> rank -> select /
 * cross / mutate), replayed as one CUDA graph per generation.  GA breeding
 * (Sec. V-B comparison): stochastic universal sampling on the weights
 * floor(clamp(F, 0, 1) 2^32) of the working-precision fitness, one-point
 * crossover of children (2m, 2m+1), per-gene replacement with probability
 * ga_mutation_rate, and child 0 = the best circuit by (working-precision F
 * desc, cost asc, index asc).  With h_reports
 * (n_probs entries) the call then copies one qe_report per search, synchronises
 * and returns QE_ENUMERIC if any search's error_word is set; with h_reports ==
 * NULL it only enqueues the generations on the stream and returns. */
qe_status qe_step(qe_ctx *ctx, uint32_t n_gen, qe_report *h_reports);

/* FMA throughput of the current GPU in binary32 and binary64 (TFLOP/s, an FMA
 * counted as two flops), measured with independent FMA chains on every SM.
 * Not part of the method: the denominators of the arithmetic rooflines of the
 * circuit and rescoring kernels.  Allocates and frees a small device buffer;
 * synchronises. */
qe_status qe_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops);

/* Launch-plan autotuner.  A generation graph can be launched in several ways
 * that give bit-identical results: with or without a launch-completion edge
 * that lets the previous generation's ranking selection start before the
 * circuit kernels fill the GPU, and with the circuit kernels' persistent grid
 * at the resident block count, one block per SM less (room for the ranking
 * chain), or one warp per circuit in a single wave, and, when searches of
 * several qubit counts share the context, with their circuit kernels one after
 * the other or on parallel streams.  qe_autotune runs 1 + gens_per_plan
 * (1..64) generations of every search with each plan (up to twelve), times the
 * last gens_per_plan on the stream with CUDA events, and keeps the fastest for
 * every later qe_step.  These are real generations: they
 * advance the searches exactly as qe_step would (qe_generation counts them).
 * With n_plans != NULL, h_ms receives up to *n_plans mean generation times (ms,
 * in plan order: sequential widths, then parallel; within each, with the edge,
 * then without; grids in the order above) and *n_plans the number of plans
 * tried.  Synchronises.  QE_ESTATE while stage
 * timing is on. */
qe_status qe_autotune(qe_ctx *ctx, uint32_t gens_per_plan, float *h_ms, uint32_t *n_plans);
/* The launch plan in use, as text (NUL-terminated, truncated to len). */
qe_status qe_launch_plan(const qe_ctx *ctx, char *h_buf, size_t len);

/* Stage timing.  qe_stage_timing(ctx, 1) rebuilds the generation graph with
 * CUDA events recorded between its kernels (on the stream each kernel runs
 * on); qe_stage_times then gives, for the last generation run, ms[0] circuit
 * kernels (sample + compose + score + segment-fitness scatter), ms[1] ranking
 * selection, ms[2] binary64 rescoring, ms[3] ranking sort, ms[4] update
 * (elitism + mutation, concurrent with ms[1..3]), ms[5] the whole generation.
 * Under mode 1 ms[0] and ms[1] run from the start of the generation, so they
 * include waiting on the stages that run beside them.  qe_stage_timing(ctx, 2)
 * serialises the generation instead: every kernel on one stream in the order
 * circuits, update, ranking (no launch-completion edge), so each interval is
 * that stage's own duration with nothing running beside it (ms[1] then runs
 * from the end of the update); the results are the same as under mode 0.
 * 0 turns timing off; other values are QE_EINVAL.  qe_stage_times
 * synchronises.  Timing adds a few event records per generation. */
qe_status qe_stage_timing(qe_ctx *ctx, int enable);
qe_status qe_stage_times(qe_ctx *ctx, float *ms);

/* The last generation of search prob as run by qe_step: its circuits
 * h_gate_idx[P*L], segment ids h_seg_id[P*L] (QEQEA), working-precision
 * fitness widened to double h_fitness[P], and top-k h_topk[max(topk,1)].
 * Any pointer may be NULL.  Synchronises.  QE_ESTATE if no generation has run
 * since qe_init or qe_load (a checkpoint does not hold the last generation). */
qe_status qe_last_generation(qe_ctx *ctx, uint32_t prob, uint8_t *h_gate_idx, uint32_t *h_seg_id,
                             double *h_fitness, qe_ranked *h_topk);

/* Bytes of one search's encoding state in the qe_get_state layout:
 *   QEQEA: cur[S][8] float, best[S][8] float, best_f[S] float, S = R*P*L, with
 *          the 8 floats of a segment {q0.re, q0.im, q1.re, q1.im, q2.re, q2.im,
 *          b0, b1} (qutrit amplitudes, then qubit amplitudes);
 *   GA:    genome[P][L] uint8, the population the next qe_step generation
 *          evaluates (gene values below the library size; qe_set_state returns
 *          QE_EINVAL for any other value); on QE_LIB_ISING followed by
 *          angle[P][L][2] float, each gene's angle as the qubit amplitudes
 *          (cos t, sin t). */
qe_status qe_state_bytes(const qe_ctx *ctx, uint32_t prob, size_t *bytes);
/* Copy the state out to / in from host memory of exactly qe_state_bytes bytes.
 * Synchronises. */
qe_status qe_get_state(qe_ctx *ctx, uint32_t prob, void *h_buf, size_t bytes);
qe_status qe_set_state(qe_ctx *ctx, uint32_t prob, const void *h_buf, size_t bytes);

/* Dense target (Eq. (11) with a general unitary T instead of the permutation
 * target_perm).  h_target: host T[i][j] as (re, im) doubles at 2 (i N + j),
 * N = 2^n_qubits, copied; NULL restores the permutation.  The fitness is then
 * f = 1 - sqrt((N - |tr(S^dag T)|) / N) with tr(S^dag T) = sum_j (S^dag T)_jj,
 * (S^dag T)_jj = sum_i conj(S_ij) T_ij (binary64: i ascending within each j,
 * then j ascending).  QE_EUNSUPPORTED for QE_FIT_PROB searches (the
 * probability overlap is defined for permutations); QE_EINVAL unless every
 * entry is finite and T^dag T = I to 1e-6.  A pending generation is ranked
 * first against the old target; the best-so-far record is kept.  Applies to
 * qe_step, qe_eval and qe_eval_host.  Synchronises. */
qe_status qe_set_target(qe_ctx *ctx, uint32_t prob, const double *h_target);

/* Checkpoint / resume.  Every random draw is a Philox function of (seed,
 * generation, ...) (Sec. IV-D sampling, Sec. IV-F mutation, Sec. V-B GA), so a
 * run's whole state is each search's encoding state (the qe_get_state
 * layout), its best-so-far record and target, and the generation counter; a
 * context that
 * loads a checkpoint continues the saved run bit for bit.
 *
 * qe_save ranks a pending last generation, then writes the file at path (a
 * temporary beside it, renamed over it once complete): a 48-byte header
 * {"QECKPT1\0", version 1, n_probs, generation, sizeof(qe_problem),
 * sizeof(qe_report), 0, payload bytes, FNV-1a 64-bit hash of the payload},
 * then the payload {qe_problem[n_probs], qe_report[n_probs] (the records as
 * qe_step reports them), and per search a uint64 byte count and its
 * qe_get_state bytes, then a uint64 byte count (0, or 16 N^2) and its dense
 * target as qe_set_target takes it}, little-endian.  Synchronises.  QE_EIO if the file
 * cannot be written (the previous file, if any, is left in place).
 *
 * qe_load reads a checkpoint into a context created with the same problems
 * (byte-equal qe_problem arrays): encoding state, records, dense targets and
 * generation counter; the launch plan is kept.  It checks the whole file first (magic,
 * version, sizes, hash, problems, record generations, gene values) and
 * returns QE_EINVAL with nothing changed if any check fails, QE_EIO if the
 * file cannot be read.  Synchronises.
 *
 * qe_checkpoint_info reads and checks a checkpoint without a context or GPU:
 * *n_probs and *gen (either may be NULL), and the problems into h_probs when
 * capacity >= *n_probs (so qe_init can recreate the context). */
qe_status qe_save(qe_ctx *ctx, const char *path);
qe_status qe_load(qe_ctx *ctx, const char *path);
qe_status qe_checkpoint_info(const char *path, qe_problem *h_probs, uint32_t capacity,
                             uint32_t *n_probs, uint32_t *gen);

/* Generations completed by qe_step. */
qe_status qe_generation(const qe_ctx *ctx, uint32_t *gen);

/* Evaluation and ranking without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc -- code running
 * while a host framework's caching allocator owns the device memory, plugins
 * in a process whose memory budget is fixed up front, loops that must never
 * block in an allocator.  It needs no context: given one search description
 * (host struct; encoding, seed and mutation fields are ignored), n_circuits
 * gate strings d_gate_idx[c*L + t] on the device, it writes their fitness to
 * d_fitness (float, or double for QE_PREC_FP64; the same arithmetic as
 * qe_eval) and, if d_topk is not NULL, the best min(max(topk,1), n_circuits)
 * circuits rescored in binary64 and sorted by (fitness desc, cost asc, index
 * asc) to the DEVICE array d_topk.  Discrete libraries only (QE_LIB_ISING is
 * QE_EINVAL here).  All work is enqueued on cuda_stream; the
 * call does not synchronise.  Scratch comes from one static device array of
 * the library (about 1.25 MiB, held by every GPU that loads the library until
 * the process exits), so n_circuits is limited to 65536 (QE_EINVAL above it)
 * and calls that overlap on the GPU -- on different streams, or from
 * different threads -- race on that scratch.  The first call on a device
 * looks up the array's device address and launch shapes, so make that first
 * call before any stream capture; under lazy module loading (the CUDA default
 * since 12.2) it also loads the library's code for that device, and the
 * driver allocates the array then, so make the first call while allocation
 * is still allowed.  Calls after it call no cudaMalloc, cudaFree or other
 * allocating routine.  Errors are returned as a status with a message written
 * to h_msg (msg_len bytes, may be NULL); the first N entries of
 * prob->target_perm (held in the struct) must be a permutation of 0..N-1
 * (QE_EINVAL otherwise).  An invalid gate index gives that
 * circuit a NaN fitness and leaves d_topk unspecified (the call does not
 * synchronise, so it cannot report it): pass valid indices, or check
 * d_fitness.  QE_PREC_SPLIT_TC is QE_EUNSUPPORTED. */
qe_status qe_eval_rank_static(const qe_problem *prob, const uint8_t *d_gate_idx,
                              uint32_t n_circuits, void *d_fitness, qe_ranked *d_topk,
                              void *cuda_stream, char *h_msg, size_t msg_len);

/* Last error message of ctx ("" if none); static text when ctx is NULL. */
const char *qe_last_error(const qe_ctx *ctx);

/* Free all device and host memory of ctx (NULL is allowed). */
void qe_destroy(qe_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
