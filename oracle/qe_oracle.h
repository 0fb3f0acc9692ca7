/*
 * qe_oracle.h -- plain FP64 CPU oracle for the batched QEQEA fitness path
 * (Krylov & Lukac, "Quantum Encoded Quantum Evolutionary Algorithm for the
 * Design of Quantum Circuits", arXiv:1809.11134).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs may load this library. It shares no code,
 * header, table or constant generator with the CUDA library; the product path
 * never calls it.
 *
 * Every routine is a slow, literal restatement of the paper's steps:
 * gates are expanded to dense 2^n x 2^n matrices by Kronecker products
 * (Sec. IV-C, step 4), circuits are composed by dense complex matmul, and the
 * fitness is Eq. (11) written out.  All arithmetic is IEEE binary64 with no
 * FMA contraction (built with -ffp-contract=off).
 *
 * Conventions where the paper is silent (each is listed as a reading in the
 * design notes):
 *   - wire w is bit (n-1-w) of a basis index (wire 0 = most significant bit);
 *   - S = G_{L-1} ... G_1 G_0, slot 0 is applied first;
 *   - discrete library order: [I] then, for c, for t != c: CNOT, CV, CV^dag
 *     on (c -> t), then for each wire w: H, T, T^dag;
 *   - regions: one per ordered pair (qutrit picks CNOT/CV/CV^dag), then one per
 *     wire when H/T/T^dag are in the library (qutrit picks H/T/T^dag);
 *   - with the identity in the library every segment also carries a qubit
 *     whose outcome 1 means "gate present";
 *   - Ising library: regions = the n wires (the qutrit picks the axis x/y/z of
 *     a rotation on that wire, Sec. IV-A) then the n(n-1)/2 wire pairs i < j
 *     in lexicographic order (an interaction template); library index
 *     3w + k = R_{x,y,z}(theta) on wire w, then 3n + pair = J on that pair;
 *     the angle theta of a slot is the angle of the sampled segment's qubit
 *     amplitudes (b0, b1) = (cos theta, sin theta), theta in [0, 2 pi), and
 *     the gates take cos(theta/2) = sgn(b1) sqrt((1 + b0)/2),
 *     sin(theta/2) = sqrt((1 - b0)/2) (sgn(b1) = -1 iff b1 < 0), binary64;
 *     J(theta) = exp(-i theta/2 D) with D the +-1 template diagonal
 *     z_i z_j (z = +1 for bit 0, -1 for bit 1).
 *
 * Measurement and mutation arithmetic is binary32 (the state's precision),
 * each operation rounded in the written order; the decision "x < cdf" is thus
 * taken in the same precision on both sides.  Composition and fitness are
 * binary64.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (published Philox test vectors, Table 1 indices, Table 2/3 values,
 * textbook NCV identities, exact-arithmetic recomputation, brute force,
 * closed-form SU(3) special cases, chi-square sampling).  The GA operators
 * (SUS, one-point crossover, per-gene mutation) are pinned only by
 * invariants and brute-force counts on tiny inputs.
 */
#ifndef QE_ORACLE_H
#define QE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* library bits */
#define ORC_LIB_NCV 1u
#define ORC_LIB_HT 2u
#define ORC_LIB_IDENTITY 4u
#define ORC_LIB_ISING 8u /* the paper's own library (Sec. III, IV-A): alone, never mixed */

/* gate kinds */
#define ORC_I 0
#define ORC_CNOT 1
#define ORC_CV 2
#define ORC_CVDG 3
#define ORC_H 4
#define ORC_T 5
#define ORC_TDG 6
#define ORC_RX 7 /* Eq. (3) */
#define ORC_RY 8 /* Eq. (4) */
#define ORC_RZ 9 /* Eq. (5) */
#define ORC_J 10 /* interaction template J_ij (Sec. III, IV-A) */

/* fitness kinds */
#define ORC_FIT_TRACE 0 /* Eq. (11) as printed: |tr(S^dag T)| */
#define ORC_FIT_PROB 1  /* probability overlap sum_j |S_{pi(j) j}|^2 */

#define ORC_Q 4096 /* mutation magnitude quantisation */

typedef struct {
  uint32_t n;            /* qubits (numberOfWires), 1..5 */
  uint32_t L;            /* circuit length (sizeOfIndividual) */
  uint32_t P;            /* population (sizeOfPopulation) */
  uint32_t library;      /* ORC_LIB_* bits */
  uint32_t fitness_kind; /* ORC_FIT_* */
  uint32_t run;          /* index of this search; goes into Philox counter word 3 */
  uint64_t seed;         /* Philox key */
  double p_mutation;     /* probabilityOfMutation, per individual per generation */
  double mutation_range; /* mutationRange, radians */
  double cost_weight;    /* lambda: F = f - lambda * cost / L */
  uint8_t perm[32];      /* target: T|j> = |perm[j]> */
  uint32_t shots;        /* qutrit measurements per slot, majority taken (Sec. IV-A1); 0 or 1 = one */
  const double *target;  /* dense target unitary, T[i][j] = (re, im) at 2 (i N + j), read by the
                            trace fitness of Eq. (11); NULL = the permutation perm */
} oracle_problem;

/* ---- Philox4x32-10 (Salmon et al., SC'11) ---- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- library / population geometry (Sec. IV-B, Eqs. (7)-(10)) ---- */
uint32_t oracle_num_gates(uint32_t n, uint32_t library);
uint32_t oracle_num_regions(uint32_t n, uint32_t library);
/* kind/control/target of library index g; returns 0 on success, -1 if g is out of range */
int oracle_gate_desc(uint32_t n, uint32_t library, uint32_t g, int *kind, int *ctrl, int *tgt);
/* library index chosen when region r's qutrit is measured as k (and the qubit says present) */
uint32_t oracle_region_gate(uint32_t n, uint32_t library, uint32_t r, uint32_t k);
uint64_t oracle_segment_index(uint64_t r, uint64_t i, uint64_t t, uint64_t L, uint64_t P);
uint64_t oracle_num_segments(const oracle_problem *p);

/* ---- Ising angles: cos/sin of theta/2 from a slot's qubit amplitudes ---- */
void oracle_half_angle(float b0, float b1, double *c, double *s);

/* ---- gates, composition, score (Sec. III, IV-C, IV-E) ---- */
/* The *_amp forms take, for the Ising library, the sampled qubit amplitudes
   (b0, b1) of every slot (amps[2t], amps[2t+1]); the other libraries ignore
   them (amps may be NULL).  The forms without amps are the discrete-library
   calls (an Ising gate without an angle yields NaN). */
void oracle_gate_matrix_amp(uint32_t n, uint32_t library, uint32_t g, float b0, float b1,
                            double *re, double *im);
void oracle_compose_amp(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates,
                        const float *amps, double *S_re, double *S_im);
/* dense N x N complex matrix of library gate g, row-major, re/im planes */
void oracle_gate_matrix(uint32_t n, uint32_t library, uint32_t g, double *re, double *im);
/* S = G_{L-1} ... G_0 for one circuit */
void oracle_compose(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates, double *S_re,
                    double *S_im);
/* fitness of an N x N matrix against the permutation target */
/* Eq. (11) against a dense target T (interleaved as oracle_problem.target):
   |tr(S^dag T)| with the diagonal elements of S^dag T each summed over i
   ascending, then the trace over j ascending. */
double oracle_score_dense(uint32_t n, const double *S_re, const double *S_im, const double *T);
double oracle_score(uint32_t n, const double *S_re, const double *S_im, const uint8_t *perm,
                    uint32_t fitness_kind);
uint32_t oracle_cost(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates);
/* F[c] = f(S_c) - lambda*cost_c/L for n_circuits circuits gates[c*L + t] */
void oracle_eval(const oracle_problem *p, const uint8_t *gates, uint32_t n_circuits, double *F,
                 uint32_t *cost);
/* the same with each circuit's slot amplitudes at amps + c*2L */
void oracle_eval_amp(const oracle_problem *p, const uint8_t *gates, const float *amps,
                     uint32_t n_circuits, double *F, uint32_t *cost);
/* useful real ops of one circuit (gate-count model, see design notes) */
uint64_t oracle_useful_flops(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates);

/* ---- encoding state: 8 floats per segment {q0re,q0im,q1re,q1im,q2re,q2im,b0,b1} ---- */
void oracle_init_state(const oracle_problem *p, float *cur, float *best, float *best_f);

/* ---- circuit construction by measurement (Sec. IV-D, Eq. (10)) ---- */
void oracle_sample(const oracle_problem *p, const float *cur, uint32_t gen, uint8_t *gate_idx,
                   uint32_t *seg_id);
/* the same, also writing every slot's qubit amplitudes (2 floats per slot) to amps */
void oracle_sample_amp(const oracle_problem *p, const float *cur, uint32_t gen, uint8_t *gate_idx,
                       uint32_t *seg_id, float *amps);

/* ---- segment fitness, elitism, adaptive mutation (Sec. IV-E1, IV-F) ---- */
void oracle_update(const oracle_problem *p, float *cur, float *best, float *best_f, uint32_t gen,
                   const uint32_t *seg_id, const double *fitness);
/* SU(3) operator of Eq. (12); params = {th1,th2,th3,ph1,...,ph5} given as cos/sin pairs */
void oracle_su3(const double *cosv, const double *sinv, double *U_re, double *U_im);
/* Eq. (12) evaluated in binary32 in the same order (used by the mutation) */
void oracle_su3_f32(const float *cosv, const float *sinv, float *U_re, float *U_im);
/* same from raw angles (libm cos/sin) */
void oracle_su3_angles(const double params[8], double *U_re, double *U_im);

/* ---- ranking ---- */
/* indices of the k best circuits by (F desc, cost asc, c asc) */
void oracle_topk(const double *F, const uint32_t *cost, uint32_t n, uint32_t k, uint32_t *idx);

/* ---- one whole generation: sample -> eval -> rank -> update ---- */
typedef struct {
  uint32_t generation;
  uint32_t best_circuit; /* circuit index of this generation's best */
  double best_fitness;   /* best F seen so far (all generations) */
  double gen_best_fitness;
  double mean_fitness;
  uint64_t useful_flops;
  uint32_t best_cost;
  uint32_t best_gen;     /* generation in which best_fitness was found */
  uint8_t best_gates[64];
  float best_amps[128]; /* Ising: the best circuit's slot amplitudes */
} oracle_report;

void oracle_step(const oracle_problem *p, float *cur, float *best, float *best_f, uint32_t gen,
                 uint32_t topk, uint8_t *gate_idx, uint32_t *seg_id, double *F, uint32_t *cost,
                 uint32_t *topk_idx, oracle_report *rep);

/* ---- classical GA on the same evaluation (integer-string genomes) ---- */
void oracle_ga_init(const oracle_problem *p, uint32_t G, uint8_t *genome);
/* one generation: SUS selection on F, one-point crossover, per-gene mutation, elitism */
void oracle_ga_next(const oracle_problem *p, uint32_t G, uint32_t gen, double ga_rate,
                    const uint8_t *genome, const double *F, const uint32_t *cost, uint8_t *out);
/* the paper's own GA comparator on the Ising library (Sec. V-B): every gene is
   a gate and its angle (qubit amplitudes, 2 floats); angles start uniform on
   multiples of 2 pi / Q; two-point crossover; per gene, with probability
   ga_rate a fresh gate and angle, else with probability ga_rate the angle
   turned by +-m mutationRange / Q, m uniform in [0, Q] */
void oracle_ga_init_amp(const oracle_problem *p, uint32_t G, uint8_t *genome, float *amps);
void oracle_ga_next_amp(const oracle_problem *p, uint32_t G, uint32_t gen, double ga_rate,
                        const uint8_t *genome, const float *amps, const double *F,
                        const uint32_t *cost, uint8_t *out, float *out_amps);

#ifdef __cplusplus
}
#endif
#endif
