/*
 * qe_oracle.c -- plain FP64 CPU oracle for the batched QEQEA fitness path
 * (arXiv:1809.11134).  TEST INFRASTRUCTURE ONLY: loaded by tests/, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline and reference legs,
 * never by the product path.  Shares no code with the CUDA library.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared (see oracle/build.py).
 * No FMA contraction anywhere: every product and sum is rounded on its own,
 * in the order written here, which is the order the design notes fix.
 */
#include "qe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* 1/sqrt(2) as the nearest binary64 value */
static const double ORC_H_COEF = 0x1.6a09e667f3bcdp-1;

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies whose
 * high/low halves are xor-mixed with the other counter words and the key;
 * the key is bumped by the Weyl constants between rounds.
 * ====================================================================== */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* draws for (a, b, gen, stream) of search p */
static void draw(const oracle_problem *p, uint32_t a, uint32_t b, uint32_t gen, uint32_t stream,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {a, b, gen, (p->run << 4) | stream};
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  oracle_philox4x32_10(ctr, key, out);
}

/* integer in [0, m) */
static uint32_t below(uint32_t u, uint32_t m) { return (uint32_t)(((uint64_t)u * m) >> 32); }
/* real in (0, 1), binary64: (u + 1/2) 2^-32 */
static double unit(uint32_t u) { return ((double)u + 0.5) * 0x1p-32; }
/* real in (0, 1), binary32: the top 23 bits plus 1/2, times 2^-23 (exact) */
static float unit32(uint32_t u) { return ((float)(u >> 9) + 0.5f) * 0x1p-23f; }

/* streams of the Philox counter's last word */
enum { ST_SAMPLE = 0, ST_MUT_DECIDE = 1, ST_MUT_SEG = 2, ST_SHOT = 3, ST_GA = 4, ST_GA_INIT = 5 };

/* ======================================================================
 * Library and population geometry.
 * ====================================================================== */
/* Ising library: the n wires, then the n(n-1)/2 pairs i < j */
static int is_ising(uint32_t library) { return library == ORC_LIB_ISING; }

uint32_t oracle_num_regions(uint32_t n, uint32_t library) {
  if (is_ising(library)) return n + n * (n - 1) / 2;
  uint32_t r = 0;
  if (library & ORC_LIB_NCV) r += n * (n - 1);
  if (library & ORC_LIB_HT) r += n;
  return r;
}

uint32_t oracle_num_gates(uint32_t n, uint32_t library) {
  if (is_ising(library)) return 3 * n + n * (n - 1) / 2;
  return ((library & ORC_LIB_IDENTITY) ? 1u : 0u) + 3u * oracle_num_regions(n, library);
}

int oracle_gate_desc(uint32_t n, uint32_t library, uint32_t g, int *kind, int *ctrl, int *tgt) {
  uint32_t G = oracle_num_gates(n, library);
  if (g >= G) return -1;
  uint32_t code = g;
  *ctrl = -1;
  *tgt = -1;
  if (is_ising(library)) {
    if (g < 3 * n) {
      *tgt = (int)(g / 3);
      *kind = (g % 3 == 0) ? ORC_RX : (g % 3 == 1) ? ORC_RY : ORC_RZ;
      return 0;
    }
    /* pair number g - 3n in lexicographic order of (i, j), i < j */
    uint32_t q = g - 3 * n;
    for (uint32_t i = 0; i < n; ++i)
      for (uint32_t j = i + 1; j < n; ++j) {
        if (q == 0) {
          *ctrl = (int)i;
          *tgt = (int)j;
          *kind = ORC_J;
          return 0;
        }
        --q;
      }
    return -1;
  }
  if (library & ORC_LIB_IDENTITY) {
    if (g == 0) {
      *kind = ORC_I;
      return 0;
    }
    code = g - 1;
  }
  uint32_t npair = (library & ORC_LIB_NCV) ? n * (n - 1) : 0;
  uint32_t r = code / 3, k = code % 3;
  if (r < npair) {
    uint32_t c = r / (n - 1), t = r % (n - 1);
    if (t >= c) t += 1;
    *ctrl = (int)c;
    *tgt = (int)t;
    *kind = (k == 0) ? ORC_CNOT : (k == 1) ? ORC_CV : ORC_CVDG;
  } else {
    *tgt = (int)(r - npair);
    *kind = (k == 0) ? ORC_H : (k == 1) ? ORC_T : ORC_TDG;
  }
  return 0;
}

uint32_t oracle_region_gate(uint32_t n, uint32_t library, uint32_t r, uint32_t k) {
  if (is_ising(library)) return r < n ? 3 * r + k : 3 * n + (r - n);
  return ((library & ORC_LIB_IDENTITY) ? 1u : 0u) + 3u * r + k;
}

/* Eq. (10): segmentIndex = region * L * P + individual * L + position */
uint64_t oracle_segment_index(uint64_t r, uint64_t i, uint64_t t, uint64_t L, uint64_t P) {
  return r * L * P + i * L + t;
}

/* Eq. (8) generalised: regions * sizeOfPopulation * sizeOfIndividual */
uint64_t oracle_num_segments(const oracle_problem *p) {
  return (uint64_t)oracle_num_regions(p->n, p->library) * p->L * p->P;
}

/* ======================================================================
 * Gates (Sec. III; the discrete CNOT/CV/CV^dag/H/T library), expanded to the
 * full register width by Kronecker products (Sec. IV-C, steps 3-4).
 * ====================================================================== */
typedef struct {
  double re, im;
} cplx;

static cplx cmul(cplx a, cplx b) {
  cplx r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  return r;
}
static cplx cadd(cplx a, cplx b) {
  cplx r;
  r.re = a.re + b.re;
  r.im = a.im + b.im;
  return r;
}

/* cos(theta/2), sin(theta/2) of the angle of the amplitudes (b0, b1) =
   (cos theta, sin theta), theta in [0, 2 pi): sin(theta/2) >= 0, and
   cos(theta/2) < 0 exactly when theta > pi, i.e. b1 < 0 */
void oracle_half_angle(float b0, float b1, double *c, double *s) {
  double a = (1.0 + (double)b0) * 0.5, b = (1.0 - (double)b0) * 0.5;
  if (a < 0.0) a = 0.0;
  if (b < 0.0) b = 0.0;
  *c = (b1 < 0.0f) ? -sqrt(a) : sqrt(a);
  *s = sqrt(b);
}

/* 2x2 single-qubit operator acting on the target wire; (c, s) = cos/sin of
   theta/2 for the rotations of Eqs. (3)-(5) */
static void gate_2x2(int kind, double c, double s, cplx u[2][2]) {
  const double h = ORC_H_COEF;
  cplx z = {0.0, 0.0}, one = {1.0, 0.0};
  u[0][0] = one;
  u[0][1] = z;
  u[1][0] = z;
  u[1][1] = one;
  switch (kind) {
    case ORC_CNOT: /* X */
      u[0][0] = z;
      u[0][1] = one;
      u[1][0] = one;
      u[1][1] = z;
      break;
    case ORC_CV: /* V = (1/2)[[1+i, 1-i], [1-i, 1+i]], V^2 = X */
      u[0][0] = (cplx){0.5, 0.5};
      u[0][1] = (cplx){0.5, -0.5};
      u[1][0] = (cplx){0.5, -0.5};
      u[1][1] = (cplx){0.5, 0.5};
      break;
    case ORC_CVDG: /* V^dag */
      u[0][0] = (cplx){0.5, -0.5};
      u[0][1] = (cplx){0.5, 0.5};
      u[1][0] = (cplx){0.5, 0.5};
      u[1][1] = (cplx){0.5, -0.5};
      break;
    case ORC_H:
      u[0][0] = (cplx){h, 0.0};
      u[0][1] = (cplx){h, 0.0};
      u[1][0] = (cplx){h, 0.0};
      u[1][1] = (cplx){-h, 0.0};
      break;
    case ORC_T: /* diag(1, e^{i pi/4}) */
      u[1][1] = (cplx){h, h};
      break;
    case ORC_TDG:
      u[1][1] = (cplx){h, -h};
      break;
    case ORC_RX: /* Eq. (3): [[c, -i s], [-i s, c]] */
      u[0][0] = (cplx){c, 0.0};
      u[0][1] = (cplx){0.0, -s};
      u[1][0] = (cplx){0.0, -s};
      u[1][1] = (cplx){c, 0.0};
      break;
    case ORC_RY: /* Eq. (4): [[c, -s], [s, c]] */
      u[0][0] = (cplx){c, 0.0};
      u[0][1] = (cplx){-s, 0.0};
      u[1][0] = (cplx){s, 0.0};
      u[1][1] = (cplx){c, 0.0};
      break;
    case ORC_RZ: /* Eq. (5): diag(e^{-i theta/2}, e^{i theta/2}) */
      u[0][0] = (cplx){c, -s};
      u[1][1] = (cplx){c, s};
      break;
    default:
      break;
  }
}

/* out (2a x 2a) = A (a x a) (x) B (2 x 2) */
static void kron2(const cplx *A, uint32_t a, cplx B[2][2], cplx *out) {
  uint32_t w = 2 * a;
  for (uint32_t i = 0; i < a; ++i)
    for (uint32_t j = 0; j < a; ++j)
      for (uint32_t k = 0; k < 2; ++k)
        for (uint32_t l = 0; l < 2; ++l) out[(2 * i + k) * w + (2 * j + l)] = cmul(A[i * a + j], B[k][l]);
}

/* M_0 (x) M_1 (x) ... (x) M_{n-1}, wire 0 leftmost (most significant) */
static void kron_chain(uint32_t n, cplx (*M)[2][2], cplx *out) {
  uint32_t N = 1u << n;
  cplx *a = (cplx *)malloc(sizeof(cplx) * N * N);
  cplx *b = (cplx *)malloc(sizeof(cplx) * N * N);
  a[0] = (cplx){1.0, 0.0};
  uint32_t dim = 1;
  for (uint32_t w = 0; w < n; ++w) {
    kron2(a, dim, M[w], b);
    dim *= 2;
    cplx *t = a;
    a = b;
    b = t;
  }
  memcpy(out, a, sizeof(cplx) * N * N);
  free(a);
  free(b);
}

static void dense_gate(uint32_t n, int kind, int ctrl, int tgt, double c, double s, cplx *G) {
  uint32_t N = 1u << n;
  cplx id[2][2] = {{{1.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {1.0, 0.0}}};
  cplx u[2][2];
  gate_2x2(kind, c, s, u);
  cplx (*M)[2][2] = malloc(sizeof(cplx[2][2]) * n);
  if (kind == ORC_J) {
    /* interaction template: the +-1 diagonal D = z_i z_j, then the term-wise
       exponent exp(-i theta/2 D) = c - i D s on the diagonal */
    for (uint32_t e = 0; e < N * N; ++e) G[e] = (cplx){0.0, 0.0};
    for (uint32_t b = 0; b < N; ++b) {
      int zi = ((b >> (n - 1 - (uint32_t)ctrl)) & 1u) ? -1 : 1;
      int zj = ((b >> (n - 1 - (uint32_t)tgt)) & 1u) ? -1 : 1;
      double d = (double)(zi * zj);
      G[b * N + b] = (cplx){c, -d * s};
    }
  } else if (kind == ORC_I) {
    for (uint32_t w = 0; w < n; ++w) memcpy(M[w], id, sizeof id);
    kron_chain(n, M, G);
  } else if (ctrl < 0) {
    /* I (x) ... (x) U_w (x) ... (x) I */
    for (uint32_t w = 0; w < n; ++w) memcpy(M[w], (int)w == tgt ? u : id, sizeof id);
    kron_chain(n, M, G);
  } else {
    /* |0><0|_c (x) I  +  |1><1|_c (x) U_t */
    cplx p0[2][2] = {{{1.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 0.0}}};
    cplx p1[2][2] = {{{0.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {1.0, 0.0}}};
    cplx *A = (cplx *)malloc(sizeof(cplx) * N * N);
    cplx *B = (cplx *)malloc(sizeof(cplx) * N * N);
    for (uint32_t w = 0; w < n; ++w) memcpy(M[w], (int)w == ctrl ? p0 : id, sizeof id);
    kron_chain(n, M, A);
    for (uint32_t w = 0; w < n; ++w) memcpy(M[w], (int)w == ctrl ? p1 : ((int)w == tgt ? u : id), sizeof id);
    kron_chain(n, M, B);
    for (uint32_t e = 0; e < N * N; ++e) G[e] = cadd(A[e], B[e]);
    free(A);
    free(B);
  }
  free(M);
}

/* cos/sin of theta/2 of slot t (Ising), NaN without amplitudes */
static void slot_angle(uint32_t library, const float *amps, uint32_t t, double *c, double *s) {
  if (!is_ising(library)) {
    *c = 1.0;
    *s = 0.0;
  } else if (!amps) {
    *c = *s = NAN;
  } else {
    oracle_half_angle(amps[2 * t], amps[2 * t + 1], c, s);
  }
}

void oracle_gate_matrix(uint32_t n, uint32_t library, uint32_t g, double *re, double *im) {
  oracle_gate_matrix_amp(n, library, g, NAN, NAN, re, im);
}

void oracle_gate_matrix_amp(uint32_t n, uint32_t library, uint32_t g, float b0, float b1,
                            double *re, double *im) {
  uint32_t N = 1u << n;
  int kind, ctrl, tgt;
  cplx *G = (cplx *)malloc(sizeof(cplx) * N * N);
  if (oracle_gate_desc(n, library, g, &kind, &ctrl, &tgt) != 0) {
    for (uint32_t e = 0; e < N * N; ++e) re[e] = im[e] = NAN;
    free(G);
    return;
  }
  const float ab[2] = {b0, b1};
  double c, s;
  slot_angle(library, (b0 == b0) ? ab : NULL, 0, &c, &s);
  dense_gate(n, kind, ctrl, tgt, c, s, G);
  for (uint32_t e = 0; e < N * N; ++e) {
    re[e] = G[e].re;
    im[e] = G[e].im;
  }
  free(G);
}

/* C = A B, k ascending, accumulator starting at +0 */
static void matmul(uint32_t N, const cplx *A, const cplx *B, cplx *C) {
  for (uint32_t i = 0; i < N; ++i)
    for (uint32_t j = 0; j < N; ++j) {
      cplx acc = {0.0, 0.0};
      for (uint32_t k = 0; k < N; ++k) acc = cadd(acc, cmul(A[i * N + k], B[k * N + j]));
      C[i * N + j] = acc;
    }
}

static void compose_c(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates,
                      const float *amps, cplx *S) {
  uint32_t N = 1u << n;
  cplx *G = (cplx *)malloc(sizeof(cplx) * N * N);
  cplx *T = (cplx *)malloc(sizeof(cplx) * N * N);
  for (uint32_t i = 0; i < N; ++i)
    for (uint32_t j = 0; j < N; ++j) S[i * N + j] = (cplx){i == j ? 1.0 : 0.0, 0.0};
  for (uint32_t t = 0; t < L; ++t) {
    int kind, ctrl, tgt;
    if (oracle_gate_desc(n, library, gates[t], &kind, &ctrl, &tgt) != 0) {
      for (uint32_t e = 0; e < N * N; ++e) S[e] = (cplx){NAN, NAN};
      break;
    }
    double c, s;
    slot_angle(library, amps, t, &c, &s);
    dense_gate(n, kind, ctrl, tgt, c, s, G);
    matmul(N, G, S, T); /* S <- G_t S */
    memcpy(S, T, sizeof(cplx) * N * N);
  }
  free(G);
  free(T);
}

void oracle_compose(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates, double *S_re,
                    double *S_im) {
  oracle_compose_amp(n, library, L, gates, NULL, S_re, S_im);
}

void oracle_compose_amp(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates,
                        const float *amps, double *S_re, double *S_im) {
  uint32_t N = 1u << n;
  cplx *S = (cplx *)malloc(sizeof(cplx) * N * N);
  compose_c(n, library, L, gates, amps, S);
  for (uint32_t e = 0; e < N * N; ++e) {
    S_re[e] = S[e].re;
    S_im[e] = S[e].im;
  }
  free(S);
}

/* ======================================================================
 * Eq. (11): fitness = 1 - sqrt((size - |tr(S^dag T)|) / size), size = 2^n.
 * For a permutation target T|j> = |perm[j]>, tr(S^dag T) is the sum over j
 * of conj(S[perm[j]][j]); it is accumulated with j ascending.
 * ====================================================================== */
/* Eq. (11) with a dense unitary T: tr(S^dag T) = sum_j (S^dag T)_jj, the
   diagonal element (S^dag T)_jj = sum_i conj(S_ij) T_ij. */
static double score_dense_c(uint32_t n, const cplx *S, const double *T) {
  uint32_t N = 1u << n;
  double size = (double)N;
  double tr_re = 0.0, tr_im = 0.0;
  for (uint32_t j = 0; j < N; ++j) {
    double d_re = 0.0, d_im = 0.0; /* (S^dag T)_jj */
    for (uint32_t i = 0; i < N; ++i) {
      cplx s = S[i * N + j];
      double t_re = T[2 * (i * N + j)], t_im = T[2 * (i * N + j) + 1];
      d_re = d_re + (s.re * t_re + s.im * t_im);
      d_im = d_im + (s.re * t_im - s.im * t_re);
    }
    tr_re = tr_re + d_re;
    tr_im = tr_im + d_im;
  }
  double m = sqrt(tr_re * tr_re + tr_im * tr_im);
  double d = (size - m) / size;
  if (d < 0.0) d = 0.0;
  return 1.0 - sqrt(d);
}

static double score_c(uint32_t n, const cplx *S, const uint8_t *perm, uint32_t kind) {
  uint32_t N = 1u << n;
  double size = (double)N;
  if (kind == ORC_FIT_PROB) {
    double q = 0.0;
    for (uint32_t j = 0; j < N; ++j) {
      cplx s = S[perm[j] * N + j];
      q = q + (s.re * s.re + s.im * s.im);
    }
    double d = (size - q) / size;
    if (d < 0.0) d = 0.0;
    return 1.0 - sqrt(d);
  }
  double tr_re = 0.0, tr_im = 0.0;
  for (uint32_t j = 0; j < N; ++j) {
    cplx s = S[perm[j] * N + j];
    tr_re = tr_re + s.re;
    tr_im = tr_im + (-s.im);
  }
  double m = sqrt(tr_re * tr_re + tr_im * tr_im);
  double d = (size - m) / size;
  if (d < 0.0) d = 0.0;
  return 1.0 - sqrt(d);
}

/* the fitness of a search: Eq. (11) against its permutation or dense target
   (the probability-overlap reading is defined for permutations only) */
static double score_p(const oracle_problem *p, const cplx *S) {
  if (p->target) return p->fitness_kind == ORC_FIT_PROB ? NAN : score_dense_c(p->n, S, p->target);
  return score_c(p->n, S, p->perm, p->fitness_kind);
}

double oracle_score_dense(uint32_t n, const double *S_re, const double *S_im, const double *T) {
  uint32_t N = 1u << n;
  cplx *S = (cplx *)malloc(sizeof(cplx) * N * N);
  for (uint32_t e = 0; e < N * N; ++e) S[e] = (cplx){S_re[e], S_im[e]};
  double f = score_dense_c(n, S, T);
  free(S);
  return f;
}

double oracle_score(uint32_t n, const double *S_re, const double *S_im, const uint8_t *perm,
                    uint32_t fitness_kind) {
  uint32_t N = 1u << n;
  cplx *S = (cplx *)malloc(sizeof(cplx) * N * N);
  for (uint32_t e = 0; e < N * N; ++e) S[e] = (cplx){S_re[e], S_im[e]};
  double f = score_c(n, S, perm, fitness_kind);
  free(S);
  return f;
}

/* gate cost: number of gates that are not the identity */
uint32_t oracle_cost(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates) {
  uint32_t cost = 0;
  for (uint32_t t = 0; t < L; ++t) {
    int kind, ctrl, tgt;
    if (oracle_gate_desc(n, library, gates[t], &kind, &ctrl, &tgt) != 0) continue;
    if (kind != ORC_I) cost += 1;
  }
  return cost;
}

uint64_t oracle_useful_flops(uint32_t n, uint32_t library, uint32_t L, const uint8_t *gates) {
  uint64_t N = 1ull << n, NN = N * N, total = 2 * N; /* score: N complex adds */
  for (uint32_t t = 0; t < L; ++t) {
    int kind, ctrl, tgt;
    if (oracle_gate_desc(n, library, gates[t], &kind, &ctrl, &tgt) != 0) continue;
    switch (kind) {
      case ORC_CV:
      case ORC_CVDG:
      case ORC_H:
        total += 4 * NN;
        break;
      case ORC_T:
      case ORC_TDG:
        total += 2 * NN;
        break;
      case ORC_RX: /* every amplitude: two real-by-complex products and a sum */
      case ORC_RY:
      case ORC_RZ: /* every amplitude: one complex product */
      case ORC_J:
        total += 6 * NN;
        break;
      default:
        break;
    }
  }
  return total;
}

void oracle_eval(const oracle_problem *p, const uint8_t *gates, uint32_t n_circuits, double *F,
                 uint32_t *cost) {
  oracle_eval_amp(p, gates, NULL, n_circuits, F, cost);
}

void oracle_eval_amp(const oracle_problem *p, const uint8_t *gates, const float *amps,
                     uint32_t n_circuits, double *F, uint32_t *cost) {
  uint32_t N = 1u << p->n;
  cplx *S = (cplx *)malloc(sizeof(cplx) * N * N);
  for (uint32_t c = 0; c < n_circuits; ++c) {
    const uint8_t *g = gates + (uint64_t)c * p->L;
    compose_c(p->n, p->library, p->L, g, amps ? amps + (uint64_t)c * 2 * p->L : NULL, S);
    double f = score_p(p, S);
    uint32_t k = oracle_cost(p->n, p->library, p->L, g);
    double pen = p->cost_weight * ((double)k / (double)p->L);
    F[c] = f - pen;
    if (cost) cost[c] = k;
  }
  free(S);
}

/* ======================================================================
 * Encoding state (Sec. IV-A, IV-B): every segment holds one qutrit
 * (3 complex amplitudes) and one qubit (2 real amplitudes).  Initial state is
 * uniform: qutrit amplitudes 1/sqrt(3), qubit amplitudes 1/sqrt(2).
 * ====================================================================== */
void oracle_init_state(const oracle_problem *p, float *cur, float *best, float *best_f) {
  uint64_t S = oracle_num_segments(p);
  float a = (float)(1.0 / sqrt(3.0));
  float b = (float)ORC_H_COEF;
  for (uint64_t s = 0; s < S; ++s) {
    float *q = cur + 8 * s;
    q[0] = a;
    q[1] = 0.0f;
    q[2] = a;
    q[3] = 0.0f;
    q[4] = a;
    q[5] = 0.0f;
    q[6] = b;
    q[7] = b;
    memcpy(best + 8 * s, q, 8 * sizeof(float));
    best_f[s] = -1.0f;
  }
}

/* ======================================================================
 * Circuit construction (Sec. IV-D): for every circuit c and slot t draw
 * whichIndividual in [0, P) and whichRotationOrInteraction in [0, R), form
 * the segment index of Eq. (10), then measure that segment's qutrit (and, if
 * the identity is in the library, its qubit) to obtain the gate.
 * ====================================================================== */
void oracle_sample(const oracle_problem *p, const float *cur, uint32_t gen, uint8_t *gate_idx,
                   uint32_t *seg_id) {
  oracle_sample_amp(p, cur, gen, gate_idx, seg_id, NULL);
}

void oracle_sample_amp(const oracle_problem *p, const float *cur, uint32_t gen, uint8_t *gate_idx,
                       uint32_t *seg_id, float *amps) {
  uint32_t R = oracle_num_regions(p->n, p->library);
  /* discrete libraries with the identity: the qubit decides "gate present";
     Ising: the qubit holds the angle and is not measured */
  int has_qubit = (p->library & ORC_LIB_IDENTITY) != 0 && !is_ising(p->library);
  for (uint32_t c = 0; c < p->P; ++c)
    for (uint32_t t = 0; t < p->L; ++t) {
      uint32_t u[4];
      draw(p, c, t, gen, ST_SAMPLE, u);
      uint32_t i = below(u[0], p->P);
      uint32_t r = below(u[1], R);
      uint64_t seg = oracle_segment_index(r, i, t, p->L, p->P);
      const float *q = cur + 8 * seg;
      /* qutrit measurement: outcome k with probability |q_k|^2 / sum, the
         cumulative comparison taken in binary32 */
      float p0 = q[0] * q[0] + q[1] * q[1];
      float p1 = q[2] * q[2] + q[3] * q[3];
      float p2 = q[4] * q[4] + q[5] * q[5];
      float p01 = p0 + p1;
      float s = p01 + p2;
      uint32_t k;
      if (p->shots <= 1) {
        float x = unit32(u[2]) * s;
        k = (x < p0) ? 0u : ((x < p01) ? 1u : 2u);
      } else {
        /* Sec. IV-A1: the qutrit is measured K times and the most frequent
           outcome taken (the lowest outcome on a tie); shot j uses word j mod 4
           of the draw (c, t + 64 floor(j / 4), gen) of its own stream */
        uint32_t count[3] = {0, 0, 0};
        for (uint32_t j = 0; j < p->shots; ++j) {
          uint32_t w[4];
          draw(p, c, t + 64u * (j / 4u), gen, ST_SHOT, w);
          float x = unit32(w[j % 4u]) * s;
          count[(x < p0) ? 0 : ((x < p01) ? 1 : 2)] += 1;
        }
        k = 0;
        if (count[1] > count[k]) k = 1;
        if (count[2] > count[k]) k = 2;
      }
      uint32_t g = oracle_region_gate(p->n, p->library, r, k);
      if (has_qubit) {
        /* qubit measurement: outcome 1 (gate present) with probability b1^2/(b0^2+b1^2) */
        float B0 = q[6] * q[6];
        float B1 = q[7] * q[7];
        float y = unit32(u[3]) * (B0 + B1);
        if (y < B0) g = 0; /* identity */
      }
      gate_idx[(uint64_t)c * p->L + t] = (uint8_t)g;
      seg_id[(uint64_t)c * p->L + t] = (uint32_t)seg;
      if (amps) {
        amps[2 * ((uint64_t)c * p->L + t)] = q[6];
        amps[2 * ((uint64_t)c * p->L + t) + 1] = q[7];
      }
    }
}

/* ======================================================================
 * Eq. (12): the SU(3) operator used to mutate a qutrit, with c_k = cos th_k,
 * s_k = sin th_k and E(x) = e^{i x}.  Products are evaluated left to right in
 * the printed order; phase factors are multiplied as complex numbers.
 * Index convention of cosv/sinv: 0..2 = th1..th3, 3..7 = ph1..ph5.
 * ====================================================================== */
static cplx ephase(const double *cosv, const double *sinv, int idx, double sign) {
  cplx e;
  e.re = cosv[idx];
  e.im = sign * sinv[idx];
  return e;
}
static cplx cscale(cplx a, double s) {
  cplx r;
  r.re = a.re * s;
  r.im = a.im * s;
  return r;
}
static cplx csub(cplx a, cplx b) {
  cplx r;
  r.re = a.re - b.re;
  r.im = a.im - b.im;
  return r;
}
static cplx cneg(cplx a) {
  cplx r;
  r.re = -a.re;
  r.im = -a.im;
  return r;
}

void oracle_su3(const double *cv, const double *sv, double *U_re, double *U_im) {
  double c1 = cv[0], c2 = cv[1], c3 = cv[2];
  double s1 = sv[0], s2 = sv[1], s3 = sv[2];
#define EP(k) ephase(cv, sv, 2 + (k), 1.0)  /* e^{+i phi_k} */
#define EM(k) ephase(cv, sv, 2 + (k), -1.0) /* e^{-i phi_k} */
  cplx U[9];
  /* row 0 */
  U[0] = cscale(cscale(EP(1), c1), c2);
  U[1] = cscale(EP(3), s1);
  U[2] = cscale(cscale(EP(4), c1), s2);
  /* row 1 */
  U[3] = csub(cscale(cscale(cmul(EM(4), EM(5)), s2), s3),
              cscale(cscale(cscale(cmul(cmul(EP(1), EP(2)), EM(3)), s1), c2), c3));
  U[4] = cscale(cscale(EP(2), c1), c3);
  U[5] = csub(cneg(cscale(cscale(cmul(EM(1), EM(5)), c2), s3)),
              cscale(cscale(cscale(cmul(cmul(EP(2), EM(3)), EP(4)), s1), s2), c3));
  /* row 2 */
  U[6] = csub(cneg(cscale(cscale(cmul(EM(2), EM(4)), s2), c3)),
              cscale(cscale(cscale(cmul(cmul(EP(1), EM(3)), EP(5)), s1), c2), s3));
  U[7] = cscale(cscale(EP(5), c1), s3);
  U[8] = csub(cscale(cscale(cmul(EM(1), EM(2)), c2), c3),
              cscale(cscale(cscale(cmul(cmul(EM(3), EP(4)), EP(5)), s1), s2), s3));
#undef EP
#undef EM
  for (int e = 0; e < 9; ++e) {
    U_re[e] = U[e].re;
    U_im[e] = U[e].im;
  }
}

void oracle_su3_angles(const double params[8], double *U_re, double *U_im) {
  double cv[8], sv[8];
  for (int k = 0; k < 8; ++k) {
    cv[k] = cos(params[k]);
    sv[k] = sin(params[k]);
  }
  oracle_su3(cv, sv, U_re, U_im);
}

/* ======================================================================
 * Segment fitness, elitism and adaptive mutation (Sec. IV-E1, IV-F).
 * ====================================================================== */
static const double ORC_PI = 3.14159265358979323846;

/* binary32 complex helpers for the mutation arithmetic */
typedef struct {
  float re, im;
} fcplx;
static fcplx fmulc(fcplx a, fcplx b) {
  fcplx r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  return r;
}
static fcplx faddc(fcplx a, fcplx b) {
  fcplx r;
  r.re = a.re + b.re;
  r.im = a.im + b.im;
  return r;
}
static fcplx fsubc(fcplx a, fcplx b) {
  fcplx r;
  r.re = a.re - b.re;
  r.im = a.im - b.im;
  return r;
}
static fcplx fscale(fcplx a, float s) {
  fcplx r;
  r.re = a.re * s;
  r.im = a.im * s;
  return r;
}
static fcplx fnegc(fcplx a) {
  fcplx r;
  r.re = -a.re;
  r.im = -a.im;
  return r;
}

/* Eq. (12) in binary32, the same evaluation order as oracle_su3 */
void oracle_su3_f32(const float *cv, const float *sv, float *U_re, float *U_im) {
  float c1 = cv[0], c2 = cv[1], c3 = cv[2];
  float s1 = sv[0], s2 = sv[1], s3 = sv[2];
#define EP(k) ((fcplx){cv[2 + (k)], sv[2 + (k)]})
#define EM(k) ((fcplx){cv[2 + (k)], -sv[2 + (k)]})
  fcplx U[9];
  U[0] = fscale(fscale(EP(1), c1), c2);
  U[1] = fscale(EP(3), s1);
  U[2] = fscale(fscale(EP(4), c1), s2);
  U[3] = fsubc(fscale(fscale(fmulc(EM(4), EM(5)), s2), s3),
               fscale(fscale(fscale(fmulc(fmulc(EP(1), EP(2)), EM(3)), s1), c2), c3));
  U[4] = fscale(fscale(EP(2), c1), c3);
  U[5] = fsubc(fnegc(fscale(fscale(fmulc(EM(1), EM(5)), c2), s3)),
               fscale(fscale(fscale(fmulc(fmulc(EP(2), EM(3)), EP(4)), s1), s2), c3));
  U[6] = fsubc(fnegc(fscale(fscale(fmulc(EM(2), EM(4)), s2), c3)),
               fscale(fscale(fscale(fmulc(fmulc(EP(1), EM(3)), EP(5)), s1), c2), s3));
  U[7] = fscale(fscale(EP(5), c1), s3);
  U[8] = fsubc(fscale(fscale(fmulc(EM(1), EM(2)), c2), c3),
               fscale(fscale(fscale(fmulc(fmulc(EM(3), EP(4)), EP(5)), s1), s2), s3));
#undef EP
#undef EM
  for (int e = 0; e < 9; ++e) {
    U_re[e] = U[e].re;
    U_im[e] = U[e].im;
  }
}

/* cos/sin of m * step for m in [0, Q], computed in binary64 and rounded */
static void trig_f32(double step, uint32_t m, float *c, float *s) {
  double ang = (double)m * step;
  *c = (float)cos(ang);
  *s = (float)sin(ang);
}

/* Adaptive mutation of one segment (Sec. IV-F).  e = 1 - segmentFitness.
   - qubit: rotate (b0, b1) by +-(1 - f) * mutationRange, quantised to range/Q
   - qutrit: one of the eight Eq. (12) parameters is set to a uniform draw from
     its domain times (1 - f), quantised to domain/Q; the rest are zero. */
static void mutate_segment(const oracle_problem *p, float *q, float bf, uint32_t gen, uint64_t seg,
                           int has_qubit) {
  uint32_t w[4];
  draw(p, (uint32_t)seg, 0, gen, ST_MUT_SEG, w);
  float fc = bf < 0.0f ? 0.0f : (bf > 1.0f ? 1.0f : bf);
  float e = 1.0f - fc;
  if (!(e == e)) e = 1.0f; /* a NaN best fitness mutates fully */
  if (has_qubit && w[0] < 0x80000000u) {
    uint32_t m = (uint32_t)floorf(e * (float)ORC_Q);
    float c, s;
    trig_f32(p->mutation_range / (double)ORC_Q, m, &c, &s);
    if (w[1] & 1u) s = -s;
    float R[2][2] = {{c, -s}, {s, c}};
    float b[2] = {q[6], q[7]};
    for (int a = 0; a < 2; ++a) {
      float acc = 0.0f;
      for (int k = 0; k < 2; ++k) acc = acc + R[a][k] * b[k];
      q[6 + a] = acc;
    }
    return;
  }
  uint32_t j = below(w[1], 8);
  uint32_t m = (uint32_t)floorf((unit32(w[2]) * e) * (float)ORC_Q);
  double domain = (j < 3) ? (ORC_PI / 2.0) : (2.0 * ORC_PI);
  float cv[8], sv[8];
  for (int k = 0; k < 8; ++k) {
    cv[k] = 1.0f;
    sv[k] = 0.0f;
  }
  trig_f32(domain / (double)ORC_Q, m, &cv[j], &sv[j]);
  float Ur[9], Ui[9];
  oracle_su3_f32(cv, sv, Ur, Ui);
  fcplx in[3] = {{q[0], q[1]}, {q[2], q[3]}, {q[4], q[5]}};
  for (int a = 0; a < 3; ++a) {
    fcplx acc = {0.0f, 0.0f};
    for (int k = 0; k < 3; ++k) acc = faddc(acc, fmulc((fcplx){Ur[3 * a + k], Ui[3 * a + k]}, in[k]));
    q[2 * a] = acc.re;
    q[2 * a + 1] = acc.im;
  }
}

void oracle_update(const oracle_problem *p, float *cur, float *best, float *best_f, uint32_t gen,
                   const uint32_t *seg_id, const double *fitness) {
  uint64_t S = oracle_num_segments(p);
  uint32_t R = oracle_num_regions(p->n, p->library);
  /* the qubit exists with the identity (gate present) and in the Ising
     library (the angle); either may be mutated */
  int has_qubit = (p->library & (ORC_LIB_IDENTITY | ORC_LIB_ISING)) != 0;
  float *sf = (float *)malloc(sizeof(float) * (S ? S : 1));
  uint8_t *touched = (uint8_t *)calloc(S ? S : 1, 1);
  /* segment fitness: a segment takes the fitness of the circuit that used it
     (rounded to binary32); when several circuits used it in this generation it
     takes the largest */
  for (uint64_t c = 0; c < p->P; ++c)
    for (uint64_t t = 0; t < p->L; ++t) {
      uint64_t seg = seg_id[c * p->L + t];
      float f = (float)fitness[c];
      if (!touched[seg] || f > sf[seg]) sf[seg] = f;
      touched[seg] = 1;
    }
  /* elitism: keep the state if it beat the segment's best so far, else revert */
  for (uint64_t seg = 0; seg < S; ++seg) {
    if (!touched[seg]) continue;
    if (sf[seg] > best_f[seg]) {
      memcpy(best + 8 * seg, cur + 8 * seg, 8 * sizeof(float));
      best_f[seg] = sf[seg];
    } else {
      memcpy(cur + 8 * seg, best + 8 * seg, 8 * sizeof(float));
    }
  }
  /* mutation: each individual changes with probabilityOfMutation; all of its
     segments (every region, every position) are then mutated */
  for (uint32_t i = 0; i < p->P; ++i) {
    uint32_t v[4];
    draw(p, i, 0, gen, ST_MUT_DECIDE, v);
    if (!(unit(v[0]) < p->p_mutation)) continue;
    for (uint32_t r = 0; r < R; ++r)
      for (uint32_t t = 0; t < p->L; ++t) {
        uint64_t seg = oracle_segment_index(r, i, t, p->L, p->P);
        mutate_segment(p, cur + 8 * seg, best_f[seg], gen, seg, has_qubit);
      }
  }
  free(sf);
  free(touched);
}

/* ======================================================================
 * Ranking by (F desc, cost asc, circuit asc) -- a total order.
 * ====================================================================== */
typedef struct {
  double F;
  uint32_t cost, c;
} rank_item;

static int rank_cmp(const void *a, const void *b) {
  const rank_item *x = (const rank_item *)a, *y = (const rank_item *)b;
  if (x->F > y->F) return -1;
  if (x->F < y->F) return 1;
  if (x->cost < y->cost) return -1;
  if (x->cost > y->cost) return 1;
  return (x->c < y->c) ? -1 : (x->c > y->c);
}

void oracle_topk(const double *F, const uint32_t *cost, uint32_t n, uint32_t k, uint32_t *idx) {
  rank_item *it = (rank_item *)malloc(sizeof(rank_item) * (n ? n : 1));
  for (uint32_t c = 0; c < n; ++c) {
    it[c].F = F[c];
    it[c].cost = cost[c];
    it[c].c = c;
  }
  qsort(it, n, sizeof(rank_item), rank_cmp);
  for (uint32_t j = 0; j < k && j < n; ++j) idx[j] = it[j].c;
  free(it);
}

/* ======================================================================
 * One generation of the search: sample P circuits, evaluate, rank, update.
 * rep carries the best-so-far record in and out (best_fitness < -1e300 on
 * the first call means "none yet").
 * ====================================================================== */
void oracle_step(const oracle_problem *p, float *cur, float *best, float *best_f, uint32_t gen,
                 uint32_t topk, uint8_t *gate_idx, uint32_t *seg_id, double *F, uint32_t *cost,
                 uint32_t *topk_idx, oracle_report *rep) {
  float *amps = NULL;
  if (is_ising(p->library)) amps = (float *)malloc(sizeof(float) * 2 * (uint64_t)p->P * p->L);
  oracle_sample_amp(p, cur, gen, gate_idx, seg_id, amps);
  oracle_eval_amp(p, gate_idx, amps, p->P, F, cost);
  uint32_t k = topk ? topk : 1;
  uint32_t *tk = topk_idx;
  uint32_t local[1];
  if (!tk) tk = local, k = 1;
  oracle_topk(F, cost, p->P, k, tk);
  uint32_t b = tk[0];
  double mean = 0.0;
  uint64_t flops = 0;
  for (uint32_t c = 0; c < p->P; ++c) {
    mean = mean + F[c];
    flops += oracle_useful_flops(p->n, p->library, p->L, gate_idx + (uint64_t)c * p->L);
    /* a dense score: four products and four sums per element instead of N complex adds */
    if (p->target) flops += 8ull * (1ull << (2 * p->n)) - 2ull * (1ull << p->n);
  }
  rep->generation = gen;
  rep->best_circuit = b;
  rep->gen_best_fitness = F[b];
  rep->mean_fitness = mean / (double)p->P;
  rep->useful_flops = flops;
  if (F[b] > rep->best_fitness || (F[b] == rep->best_fitness && cost[b] < rep->best_cost)) {
    rep->best_fitness = F[b];
    rep->best_cost = cost[b];
    rep->best_gen = gen;
    memset(rep->best_gates, 0, sizeof rep->best_gates);
    memcpy(rep->best_gates, gate_idx + (uint64_t)b * p->L, p->L);
    memset(rep->best_amps, 0, sizeof rep->best_amps);
    if (amps) memcpy(rep->best_amps, amps + (uint64_t)b * 2 * p->L, sizeof(float) * 2 * p->L);
  }
  free(amps);
  oracle_update(p, cur, best, best_f, gen, seg_id, F);
}

/* ======================================================================
 * Classical GA on the same evaluation (the comparison algorithm of
 * Sec. V-B, with the integer-string encoding, one-point crossover and
 * per-gene mutation of the 5-qubit workload).
 *   - selection: stochastic universal sampling on the weights
 *     floor(clamp(F, 0, 1) 2^32) (integers, so every prefix sum is exact),
 *     pointers s + m floor(W/P) with one offset s drawn per generation
 *     (identity selection when floor(W/P) = 0);
 *   - the selected parents, in pointer order, are paired (2m, 2m+1) and
 *     crossed at cut = 1 + below(u, L-1) (no crossover when L == 1);
 *   - each gene is replaced with probability ga_rate by a uniform gate;
 *   - elitism: the best genome of the parent generation is copied to slot 0.
 * ====================================================================== */
void oracle_ga_init(const oracle_problem *p, uint32_t G, uint8_t *genome) {
  for (uint32_t c = 0; c < p->P; ++c)
    for (uint32_t t = 0; t < p->L; ++t) {
      uint32_t u[4];
      draw(p, c, t, 0, ST_GA_INIT, u);
      genome[(uint64_t)c * p->L + t] = (uint8_t)below(u[0], G);
    }
}

/* SUS weight of a circuit: max(F, 0) clamped to 1, as a 32-bit fixed-point integer */
static uint64_t sus_weight(double F) {
  double x = F > 0.0 ? (F < 1.0 ? F : 1.0) : 0.0;
  return (uint64_t)floor(x * 4294967296.0);
}

void oracle_ga_next(const oracle_problem *p, uint32_t G, uint32_t gen, double ga_rate,
                    const uint8_t *genome, const double *F, const uint32_t *cost, uint8_t *out) {
  uint32_t P = p->P, L = p->L;
  uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * P);
  uint64_t W = 0;
  for (uint32_t c = 0; c < P; ++c) {
    W += sus_weight(F[c]);
    cum[c] = W;
  }
  uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * P);
  uint32_t u[4];
  draw(p, 0, 0, gen, ST_GA, u);
  uint64_t D = W / P; /* pointer spacing */
  if (D > 0) {
    /* pointers s + m D with s uniform in [0, D); parent = first c with cum[c] > pointer */
    uint64_t r64 = ((uint64_t)u[1] << 32) | u[0];
    uint64_t s0 = (uint64_t)(((unsigned __int128)r64 * D) >> 64);
    uint32_t c = 0;
    for (uint32_t m = 0; m < P; ++m) {
      uint64_t ptr = s0 + (uint64_t)m * D;
      while (c + 1 < P && !(cum[c] > ptr)) ++c;
      parent[m] = c;
    }
  } else {
    for (uint32_t m = 0; m < P; ++m) parent[m] = m;
  }
  /* crossover */
  for (uint32_t m = 0; m < P; m += 2) {
    const uint8_t *a = genome + (uint64_t)parent[m] * L;
    uint8_t *oa = out + (uint64_t)m * L;
    if (m + 1 >= P) {
      memcpy(oa, a, L);
      break;
    }
    const uint8_t *b = genome + (uint64_t)parent[m + 1] * L;
    uint8_t *ob = out + (uint64_t)(m + 1) * L;
    uint32_t cut = L;
    if (L > 1) {
      uint32_t v[4];
      draw(p, m / 2, 1, gen, ST_GA, v);
      cut = 1 + below(v[0], L - 1);
    }
    for (uint32_t t = 0; t < L; ++t) {
      oa[t] = t < cut ? a[t] : b[t];
      ob[t] = t < cut ? b[t] : a[t];
    }
  }
  /* per-gene mutation */
  for (uint32_t c = 0; c < P; ++c)
    for (uint32_t t = 0; t < L; ++t) {
      uint32_t v[4];
      draw(p, c, 2 + t, gen, ST_GA, v);
      if (unit(v[0]) < ga_rate) out[(uint64_t)c * L + t] = (uint8_t)below(v[1], G);
    }
  /* elitism */
  uint32_t bidx;
  oracle_topk(F, cost, P, 1, &bidx);
  memcpy(out, genome + (uint64_t)bidx * L, L);
  free(cum);
  free(parent);
}

/* ======================================================================
 * The paper's GA comparator on the Ising library (Sec. V-B): genes are
 * (gate, angle) pairs, the angle kept as qubit amplitudes like the QEQEA
 * slots; selection as above (SUS), two-point crossover, and a real-valued
 * mutation of the angle besides the replacement of whole genes.
 * ====================================================================== */
void oracle_ga_init_amp(const oracle_problem *p, uint32_t G, uint8_t *genome, float *amps) {
  for (uint32_t c = 0; c < p->P; ++c)
    for (uint32_t t = 0; t < p->L; ++t) {
      uint32_t u[4];
      uint64_t e = (uint64_t)c * p->L + t;
      draw(p, c, t, 0, ST_GA_INIT, u);
      genome[e] = (uint8_t)below(u[0], G);
      trig_f32((2.0 * ORC_PI) / (double)ORC_Q, below(u[1], ORC_Q), &amps[2 * e], &amps[2 * e + 1]);
    }
}

void oracle_ga_next_amp(const oracle_problem *p, uint32_t G, uint32_t gen, double ga_rate,
                        const uint8_t *genome, const float *amps, const double *F,
                        const uint32_t *cost, uint8_t *out, float *out_amps) {
  uint32_t P = p->P, L = p->L;
  uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * P);
  uint64_t W = 0;
  for (uint32_t c = 0; c < P; ++c) {
    W += sus_weight(F[c]);
    cum[c] = W;
  }
  uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * P);
  uint32_t u[4];
  draw(p, 0, 0, gen, ST_GA, u);
  uint64_t D = W / P;
  if (D > 0) {
    uint64_t r64 = ((uint64_t)u[1] << 32) | u[0];
    uint64_t s0 = (uint64_t)(((unsigned __int128)r64 * D) >> 64);
    uint32_t c = 0;
    for (uint32_t m = 0; m < P; ++m) {
      uint64_t ptr = s0 + (uint64_t)m * D;
      while (c + 1 < P && !(cum[c] > ptr)) ++c;
      parent[m] = c;
    }
  } else {
    for (uint32_t m = 0; m < P; ++m) parent[m] = m;
  }
  /* two-point crossover: the genes in [lo, hi) come from the other parent */
  for (uint32_t m = 0; m < P; m += 2) {
    uint64_t a = (uint64_t)parent[m] * L, oa = (uint64_t)m * L;
    if (m + 1 >= P) {
      memcpy(out + oa, genome + a, L);
      memcpy(out_amps + 2 * oa, amps + 2 * a, 2 * L * sizeof(float));
      break;
    }
    uint64_t b = (uint64_t)parent[m + 1] * L, ob = (uint64_t)(m + 1) * L;
    uint32_t lo = L, hi = L;
    if (L > 1) {
      uint32_t v[4];
      draw(p, m / 2, 1, gen, ST_GA, v);
      uint32_t x = 1 + below(v[0], L - 1), y = 1 + below(v[1], L - 1);
      lo = x < y ? x : y;
      hi = x < y ? y : x;
    }
    for (uint32_t t = 0; t < L; ++t) {
      int swap = t >= lo && t < hi;
      uint64_t sa = swap ? b : a, sb = swap ? a : b;
      out[oa + t] = genome[sa + t];
      out[ob + t] = genome[sb + t];
      out_amps[2 * (oa + t)] = amps[2 * (sa + t)];
      out_amps[2 * (oa + t) + 1] = amps[2 * (sa + t) + 1];
      out_amps[2 * (ob + t)] = amps[2 * (sb + t)];
      out_amps[2 * (ob + t) + 1] = amps[2 * (sb + t) + 1];
    }
  }
  /* per-gene mutation: a fresh gene, or the angle turned by +-m range/Q */
  for (uint32_t c = 0; c < P; ++c)
    for (uint32_t t = 0; t < L; ++t) {
      uint32_t v[4];
      uint64_t e = (uint64_t)c * L + t;
      draw(p, c, 2 + t, gen, ST_GA, v);
      if (unit(v[0]) < ga_rate) {
        out[e] = (uint8_t)below(v[1], G);
        trig_f32((2.0 * ORC_PI) / (double)ORC_Q, below(v[2], ORC_Q), &out_amps[2 * e],
                 &out_amps[2 * e + 1]);
      } else if (unit(v[3]) < ga_rate) {
        float cs, sn;
        trig_f32(p->mutation_range / (double)ORC_Q, below(v[2], ORC_Q + 1), &cs, &sn);
        if (v[1] & 1u) sn = -sn;
        float R[2][2] = {{cs, -sn}, {sn, cs}};
        float b[2] = {out_amps[2 * e], out_amps[2 * e + 1]};
        for (int r = 0; r < 2; ++r) {
          float acc = 0.0f;
          for (int k = 0; k < 2; ++k) acc = acc + R[r][k] * b[k];
          out_amps[2 * e + r] = acc;
        }
      }
    }
  /* elitism: the best genome of the parent generation, angles included */
  uint32_t bidx;
  oracle_topk(F, cost, P, 1, &bidx);
  memcpy(out, genome + (uint64_t)bidx * L, L);
  memcpy(out_amps, amps + 2 * (uint64_t)bidx * L, 2 * L * sizeof(float));
  free(cum);
  free(parent);
}
