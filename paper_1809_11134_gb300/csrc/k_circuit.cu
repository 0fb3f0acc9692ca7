// k_circuit.cu -- one warp per circuit: measure the encoding into gates
// (Sec. IV-D), compose the circuit unitary in registers (Sec. IV-C), score it
// (Eq. (11)) and scatter the fitness to the segments that built it
// (Sec. IV-E1).
//
// Gate application.  A library gate becomes an "op" byte: ops 0 .. 2n(n-1)-1
// are pair gates (2*pair + 0 = CNOT, 2*pair + 1 = CV or CV^dag), the next 2n
// ops are wire gates (2*n(n-1) + 2w + 0 = H, + 1 = T or T^dag); bit 7 carries
// the sign sigma (-1 for the daggers) and 0xff is the identity.  Every op is a
// compile-time case of one switch, so the row pairs it touches are fixed
// register indices (or one lane-xor shuffle when the target wire is a lane
// bit); the op is warp-uniform, so the switch never diverges.
//
// Two arithmetics:
//  * binary32 (working precision): any operation order, FMA allowed;
//  * binary64 canonical: every nonzero term of the dense product
//    G_t * S (k ascending, complex product (ar br - ai bi, ar bi + ai br),
//    every operation rounded) computed with _rn intrinsics in the same order,
//    so results equal the dense oracle's (terms with a zero coefficient add
//    exact zeros; only signs of zero can differ).  The score sums
//    S[perm[j]][j] with j ascending.
#include "qe_dev.cuh"
#include "qe_host.h"

namespace qe {

enum Kind { kCnot = 0, kCvx = 1, kHad = 2, kTx = 3, kRx = 4, kRy = 5, kRz = 6, kJzz = 7 };

// ------------------------------------------------------------------ arithmetic
template <typename R, bool CANON>
struct Ar;

template <>
struct Ar<float, false> {
  // CV (s=+1) / CV^dag (s=-1) on a register pair (x = bit-0 row, y = bit-1 row)
  static __device__ __forceinline__ void cvx_pair(float &xr, float &xi, float &yr, float &yi,
                                                  float s) {
    const float s1 = xr + yr, s2 = xi + yi, d1 = xr - yr, d2 = xi - yi;
    const float h1 = 0.5f * s1, h2 = 0.5f * s2, hs = 0.5f * s;
    xr = fmaf(-hs, d2, h1);
    xi = fmaf(hs, d1, h2);
    yr = fmaf(hs, d2, h1);
    yi = fmaf(-hs, d1, h2);
  }
  // new value of this lane's row given the partner's: A(m) + B(p) for both rows
  static __device__ __forceinline__ void cvx_lane(float &mr, float &mi, float pr, float pi,
                                                  float s) {
    const float a = mr + pr, b = mi + pi, c = mi - pi, d = mr - pr;
    const float hs = 0.5f * s;
    mr = fmaf(-hs, c, 0.5f * a);
    mi = fmaf(hs, d, 0.5f * b);
  }
  static __device__ __forceinline__ void had_pair(float &xr, float &xi, float &yr, float &yi) {
    const float s1 = xr + yr, s2 = xi + yi, d1 = xr - yr, d2 = xi - yi;
    xr = kH32 * s1;
    xi = kH32 * s2;
    yr = kH32 * d1;
    yi = kH32 * d2;
  }
  static __device__ __forceinline__ void had_lane(float &mr, float &mi, float pr, float pi,
                                                  bool up) {
    mr = kH32 * (up ? pr - mr : mr + pr);
    mi = kH32 * (up ? pi - mi : mi + pi);
  }
  // y <- (h + i s h) y
  static __device__ __forceinline__ void tx(float &yr, float &yi, float s) {
    const float r = yr, i = yi;
    yr = kH32 * fmaf(-s, i, r);
    yi = kH32 * fmaf(s, r, i);
  }
  // Ising rotations (Eqs. (3)-(5)) with c = cos(theta/2), s = sin(theta/2):
  // the new value of row m given the partner row p; up = this row's target bit
  static __device__ __forceinline__ void rx_lane(float &mr, float &mi, float pr, float pi,
                                                 float c, float s) {
    const float r = mr, i = mi;  // c m - i s p
    mr = fmaf(s, pi, c * r);
    mi = fmaf(-s, pr, c * i);
  }
  static __device__ __forceinline__ void ry_lane(float &mr, float &mi, float pr, float pi,
                                                 bool up, float c, float s) {
    const float t = up ? s : -s;  // row 0: c m - s p; row 1: s p + c m
    mr = fmaf(t, pr, c * mr);
    mi = fmaf(t, pi, c * mi);
  }
  // m <- (c - i d s) m, d = +-1 (R_z: d = +1 on target bit 0; J: d = z_i z_j)
  static __device__ __forceinline__ void phase(float &mr, float &mi, float c, float ds) {
    const float r = mr, i = mi;
    mr = fmaf(ds, i, c * r);
    mi = fmaf(-ds, r, c * i);
  }
};

template <>
struct Ar<double, true> {
  // x' = A(x) + B(y), y' = B(x) + A(y) with A(z) = (1+si)/2 z, B(z) = (1-si)/2 z:
  // each half-product is 0.5 * (z.re -+ s z.im) (one rounding: fma with s = +-1
  // is exact up to the final rounding), the row sum adds the two.
  static __device__ __forceinline__ void cvx_pair(double &xr, double &xi, double &yr, double &yi,
                                                  double s) {
    const double a1 = __fma_rn(-s, xi, xr), a2 = __fma_rn(s, xr, xi);
    const double b1 = __fma_rn(s, yi, yr), b2 = __fma_rn(-s, yr, yi);
    const double c1 = __fma_rn(s, xi, xr), c2 = __fma_rn(-s, xr, xi);
    const double d1 = __fma_rn(-s, yi, yr), d2 = __fma_rn(s, yr, yi);
    xr = __dmul_rn(0.5, __dadd_rn(a1, b1));
    xi = __dmul_rn(0.5, __dadd_rn(a2, b2));
    yr = __dmul_rn(0.5, __dadd_rn(c1, d1));
    yi = __dmul_rn(0.5, __dadd_rn(c2, d2));
  }
  static __device__ __forceinline__ void cvx_lane(double &mr, double &mi, double pr, double pi,
                                                  double s) {
    const double a1 = __fma_rn(-s, mi, mr), a2 = __fma_rn(s, mr, mi);
    const double b1 = __fma_rn(s, pi, pr), b2 = __fma_rn(-s, pr, pi);
    mr = __dmul_rn(0.5, __dadd_rn(a1, b1));
    mi = __dmul_rn(0.5, __dadd_rn(a2, b2));
  }
  // x' = h x + h y, y' = h x + (-h) y, each product rounded, then the sum
  static __device__ __forceinline__ void had_pair(double &xr, double &xi, double &yr,
                                                  double &yi) {
    const double hxr = __dmul_rn(kH64, xr), hxi = __dmul_rn(kH64, xi);
    const double hyr = __dmul_rn(kH64, yr), hyi = __dmul_rn(kH64, yi);
    xr = __dadd_rn(hxr, hyr);
    xi = __dadd_rn(hxi, hyi);
    yr = __dsub_rn(hxr, hyr);
    yi = __dsub_rn(hxi, hyi);
  }
  static __device__ __forceinline__ void had_lane(double &mr, double &mi, double pr, double pi,
                                                  bool up) {
    const double hm_r = __dmul_rn(kH64, mr), hm_i = __dmul_rn(kH64, mi);
    const double hp_r = __dmul_rn(kH64, pr), hp_i = __dmul_rn(kH64, pi);
    mr = up ? __dsub_rn(hp_r, hm_r) : __dadd_rn(hm_r, hp_r);
    mi = up ? __dsub_rn(hp_i, hm_i) : __dadd_rn(hm_i, hp_i);
  }
  // y' = (h, s h) y = (h yr - s (h yi), h yi + s (h yr))
  static __device__ __forceinline__ void tx(double &yr, double &yi, double s) {
    const double hr = __dmul_rn(kH64, yr), hi = __dmul_rn(kH64, yi);
    yr = __fma_rn(-s, hi, hr);
    yi = __fma_rn(s, hr, hi);
  }
  // Ising rotations, the dense product's two nonzero terms per row: each
  // complex product (a.re b.re - a.im b.im, a.re b.im + a.im b.re) has one
  // zero coefficient part, so it is one rounded product per component; the
  // row sum adds the two terms (order-free: two addends)
  static __device__ __forceinline__ void rx_lane(double &mr, double &mi, double pr, double pi,
                                                 double c, double s) {
    // c m + (-i s) p = (c mr + s pi, c mi - s pr)
    const double r = mr, i = mi;
    mr = __dadd_rn(__dmul_rn(c, r), __dmul_rn(s, pi));
    mi = __dadd_rn(__dmul_rn(c, i), __dmul_rn(-s, pr));
  }
  static __device__ __forceinline__ void ry_lane(double &mr, double &mi, double pr, double pi,
                                                 bool up, double c, double s) {
    // row 0: c m + (-s) p; row 1: s p + c m
    const double t = up ? s : -s;
    mr = __dadd_rn(__dmul_rn(c, mr), __dmul_rn(t, pr));
    mi = __dadd_rn(__dmul_rn(c, mi), __dmul_rn(t, pi));
  }
  // m <- (c, -d s) m, one term: (c mr - (-d s) mi, c mi + (-d s) mr)
  static __device__ __forceinline__ void phase(double &mr, double &mi, double c, double ds) {
    const double gi = -ds, r = mr, i = mi;
    mr = __dsub_rn(__dmul_rn(c, r), __dmul_rn(gi, i));
    mi = __dadd_rn(__dmul_rn(c, i), __dmul_rn(gi, r));
  }
};

// ------------------------------------------------------------------ one gate
template <int NQ, typename R, bool CANON, int KIND, int CW, int TW, int WB = 0>
__device__ __forceinline__ void apply_gate(R (&re)[Lay<NQ, WB>::ROWS], R (&im)[Lay<NQ, WB>::ROWS],
                                           int lane, R s) {
  using Ly = Lay<NQ, WB>;
  using A = Ar<R, CANON>;
  constexpr int tb = NQ - 1 - TW;                 // target row bit
  constexpr int cb = CW < 0 ? -1 : NQ - 1 - CW;   // control row bit
  constexpr bool T_REG = tb < Ly::RBR;
  constexpr bool C_REG = cb >= 0 && cb < Ly::RBR;
  constexpr bool C_LANE = cb >= Ly::RBR;
  bool cl = true;
  if constexpr (C_LANE) cl = (lane >> (Ly::CB + cb - Ly::RBR)) & 1;

  if constexpr (KIND == kTx) {
    // diagonal: rows whose target bit is 1 take the phase
    if constexpr (T_REG) {
#pragma unroll
      for (int r = 0; r < Ly::ROWS; ++r)
        if ((r >> tb) & 1) A::tx(re[r], im[r], s);
    } else {
      const bool up = (lane >> (Ly::CB + tb - Ly::RBR)) & 1;
#pragma unroll
      for (int r = 0; r < Ly::ROWS; ++r) {
        R a = re[r], b = im[r];
        A::tx(a, b, s);
        re[r] = up ? a : re[r];
        im[r] = up ? b : im[r];
      }
    }
  } else if constexpr (T_REG) {
#pragma unroll
    for (int r0 = 0; r0 < Ly::ROWS; ++r0) {
      if ((r0 >> tb) & 1) continue;
      if (C_REG && !((r0 >> cb) & 1)) continue;
      const int r1 = r0 | (1 << tb);
      R xr = re[r0], xi = im[r0], yr = re[r1], yi = im[r1];
      if constexpr (KIND == kCnot) {
        R t0 = xr, t1 = xi;
        xr = yr;
        xi = yi;
        yr = t0;
        yi = t1;
      } else if constexpr (KIND == kCvx) {
        A::cvx_pair(xr, xi, yr, yi, s);
      } else {
        A::had_pair(xr, xi, yr, yi);
      }
      if constexpr (C_LANE) {
        re[r0] = cl ? xr : re[r0];
        im[r0] = cl ? xi : im[r0];
        re[r1] = cl ? yr : re[r1];
        im[r1] = cl ? yi : im[r1];
      } else {
        re[r0] = xr;
        im[r0] = xi;
        re[r1] = yr;
        im[r1] = yi;
      }
    }
  } else {
    constexpr int tl = Ly::CB + tb - Ly::RBR;  // lane bit of the target
    const bool up = (lane >> tl) & 1;
#pragma unroll
    for (int r = 0; r < Ly::ROWS; ++r) {
      if (C_REG && !((r >> cb) & 1)) continue;
      const R pr = __shfl_xor_sync(kFull, re[r], 1 << tl);
      const R pi = __shfl_xor_sync(kFull, im[r], 1 << tl);
      R mr = re[r], mi = im[r];
      if constexpr (KIND == kCnot) {
        mr = pr;
        mi = pi;
      } else if constexpr (KIND == kCvx) {
        A::cvx_lane(mr, mi, pr, pi, s);
      } else {
        A::had_lane(mr, mi, pr, pi, up);
      }
      re[r] = cl ? mr : re[r];
      im[r] = cl ? mi : im[r];
    }
  }
}

// Ising gate of kind R_x / R_y / R_z on wire TW, or the interaction template on
// wires (WI, TW); c = cos(theta/2), s = sin(theta/2) of the slot
template <int NQ, typename R, bool CANON, int KIND, int WI, int TW, int WB = 0>
__device__ __forceinline__ void apply_ising(R (&re)[Lay<NQ, WB>::ROWS], R (&im)[Lay<NQ, WB>::ROWS],
                                            int lane, R c, R s) {
  using Ly = Lay<NQ, WB>;
  using A = Ar<R, CANON>;
  constexpr int tb = NQ - 1 - TW;  // row bit of wire TW
  constexpr bool T_REG = tb < Ly::RBR;
  if constexpr (KIND == kRz || KIND == kJzz) {
    // diagonal: row i takes (c - i d s), d = +1 where the wire's bit is 0 (R_z),
    // d = z_i z_j (J)
    constexpr int ib = KIND == kJzz ? NQ - 1 - WI : 0;
    constexpr bool I_REG = ib < Ly::RBR;
    int lt = 0, li = 0;
    if constexpr (!T_REG) lt = (lane >> (Ly::CB + tb - Ly::RBR)) & 1;
    if constexpr (KIND == kJzz && !I_REG) li = (lane >> (Ly::CB + ib - Ly::RBR)) & 1;
#pragma unroll
    for (int r = 0; r < Ly::ROWS; ++r) {
      const int bt = T_REG ? ((r >> tb) & 1) : lt;
      int odd = bt;
      if constexpr (KIND == kJzz) odd ^= I_REG ? ((r >> ib) & 1) : li;
      A::phase(re[r], im[r], c, odd ? -s : s);
    }
  } else if constexpr (T_REG) {
#pragma unroll
    for (int r0 = 0; r0 < Ly::ROWS; ++r0) {
      if ((r0 >> tb) & 1) continue;
      const int r1 = r0 | (1 << tb);
      R xr = re[r0], xi = im[r0], yr = re[r1], yi = im[r1];
      if constexpr (KIND == kRx) {
        A::rx_lane(re[r0], im[r0], yr, yi, c, s);
        A::rx_lane(re[r1], im[r1], xr, xi, c, s);
      } else {
        A::ry_lane(re[r0], im[r0], yr, yi, false, c, s);
        A::ry_lane(re[r1], im[r1], xr, xi, true, c, s);
      }
    }
  } else {
    constexpr int tl = Ly::CB + tb - Ly::RBR;  // lane bit of the target
    const bool up = (lane >> tl) & 1;
#pragma unroll
    for (int r = 0; r < Ly::ROWS; ++r) {
      const R pr = __shfl_xor_sync(kFull, re[r], 1 << tl);
      const R pi = __shfl_xor_sync(kFull, im[r], 1 << tl);
      if constexpr (KIND == kRx) A::rx_lane(re[r], im[r], pr, pi, c, s);
      else A::ry_lane(re[r], im[r], pr, pi, up, c, s);
    }
  }
}

// wires of interaction template q (pairs i < j, lexicographic)
constexpr int jpair_i(int nq, int q) {
  int i = 0;
  while (i < nq && q >= nq - 1 - i) {
    q -= nq - 1 - i;
    ++i;
  }
  return i;
}
constexpr int jpair_j(int nq, int q) {
  int i = 0;
  while (i < nq && q >= nq - 1 - i) {
    q -= nq - 1 - i;
    ++i;
  }
  return i + 1 + q;
}

constexpr int pair_ctrl(int nq, int pr) { return nq > 1 ? pr / (nq - 1) : 0; }
constexpr int pair_tgt(int nq, int pr) {
  return nq > 1 ? ((pr % (nq - 1)) >= pair_ctrl(nq, pr) ? (pr % (nq - 1)) + 1 : (pr % (nq - 1)))
                : 0;
}

template <int NQ, typename R, bool CANON, int OP, int WB = 0>
__device__ __forceinline__ void apply_op(R (&re)[Lay<NQ, WB>::ROWS], R (&im)[Lay<NQ, WB>::ROWS],
                                         int lane, R s, R ic, R is) {
  constexpr int NP = NQ * (NQ - 1);
  if constexpr (OP >= kOpIsingJ) {
    constexpr int q = OP - kOpIsingJ;
    apply_ising<NQ, R, CANON, kJzz, jpair_i(NQ, q), jpair_j(NQ, q), WB>(re, im, lane, ic, is);
  } else if constexpr (OP >= kOpIsingRot) {
    constexpr int w = (OP - kOpIsingRot) / 3, k = (OP - kOpIsingRot) % 3;
    apply_ising<NQ, R, CANON, k == 0 ? kRx : (k == 1 ? kRy : kRz), 0, w, WB>(re, im, lane, ic,
                                                                             is);
  } else if constexpr (OP < 2 * NP) {
    constexpr int pr = OP >> 1;
    apply_gate<NQ, R, CANON, (OP & 1) ? kCvx : kCnot, pair_ctrl(NQ, pr), pair_tgt(NQ, pr), WB>(
        re, im, lane, s);
  } else {
    constexpr int w = (OP - 2 * NP) >> 1;
    apply_gate<NQ, R, CANON, (OP & 1) ? kTx : kHad, -1, w, WB>(re, im, lane, s);
  }
}

// a kernel compiles either the discrete ops or the Ising ops (ISING)
#define QE_CASE(k)                                                      \
  case k:                                                               \
    if constexpr (!ISING && (k) < 2 * NQ * NQ)                          \
      apply_op<NQ, R, CANON, (k), WB>(re, im, lane, s, ic, is);         \
    break;
// Ising rotations exist for wires < NQ, templates for pairs < NQ (NQ - 1) / 2
#define QE_ICASE(k)                                                     \
  case kOpIsingRot + (k):                                               \
    if constexpr (ISING && (k) < 3 * NQ)                                \
      apply_op<NQ, R, CANON, kOpIsingRot + (k), WB>(re, im, lane, s, ic, is); \
    break;
#define QE_JCASE(k)                                                     \
  case kOpIsingJ + (k):                                                 \
    if constexpr (ISING && (k) < NQ * (NQ - 1) / 2)                     \
      apply_op<NQ, R, CANON, kOpIsingJ + (k), WB>(re, im, lane, s, ic, is); \
    break;

template <int NQ, typename R, bool CANON, bool ISING, int WB = 0>
__device__ __forceinline__ void dispatch(int op, R (&re)[Lay<NQ, WB>::ROWS],
                                         R (&im)[Lay<NQ, WB>::ROWS], int lane, R s, R ic, R is) {
  switch (op) {
    QE_CASE(0) QE_CASE(1) QE_CASE(2) QE_CASE(3) QE_CASE(4) QE_CASE(5) QE_CASE(6) QE_CASE(7)
    QE_CASE(8) QE_CASE(9) QE_CASE(10) QE_CASE(11) QE_CASE(12) QE_CASE(13) QE_CASE(14)
    QE_CASE(15) QE_CASE(16) QE_CASE(17) QE_CASE(18) QE_CASE(19) QE_CASE(20) QE_CASE(21)
    QE_CASE(22) QE_CASE(23) QE_CASE(24) QE_CASE(25) QE_CASE(26) QE_CASE(27) QE_CASE(28)
    QE_CASE(29) QE_CASE(30) QE_CASE(31) QE_CASE(32) QE_CASE(33) QE_CASE(34) QE_CASE(35)
    QE_CASE(36) QE_CASE(37) QE_CASE(38) QE_CASE(39) QE_CASE(40) QE_CASE(41) QE_CASE(42)
    QE_CASE(43) QE_CASE(44) QE_CASE(45) QE_CASE(46) QE_CASE(47) QE_CASE(48) QE_CASE(49)
    QE_ICASE(0) QE_ICASE(1) QE_ICASE(2) QE_ICASE(3) QE_ICASE(4) QE_ICASE(5) QE_ICASE(6)
    QE_ICASE(7) QE_ICASE(8) QE_ICASE(9) QE_ICASE(10) QE_ICASE(11) QE_ICASE(12) QE_ICASE(13)
    QE_ICASE(14)
    QE_JCASE(0) QE_JCASE(1) QE_JCASE(2) QE_JCASE(3) QE_JCASE(4) QE_JCASE(5) QE_JCASE(6)
    QE_JCASE(7) QE_JCASE(8) QE_JCASE(9)
    default:
      break;
  }
}
#undef QE_CASE
#undef QE_ICASE
#undef QE_JCASE

// ------------------------------------------------------------------ 5 qubits: target at bit 0
// With n = 5 a lane holds a whole column (32 rows, all in registers).  A switch
// with one case per (kind, control, target) would be ~50 cases of unrolled
// register updates, more code than the instruction cache holds.  Instead the
// kernel keeps a map from wires to physical row bits: before each gate the
// target wire's bit is exchanged with bit 0 (4 static cases of register moves),
// then the gate acts on bit 0 with its control at any other bit (CNOT, CV:
// 4 cases each; H, T: 1 each).  Binary32 translates rows through the map only
// at the end.  Binary64 uses the same gate code: every row of a one- or
// two-wire gate has two nonzero terms, whose sum does not depend on their
// order, so each row gets the dense product's value wherever it sits; the map
// is brought back to the identity before the score, which sums in the
// oracle's row order.
template <typename R>
__device__ __forceinline__ void xchg(R &a, R &b) {
  const R t = a;
  a = b;
  b = t;
}

// exchange physical row bits 0 and B of the column
template <int B, typename R>
__device__ __forceinline__ void swap_bit0(R (&re)[32], R (&im)[32]) {
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    if ((r & 1) && !((r >> B) & 1)) {
      const int q = (r ^ 1) | (1 << B);
      xchg(re[r], re[q]);
      xchg(im[r], im[q]);
    }
  }
}

template <typename R>
__device__ __forceinline__ void swap_bit0_dyn(int b, R (&re)[32], R (&im)[32]) {
  switch (b) {
    case 1: swap_bit0<1>(re, im); break;
    case 2: swap_bit0<2>(re, im); break;
    case 3: swap_bit0<3>(re, im); break;
    default: swap_bit0<4>(re, im); break;
  }
}

// gate of kind K on target bit 0, control at bit CB (-1: none); for the
// interaction template CB is the bit of its other wire.  ic/is: cos/sin of
// theta/2 (Ising kinds)
template <int K, int CB, typename R, bool CANON>
__device__ __forceinline__ void gate_bit0(R (&re)[32], R (&im)[32], R s, R ic, R is) {
  using A = Ar<R, CANON>;
  if constexpr (K == kRz || K == kJzz) {
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      int odd = r & 1;
      if constexpr (K == kJzz) odd ^= (r >> CB) & 1;
      A::phase(re[r], im[r], ic, odd ? -is : is);
    }
    return;
  }
#pragma unroll
  for (int r0 = 0; r0 < 32; r0 += 2) {
    if (K != kRx && K != kRy && CB >= 0 && !((r0 >> CB) & 1)) continue;
    const int r1 = r0 | 1;
    if constexpr (K == kRx || K == kRy) {
      const R xr = re[r0], xi = im[r0], yr = re[r1], yi = im[r1];
      if constexpr (K == kRx) {
        A::rx_lane(re[r0], im[r0], yr, yi, ic, is);
        A::rx_lane(re[r1], im[r1], xr, xi, ic, is);
      } else {
        A::ry_lane(re[r0], im[r0], yr, yi, false, ic, is);
        A::ry_lane(re[r1], im[r1], xr, xi, true, ic, is);
      }
    } else if constexpr (K == kCnot) {
      xchg(re[r0], re[r1]);
      xchg(im[r0], im[r1]);
    } else if constexpr (K == kCvx) {
      A::cvx_pair(re[r0], im[r0], re[r1], im[r1], s);
    } else if constexpr (K == kHad) {
      A::had_pair(re[r0], im[r0], re[r1], im[r1]);
    } else {
      A::tx(re[r1], im[r1], s);
    }
  }
}

// the wire at physical bit b moves to bit 0 and the wire at bit 0 to bit b
__device__ __forceinline__ void remap5(int b, uint32_t &pos, uint32_t &inv) {
  const int w0 = inv & 7, wb = (inv >> (3 * b)) & 7;
  pos = (pos & ~(7u << (3 * w0))) | ((uint32_t)b << (3 * w0));
  pos &= ~(7u << (3 * wb));
  inv = (inv & ~(7u << (3 * b))) | ((uint32_t)w0 << (3 * b));
  inv = (inv & ~7u) | (uint32_t)wb;
}

// apply one op: wire bits in pos (3 bits per wire), wire at each bit in inv
template <bool ISING, typename R, bool CANON>
__device__ __forceinline__ void apply5(int op, uint32_t &pos, uint32_t &inv, R (&re)[32],
                                       R (&im)[32], R ic, R is) {
  constexpr int NP2 = 2 * 5 * 4;
  const int o = op & 0x7f;
  const R s = (op & kOpNeg) ? R(-1) : R(1);
  int kind, tw, cw = -1;
  if (ISING && o >= kOpIsingJ) {
    // template on wires (i, j): j goes to bit 0, i is the "control" bit
    int q = o - kOpIsingJ, i = 0;
    while (q >= 4 - i) {
      q -= 4 - i;
      ++i;
    }
    cw = i;
    tw = i + 1 + q;
    kind = kJzz;
  } else if (ISING) {
    tw = (o - kOpIsingRot) / 3;
    kind = kRx + (o - kOpIsingRot) % 3;
  } else if (o < NP2) {
    const int pr = o >> 1;
    cw = pr >> 2;
    const int tt = pr & 3;
    tw = tt >= cw ? tt + 1 : tt;
    kind = (o & 1) ? kCvx : kCnot;
  } else {
    tw = (o - NP2) >> 1;
    kind = (o & 1) ? kTx : kHad;
  }
  const int b = (pos >> (3 * tw)) & 7;
  if (b != 0) {
    swap_bit0_dyn(b, re, im);
    remap5(b, pos, inv);
  }
  const int cb = cw < 0 ? 0 : (int)((pos >> (3 * cw)) & 7);
  if constexpr (ISING) {
    switch (kind * 5 + cb) {
      case kRx * 5: gate_bit0<kRx, -1, R, CANON>(re, im, s, ic, is); break;
      case kRy * 5: gate_bit0<kRy, -1, R, CANON>(re, im, s, ic, is); break;
      case kRz * 5: gate_bit0<kRz, -1, R, CANON>(re, im, s, ic, is); break;
      case kJzz * 5 + 1: gate_bit0<kJzz, 1, R, CANON>(re, im, s, ic, is); break;
      case kJzz * 5 + 2: gate_bit0<kJzz, 2, R, CANON>(re, im, s, ic, is); break;
      case kJzz * 5 + 3: gate_bit0<kJzz, 3, R, CANON>(re, im, s, ic, is); break;
      default: gate_bit0<kJzz, 4, R, CANON>(re, im, s, ic, is); break;
    }
    return;
  }
  switch (kind * 5 + cb) {
    case kCnot * 5 + 1: gate_bit0<kCnot, 1, R, CANON>(re, im, s, ic, is); break;
    case kCnot * 5 + 2: gate_bit0<kCnot, 2, R, CANON>(re, im, s, ic, is); break;
    case kCnot * 5 + 3: gate_bit0<kCnot, 3, R, CANON>(re, im, s, ic, is); break;
    case kCnot * 5 + 4: gate_bit0<kCnot, 4, R, CANON>(re, im, s, ic, is); break;
    case kCvx * 5 + 1: gate_bit0<kCvx, 1, R, CANON>(re, im, s, ic, is); break;
    case kCvx * 5 + 2: gate_bit0<kCvx, 2, R, CANON>(re, im, s, ic, is); break;
    case kCvx * 5 + 3: gate_bit0<kCvx, 3, R, CANON>(re, im, s, ic, is); break;
    case kCvx * 5 + 4: gate_bit0<kCvx, 4, R, CANON>(re, im, s, ic, is); break;
    case kHad * 5: gate_bit0<kHad, -1, R, CANON>(re, im, s, ic, is); break;
    default: gate_bit0<kTx, -1, R, CANON>(re, im, s, ic, is); break;
  }
}

// bring the map back to the identity (wire w at physical bit 4 - w) by
// exchanges of bit 0 with another bit: each exchange sends the wire at bit 0
// home, or, when it is home, brings a misplaced wire to bit 0 (at most 8)
template <typename R>
__device__ __forceinline__ void restore5(uint32_t &pos, uint32_t &inv, R (&re)[32],
                                         R (&im)[32]) {
  for (int it = 0; it < 8; ++it) {
    const int w0 = inv & 7;
    int b = 4 - w0;  // the home bit of the wire at bit 0
    if (b == 0) {
      for (int c = 4; c >= 1; --c)
        if ((int)((inv >> (3 * c)) & 7) != 4 - c) b = c;
      if (b == 0) return;  // every wire is home
    }
    swap_bit0_dyn(b, re, im);
    remap5(b, pos, inv);
  }
}

// physical row of logical row x under the map
__device__ __forceinline__ int phys_row5(int x, uint32_t pos) {
  int p = 0;
#pragma unroll
  for (int w = 0; w < 5; ++w) p |= ((x >> (4 - w)) & 1) << ((pos >> (3 * w)) & 7);
  return p;
}

// real operations of one op on an N x N state (gate-count work model)
__device__ __forceinline__ uint32_t op_work(const DevProblem &p, int op) {
  if (op == kOpIdentity) return 0;
  const int o = op & 0x7f;
  const uint32_t NN = p.N * p.N;
  if (o >= kOpIsingRot) return 6 * NN;  // R_x/R_y/R_z/J: six real ops per amplitude
  const int np2 = 2 * (int)(p.n * (p.n - 1));
  if (o < np2) return (o & 1) ? 4 * NN : 0;  // CV: 4N^2, CNOT: 0
  return (o & 1) ? 2 * NN : 4 * NN;          // T: 2N^2, H: 4N^2
}

__device__ __forceinline__ void prefetch_l2(const void *ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// If individual i mutates in this generation, list it for the update, which
// will walk all of its R*L segments (their 64-B records and fitness pairs);
// when the update's lines fit in L2 (p.prefetch), prefetch them into L2 from
// the circuit kernel so that the update, which is latency-bound, finds them
// there (with more lines than L2 holds they would be evicted before use).
__device__ __forceinline__ void prefetch_mutated(const DevProblem &p, uint32_t i, uint32_t gen,
                                                 int lane) {
  const uint4 v = draw(p, i, 0, gen, kStMutDecide);
  if (lane == 0 && i == 0) p.mut_cnt[(gen + 1u) & 1u] = 0u;  // the next generation's list
  if (!((unsigned long long)v.x < p.mut_T)) return;
  // list the individual for the update's mutation role (any order: the
  // individuals' segments are disjoint)
  if (lane == 0) p.mut_list[(size_t)(gen & 1u) * p.P + atomicAdd(p.mut_cnt + (gen & 1u), 1u)] = i;
  if (!p.prefetch) return;
  const uint32_t RL = p.R * p.L;
  for (uint32_t x = lane; x < RL; x += 32) {
    const uint32_t r = x / p.L, t = x - r * p.L;
    const uint32_t seg = r * p.LP + i * p.L + t;
    prefetch_l2(cur_of(p, seg));
    if ((t & 7) == 0) prefetch_l2(key_of(p, seg));
  }
}

// ------------------------------------------------------------------ sampling
// Sec. IV-A1: the qutrit measured K > 1 times, the most frequent outcome kept
// (the lowest on a tie).  Shot j compares word j mod 4 of the Philox draw
// (c, t + 64 floor(j / 4), gen, stream 3) with the same binary32 CDF as one
// measurement.  The circuit kernel never runs it (its register budget is
// tight): searches with K > 1 are measured by k_presample ahead of it.
__device__ __forceinline__ uint32_t measure_shots(const DevProblem &p, uint32_t c, uint32_t t,
                                               uint32_t gen, float p0, float p01, float s) {
  uint32_t n0 = 0, n1 = 0, n2 = 0;
  const uint32_t K = p.shots;
  for (uint32_t j = 0; j < K; j += 4) {
    const uint4 w = draw(p, c, t + 64u * (j >> 2), gen, kStShot);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      if (j + q < K) {
        const float x = __fmul_rn(unit32(ws[q]), s);
        if (x < p0) ++n0;
        else if (x < p01) ++n1;
        else ++n2;
      }
    }
  }
  uint32_t k = 0, best = n0;
  if (n1 > best) {
    k = 1;
    best = n1;
  }
  if (n2 > best) k = 2;
  return k;
}

// Sec. IV-D: draw whichIndividual and whichRotationOrInteraction, form the
// segment index (Eq. (10)), measure the segment's qutrit (and qubit) in binary32
// (SHOTS: K times when the search asks for it).
template <bool ISING, bool SHOTS = false>
__device__ __forceinline__ void sample_slot(const DevProblem &p, uint32_t c, uint32_t t,
                                            uint32_t gen, uint32_t &g_out, uint32_t &seg_out,
                                            float2 &amp_out) {
  const uint4 u = draw(p, c, t, gen, kStSample);
  const uint32_t i = below(u.x, p.P), r = below(u.y, p.R);
  const uint32_t seg = r * p.LP + i * p.L + t;
  const float4 a = __ldg(cur_of(p, seg));
  const float4 b = __ldg(cur_of(p, seg) + 1);
  // the update reads this segment's best record next: bring it into L2 now
  if (p.prefetch) prefetch_l2(best_of(p, seg));
  const float p0 = __fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y));
  const float p1 = __fadd_rn(__fmul_rn(a.z, a.z), __fmul_rn(a.w, a.w));
  const float p2 = __fadd_rn(__fmul_rn(b.x, b.x), __fmul_rn(b.y, b.y));
  const float p01 = __fadd_rn(p0, p1);
  const float s = __fadd_rn(p01, p2);
  uint32_t k;
  if (SHOTS && p.shots > 1) {
    k = measure_shots(p, c, t, gen, p0, p01, s);
  } else {
    const float x = __fmul_rn(unit32(u.z), s);
    k = (x < p0) ? 0u : ((x < p01) ? 1u : 2u);
  }
  uint32_t g = p.base + 3u * r + k;
  if constexpr (ISING) {
    if (r >= p.n) g = 3u * p.n + (r - p.n);  // the interaction template of that pair
    amp_out = make_float2(b.z, b.w);         // the slot's angle; the qubit is not measured
  } else if (p.measure_qubit) {
    const float B0 = __fmul_rn(b.z, b.z), B1 = __fmul_rn(b.w, b.w);
    const float y = __fmul_rn(unit32(u.w), __fadd_rn(B0, B1));
    if (y < B0) g = 0;
  }
  g_out = g;
  seg_out = seg;
}

// cos(theta/2), sin(theta/2) of a slot's amplitudes (b0, b1) = (cos theta,
// sin theta), theta in [0, 2 pi): sgn(b1) sqrt((1 + b0)/2), sqrt((1 - b0)/2);
// binary64 with every operation rounded (so it equals the oracle's), binary32
// otherwise
__device__ __forceinline__ void half_angle(float b0, float b1, double &c, double &s) {
  double a = __dmul_rn(__dadd_rn(1.0, (double)b0), 0.5);
  double b = __dmul_rn(__dsub_rn(1.0, (double)b0), 0.5);
  if (a < 0.0) a = 0.0;
  if (b < 0.0) b = 0.0;
  c = __dsqrt_rn(a);
  if (b1 < 0.f) c = -c;
  s = __dsqrt_rn(b);
}
__device__ __forceinline__ void half_angle(float b0, float b1, float &c, float &s) {
  const float a = fmaxf(0.f, (1.f + b0) * 0.5f), b = fmaxf(0.f, (1.f - b0) * 0.5f);
  c = sqrtf(a);
  if (b1 < 0.f) c = -c;
  s = sqrtf(b);
}

// ------------------------------------------------------------------ one circuit
struct CircuitOut {
  double F;       // fitness (binary64 for CANON; widened binary32 otherwise)
  uint32_t cost;  // non-identity gates
  uint32_t work;  // useful real operations
  bool bad;       // an op byte was invalid
};

// Eq. (11) in binary32 from every lane's share (vr, vi) of the trace (or, for
// the probability overlap, of its row's amplitude), minus the cost penalty pen
__device__ __forceinline__ double fitness32(const DevProblem &p, float vr, float vi, double pen,
                                            int N) {
  float a, b;
  if (p.fit_kind == 1) {
    a = vr * vr + vi * vi;
    b = 0.f;
  } else {
    a = vr;
    b = vi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    b += __shfl_xor_sync(kFull, b, o);
  }
  const float size = (float)N, inv = 1.f / (float)N;
  float d;
  if (p.fit_kind == 1) {
    d = (size - a) * inv;
  } else {
    d = (size - sqrtf(a * a + b * b)) * inv;
  }
  d = fmaxf(d, 0.f);
  const float f = 1.f - sqrtf(d);
  return pen == 0.0 ? (double)f : (double)(float)((double)f - pen);
}

// ------------------------------------------------------------------ 5 qubits in shared memory
// Binary32 composition of a 5-qubit circuit with the unitary in shared memory:
// lane j owns column j (32 rows of 8 B, 256 B apart, so a warp's access to one
// row is 256 contiguous bytes), and rows are addressed through a map from
// logical to physical rows that is linear over GF(2): physical row A x, with
// the columns a_k = A e_k of A packed 5 bits each.  A gate on logical target
// bit t (control c) pairs logical rows x and x ^ e_t, i.e. physical rows p and
// p ^ a_t; the rows of a gate are enumerated in Gray-code order over the
// columns of the free bits, one XOR per row.  A CNOT moves no data: it maps
// logical row x to x ^ x_c e_t, which is the column update a_c ^= a_t.  Every
// pair gets the same binary32 operations as in the register kernels.
struct Op5Table {
  uint32_t v[40 + 10];
};
// op byte -> kind | target bit << 2 | control bit << 5 (7 = none) | free
// bits (ascending, 3 bits each) << 8: pair ops 0..39 (2 * pair + {CNOT, CV})
// and wire ops 40..49 (H, T), wire w at bit 4 - w
constexpr uint32_t op5_fields(int o) {
  int kind = 0, tw = 0, cw = -1;
  if (o < 40) {
    const int pr = o >> 1, tt = pr & 3;
    cw = pr >> 2;
    tw = tt >= cw ? tt + 1 : tt;
    kind = (o & 1) ? kCvx : kCnot;
  } else {
    tw = (o - 40) >> 1;
    kind = (o & 1) ? kTx : kHad;
  }
  const int tb = 4 - tw, cb = cw < 0 ? 7 : 4 - cw;
  uint32_t v = (uint32_t)kind | ((uint32_t)tb << 2) | ((uint32_t)cb << 5);
  int k = 0;
  for (int b = 0; b < 5; ++b)
    if (b != tb && b != cb) v |= (uint32_t)b << (8 + 3 * k++);
  return v;
}
constexpr Op5Table make_op5() {
  Op5Table t{};
  for (int o = 0; o < 50; ++o) t.v[o] = op5_fields(o);
  return t;
}
__constant__ Op5Table c_op5 = make_op5();

constexpr uint32_t kMap5Identity = 1u | (2u << 5) | (4u << 10) | (8u << 15) | (16u << 20);

__device__ __forceinline__ uint32_t col5(uint32_t A, uint32_t k) { return (A >> (5 * k)) & 31u; }

// physical row of logical row x
__device__ __forceinline__ uint32_t phys5(uint32_t A, uint32_t x) {
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) r ^= ((x >> k) & 1u) ? col5(A, k) : 0u;
  return r;
}

constexpr int ctz_c(int v) {
  int n = 0;
  while (!(v & 1)) {
    v >>= 1;
    ++n;
  }
  return n;
}

// the free-bit columns g[0..M) and the Gray-code order of 2^M rows from q:
// row i of the gate is q ^ (XOR of g[b] over the bits b of gray(i))
template <int M>
__device__ __forceinline__ void gray_rows(uint32_t q, const uint32_t (&g)[4], uint32_t (&rows)[1 << M]) {
#pragma unroll
  for (int i = 0; i < (1 << M); ++i) {
    rows[i] = q;
    if (i + 1 < (1 << M)) q ^= g[ctz_c(i + 1)];
  }
}

template <int KIND, int M>
__device__ __forceinline__ void gate5_smem(float2 *col, uint32_t q, uint32_t at,
                                           const uint32_t (&g)[4], float s) {
  using A = Ar<float, false>;
  uint32_t rows[1 << M];
  gray_rows<M>(q, g, rows);
  // four pairs (or rows) per batch: every load of a batch before its stores
#pragma unroll
  for (int b = 0; b < (1 << M); b += 4) {
    if constexpr (KIND == kTx) {
      float2 y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = col[rows[b + u] << 5];
#pragma unroll
      for (int u = 0; u < 4; ++u) A::tx(y[u].x, y[u].y, s);
#pragma unroll
      for (int u = 0; u < 4; ++u) col[rows[b + u] << 5] = y[u];
    } else {
      float2 x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = col[rows[b + u] << 5];
        y[u] = col[(rows[b + u] ^ at) << 5];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if constexpr (KIND == kCvx) A::cvx_pair(x[u].x, x[u].y, y[u].x, y[u].y, s);
        else A::had_pair(x[u].x, x[u].y, y[u].x, y[u].y);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        col[rows[b + u] << 5] = x[u];
        col[(rows[b + u] ^ at) << 5] = y[u];
      }
    }
  }
}

// the whole circuit: gates from the op bytes (slots t < L, ops0 for t < 32 and
// ops1 above, by lane t & 31), then this lane's share of the score and, if
// S_out is given, the unitary; blocks of 128 threads (four circuits)
template <bool DENSE_OK>
__device__ __forceinline__ CircuitOut compose5_smem(const DevProblem &p, int lane, uint32_t ops0,
                                                    uint32_t ops1, float *S_out) {
  __shared__ float2 s_state[4][32 * 32];
  float2 *col = &s_state[(threadIdx.x >> 5) & 3][lane];
  const uint32_t cost = __reduce_add_sync(kFull, (ops0 != kOpIdentity) + (ops1 != kOpIdentity));
  const uint32_t work = __reduce_add_sync(kFull, op_work(p, (int)ops0) + op_work(p, (int)ops1));
#pragma unroll
  for (int r = 0; r < 32; ++r) col[r << 5] = make_float2(r == lane ? 1.f : 0.f, 0.f);
  uint32_t Amap = kMap5Identity;
  const uint32_t L = p.L;
  for (uint32_t t = 0; t < L; ++t) {
    const uint32_t src = t < 32 ? ops0 : ops1;
    const int op = __shfl_sync(kFull, (int)src, (int)(t & 31));
    if (op == kOpIdentity) continue;
    const uint32_t d = c_op5.v[op & 0x7f];
    const float s = (op & kOpNeg) ? -1.f : 1.f;
    const uint32_t kind = d & 3u, tb = (d >> 2) & 7u, cb = (d >> 5) & 7u;
    const uint32_t at = col5(Amap, tb);
    if (kind == kCnot) {
      Amap ^= at << (5 * cb);
      continue;
    }
    const uint32_t g[4] = {col5(Amap, (d >> 8) & 7u), col5(Amap, (d >> 11) & 7u),
                           col5(Amap, (d >> 14) & 7u), col5(Amap, (d >> 17) & 7u)};
    if (kind == kCvx) gate5_smem<kCvx, 3>(col, col5(Amap, cb), at, g, s);
    else if (kind == kHad) gate5_smem<kHad, 4>(col, 0u, at, g, s);
    else gate5_smem<kTx, 4>(col, at, at, g, s);
  }
  CircuitOut out;
  out.cost = cost;
  out.work = work + 2u * 32u;
  out.bad = false;
  const int j = lane;
  if (S_out) {
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const float2 v = col[phys5(Amap, (uint32_t)i) << 5];
      S_out[2 * (i * 32 + j)] = v.x;
      S_out[2 * (i * 32 + j) + 1] = v.y;
    }
  }
  float vr = 0.f, vi = 0.f;
  const bool dense = DENSE_OK && p.dense != 0;
  if (!dense) {
    const float2 v = col[phys5(Amap, p.perm[j]) << 5];
    vr = v.x;
    vi = v.y;
  } else {
    // (S^dag T)_jj = sum_i conj(S_ij) T_ij, rows in Gray-code order
    out.work += 8u * 32u * 32u - 2u * 32u;
    uint32_t x = 0;
    for (int i = 0; i < 32; ++i) {
      const float2 v = col[phys5(Amap, x) << 5];
      const float2 tt = __ldg(p.tgt32 + x * 32 + j);
      vr = fmaf(v.x, tt.x, fmaf(v.y, tt.y, vr));
      vi = fmaf(v.x, tt.y, fmaf(-v.y, tt.x, vi));
      x ^= 1u << __ffs(i + 1) - 1;
    }
  }
  const double pen =
      p.cost_weight == 0.0 ? 0.0 : __dmul_rn(p.cost_weight, __ddiv_rn((double)cost, (double)p.L));
  out.F = fitness32(p, vr, vi, pen, 32);
  return out;
}

// 5-qubit binary32 composition on the Ising library (Sec. III: R_x, R_y, R_z
// per wire, the interaction templates J_ij per pair) in shared memory, one
// column per lane as above; the library has no CNOT, so rows are not mapped.
// Of the 25 ops, the diagonal ones (R_z and every J) are deferred: a diagonal
// factor D[p] per row, shared by the warp's 32 columns, accumulates their
// phases (lane p updates D[p]: no row of S is touched), and the next R_x or
// R_y, which reads every row anyway, multiplies each row by its D[p] as it
// loads it and then resets D to 1.  A diagonal op thus moves 512 B of shared
// memory instead of the whole 8 KB column set twice.  Binary32 only: the
// phases of consecutive diagonal ops are multiplied together before they
// reach S, which changes the rounding (the binary64 kernels, which match the
// oracle bit for bit, apply every gate in order).
template <bool DENSE_OK>
__device__ __forceinline__ CircuitOut compose5_smem_ising(const DevProblem &p, int lane,
                                                          uint32_t ops0, uint32_t ops1,
                                                          float *S_out, float ic0, float is0,
                                                          float ic1, float is1) {
  using A = Ar<float, false>;
  __shared__ float2 s_state[4][32 * 32];
  __shared__ float2 s_diag[4][32];
  const int w = (threadIdx.x >> 5) & 3;
  float2 *col = &s_state[w][lane];
  float2 *D = s_diag[w];
  const uint32_t cost = __reduce_add_sync(kFull, (ops0 != kOpIdentity) + (ops1 != kOpIdentity));
  const uint32_t work = __reduce_add_sync(kFull, op_work(p, (int)ops0) + op_work(p, (int)ops1));
  __syncwarp();  // the previous circuit's reads of D
#pragma unroll
  for (int r = 0; r < 32; ++r) col[r << 5] = make_float2(r == lane ? 1.f : 0.f, 0.f);
  bool pending = false;  // D holds phases not yet applied to S
  const uint32_t L = p.L;
  for (uint32_t t = 0; t < L; ++t) {
    const uint32_t src = t < 32 ? ops0 : ops1;
    const int op = __shfl_sync(kFull, (int)src, (int)(t & 31));
    if (op == kOpIdentity) continue;
    const float c = __shfl_sync(kFull, t < 32 ? ic0 : ic1, (int)(t & 31));
    const float sn = __shfl_sync(kFull, t < 32 ? is0 : is1, (int)(t & 31));
    const int o = op & 0x7f;
    if (o >= kOpIsingJ || (o - kOpIsingRot) % 3 == 2) {
      // R_z on wire w (row bit tb): rows with bit 0 take c - i s, bit 1 c + i s;
      // J on wires (i, j): c - i s where the two bits agree, c + i s elsewhere
      int tb, ib = -1;
      if (o >= kOpIsingJ) {
        int q = o - kOpIsingJ, i = 0;
        while (q >= 4 - i) {
          q -= 4 - i;
          ++i;
        }
        tb = 4 - (i + 1 + q);
        ib = 4 - i;
      } else {
        tb = 4 - (o - kOpIsingRot) / 3;
      }
      int odd = (lane >> tb) & 1;
      if (ib >= 0) odd ^= (lane >> ib) & 1;
      const float ds = odd ? -sn : sn;
      float2 v = pending ? D[lane] : make_float2(1.f, 0.f);
      A::phase(v.x, v.y, c, ds);
      D[lane] = v;
      pending = true;
      continue;
    }
    // R_x or R_y on wire w: row pairs (r, r | 1 << tb), each row first taking
    // its pending phase
    const int k = (o - kOpIsingRot) % 3;
    const int tb = 4 - (o - kOpIsingRot) / 3;
    if (pending) __syncwarp();  // the lanes' writes of D
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const int r0 = ((i >> tb) << (tb + 1)) | (i & ((1 << tb) - 1));
      const int r1 = r0 | (1 << tb);
      float2 x = col[r0 << 5], y = col[r1 << 5];
      if (pending) {
        const float2 d0 = D[r0], d1 = D[r1];
        const float xr = x.x, yr = y.x;
        x.x = d0.x * xr - d0.y * x.y;
        x.y = d0.x * x.y + d0.y * xr;
        y.x = d1.x * yr - d1.y * y.y;
        y.y = d1.x * y.y + d1.y * yr;
      }
      const float2 x0 = x, y0 = y;
      if (k == 0) {
        A::rx_lane(x.x, x.y, y0.x, y0.y, c, sn);
        A::rx_lane(y.x, y.y, x0.x, x0.y, c, sn);
      } else {
        A::ry_lane(x.x, x.y, y0.x, y0.y, false, c, sn);
        A::ry_lane(y.x, y.y, x0.x, x0.y, true, c, sn);
      }
      col[r0 << 5] = x;
      col[r1 << 5] = y;
    }
    if (pending) {
      __syncwarp();  // every lane has read D
      D[lane] = make_float2(1.f, 0.f);
      pending = false;
    }
  }
  if (pending) __syncwarp();
  // the logical rows of S with their pending phases
  auto row = [&](int i) {
    float2 v = col[i << 5];
    if (pending) {
      const float2 d = D[i];
      const float vr = v.x;
      v.x = d.x * vr - d.y * v.y;
      v.y = d.x * v.y + d.y * vr;
    }
    return v;
  };
  CircuitOut out;
  out.cost = cost;
  out.work = work + 2u * 32u;
  out.bad = false;
  const int j = lane;
  if (S_out) {
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const float2 v = row(i);
      S_out[2 * (i * 32 + j)] = v.x;
      S_out[2 * (i * 32 + j) + 1] = v.y;
    }
  }
  float vr = 0.f, vi = 0.f;
  const bool dense = DENSE_OK && p.dense != 0;
  if (!dense) {
    const float2 v = row(p.perm[j]);
    vr = v.x;
    vi = v.y;
  } else {
    out.work += 8u * 32u * 32u - 2u * 32u;
    for (int i = 0; i < 32; ++i) {
      const float2 v = row(i);
      const float2 tt = __ldg(p.tgt32 + i * 32 + j);
      vr = fmaf(v.x, tt.x, fmaf(v.y, tt.y, vr));
      vi = fmaf(v.x, tt.y, fmaf(-v.y, tt.x, vi));
    }
  }
  const double pen =
      p.cost_weight == 0.0 ? 0.0 : __dmul_rn(p.cost_weight, __ddiv_rn((double)cost, (double)p.L));
  out.F = fitness32(p, vr, vi, pen, 32);
  return out;
}

// the group of 2^WB warps that shares one circuit (binary64, WB > 0): this
// warp's index in it, the group's named barrier and its shared-memory row of
// per-column score terms
struct Split {
  int sub = 0;
  int bar = 0;
  double2 *sv = nullptr;
};

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ops0/ops1: this lane's op bytes for slots lane and lane + 32
// ic0/is0, ic1/is1: cos/sin of theta/2 of this lane's slots (Ising)
// DENSE_OK = false compiles the dense-target score out (permutation targets only)
// WB > 0 (binary64 only): this warp composes its 2^-WB share of the columns;
// the score's terms meet in sp.sv and lane 0 of warp sp.sub == 0 folds them
// (out.F is valid there only)
template <int NQ, typename R, bool CANON, bool ISING = false, bool DENSE_OK = true, int WB = 0>
__device__ __forceinline__ CircuitOut compose_score(const DevProblem &p, int lane, uint32_t ops0,
                                                    uint32_t ops1, R *S_out, R ic0 = R(1),
                                                    R is0 = R(0), R ic1 = R(1), R is1 = R(0),
                                                    const Split &sp = Split{}) {
  static_assert(WB == 0 || CANON, "the column split is a binary64 form");
  if constexpr (NQ == 5 && !CANON && !ISING) {
    return compose5_smem<DENSE_OK>(p, lane, ops0, ops1, (float *)S_out);
  } else if constexpr (NQ == 5 && !CANON && ISING) {
    return compose5_smem_ising<DENSE_OK>(p, lane, ops0, ops1, (float *)S_out, (float)ic0,
                                         (float)is0, (float)ic1, (float)is1);
  } else {
  using Ly = Lay<NQ, WB>;
  constexpr int N = Ly::N;
  const int j = (sp.sub << Ly::CB) | (lane & ((1 << Ly::CB) - 1));
  const int grp = (lane >> Ly::CB) & ((1 << Ly::RBL) - 1);
  const bool shadow = (lane >> (Ly::CB + Ly::RBL)) != 0;
  R re[Ly::ROWS], im[Ly::ROWS];
#pragma unroll
  for (int r = 0; r < Ly::ROWS; ++r) {
    re[r] = (((grp << Ly::RBR) | r) == j) ? R(1) : R(0);
    im[r] = R(0);
  }
  // gate cost and work of this lane's slots, reduced once (identity ops and
  // the slots beyond L carry kOpIdentity)
  const uint32_t cost = __reduce_add_sync(kFull, (ops0 != kOpIdentity) + (ops1 != kOpIdentity));
  const uint32_t work = __reduce_add_sync(kFull, op_work(p, (int)ops0) + op_work(p, (int)ops1));
  const uint32_t L = p.L;
  // 5 qubits: wire w starts at physical bit 4 - w (pos), bit b holds wire
  // 4 - b (inv); binary32 translates rows through the map at the output,
  // binary64 restores the identity map after the last gate
  constexpr bool kMap5 = NQ == 5 && WB == 0;
  constexpr bool kMapped = NQ == 5 && !CANON;
  uint32_t pos = 0, inv = 0;
  if constexpr (kMap5) {
#pragma unroll
    for (int w = 0; w < 5; ++w) {
      pos |= (uint32_t)(4 - w) << (3 * w);
      inv |= (uint32_t)w << (3 * (4 - w));
    }
  }
  // the non-identity slots in ascending order: slots 0..31 from the lanes'
  // ops0, then 32..63 from ops1 (slots at or beyond L carry kOpIdentity)
  for (int half = 0; half < (L > 32u ? 2 : 1); ++half) {
    const uint32_t src = half ? ops1 : ops0;
    uint32_t m = __ballot_sync(kFull, src != kOpIdentity);
    while (m) {
      const int t = __ffs(m) - 1;
      m &= m - 1;
      const int op = __shfl_sync(kFull, (int)src, t);
      R ic = R(1), is = R(0);
      if constexpr (ISING) {
        ic = __shfl_sync(kFull, half ? ic1 : ic0, t);
        is = __shfl_sync(kFull, half ? is1 : is0, t);
      }
      if constexpr (kMap5) {
        apply5<ISING, R, CANON>(op, pos, inv, re, im, ic, is);
      } else {
        const R s = (op & kOpNeg) ? R(-1) : R(1);
        dispatch<NQ, R, CANON, ISING, WB>(op & 0x7f, re, im, lane, s, ic, is);
      }
    }
  }
  if constexpr (kMap5 && !kMapped) restore5(pos, inv, re, im);
  CircuitOut out;
  out.cost = cost;
  out.work = work + 2u * N;
  out.bad = false;
  if (S_out) {
    if (!shadow) {
#pragma unroll
      for (int r = 0; r < Ly::ROWS; ++r) {
        int i = (grp << Ly::RBR) | r;
        if constexpr (kMapped) {
          // logical row of physical row r: bit b of r is wire inv[b]
          int x = 0;
#pragma unroll
          for (int b = 0; b < 5; ++b) x |= ((r >> b) & 1) << (4 - (int)((inv >> (3 * b)) & 7));
          i = x;
        }
        S_out[2 * (i * N + j)] = re[r];
        S_out[2 * (i * N + j) + 1] = im[r];
      }
    }
  }
  // this lane's S[perm[j]][j], if it holds that row.  Picked by an arithmetic
  // blend (exact: one term has weight 1, the rest weight 0) so that the state
  // array is never indexed dynamically and stays in registers.
  R vr = R(0), vi = R(0);
  const bool dense = DENSE_OK && p.dense != 0;
  if (dense) out.work += 8u * N * N - 2u * N;  // the dense score
  if (!dense) {
    int pj = p.perm[j];
    if constexpr (kMapped) pj = phys_row5(pj, pos);
    const uint32_t own = (!shadow && (pj >> Ly::RBR) == grp) ? (1u << (pj & (Ly::ROWS - 1))) : 0u;
#pragma unroll
    for (int r = 0; r < Ly::ROWS; ++r) {
      const R m = (R)((own >> r) & 1u);
      vr = fma(m, re[r], vr);
      vi = fma(m, im[r], vi);
    }
  } else if constexpr (!CANON) {
    // dense target, binary32: this lane's rows of the diagonal element
    // (S^dag T)_jj = sum_i conj(S_ij) T_ij, any order
    if (!shadow) {
#pragma unroll
      for (int r = 0; r < Ly::ROWS; ++r) {
        int i = (grp << Ly::RBR) | r;
        if constexpr (kMapped) {
          int x = 0;
#pragma unroll
          for (int b = 0; b < 5; ++b) x |= ((r >> b) & 1) << (4 - (int)((inv >> (3 * b)) & 7));
          i = x;
        }
        const float2 t = __ldg(p.tgt32 + i * N + j);
        vr = fmaf(re[r], t.x, fmaf(im[r], t.y, vr));
        vi = fmaf(re[r], t.y, fmaf(-im[r], t.x, vi));
      }
    }
  }
  const double pen =
      p.cost_weight == 0.0 ? 0.0 : __dmul_rn(p.cost_weight, __ddiv_rn((double)cost, (double)p.L));
  if constexpr (CANON) {
    // sequential sum over j ascending, on lane 0 (the values arrive by shuffle;
    // the binary64 arithmetic runs on one lane only)
    double a = 0.0, b = 0.0;
    if (dense) {
      // the oracle's order: each diagonal element (S^dag T)_jj summed over rows
      // i ascending (row group g continues group g - 1's sum), then the trace
      // over j ascending
      double dr = 0.0, di = 0.0;
#pragma unroll
      for (int g2 = 0; g2 < (1 << Ly::RBL); ++g2) {
        if (g2 > 0) {
          const double ur = __shfl_up_sync(kFull, dr, 1 << Ly::CB);
          const double ui = __shfl_up_sync(kFull, di, 1 << Ly::CB);
          if (grp == g2) {
            dr = ur;
            di = ui;
          }
        }
        if (grp == g2 && !shadow) {
#pragma unroll
          for (int r = 0; r < Ly::ROWS; ++r) {
            const double2 t = __ldg(p.tgt64 + ((g2 << Ly::RBR) | r) * N + j);
            dr = __dadd_rn(dr, __dadd_rn(__dmul_rn((double)re[r], t.x), __dmul_rn((double)im[r], t.y)));
            di = __dadd_rn(di, __dsub_rn(__dmul_rn((double)re[r], t.y), __dmul_rn((double)im[r], t.x)));
          }
        }
      }
      if constexpr (WB > 0) {
        if (grp == (1 << Ly::RBL) - 1 && !shadow) sp.sv[j] = make_double2(dr, di);
      } else {
        const int last = ((1 << Ly::RBL) - 1) << NQ;
        for (int jj = 0; jj < N; ++jj) {
          const double xr = __shfl_sync(kFull, dr, last | jj), xi = __shfl_sync(kFull, di, last | jj);
          if (lane == 0) {
            a = __dadd_rn(a, xr);
            b = __dadd_rn(b, xi);
          }
        }
      }
    } else if constexpr (WB > 0) {
      if (!shadow && (p.perm[j] >> Ly::RBR) == grp) sp.sv[j] = make_double2(vr, vi);
    } else {
      for (int jj = 0; jj < N; ++jj) {
        const int owner = ((p.perm[jj] >> Ly::RBR) << NQ) | jj;
        const double xr = __shfl_sync(kFull, vr, owner), xi = __shfl_sync(kFull, vi, owner);
        if (lane == 0) {
          if (p.fit_kind == 1) {
            a = __dadd_rn(a, __dadd_rn(__dmul_rn(xr, xr), __dmul_rn(xi, xi)));
          } else {
            a = __dadd_rn(a, xr);
            b = __dadd_rn(b, -xi);
          }
        }
      }
    }
    if constexpr (WB > 0) {
      // the same sums in the same order (columns ascending), from shared memory
      named_sync(sp.bar, 32 << WB);
      if (sp.sub == 0 && lane == 0) {
        for (int jj = 0; jj < N; ++jj) {
          const double xr = sp.sv[jj].x, xi = sp.sv[jj].y;
          if (dense) {
            a = __dadd_rn(a, xr);
            b = __dadd_rn(b, xi);
          } else if (p.fit_kind == 1) {
            a = __dadd_rn(a, __dadd_rn(__dmul_rn(xr, xr), __dmul_rn(xi, xi)));
          } else {
            a = __dadd_rn(a, xr);
            b = __dadd_rn(b, -xi);
          }
        }
      }
      named_sync(sp.bar, 32 << WB);  // sp.sv is free for the group's next circuit
    }
    double F = 0.0;
    if (lane == 0) {
      // (size - x) / size: size = N is a power of two, so the division is the
      // exact scaling by 1/N (identical result, no binary64 division sequence)
      const double size = (double)N, inv = 1.0 / (double)N;
      double d;
      if (p.fit_kind == 1) {
        d = __dmul_rn(__dsub_rn(size, a), inv);
      } else {
        const double m = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
        d = __dmul_rn(__dsub_rn(size, m), inv);
      }
      if (d < 0.0) d = 0.0;
      const double f = __dsub_rn(1.0, __dsqrt_rn(d));
      F = __dsub_rn(f, pen);
    }
    out.F = __shfl_sync(kFull, F, 0);
  } else {
    out.F = fitness32(p, (float)vr, (float)vi, pen, N);
  }
  return out;
  }
}

// op byte of library gate g (kOpIdentity also for out-of-range g; bad flags it)
__device__ __forceinline__ uint32_t op_of(const DevProblem &p, uint32_t g, bool &bad) {
  if (g >= p.G) {
    bad = true;
    return kOpIdentity;
  }
  return p.gop[g];
}

__device__ __forceinline__ uint32_t find_problem(const uint32_t *prefix, uint32_t n, uint32_t x) {
  // largest q with prefix[q] <= x
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------ kernels
// Whole generation for a group of searches: sample, compose, score, scatter.
// minimum resident 256-thread blocks per SM: the 5-qubit binary32 kernel is
// capped at 128 registers (its 64 state registers plus temporaries); the
// scheduler otherwise interleaves every row pair of a gate and asks for ~190.
//
// The 5-qubit binary32 kernel runs 128-thread blocks (four circuits, 32 KB of
// shared memory for their unitaries, see compose5_smem): six fit an SM's
// shared memory, so each thread may use 85 registers (its Ising variant too,
// with 1 KB more for the deferred diagonal factors).
template <int NQ, bool CANON>
constexpr int block_threads() {
  return (NQ == 5 && !CANON) ? 128 : 256;
}
// log2 of the warps per circuit.  binary64 at 5 qubits: each circuit's
// columns on 4 warps (8 rows per lane: ~120 registers without spills instead
// of 255 with spills); at 4 qubits on 2 warps (4 rows per lane, 80 registers
// instead of 108: 4.76 -> 4.65 ms for 65 536 circuits of 32 gates; 4 warps
// took 5.57 ms); at 3 qubits one warp (2 warps: 0.136 -> 0.163 ms)
template <int NQ, bool CANON>
constexpr int circuit_split() {
  return CANON ? (NQ == 5 ? 2 : (NQ == 4 ? 1 : 0)) : 0;
}
template <int NQ, bool CANON, bool ISING>
constexpr int min_blocks() {
  return (NQ == 5 && !CANON) ? 6 : ((NQ <= 3 && !CANON) ? 6 : 1);
}

// EXT: the group holds a search measured K > 1 times (k_presample) or one with
// a dense target; without it both paths are compiled out of the kernel
template <int NQ, typename R, bool CANON, bool ISING, bool EXT>
__global__ void __launch_bounds__(block_threads<NQ, CANON>(), min_blocks<NQ, CANON, ISING>()) k_step(const DevProblem *__restrict__ probs,
                                              const uint32_t *__restrict__ group,
                                              const uint32_t *__restrict__ prefix,
                                              uint32_t n_group, uint32_t total, DevGlobal g) {
  constexpr int WB = circuit_split<NQ, CANON>();
  const int lane = threadIdx.x & 31;
  const int sub = (threadIdx.x >> 5) & ((1 << WB) - 1);  // warp within the circuit's group
  __shared__ double2 s_terms[WB ? (block_threads<NQ, CANON>() / 32) >> WB : 1][32];
  Split sp;
  sp.sub = sub;
  sp.bar = 1 + ((threadIdx.x >> 5) >> WB);
  sp.sv = s_terms[WB ? (threadIdx.x >> 5) >> WB : 0];
  const uint32_t gen = *g.gen;
  const uint32_t nw = (gridDim.x * blockDim.x) >> (5 + WB);
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> (5 + WB); w < total; w += nw) {
    const uint32_t q = find_problem(prefix, n_group, w);
    const DevProblem &p = probs[group[q]];
    const uint32_t c = w - prefix[q];
    const uint32_t par = gen & 1u;  // generation buffer
    uint8_t *gate_idx = p.gate_idx + (size_t)par * p.P * p.L;
    uint32_t o0 = kOpIdentity, o1 = kOpIdentity, seg0 = 0, seg1 = 0;
    bool bad = false;
    const bool qeqea = p.enc == kEncQeqea;
    float2 a0 = make_float2(1.f, 0.f), a1 = a0;  // Ising: the slots' angles
    if (EXT && qeqea && p.shots > 1) {
      // measured K times by k_presample ahead of this kernel
      if ((uint32_t)lane < p.L) {
        o0 = op_of(p, gate_idx[(size_t)c * p.L + lane], bad);
        seg0 = p.seg_id[(size_t)c * p.L + lane];
      }
      if ((uint32_t)lane + 32 < p.L) {
        o1 = op_of(p, gate_idx[(size_t)c * p.L + lane + 32], bad);
        seg1 = p.seg_id[(size_t)c * p.L + lane + 32];
      }
      if constexpr (ISING) {
        const float2 *amps = p.amps + (size_t)par * p.P * p.L + (size_t)c * p.L;
        if ((uint32_t)lane < p.L) a0 = amps[lane];
        if ((uint32_t)lane + 32 < p.L) a1 = amps[lane + 32];
      }
      if (sub == 0) prefetch_mutated(p, c, gen, lane);
    } else if (qeqea) {
      float2 *amps = ISING ? p.amps + (size_t)par * p.P * p.L + (size_t)c * p.L : nullptr;
      // (with the columns split over a group of warps every warp samples the
      // same slots; the first one writes them, lists the mutation and scatters)
      if ((uint32_t)lane < p.L) {
        uint32_t gg;
        sample_slot<ISING>(p, c, lane, gen, gg, seg0, a0);
        if (sub == 0) {
          gate_idx[(size_t)c * p.L + lane] = (uint8_t)gg;
          p.seg_id[(size_t)c * p.L + lane] = seg0;
          if constexpr (ISING) amps[lane] = a0;
        }
        o0 = op_of(p, gg, bad);
      }
      if ((uint32_t)lane + 32 < p.L) {
        uint32_t gg;
        sample_slot<ISING>(p, c, lane + 32, gen, gg, seg1, a1);
        if (sub == 0) {
          gate_idx[(size_t)c * p.L + lane + 32] = (uint8_t)gg;
          p.seg_id[(size_t)c * p.L + lane + 32] = seg1;
          if constexpr (ISING) amps[lane + 32] = a1;
        }
        o1 = op_of(p, gg, bad);
      }
      if (sub == 0) prefetch_mutated(p, c, gen, lane);
    } else {
      // GA: this generation's genome, bred by the previous generation (k_ga_next)
      if ((uint32_t)lane < p.L) o0 = op_of(p, gate_idx[(size_t)c * p.L + lane], bad);
      if ((uint32_t)lane + 32 < p.L) o1 = op_of(p, gate_idx[(size_t)c * p.L + lane + 32], bad);
      if constexpr (ISING) {  // and the genes' angles
        const float2 *amps = p.amps + (size_t)par * p.P * p.L + (size_t)c * p.L;
        if ((uint32_t)lane < p.L) a0 = amps[lane];
        if ((uint32_t)lane + 32 < p.L) a1 = amps[lane + 32];
      }
    }
    R ic0 = R(1), is0 = R(0), ic1 = R(1), is1 = R(0);
    if constexpr (ISING) {
      half_angle(a0.x, a0.y, ic0, is0);
      half_angle(a1.x, a1.y, ic1, is1);
    }
    CircuitOut out = compose_score<NQ, R, CANON, ISING, EXT, WB>(p, lane, o0, o1, (R *)nullptr,
                                                                  ic0, is0, ic1, is1, sp);
    if (sub != 0) continue;  // the score is on the group's first warp
    const bool nonfinite = !isfinite(out.F);
    if (lane == 0) {
      if constexpr (CANON) p.fit64[(size_t)par * p.P + c] = out.F;
      else p.fit32[(size_t)par * p.P + c] = (float)out.F;
      p.meta[(size_t)par * p.P + c] = out.cost | (out.work << 8);
      if (nonfinite) atomicOr(g.err, kErrNonFinite);
    }
    if (!nonfinite && qeqea) {
      const uint32_t key = fkey((float)out.F);
      if ((uint32_t)lane < p.L) atomicMax(key_of(p, seg0), key);
      if ((uint32_t)lane + 32 < p.L) atomicMax(key_of(p, seg1), key);
    }
  }
}

// Measurement ahead of the circuit kernel for the searches that measure each
// qutrit K > 1 times: one thread per slot over all of them (prefix sums of
// P * L), writing this generation's gate_idx, seg_id and (Ising) angles.
__global__ void __launch_bounds__(256) k_presample(const DevProblem *__restrict__ probs,
                                                   const uint32_t *__restrict__ ids,
                                                   const unsigned long long *__restrict__ prefix,
                                                   uint32_t n_ids, unsigned long long total,
                                                   DevGlobal g) {
  const uint32_t gen = *g.gen;
  const uint32_t par = gen & 1u;
  for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       e < total; e += (unsigned long long)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_ids;  // the search holding slot e
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (prefix[mid] <= e) lo = mid;
      else hi = mid;
    }
    const DevProblem &p = probs[ids[lo]];
    const size_t x = (size_t)(e - prefix[lo]);
    const uint32_t c = (uint32_t)(x / p.L), t = (uint32_t)(x % p.L);
    uint32_t gg, seg;
    float2 amp;
    if (p.ising) {
      sample_slot<true, true>(p, c, t, gen, gg, seg, amp);
      p.amps[(size_t)par * p.P * p.L + x] = amp;
    } else {
      sample_slot<false, true>(p, c, t, gen, gg, seg, amp);
    }
    p.gate_idx[(size_t)par * p.P * p.L + x] = (uint8_t)gg;
    p.seg_id[x] = seg;
  }
}

// Measurement only (qe_sample).
__global__ void __launch_bounds__(256) k_sample(const DevProblem *__restrict__ probs,
                                                uint32_t prob, uint32_t gen, uint8_t *gate_idx,
                                                uint32_t *seg_id) {
  const DevProblem &p = probs[prob];
  const size_t n = (size_t)p.P * p.L;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const uint32_t c = (uint32_t)(e / p.L), t = (uint32_t)(e % p.L);
    uint32_t gg, seg;
    float2 amp;
    if (p.ising) sample_slot<true, true>(p, c, t, gen, gg, seg, amp);
    else sample_slot<false, true>(p, c, t, gen, gg, seg, amp);
    gate_idx[e] = (uint8_t)gg;
    seg_id[e] = seg;
  }
}

// One caller-provided circuit: its gate string g_c (and Ising slot angles a_c)
// composed and scored by the circuit's warp group; lane 0 of its first warp
// stores the fitness (NaN for an invalid gate index) and cost, and sets the
// error word.
template <int NQ, typename R, bool CANON, bool ISING>
__device__ __forceinline__ void eval_one(const DevProblem &p, int lane, const Split &sp,
                                         const uint8_t *__restrict__ g_c,
                                         const float2 *__restrict__ a_c, R *fit_c,
                                         uint32_t *cost_c, R *S_c, const DevGlobal &g) {
  constexpr int WB = circuit_split<NQ, CANON>();
  bool bad = false;
  uint32_t o0 = kOpIdentity, o1 = kOpIdentity;
  if ((uint32_t)lane < p.L) o0 = op_of(p, g_c[lane], bad);
  if ((uint32_t)lane + 32 < p.L) o1 = op_of(p, g_c[lane + 32], bad);
  const bool anybad = __any_sync(kFull, bad);
  R ic0 = R(1), is0 = R(0), ic1 = R(1), is1 = R(0);
  if constexpr (ISING) {
    if ((uint32_t)lane < p.L) {
      const float2 a = a_c[lane];
      half_angle(a.x, a.y, ic0, is0);
    }
    if ((uint32_t)lane + 32 < p.L) {
      const float2 a = a_c[lane + 32];
      half_angle(a.x, a.y, ic1, is1);
    }
  }
  CircuitOut out =
      compose_score<NQ, R, CANON, ISING, true, WB>(p, lane, o0, o1, S_c, ic0, is0, ic1, is1, sp);
  if (lane == 0 && sp.sub == 0) {
    double F = anybad ? __longlong_as_double(0x7ff8000000000000ll) : out.F;
    if (fit_c) *fit_c = (R)F;
    if (cost_c) *cost_c = out.cost;
    if (anybad) atomicOr(g.err, kErrBadGate);
    else if (!isfinite(F)) atomicOr(g.err, kErrNonFinite);
  }
}

// this thread's place in its circuit's warp group (binary64 at 5 qubits: four
// warps per circuit, the score's terms in s_terms)
#define QE_EVAL_SPLIT(NQ, CANON)                                                    \
  constexpr int WB = circuit_split<NQ, CANON>();                                    \
  const int lane = threadIdx.x & 31;                                                \
  __shared__ double2 s_terms[WB ? (block_threads<NQ, CANON>() / 32) >> WB : 1][32]; \
  Split sp;                                                                         \
  sp.sub = (threadIdx.x >> 5) & ((1 << WB) - 1);                                    \
  sp.bar = 1 + ((threadIdx.x >> 5) >> WB);                                          \
  sp.sv = s_terms[WB ? (threadIdx.x >> 5) >> WB : 0];                               \
  const uint32_t nw = (gridDim.x * blockDim.x) >> (5 + WB);                         \
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> (5 + WB);

// Fitness (and optionally the unitaries) of caller-provided gate strings
// (Ising: with every slot's angle as qubit amplitudes in amps).
template <int NQ, typename R, bool CANON, bool ISING>
__global__ void __launch_bounds__(block_threads<NQ, CANON>(), min_blocks<NQ, CANON, ISING>()) k_eval(const DevProblem *__restrict__ probs, uint32_t prob,
                                              const uint8_t *__restrict__ gates,
                                              const float2 *__restrict__ amps, uint32_t n,
                                              R *fit, uint32_t *cost, R *S, DevGlobal g) {
  QE_EVAL_SPLIT(NQ, CANON)
  const DevProblem &p = probs[prob];
  const size_t NN2 = 2 * (size_t)p.N * p.N;
  for (uint32_t c = w0; c < n; c += nw)
    eval_one<NQ, R, CANON, ISING>(p, lane, sp, gates + (size_t)c * p.L,
                                  ISING ? amps + (size_t)c * p.L : nullptr,
                                  fit ? fit + c : nullptr, cost ? cost + c : nullptr,
                                  S ? S + NN2 * c : nullptr, g);
}

// Several searches' caller-provided circuits of one width in one launch (the
// batched host call): circuit w of the launch belongs to the job whose first
// circuit is the largest first <= w.
template <int NQ, typename R, bool CANON>
__global__ void __launch_bounds__(block_threads<NQ, CANON>(), min_blocks<NQ, CANON, false>()) k_eval_jobs(const DevProblem *__restrict__ probs,
                                                   const EvalJob *__restrict__ jobs,
                                                   uint32_t n_jobs, uint32_t total, DevGlobal g) {
  wait_predecessor();  // the batch graph's copy of the gate strings
  QE_EVAL_SPLIT(NQ, CANON)
  for (uint32_t w = w0; w < total; w += nw) {
    uint32_t lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (jobs[mid].first <= w) lo = mid;
      else hi = mid;
    }
    const EvalJob &j = jobs[lo];
    const DevProblem &p = probs[j.prob];
    const uint32_t c = w - j.first;
    eval_one<NQ, R, CANON, false>(p, lane, sp, j.gates + (size_t)c * p.L, nullptr,
                                  (R *)j.fit + c, j.cost + c, nullptr, g);
  }
}
#undef QE_EVAL_SPLIT

// Binary64 rescoring of ranking candidates: list entries are problem << 20 | slot,
// the circuit is cand[slot] of that problem, gates (and Ising angles) come from
// gtab[problem] (a batch of several searches' caller circuits), else gsrc/asrc
// (NULL = the problem's own generation buffers).  One launch per
// (qubit count, library kind) present; other entries are skipped.
// warps per binary64 rescoring candidate, log2: 2 at 3 qubits (one row per
// lane), 4 at 4 and 5 qubits
template <int NQ>
constexpr int rescore_split() {
  return NQ == 3 ? 1 : (NQ >= 4 ? 2 : 0);
}
constexpr int rescore_split_of(uint32_t nq) { return nq == 3 ? 1 : (nq >= 4 ? 2 : 0); }

template <int NQ, bool ISING>
__global__ void __launch_bounds__(256) k_rescore(const DevProblem *__restrict__ probs,
                                                 const uint8_t *__restrict__ gsrc,
                                                 const float2 *__restrict__ asrc, int pipelined,
                                                 const uint8_t *const *__restrict__ gtab,
                                                 DevGlobal g) {
  wait_predecessor();  // the selection's candidates and chain flag
  // 2^WB warps per candidate, each composing a share of its columns: a
  // binary64 instruction of one warp issues once per ~68 cycles on GB300's
  // thin binary64 pipe, so a candidate's latency shrinks with the warps that
  // share it (up to the SM's rate, ~3.4 warps' worth)
  constexpr int WB = rescore_split<NQ>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp >> WB, sub = warp & ((1 << WB) - 1);
  const uint32_t groups = (blockDim.x >> 5) >> WB;
  const uint32_t ng = gridDim.x * groups;
  __shared__ double2 s_terms[256 / 32][32];
  Split sp;
  sp.sub = sub;
  sp.bar = 1 + grp;
  sp.sv = s_terms[grp];
  if (pipelined && !*g.rank_active) return;
  const uint32_t par = pipelined ? ((*g.gen - 1u) & 1u) : 0u;
  const uint32_t total = *g.rescore_n;
  // entries are dealt block-first (entry w -> block w % gridDim) so that a
  // short queue spreads one binary64 circuit per SM before doubling up
  for (uint32_t w = blockIdx.x + gridDim.x * grp; w < total; w += ng) {
    const uint32_t ent = g.rescore_list[w];
    const DevProblem &p = probs[ent >> 20];
    if (p.n != (uint32_t)NQ || (p.ising != 0) != ISING) continue;
    const uint32_t slot = ent & 0xfffffu;
    const uint32_t c = p.cand[slot];
    const uint8_t *gates =
        (gtab ? gtab[ent >> 20] : gsrc ? gsrc : p.gate_idx + (size_t)par * p.P * p.L) +
        (size_t)c * p.L;
    bool bad = false;
    uint32_t o0 = kOpIdentity, o1 = kOpIdentity;
    if ((uint32_t)lane < p.L) o0 = op_of(p, gates[lane], bad);
    if ((uint32_t)lane + 32 < p.L) o1 = op_of(p, gates[lane + 32], bad);
    const bool anybad = __any_sync(kFull, bad);
    double ic0 = 1.0, is0 = 0.0, ic1 = 1.0, is1 = 0.0;
    if constexpr (ISING) {
      const float2 *am =
          (asrc ? asrc : p.amps + (size_t)par * p.P * p.L) + (size_t)c * p.L;
      if ((uint32_t)lane < p.L) half_angle(am[lane].x, am[lane].y, ic0, is0);
      if ((uint32_t)lane + 32 < p.L) half_angle(am[lane + 32].x, am[lane + 32].y, ic1, is1);
    }
    const double F32 = p.cand_f[slot];  // the binary32 fitness the selection ranked by
    CircuitOut out = compose_score<NQ, double, true, ISING, true, WB>(
        p, lane, o0, o1, (double *)nullptr, ic0, is0, ic1, is1, sp);
    if (lane == 0 && sub == 0) {
      p.cand_f[slot] = anybad ? __longlong_as_double(0x7ff8000000000000ll) : out.F;
      // the exactness of the top-k rests on every binary64 fitness lying in the
      // interval its binary32 fitness implies: check it on every candidate
      float lo, hi;
      guard_band(p, (float)F32, out.cost, lo, hi);
      if (!anybad && F32 == F32 && !(out.F >= (double)lo && out.F <= (double)hi))
        atomicOr(g.err, kErrGuardBand);
    }
  }
}

// ------------------------------------------------------------------ launchers
#define QE_NQ_SWITCH(n, X) \
  switch (n) {             \
    case 1: X(1); break;   \
    case 2: X(2); break;   \
    case 3: X(3); break;   \
    case 4: X(4); break;   \
    default: X(5); break;  \
  }

cudaError_t launch_step(const LaunchCfg &lc, uint32_t n, const DevProblem *probs,
                        const uint32_t *group, const uint32_t *prefix, uint32_t n_group,
                        uint32_t total, bool canon, bool ising, bool ext, const DevGlobal &g,
                        cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  uint32_t per = canon ? lc.step64[n] : lc.step32[n];
  if (lc.grid_mode == 1 && per > 1) per -= 1;
  if (lc.grid_mode == 2) per = 0xffffu;  // every circuit's warp in one launch
#define QE_LK(NQ, R, C, I)                                                                \
  {                                                                                       \
    constexpr int bt = block_threads<NQ, C>();                                            \
    const dim3 grid = grid_for(lc, total, per, (bt / 32) >> circuit_split<NQ, C>());      \
    if (ext)                                                                              \
      k_step<NQ, R, C, I, true><<<grid, bt, 0, st>>>(probs, group, prefix, n_group, total, g); \
    else                                                                                  \
      k_step<NQ, R, C, I, false><<<grid, bt, 0, st>>>(probs, group, prefix, n_group, total, g); \
  }
#define QE_L(NQ)                                                                          \
  if (canon) {                                                                            \
    if (ising) QE_LK(NQ, double, true, true) else QE_LK(NQ, double, true, false)          \
  } else {                                                                                \
    if (ising) QE_LK(NQ, float, false, true) else QE_LK(NQ, float, false, false)          \
  }
  QE_NQ_SWITCH(n, QE_L)
#undef QE_L
#undef QE_LK
  return cudaGetLastError();
}

cudaError_t launch_presample(const LaunchCfg &lc, const DevProblem *probs, const uint32_t *ids,
                             const unsigned long long *prefix, uint32_t n_ids,
                             unsigned long long total, const DevGlobal &g, cudaStream_t st) {
  if (!n_ids || !total) return cudaSuccess;
  unsigned long long blocks = (total + 255) / 256;
  const unsigned long long cap = (unsigned long long)lc.num_sms * 16;
  if (blocks > cap) blocks = cap;
  k_presample<<<(uint32_t)blocks, 256, 0, st>>>(probs, ids, prefix, n_ids, total, g);
  return cudaGetLastError();
}

cudaError_t launch_sample(const LaunchCfg &lc, const DevProblem *probs, uint32_t prob, uint32_t P,
                          uint32_t L, uint32_t gen, uint8_t *gate_idx, uint32_t *seg_id,
                          cudaStream_t st) {
  const size_t n = (size_t)P * L;
  uint32_t blocks = (uint32_t)((n + 255) / 256);
  const uint32_t cap = lc.num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_sample<<<blocks, 256, 0, st>>>(probs, prob, gen, gate_idx, seg_id);
  return cudaGetLastError();
}

cudaError_t launch_eval(const LaunchCfg &lc, uint32_t nq, const DevProblem *probs, uint32_t prob,
                        bool canon, const uint8_t *gates, const float2 *amps, uint32_t n,
                        void *fit, uint32_t *cost, void *S, const DevGlobal &g,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const uint32_t per = canon ? lc.step64[nq] : lc.step32[nq];
  const bool ising = amps != nullptr;
#define QE_LK(NQ, R, C, I)                                                                 \
  {                                                                                        \
    constexpr int bt = block_threads<NQ, C>();                                             \
    k_eval<NQ, R, C, I><<<grid_for(lc, n, per, (bt / 32) >> circuit_split<NQ, C>()), bt, 0, st>>>( \
        probs, prob, gates, amps, n, (R *)fit, cost, (R *)S, g);                           \
  }
#define QE_L(NQ)                                                                           \
  if (canon) {                                                                             \
    if (ising) QE_LK(NQ, double, true, true) else QE_LK(NQ, double, true, false)           \
  } else {                                                                                 \
    if (ising) QE_LK(NQ, float, false, true) else QE_LK(NQ, float, false, false)           \
  }
  QE_NQ_SWITCH(nq, QE_L)
#undef QE_L
#undef QE_LK
  return cudaGetLastError();
}

cudaError_t launch_eval_jobs(const LaunchCfg &lc, uint32_t nq, bool canon,
                             const DevProblem *probs, const EvalJob *jobs, uint32_t n_jobs,
                             uint32_t total, const DevGlobal &g, cudaStream_t st) {
  if (total == 0 || n_jobs == 0) return cudaSuccess;
  const uint32_t per = canon ? lc.step64[nq] : lc.step32[nq];
#define QE_LK(NQ, R, C)                                                                    \
  {                                                                                        \
    constexpr int bt = block_threads<NQ, C>();                                             \
    k_eval_jobs<NQ, R, C><<<grid_for(lc, total, per, (bt / 32) >> circuit_split<NQ, C>()), bt, 0, \
                            st>>>(probs, jobs, n_jobs, total, g);                          \
  }
#define QE_L(NQ)                                                                           \
  if (canon) QE_LK(NQ, double, true) else QE_LK(NQ, float, false)
  QE_NQ_SWITCH(nq, QE_L)
#undef QE_L
#undef QE_LK
  return cudaGetLastError();
}

cudaError_t launch_rescore(const LaunchCfg &lc, uint32_t nq, bool ising, const DevProblem *probs,
                           const uint8_t *gsrc, const float2 *asrc, bool pipelined,
                           const DevGlobal &g, cudaStream_t st, const uint8_t *const *gtab,
                           uint32_t expect) {
  // enough blocks for `expect` candidates (any count is handled: the loop
  // strides over the queue), at most the resident grid
  uint32_t blocks = lc.num_sms * lc.step64[nq];
  if (expect) {
    const uint32_t per_block = (256 / 32) >> rescore_split_of(nq);
    const uint32_t want = (expect + per_block - 1) / per_block;
    if (want < blocks) blocks = want;
  }
  const int pl = pipelined ? 1 : 0;
#define QE_L(NQ)                                                                           \
  if (ising)                                                                               \
    k_rescore<NQ, true><<<blocks, 256, 0, st>>>(probs, gsrc, asrc, pl, gtab, g);            \
  else                                                                                     \
    k_rescore<NQ, false><<<blocks, 256, 0, st>>>(probs, gsrc, asrc, pl, gtab, g);
  QE_NQ_SWITCH(nq, QE_L)
#undef QE_L
  return cudaGetLastError();
}

bool is_circuit_kernel(const void *f) {
#define QE_K(NQ)                                                                          \
  if (f == (const void *)k_step<NQ, float, false, false, false> ||                        \
      f == (const void *)k_step<NQ, double, true, false, false> ||                        \
      f == (const void *)k_step<NQ, float, false, true, false> ||                         \
      f == (const void *)k_step<NQ, double, true, true, false> ||                         \
      f == (const void *)k_step<NQ, float, false, false, true> ||                         \
      f == (const void *)k_step<NQ, double, true, false, true> ||                         \
      f == (const void *)k_step<NQ, float, false, true, true> ||                          \
      f == (const void *)k_step<NQ, double, true, true, true>)                            \
    return true;
  QE_K(1) QE_K(2) QE_K(3) QE_K(4) QE_K(5)
#undef QE_K
  return false;
}

bool is_eval_jobs_kernel(const void *f) {
#define QE_K(NQ)                                                                             \
  if (f == (const void *)k_eval_jobs<NQ, float, false> ||                                    \
      f == (const void *)k_eval_jobs<NQ, double, true>)                                      \
    return true;
  QE_K(1) QE_K(2) QE_K(3) QE_K(4) QE_K(5)
#undef QE_K
  return false;
}

bool is_rescore_kernel(const void *f) {
#define QE_K(NQ)                                                                         \
  if (f == (const void *)k_rescore<NQ, false> || f == (const void *)k_rescore<NQ, true>) \
    return true;
  QE_K(1) QE_K(2) QE_K(3) QE_K(4) QE_K(5)
#undef QE_K
  return false;
}

cudaError_t query_circuit_occupancy(LaunchCfg &lc) {
  cudaError_t e = cudaSuccess;
  int b = 0;
  // the 5-qubit binary32 kernels keep their unitaries in shared memory: ask
  // for the largest shared-memory carveout so that six blocks fit an SM
  const void *smem5[] = {(const void *)k_step<5, float, false, false, false>,
                         (const void *)k_step<5, float, false, false, true>,
                         (const void *)k_eval<5, float, false, false>,
                         (const void *)k_step<5, float, false, true, false>,
                         (const void *)k_step<5, float, false, true, true>,
                         (const void *)k_eval<5, float, false, true>};
  for (const void *f : smem5)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
#define QE_Q(NQ)                                                                            \
  if (e == cudaSuccess)                                                                     \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<NQ, float, false, false, false>, \
                                                      block_threads<NQ, false>(), 0);       \
  lc.step32[NQ] = b > 0 ? b : 1;                                                            \
  if (e == cudaSuccess)                                                                     \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<NQ, double, true, false, false>, \
                                                      block_threads<NQ, true>(), 0);        \
  lc.step64[NQ] = b > 0 ? b : 1;
  QE_Q(1) QE_Q(2) QE_Q(3) QE_Q(4) QE_Q(5)
#undef QE_Q
  return e;
}

}  // namespace qe
