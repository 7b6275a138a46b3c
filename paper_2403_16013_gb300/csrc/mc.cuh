// mc.cuh - device library of error-free transformations and multi-component
// (DD / TD / QD, L = 2 / 3 / 4 binary64 limbs) real and complex arithmetic.
//
// The paper (Sec. 1, Sec. 2.2) builds its complex DD/TD/QD operations on
// multi-component real arithmetic without printing the algorithms.  This file
// implements them from the published building blocks:
//   * TwoSum (Knuth): s = RN(a+b), e = a+b-s exactly, 6 flops, any a, b;
//   * TwoProd with FMA: p = RN(ab), e = fma(a,b,-p) = ab-p exactly, 2 flops;
//   * a leveled accumulator: level k collects terms of order u^k (u = 2^-53)
//     exactly with TwoSum and passes each rounding error down to level k+1;
//     only the last level (order u^(L-1)) is summed with plain rounding.
//     Products keep the limb pairs (i, j) with i + j <= L-1 (TwoProd for
//     i + j <= L-2, a plain FMA into the last level for i + j = L-1); the
//     dropped pairs are below u^L relative.  This is the compensated-dot idea
//     of Ogita, Rump and Oishi (Dot2) carried to L levels;
//   * renormalisation: a bottom-up TwoSum pass (VecSum) followed by a
//     top-down TwoSum pass; both are error-free, so the value of the
//     accumulator is kept exactly while it is put back into nonoverlapping
//     limbs.
// Every floating-point operation is written with the _rn intrinsics, so the
// compiler can neither contract nor reassociate them (the library is also
// built with -fmad=false).  Divisions call CUDA's correctly rounded __ddiv_rn.
#pragma once

#include <cstdint>

namespace mclu {

// ------------------------------------------------------------------ EFTs --

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  double x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  double br = __dsub_rn(b, bv);
  double ar = __dsub_rn(a, av);
  s = x;
  e = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e) {
  double x = __dmul_rn(a, b);
  e = __fma_rn(a, b, -x);
  p = x;
}

// Integer views (ALU pipe, not the FP64 pipe).
__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_neg(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ double flip(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
// Monotone integer key of a double (total order consistent with < for non-NaN).
__device__ __forceinline__ long long order_key(double x) {
  long long i = __double_as_longlong(x);
  return i >= 0 ? i : (i ^ 0x7fffffffffffffffLL);
}

// ------------------------------------------------------------ MC values --

template <int L>
struct R {  // real multi-component value: x[0] + ... + x[L-1]
  double x[L];
};

template <int L>
struct Z {  // complex: separate real and imaginary MC parts (Sec. 2.2)
  R<L> re, im;
};

template <int L>
__device__ __forceinline__ R<L> r_zero() {
  R<L> r;
#pragma unroll
  for (int i = 0; i < L; i++) r.x[i] = 0.0;
  return r;
}

template <int L>
__device__ __forceinline__ Z<L> z_zero() {
  Z<L> r;
  r.re = r_zero<L>();
  r.im = r_zero<L>();
  return r;
}

template <int L>
__device__ __forceinline__ R<L> r_neg(const R<L> &a) {
  R<L> r;
#pragma unroll
  for (int i = 0; i < L; i++) r.x[i] = flip(a.x[i]);
  return r;
}

template <int L>
__device__ __forceinline__ R<L> r_abs(const R<L> &a) {
  return is_neg(a.x[0]) ? r_neg(a) : a;
}

template <int L>
__device__ __forceinline__ Z<L> z_conj(const Z<L> &a) {
  Z<L> r;
  r.re = a.re;
  r.im = r_neg(a.im);
  return r;
}

template <int L>
__device__ __forceinline__ Z<L> z_neg(const Z<L> &a) {
  Z<L> r;
  r.re = r_neg(a.re);
  r.im = r_neg(a.im);
  return r;
}

// Renormalise N doubles in place: bottom-up TwoSum pass, then a top-down
// TwoSum pass over the remaining pairs.  Exact; leaves nonoverlapping limbs
// with leading zeros moved out of the way.
template <int N>
__device__ __forceinline__ void renorm_n(double *x) {
  if constexpr (N == 1) {
    return;
  } else {
    double c = x[N - 1];
#pragma unroll
    for (int i = N - 2; i >= 0; i--) {
      double h, l;
      two_sum(x[i], c, h, l);
      x[i + 1] = l;
      c = h;
    }
    x[0] = c;
#pragma unroll
    for (int i = 1; i < N - 1; i++) {
      double h, l;
      two_sum(x[i], x[i + 1], h, l);
      x[i] = h;
      x[i + 1] = l;
    }
    // A zero limb above a nonzero one can survive both passes only for N >= 4;
    // shift such limbs up (integer selects, no FP64 work).
    if constexpr (N >= 4) {
#pragma unroll
      for (int p = 0; p < N - 2; p++) {
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
          bool z = is_zero(x[i]);
          double a = x[i], b = x[i + 1];
          x[i] = z ? b : a;
          x[i + 1] = z ? 0.0 : b;
        }
      }
    }
  }
}

// ------------------------------------------------------ leveled accumulator --

template <int L>
struct Acc {
  double s[L];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < L; i++) s[i] = 0.0;
  }
  __device__ __forceinline__ void set(const R<L> &c) {
#pragma unroll
    for (int i = 0; i < L; i++) s[i] = c.x[i];
  }

  // add v (a term of order u^LV) exactly into level LV, errors cascade down
  template <int LV>
  __device__ __forceinline__ void dep(double v) {
    if constexpr (LV >= L - 1) {
      s[L - 1] = __dadd_rn(s[L - 1], v);
    } else {
      double h, e;
      two_sum(s[LV], v, h, e);
      s[LV] = h;
      dep<LV + 1>(e);
    }
  }

  // s += a * b (NEG: s -= a * b; the sign is folded into the multiplies)
  template <bool NEG = false>
  __device__ __forceinline__ void add_prod(const R<L> &A, const R<L> &B) {
    const double *b = B.x;
    double a[L];
#pragma unroll
    for (int q = 0; q < L; q++) a[q] = NEG ? -A.x[q] : A.x[q];
    if constexpr (L == 2) {
      double p, e;
      two_prod(a[0], b[0], p, e);
      dep<0>(p);
      s[1] = __dadd_rn(s[1], e);
      s[1] = __fma_rn(a[0], b[1], s[1]);
      s[1] = __fma_rn(a[1], b[0], s[1]);
    } else if constexpr (L == 3) {
      double p00, e00, p01, e01, p10, e10;
      two_prod(a[0], b[0], p00, e00);
      two_prod(a[0], b[1], p01, e01);
      two_prod(a[1], b[0], p10, e10);
      dep<0>(p00);
      dep<1>(e00);
      dep<1>(p01);
      dep<1>(p10);
      s[2] = __dadd_rn(s[2], e01);
      s[2] = __dadd_rn(s[2], e10);
      s[2] = __fma_rn(a[0], b[2], s[2]);
      s[2] = __fma_rn(a[1], b[1], s[2]);
      s[2] = __fma_rn(a[2], b[0], s[2]);
    } else {
      static_assert(L == 4, "L must be 2, 3 or 4");
      double p00, e00, p01, e01, p10, e10, p02, e02, p11, e11, p20, e20;
      two_prod(a[0], b[0], p00, e00);
      two_prod(a[0], b[1], p01, e01);
      two_prod(a[1], b[0], p10, e10);
      two_prod(a[0], b[2], p02, e02);
      two_prod(a[1], b[1], p11, e11);
      two_prod(a[2], b[0], p20, e20);
      dep<0>(p00);
      dep<1>(e00);
      dep<1>(p01);
      dep<1>(p10);
      dep<2>(e01);
      dep<2>(e10);
      dep<2>(p02);
      dep<2>(p11);
      dep<2>(p20);
      s[3] = __dadd_rn(s[3], e02);
      s[3] = __dadd_rn(s[3], e11);
      s[3] = __dadd_rn(s[3], e20);
      s[3] = __fma_rn(a[0], b[3], s[3]);
      s[3] = __fma_rn(a[1], b[2], s[3]);
      s[3] = __fma_rn(a[2], b[1], s[3]);
      s[3] = __fma_rn(a[3], b[0], s[3]);
    }
  }

  // s = a * b for an empty accumulator (skips the TwoSums against zeros)
  __device__ __forceinline__ void set_prod(const R<L> &A, const R<L> &B) {
    const double *a = A.x, *b = B.x;
    if constexpr (L == 2) {
      two_prod(a[0], b[0], s[0], s[1]);
      s[1] = __fma_rn(a[0], b[1], s[1]);
      s[1] = __fma_rn(a[1], b[0], s[1]);
    } else if constexpr (L == 3) {
      double e01, e10, p01, p10;
      two_prod(a[0], b[0], s[0], s[1]);
      two_prod(a[0], b[1], p01, e01);
      two_prod(a[1], b[0], p10, e10);
      s[2] = e01;
      dep<1>(p01);
      dep<1>(p10);
      s[2] = __dadd_rn(s[2], e10);
      s[2] = __fma_rn(a[0], b[2], s[2]);
      s[2] = __fma_rn(a[1], b[1], s[2]);
      s[2] = __fma_rn(a[2], b[0], s[2]);
    } else {
      double p01, e01, p10, e10, p02, e02, p11, e11, p20, e20;
      two_prod(a[0], b[0], s[0], s[1]);
      two_prod(a[0], b[1], p01, e01);
      two_prod(a[1], b[0], p10, e10);
      two_prod(a[0], b[2], p02, e02);
      two_prod(a[1], b[1], p11, e11);
      two_prod(a[2], b[0], p20, e20);
      s[2] = e01;
      s[3] = e02;
      dep<1>(p01);
      dep<1>(p10);
      dep<2>(e10);
      dep<2>(p02);
      dep<2>(p11);
      dep<2>(p20);
      s[3] = __dadd_rn(s[3], e11);
      s[3] = __dadd_rn(s[3], e20);
      s[3] = __fma_rn(a[0], b[3], s[3]);
      s[3] = __fma_rn(a[1], b[2], s[3]);
      s[3] = __fma_rn(a[2], b[1], s[3]);
      s[3] = __fma_rn(a[3], b[0], s[3]);
    }
  }

  // s += q * b for a binary64 q
  __device__ __forceinline__ void add_prod1(double q, const R<L> &B) {
    const double *b = B.x;
    double p, e;
    two_prod(q, b[0], p, e);
    dep<0>(p);
    if constexpr (L == 2) {
      s[1] = __dadd_rn(s[1], e);
      s[1] = __fma_rn(q, b[1], s[1]);
    } else if constexpr (L == 3) {
      double p1, e1;
      two_prod(q, b[1], p1, e1);
      dep<1>(e);
      dep<1>(p1);
      s[2] = __dadd_rn(s[2], e1);
      s[2] = __fma_rn(q, b[2], s[2]);
    } else {
      double p1, e1, p2, e2;
      two_prod(q, b[1], p1, e1);
      two_prod(q, b[2], p2, e2);
      dep<1>(e);
      dep<1>(p1);
      dep<2>(e1);
      dep<2>(p2);
      s[3] = __dadd_rn(s[3], e2);
      s[3] = __fma_rn(q, b[3], s[3]);
    }
  }

  // s += c (an L-limb value, limb l deposited at level l)
  __device__ __forceinline__ void add(const R<L> &c) {
    dep<0>(c.x[0]);
    if constexpr (L >= 2) dep<1>(c.x[1]);
    if constexpr (L >= 3) dep<2>(c.x[2]);
    if constexpr (L >= 4) dep<3>(c.x[3]);
  }

  // s += sign * t (another accumulator, level by level)
  __device__ __forceinline__ void add_acc(const Acc<L> &t, bool negate) {
    dep<0>(negate ? flip(t.s[0]) : t.s[0]);
    if constexpr (L >= 2) dep<1>(negate ? flip(t.s[1]) : t.s[1]);
    if constexpr (L >= 3) dep<2>(negate ? flip(t.s[2]) : t.s[2]);
    if constexpr (L >= 4) dep<3>(negate ? flip(t.s[3]) : t.s[3]);
  }

  __device__ __forceinline__ R<L> result() const {
    R<L> r;
#pragma unroll
    for (int i = 0; i < L; i++) r.x[i] = s[i];
    renorm_n<L>(r.x);
    return r;
  }
};

// ------------------------------------------------------- real operations --

// Accurate addition: every limb of both operands is summed exactly on L
// levels plus one guard level, then renormalised and rounded to L limbs, so
// cancellation in the leading limbs keeps relative accuracy.
template <int L>
__device__ __forceinline__ R<L> r_add(const R<L> &a, const R<L> &b) {
  Acc<L + 1> t;
#pragma unroll
  for (int i = 0; i < L; i++) t.s[i] = a.x[i];
  t.s[L] = 0.0;
  t.template dep<0>(b.x[0]);
  if constexpr (L >= 2) t.template dep<1>(b.x[1]);
  if constexpr (L >= 3) t.template dep<2>(b.x[2]);
  if constexpr (L >= 4) t.template dep<3>(b.x[3]);
  renorm_n<L + 1>(t.s);
  R<L> r;
#pragma unroll
  for (int i = 0; i < L; i++) r.x[i] = t.s[i];
  return r;
}

template <int L>
__device__ __forceinline__ R<L> r_sub(const R<L> &a, const R<L> &b) {
  return r_add<L>(a, r_neg<L>(b));
}

template <int L>
__device__ __forceinline__ R<L> r_mul(const R<L> &a, const R<L> &b) {
  Acc<L> t;
  t.set_prod(a, b);
  return t.result();
}

// Long division: q_k = RN(r_k[0] / b[0]), r_{k+1} = r_k - q_k b (L levels),
// L+1 quotient digits renormalised to L limbs.
template <int L>
__device__ __forceinline__ R<L> r_div(const R<L> &a, const R<L> &b) {
  double q[L + 1];
  R<L> r = a;
#pragma unroll
  for (int k = 0; k <= L; k++) {
    q[k] = __ddiv_rn(r.x[0], b.x[0]);
    if (k < L) {
      Acc<L> t;
      t.set(r);
      t.add_prod1(flip(q[k]), b);
      r = t.result();
    }
  }
  renorm_n<L + 1>(q);
  R<L> z;
#pragma unroll
  for (int i = 0; i < L; i++) z.x[i] = q[i];
  return z;
}

// Lexicographic comparison of renormalised values (nonoverlapping limbs):
// returns true if a > b.  Integer compares only.
template <int L>
__device__ __forceinline__ bool r_gt(const R<L> &a, const R<L> &b) {
#pragma unroll
  for (int i = 0; i < L; i++) {
    long long ka = order_key(a.x[i]), kb = order_key(b.x[i]);
    if (ka != kb) return ka > kb;
  }
  return false;
}

// ---------------------------------------------------- complex operations --

template <int L>
__device__ __forceinline__ Z<L> z_add(const Z<L> &a, const Z<L> &b) {
  Z<L> r;
  r.re = r_add<L>(a.re, b.re);
  r.im = r_add<L>(a.im, b.im);
  return r;
}

template <int L>
__device__ __forceinline__ Z<L> z_sub(const Z<L> &a, const Z<L> &b) {
  Z<L> r;
  r.re = r_sub<L>(a.re, b.re);
  r.im = r_sub<L>(a.im, b.im);
  return r;
}

// Eq. (1), each part accumulated on the leveled accumulator:
// Re = Re a Re b - Im a Im b,  Im = Re a Im b + Im a Re b.
template <int L>
__device__ __forceinline__ Z<L> z_mul(const Z<L> &a, const Z<L> &b) {
  Z<L> r;
  Acc<L> t;
  t.set_prod(a.re, b.re);
  t.template add_prod<true>(a.im, b.im);
  r.re = t.result();
  t.set_prod(a.re, b.im);
  t.add_prod(a.im, b.re);
  r.im = t.result();
  return r;
}

// Eq. (2): t1 = Re a Re b, t2 = Im a Im b, Re = t1 - t2,
// Im = (Re a + Im a)(Re b + Im b) - (t1 + t2), every step rounded to L limbs.
template <int L>
__device__ __forceinline__ Z<L> z_mul3m(const Z<L> &a, const Z<L> &b) {
  R<L> t1 = r_mul<L>(a.re, b.re);
  R<L> t2 = r_mul<L>(a.im, b.im);
  R<L> t3 = r_mul<L>(r_add<L>(a.re, a.im), r_add<L>(b.re, b.im));
  Z<L> r;
  r.re = r_sub<L>(t1, t2);
  r.im = r_sub<L>(t3, r_add<L>(t1, t2));
  return r;
}

// |a|^2 = Re a^2 + Im a^2
template <int L>
__device__ __forceinline__ R<L> z_norm2(const Z<L> &a) {
  Acc<L> t;
  t.set_prod(a.re, a.re);
  t.add_prod(a.im, a.im);
  return t.result();
}

// 1/d by Newton's iteration r <- r + r (1 - d r) from the binary64
// reciprocal of the leading limb: one step reaches double-double accuracy,
// a second step (in L-limb arithmetic) triple/quad-double accuracy.  Shorter
// dependent chains than long division, which matters on the latency-bound
// panel path.
template <int L>
__device__ __forceinline__ R<L> r_recip(const R<L> &d) {
  const double r0 = __ddiv_rn(1.0, d.x[0]);
  // e = 1 - d r0 (leveled, L limbs), then r = r0 + r0 e
  Acc<L> t;
  t.zero();
  t.s[0] = 1.0;
  t.add_prod1(flip(r0), d);
  const R<L> e = t.result();
  Acc<L> u;
  u.zero();
  u.s[0] = r0;
  u.add_prod1(r0, e);
  R<L> r = u.result();
  if constexpr (L >= 3) {
    Acc<L> t2;
    t2.zero();
    t2.s[0] = 1.0;
    t2.template add_prod<true>(d, r);
    const R<L> e2 = t2.result();
    Acc<L> u2;
    u2.set(r);
    u2.add_prod(r, e2);
    r = u2.result();
  }
  return r;
}

// 1/(a + bi) = (a - bi) / (a^2 + b^2)
template <int L>
__device__ __forceinline__ Z<L> z_inv(const Z<L> &a) {
  const R<L> rinv = r_recip<L>(z_norm2<L>(a));
  Z<L> r;
  r.re = r_mul<L>(a.re, rinv);
  r.im = r_neg<L>(r_mul<L>(a.im, rinv));
  return r;
}

// 1/p by Newton's method from a binary64 seed: a shorter chain of FP64
// instructions than conj(p)/|p|^2 with a multi-component reciprocal (the
// pivot reciprocal of the panel, which every column waits for).
//   seed   r0 = conj(p0) RN(1/RN(|p0|^2)), p0 = a0 + b0 i the leading limbs:
//          relative error a few units of 2^-53;
//   resid  e = 1 - p r0, of order 2^-52.  Its leading terms cancel:
//          a0 Re r0 and -b0 Im r0 lie in [0, 1] and add up to about 1, so
//          1 minus the larger one is split exactly into a rounded value and
//          its error (Fast2Sum), and the rounded value nearly cancels the
//          smaller one; a0 Im r0 and b0 Re r0 are nearly opposite, so their
//          sum is exact.  The TwoProd and Fast2Sum errors and the products
//          with the lower limbs are added in binary64: absolute error about
//          2^-105;
//   finish r = r0 (1 + e + e^2) (1/p = r0 / (1 - e)), the correction in
//          binary64 and added to r0 with TwoSum: relative error of order
//          |e|^3 + 2^-105.
// The real and imaginary parts of e and of r are independent chains (the
// panel runs them on two SMSPs).  L >= 3 adds one Newton step in L-limb
// arithmetic (rcp_prod, rcp_resid_l, rcp_newton below).
struct RcpSeed {
  double rr, ri;  // Re r0, Im r0
};

__device__ __forceinline__ RcpSeed rcp_seed(double a0, double b0) {
  const double d = __fma_rn(a0, a0, __dmul_rn(b0, b0));
  const double q = __drcp_rn(d);
  return {__dmul_rn(a0, q), flip(__dmul_rn(b0, q))};
}

// Re e = 1 - (a Re r0 - b Im r0)
template <int L>
__device__ __forceinline__ double rcp_resid_re(const R<L> &a, const R<L> &b, const RcpSeed &s) {
  double p1, e1, p2, e2;
  two_prod(a.x[0], s.rr, p1, e1);  // p1 >= 0
  two_prod(b.x[0], s.ri, p2, e2);  // p2 <= 0
  // the larger of p1 and -p2 (integer compare of nonnegative doubles) is
  // subtracted from 1 first, its rounding error kept (Fast2Sum: 1 is not
  // smaller in magnitude); the result then nearly cancels the other product
  const bool big1 = __double_as_longlong(p1) >= __double_as_longlong(flip(p2));
  const double c = big1 ? __dsub_rn(1.0, p1) : __dadd_rn(1.0, p2);
  const double cl = big1 ? __dsub_rn(__dsub_rn(1.0, c), p1) : __dadd_rn(__dsub_rn(1.0, c), p2);
  const double s0 = big1 ? __dadd_rn(c, p2) : __dsub_rn(c, p1);
  double t = __dadd_rn(__dsub_rn(e2, e1), cl);
  t = __fma_rn(flip(a.x[1]), s.rr, t);
  t = __fma_rn(b.x[1], s.ri, t);
  return __dadd_rn(s0, t);
}

// Im e = -(a Im r0 + b Re r0)
template <int L>
__device__ __forceinline__ double rcp_resid_im(const R<L> &a, const R<L> &b, const RcpSeed &s) {
  double q1, f1, q2, f2;
  two_prod(a.x[0], s.ri, q1, f1);
  two_prod(b.x[0], s.rr, q2, f2);
  const double s0 = __dadd_rn(q1, q2);  // exact: q1 and q2 are nearly opposite
  double t = __dadd_rn(f1, f2);
  t = __fma_rn(a.x[1], s.ri, t);
  t = __fma_rn(b.x[1], s.rr, t);
  return flip(__dadd_rn(s0, t));
}

// One part of r0 (1 + e + e^2): IM = false the real part, true the imaginary
// part, as a two-limb value (limbs 2 .. L-1 zero).
template <int L, bool IM>
__device__ __forceinline__ R<L> rcp_finish(const RcpSeed &s, double er, double ei) {
  // u = e + e^2
  const double ur = __dadd_rn(er, __fma_rn(er, er, flip(__dmul_rn(ei, ei))));
  const double ui = __fma_rn(__dadd_rn(er, er), ei, ei);
  // delta = r0 u
  const double d = IM ? __fma_rn(s.rr, ui, __dmul_rn(s.ri, ur)) : __fma_rn(s.rr, ur, flip(__dmul_rn(s.ri, ui)));
  R<L> r = r_zero<L>();
  two_sum(IM ? s.ri : s.rr, d, r.x[0], r.x[1]);
  return r;
}

// L >= 3: one Newton step from the two-limb r (rcp_finish) to L limbs.
//   e = 1 - p r with the four real products P_xy = p_x r_y (x, y in re, im;
//   p_x L limbs, r_y two) summed on leveled accumulators: e is of order
//   2^-104 and exact to about 2^-212 after its leading terms cancel, so two
//   limbs of it suffice;
//   r' = r + r (e + e^2): the products r e (two-limb by two-limb, TwoProd on
//   the leading limbs) and the second-order term added to r's limbs on the
//   levels of an L-limb accumulator: relative error of order |e|^3 + 2^-53L.
// The products, the two parts of e and the two parts of r' are independent
// chains (the TD / QD panel spreads them over warps).
template <int L>
__device__ __forceinline__ void rcp_prod(Acc<L> &P, const R<L> &px, double y0, double y1) {
  P.zero();
  P.add_prod1(y0, px);
  P.add_prod1(y1, px);
}

// Re e = 1 - P_rr + P_ii (IM false), Im e = -(P_ri + P_ir) (IM true).  The
// leading levels cancel down to about 2^-105, where one renormalisation
// leaves its two leading limbs overlapping (the pair then misses terms of
// order 2^-159); a second pass makes them nonoverlapping (the pair within
// about 2^-211 of the sum).
template <int L, bool IM>
__device__ __forceinline__ R<L> rcp_resid_l(const Acc<L> &Pa, const Acc<L> &Pb) {
  Acc<L> t;
  t.zero();
  if (!IM) t.s[0] = 1.0;
  t.add_acc(Pa, true);
  t.add_acc(Pb, IM);
  R<L> e = t.result();
  renorm_n<L>(e.x);
  return e;
}

// part IM of r' = r + r e + r e^2 (r, e: two limbs per part)
template <int L, bool IM>
__device__ __forceinline__ R<L> rcp_newton(const double (&r)[4], const double (&e)[4]) {
  const double rr0 = r[0], rr1 = r[1], ri0 = r[2], ri1 = r[3];
  const double er0 = e[0], er1 = e[1], ei0 = e[2], ei1 = e[3];
  Acc<L> u;
  u.zero();
  u.s[0] = IM ? ri0 : rr0;
  u.s[1] = IM ? ri1 : rr1;
  double p, q;
  // leading products: Re: rr0 er0 - ri0 ei0, Im: rr0 ei0 + ri0 er0
  two_prod(rr0, IM ? ei0 : er0, p, q);
  u.template dep<2>(p);
  u.template dep<3>(q);
  two_prod(IM ? ri0 : flip(ri0), IM ? er0 : ei0, p, q);
  u.template dep<2>(p);
  u.template dep<3>(q);
  // the remaining first-order terms and e^2 = (er0^2 - ei0^2) + 2 er0 ei0 i
  double t = 0.0;
  if (!IM) {
    t = __fma_rn(rr0, er1, t);
    t = __fma_rn(rr1, er0, t);
    t = __fma_rn(flip(ri0), ei1, t);
    t = __fma_rn(flip(ri1), ei0, t);
    t = __fma_rn(rr1, er1, t);
    t = __fma_rn(flip(ri1), ei1, t);
  } else {
    t = __fma_rn(rr0, ei1, t);
    t = __fma_rn(rr1, ei0, t);
    t = __fma_rn(ri0, er1, t);
    t = __fma_rn(ri1, er0, t);
    t = __fma_rn(rr1, ei1, t);
    t = __fma_rn(ri1, er1, t);
  }
  const double e2r = __fma_rn(er0, er0, flip(__dmul_rn(ei0, ei0)));
  const double e2i = __dmul_rn(__dadd_rn(er0, er0), ei0);
  if (!IM) {
    t = __fma_rn(rr0, e2r, t);
    t = __fma_rn(flip(ri0), e2i, t);
  } else {
    t = __fma_rn(rr0, e2i, t);
    t = __fma_rn(ri0, e2r, t);
  }
  u.template dep<3>(t);
  return u.result();
}

template <int L>
__device__ __forceinline__ Z<L> z_inv_newton(const Z<L> &p) {
  const RcpSeed s = rcp_seed(p.re.x[0], p.im.x[0]);
  const double er = rcp_resid_re<L>(p.re, p.im, s);
  const double ei = rcp_resid_im<L>(p.re, p.im, s);
  Z<L> r;
  r.re = rcp_finish<L, false>(s, er, ei);
  r.im = rcp_finish<L, true>(s, er, ei);
  if constexpr (L >= 3) {
    const double r2[4] = {r.re.x[0], r.re.x[1], r.im.x[0], r.im.x[1]};
    Acc<L> Prr, Pii, Pri, Pir;
    rcp_prod<L>(Prr, p.re, r2[0], r2[1]);
    rcp_prod<L>(Pii, p.im, r2[2], r2[3]);
    rcp_prod<L>(Pri, p.re, r2[2], r2[3]);
    rcp_prod<L>(Pir, p.im, r2[0], r2[1]);
    const R<L> e_re = rcp_resid_l<L, false>(Prr, Pii);
    const R<L> e_im = rcp_resid_l<L, true>(Pri, Pir);
    const double e2[4] = {e_re.x[0], e_re.x[1], e_im.x[0], e_im.x[1]};
    r.re = rcp_newton<L, false>(r2, e2);
    r.im = rcp_newton<L, true>(r2, e2);
  }
  return r;
}

// a / b = a conj(b) / |b|^2 with both real parts divided by long division
template <int L>
__device__ __forceinline__ Z<L> z_div(const Z<L> &a, const Z<L> &b) {
  Z<L> num = z_mul<L>(a, z_conj<L>(b));
  R<L> d = z_norm2<L>(b);
  Z<L> r;
  r.re = r_div<L>(num.re, d);
  r.im = r_div<L>(num.im, d);
  return r;
}

// cabs1(z) = |Re z| + |Im z| (the pivot key; LAPACK's izamax measure)
template <int L>
__device__ __forceinline__ R<L> z_abs1(const Z<L> &a) {
  return r_add<L>(r_abs<L>(a.re), r_abs<L>(a.im));
}

// Pivot key: cabs1 with its two leading limbs made a TwoSum pair, so that
// limb 0 is the rounded value of limbs 0 + 1 and the lexicographic comparison
// of r_gt orders keys by value (exactly for DD; for TD/QD up to ties in the
// third limb).
template <int L>
__device__ __forceinline__ R<L> pivot_key(const Z<L> &a) {
  R<L> k = z_abs1<L>(a);
  double h, l;
  two_sum(k.x[0], k.x[1], h, l);
  k.x[0] = h;
  k.x[1] = l;
  return k;
}

// c - a b on the leveled accumulator (one renormalisation per part)
template <int L>
__device__ __forceinline__ Z<L> z_fms(const Z<L> &c, const Z<L> &a, const Z<L> &b) {
  Z<L> r;
  Acc<L> t;
  t.set(c.re);
  t.template add_prod<true>(a.re, b.re);
  t.template add_prod<false>(a.im, b.im);
  r.re = t.result();
  t.set(c.im);
  t.template add_prod<true>(a.re, b.im);
  t.template add_prod<true>(a.im, b.re);
  r.im = t.result();
  return r;
}

// ---------------------------------------------------------- plane access --

// A complex L-limb matrix: 2L column-major planes, plane (c,l) at
// p + (c*L + l)*ps, element (i,j) at offset j*ld + i.
struct View {
  double *p;
  int64_t ld;
  int64_t ps;
};

template <int L>
__device__ __forceinline__ Z<L> ldz(const View &v, int64_t i, int64_t j) {
  Z<L> z;
  const int64_t o = j * v.ld + i;
#pragma unroll
  for (int l = 0; l < L; l++) {
    z.re.x[l] = v.p[(int64_t)l * v.ps + o];
    z.im.x[l] = v.p[(int64_t)(L + l) * v.ps + o];
  }
  return z;
}

template <int L>
__device__ __forceinline__ void stz(const View &v, int64_t i, int64_t j, const Z<L> &z) {
  const int64_t o = j * v.ld + i;
#pragma unroll
  for (int l = 0; l < L; l++) {
    v.p[(int64_t)l * v.ps + o] = z.re.x[l];
    v.p[(int64_t)(L + l) * v.ps + o] = z.im.x[l];
  }
}

}  // namespace mclu
