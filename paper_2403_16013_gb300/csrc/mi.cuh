// mi.cuh - complex multi-component arithmetic on the integer pipes.
//
// The DD/TD/QD operations of Sec. 2 (complex multiply-subtract, product,
// cabs1, reciprocal) computed as exact fixed-point sums of the binary64 limbs
// and limb products of the operands, rounded once to L limbs (greedy round to
// nearest even per limb): one rounding per operation, like the oracle's
// exact-then-round operations, using integer instructions only.
//
// They are exposed through mclu_vec_op (ops 20-23) and are not used by the
// factorisation: on GB300 an FP64 instruction holds its SMSP for 64 cycles,
// but the integer emulation of a limb product and its placement costs about
// 25 times the instructions of the TwoProd/TwoSum forms of mc.cuh, and in the
// cooperative panel these versions measured two times slower.
//
// Frame: W 32-bit words, two's complement, bit 0 of weight 2^E.  E is set
// 32 W - 4 bits below an upper bound 2^T of the terms, so the sum cannot
// overflow; a term's bits below 2^E are truncated, which leaves an error
// below 2^(T - 32W + 8) -- far below the last limb (W = 6 / 8 / 9 for
// DD / TD / QD keeps 70 or more bits below the L limbs).  Limb products
// a_i b_j with i + j > L lie below the last limb's rounding and are left
// out.
#pragma once

#include "mc.cuh"

namespace mclu {
namespace mi {

template <int L>
struct Frame;
template <>
struct Frame<2> {
  static constexpr int W = 6;
};
template <>
struct Frame<3> {
  static constexpr int W = 8;
};
template <>
struct Frame<4> {
  static constexpr int W = 9;
};

// |x| = m 2^e with m < 2^53 (m = 0 for zero)
struct Lb {
  uint64_t m;
  int e;
  bool neg;
};

__device__ __forceinline__ Lb lb(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  Lb r;
  r.neg = (b >> 63) != 0;
  r.m = (b & 0xFFFFFFFFFFFFFULL) | (ex ? (1ULL << 52) : 0ULL);
  r.e = (ex ? ex : 1) - 1075;
  return r;
}

// exclusive bound exponent of |x|: |x| < 2^top (a very small value for zero)
__device__ __forceinline__ int top_of(const Lb &a) { return a.m ? a.e + 64 - __clzll((long long)a.m) : -100000; }

template <int W>
struct Fx {
  uint32_t w[W];
  int E;

  // frame for terms bounded by 2^T in total
  __device__ __forceinline__ void init(int T) {
    E = T + 4 - 32 * W;
#pragma unroll
    for (int i = 0; i < W; i++) w[i] = 0u;
  }

  // += (neg ? -1 : 1) (hi:lo) 2^e, (hi:lo) < 2^124, bits below 2^E dropped
  __device__ __forceinline__ void add(uint64_t lo, uint64_t hi, int e, bool neg) {
    const int s = e - E;
    // left placement (s >= 0): (hi:lo) << bs at word ws
    const int sl = s > 0 ? s : 0;
    const int ws = sl >> 5, bs = sl & 31;
    const uint64_t l2 = lo << bs;
    const uint64_t h2 = (hi << bs) | (bs ? (lo >> (64 - bs)) : 0ULL);
    const uint32_t t4l = bs ? (uint32_t)(hi >> (64 - bs)) : 0u;
    // right placement (s < 0): (hi:lo) >> r at word 0
    const int r = s < 0 ? min(-s, 127) : 0;
    const uint64_t rlo = r == 0 ? lo : (r < 64 ? ((lo >> r) | (hi << (64 - r))) : (hi >> (r - 64)));
    const uint64_t rhi = r < 64 ? (hi >> r) : 0ULL;
    const bool right = s < 0;
    const uint64_t plo = right ? rlo : l2, phi = right ? rhi : h2;
    const uint32_t t0 = (uint32_t)plo, t1 = (uint32_t)(plo >> 32), t2 = (uint32_t)phi, t3 = (uint32_t)(phi >> 32);
    const uint32_t t4 = right ? 0u : t4l;
    const int base = right ? 0 : ws;
    const uint32_t inv = neg ? 0xFFFFFFFFu : 0u;
    uint64_t carry = neg ? 1ULL : 0ULL;
#pragma unroll
    for (int i = 0; i < W; i++) {
      const int k = i - base;
      uint32_t v = (k == 0) ? t0 : (k == 1) ? t1 : (k == 2) ? t2 : (k == 3) ? t3 : (k == 4) ? t4 : 0u;
      v ^= inv;
      const uint64_t t = (uint64_t)w[i] + v + carry;
      w[i] = (uint32_t)t;
      carry = t >> 32;
    }
  }

  __device__ __forceinline__ void add_limb(const Lb &a, bool flip) { add(a.m, 0ULL, a.e, a.neg != flip); }

  // += a b (flip: -= a b), the exact 106-bit product of two limbs
  __device__ __forceinline__ void add_prod(const Lb &a, const Lb &b, bool flip) {
    const uint64_t lo = a.m * b.m, hi = __umul64hi(a.m, b.m);
    add(lo, hi, a.e + b.e, (a.neg != b.neg) != flip);
  }

  // Round the frame to L limbs (greedy round to nearest even).
  template <int L>
  __device__ __forceinline__ void round(R<L> &out) const {
    uint32_t Rw[W];
    bool neg = (int32_t)w[W - 1] < 0;
    {
      const uint32_t inv = neg ? 0xFFFFFFFFu : 0u;
      uint64_t carry = neg ? 1ULL : 0ULL;
#pragma unroll
      for (int i = 0; i < W; i++) {
        const uint64_t t = (uint64_t)(w[i] ^ inv) + carry;
        Rw[i] = (uint32_t)t;
        carry = t >> 32;
      }
    }
#pragma unroll
    for (int l = 0; l < L; l++) {
      int tw = -1;
#pragma unroll
      for (int i = 0; i < W; i++) tw = Rw[i] ? i : tw;
      uint32_t h = 0, m = 0, q = 0, below = 0;
#pragma unroll
      for (int i = 0; i < W; i++) {
        h = (i == tw) ? Rw[i] : h;
        m = (i == tw - 1) ? Rw[i] : m;
        q = (i == tw - 2) ? Rw[i] : q;
        below |= (i < tw - 2) ? Rw[i] : 0u;
      }
      const bool zero = tw < 0;
      const int z = __clz(h | (zero ? 1u : 0u));
      const uint32_t W2 = z ? (h << z) | (m >> (32 - z)) : h;
      const uint32_t W1 = z ? (m << z) | (q >> (32 - z)) : m;
      const uint32_t W0 = z ? (q << z) : q;
      const uint64_t mwin = ((uint64_t)W2 << 21) | (W1 >> 11);  // 53 bits below the leading one
      const uint32_t rbit = (W1 >> 10) & 1u;
      const uint32_t sticky = (W1 & 0x3FFu) | W0 | below;
      const int top_bit = 32 * tw + 31 - z;
      const int lo = top_bit - 52;  // frame position of the mantissa LSB
      const bool big = lo > 0;
      const uint64_t small = (uint64_t)Rw[0] | ((uint64_t)Rw[1] << 32);  // whole value when lo <= 0
      const uint64_t mant = big ? mwin : small;
      const bool up = big && rbit && (sticky || (mant & 1ULL));
      int ex = (big ? lo : 0) + E;
      uint64_t mm = mant + (up ? 1ULL : 0ULL);
      const bool cout = (mm >> 53) != 0;
      mm = cout ? (mm >> 1) : mm;
      ex += cout ? 1 : 0;
      const int msb = 63 - __clzll((long long)(mm | 1ULL));
      mm <<= (52 - msb);
      ex -= (52 - msb);
      const unsigned long long bits = ((unsigned long long)(neg ? 1 : 0) << 63) |
                                      ((unsigned long long)(ex + 52 + 1023) << 52) | (mm & 0xFFFFFFFFFFFFFULL);
      out.x[l] = zero ? 0.0 : __longlong_as_double((long long)bits);
      // remainder below lo, complemented within lo bits if rounded up
      const int lw = big ? (lo >> 5) : -1, lbit = lo & 31;
      const uint32_t lmask = lbit ? ((1u << lbit) - 1u) : 0u;
      uint64_t carry = 1;
#pragma unroll
      for (int i = 0; i < W; i++) {
        const uint32_t keep = (i < lw) ? Rw[i] : (i == lw ? (Rw[i] & lmask) : 0u);
        const uint32_t cinv = (i < lw) ? ~Rw[i] : (i == lw ? (~Rw[i] & lmask) : 0u);
        const uint64_t t = (uint64_t)cinv + carry;
        const uint32_t comp = (i < lw) ? (uint32_t)t : (i == lw ? ((uint32_t)t & lmask) : 0u);
        carry = (i < lw) ? (t >> 32) : 0;
        Rw[i] = up ? comp : keep;
      }
      neg = up ? !neg : neg;
    }
  }
};

template <int L>
struct ZL {  // the limbs of a complex value, unpacked once
  Lb re[L], im[L];
};

template <int L>
__device__ __forceinline__ ZL<L> unpack(const Z<L> &a) {
  ZL<L> r;
#pragma unroll
  for (int q = 0; q < L; q++) {
    r.re[q] = lb(a.re.x[q]);
    r.im[q] = lb(a.im.x[q]);
  }
  return r;
}

// frame += (flip ? -1 : 1) x y over the limb products of order <= L
template <int L, int W>
__device__ __forceinline__ void add_mul(Fx<W> &f, const Lb (&x)[L], const Lb (&y)[L], bool flip) {
#pragma unroll
  for (int i = 0; i < L; i++)
#pragma unroll
    for (int j = 0; j < L; j++)
      if (i + j <= L) f.add_prod(x[i], y[j], flip);
}

template <int L>
__device__ __forceinline__ int prod_top(const Lb (&x)[L], const Lb (&y)[L]) {
  return top_of(x[0]) + top_of(y[0]) + 1;
}

// c - a b (Eq. 1 form: Re = c_re - a_re b_re + a_im b_im, Im = c_im - a_re b_im - a_im b_re)
template <int L>
__device__ __forceinline__ Z<L> zi_fms(const Z<L> &c, const ZL<L> &a, const ZL<L> &b) {
  constexpr int W = Frame<L>::W;
  Z<L> r;
  Lb cl[L];
  {
#pragma unroll
    for (int q = 0; q < L; q++) cl[q] = lb(c.re.x[q]);
    Fx<W> f;
    f.init(max(top_of(cl[0]) + 1, max(prod_top<L>(a.re, b.re), prod_top<L>(a.im, b.im))) + 2);
#pragma unroll
    for (int q = 0; q < L; q++) f.add_limb(cl[q], false);
    add_mul<L, W>(f, a.re, b.re, true);
    add_mul<L, W>(f, a.im, b.im, false);
    f.template round<L>(r.re);
  }
  {
#pragma unroll
    for (int q = 0; q < L; q++) cl[q] = lb(c.im.x[q]);
    Fx<W> f;
    f.init(max(top_of(cl[0]) + 1, max(prod_top<L>(a.re, b.im), prod_top<L>(a.im, b.re))) + 2);
#pragma unroll
    for (int q = 0; q < L; q++) f.add_limb(cl[q], false);
    add_mul<L, W>(f, a.re, b.im, true);
    add_mul<L, W>(f, a.im, b.re, true);
    f.template round<L>(r.im);
  }
  return r;
}

// a b (Eq. 1)
template <int L>
__device__ __forceinline__ Z<L> zi_mul(const ZL<L> &a, const ZL<L> &b) {
  constexpr int W = Frame<L>::W;
  Z<L> r;
  {
    Fx<W> f;
    f.init(max(prod_top<L>(a.re, b.re), prod_top<L>(a.im, b.im)) + 2);
    add_mul<L, W>(f, a.re, b.re, false);
    add_mul<L, W>(f, a.im, b.im, true);
    f.template round<L>(r.re);
  }
  {
    Fx<W> f;
    f.init(max(prod_top<L>(a.re, b.im), prod_top<L>(a.im, b.re)) + 2);
    add_mul<L, W>(f, a.re, b.im, false);
    add_mul<L, W>(f, a.im, b.re, false);
    f.template round<L>(r.im);
  }
  return r;
}

// cabs1(a) = |Re a| + |Im a|, rounded to L limbs (a canonical key: limbwise
// lexicographic order is value order)
template <int L>
__device__ __forceinline__ R<L> zi_abs1(const ZL<L> &a) {
  constexpr int W = Frame<L>::W;
  Fx<W> f;
  f.init(max(top_of(a.re[0]), top_of(a.im[0])) + 2);
  const bool fr = a.re[0].neg, fi = a.im[0].neg;
#pragma unroll
  for (int q = 0; q < L; q++) {
    f.add_limb(a.re[q], fr);
    f.add_limb(a.im[q], fi);
  }
  R<L> k;
  f.template round<L>(k);
  return k;
}

// 1/a = conj(a) / |a|^2: D = |a|^2 rounded to L limbs, x0 = 1/D0 (binary64),
// then Newton steps x <- x + x (1 - D x), each residual 1 - D x and each
// update formed exactly in a frame and rounded to L limbs (the precision
// doubles per step: two steps for DD and TD, three for QD), then
// Re = Re(a) x, Im = -Im(a) x.
template <int L>
__device__ __forceinline__ Z<L> zi_inv(const ZL<L> &a) {
  constexpr int W = Frame<L>::W;
  constexpr int ITER = L == 4 ? 3 : 2;
  R<L> D;
  {
    Fx<W> f;
    f.init(max(prod_top<L>(a.re, a.re), prod_top<L>(a.im, a.im)) + 2);
    add_mul<L, W>(f, a.re, a.re, false);
    add_mul<L, W>(f, a.im, a.im, false);
    f.template round<L>(D);
  }
  Lb dl[L], xl[L];
#pragma unroll
  for (int q = 0; q < L; q++) dl[q] = lb(D.x[q]);
  R<L> x;
#pragma unroll
  for (int q = 0; q < L; q++) x.x[q] = 0.0;
  x.x[0] = 1.0 / D.x[0];
#pragma unroll
  for (int it = 0; it < ITER; it++) {
#pragma unroll
    for (int q = 0; q < L; q++) xl[q] = lb(x.x[q]);
    R<L> e;
    {
      Fx<W> f;
      f.init(2 + 2);  // |1| and |D x| are below 2
      f.add(1ULL << 52, 0ULL, -52, false);
      add_mul<L, W>(f, dl, xl, true);
      f.template round<L>(e);
    }
    Lb el[L];
#pragma unroll
    for (int q = 0; q < L; q++) el[q] = lb(e.x[q]);
    Fx<W> f;
    f.init(top_of(xl[0]) + 2);
#pragma unroll
    for (int q = 0; q < L; q++) f.add_limb(xl[q], false);
    add_mul<L, W>(f, xl, el, false);
    f.template round<L>(x);
  }
#pragma unroll
  for (int q = 0; q < L; q++) xl[q] = lb(x.x[q]);
  Z<L> r;
  {
    Fx<W> f;
    f.init(prod_top<L>(a.re, xl) + 2);
    add_mul<L, W>(f, a.re, xl, false);
    f.template round<L>(r.re);
  }
  {
    Fx<W> f;
    f.init(prod_top<L>(a.im, xl) + 2);
    add_mul<L, W>(f, a.im, xl, true);
    f.template round<L>(r.im);
  }
  return r;
}

}  // namespace mi
}  // namespace mclu
