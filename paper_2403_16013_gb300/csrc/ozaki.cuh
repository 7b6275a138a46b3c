// ozaki.cuh - Ozaki-scheme complex multi-component matrix product on the
// GB300 tensor cores (tcgen05, bf16 inputs, fp32 accumulation in TMEM).
//
// The Ozaki scheme (Sec. 2.3, Fig. 4 of the paper) splits the operands of a
// matrix product into slices whose pairwise products are computed without
// rounding by a short-precision GEMM and then summed in multi-component
// arithmetic.  The paper uses binary64 DGEMM slices on a CPU.  On GB300 the
// FP64 pipe and the INT8 tensor path are slow, so this file uses the bf16
// tensor-core path instead and keeps everything around it off the FP64 pipe:
//
//  Split (integer ALU only).  Row i of A gets the power-of-two scale
//  2^Ea_i with |A_ij| < 2^(Ea_i - 1) for all j (column j of B: 2^Eb_j).  Each
//  element's limbs are truncated toward zero into the two's-complement
//  integer T = sum_l trunc(x_l 2^(beta S - E)), |T| < 2^(beta S - 1), and T is
//  written in S balanced base-2^beta digits a_0 .. a_{S-1} (|a_p| <= 2^(beta-1)),
//  each exactly representable in bf16: x ~ 2^E sum_p a_p 2^(-beta (p+1)).
//  The complex product is made real ("realified"): A_r = [Re A | Im A] and
//  B_r has the columns [Re B; -Im B] (real part of the product) and
//  [Im B; Re B] (imaginary part), interleaved, so one real GEMM gives Eq. (1).
//
//  Products (tcgen05.mma kind::f16, M = 128, N = 32 or 16, K = 16).  Slice
//  pairs (p, q) with p + q <= S - 1 are kept; pair products with the same
//  p + q = d go to one TMEM fp32 accumulator D_d.  Every digit product is an
//  integer of at most 2^12 (beta = 7), a K = 64 chunk has at most S pairs per
//  diagonal, and chunks_per_fold chunks accumulate before the epilogue reads
//  them, so every partial sum is an integer of at most 2^24: the fp32
//  accumulation is exact.
//
//  Epilogue (integer ALU only).  F = sum_d D_d 2^(beta (S-1-d)) is folded into
//  a register-resident fixed-point integer; the product is
//  P = F 2^(Ea + Eb - beta (S+1)).  C - P is formed exactly in a wider integer
//  frame and rounded back to L binary64 limbs (round to nearest, greedy).
//
// Error: truncating the limbs costs at most L units of 2^(E - beta S) per
// element and the dropped pairs (p + q >= S) less than S K 2^(2beta - 2)
// units of 2^(Ea + Eb - beta (S+1)); with beta S >= 53 L + 6 both stay below
// the L-limb rounding level relative to max|A_i.| max|B_.j|.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>

#include "mc.cuh"

namespace mclu {
namespace oz {

template <int L>
struct Cfg;
// beta: digit bits; S: slices; N: realified columns per tile; FW: 32-bit words of
// the fold accumulator F; TW: words of the split integer T; RW: words of the
// final C - P frame; GS: diagonals pre-combined in int64 (GS diagonals of at
// most 2^24, shifted by beta each, stay below 2^60); EW: epilogue warps
// (16 for DD's 32-column tiles, 8 for the 16-column TD/QD tiles: measured);
// EF: fold each group of diagonals as soon as its products are done (1) or
// all groups after the last one (0) -- measured faster for DD, slower for
// TD/QD.
template <>
struct Cfg<2> {
  static constexpr int BETA = 7, S = 16, N = 32, FW = 5, TW = 4, RW = 6, GS = 6, EW = 16, EF = 1;
};
template <>
struct Cfg<3> {
  static constexpr int BETA = 7, S = 24, N = 16, FW = 7, TW = 6, RW = 8, GS = 6, EW = 8, EF = 0;
};
template <>
struct Cfg<4> {
  static constexpr int BETA = 7, S = 32, N = 16, FW = 9, TW = 8, RW = 10, GS = 6, EW = 8, EF = 0;
};

// Slices kept per operand when the caller asks for the default (ozaki_slices
// = 0): the full S of the precision.
template <int L>
constexpr int default_slices() {
  return Cfg<L>::S;
}

constexpr int KC = 64;         // realified K per chunk (32 complex columns of A)

// K chunks whose products accumulate in TMEM before the epilogue folds them:
// the largest c with c KC S 2^(2 beta - 2) <= 2^24, so that every partial
// sum of a diagonal (at most S digit products of at most 2^(2 beta - 2) per K
// index) is an integer of at most 2^24 and the fp32 accumulation stays exact.
// DD (beta 7, S 16): 4 chunks, i.e. a whole trailing update of nb = 128; TD,
// QD: 2.
template <int L>
__host__ __device__ constexpr int chunks_per_fold() {
  return (int)((1LL << 24) / ((long long)KC * Cfg<L>::S * (1LL << (2 * Cfg<L>::BETA - 2))));
}
static_assert(chunks_per_fold<2>() == 4 && chunks_per_fold<3>() == 2 && chunks_per_fold<4>() == 2,
              "fold groups of K chunks");
constexpr int NB_MAX = KC / 2; // complex panel width per chunk
constexpr int BM = 128;        // tile rows (TMEM lanes)
constexpr int NST = 4;         // A pipeline stages
constexpr int NSB = 2;         // B buffers (one K chunk's slices each)
// warp 0: A producer, warp 1: TMEM owner and MMA issuer, warp 2: B producer,
// then EW epilogue warps
template <int L>
constexpr int threads_of() {
  return 32 * (3 + Cfg<L>::EW);
}
constexpr int TMEM_COLS = 512;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz: bound on every wait

// ------------------------------------------------------------ PTX wrappers --

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused with 128B swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D fp32, A/B bf16, both K-major, M = 128, N.
template <int N>
__device__ __forceinline__ uint32_t umma_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
// The same for a runtime N (a multiple of 16, 16 .. 256).
__device__ __forceinline__ uint32_t umma_idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[NC]);

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

template <>
__device__ __forceinline__ void tmem_ld<4>(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------- multiword integers --
// Little-endian arrays of 32-bit words, two's complement.

// Unpacked binary64: x = (-1)^neg * mant * 2^e, mant < 2^53 (0 for x = 0).
struct Unpacked {
  uint64_t mant;
  int e;
  bool neg;
};

__device__ __forceinline__ Unpacked unpack(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  Unpacked u;
  u.neg = (b >> 63) != 0;
  u.mant = (b & 0xFFFFFFFFFFFFFULL) | (ex ? (1ULL << 52) : 0ULL);
  u.e = (ex ? ex : 1) - 1075;
  return u;
}

// floor(log2|x|) of a nonzero normal double (integer bit view).
__device__ __forceinline__ int ilogb_bits(double x) {
  return (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7FF) - 1023;
}

// acc += sign * trunc(mant * 2^s) for a runtime shift s (acc has W words).
template <int W>
__device__ __forceinline__ void add_shifted(uint32_t (&acc)[W], uint64_t mant, int s, bool neg) {
  if (mant == 0) return;
  uint32_t t0, t1, t2;
  int ws;
  if (s < 0) {
    if (s <= -64) return;
    const uint64_t v = mant >> (-s);
    t0 = (uint32_t)v;
    t1 = (uint32_t)(v >> 32);
    t2 = 0;
    ws = 0;
  } else {
    ws = s >> 5;
    const int bs = s & 31;
    const uint64_t lo = mant << bs;                       // low 64 bits
    const uint64_t hi = bs ? (mant >> (64 - bs)) : 0ULL;  // bits above 64
    t0 = (uint32_t)lo;
    t1 = (uint32_t)(lo >> 32);
    t2 = (uint32_t)hi;
  }
  // two's complement add (or subtract) of the 3-word value placed at word ws
  uint64_t carry = neg ? 1ULL : 0ULL;
#pragma unroll
  for (int w = 0; w < W; w++) {
    uint32_t v = (w == ws) ? t0 : (w == ws + 1) ? t1 : (w == ws + 2) ? t2 : 0u;
    if (neg) v = ~v;
    const uint64_t t = (uint64_t)acc[w] + v + carry;
    acc[w] = (uint32_t)t;
    carry = t >> 32;
  }
}

// --------------------------------------------------------------- split --

// Power-of-two scales: Ea_i over row i of the m x k block A (both parts, all
// columns), Eb_j over column j of the k x n block B.  E = max floor(log2
// |leading limb|) + 2, so |x| < 2^(E-1).

// Balanced base-2^BETA digits of x / 2^E (S digits, most significant first).
template <int L>
__device__ __forceinline__ void digits_of(const double (&x)[L], int E, float (&dg)[Cfg<L>::S]) {
  constexpr int BETA = Cfg<L>::BETA, S = Cfg<L>::S, TW = Cfg<L>::TW;
  uint32_t T[TW];
#pragma unroll
  for (int w = 0; w < TW; w++) T[w] = 0;
#pragma unroll
  for (int l = 0; l < L; l++) {
    if (is_zero(x[l])) continue;
    const Unpacked u = unpack(x[l]);
    add_shifted<TW>(T, u.mant, u.e + BETA * S - E, u.neg);
  }
  constexpr uint32_t MASK = (1u << BETA) - 1, HALF = 1u << (BETA - 1);
#pragma unroll
  for (int p = S - 1; p >= 0; p--) {
    const uint32_t b = T[0] & MASK;
    const int d = (b >= HALF && p > 0) ? (int)b - (1 << BETA) : (int)b;
    dg[p] = (float)(p > 0 ? d : (int)(T[0]));  // top digit: the remaining signed value
    // T = (T - d) >> BETA  (arithmetic)
    if (p > 0) {
      uint64_t carry = (d < 0) ? 1ULL : 0ULL;  // subtracting a negative digit adds 2^BETA - b
      // T + (b >= HALF ? 2^BETA : 0) - b  ==  T - d : clear the low bits, add 2^BETA if negative digit
      T[0] &= ~MASK;
      if (carry) {
        uint64_t c = 1ULL << BETA;
#pragma unroll
        for (int w = 0; w < TW; w++) {
          const uint64_t t = (uint64_t)T[w] + (uint32_t)c;
          T[w] = (uint32_t)t;
          c = t >> 32;
        }
      }
#pragma unroll
      for (int w = 0; w < TW - 1; w++) T[w] = (T[w] >> BETA) | (T[w + 1] << (32 - BETA));
      T[TW - 1] = (uint32_t)((int32_t)T[TW - 1] >> BETA);
    }
  }
}

// Slice layout.  A: [chunk][S][Mpad][64] bf16 for 32 complex columns per
// chunk: columns 0..31 hold Re, 32..63 Im.  B: [chunk][S][Npad][64] with
// Npad >= 2n: row 2j = [Re B_.j ; -Im B_.j], row 2j+1 = [Im B_.j ; Re B_.j]
// (K index: 0..31 first half, 32..63 second).

// Scales and slices of both operands in one launch: warp v < Mpad takes row
// v of A (its scale Ea over the whole row, then its slices chunk by chunk,
// one column a lane), warp Mpad + j column j of B (Eb, then its slices, one
// row a lane).  Padding rows and columns get zero slices and scale 0.
template <int L>
__global__ void k_oz_split_ab(View A, View B, int64_t m, int64_t n, int64_t k, int *Ea, int *Eb,
                              __nv_bfloat16 *as, __nv_bfloat16 *bs, int64_t Mpad, int64_t Npad, int nchunks, int Se) {
  constexpr int S = Cfg<L>::S;
  const int lane = threadIdx.x & 31;
  const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool aside = v < Mpad;
  const int64_t idx = aside ? v : v - Mpad;  // row of A or column of B
  if (!aside && 2 * idx >= Npad) return;
  const View X = aside ? A : B;
  const bool real = aside ? idx < m : idx < n;
  // element t of this row (A) or column (B)
  auto off = [&](int64_t t) -> int64_t { return aside ? t * X.ld + idx : idx * X.ld + t; };
  int e = -100000;
  if (real) {
    for (int64_t t = lane; t < k; t += 32) {
      const int64_t o = off(t);
      const double re = X.p[o], im = X.p[(int64_t)L * X.ps + o];
      if (!is_zero(re)) e = max(e, ilogb_bits(re));
      if (!is_zero(im)) e = max(e, ilogb_bits(im));
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, d));
  const int E = (e == -100000) ? 0 : e + 2;
  if (lane == 0) (aside ? Ea : Eb)[idx] = E;
  for (int c = 0; c < nchunks; c++) {
    const int64_t t = (int64_t)c * NB_MAX + lane;
    const bool ok = real && t < k;
    if (aside) {
#pragma unroll
      for (int part = 0; part < 2; part++) {
        double x[L];
#pragma unroll
        for (int l = 0; l < L; l++) x[l] = ok ? X.p[(int64_t)(part * L + l) * X.ps + off(t)] : 0.0;
        float dg[S];
        digits_of<L>(x, E, dg);
        __nv_bfloat16 *o = as + (((int64_t)c * S) * Mpad + idx) * KC + part * NB_MAX + lane;
#pragma unroll
        for (int p = 0; p < S; p++)
          if (p < Se) o[(int64_t)p * Mpad * KC] = __float2bfloat16_rn(dg[p]);
      }
    } else {
      float dre[S], dim[S];
      double x[L];
#pragma unroll
      for (int l = 0; l < L; l++) x[l] = ok ? X.p[(int64_t)l * X.ps + off(t)] : 0.0;
      digits_of<L>(x, E, dre);
#pragma unroll
      for (int l = 0; l < L; l++) x[l] = ok ? X.p[(int64_t)(L + l) * X.ps + off(t)] : 0.0;
      digits_of<L>(x, E, dim);
      __nv_bfloat16 *o0 = bs + (((int64_t)c * S) * Npad + 2 * idx) * KC;
      __nv_bfloat16 *o1 = o0 + KC;
#pragma unroll
      for (int q = 0; q < S; q++) {
        if (q >= Se) break;
        const int64_t so = (int64_t)q * Npad * KC;
        o0[so + lane] = __float2bfloat16_rn(dre[q]);
        o0[so + NB_MAX + lane] = __float2bfloat16_rn(-dim[q]);
        o1[so + lane] = __float2bfloat16_rn(dim[q]);
        o1[so + NB_MAX + lane] = __float2bfloat16_rn(dre[q]);
      }
    }
  }
}

// ------------------------------------------------------ final C - P step --

// Word idx of a register array (select chain, no dynamic indexing).
template <int W>
__device__ __forceinline__ uint32_t word_at(const uint32_t (&F)[W], int idx, uint32_t fill) {
  uint32_t r = fill;
#pragma unroll
  for (int w = 0; w < W; w++) r = (w == idx) ? F[w] : r;
  return r;
}

// F += G * 2^SHIFT for a signed 64-bit G with |G| < 2^60 (compile-time shift).
template <int W, int SHIFT>
__device__ __forceinline__ void fold64(uint32_t (&F)[W], long long G) {
  constexpr int WS = SHIFT / 32, BS = SHIFT % 32;
  const uint32_t sx = G < 0 ? 0xFFFFFFFFu : 0u;
  // G << BS as a 96-bit two's complement value (w0, w1, w2)
  const unsigned long long ug = (unsigned long long)G;
  const uint32_t g0 = (uint32_t)ug, g1 = (uint32_t)(ug >> 32);
  const uint32_t w0 = BS ? (g0 << BS) : g0;
  const uint32_t w1 = BS ? ((g1 << BS) | (g0 >> (32 - BS))) : g1;
  const uint32_t w2 = BS ? ((sx << BS) | (g1 >> (32 - BS))) : sx;
  uint64_t carry = 0;
#pragma unroll
  for (int w = WS; w < W; w++) {
    const uint32_t add = (w == WS) ? w0 : (w == WS + 1) ? w1 : (w == WS + 2) ? w2 : sx;
    const uint64_t t = (uint64_t)F[w] + add + carry;
    F[w] = (uint32_t)t;
    carry = t >> 32;
  }
}

// Per-thread scratch in shared memory, interleaved so that the threads of a
// warp touch consecutive words (no bank conflicts).  Runtime-indexed word
// accesses go here (load/store pipe) instead of register select chains.
struct Scratch {
  uint32_t *p;
  int stride;
  __device__ __forceinline__ uint32_t &operator[](int w) const { return p[w * stride]; }
};

// acc (RW words, two's complement, registers) += sign * trunc(mant * 2^s)
// with the runtime placement done through the scratch.
template <int RW>
__device__ __forceinline__ void add_limb(uint32_t (&acc)[RW], uint64_t mant, int s, bool neg, const Scratch &sc) {
  if (mant == 0) return;
  uint32_t t0, t1, t2;
  int ws;
  if (s < 0) {
    if (s <= -64) return;
    const uint64_t v = mant >> (-s);
    t0 = (uint32_t)v;
    t1 = (uint32_t)(v >> 32);
    t2 = 0;
    ws = 0;
  } else {
    ws = s >> 5;
    const int bs = s & 31;
    const uint64_t lo = mant << bs;
    t0 = (uint32_t)lo;
    t1 = (uint32_t)(lo >> 32);
    t2 = bs ? (uint32_t)(mant >> (64 - bs)) : 0u;
  }
#pragma unroll
  for (int w = 0; w < RW + 2; w++) sc[w] = 0u;
  sc[ws] = t0;
  sc[ws + 1] = t1;
  sc[ws + 2] = t2;
  uint64_t carry = neg ? 1ULL : 0ULL;
#pragma unroll
  for (int w = 0; w < RW; w++) {
    uint32_t v = sc[w];
    if (neg) v = ~v;
    const uint64_t t = (uint64_t)acc[w] + v + carry;
    acc[w] = (uint32_t)t;
    carry = t >> 32;
  }
}

// out = C - F 2^eF (BETA) or F 2^eF, rounded to L limbs (greedy round to
// nearest even).  The remainder is kept in sign-magnitude form; every limb
// reads a 96-bit window at the leading word, rounds, and keeps the bits below
// the rounding position (complemented if it rounded up).
template <int L, int FW, int RW, bool BETA>
__device__ __forceinline__ void finish2(const uint32_t (&F)[FW], int eF, const double (&c)[L], double (&out)[L],
                                        const Scratch &sc) {
  const bool fneg = (int32_t)F[FW - 1] < 0;
  int topF = -1;
#pragma unroll
  for (int w = 0; w < FW; w++) {
    const uint32_t v = fneg ? ~F[w] : F[w];
    if (v) topF = 32 * w + 31 - __clz(v);
  }
  int top = (topF >= 0) ? eF + topF + 1 : -100000;
  if (BETA && !is_zero(c[0])) top = max(top, ilogb_bits(c[0]) + 2);
  if (top == -100000) {
#pragma unroll
    for (int l = 0; l < L; l++) out[l] = 0.0;
    return;
  }
  top += 2;
  const int lsb = max(eF, top - (32 * RW - 2));
  uint32_t R[RW];
  if (lsb == eF) {  // common case: F enters the frame unshifted
    const uint32_t sx = fneg ? 0xFFFFFFFFu : 0u;
    uint64_t carry = BETA ? 1ULL : 0ULL;  // R = -F (BETA) or F
#pragma unroll
    for (int w = 0; w < RW; w++) {
      const uint32_t v = (w < FW) ? F[w] : sx;
      const uint64_t t = (uint64_t)(BETA ? ~v : v) + carry;
      R[w] = (uint32_t)t;
      carry = t >> 32;
    }
  } else {  // C dominates: F shifted right into C's frame (truncation below lsb)
#pragma unroll
    for (int w = 0; w < RW; w++) R[w] = 0;
    const int s = lsb - eF, ws = s >> 5, bs = s & 31;
    const uint32_t sx = fneg ? 0xFFFFFFFFu : 0u;
    uint64_t carry = BETA ? 1ULL : 0ULL;
#pragma unroll
    for (int w = 0; w < RW; w++) {
      const uint32_t lo = word_at<FW>(F, w + ws, sx);
      const uint32_t hi = word_at<FW>(F, w + ws + 1, sx);
      const uint32_t v = bs ? ((lo >> bs) | (hi << (32 - bs))) : lo;
      const uint64_t t = (uint64_t)R[w] + (uint32_t)(BETA ? ~v : v) + carry;
      R[w] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  if (BETA) {
#pragma unroll
    for (int l = 0; l < L; l++) {
      if (is_zero(c[l])) continue;
      const Unpacked u = unpack(c[l]);
      add_limb<RW>(R, u.mant, u.e - lsb, u.neg, sc);
    }
  }
  // sign-magnitude
  bool neg = (int32_t)R[RW - 1] < 0;
  {
    uint64_t carry = neg ? 1ULL : 0ULL;
#pragma unroll
    for (int w = 0; w < RW; w++) {
      const uint64_t t = (uint64_t)(neg ? ~R[w] : R[w]) + carry;
      R[w] = (uint32_t)t;
      carry = t >> 32;
    }
  }
#pragma unroll
  for (int l = 0; l < L; l++) {
    int tw = -1;
#pragma unroll
    for (int w = 0; w < RW; w++)
      if (R[w]) tw = w;
    if (tw < 0) {
      out[l] = 0.0;
      continue;
    }
    // scratch: words of |R| and prefix ORs (sticky below the window)
    uint32_t orb = 0;
#pragma unroll
    for (int w = 0; w < RW; w++) {
      sc[w] = R[w];
      sc[RW + w] = orb;  // OR of words [0, w)
      orb |= R[w];
    }
    const uint32_t h = sc[tw];
    const uint32_t m = tw >= 1 ? sc[tw - 1] : 0u;
    const uint32_t q = tw >= 2 ? sc[tw - 2] : 0u;
    const uint32_t below = tw >= 2 ? sc[RW + tw - 2] : 0u;
    const int z = __clz(h);  // h != 0
    // 96-bit window (h:m:q) << z: leading bit at window bit 95
    const uint32_t W2 = z ? (h << z) | (m >> (32 - z)) : h;
    const uint32_t W1 = z ? (m << z) | (q >> (32 - z)) : m;
    const uint32_t W0 = z ? (q << z) : q;
    uint64_t mant = ((uint64_t)W2 << 21) | (W1 >> 11);          // bits 95..43 (53 bits)
    const uint32_t rbit = (W1 >> 10) & 1u;                      // bit 42
    const uint32_t sticky = (W1 & 0x3FFu) | W0 | below;         // bits 41..0 and lower words
    const int top_bit = 32 * tw + 31 - z;                       // position of the leading bit in R
    const int lo = top_bit - 52;                                // position of the mantissa LSB
    bool up = false;
    if (lo > 0) {
      up = rbit && (sticky || (mant & 1ULL));
    } else {  // the whole value fits: exact
      mant = 0;
#pragma unroll
      for (int w = 0; w < 2 && w < RW; w++) mant |= (uint64_t)R[w] << (32 * w);
    }
    int ex = (lo > 0 ? lo : 0) + lsb;  // value = mant * 2^ex
    uint64_t mm = mant + (up ? 1ULL : 0ULL);
    if (mm >> 53) {
      mm >>= 1;
      ex += 1;
    }
    {  // normalise (only the exact small case can have fewer than 53 bits)
      const int msb = 63 - __clzll((long long)mm);
      mm <<= (52 - msb);
      ex -= (52 - msb);
    }
    const unsigned long long bits = ((unsigned long long)(neg ? 1 : 0) << 63) |
                                    ((unsigned long long)(ex + 52 + 1023) << 52) | (mm & 0xFFFFFFFFFFFFFULL);
    out[l] = __longlong_as_double((long long)bits);
    // remainder: the bits of |R| below lo, complemented within lo bits if rounded up
    if (lo <= 0) {
#pragma unroll
      for (int w = 0; w < RW; w++) R[w] = 0;
    } else {
      const int lw = lo >> 5, lb = lo & 31;
      const uint32_t lmask = lb ? ((1u << lb) - 1u) : 0u;
#pragma unroll
      for (int w = 0; w < RW; w++) R[w] = (w < lw) ? R[w] : (w == lw ? (R[w] & lmask) : 0u);
      if (up) {  // 2^lo - rest
        uint64_t carry = 1;
#pragma unroll
        for (int w = 0; w < RW; w++) {
          const uint32_t inv = (w < lw) ? ~R[w] : (w == lw ? (~R[w] & lmask) : 0u);
          const uint64_t t = (uint64_t)inv + carry;
          R[w] = (w < lw) ? (uint32_t)t : (w == lw ? ((uint32_t)t & lmask) : 0u);
          carry = (w < lw) ? (t >> 32) : 0;
        }
        neg = !neg;
      }
    }
  }
}

// Fold diagonals D0 .. D0+G-1 (G = min(GS, S - D0)) of the TMEM accumulators
// into F: G_c = sum_t D_{D0+t} 2^(beta (G-1-t)) exactly in int64, then one
// multiword addition at shift beta (S - D0 - G).  Group g of diagonals is
// complete once the products of A slices 0 .. D0+G-1 are done: the warp
// waits for that group's commit barrier (lane 0 waits, the outcome is
// broadcast so the warp stays converged for the .sync.aligned loads).
template <int L, int NH, int D0>
__device__ __forceinline__ bool fold_diagonals(uint32_t (&F)[NH][Cfg<L>::FW], uint32_t tbase, uint64_t *bar_grp,
                                               uint32_t parity, int lane, int Se) {
  constexpr int S = Cfg<L>::S, N = Cfg<L>::N, BETA = Cfg<L>::BETA, FW = Cfg<L>::FW;
  constexpr int GS = Cfg<L>::GS;
  constexpr int G = (S - D0) < GS ? (S - D0) : GS;
  if (D0 >= Se) return true;  // diagonals of dropped slice pairs: nothing was accumulated
  if (Cfg<L>::EF || D0 == 0) {
    int got = 0;
    if (lane == 0) got = mbar_wait(&bar_grp[Cfg<L>::EF ? D0 / GS : (Se - 1) / GS], parity) ? 1 : 0;
    got = __shfl_sync(0xffffffffu, got, 0);
    if (!got) return false;
    __syncwarp();
    tc_fence_after();
  }
  long long g[NH];
#pragma unroll
  for (int cc = 0; cc < NH; cc++) g[cc] = 0;
#pragma unroll
  for (int t = 0; t < G; t++) {
    uint32_t v[NH];
#pragma unroll
    for (int cc = 0; cc < NH; cc++) v[cc] = 0u;  // 0.0f: a diagonal past the last kept one
    if (D0 + t < Se) {                          // warp-uniform
      tmem_ld<NH>(tbase + (uint32_t)((D0 + t) * N), v);
      tmem_wait_ld();
    }
#pragma unroll
    for (int cc = 0; cc < NH; cc++) g[cc] = g[cc] * (1LL << BETA) + (long long)__float2int_rz(__uint_as_float(v[cc]));
  }
#pragma unroll
  for (int cc = 0; cc < NH; cc++) fold64<FW, BETA *(S - D0 - G)>(F[cc], g[cc]);
  if constexpr (D0 + G < S)
    return fold_diagonals<L, NH, D0 + G>(F, tbase, bar_grp, parity, lane, Se);
  else
    return true;
}

// ---------------------------------------------------------------- GEMM --

// C (m x n complex) = C - A B (BETA) or A B, from the slices of A (rows) and
// B (columns) cut by k_oz_split_ab.  Persistent: one CTA per SM
// walks the (row tile, column tile) grid.  Warp 0 lane 0: TMA producer of
// the A slices (NST-stage ring).  Warp 1: TMEM owner and MMA issuer (lane 0).
// Warp 2 lane 0: TMA producer of the B slices (NSB chunk buffers, so the next
// chunk loads during the current one's MMAs).  Warps 3 .. 2+EW: epilogue.
template <int L, bool BETA>
__global__ void __launch_bounds__(threads_of<L>(), 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, View C, int64_t m,
              int64_t n, int nchunks, int Mpad, int Npad, const int *Ea, const int *Eb, int *status, int Se) {
  using CF = Cfg<L>;
  constexpr int S = CF::S, N = CF::N, BETA_B = CF::BETA, FW = CF::FW, RW = CF::RW;
  constexpr int CPF = chunks_per_fold<L>();
  constexpr int A_BYTES = BM * KC * 2;  // 16 KB
  constexpr int B_TILE = N * KC * 2;    // 4 KB or 2 KB (multiples of 1024 B)
  constexpr int B_BYTES = S * B_TILE;
  constexpr int EPI_WARPS = Cfg<L>::EW;
  constexpr int NPART = EPI_WARPS / 4;   // epilogue warps per TMEM lane quarter
  constexpr int NH = N / NPART;          // columns per epilogue thread
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sB = base;                  // NSB buffers of B_BYTES
  uint8_t *sA = base + NSB * B_BYTES;
  __shared__ __align__(8) uint64_t bar_afull[NST], bar_aempty[NST];
  __shared__ __align__(8) uint64_t bar_bfull[NSB], bar_bempty[NSB], bar_accempty;
  constexpr int NGRP = (S + CF::GS - 1) / CF::GS;  // fold groups of diagonals
  __shared__ __align__(8) uint64_t bar_grp[NGRP];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_err;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; i++) {
      mbar_init(&bar_afull[i], 1);
      mbar_init(&bar_aempty[i], 1);
    }
    for (int i = 0; i < NSB; i++) {
      mbar_init(&bar_bfull[i], 1);
      mbar_init(&bar_bempty[i], 1);
    }
    for (int i = 0; i < NGRP; i++) mbar_init(&bar_grp[i], 1);
    mbar_init(&bar_accempty, EPI_WARPS);
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  // Tiles in column-major order: consecutive CTAs take the row tiles of one
  // column tile, so a wave reads a few B tiles and all of A (a few tens of
  // MB at n = 4096), which stay in L2; in row-major order each B tile came
  // back only after a whole row of tiles and was read again from DRAM.
  const int64_t mt = (m + BM - 1) / BM, nt = Npad / N, total = mt * nt;

  if (warp == 2) {
    if (lane == 0) {  // -------------------------------------- B producer
      // the Se B slices of each K chunk into one of NSB buffers: the next
      // chunk's slices load while the MMAs of the current chunk run
      uint32_t r = 0;
      for (int64_t t = blockIdx.x; t < total && !s_err; t += gridDim.x) {
        const int ntile = (int)(t / mt);  // column-major tile order (see above)
        for (int c = 0; c < nchunks; c++, r++) {
          const int b = (int)(r % NSB);
          if (!mbar_wait(&bar_bempty[b], ((r / NSB) & 1) ^ 1)) {
            s_err = 1;
            break;
          }
          mbar_expect_tx(&bar_bfull[b], (uint32_t)(Se * B_TILE));
          for (int q = 0; q < Se; q++)
            tma_load_2d(sB + b * B_BYTES + q * B_TILE, &tmB, &bar_bfull[b], 0, (c * S + q) * Npad + ntile * N);
        }
      }
      // drain: wait for the last loads of every buffer to land before leaving
      for (int i = 0; i < NSB && r > 0; i++) {
        const uint32_t it = r - 1 - i;
        if ((int)it < 0) break;
        mbar_wait(&bar_bfull[it % NSB], (it / NSB) & 1);
      }
    }
  } else if (warp == 0) {
    if (lane == 0) {  // -------------------------------------- A producer
      uint32_t a_it = 0;
      for (int64_t t = blockIdx.x; t < total && !s_err; t += gridDim.x) {
        const int mtile = (int)(t % mt);
        for (int c = 0; c < nchunks; c++) {
          for (int p = 0; p < Se; p++, a_it++) {
            const int st = a_it % NST;
            const uint32_t ph = (a_it / NST) & 1;
            if (!mbar_wait(&bar_aempty[st], ph ^ 1)) {
              s_err = 2;
              break;
            }
            mbar_expect_tx(&bar_afull[st], A_BYTES);
            tma_load_2d(sA + st * A_BYTES, &tmA, &bar_afull[st], 0, (c * S + p) * Mpad + mtile * BM);
          }
          if (s_err) break;
        }
      }
      // drain: wait for the last loads of every stage to land before leaving
      for (int i = 0; i < NST && a_it > 0; i++) {
        const uint32_t it = a_it - 1 - i;
        if ((int)it < 0) break;
        mbar_wait(&bar_afull[it % NST], (it / NST) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // --------------------------------------------- MMA
      uint32_t a_it = 0, r = 0, g = 0;  // r: K chunks (B pipeline), g: fold groups (TMEM)
      for (int64_t t = blockIdx.x; t < total && !s_err; t += gridDim.x) {
        for (int c = 0; c < nchunks; c++, r++) {
          // a fold group of CPF chunks accumulates in TMEM: its first chunk
          // overwrites the diagonals once the epilogue has read the previous
          // group, its last chunk signals the diagonal groups
          const bool gfirst = c % CPF == 0, glast = c % CPF == CPF - 1 || c == nchunks - 1;
          const int b = (int)(r % NSB);
          if ((gfirst && !mbar_wait(&bar_accempty, (g & 1) ^ 1)) || !mbar_wait(&bar_bfull[b], (r / NSB) & 1)) {
            s_err = 3;
            break;
          }
          tc_fence_after();
          for (int p = 0; p < Se; p++, a_it++) {
            const int st = a_it % NST;
            if (!mbar_wait(&bar_afull[st], (a_it / NST) & 1)) {
              s_err = 4;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + st * A_BYTES);
            // The Se kept B slices lie back to back in one K-major,
            // 128-byte-swizzled layout (each a multiple of 1024 bytes), so A_p
            // times slices 0 .. Se-1-p is one product with (Se - p) N columns,
            // landing on the TMEM column blocks of diagonals p .. Se-1 (split
            // at 256 columns).
            const int ncols = (Se - p) * N;
            for (int c0 = 0; c0 < ncols; c0 += 256) {
              const int nn = min(256, ncols - c0);
              const uint32_t b0 = smem_u32(sB + b * B_BYTES) + (uint32_t)(c0 * KC * 2);
              const uint32_t d = tmem + (uint32_t)(p * N + c0);
              const uint32_t idesc = umma_idesc_n(nn);
#pragma unroll
              for (int ks = 0; ks < KC / 16; ks++)
                umma_bf16(d, umma_desc(a0 + ks * 32), umma_desc(b0 + ks * 32), idesc,
                          (p > 0 || ks > 0 || !gfirst) ? 1u : 0u);
            }
            umma_commit(&bar_aempty[st]);
            // diagonals of the group ending at p are complete: let the
            // epilogue fold them while the later slices multiply
            if (glast && ((p + 1) % CF::GS == 0 || p == Se - 1)) umma_commit(&bar_grp[p / CF::GS]);
          }
          if (s_err) break;
          umma_commit(&bar_bempty[b]);
          if (glast) g++;
        }
      }
    }
  } else {  // ---------------------------------------------------- epilogue
    // TMEM lanes [32 (warp % 4), + 32) are the ones a warp may access
    const int quarter = warp & 3, half = (warp - 3) >> 2;  // half: column part 0 .. NPART-1
    const int row = quarter * 32 + lane;
    const int etid = threadIdx.x - 96;  // 0 .. 32 * EPI_WARPS - 1
    const Scratch sc{reinterpret_cast<uint32_t *>(sA + NST * A_BYTES) + etid, EPI_WARPS * 32};
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * NH);
    uint32_t g = 0;  // fold groups
    const int ngroups = (nchunks + CPF - 1) / CPF;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
      const int mtile = (int)(t % mt), ntile = (int)(t / mt);
      uint32_t F[NH][FW];
#pragma unroll
      for (int cc = 0; cc < NH; cc++)
#pragma unroll
        for (int w = 0; w < FW; w++) F[cc][w] = 0;
      bool ok = true;
      for (int gi = 0; gi < ngroups; gi++, g++) {
        // diagonal d sits in TMEM columns [d N, d N + N), summed over the
        // group's K chunks; each group of diagonals is folded as soon as its
        // commit barrier completes
        if (!fold_diagonals<L, NH, 0>(F, tbase, bar_grp, g & 1, lane, Se)) {
          if (lane == 0) s_err = 5;
          ok = false;
          break;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_accempty);
      }
      if (!ok) break;
      // C - P for this thread's row and columns
      const int64_t i = (int64_t)mtile * BM + row;
      if (i < m) {
        const int ea = Ea[i];
#pragma unroll 1
        for (int cc = 0; cc < NH; cc++) {
          const int64_t jj = (int64_t)ntile * N + half * NH + cc;
          const int64_t j = jj >> 1;
          const int part = (int)(jj & 1);
          if (j >= n) continue;
          const int eF = ea + Eb[j] - BETA_B * (S + 1);
          double cv[L], ov[L];
          double *cp = C.p + (int64_t)(part * L) * C.ps + j * C.ld + i;
#pragma unroll
          for (int l = 0; l < L; l++) cv[l] = BETA ? cp[(int64_t)l * C.ps] : 0.0;
          uint32_t f[FW];  // column cc of F, selected without dynamic register indexing
#pragma unroll
          for (int w = 0; w < FW; w++) {
            uint32_t v = 0;
#pragma unroll
            for (int c2 = 0; c2 < NH; c2++) v = (c2 == cc) ? F[c2][w] : v;
            f[w] = v;
          }
          finish2<L, FW, RW, BETA>(f, eF, cv, ov, sc);
#pragma unroll
          for (int l = 0; l < L; l++) cp[(int64_t)l * C.ps] = ov[l];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
  if (threadIdx.x == 0 && s_err) atomicOr(status, 1 << s_err);
}


// ---------------------------------------------------------------- host --

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// 2-D bf16 tensor map over `rows` rows of KC elements (128 B), box KC x box_rows,
// 128-byte swizzle (matches the UMMA K-major SW128 layout).
inline int make_map(CUtensorMap *map, void *base, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return (int)cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)KC, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)KC * 2};
  cuuint32_t box[2] = {(cuuint32_t)KC, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

template <int L>
struct Sizes {
  int64_t nchunks, Mpad, Npad;
  size_t a_bytes, b_bytes, total;
};

template <int L>
inline Sizes<L> sizes(int64_t m, int64_t n, int64_t k) {
  Sizes<L> z;
  z.nchunks = (k + NB_MAX - 1) / NB_MAX;
  z.Mpad = rup(m > 0 ? m : 1, BM);
  z.Npad = rup(2 * (n > 0 ? n : 1), Cfg<L>::N);
  z.a_bytes = (size_t)z.nchunks * Cfg<L>::S * z.Mpad * KC * 2;
  z.b_bytes = (size_t)z.nchunks * Cfg<L>::S * z.Npad * KC * 2;
  z.total = z.a_bytes + z.b_bytes + (size_t)(z.Mpad + z.Npad + 64) * sizeof(int) + 1024;
  return z;
}

template <int L>
inline size_t ws_bytes(int64_t m, int64_t n, int64_t k) {
  return sizes<L>(m, n, k).total;
}

inline int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// Scales and slices of A (m x k, rows) and B (k x n, columns) into ws.
template <int L>
int split(View A, View B, int64_t m, int64_t n, int64_t k, void *ws, cudaStream_t s, void (*note)(),
          int Se = Cfg<L>::S) {
  const Sizes<L> z = sizes<L>(m, n, k);
  char *w = (char *)ws;
  __nv_bfloat16 *as = (__nv_bfloat16 *)w;
  __nv_bfloat16 *bs = (__nv_bfloat16 *)(w + z.a_bytes);
  int *Ea = (int *)(w + z.a_bytes + z.b_bytes);
  int *Eb = Ea + z.Mpad;
  const int64_t warps = z.Mpad + z.Npad / 2;
  k_oz_split_ab<L><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(A, B, m, n, k, Ea, Eb, as, bs, z.Mpad, z.Npad,
                                                                        (int)z.nchunks, Se);
  note();
  return (int)cudaGetLastError();
}

// C = C - A B (beta) or A B with the Ozaki scheme.  ws: ws_bytes<L>(m, n, k);
// status: device int, OR-ed with a nonzero code if a pipeline wait timed out.
// Se: slices kept per operand (1 .. S; pairs p + q <= Se - 1 are multiplied).
template <int L>
int gemm(bool beta, View A, View B, View C, int64_t m, int64_t n, int64_t k, void *ws, int *status, cudaStream_t s,
         void (*note)(), int Se = Cfg<L>::S) {
  if (Se < 1 || Se > Cfg<L>::S) return (int)cudaErrorInvalidValue;
  if (m <= 0 || n <= 0) return 0;
  if (k == 0) {  // nothing to multiply (and nothing to split): C unchanged (beta) or zero
    if (!beta) {
      for (int pl = 0; pl < 2 * L; pl++) {
        cudaError_t e = cudaMemset2DAsync(C.p + (int64_t)pl * C.ps, C.ld * sizeof(double), 0, m * sizeof(double), n, s);
        if (e != cudaSuccess) return (int)e;
      }
    }
    return 0;
  }
  const Sizes<L> z = sizes<L>(m, n, k);
  int rc = split<L>(A, B, m, n, k, ws, s, note, Se);
  if (rc) return rc;
  char *w = (char *)ws;
  int *Ea = (int *)(w + z.a_bytes + z.b_bytes);
  int *Eb = Ea + z.Mpad;
  CUtensorMap tmA, tmB;
  rc = make_map(&tmA, w, (uint64_t)z.nchunks * Cfg<L>::S * z.Mpad, BM);
  if (rc) return rc;
  rc = make_map(&tmB, w + z.a_bytes, (uint64_t)z.nchunks * Cfg<L>::S * z.Npad, Cfg<L>::N);
  if (rc) return rc;
  constexpr int A_BYTES = BM * KC * 2, B_BYTES = Cfg<L>::S * Cfg<L>::N * KC * 2;
  constexpr int SCR_BYTES = (2 * Cfg<L>::RW + 2) * Cfg<L>::EW * 32 * 4;  // epilogue scratch
  constexpr int THREADS = threads_of<L>();
  // at least ~116 KB so that a single CTA (and its 512 TMEM columns) fits per SM
  const int smem = std::max(NSB * B_BYTES + NST * A_BYTES + SCR_BYTES + 1024, 116 * 1024);
  static_assert(NSB * B_BYTES + NST * A_BYTES + SCR_BYTES + 1024 <= 227 * 1024, "shared memory of k_oz_gemm");
  const int64_t tiles = ((m + BM - 1) / BM) * (z.Npad / Cfg<L>::N);
  const int grid = (int)std::min<int64_t>(tiles, sm_count());
  if (beta) {
    auto kern = k_oz_gemm<L, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<grid, THREADS, smem, s>>>(tmA, tmB, C, m, n, (int)z.nchunks, (int)z.Mpad, (int)z.Npad, Ea, Eb, status, Se);
  } else {
    auto kern = k_oz_gemm<L, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<grid, THREADS, smem, s>>>(tmA, tmB, C, m, n, (int)z.nchunks, (int)z.Mpad, (int)z.Npad, Ea, Eb, status, Se);
  }
  note();
  return (int)cudaGetLastError();
}

}  // namespace oz
}  // namespace mclu
