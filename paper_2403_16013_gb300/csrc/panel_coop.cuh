// panel_coop.cuh - persistent cooperative panel factorisation (Sec. 3: the
// unblocked partial-pivoting factorisation of one panel of width nb).
//
// One cooperative launch factors the whole panel rows [j0, n) x columns
// [j0, jend): each CTA keeps a contiguous block of panel rows in shared
// memory for all nb columns, so a column step needs no kernel launch and no
// global-memory traffic except the pivot exchange.  Per column j:
//   1. every CTA picks its candidate among its rows i >= j (column j is up
//      to date) by the leading-limb key k0 (full cabs1 keys only where two
//      k0 are near) and writes (k0, row) to its key slot as two
//      self-validating words that carry the column (no fence), the
//      candidate's full key under a release stamp;
//   2. it then applies the pending rank-1 update of column j-1 to the
//      columns after j (one step of lookahead: only column j was updated
//      before the keys), first to its best row and to row j, which it
//      publishes (all nb columns) together with the reciprocal of its best
//      value under a release flag stamped with the column, then to its other
//      rows;
//   3. meanwhile one warp reads every CTA's key slot (bounded polling until
//      both words carry the column; integer comparisons only; same winner p
//      everywhere, ties to the lowest row; the full keys are read only for
//      slots whose k0 are near the largest), waits for
//      the winner's flag, stages its row and swaps rows j and p where this
//      CTA owns them (both were published rows, so the update of step 2
//      never touches them);
//   4. every CTA scales its rows below j by the winner's reciprocal (the
//      multipliers) and updates column j+1 of those rows, renormalised for
//      the next keys; the other columns wait for step 2 of the next column.
//      (DD: the candidate also publishes v = r u_{j,j+1}, so that column j+1
//      is a_{i,j+1} - a_ij v, formed at the same time as the multipliers.)
// Updated elements stay in leveled-accumulator form (no renormalisation)
// except the next pivot column; rows are renormalised when written back.
// Slots, row buffers and pivot rows alternate between two buffers by column
// parity: a CTA rewrites a buffer two columns later, once every CTA has
// stamped the column in between, which each does only after reading it.
// Every wait is bounded (clock64 budget); a timeout sets *status and every
// CTA returns.
#pragma once

#include "lu_kernels.cuh"

namespace mclu {

constexpr int COOP_T = 256;
constexpr int COOP_GMAX = 256;                  // most CTAs of one cooperative panel launch
constexpr long long COOP_WAIT = 2000000000LL;  // ~1 s at 2 GHz
constexpr int COOP_KS = 16;                     // doubles per key slot (one 128-byte line)

struct CoopWS {
  int *status;    // nonzero: a wait timed out
  double *kslot;  // [2][G][COOP_KS] by column parity: header words, full key, stamp 2 (see the key slot below)
  double *prow;   // [2][G][nb][2L] best row of each CTA, by column parity
  double *srow;   // [2][nb][2L] row j, by column parity
  int *rcp_flag;  // [2G] column stamp (j + 1) of the reciprocal and rows of each slot
  double *vnext;  // [2G][2L] v = r u of each slot's candidate, u its element in the next column (DD)
  int *v_flag;    // [2G] column stamp (j + 1) of vnext of each slot
};

// Barrier over the `count` threads (whole warps) that execute it with this id
// (id 0 is __syncthreads).
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Arrive at that barrier without waiting (the producers of a bar.sync).
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Bounded wait until *flag == v; false on timeout.
__device__ __forceinline__ bool coop_wait_flag(const int *flag, int v) {
  const long long t0 = clock64();
  while (ld_acquire(flag) != v)
    if (clock64() - t0 > COOP_WAIT) return false;
  return true;
}

// ----------------------------------------------------------- pivot keys --
// The pivot key of partial pivoting is cabs1 = |Re a| + |Im a| of the
// multi-component value (pivot_key: an accurate L-limb addition, tens of
// FP64 instructions in a dependent chain).  The leading limbs decide it
// almost always, for one FP64 addition: with ulp-nonoverlapping limbs
// (|x_{l+1}| <= ulp(x_l)) the lower limbs change |Re a| and |Im a| by at
// most 2^-52 of their leading limbs, and k0 = RN(|Re a_0| + |Im a_0|) adds a
// rounding of 2^-53, so the exact key K satisfies |K - k0| < 2^-51 k0.  A k0
// ahead of another by more than 32 ulps (more than 2^-48 relative: ulp(x) >
// 2^-53 |x|) therefore belongs to the larger exact key; keys within 32 ulps
// of the largest k0 ("near") are compared in full.

constexpr long long KEY_NEAR_ULPS = 32;

// k0 of row r of panel column c (the pivot column is renormalised, so its
// limbs are ulp-nonoverlapping); the sign bits are cleared on the integer pipe.
template <int L>
__device__ __forceinline__ double cheap_key(const double *sp, int c, int rpc, int r) {
  const double *d = sp + (size_t)c * 2 * L * rpc + r;
  const double re = __longlong_as_double(__double_as_longlong(d[0]) & 0x7fffffffffffffffLL);
  const double im = __longlong_as_double(__double_as_longlong(d[(size_t)L * rpc]) & 0x7fffffffffffffffLL);
  return __dadd_rn(re, im);
}

// k0 within KEY_NEAR_ULPS of kmax (both keys are >= 0, k0 <= kmax)
__device__ __forceinline__ bool key_near(double k0, double kmax) {
  return order_key(kmax) - order_key(k0) <= KEY_NEAR_ULPS;
}

// Key slot of one CTA for one column parity (COOP_KS doubles = one 128-byte
// line).  The common path is two 64-bit words, each of which validates
// itself, so a reader needs neither a fence nor a second round trip:
//   word 0: the column stamp (j + 1) in the high 32 bits, the candidate row
//           in bits 0..30 (INT_MAX: no candidate), bit 31 set when k0 is
//           exactly zero;
//   word 1: the bits of k0 (-1.0: no candidate) with the low KEY_STAMP_BITS
//           mantissa bits replaced by the low bits of the stamp.
// A 64-bit aligned access is single-copy atomic, so a word that shows this
// column's stamp holds this column's value (word 0 is still stored with
// release and the reader fences once after its polling: that orders each
// CTA's reads of the pivot rows of column j before its stamp of column j+1,
// which the owner of those row buffers awaits before it rewrites them); stale words hold an earlier
// column (the stamp bits of word 1 repeat only after 2^20 columns, far
// beyond any order that fits in memory).  Truncating k0 to its high bits is
// monotone, so the truncated keys order the candidates except within
// KEY_SLOT_NEAR of each other, where the full keys decide.  Those follow in
// doubles 2 .. L+1 under stamp 2 (an int in double L+2, released).
constexpr int KEY_STAMP_BITS = 20;
constexpr unsigned long long KEY_STAMP_MASK = (1ull << KEY_STAMP_BITS) - 1;
// |exact key - k0| < 2^-51 k0 and the truncation removes less than 2^-32 k0,
// so truncated keys further apart than 2^-30.9 (relative) are ordered as the
// exact keys; 2^23 units of the order key is 2^-30 or more.
constexpr long long KEY_SLOT_NEAR = 1ll << 23;


template <int L>
__device__ __forceinline__ int *slot_stamp2(double *slot) {
  return reinterpret_cast<int *>(slot + L + 2);
}

// Publication of this CTA's candidate (one thread): the two header words;
// with has_key, the full key under stamp 2 as well.
template <int L>
__device__ __forceinline__ void publish_key_slot(double *slot, int64_t j, int cand, double k0, bool has_key,
                                                 const double *key) {
  const unsigned long long stamp = (unsigned long long)(j + 1);
  if (has_key) {
#pragma unroll
    for (int l = 0; l < L; l++) slot[2 + l] = key[l];
    st_release(slot_stamp2<L>(slot), (int)(j + 1));
  }
  const unsigned long long kb = (unsigned long long)__double_as_longlong(k0);
  const unsigned zero = kb == 0 ? 0x80000000u : 0u;
  unsigned long long *w = reinterpret_cast<unsigned long long *>(slot);
  st_relaxed_u64(w + 1, (kb & ~KEY_STAMP_MASK) | (stamp & KEY_STAMP_MASK));
  st_release_u64(w, (stamp << 32) | (unsigned)((unsigned)cand & 0x7fffffffu) | zero);
}

// The full key of a candidate chosen by k0 alone, published under stamp 2.
template <int L>
__device__ __forceinline__ void publish_full_key(double *slot, int64_t j, const R<L> &key) {
#pragma unroll
  for (int l = 0; l < L; l++) slot[2 + l] = key.x[l];
  st_release(slot_stamp2<L>(slot), (int)(j + 1));
}

struct Winner {
  int64_t p;  // pivot row (j for a zero column)
  int part;   // key slot of the winner, -1 if none
  bool zero;  // every candidate key is zero
  bool ok;    // false: a wait ran out
};

// The pivot of column j over all G key slots of parity par, run by one warp:
// lane l takes slots l, l + 32, ...; it polls both header words of each
// until they carry the column (bounded), keeping the values it validated.
// The largest truncated k0 (ties: the lowest row) wins unless another slot's
// truncated k0 is within KEY_SLOT_NEAR; then the full keys of the near slots
// are awaited (stamp 2, acquire) and compared.  Integer operations only,
// except on that rare path.
template <int L>
__device__ Winner exchange_winner(const CoopWS &cw, int par, int G, int64_t j, int lane) {
  constexpr int KMAX = COOP_GMAX / 32;
  const unsigned long long stamp = (unsigned long long)(j + 1);
  long long keys[KMAX];  // truncated k0 bits (negative: no candidate)
  int rows[KMAX];
  unsigned zflag = 0;    // slots whose k0 is exactly zero
  unsigned pendk = 0;
#pragma unroll
  for (int k = 0; k < KMAX; k++) {
    keys[k] = LLONG_MIN;
    rows[k] = INT_MAX;
    if (lane + 32 * k < G) pendk |= 1u << k;
  }
  bool ok = true;
  const long long t0 = clock64();
  while (pendk) {
#pragma unroll
    for (int k = 0; k < KMAX; k++)
      if ((pendk >> k) & 1u) {
        const unsigned long long *w =
            reinterpret_cast<const unsigned long long *>(cw.kslot + ((size_t)par * G + lane + 32 * k) * COOP_KS);
        const unsigned long long w0 = ld_relaxed_u64(w), w1 = ld_relaxed_u64(w + 1);
        if ((w0 >> 32) == stamp && (w1 & KEY_STAMP_MASK) == (stamp & KEY_STAMP_MASK)) {
          keys[k] = (long long)(w1 & ~KEY_STAMP_MASK);
          rows[k] = (int)(w0 & 0x7fffffffu);
          if (w0 & 0x80000000u) zflag |= 1u << k;
          pendk &= ~(1u << k);
        }
      }
    if (pendk && clock64() - t0 > COOP_WAIT) {
      ok = false;
      break;
    }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  Winner res{j, -1, true, __all_sync(0xffffffffu, ok)};
  if (!res.ok) return res;
  // this lane's best slot, then the warp's: largest key, then lowest row
  long long bk = LLONG_MIN;
  int bi = INT_MAX, bq = -1;
  bool bz = false;
#pragma unroll
  for (int k = 0; k < KMAX; k++)
    if (rows[k] != INT_MAX && (keys[k] > bk || (keys[k] == bk && rows[k] < bi))) {
      bk = keys[k];
      bi = rows[k];
      bq = par * G + lane + 32 * k;
      bz = (zflag >> k) & 1u;
    }
  const unsigned long long u = (unsigned long long)bk ^ 0x8000000000000000ull;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, (unsigned)(u >> 32));
  const unsigned mlo = __reduce_max_sync(0xffffffffu, (unsigned)(u >> 32) == mhi ? (unsigned)u : 0u);
  const bool top = (unsigned)(u >> 32) == mhi && (unsigned)u == mlo;
  const int wrow = (int)__reduce_min_sync(0xffffffffu, top ? (unsigned)bi : 0xffffffffu);
  const long long kmax = (long long)((((unsigned long long)mhi << 32) | mlo) ^ 0x8000000000000000ull);
  bool nearx = false;
  if (kmax >= 0) {
#pragma unroll
    for (int k = 0; k < KMAX; k++)
      if (rows[k] != INT_MAX && keys[k] >= 0 && rows[k] != wrow && kmax - keys[k] <= KEY_SLOT_NEAR) nearx = true;
  }
  int my = top && bi == wrow ? bi : INT_MAX, myq = bq;
  bool zero = kmax < 0 || __any_sync(0xffffffffu, top && bi == wrow && bz);
  int win = wrow;
  if (__any_sync(0xffffffffu, nearx)) {
    // full keys of the slots within the window of the largest truncated k0
    R<L> fk = invalid_key<L>();
    int fi = INT_MAX, fq = -1;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
      if (rows[k] == INT_MAX || keys[k] < 0 || kmax - keys[k] > KEY_SLOT_NEAR) continue;
      double *slot = cw.kslot + ((size_t)par * G + lane + 32 * k) * COOP_KS;
      if (!coop_wait_flag(slot_stamp2<L>(slot), (int)stamp)) {
        ok = false;
        continue;
      }
      R<L> kk;
#pragma unroll
      for (int l = 0; l < L; l++) kk.x[l] = __ldcg(slot + 2 + l);
      if (better<L>(kk, rows[k], fk, fi)) {
        fk = kk;
        fi = rows[k];
        fq = par * G + lane + 32 * k;
      }
    }
    res.ok = __all_sync(0xffffffffu, ok);
    if (!res.ok) return res;
    my = fi;
    myq = fq;
    warp_argmax<L>(fk, fi);
    win = fi;
    zero = !(fk.x[0] > 0.0);
  }
  const unsigned own = __ballot_sync(0xffffffffu, my == win && my != INT_MAX);
  res.part = own ? __shfl_sync(0xffffffffu, myq, __ffs(own) - 1) : -1;
  res.zero = zero;
  res.p = (win == INT_MAX || zero) ? j : win;
  return res;
}

// Factor panel columns [j0, jend) of rows [j0, n).  CTA b owns rows
// [j0 + b*rpc, j0 + min((b+1)*rpc, n - j0)).  Shared memory: the owned rows,
// [col][component][row] with the row fastest (consecutive threads take
// consecutive rows: no bank conflicts), then the pivot rows of the two column
// parities [col][component], then the multipliers' four partial products
// [4][row][L].  Slot of this CTA for column parity par: par * G + b.
template <int L>
__global__ void __launch_bounds__(COOP_T) k_panel_coop(View A, int64_t n, int64_t j0, int64_t jend, int rpc,
                                                      int32_t *ipiv, PanelWS<L> ws, CoopWS cw) {
  extern __shared__ double sp[];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int nb = (int)(jend - j0);
  const int G = (int)gridDim.x, b = (int)blockIdx.x;
  const int64_t rbeg = j0 + (int64_t)b * rpc;
  const int64_t rend = min(n, rbeg + rpc);
  const int nr = (int)max((int64_t)0, rend - rbeg);
  const int RW = nb * 2 * L;             // doubles per panel row
  double *su2 = sp + (size_t)rpc * RW;   // pivot rows [2][col][2L]
  double *mscr = su2 + 2 * (size_t)RW;   // [4][rpc][L] the multipliers' partial products
  auto ldp = [&](int r, int c) {
    Z<L> z;
    const double *d = sp + (size_t)c * 2 * L * rpc + r;
#pragma unroll
    for (int q = 0; q < L; q++) {
      z.re.x[q] = d[(size_t)q * rpc];
      z.im.x[q] = d[(size_t)(L + q) * rpc];
    }
    return z;
  };
  auto stp = [&](int r, int c, const Z<L> &z) {
    double *d = sp + (size_t)c * 2 * L * rpc + r;
#pragma unroll
    for (int q = 0; q < L; q++) {
      d[(size_t)q * rpc] = z.re.x[q];
      d[(size_t)(L + q) * rpc] = z.im.x[q];
    }
  };
  // element t = c * 2L + q of row r (the global row-slot format)
  auto rowel = [&](int r, int t) -> double & { return sp[(size_t)t * rpc + r]; };
  // element (r, c) minus l u, l = column jm of row r, u = element c of the
  // pivot row su; the result stays in accumulator form (its levels)
  auto upd = [&](int r, int c, int jm, const double *su) {
    Z<L> u;
#pragma unroll
    for (int q = 0; q < L; q++) {
      u.re.x[q] = su[c * 2 * L + q];
      u.im.x[q] = su[c * 2 * L + L + q];
    }
    const Z<L> a = ldp(r, c);
    Acc<L> re, im;
    re.set(a.re);
    im.set(a.im);
    acc_csub<L>(re, im, ldp(r, jm), u);
    Z<L> z;
#pragma unroll
    for (int q = 0; q < L; q++) {
      z.re.x[q] = re.s[q];
      z.im.x[q] = im.s[q];
    }
    return z;
  };  // one component of upd (h = 0: Re, 1: Im), stored in place: the pending
  // update in items of half the FP64 work, so that a warp that joins late
  // holds the others up by less
  auto upd1 = [&](int r, int c, int jm, const double *su, int h) {
    R<L> ur, ui;
#pragma unroll
    for (int q = 0; q < L; q++) {
      ur.x[q] = su[c * 2 * L + q];
      ui.x[q] = su[c * 2 * L + L + q];
    }
    const Z<L> lv = ldp(r, jm);
    double *d = sp + (size_t)c * 2 * L * rpc + r + (size_t)(h * L) * rpc;
    Acc<L> t;
    R<L> a;
#pragma unroll
    for (int q = 0; q < L; q++) a.x[q] = d[(size_t)q * rpc];
    t.set(a);
    if (h == 0) {  // Re a - Re l Re u + Im l Im u
      t.template add_prod<true>(lv.re, ur);
      t.template add_prod<false>(lv.im, ui);
    } else {       // Im a - Re l Im u - Im l Re u
      t.template add_prod<true>(lv.re, ui);
      t.template add_prod<true>(lv.im, ur);
    }
#pragma unroll
    for (int q = 0; q < L; q++) d[(size_t)q * rpc] = t.s[q];
  };

  // load the owned rows
  for (int t = tid; t < nr * nb; t += COOP_T) {
    const int r = t % nr, c = t / nr;
    stp(r, c, ldz<L>(A, rbeg + r, j0 + c));
  }
  __shared__ int s_zero, s_next, s_pend, s_ok, s_cand, s_fast;
  __shared__ double s_rcp[2 * L], s_v[2 * L], s_key[L], s_k0;
  // The CTA's candidate for panel column c among its rows i >= jrow: the
  // largest k0 (one FP64 addition per row), unless another row's k0 is near
  // it; then the full keys of the near rows decide (s_fast = 0, s_key the
  // full key).  s_k0 is the largest k0 either way.
  //   select_block: all threads (barriers inside);
  //   select_warp0: warp 0 alone when the CTA has at most 32 rows (one row a
  //   lane, warp shuffles only): run at the end of the previous column, right
  //   after warps 0 and 1 have formed column c, it saves the column start
  //   four block barriers.
  const bool fused = rpc <= 32;
  auto select_block = [&](int jc, int64_t j) {
    {
      R<1> k1 = invalid_key<1>();
      int idx = INT_MAX;
      for (int r = tid; r < nr; r += COOP_T) {
        const int64_t i = rbeg + r;
        if (i < j) continue;
        R<1> k;
        k.x[0] = cheap_key<L>(sp, jc, rpc, r);
        if (better<1>(k, (int)i, k1, idx)) {
          k1 = k;
          idx = (int)i;
        }
      }
      block_argmax<1>(k1, idx, tid, COOP_T);
      if (tid == 0) {
        s_k0 = k1.x[0];
        s_cand = idx;
      }
      __syncthreads();
      const double kmax = s_k0;
      const int c0 = s_cand;
      bool mynear = false;
      if (c0 != INT_MAX) {
        for (int r = tid; r < nr; r += COOP_T) {
          const int64_t i = rbeg + r;
          if (i >= j && i != c0 && key_near(cheap_key<L>(sp, jc, rpc, r), kmax)) mynear = true;
        }
      }
      if (__syncthreads_or(mynear)) {
        R<L> key = invalid_key<L>();
        int id2 = INT_MAX;
        for (int r = tid; r < nr; r += COOP_T) {
          const int64_t i = rbeg + r;
          if (i < j || !key_near(cheap_key<L>(sp, jc, rpc, r), kmax)) continue;
          const R<L> k = pivot_key<L>(ldp(r, jc));
          if (better<L>(k, (int)i, key, id2)) {
            key = k;
            id2 = (int)i;
          }
        }
        block_argmax<L>(key, id2, tid, COOP_T);
        if (tid == 0) {
#pragma unroll
          for (int l = 0; l < L; l++) s_key[l] = key.x[l];
          s_cand = id2;
          s_fast = 0;
        }
      } else if (tid == 0) {
        s_fast = 1;
      }
      __syncthreads();
    }
  };
  auto select_warp0 = [&](int c, int64_t jrow) {
    const int64_t i = rbeg + lane;
    const bool act = lane < nr && i >= jrow;
    R<1> k;
    k.x[0] = act ? cheap_key<L>(sp, c, rpc, lane) : -1.0;
    R<1> kk = k;
    int ii = act ? (int)i : INT_MAX;
    warp_argmax<1>(kk, ii);
    const bool nearl = act && ii != INT_MAX && key_near(k.x[0], kk.x[0]);  // the winner included
    if (__any_sync(0xffffffffu, nearl && (int)i != ii)) {
      R<L> fk = nearl ? pivot_key<L>(ldp(lane, c)) : invalid_key<L>();
      int fi = nearl ? (int)i : INT_MAX;
      warp_argmax<L>(fk, fi);
      if (lane == 0) {
#pragma unroll
        for (int l = 0; l < L; l++) s_key[l] = fk.x[l];
        s_cand = fi;
        s_k0 = kk.x[0];
        s_fast = 0;
      }
    } else if (lane == 0) {
      s_cand = ii;
      s_k0 = kk.x[0];
      s_fast = 1;
    }
  };
  if (tid == 0) {
    s_next = 0;
    s_pend = 0;
    s_ok = 1;
  }
  if (fused && w == 0) select_warp0(0, j0);
  __syncthreads();
  for (int jc = 0; jc < nb; jc++) {
    const int64_t j = j0 + jc;
    const int par = jc & 1;
    double *su = su2 + (size_t)par * RW;                 // pivot row of column jc
    const double *sprev = su2 + (size_t)(par ^ 1) * RW;  // pivot row of column jc - 1
    const bool pend = s_pend != 0;  // the update of columns jc+1.. from column jc-1 is pending
    const int q = par * G + b;
    // 1. the CTA's candidate among its rows i >= j (with at most 32 rows a
    //    CTA, warp 0 chose it at the end of the previous column)
    if (!fused) select_block(jc, j);
    const int cand = s_cand;
    const bool fast = s_fast != 0;
    const bool has = cand != INT_MAX;                                // uniform over the CTA
    const int cr = has ? (int)(cand - rbeg) : -1;                    // local row of the candidate
    const int jr = (j >= rbeg && j < rend) ? (int)(j - rbeg) : -1;  // local row j
    // 2. warps 0 and 1: the reciprocal 1/p of the candidate by Newton's
    //    method from a binary64 seed (z_inv_newton: the real and imaginary
    //    parts of the residual and of the result on SMSPs 0 and 1; warps 4
    //    and 5 keep off those two FP64 units meanwhile);
    //    warps 2 and 7: the pending update of the candidate row and of row j,
    //    published to their slots; once all four are done thread 0 releases
    //    the flag.  Warp 3 publishes the key and does step 3 at the same time
    //    (it needs no FP64 unit until the swap).  The rest of the pending
    //    update goes in 32-element pieces to whole warps: 6 at once, the
    //    others when free.
    __shared__ double s_r[2 * L];  // this CTA's candidate's reciprocal (re limbs, im limbs)
    const bool vnx = L == 2 && has && jc + 1 < nb;  // publish v = r u_{cand, jc+1}
    if ((w & 2) == 0) {
      __shared__ double s_e[2];  // Re e, Im e of the Newton step
      const bool act = has && lane == 0 && w < 2;
      Z<L> pv;
      RcpSeed sd;
      if (act) {
        pv = ldp(cr, jc);
        sd = rcp_seed(pv.re.x[0], pv.im.x[0]);
        s_e[w] = w == 0 ? rcp_resid_re<L>(pv.re, pv.im, sd) : rcp_resid_im<L>(pv.re, pv.im, sd);
      }
      named_sync(1, 128);
      if (act) {
        R<L> v;
        if constexpr (L == 2) {
          v = w == 0 ? rcp_finish<L, false>(sd, s_e[0], s_e[1]) : rcp_finish<L, true>(sd, s_e[0], s_e[1]);
        } else {  // (the team kernel factors TD and QD panels)
          const Z<L> z = z_inv_newton<L>(pv);
          v = w == 0 ? z.re : z.im;
        }
#pragma unroll
        for (int l = 0; l < L; l++) {
          ws.part_rcp[(int64_t)q * 2 * L + w * L + l] = v.x[l];
          s_r[w * L + l] = v.x[l];
        }
      }
      named_sync(1, 128);
      if (w == 5 && lane == 0 && has && fast)  // off the reciprocal's SMSPs' critical window
        publish_full_key<L>(cw.kslot + (size_t)q * COOP_KS, j, pivot_key<L>(ldp(cr, jc)));
    } else if (w == 2 || w == 7) {
      // warp 2: the candidate row (and the row-j slot when it is row j);
      // warp 7: row j when it is another row of this CTA
      const int r = w == 2 ? cr : (jr != cr ? jr : -1);
      if (r >= 0) {
        double *dst = w == 2 ? cw.prow + (size_t)q * RW : cw.srow + (size_t)par * RW;
        double *dst2 = (w == 2 && jr == cr) ? cw.srow + (size_t)par * RW : nullptr;
        for (int c = lane; c < nb; c += 32) {
          Z<L> z;
          if (pend && c > jc) {
            z = upd(r, c, jc - 1, sprev);
            stp(r, c, z);
          } else {
            z = ldp(r, c);
          }
#pragma unroll
          for (int l = 0; l < L; l++) {
            dst[c * 2 * L + l] = z.re.x[l];
            dst[c * 2 * L + L + l] = z.im.x[l];
          }
          if (dst2) {
#pragma unroll
            for (int l = 0; l < L; l++) {
              dst2[c * 2 * L + l] = z.re.x[l];
              dst2[c * 2 * L + L + l] = z.im.x[l];
            }
          }
        }
      }
      named_arrive(3, 96);  // rows cr and jr are final: warp 3 may swap them
      if (w == 2) named_arrive(4, 64);  // warp 6 may take SMSP 2's FP64 unit
    }
    if (w == 0 || w == 1 || w == 2 || w == 7) {
      named_sync(2, 128);
      if (has && tid == 0) st_release(cw.rcp_flag + q, (int)(j + 1));
      if (vnx && w < 2) {
        // v = r u on warps 0 (Re) and 1 (Im), u the candidate row's element
        // of column jc+1 (final: warp 2 updated it)
        if (lane == 0) {
          const Z<L> u = ldp(cr, jc + 1);
          R<L> rre, rim;
#pragma unroll
          for (int l = 0; l < L; l++) {
            rre.x[l] = s_r[l];
            rim.x[l] = s_r[L + l];
          }
          Acc<L> t;
          t.set_prod(rre, w == 0 ? u.re : u.im);
          if (w == 0)
            t.template add_prod<true>(rim, u.im);
          else
            t.template add_prod<false>(rim, u.re);
          const R<L> v = t.result();
#pragma unroll
          for (int l = 0; l < L; l++) cw.vnext[(int64_t)q * 2 * L + w * L + l] = v.x[l];
        }
        named_sync(6, 64);
        if (tid == 0) st_release(cw.v_flag + q, (int)(j + 1));
      }
    }
    if (w == 3) {
      if (lane == 0) {  // this CTA's candidate (k0, row; the full key if known) to its slot
        R<L> inv = invalid_key<L>();
        publish_key_slot<L>(cw.kslot + (size_t)q * COOP_KS, j, cand, has ? s_k0 : -1.0, !has || !fast,
                            has ? s_key : inv.x);
      }
      // 3. the winner over all key slots of this column
      const Winner win = exchange_winner<L>(cw, par, G, j, lane);
      bool ok = win.ok;
      const bool zero = win.zero;
      const int64_t p = win.p;
      const int part = win.part;
      const bool own_p = p != j && p >= rbeg && p < rend;
      if (ok && !zero && lane == 0) {
        // the winner's reciprocal and row; row j where this CTA owns row p
        ok = coop_wait_flag(cw.rcp_flag + part, (int)(j + 1)) &&
             (!own_p || coop_wait_flag(cw.rcp_flag + par * G + (int)((j - j0) / rpc), (int)(j + 1)));
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok && !zero) {
        const double *prow = cw.prow + (size_t)part * RW;
        for (int t = lane; t < RW; t += 32) su[t] = __ldcg(prow + t);
        if (lane < 2 * L) s_rcp[lane] = __ldcg(ws.part_rcp + (int64_t)part * 2 * L + lane);
      }
      named_sync(3, 96);  // warps 2 and 7 are done with rows cr and jr
      if (ok && !zero) {
        if (own_p) {
          const double *srow = cw.srow + (size_t)par * RW;
          for (int t = lane; t < RW; t += 32) rowel((int)(p - rbeg), t) = __ldcg(srow + t);
        }
        if (p != j && jr >= 0)
          for (int t = lane; t < RW; t += 32) rowel(jr, t) = su[t];
        if (L == 2 && jc + 1 < nb) {  // the winner's v, published after its reciprocal
          if (lane == 0) ok = coop_wait_flag(cw.v_flag + part, (int)(j + 1));
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (ok && lane < 2 * L) s_v[lane] = __ldcg(cw.vnext + (int64_t)part * 2 * L + lane);
        }
      }
      if (lane == 0) {
        if (!ok) {
          atomicOr(cw.status, 1);
          s_ok = 0;
        }
        s_zero = zero ? 1 : 0;
        if (ok && b == 0) {
          ipiv[j] = (int32_t)(p + 1);
          if (zero && *ws.info == 0) *ws.info = (int)(j + 1);
        }
      }
    } else {
      // warp 6 shares SMSP 2 with warp 2: it starts its share of the pending
      // update once the candidate row (on the path to the flag) is done
      if (w == 6) named_sync(4, 64);
    }
    if (w != 3 && pend) {
      const int rlo = (int)max((int64_t)0, j - rbeg);  // rows i > j - 1
      const int nrow = nr - rlo, ncol = nb - jc - 1;
      const int per = nrow > 0 ? nrow * ncol : 0;     // elements
      const int half = (per + 31) / 32 * 32;          // items of one component, whole warps
      for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&s_next, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= 2 * half) break;
        const int h = base >= half ? 1 : 0;  // uniform over the warp
        const int t = base - h * half + lane;
        if (t < per) {
          const int rr = rlo + t % nrow, cc = jc + 1 + t / nrow;
          if (rr != cr && rr != jr) upd1(rr, cc, jc - 1, sprev, h);
        }
      }
    }
    __syncthreads();
    if (!s_ok) return;
    if (s_zero) {  // nothing to eliminate in this column; no swap; the next
                   // pivot column is renormalised for its keys
      if (jc + 1 < nb) {
        for (int rr = tid; rr < nr; rr += COOP_T) {
          if (rbeg + rr <= j) continue;
          const Z<L> a = ldp(rr, jc + 1);
          Acc<L> re, im;
          re.set(a.re);
          im.set(a.im);
          Z<L> z;
          z.re = re.result();
          z.im = im.result();
          stp(rr, jc + 1, z);
        }
        if (fused) {
          __syncthreads();
          if (w == 0) select_warp0(jc + 1, j + 1);
        }
      }
      if (tid == 0) {
        s_pend = 0;
        s_next = 0;
      }
      __syncthreads();
      continue;
    }
    {
      Z<L> r;
#pragma unroll
      for (int l = 0; l < L; l++) {
        r.re.x[l] = s_rcp[l];
        r.im.x[l] = s_rcp[L + l];
      }
      // the multipliers' combination (warps 0 and 1): Re l = P0 - P1,
      // Im l = P2 + P3, written to column jc
      auto combine_l = [&]() {
        for (int rr = lane; rr < nr; rr += 32) {
          if (rbeg + rr <= j) continue;
          Acc<L> t, o;
#pragma unroll
          for (int l = 0; l < L; l++) {
            t.s[l] = mscr[((size_t)(2 * w) * rpc + rr) * L + l];
            o.s[l] = mscr[((size_t)(2 * w + 1) * rpc + rr) * L + l];
          }
          t.add_acc(o, w == 0);
          const R<L> v = t.result();
          double *d = sp + (size_t)jc * 2 * L * rpc + rr + (size_t)(w * L) * rpc;
#pragma unroll
          for (int l = 0; l < L; l++) d[(size_t)l * rpc] = v.x[l];
        }
      };
      // column cc's part h (0: Re, 1: Im) from the products P_{b+2h},
      // P_{b+2h+1}: Re a - P0 + P1, Im a - P2 - P3, renormalised for its keys
      auto combine_next = [&](int cc, int h, int b) {
        for (int rr = lane; rr < nr; rr += 32) {
          if (rbeg + rr <= j) continue;
          const Z<L> a = ldp(rr, cc);
          Acc<L> t, o;
          t.set(h == 0 ? a.re : a.im);
#pragma unroll
          for (int l = 0; l < L; l++) o.s[l] = mscr[((size_t)(b + 2 * h) * rpc + rr) * L + l];
          t.add_acc(o, true);
#pragma unroll
          for (int l = 0; l < L; l++) o.s[l] = mscr[((size_t)(b + 2 * h + 1) * rpc + rr) * L + l];
          t.add_acc(o, h == 1);
          const R<L> v = t.result();
          double *d = sp + (size_t)cc * 2 * L * rpc + rr + (size_t)(h * L) * rpc;
#pragma unroll
          for (int l = 0; l < L; l++) d[(size_t)l * rpc] = v.x[l];
        }
      };
      // product p of x (0: Re x Re y, 1: Im x Im y, 2: Re x Im y, 3: Im x Re y)
      // for the rows below j into mscr[slot]
      auto products = [&](int p, int slot, int c, const double *y2) {
        R<L> y;
#pragma unroll
        for (int l = 0; l < L; l++) y.x[l] = y2[((p == 0 || p == 3) ? 0 : L) + l];
        for (int rr = lane; rr < nr; rr += 32) {
          if (rbeg + rr <= j) continue;
          const Z<L> x = ldp(rr, c);
          Acc<L> t;
          t.set_prod((p == 0 || p == 2) ? x.re : x.im, y);
#pragma unroll
          for (int l = 0; l < L; l++) mscr[((size_t)slot * rpc + rr) * L + l] = t.s[l];
        }
      };
      if (L == 2 && jc + 1 < nb) {
        // 4. (DD) the multipliers l = a r and column jc+1 = a' - a v at once:
        //    warps 0..3 (one per SMSP) form the four real products of a r,
        //    warps 4..7 those of a v; then warps 0 and 1 combine l while
        //    warps 2 and 3 combine column jc+1
        const int cc = jc + 1;
        products(w & 3, w, jc, w < 4 ? s_rcp : s_v);
        __syncthreads();
        if (w < 2)
          combine_l();
        else if (w < 4)
          combine_next(cc, w - 2, 4);
        if (fused && w < 4) {  // column cc is final on warps 0..3: the next candidate
          named_sync(5, 128);
          if (w == 0) select_warp0(cc, j + 1);
        }
      } else {
        // 4. multipliers l = a r of the rows below j: warps 0..3 (one per
        //    SMSP, each with its own FP64 unit) form the four real products
        //    Re a Re r, Im a Im r, Re a Im r, Im a Re r on leveled
        //    accumulators; warps 0 and 1 then form Re l = P0 - P1 and
        //    Im l = P2 + P3
        if (w < 4) products(w, w, jc, s_rcp);
        __syncthreads();
        if (w < 2) combine_l();
        __syncthreads();
        // the next pivot column jc+1 now, renormalised for its keys (the
        // columns after it wait for the next column's step 2), split like
        // the multipliers: warps 0..3 form Re l Re u, Im l Im u, Re l Im u,
        // Im l Re u; warps 0 and 1 take a - P0 + P1 and a - P2 - P3
        if (jc + 1 < nb) {
          const int cc = jc + 1;
          if (w < 4) products(w, w, jc, su + cc * 2 * L);
          __syncthreads();
          if (w < 2) combine_next(cc, w, 0);
          if (fused && w < 2) {  // column cc is final on warps 0 and 1: the next candidate
            named_sync(5, 64);
            if (w == 0) select_warp0(cc, j + 1);
          }
        }
      }
      if (tid == 0) {
        s_pend = jc + 2 < nb ? 1 : 0;
        s_next = 0;
      }
    }
    __syncthreads();
  }
  // write the owned rows back, renormalised (elements that left the active
  // rows, such as the U part of each pivot row, may still hold accumulator levels)
  for (int t = tid; t < nr * nb; t += COOP_T) {
    const int r = t % nr, c = t / nr;
    const Z<L> a = ldp(r, c);
    Acc<L> re, im;
    re.set(a.re);
    im.set(a.im);
    Z<L> z;
    z.re = re.result();
    z.im = im.result();
    stz<L>(A, rbeg + r, j0 + c, z);
  }
}

}  // namespace mclu
