// panel_coop.cuh - persistent cooperative panel factorisation (Sec. 3: the
// unblocked partial-pivoting factorisation of one panel of width nb).
//
// One cooperative launch factors the whole panel rows [j0, n) x columns
// [j0, jend): each CTA keeps a contiguous block of panel rows in shared
// memory for all nb columns, so a column step needs no kernel launch and no
// global-memory traffic except the pivot exchange.  Per column j, with one
// grid barrier:
//   1. every CTA computes cabs1 keys of its rows i >= j; its best (key, row)
//      goes to a global partial, its best row (all nb columns) to a global
//      row slot, and the owner of row j also publishes row j; the CTA then
//      arrives at the grid barrier and, while the others arrive, computes the
//      reciprocal of its best value and publishes it with a release flag
//      stamped with the column;                                -> grid barrier
//   2. every CTA reduces all partials (same winner p everywhere; ties to the
//      lowest row), waits for the winner's reciprocal flag (bounded) and
//      reads the winner's row from its slot;
//   3. the owners swap rows j and p in shared memory, every CTA scales its
//      rows below j by the winner's reciprocal and applies the rank-1 update
//      to the remaining panel columns.  Updated elements stay in leveled-
//      accumulator form (no renormalisation) except the next pivot column;
//      rows are renormalised when written back.
// Partials and row slots alternate between two buffers by column parity: a
// buffer is rewritten two columns later, after a barrier that every CTA
// reaches only once it has finished reading it.
// Grid barriers are counter + generation in global memory with a bounded
// spin (clock64 budget); a timeout sets *status and every CTA returns.
#pragma once

#include "lu_kernels.cuh"

namespace mclu {

constexpr int COOP_T = 256;
constexpr int COOP_GMAX = 256;                  // most CTAs of one cooperative panel launch
constexpr long long COOP_WAIT = 2000000000LL;  // ~1 s at 2 GHz

struct CoopWS {
  unsigned *bar_count;  // arrival counter
  unsigned *bar_gen;    // generation
  int *status;          // nonzero: a barrier timed out
  double *prow;         // [2][G][nb][2L] best row of each CTA, by column parity
  double *srow;         // [2][nb][2L] row j, by column parity
  int *rcp_flag;        // [2G] column stamp (j + 1) of the reciprocal in each partial slot
};

// Split grid barrier: arrive returns the generation to wait for; wait spins
// (bounded) until it has passed.  Returns false on timeout.
__device__ __forceinline__ unsigned coop_arrive(const CoopWS &cw, unsigned nblocks) {
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = cw.bar_gen;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(cw.bar_count, 1u) == nblocks - 1) {
      *cw.bar_count = 0;
      __threadfence();
      atomicAdd(cw.bar_gen, 1u);
    }
    s_gen = g;
  }
  __syncthreads();
  return s_gen;
}

__device__ __forceinline__ bool coop_wait(const CoopWS &cw, unsigned g) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *gen = cw.bar_gen;
    const long long t0 = clock64();
    while (*gen == g) {
      if (clock64() - t0 > COOP_WAIT) {
        ok = 0;
        atomicOr(cw.status, 1);
        break;
      }
    }
    __threadfence();
    s_ok = ok && (*(volatile int *)cw.status == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Sense-reversal grid barrier with a bounded wait.  Returns false on timeout.
__device__ __forceinline__ bool coop_barrier(const CoopWS &cw, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *gen = cw.bar_gen;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(cw.bar_count, 1u) == nblocks - 1) {
      *cw.bar_count = 0;
      __threadfence();
      atomicAdd(cw.bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > COOP_WAIT) {
          ok = 0;
          atomicOr(cw.status, 1);
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && (*(volatile int *)cw.status == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Factor panel columns [j0, jend) of rows [j0, n).  CTA b owns rows
// [j0 + b*rpc, j0 + min((b+1)*rpc, n - j0)).  Shared memory: the owned rows,
// [col][component][row] with the row fastest (consecutive threads take
// consecutive rows: no bank conflicts), then the pivot row of the current
// column [col][component], then the multipliers' four partial products
// [4][row][L].  Partial slots: par * G + b for column parity par.
template <int L>
__global__ void __launch_bounds__(COOP_T) k_panel_coop(View A, int64_t n, int64_t j0, int64_t jend, int rpc,
                                                      int32_t *ipiv, PanelWS<L> ws, CoopWS cw) {
  extern __shared__ double sp[];
  const int tid = threadIdx.x;
  const int nb = (int)(jend - j0);
  const int G = (int)gridDim.x, b = (int)blockIdx.x;
  const int64_t rbeg = j0 + (int64_t)b * rpc;
  const int64_t rend = min(n, rbeg + rpc);
  const int nr = (int)max((int64_t)0, rend - rbeg);
  const int RW = nb * 2 * L;  // doubles per panel row
  double *su = sp + (size_t)rpc * RW;  // pivot row [col][2L]
  double *mscr = su + RW;              // [4][rpc][L] the multipliers' partial products
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
  // load the owned rows
  for (int t = tid; t < nr * nb; t += COOP_T) {
    const int r = t % nr, c = t / nr;
    stp(r, c, ldz<L>(A, rbeg + r, j0 + c));
  }
  __syncthreads();
  __shared__ int s_p, s_zero, s_part;
  for (int jc = 0; jc < nb; jc++) {
    const int64_t j = j0 + jc;
    const int par = jc & 1;
    // 1. keys of the rows i >= j of this CTA
    R<L> key = invalid_key<L>();
    int idx = INT_MAX;
    for (int r = tid; r < nr; r += COOP_T) {
      const int64_t i = rbeg + r;
      if (i < j) continue;
      const R<L> k = pivot_key<L>(ldp(r, jc));
      if (better<L>(k, (int)i, key, idx)) {
        key = k;
        idx = (int)i;
      }
    }
    const int cand = write_partial_key<L>(key, idx, ws, par * G + b, tid, COOP_T);
    // publish this CTA's best row and, from its owner, row j
    if (cand != INT_MAX) {
      double *dst = cw.prow + ((size_t)par * G + b) * RW;
      const int r = (int)(cand - rbeg);
      for (int t = tid; t < RW; t += COOP_T) dst[t] = rowel(r, t);
    }
    if (j >= rbeg && j < rend) {
      double *dst = cw.srow + (size_t)par * RW;
      const int r = (int)(j - rbeg);
      for (int t = tid; t < RW; t += COOP_T) dst[t] = rowel(r, t);
    }
    const unsigned gen = coop_arrive(cw, G);
    // the reciprocal 1/p = conj(p) / |p|^2 of this CTA's candidate, while the
    // other CTAs arrive, split over warps 0 and 1 (two SMSPs, two FP64
    // units): Re p^2 and Im p^2 in parallel, the real reciprocal x of |p|^2
    // on warp 0, then Re p x and -Im p x in parallel; published with a
    // release flag stamped with the column
    {
      __shared__ double s_inv[2 * L];  // Im p^2 accumulator, then x
      const int w = tid >> 5, lane = tid & 31;
      const bool has = cand != INT_MAX;  // uniform over the CTA
      const bool act = has && lane == 0 && w < 2;
      const int q = par * G + b;
      Z<L> pv;
      Acc<L> t;
      if (act) {
        pv = ldp((int)(cand - rbeg), jc);
        const R<L> h = w == 0 ? pv.re : pv.im;
        t.set_prod(h, h);
        if (w == 1) {
#pragma unroll
          for (int l = 0; l < L; l++) s_inv[l] = t.s[l];
        }
      }
      __syncthreads();
      if (has && tid == 0) {
        Acc<L> o;
#pragma unroll
        for (int l = 0; l < L; l++) o.s[l] = s_inv[l];
        t.add_acc(o, false);
        const R<L> x = r_recip<L>(t.result());
#pragma unroll
        for (int l = 0; l < L; l++) s_inv[L + l] = x.x[l];
      }
      __syncthreads();
      if (act) {
        R<L> x;
#pragma unroll
        for (int l = 0; l < L; l++) x.x[l] = s_inv[L + l];
        R<L> v = r_mul<L>(w == 0 ? pv.re : pv.im, x);
        if (w == 1) v = r_neg<L>(v);
#pragma unroll
        for (int l = 0; l < L; l++) ws.part_rcp[(int64_t)q * 2 * L + w * L + l] = v.x[l];
        __threadfence();
      }
      __syncthreads();
      if (has && tid == 0) st_release(cw.rcp_flag + q, (int)(j + 1));
    }
    if (!coop_wait(cw, gen)) return;
    // 2. reduce the partials (every CTA, same result)
    {
      R<L> bk = invalid_key<L>();
      int bi = INT_MAX, bq = -1;
      for (int q = par * G + tid; q < par * G + G; q += COOP_T) {
        R<L> k;
#pragma unroll
        for (int l = 0; l < L; l++) k.x[l] = __ldcg(ws.part_key + (int64_t)q * L + l);
        const int i = __ldcg(ws.part_idx + q);
        if (better<L>(k, i, bk, bi)) {
          bk = k;
          bi = i;
          bq = q;
        }
      }
      const int my = bi;
      block_argmax<L>(bk, bi, tid, COOP_T);
      if (tid == 0) {
        const bool zero = !(bk.x[0] > 0.0);
        s_p = (bi == INT_MAX || zero) ? (int)j : bi;
        s_zero = zero ? 1 : 0;
      }
      __syncthreads();
      if (my == s_p && my != INT_MAX && !s_zero) s_part = bq;
      __syncthreads();
    }
    const int64_t p = s_p;
    const bool zero = s_zero != 0;
    if (b == 0 && tid == 0) {
      ipiv[j] = (int32_t)(p + 1);
      if (zero && *ws.info == 0) *ws.info = (int)(j + 1);
    }
    if (zero) {  // nothing to eliminate in this column; no swap; the next
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
      }
      __syncthreads();
      continue;
    }
    // 3. wait for the winner's reciprocal (bounded), stage the pivot row
    //    (row p before the swap), swap, scale, update
    {
      __shared__ int s_rok;
      if (tid == 0) {
        int ok = 1;
        const long long t0 = clock64();
        while (ld_acquire(cw.rcp_flag + s_part) != (int)(j + 1)) {
          if (clock64() - t0 > COOP_WAIT) {
            ok = 0;
            atomicOr(cw.status, 1);
            break;
          }
        }
        s_rok = ok;
      }
      __syncthreads();
      if (!s_rok) return;
    }
    const double *prow = cw.prow + (size_t)s_part * RW;
    for (int t = tid; t < RW; t += COOP_T) su[t] = __ldcg(prow + t);
    __syncthreads();
    if (p != j) {
      const double *srow = cw.srow + (size_t)par * RW;
      if (p >= rbeg && p < rend)
        for (int t = tid; t < RW; t += COOP_T) rowel((int)(p - rbeg), t) = __ldcg(srow + t);
      if (j >= rbeg && j < rend)
        for (int t = tid; t < RW; t += COOP_T) rowel((int)(j - rbeg), t) = su[t];
    }
    __syncthreads();
    {
      Z<L> r;
#pragma unroll
      for (int q = 0; q < L; q++) {
        r.re.x[q] = __ldcg(ws.part_rcp + (int64_t)s_part * 2 * L + q);
        r.im.x[q] = __ldcg(ws.part_rcp + (int64_t)s_part * 2 * L + L + q);
      }
      // multipliers l = a r of the rows below j: warps 0..3 (one per SMSP,
      // each with its own FP64 unit) form the four real products
      // Re a Re r, Im a Im r, Re a Im r, Im a Re r on leveled accumulators;
      // warps 0 and 1 then form Re l = P0 - P1 and Im l = P2 + P3
      {
        const int w = tid >> 5, lane = tid & 31;
        if (w < 4) {
          const R<L> y = (w == 0 || w == 3) ? r.re : r.im;
          for (int rr = lane; rr < nr; rr += 32) {
            if (rbeg + rr <= j) continue;
            const Z<L> a = ldp(rr, jc);
            Acc<L> t;
            t.set_prod((w == 0 || w == 2) ? a.re : a.im, y);
#pragma unroll
            for (int q = 0; q < L; q++) mscr[((size_t)w * rpc + rr) * L + q] = t.s[q];
          }
        }
        __syncthreads();
        if (w < 2) {
          for (int rr = lane; rr < nr; rr += 32) {
            if (rbeg + rr <= j) continue;
            Acc<L> t, o;
#pragma unroll
            for (int q = 0; q < L; q++) {
              t.s[q] = mscr[((size_t)(2 * w) * rpc + rr) * L + q];
              o.s[q] = mscr[((size_t)(2 * w + 1) * rpc + rr) * L + q];
            }
            t.add_acc(o, w == 0);
            const R<L> v = t.result();
            double *d = sp + (size_t)jc * 2 * L * rpc + rr + (size_t)(w * L) * rpc;
#pragma unroll
            for (int q = 0; q < L; q++) d[(size_t)q * rpc] = v.x[q];
          }
        }
      }
      __syncthreads();
      // rank-1 update of columns jc+1 .. nb-1 with the staged pivot row
      const int ncol = nb - jc - 1;
      for (int t = tid; t < nr * ncol; t += COOP_T) {
        const int rr = t % nr, cc = jc + 1 + t / nr;
        if (rbeg + rr <= j) continue;
        Z<L> u;
#pragma unroll
        for (int q = 0; q < L; q++) {
          u.re.x[q] = su[cc * 2 * L + q];
          u.im.x[q] = su[cc * 2 * L + L + q];
        }
        // the element stays in accumulator form (its levels) between
        // columns; the next pivot column is renormalised here
        const Z<L> a = ldp(rr, cc);
        Acc<L> re, im;
        re.set(a.re);
        im.set(a.im);
        acc_csub<L>(re, im, ldp(rr, jc), u);
        Z<L> z;
        if (cc == jc + 1) {
          z.re = re.result();
          z.im = im.result();
        } else {
#pragma unroll
          for (int q = 0; q < L; q++) {
            z.re.x[q] = re.s[q];
            z.im.x[q] = im.s[q];
          }
        }
        stp(rr, cc, z);
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
