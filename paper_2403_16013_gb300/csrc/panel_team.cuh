// panel_team.cuh - the cooperative panel factorisation of panel_coop.cuh
// with the rank-1 update of each column run by a team of its own (Sec. 3:
// the unblocked partial-pivoting factorisation of one panel of width nb).
//
// Same data layout, key-slot exchange and row publication as k_panel_coop;
// the CTA's warps split into two teams that meet only at named barriers:
//   * the factor team (warps 0-3) computes the keys, the candidate's
//     reciprocal (warps 0, 1), the exchange (warp 3: key slots, winner's
//     flag, pivot row, swap), publishes the candidate row and row j (warp 2)
//     once the update team is done with the previous column, then the
//     multipliers and the next pivot column (four real products on four
//     warps);
//   * the update team (warps 5-7; warp 4 only keeps the barrier counts)
//     applies column j-1's rank-1 update to the columns after j from the
//     moment column j-1's multipliers are final until the factor team needs
//     the rows for column j: it overlaps the factor team's update of the
//     next pivot column, its keys, reciprocal and exchange instead of only
//     the exchange.
// With TD and QD the long reciprocal chain leaves room for the whole update
// (measured at n = 4096: panel TD 128.3 -> 123.1 ms, QD 282.3 -> 266.1 ms);
// with DD the shorter chain does not, and k_panel_coop stays faster.
// Every global wait is bounded (clock64 budget); a timeout sets *status, the
// factor team releases the update team at its next go signal and the CTA
// returns without writing back.
#pragma once

#include "panel_coop.cuh"

namespace mclu {

// Named barriers of k_panel_team (id 0 is __syncthreads): the factor team
// is warps 0-3, the update team warps 4-7.
constexpr int BAR_MAIN = 1;  // factor team (128)
constexpr int BAR_RCP = 2;   // warps 0 and 1 (64)
constexpr int BAR_DONE = 3;  // update team arrives, warps 0-2 wait (224)
constexpr int BAR_PUB = 4;   // warps 0-2 (96)
constexpr int BAR_SWAP = 5;  // warps 0-2 arrive, warp 3 waits (128)
constexpr int BAR_GO = 6;    // factor team arrives, update team waits (256)

// Factor panel columns [j0, jend) of rows [j0, n).  CTA b owns rows
// [j0 + b*rpc, j0 + min((b+1)*rpc, n - j0)).  Shared memory: the owned rows,
// [col][component][row] with the row fastest (consecutive threads take
// consecutive rows: no bank conflicts), then the pivot rows of the two column
// parities [col][component], then the multipliers' four partial products
// [4][row][L].  Slot of this CTA for column parity par: par * G + b.
template <int L>
__global__ void __launch_bounds__(COOP_T) k_panel_team(View A, int64_t n, int64_t j0, int64_t jend, int rpc,
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
  };
  // load the owned rows
  for (int t = tid; t < nr * nb; t += COOP_T) {
    const int r = t % nr, c = t / nr;
    stp(r, c, ldz<L>(A, rbeg + r, j0 + c));
  }
  __shared__ int s_zero, s_pend, s_ok, s_cand, s_fast, s_near;
  __shared__ double s_rcp[2 * L], s_key[L], s_k0;
  __shared__ double s_bk[4 * L];
  __shared__ int s_bi[4];
  if (tid == 0) {
    s_pend = 0;
    s_ok = 1;
  }
  __syncthreads();
  if (w >= 4) {
    // ------------------------------------------------------- update team
    // Iteration jc: the pending rank-1 update of column jc-1 (rows i >= j,
    // columns jc+1 ..), from the go signal the factor team gives once the
    // multipliers of column jc-1 are final, to the done signal it waits for
    // before publishing rows of column jc.
    // The update runs on warps 5, 6 and 7 (SMSPs 1, 2, 3); warp 4 stays
    // off SMSP 0, whose FP64 unit carries the factor team's serial chain
    // (measured: with warp 4 and per-component items, TD panel 94.1 ->
    // 96.7 ms, QD 189.0 -> 187.0 ms at n = 4096).
    const int ut = tid - 160;  // warps 5..7: 0 .. 95
    for (int jc = 0; jc < nb; jc++) {
      named_sync(BAR_GO, 256);
      if (!s_ok) break;
      if (s_pend && ut >= 0) {
        const int64_t j = j0 + jc;
        const double *sprev = su2 + (size_t)((jc & 1) ^ 1) * RW;
        const int rlo = (int)max((int64_t)0, j - rbeg);  // rows i > j - 1
        const int nrow = nr - rlo, ncol = nb - jc - 1;
        const int tot = nrow > 0 ? nrow * ncol : 0;
        for (int t = ut; t < tot; t += 96) {
          const int rr = rlo + t % nrow, cc = jc + 1 + t / nrow;
          stp(rr, cc, upd(rr, cc, jc - 1, sprev));
        }
      }
      named_arrive(BAR_DONE, 224);
    }
  } else {
    // ------------------------------------------------------- factor team
    named_arrive(BAR_GO, 256);  // iteration 0 of the update team: nothing pending
    for (int jc = 0; jc < nb; jc++) {
      const int64_t j = j0 + jc;
      const int par = jc & 1;
      double *su = su2 + (size_t)par * RW;  // pivot row of column jc
      const int q = par * G + b;
      // 1. the CTA's candidate among its rows i >= j (column jc is up to
      //    date): the largest k0 (one FP64 addition per row), unless another
      //    row's k0 is near it; then the full keys of the near rows decide
      //    (s_fast = 0, s_key the full key)
      {
        R<1> k1 = invalid_key<1>();
        int idx = INT_MAX;
        for (int r = tid; r < nr; r += 128) {
          const int64_t i = rbeg + r;
          if (i < j) continue;
          R<1> k;
          k.x[0] = cheap_key<L>(sp, jc, rpc, r);
          if (better<1>(k, (int)i, k1, idx)) {
            k1 = k;
            idx = (int)i;
          }
        }
        warp_argmax<1>(k1, idx);
        if (lane == 0) {
          s_bk[w * L] = k1.x[0];
          s_bi[w] = idx;
        }
        if (tid == 0) s_near = 0;
        named_sync(BAR_MAIN, 128);
        if (tid == 0) {
#pragma unroll
          for (int v = 1; v < 4; v++) {
            R<1> k;
            k.x[0] = s_bk[v * L];
            if (better<1>(k, s_bi[v], k1, idx)) {
              k1 = k;
              idx = s_bi[v];
            }
          }
          s_k0 = k1.x[0];
          s_cand = idx;
        }
        named_sync(BAR_MAIN, 128);
        const double kmax = s_k0;
        const int c0 = s_cand;
        if (c0 != INT_MAX) {
          for (int r = tid; r < nr; r += 128) {
            const int64_t i = rbeg + r;
            if (i >= j && i != c0 && key_near(cheap_key<L>(sp, jc, rpc, r), kmax)) s_near = 1;
          }
        }
        named_sync(BAR_MAIN, 128);
        const bool near = s_near != 0;
        if (near) {
          R<L> key = invalid_key<L>();
          idx = INT_MAX;
          for (int r = tid; r < nr; r += 128) {
            const int64_t i = rbeg + r;
            if (i < j || !key_near(cheap_key<L>(sp, jc, rpc, r), kmax)) continue;
            const R<L> k = pivot_key<L>(ldp(r, jc));
            if (better<L>(k, (int)i, key, idx)) {
              key = k;
              idx = (int)i;
            }
          }
          warp_argmax<L>(key, idx);
          if (lane == 0) {
#pragma unroll
            for (int l = 0; l < L; l++) s_bk[w * L + l] = key.x[l];
            s_bi[w] = idx;
          }
          named_sync(BAR_MAIN, 128);
          if (tid == 0) {
#pragma unroll
            for (int v = 1; v < 4; v++) {
              R<L> k;
#pragma unroll
              for (int l = 0; l < L; l++) k.x[l] = s_bk[v * L + l];
              if (better<L>(k, s_bi[v], key, idx)) {
                key = k;
                idx = s_bi[v];
              }
            }
#pragma unroll
            for (int l = 0; l < L; l++) s_key[l] = key.x[l];
            s_cand = idx;
          }
        }
        if (tid == 0) s_fast = near ? 0 : 1;
        named_sync(BAR_MAIN, 128);
      }
      const int cand = s_cand;
      const bool fast = s_fast != 0;
      const bool has = cand != INT_MAX;                                // uniform over the CTA
      const int cr = has ? (int)(cand - rbeg) : -1;                    // local row of the candidate
      const int jr = (j >= rbeg && j < rend) ? (int)(j - rbeg) : -1;  // local row j
      if (w < 3) {
        // 2. warps 0 and 1: the reciprocal 1/p of the candidate (Newton's
        //    method, its real and imaginary chains on SMSPs 0 and 1); then,
        //    once the update team is done with column
        //    jc-1, warp 2 publishes the candidate row and row j, and thread 0
        //    releases the slot's flag
        if (w < 2) {
          // 1/p by Newton's method (z_inv_newton): the binary64 seed and the
          // two-limb step with the real part on warp 0 and the imaginary part
          // on warp 1, then the L-limb step: warp 0 forms P_rr, P_ii and Re e,
          // warp 1 P_ri, P_ir and Im e, and each its part of r'
          __shared__ double s_e[2], s_r2[4], s_el[4];
          const bool act = has && lane == 0;
          Z<L> pv;
          RcpSeed sd;
          if (act) {
            pv = ldp(cr, jc);
            sd = rcp_seed(pv.re.x[0], pv.im.x[0]);
            s_e[w] = w == 0 ? rcp_resid_re<L>(pv.re, pv.im, sd) : rcp_resid_im<L>(pv.re, pv.im, sd);
          }
          named_sync(BAR_RCP, 64);
          R<L> v;
          if (act) {
            v = w == 0 ? rcp_finish<L, false>(sd, s_e[0], s_e[1]) : rcp_finish<L, true>(sd, s_e[0], s_e[1]);
            s_r2[2 * w] = v.x[0];
            s_r2[2 * w + 1] = v.x[1];
          }
          if constexpr (L >= 3) {
            named_sync(BAR_RCP, 64);
            const double r2[4] = {s_r2[0], s_r2[1], s_r2[2], s_r2[3]};
            if (act) {
              Acc<L> Pa, Pb;
              rcp_prod<L>(Pa, pv.re, r2[2 * w], r2[2 * w + 1]);  // P_rr (warp 0), P_ri (warp 1)
              rcp_prod<L>(Pb, pv.im, r2[2 - 2 * w], r2[3 - 2 * w]);  // P_ii, P_ir
              const R<L> e = w == 0 ? rcp_resid_l<L, false>(Pa, Pb) : rcp_resid_l<L, true>(Pa, Pb);
              s_el[2 * w] = e.x[0];
              s_el[2 * w + 1] = e.x[1];
            }
            named_sync(BAR_RCP, 64);
            if (act) {
              const double e2[4] = {s_el[0], s_el[1], s_el[2], s_el[3]};
              v = w == 0 ? rcp_newton<L, false>(r2, e2) : rcp_newton<L, true>(r2, e2);
            }
          }
          if (act) {
#pragma unroll
            for (int l = 0; l < L; l++) ws.part_rcp[(int64_t)q * 2 * L + w * L + l] = v.x[l];
          }
        }
        if (w == 2 && lane == 0 && has && fast)  // the full key, off the reciprocal's SMSPs
          publish_full_key<L>(cw.kslot + (size_t)q * COOP_KS, j, pivot_key<L>(ldp(cr, jc)));
        named_sync(BAR_DONE, 224);  // the update of column jc-1 is complete
        if (w == 2) {
          if (cr >= 0) {
            double *dst = cw.prow + (size_t)q * RW;
            for (int t = lane; t < RW; t += 32) dst[t] = rowel(cr, t);
          }
          if (jr >= 0) {
            double *dst = cw.srow + (size_t)par * RW;
            for (int t = lane; t < RW; t += 32) dst[t] = rowel(jr, t);
          }
        }
        named_sync(BAR_PUB, 96);
        if (has && tid == 0) {
          __threadfence();
          st_release(cw.rcp_flag + q, (int)(j + 1));
        }
        named_arrive(BAR_SWAP, 128);  // rows cr and jr are final: warp 3 may swap them
      } else {
        // 3. warp 3: this CTA's candidate (k0, row; the full key when known)
        //    to its slot, stamped; then the winner over all key slots of this
        //    column (exchange_winner)
        if (lane == 0) {
          R<L> inv = invalid_key<L>();
          publish_key_slot<L>(cw.kslot + (size_t)q * COOP_KS, j, cand, has ? s_k0 : -1.0, !has || !fast,
                              has ? s_key : inv.x);
        }
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
        named_sync(BAR_SWAP, 128);  // the update of column jc-1 is complete
        if (ok && !zero) {
          if (own_p) {
            const double *srow = cw.srow + (size_t)par * RW;
            for (int t = lane; t < RW; t += 32) rowel((int)(p - rbeg), t) = __ldcg(srow + t);
          }
          if (p != j && jr >= 0)
            for (int t = lane; t < RW; t += 32) rowel(jr, t) = su[t];
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
      }
      named_sync(BAR_MAIN, 128);
      if (!s_ok) {  // release the update team (it stops at its next go signal)
        if (jc + 1 < nb) named_arrive(BAR_GO, 256);
        break;
      }
      if (s_zero) {  // nothing to eliminate in this column; no swap; the next
                     // pivot column is renormalised for its keys
        if (jc + 1 < nb) {
          for (int rr = tid; rr < nr; rr += 128) {
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
          if (tid == 0) s_pend = 0;
          named_sync(BAR_MAIN, 128);
          named_arrive(BAR_GO, 256);
        }
        continue;
      }
      Z<L> r;
#pragma unroll
      for (int l = 0; l < L; l++) {
        r.re.x[l] = s_rcp[l];
        r.im.x[l] = s_rcp[L + l];
      }
      // 4. multipliers l = a r of the rows below j: warps 0..3 (one per
      //    SMSP, each with its own FP64 unit) form the four real products
      //    Re a Re r, Im a Im r, Re a Im r, Im a Re r on leveled
      //    accumulators; warps 0 and 1 then form Re l = P0 - P1 and
      //    Im l = P2 + P3
      {
        const R<L> y = (w == 0 || w == 3) ? r.re : r.im;
        for (int rr = lane; rr < nr; rr += 32) {
          if (rbeg + rr <= j) continue;
          const Z<L> a = ldp(rr, jc);
          Acc<L> t;
          t.set_prod((w == 0 || w == 2) ? a.re : a.im, y);
#pragma unroll
          for (int l = 0; l < L; l++) mscr[((size_t)w * rpc + rr) * L + l] = t.s[l];
        }
      }
      named_sync(BAR_MAIN, 128);
      if (w < 2) {
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
      }
      if (jc + 1 < nb) {
        if (tid == 0) s_pend = jc + 2 < nb ? 1 : 0;
        named_sync(BAR_MAIN, 128);
        // the multipliers of column jc are final: the update team takes
        // columns jc+2 .. while this team updates column jc+1, renormalised
        // for its keys, split like the multipliers: warps 0..3 form
        // Re l Re u, Im l Im u, Re l Im u, Im l Re u; warps 0 and 1 take
        // a - P0 + P1 and a - P2 - P3
        named_arrive(BAR_GO, 256);
        const int cc = jc + 1;
        {
          R<L> y;
#pragma unroll
          for (int l = 0; l < L; l++) y.x[l] = su[cc * 2 * L + ((w == 0 || w == 3) ? 0 : L) + l];
          for (int rr = lane; rr < nr; rr += 32) {
            if (rbeg + rr <= j) continue;
            const Z<L> lv = ldp(rr, jc);
            Acc<L> t;
            t.set_prod((w == 0 || w == 2) ? lv.re : lv.im, y);
#pragma unroll
            for (int l = 0; l < L; l++) mscr[((size_t)w * rpc + rr) * L + l] = t.s[l];
          }
        }
        named_sync(BAR_MAIN, 128);
        if (w < 2) {
          for (int rr = lane; rr < nr; rr += 32) {
            if (rbeg + rr <= j) continue;
            const Z<L> a = ldp(rr, cc);
            Acc<L> t, o;
            t.set(w == 0 ? a.re : a.im);
#pragma unroll
            for (int l = 0; l < L; l++) o.s[l] = mscr[((size_t)(2 * w) * rpc + rr) * L + l];
            t.add_acc(o, true);
#pragma unroll
            for (int l = 0; l < L; l++) o.s[l] = mscr[((size_t)(2 * w + 1) * rpc + rr) * L + l];
            t.add_acc(o, w == 1);
            const R<L> v = t.result();
            double *d = sp + (size_t)cc * 2 * L * rpc + rr + (size_t)(w * L) * rpc;
#pragma unroll
            for (int l = 0; l < L; l++) d[(size_t)l * rpc] = v.x[l];
          }
        }
      }
      named_sync(BAR_MAIN, 128);
    }
  }
  __syncthreads();
  if (!s_ok) return;
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
