// lu_kernels.cuh - CUDA kernels of the complex multi-component LU (Sec. 3) and
// solve (Sec. 4), templated on the limb count L (2 DD, 3 TD, 4 QD).
//
// All arithmetic is on the FP64 pipe through mc.cuh.  On GB300 the FP64 pipe
// is the scarce unit (about 1.6 results per clock per SM, against ~110 for
// FP32), so every kernel here is sized for FP64 issue, not for bandwidth:
// enough independent elements per SM to keep the FP64 pipe busy, operands
// staged in shared memory once per tile, no redundant multi-component work.
//
// Pivoting (partial pivoting of Sec. 3): the key is cabs1 = |Re| + |Im| in
// L-limb arithmetic, compared lexicographically on the renormalised limbs
// (integer compares); ties go to the lowest row.  A column's search spans
// many CTAs: each writes a partial (key, row); the CTA that arrives last on an
// atomic counter (threadfence-reduction pattern, no waiting anywhere) reduces
// the partials, swaps the pivot row inside the panel, records ipiv and info,
// and leaves the reciprocal of the pivot for the next launch.
#pragma once

#include <climits>

#include "mc.cuh"

namespace mclu {

constexpr int PANEL_T = 16;   // panel-step CTA: 16 rows x 16 columns of the panel
constexpr int SEARCH_T = 256; // threads of a pivot-search CTA
constexpr int GEMM_T = 16;    // GEMM CTA tile: 16 x 16 outputs, k staged 16 at a time

// Workspace shared by the panel kernels of one factorisation.
template <int L>
struct PanelWS {
  int *counter;     // arrival counter of the last-CTA pattern (reset by the last CTA)
  int *info;        // first zero pivot, 1-based (0 = none)
  int *zflag;       // 1 if the current pivot column was entirely zero
  double *recip;    // [2L] reciprocal of the current pivot (re limbs, im limbs)
  double *part_key; // [nparts][L]
  int *part_idx;    // [nparts]
  double *part_rcp; // [nparts][2L] reciprocal of each partial's candidate
  double *lbuf;     // [2][2L][lbuf_ld] pending multipliers of a column (double buffered)
  int64_t lbuf_ld;
};

template <int L>
__device__ __forceinline__ bool better(const R<L> &ka, int ia, const R<L> &kb, int ib) {
  if (r_gt<L>(ka, kb)) return true;
  if (r_gt<L>(kb, ka)) return false;
  return ia < ib;
}

template <int L>
__device__ __forceinline__ R<L> invalid_key_() {
  R<L> k;
#pragma unroll
  for (int l = 0; l < L; l++) k.x[l] = 0.0;
  k.x[0] = -1.0;
  return k;
}

// Warp argmax of (key, idx) under `better` (value, then the lower index).
// The leading limb decides almost always: its order key is reduced with two
// 32-bit __reduce_max_sync steps and a ballot; when several lanes share the
// largest leading limb, they are compared in full, one lane at a time.
// Every lane returns the warp's winner.
template <int L>
__device__ __forceinline__ void warp_argmax(R<L> &key, int &idx) {
  const unsigned long long u = (unsigned long long)order_key(key.x[0]) ^ 0x8000000000000000ULL;
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  unsigned cand = __ballot_sync(0xffffffffu, hi == mhi && lo == mlo);
  int win = __ffs(cand) - 1;
  // equal leading limbs: full comparison among the candidates (unless the
  // largest leading limb is negative, i.e. every lane holds the invalid key)
  if (__popc(cand) > 1 && mhi >= 0x80000000u) {
    R<L> bk;
    int bi;
#pragma unroll
    for (int l = 0; l < L; l++) bk.x[l] = __shfl_sync(0xffffffffu, key.x[l], win);
    bi = __shfl_sync(0xffffffffu, idx, win);
    cand &= cand - 1;
    while (cand) {
      const int c = __ffs(cand) - 1;
      cand &= cand - 1;
      R<L> ck;
#pragma unroll
      for (int l = 0; l < L; l++) ck.x[l] = __shfl_sync(0xffffffffu, key.x[l], c);
      const int ci = __shfl_sync(0xffffffffu, idx, c);
      if (better<L>(ck, ci, bk, bi)) {
        bk = ck;
        bi = ci;
        win = c;
      }
    }
  }
#pragma unroll
  for (int l = 0; l < L; l++) key.x[l] = __shfl_sync(0xffffffffu, key.x[l], win);
  idx = __shfl_sync(0xffffffffu, idx, win);
}

// Block-wide argmax; nthr a multiple of 32 (at most 1024); result in (key,
// idx) of thread 0.  Each warp reduces with warp_argmax, the warp results
// meet in shared memory and warp 0 reduces them.
template <int L>
__device__ void block_argmax(R<L> &key, int &idx, int tid, int nthr) {
  __shared__ double s_key[32 * L];
  __shared__ int s_idx[32];
  const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
  warp_argmax<L>(key, idx);
  if (lane == 0) {
#pragma unroll
    for (int l = 0; l < L; l++) s_key[warp * L + l] = key.x[l];
    s_idx[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    R<L> k = invalid_key_<L>();
    int i = INT_MAX;
    if (lane < nw) {
#pragma unroll
      for (int l = 0; l < L; l++) k.x[l] = s_key[lane * L + l];
      i = s_idx[lane];
    }
    warp_argmax<L>(k, i);
    if (lane == 0) {
      key = k;
      idx = i;
    }
  }
  __syncthreads();
}

template <int L>
__device__ __forceinline__ R<L> invalid_key() {
  return invalid_key_<L>();
}

// Last-CTA finalisation of the pivot of column jp: reduce nparts partials,
// record ipiv/info, swap rows jp <-> p over panel columns [j0, jend) (and the
// pending multipliers of column jcol in lbuf slot `pend` if pend >= 0), then
// compute the reciprocal of the new pivot.
template <int L>
__device__ void finalize_pivot(View A, int64_t n, int64_t jp, int64_t j0, int64_t jend, int32_t *ipiv,
                               PanelWS<L> ws, int nparts, int pend, int tid, int nthr) {
  R<L> key = invalid_key<L>();
  int idx = INT_MAX, part = -1;
  for (int q = tid; q < nparts; q += nthr) {
    R<L> k;
#pragma unroll
    for (int l = 0; l < L; l++) k.x[l] = __ldcg(ws.part_key + (int64_t)q * L + l);
    int i = __ldcg(ws.part_idx + q);
    if (better<L>(k, i, key, idx)) {
      key = k;
      idx = i;
      part = q;
    }
  }
  __shared__ int s_part;
  const int my_idx = idx;
  block_argmax<L>(key, idx, tid, nthr);
  __shared__ int s_win;
  if (tid == 0) s_win = idx;
  __syncthreads();
  if (my_idx == s_win && my_idx != INT_MAX) s_part = part;  // the thread that read the winning partial
  __syncthreads();
  __shared__ int s_p, s_zero;
  if (tid == 0) {
    bool zero = !(key.x[0] > 0.0);
    int64_t p = (idx == INT_MAX || zero) ? jp : idx;
    s_p = (int)p;
    s_zero = zero ? 1 : 0;
    ipiv[jp] = (int32_t)(p + 1);
    *ws.zflag = zero ? 1 : 0;
    if (zero && *ws.info == 0) *ws.info = (int)(jp + 1);
  }
  __syncthreads();
  const int64_t p = s_p;
  if (p != jp) {
    const int64_t w = jend - j0;
    for (int64_t t = tid; t < w * 2 * L; t += nthr) {
      int64_t c = j0 + t / (2 * L);
      int pl = (int)(t % (2 * L));
      double *P = A.p + (int64_t)pl * A.ps + c * A.ld;
      double a = P[jp], b = P[p];
      P[jp] = b;
      P[p] = a;
    }
    if (pend >= 0) {
      for (int pl = tid; pl < 2 * L; pl += nthr) {
        double *P = ws.lbuf + ((int64_t)pend * 2 * L + pl) * ws.lbuf_ld;
        double a = P[jp], b = P[p];
        P[jp] = b;
        P[p] = a;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (!s_zero) {  // the winning candidate computed its reciprocal already
#pragma unroll
      for (int l = 0; l < 2 * L; l++) ws.recip[l] = __ldcg(ws.part_rcp + (int64_t)s_part * 2 * L + l);
    }
    *ws.counter = 0;
    __threadfence();
  }
}

// Block argmax of (key, row) that also publishes the reciprocal of the
// winner's value into the block's partial q.
template <int L>
__device__ int write_partial(R<L> key, int idx, const Z<L> &rcp, PanelWS<L> ws, int q, int tid, int nthr) {
  const int my_idx = idx;
  block_argmax<L>(key, idx, tid, nthr);
  __shared__ int s_w;
  if (tid == 0) {
#pragma unroll
    for (int l = 0; l < L; l++) ws.part_key[(int64_t)q * L + l] = key.x[l];
    ws.part_idx[q] = idx;
    s_w = idx;
  }
  __syncthreads();
  const int w = s_w;
  if (my_idx == w && my_idx != INT_MAX) {
#pragma unroll
    for (int l = 0; l < L; l++) {
      ws.part_rcp[(int64_t)q * 2 * L + l] = rcp.re.x[l];
      ws.part_rcp[(int64_t)q * 2 * L + L + l] = rcp.im.x[l];
    }
  }
  return w;
}

// True in exactly one CTA per launch: the last one to arrive.
__device__ __forceinline__ bool arrive_last(int *counter, int nblocks, int tid) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    int prev = atomicAdd(counter, 1);
    s_last = (prev == nblocks - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Pivot search of column j over rows [j, n) (first column of a panel).
template <int L>
__global__ void __launch_bounds__(SEARCH_T) k_pivot_first(View A, int64_t n, int64_t j, int64_t j0, int64_t jend,
                                                          int32_t *ipiv, PanelWS<L> ws) {
  const int tid = threadIdx.x;
  const int64_t i = j + (int64_t)blockIdx.x * SEARCH_T + tid;
  R<L> key = invalid_key<L>();
  int idx = INT_MAX;
  Z<L> rcp = z_zero<L>();
  if (i < n) {
    const Z<L> a = ldz<L>(A, i, j);
    key = pivot_key<L>(a);
    idx = (int)i;
    rcp = z_inv<L>(a);  // speculative: kept only if this row wins
  }
  write_partial<L>(key, idx, rcp, ws, blockIdx.x, tid, SEARCH_T);
  if (arrive_last(ws.counter, gridDim.x, tid))
    finalize_pivot<L>(A, n, j, j0, jend, ipiv, ws, gridDim.x, -1, tid, SEARCH_T);
}

__host__ __device__ __forceinline__ int panel_colblocks(int64_t j, int64_t jend) {
  int64_t c = jend - j - 1;
  return c <= 0 ? 1 : (int)((c + PANEL_T - 1) / PANEL_T);
}

// One column step of the panel [j0, jend): scale column j by the pivot's
// reciprocal (multipliers l_i, Sec. 3 / the paper's "inv" operation), update
// the panel columns j+1..jend-1 (A_ic -= l_i A_jc), and search the pivot of
// column j+1.  Grid: (row blocks of rows j+1..n-1, column blocks).
template <int L>
__global__ void __launch_bounds__(PANEL_T *PANEL_T)
    k_panel_step(View A, int64_t n, int64_t j, int64_t j0, int64_t jend, int32_t *ipiv, PanelWS<L> ws) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PANEL_T + tx;
  const int64_t i = j + 1 + (int64_t)blockIdx.x * PANEL_T + tx;
  const bool row_ok = i < n;
  const bool via_lbuf = gridDim.y > 1;
  const int slot = (int)(j & 1);
  __shared__ double s_l[PANEL_T][2 * L];
  __shared__ double s_u[PANEL_T][2 * L];
  const int zero = *ws.zflag;

  // flush the multipliers of column j-1 if they were left in lbuf
  if (j > j0 && panel_colblocks(j - 1, jend) > 1 && blockIdx.y == 0 && ty == 1) {
    const int ps = 1 - slot;
    const int64_t fi = i;
    if (fi < n) {
#pragma unroll
      for (int pl = 0; pl < 2 * L; pl++)
        A.p[(int64_t)pl * A.ps + (j - 1) * A.ld + fi] = ws.lbuf[((int64_t)ps * 2 * L + pl) * ws.lbuf_ld + fi];
    }
    if (blockIdx.x == 0 && tx == 0) {  // row j, not in this launch's row range
#pragma unroll
      for (int pl = 0; pl < 2 * L; pl++)
        A.p[(int64_t)pl * A.ps + (j - 1) * A.ld + j] = ws.lbuf[((int64_t)ps * 2 * L + pl) * ws.lbuf_ld + j];
    }
  }

  // multipliers of this CTA's rows
  if (ty == 0) {
    Z<L> l = z_zero<L>();
    if (row_ok) {
      Z<L> a = ldz<L>(A, i, j);
      if (zero) {
        l = a;
      } else {
        Z<L> r;
#pragma unroll
        for (int q = 0; q < L; q++) {
          r.re.x[q] = ws.recip[q];
          r.im.x[q] = ws.recip[L + q];
        }
        l = z_mul<L>(a, r);
      }
      if (!via_lbuf) {
        stz<L>(A, i, j, l);
      } else if (blockIdx.y == 0) {
#pragma unroll
        for (int q = 0; q < L; q++) {
          ws.lbuf[((int64_t)slot * 2 * L + q) * ws.lbuf_ld + i] = l.re.x[q];
          ws.lbuf[((int64_t)slot * 2 * L + L + q) * ws.lbuf_ld + i] = l.im.x[q];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < L; q++) {
      s_l[tx][q] = l.re.x[q];
      s_l[tx][L + q] = l.im.x[q];
    }
  }
  // pivot-row entries of this CTA's columns
  const int64_t cbase = j + 1 + (int64_t)blockIdx.y * PANEL_T;
  if (ty == 1 && cbase + tx < jend) {
    Z<L> u = ldz<L>(A, j, cbase + tx);
#pragma unroll
    for (int q = 0; q < L; q++) {
      s_u[tx][q] = u.re.x[q];
      s_u[tx][L + q] = u.im.x[q];
    }
  }
  __syncthreads();

  const int64_t c = cbase + ty;
  Z<L> updated;
  if (row_ok && c < jend && !zero) {
    Z<L> l, u;
#pragma unroll
    for (int q = 0; q < L; q++) {
      l.re.x[q] = s_l[tx][q];
      l.im.x[q] = s_l[tx][L + q];
      u.re.x[q] = s_u[ty][q];
      u.im.x[q] = s_u[ty][L + q];
    }
    updated = z_fms<L>(ldz<L>(A, i, c), l, u);
    stz<L>(A, i, c, updated);
  } else if (row_ok && c < jend) {
    updated = ldz<L>(A, i, c);
  }

  // pivot search of column j+1 (CTAs of column block 0, threads ty == 0)
  const bool search = (j + 1 < jend);
  if (search) {
    if (blockIdx.y == 0) {
      R<L> key = invalid_key<L>();
      int idx = INT_MAX;
      Z<L> rcp = z_zero<L>();
      if (ty == 0 && row_ok) {
        key = pivot_key<L>(updated);
        idx = (int)i;
        rcp = z_inv<L>(updated);  // speculative: kept only if this row wins
      }
      write_partial<L>(key, idx, rcp, ws, blockIdx.x, tid, PANEL_T * PANEL_T);
    }
    if (arrive_last(ws.counter, gridDim.x * gridDim.y, tid))
      finalize_pivot<L>(A, n, j + 1, j0, jend, ipiv, ws, gridDim.x, via_lbuf ? slot : -1, tid, PANEL_T * PANEL_T);
  }
}

// Apply the row swaps ipiv[k0..k1) of one panel to the columns [c0, c1)
// other than [x0, x1) (x0 = x1: none excluded; the excluded range lies inside
// [c0, c1)), numbered c' = 0 .. ncols - 1, all 2L planes.  The swaps only
// touch rows [k0, k1) and their partners p >= k, so their product is a
// permutation of at most 2 (k1 - k0) rows (slot s < nb is row k0 + s, later
// slots hold the distinct partner rows at or below k1; org[s] = the row whose
// content ends in slot s's row).  Every CTA builds it in shared memory: each
// thread finds whether its partner row occurs earlier (the first occurrence
// gets a slot, numbered by a block prefix sum), then one thread applies the
// transpositions in order as swaps of org entries (two shared-memory reads
// and writes per swap).  Then each CTA gathers the moved rows of its
// LASWP_C columns into registers, plane by plane, and writes them back
// permuted.  Rows in [k0, k1) are contiguous in a column (coalesced);
// partner rows cost one sector each.  k1 - k0 <= LASWP_NB_MAX (one pivot per
// thread).
constexpr int LASWP_C = 16;        // columns per CTA
constexpr int LASWP_NB_MAX = 256;  // most swaps of one launch
constexpr int LASWP_K = 2 * LASWP_NB_MAX * LASWP_C / 256;  // moved elements a thread holds

inline size_t laswp_smem(int nb) { return (size_t)2 * nb * 2 * sizeof(int) + (size_t)4 * nb * sizeof(int) + 16; }

template <int L>
__global__ void __launch_bounds__(256) k_laswp_gather(View A, int64_t k0, int64_t k1, const int32_t *ipiv,
                                                      int64_t c0, int64_t c1, int64_t x0, int64_t x1) {
  const int nb = (int)(k1 - k0);
  extern __shared__ double lsm[];
  int *dst = reinterpret_cast<int *>(lsm);                 // [2 nb]
  int *org = dst + 2 * nb;                                 // [2 nb]
  int *piv = org + 2 * nb;                                 // [nb] the pivots, read once
  int *fidx = piv + nb;                                    // [nb] first pivot with the same partner row
  int *pslot = fidx + nb;                                  // [nb] slot of a first partner occurrence
  int *slotof = pslot + nb;                                // [nb] slot of the row swapped with row k0 + k
  __shared__ int s_cnt, s_wsum[8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < nb) piv[tid] = ipiv[k0 + tid] - 1;
  __syncthreads();
  int first = 0;
  if (tid < nb) {
    const int p = piv[tid];
    int f = -1;
    if (p >= k1) {  // a partner row below the panel's rows: its first occurrence
      f = tid;
      for (int t2 = 0; t2 < tid; t2++)
        if (piv[t2] == p) {
          f = t2;
          break;
        }
      first = f == tid;
    }
    fidx[tid] = f;
    dst[tid] = (int)k0 + tid;
    org[tid] = (int)k0 + tid;
  }
  int incl = first;  // block prefix sum of the first occurrences (8 warps)
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) s_wsum[w] = incl;
  __syncthreads();
  int base = 0;
  for (int v = 0; v < w; v++) base += s_wsum[v];
  if (first) {
    const int sl = nb + base + incl - 1;
    pslot[tid] = sl;
    dst[sl] = piv[tid];
    org[sl] = piv[tid];
  }
  if (tid == 0) {
    int tot = 0;
    for (int v = 0; v < 8; v++) tot += s_wsum[v];
    s_cnt = tot;
  }
  __syncthreads();
  if (tid < nb) {
    const int p = piv[tid];
    slotof[tid] = p < k1 ? p - (int)k0 : pslot[fidx[tid]];
  }
  __syncthreads();
  if (tid == 0) {  // the transpositions in order
    for (int k = 0; k < nb; k++) {
      const int sb = slotof[k];
      if (sb != k) {
        const int t = org[k];
        org[k] = org[sb];
        org[sb] = t;
      }
    }
  }
  __syncthreads();
  const int T = nb + s_cnt;
  const int64_t ncols = (c1 - c0) - (x1 - x0);
  const int64_t cb = (int64_t)blockIdx.x * LASWP_C;
  // each thread gathers up to LASWP_K (slot, column) elements of a plane into
  // registers before it stores any of them, so that its loads are in flight
  // together (T LASWP_C <= LASWP_K x 256 threads)
  for (int pl = 0; pl < 2 * L; pl++) {
    double *P = A.p + (int64_t)pl * A.ps;
    double v[LASWP_K];
#pragma unroll
    for (int k = 0; k < LASWP_K; k++) {
      const int t = tid + 256 * k;
      const int sl = t % T, cl = t / T;
      const int64_t cc = cb + cl;
      if (t < T * LASWP_C && cc < ncols && org[sl] != dst[sl]) {
        const int64_t c = (c0 + cc < x0) ? c0 + cc : c0 + cc + (x1 - x0);
        v[k] = P[c * A.ld + org[sl]];
      }
    }
    __syncthreads();  // every row read before any is written
#pragma unroll
    for (int k = 0; k < LASWP_K; k++) {
      const int t = tid + 256 * k;
      const int sl = t % T, cl = t / T;
      const int64_t cc = cb + cl;
      if (t < T * LASWP_C && cc < ncols && org[sl] != dst[sl]) {
        const int64_t c = (c0 + cc < x0) ? c0 + cc : c0 + cc + (x1 - x0);
        P[c * A.ld + dst[sl]] = v[k];
      }
    }
    __syncthreads();
  }
}

// acc_re + i acc_im -= a b (complex, on the leveled accumulators)
template <int L>
__device__ __forceinline__ void acc_csub(Acc<L> &re, Acc<L> &im, const Z<L> &a, const Z<L> &b) {
  re.template add_prod<true>(a.re, b.re);
  re.template add_prod<false>(a.im, b.im);
  im.template add_prod<true>(a.re, b.im);
  im.template add_prod<true>(a.im, b.re);
}

// acc_re + i acc_im += a b
template <int L>
__device__ __forceinline__ void acc_cadd(Acc<L> &re, Acc<L> &im, const Z<L> &a, const Z<L> &b) {
  re.template add_prod<false>(a.re, b.re);
  re.template add_prod<true>(a.im, b.im);
  im.template add_prod<false>(a.re, b.im);
  im.template add_prod<false>(a.im, b.re);
}

template <int L>
__device__ __forceinline__ Z<L> lds_z(const double *p) {
  Z<L> z;
#pragma unroll
  for (int q = 0; q < L; q++) {
    z.re.x[q] = p[q];
    z.im.x[q] = p[L + q];
  }
  return z;
}

template <int L>
__device__ __forceinline__ void sts_z(double *p, const Z<L> &z) {
#pragma unroll
  for (int q = 0; q < L; q++) {
    p[q] = z.re.x[q];
    p[L + q] = z.im.x[q];
  }
}

// Triangular block solve T x = b for the bs x bs diagonal block of A at
// (k0, k0) on columns of X (rows xrow0..xrow0+bs-1); rdiag (planes
// [2L][rld]) holds 1/T_kk when the diagonal is not unit.  T = A (LOWER: unit or not) or,
// with CONJT, T(r, k) = conj(A(k0+k, k0+r)).  Right-looking inside the block:
// at step k the owner of row k finalises x_k (dividing by T_kk if !UNIT) and
// every row below (LOWER) or above (!LOWER) subtracts T(r,k) x_k.
// Block: (RT rows, CT columns); grid.x over column groups.
template <int L, bool LOWER, bool UNIT, bool CONJT, bool STAGE>
__global__ void k_tri_block(View A, int64_t k0, int bs, View X, int64_t ncols, const double *rdiag, int64_t rld,
                            int64_t xrow0) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int RT = blockDim.x, CT = blockDim.y;
  const int64_t c = (int64_t)blockIdx.x * CT + ty;
  const bool ok = tx < bs && c < ncols;
  // dynamic shared memory: [STAGE: T block [bs][bs][2L] (row r, step k) and
  // diagonal reciprocals [bs][2L]], exchange slots [CT][2L]
  extern __shared__ double smem[];
  double *sT = smem;
  double *sR = sT + (STAGE ? (size_t)bs * bs * 2 * L : 0);
  double *s_x = sR + (STAGE ? (size_t)bs * 2 * L : 0);
  // stage the triangle once: T(r, k) = A(k0+r, k0+k) or conj(A(k0+k, k0+r))
  for (int t = ty * RT + tx; STAGE && t < bs * bs; t += RT * CT) {
    const int r = t % bs, kk = t / bs;
    const bool need = LOWER ? (r > kk) : (r < kk);
    Z<L> v = z_zero<L>();
    if (need) v = CONJT ? z_conj<L>(ldz<L>(A, k0 + kk, k0 + r)) : ldz<L>(A, k0 + r, k0 + kk);
#pragma unroll
    for (int q = 0; q < L; q++) {
      sT[((size_t)r * bs + kk) * 2 * L + q] = v.re.x[q];
      sT[((size_t)r * bs + kk) * 2 * L + L + q] = v.im.x[q];
    }
  }
  if (!UNIT && STAGE) {
    for (int t = ty * RT + tx; t < bs * 2 * L; t += RT * CT) {
      const int kk = t / (2 * L), q = t % (2 * L);
      sR[t] = rdiag[(int64_t)q * rld + k0 + kk];
    }
  }
  // row tx accumulates its updates on leveled accumulators and is
  // renormalised once, at the step that finalises it
  Z<L> x;
  Acc<L> are, aim;
  if (ok) {
    x = ldz<L>(X, xrow0 + tx, c);
    are.set(x.re);
    aim.set(x.im);
  }
  __syncthreads();
  for (int s = 0; s < bs; s++) {
    const int k = LOWER ? s : bs - 1 - s;
    if (ok && tx == k) {
      x.re = are.result();
      x.im = aim.result();
      if (!UNIT) {  // multiply by the precomputed reciprocal of T_kk
        Z<L> r;
#pragma unroll
        for (int q = 0; q < L; q++) {
          r.re.x[q] = STAGE ? sR[k * 2 * L + q] : rdiag[(int64_t)q * rld + k0 + k];
          r.im.x[q] = STAGE ? sR[k * 2 * L + L + q] : rdiag[(int64_t)(L + q) * rld + k0 + k];
        }
        x = z_mul<L>(x, r);
      }
#pragma unroll
      for (int q = 0; q < L; q++) {
        s_x[ty * 2 * L + q] = x.re.x[q];
        s_x[ty * 2 * L + L + q] = x.im.x[q];
      }
    }
    __syncthreads();
    if (ok && (LOWER ? tx > k : tx < k)) {
      Z<L> t, xk;
      if (STAGE) {
#pragma unroll
        for (int q = 0; q < L; q++) {
          t.re.x[q] = sT[((size_t)tx * bs + k) * 2 * L + q];
          t.im.x[q] = sT[((size_t)tx * bs + k) * 2 * L + L + q];
        }
      } else {
        t = CONJT ? z_conj<L>(ldz<L>(A, k0 + k, k0 + tx)) : ldz<L>(A, k0 + tx, k0 + k);
      }
#pragma unroll
      for (int q = 0; q < L; q++) {
        xk.re.x[q] = s_x[ty * 2 * L + q];
        xk.im.x[q] = s_x[ty * 2 * L + L + q];
      }
      acc_csub<L>(are, aim, t, xk);
    }
    __syncthreads();
  }
  if (ok) stz<L>(X, xrow0 + tx, c, x);
}

// Unit lower triangular solve T x = b for the bs x bs diagonal block of A at
// (k0, k0) on column blockIdx.x of X (rows xrow0 .. xrow0+bs-1); the
// diagonal is unit, the strictly lower part is read from A.  Thread (r, p)
// holds row r's partial accumulator p of the four real products of the
// complex update x_r -= T(r,k) x_k:
//   p = 0: Re x - sum Re T Re x     p = 1: + sum Im T Im x
//   p = 2: Im x - sum Re T Im x     p = 3: - sum Im T Re x
// so each step costs every SMSP one product (the four warp groups run on
// four FP64 units), and x_k = (P0 + P1) + i (P2 + P3) is formed when row k
// is final.  Column k of T is streamed through registers and shared memory
// ahead of its step (below).  Block (bs rounded up to 32, 4), bs <= 128.
// Columns blockIdx.x >= ncol1 are columns blockIdx.x - ncol1 of a second
// right-hand side X2 (rows xrow2 ..): two solves with the same triangle in
// one launch.
template <int L>
__global__ void __launch_bounds__(512) k_lsolve4(View A, int64_t k0, int bs, View X, int64_t xrow0, View X2,
                                                 int64_t ncol1, int64_t xrow2) {
  const int r = threadIdx.x, p = threadIdx.y;
  const int RT = blockDim.x;
  const int tid = p * RT + r;
  int64_t c = blockIdx.x;
  if (c >= ncol1) {
    X = X2;
    c -= ncol1;
    xrow0 = xrow2;
  }
  extern __shared__ double lsm4[];
  double *col = lsm4;                              // [3][RT][2L]: column k of T
  double *part = col + (size_t)3 * RT * 2 * L;     // [2][4][L]: row k's partial accumulators
  double *xk = part + 2 * 4 * L;                   // [2][2L]: x_k
  const bool own = r < bs;
  Acc<L> acc;
  acc.zero();
  if (own && (p == 0 || p == 2)) {
    const Z<L> x = ldz<L>(X, xrow0 + r, c);
    acc.set(p == 0 ? x.re : x.im);
  }
  // Column k of T (rows k+1 .. bs-1, one row per thread) is loaded into
  // registers during step k-2 and stored to shared memory during step k-1,
  // so no step waits for a global load.  Columns, partial accumulators and
  // x_k rotate through buffers (3, 2, 2), which leaves two barriers a step.
  const bool frow = tid < bs;
  Z<L> pre;
  auto load_col = [&](int k) {
    if (frow && k < bs && tid > k) pre = ldz<L>(A, k0 + tid, k0 + k);
  };
  auto store_col = [&](int k) {
    if (frow && k < bs && tid > k) {
      double *d = col + ((size_t)(k % 3) * RT + tid) * 2 * L;
#pragma unroll
      for (int q = 0; q < L; q++) {
        d[q] = pre.re.x[q];
        d[L + q] = pre.im.x[q];
      }
    }
  };
  load_col(0);
  store_col(0);
  load_col(1);
  __syncthreads();
  for (int k = 0; k < bs; k++) {
    const int par = k & 1;
    store_col(k + 1);
    load_col(k + 2);
    if (r == k) {
#pragma unroll
      for (int q = 0; q < L; q++) part[(par * 4 + p) * L + q] = acc.s[q];
    }
    __syncthreads();
    if (r == 0 && (p == 0 || p == 2)) {  // x_k: Re on (0,0), Im on (0,2)
      Acc<L> t, o;
#pragma unroll
      for (int q = 0; q < L; q++) {
        t.s[q] = part[(par * 4 + p) * L + q];
        o.s[q] = part[(par * 4 + p + 1) * L + q];
      }
      t.add_acc(o, false);
      const R<L> v = t.result();
#pragma unroll
      for (int q = 0; q < L; q++) {
        xk[par * 2 * L + (p >> 1) * L + q] = v.x[q];
        X.p[(int64_t)((p >> 1) * L + q) * X.ps + c * X.ld + xrow0 + k] = v.x[q];
      }
    }
    __syncthreads();
    if (own && r > k) {
      const double *d = col + ((size_t)(k % 3) * RT + r) * 2 * L;
      const double *xv_ = xk + par * 2 * L;
      R<L> tv, xv;
#pragma unroll
      for (int q = 0; q < L; q++) {
        tv.x[q] = d[(p == 0 || p == 2) ? q : L + q];    // Re T for p = 0, 2; Im T for p = 1, 3
        xv.x[q] = xv_[(p == 0 || p == 1) ? (p == 0 ? q : L + q) : (p == 2 ? L + q : q)];
      }
      if (p == 1)
        acc.template add_prod<false>(tv, xv);
      else
        acc.template add_prod<true>(tv, xv);
    }
  }
}

template <int L>
constexpr size_t lsolve4_smem(int RT) {
  return ((size_t)3 * RT * 2 * L + 2 * 4 * L + 2 * 2 * L) * sizeof(double);
}

// Shared memory of k_tri_block for block size bs and CT columns.
template <int L>
constexpr size_t tri_block_smem(int bs, int CT, bool stage) {
  return ((stage ? (size_t)bs * bs + bs : 0) + CT) * 2 * L * sizeof(double);
}

// X = identity (n x n planes, leading dimension ld).
template <int L>
__global__ void k_identity(View X, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int64_t i = t % n, j = t / n;
  Z<L> z = z_zero<L>();
  if (i == j) z.re.x[0] = 1.0;
  stz<L>(X, i, j, z);
}

// rdiag[k] = 1 / A_kk for the diagonal of A, planes [2L][ld].
template <int L>
__global__ void k_diag_recip(View A, int64_t n, double *rdiag, int64_t ld) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const Z<L> r = z_inv<L>(ldz<L>(A, k, k));
#pragma unroll
  for (int q = 0; q < L; q++) {
    rdiag[(int64_t)q * ld + k] = r.re.x[q];
    rdiag[(int64_t)(L + q) * ld + k] = r.im.x[q];
  }
}

// ------------------------------------------------ blocked substitution (Sec. 4)
//
// The forward and back substitutions run over SOLVE_BS x SOLVE_BS diagonal
// blocks.  The inverses of all diagonal blocks are formed first, in parallel
// (k_blk_inv); each block step is then one launch (k_blk_solve) that applies
// the block's inverse to the current residual of the block and subtracts the
// block's contribution from the remaining rows.
constexpr int SOLVE_BS = 8;

// Inverses of the diagonal blocks of the factors held in A: blockIdx.y = 0
// gives inv(L_kk) of the unit lower triangle, blockIdx.y = 1 inv(U_kk) of the
// upper triangle, whose diagonal reciprocals are rdiag (planes [2L][rld]).
// Thread c forms column c of the inverse by substitution, each entry one
// leveled accumulation: lower, x_i = -sum_{c <= j < i} L_ij x_j with x_c = 1;
// upper, x_i = -(sum_{i < j <= c} U_ij x_j) / U_ii with x_c = 1 / U_cc.
// Output W[block][2L][SOLVE_BS][SOLVE_BS], row-major (i, j), zero outside the
// block's bs x bs extent and outside the triangle.
template <int L>
__global__ void __launch_bounds__(SOLVE_BS) k_blk_inv(View A, int64_t n, double *WL, double *WU, const double *rdiag,
                                                      int64_t rld) {
  constexpr int BS = SOLVE_BS;
  __shared__ double sT[BS][BS][2 * L];  // T(i, j) of the diagonal block
  __shared__ double sX[BS][BS][2 * L];  // sX[i][c]: entry (i, c) of the inverse
  const int c = threadIdx.x;
  const int64_t blk = blockIdx.x, k0 = blk * BS;
  const int bs = (int)min((int64_t)BS, n - k0);
  const bool upper = blockIdx.y == 1;
  for (int t = c; t < BS * BS; t += BS) {
    const int i = t % BS, j = t / BS;
    Z<L> v = z_zero<L>();
    if (i < bs && j < bs && (upper ? i <= j : i > j)) v = ldz<L>(A, k0 + i, k0 + j);
    sts_z<L>(sT[i][j], v);
    sts_z<L>(sX[i][j], z_zero<L>());
  }
  __syncthreads();
  if (c < bs) {
    if (!upper) {
      Z<L> one = z_zero<L>();
      one.re.x[0] = 1.0;
      sts_z<L>(sX[c][c], one);
      for (int i = c + 1; i < bs; i++) {
        Acc<L> re, im;
        re.zero();
        im.zero();
        for (int j = c; j < i; j++) acc_csub<L>(re, im, lds_z<L>(sT[i][j]), lds_z<L>(sX[j][c]));
        Z<L> x;
        x.re = re.result();
        x.im = im.result();
        sts_z<L>(sX[i][c], x);
      }
    } else {
      auto recip = [&](int i) {
        Z<L> r;
#pragma unroll
        for (int q = 0; q < L; q++) {
          r.re.x[q] = rdiag[(int64_t)q * rld + k0 + i];
          r.im.x[q] = rdiag[(int64_t)(L + q) * rld + k0 + i];
        }
        return r;
      };
      sts_z<L>(sX[c][c], recip(c));
      for (int i = c - 1; i >= 0; i--) {
        Acc<L> re, im;
        re.zero();
        im.zero();
        for (int j = i + 1; j <= c; j++) acc_csub<L>(re, im, lds_z<L>(sT[i][j]), lds_z<L>(sX[j][c]));
        Z<L> x;
        x.re = re.result();
        x.im = im.result();
        sts_z<L>(sX[i][c], z_mul<L>(x, recip(i)));
      }
    }
  }
  __syncthreads();
  double *W = (upper ? WU : WL) + blk * 2 * L * BS * BS;
  for (int i = 0; i < BS; i++)
#pragma unroll
    for (int q = 0; q < 2 * L; q++) W[((size_t)q * BS + i) * BS + c] = sX[i][c][q];
}

// Shared memory of k_blk_solve: A tile [SOLVE_BS][32][2L], op(W) [SOLVE_BS][SOLVE_BS][2L],
// r_k and x_k [SOLVE_BS][2L] each.
template <int L>
constexpr size_t blk_solve_smem() {
  return ((size_t)SOLVE_BS * 32 + SOLVE_BS * SOLVE_BS + 2 * SOLVE_BS) * 2 * L * sizeof(double);
}

// One step of the blocked substitution for the diagonal block at k0 (bs <=
// SOLVE_BS rows) on column blockIdx.y of the residual R:
//   1. x_k = op(Wk) r_k, Wk the block's inverse (op: identity, or the
//      conjugate transpose with CONJT).  Four lanes share a row of Wk, only
//      the triangle is visited, and the partial accumulators are combined
//      through warp shuffles.  Every CTA forms x_k (a 16 x 16 product); the
//      CTAs with blockIdx.x = 0 store it in Y.
//   2. R[r] -= sum_j op(T)(r, k0+j) x_j for the rows r in [r0, r1), where
//      op(T)(r, j) = A(r, j), or conj(A(j, r)) with CONJT.  Eight lanes share a
//      row, 32 rows per CTA; the A tile is staged in shared memory (read along
//      its columns with CONJT, contiguous in memory).
// No CTA writes rows of block k of R, so every CTA reads the same r_k.
template <int L, bool LOWER, bool CONJT>
__global__ void __launch_bounds__(256) k_blk_solve(View A, int64_t k0, int bs, const double *Wk, View R, View Y,
                                                   int64_t r0, int64_t r1) {
  constexpr int BS = SOLVE_BS, TR = 32, G = 8, G1 = 4;
  extern __shared__ double bsm[];
  double(*sA)[TR][2 * L] = reinterpret_cast<double(*)[TR][2 * L]>(bsm);
  double(*sW)[BS][2 * L] = reinterpret_cast<double(*)[BS][2 * L]>(bsm + (size_t)BS * TR * 2 * L);
  double(*sR)[2 * L] = reinterpret_cast<double(*)[2 * L]>(bsm + ((size_t)BS * TR + BS * BS) * 2 * L);
  double(*sX)[2 * L] = sR + BS;
  const int tid = threadIdx.x;
  const int64_t c = blockIdx.y;
  const int64_t rbase = r0 + (int64_t)blockIdx.x * TR;
  // stage op(Wk), r_k and the A tile
  for (int t = tid; t < BS * BS * 2 * L; t += 256) {
    const int q = t / (BS * BS), ij = t % (BS * BS);
    const int i = ij / BS, j = ij % BS;
    double v;
    if (CONJT) {
      v = Wk[((size_t)q * BS + j) * BS + i];
      if (q >= L) v = -v;
    } else {
      v = Wk[((size_t)q * BS + i) * BS + j];
    }
    sW[i][j][q] = v;
  }
  for (int t = tid; t < BS; t += 256) sts_z<L>(sR[t], t < bs ? ldz<L>(R, k0 + t, c) : z_zero<L>());
  if (r1 > r0) {
    for (int t = tid; t < bs * TR; t += 256) {
      int kq, rq;
      if (CONJT) {
        kq = t % bs;
        rq = t / bs;
      } else {
        rq = t % TR;
        kq = t / TR;
      }
      const int64_t gr = rbase + rq, gk = k0 + kq;
      Z<L> v = z_zero<L>();
      if (gr < r1) v = CONJT ? z_conj<L>(ldz<L>(A, gk, gr)) : ldz<L>(A, gr, gk);
      sts_z<L>(sA[kq][rq], v);
    }
  }
  __syncthreads();
  // 1. x_k = op(Wk) r_k on the first BS * G1 threads (whole warps)
  if (tid < BS * G1) {
    const int i = tid / G1, g = tid % G1;
    Acc<L> re, im;
    re.zero();
    im.zero();
    const int jlo = LOWER ? 0 : i, jhi = LOWER ? i : bs - 1;
    for (int j = jlo + g; j <= jhi && j < bs; j += G1) acc_cadd<L>(re, im, lds_z<L>(sW[i][j]), lds_z<L>(sR[j]));
#pragma unroll
    for (int off = G1 / 2; off > 0; off >>= 1) {
      Acc<L> ore, oim;
#pragma unroll
      for (int q = 0; q < L; q++) {
        ore.s[q] = __shfl_down_sync(0xffffffffu, re.s[q], off, G1);
        oim.s[q] = __shfl_down_sync(0xffffffffu, im.s[q], off, G1);
      }
      re.add_acc(ore, false);
      im.add_acc(oim, false);
    }
    if (g == 0) {
      Z<L> x;
      x.re = re.result();
      x.im = im.result();
      sts_z<L>(sX[i], x);
      if (blockIdx.x == 0 && i < bs) stz<L>(Y, k0 + i, c, x);
    }
  }
  __syncthreads();
  if (r1 <= r0) return;
  // 2. the remaining rows lose the block's contribution
  const int g = tid & (G - 1), rloc = tid >> 3;
  const int64_t r = rbase + rloc;
  Acc<L> are, aim;
  are.zero();
  aim.zero();
  for (int kq = g; kq < bs; kq += G) acc_csub<L>(are, aim, lds_z<L>(sA[kq][rloc]), lds_z<L>(sX[kq]));
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    Acc<L> ore, oim;
#pragma unroll
    for (int q = 0; q < L; q++) {
      ore.s[q] = __shfl_down_sync(0xffffffffu, are.s[q], off, G);
      oim.s[q] = __shfl_down_sync(0xffffffffu, aim.s[q], off, G);
    }
    are.add_acc(ore, false);
    aim.add_acc(oim, false);
  }
  if (g == 0 && r < r1) {
    const Z<L> x0 = ldz<L>(R, r, c);
    are.add(x0.re);
    aim.add(x0.im);
    Z<L> z;
    z.re = are.result();
    z.im = aim.result();
    stz<L>(R, r, c, z);
  }
}

// ------------------------------------- persistent dataflow substitution
//
// The whole forward (LOWER) or backward substitution of one right-hand side
// in one cooperative launch.  Step q (q = 0 .. nblk-1) makes x of diagonal
// block b(q) = q (LOWER) or nblk-1-q.  CTA g owns the steps q = g (mod G):
// the residual of its blocks lives in its shared memory for the whole solve,
// and so does M_q = op(W_{b(q)}) op(T)(b(q), b(q-1)) of each owned step,
// formed at the start.  Iteration q of every CTA:
//   1. the owner of step q+1 forms y = op(W_{b(q+1)}) r_{b(q+1)} (all its
//      earlier terms are in) before it needs x_q;
//   2. get x_q: the owner has it; the others poll its words in Y until none
//      holds FLOW_SENT any more (every word validates itself: no flag, no
//      fence, one round trip);
//   3. the owner of step q+1 forms x_{q+1} = y - M_{q+1} x_q and stores it --
//      before any other work, since every CTA waits for it;
//   4. all other owned blocks of later steps subtract op(T)(block, b(q)) x_q.
// Y must hold FLOW_SENT in every word of the solution before the launch.  A
// wait that runs out (the co-resident cooperative launch rules this out)
// sets *status and writes NaN to every x the CTA still owed, so the failure
// shows in the result.
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Every 64-bit word of count words at p set to v.
static __global__ void k_fill_u64(unsigned long long *p, int64_t count, unsigned long long v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

constexpr int FLOW_T = 128;
constexpr long long FLOW_WAIT = 2000000000LL;  // bound on one wait, ~1 s at 2 GHz
// The value of a solution word not yet written: a signalling-NaN bit pattern,
// which no arithmetic result has (a NaN result is a quiet NaN).
constexpr unsigned long long FLOW_SENT = 0x7ff0dead5eed0000ULL;

// One warp: lane = 4 i + g handles row i (< SOLVE_BS) and the products j = g, g+4.
template <int L, bool CONJT>
struct TileRegs {
  Z<L> t[2];
  __device__ __forceinline__ void load(View A, int64_t r0, int64_t c0, int br, int bc, int lane) {
    const int i = lane >> 2, g = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = g + 4 * h;
      t[h] = z_zero<L>();
      if (i < br && j < bc) t[h] = CONJT ? z_conj<L>(ldz<L>(A, c0 + j, r0 + i)) : ldz<L>(A, r0 + i, c0 + j);
    }
  }
};

// res[i] -= sum_j T(i, j) x_j over one warp (combine of the 4 lanes of a row).
template <int L>
__device__ __forceinline__ void warp_tile_apply(const Z<L> (&t)[2], const double (*xs)[2 * L], double (*res)[2 * L],
                                                int br, int bc, int lane) {
  const int i = lane >> 2, g = lane & 3;
  Acc<L> re, im;
  re.zero();
  im.zero();
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int j = g + 4 * h;
    if (i < br && j < bc) acc_csub<L>(re, im, t[h], lds_z<L>(xs[j]));
  }
#pragma unroll
  for (int off = 2; off > 0; off >>= 1) {
    Acc<L> ore, oim;
#pragma unroll
    for (int q = 0; q < L; q++) {
      ore.s[q] = __shfl_down_sync(0xffffffffu, re.s[q], off, 4);
      oim.s[q] = __shfl_down_sync(0xffffffffu, im.s[q], off, 4);
    }
    re.add_acc(ore, false);
    im.add_acc(oim, false);
  }
  if (g == 0 && i < br) {
    const Z<L> r0 = lds_z<L>(res[i]);
    re.add(r0.re);
    im.add(r0.im);
    Z<L> z;
    z.re = re.result();
    z.im = im.result();
    sts_z<L>(res[i], z);
  }
}

// op(W) of one diagonal block, in the same lane layout (only the triangle).
template <int L, bool LOWER, bool CONJT>
struct InvRegs {
  Z<L> w[2];
  __device__ __forceinline__ void load(const double *Wb, int bs, int lane) {
    constexpr int BS = SOLVE_BS;
    const int i = lane >> 2, g = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = g + 4 * h;
      w[h] = z_zero<L>();
      if (i < bs && j < bs && (LOWER ? j <= i : j >= i)) {
#pragma unroll
        for (int q = 0; q < L; q++) {
          if (CONJT) {
            w[h].re.x[q] = Wb[((size_t)q * BS + j) * BS + i];
            w[h].im.x[q] = -Wb[((size_t)(L + q) * BS + j) * BS + i];
          } else {
            w[h].re.x[q] = Wb[((size_t)q * BS + i) * BS + j];
            w[h].im.x[q] = Wb[((size_t)(L + q) * BS + i) * BS + j];
          }
        }
      }
    }
  }
};

// x = op(W) r over one warp; returns this lane's row result in lanes g == 0.
template <int L>
__device__ __forceinline__ void warp_inv_apply(const Z<L> (&w)[2], const double (*r)[2 * L], double (*x)[2 * L],
                                               int bs, int lane) {
  const int i = lane >> 2, g = lane & 3;
  Acc<L> re, im;
  re.zero();
  im.zero();
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int j = g + 4 * h;
    if (i < bs && j < bs) acc_cadd<L>(re, im, w[h], lds_z<L>(r[j]));
  }
#pragma unroll
  for (int off = 2; off > 0; off >>= 1) {
    Acc<L> ore, oim;
#pragma unroll
    for (int q = 0; q < L; q++) {
      ore.s[q] = __shfl_down_sync(0xffffffffu, re.s[q], off, 4);
      oim.s[q] = __shfl_down_sync(0xffffffffu, im.s[q], off, 4);
    }
    re.add_acc(ore, false);
    im.add_acc(oim, false);
  }
  if (g == 0 && i < bs) {
    Z<L> z;
    z.re = re.result();
    z.im = im.result();
    sts_z<L>(x[i], z);
  }
}

// Critical step of the dataflow substitution, split by product over the four
// warps of the CTA (one SMSP and FP64 unit each): warp p forms product p of
// every complex MAC of the step for the rows i = lane / 4 (lanes g = lane % 4
// take j = g, g + 4), combines its four lanes and leaves the partial
// accumulator in part[p][i][L].
//   tile update r -= T x:  p0 -Re T Re x, p1 +Im T Im x, p2 -Re T Im x, p3 -Im T Re x
//   inverse    x = W r:    p0 +Re W Re r, p1 -Im W Im r, p2 +Re W Im r, p3 +Im W Re r
template <int L, bool INV>
__device__ __forceinline__ void warp_part(const Z<L> (&m)[2], const double (*v)[2 * L], double *part, int p, int br,
                                          int bc, bool tri_lower, bool tri, int lane) {
  const int i = lane >> 2, g = lane & 3;
  Acc<L> acc;
  acc.zero();
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int j = g + 4 * h;
    if (i < br && j < bc && (!tri || (tri_lower ? j <= i : j >= i))) {
      const Z<L> vj = lds_z<L>(v[j]);
      const R<L> &a = (p == 0 || p == 2) ? m[h].re : m[h].im;
      const R<L> &b = (p == 0 || p == 3) ? vj.re : vj.im;
      if (INV ? (p == 1) : (p != 1))
        acc.template add_prod<true>(a, b);
      else
        acc.template add_prod<false>(a, b);
    }
  }
#pragma unroll
  for (int off = 2; off > 0; off >>= 1) {
    Acc<L> o;
#pragma unroll
    for (int q = 0; q < L; q++) o.s[q] = __shfl_down_sync(0xffffffffu, acc.s[q], off, 4);
    acc.add_acc(o, false);
  }
  if (g == 0 && i < br) {
#pragma unroll
    for (int q = 0; q < L; q++) part[(p * SOLVE_BS + i) * L + q] = acc.s[q];
  }
}

// Warps 0 (real part) and 1 (imaginary part): out[i] = base[i] + P_{2w} +
// P_{2w+1} for the rows i < br (base omitted when null).
template <int L>
__device__ __forceinline__ void combine_parts(const double *part, const double (*base)[2 * L], double (*out)[2 * L],
                                              int br, int warp, int lane) {
  if (warp < 2 && lane < br) {
    Acc<L> t, o;
#pragma unroll
    for (int q = 0; q < L; q++) {
      t.s[q] = part[((2 * warp) * SOLVE_BS + lane) * L + q];
      o.s[q] = part[((2 * warp + 1) * SOLVE_BS + lane) * L + q];
    }
    t.add_acc(o, false);
    if (base) {
      R<L> b;
#pragma unroll
      for (int q = 0; q < L; q++) b.x[q] = base[lane][warp * L + q];
      t.add(b);
    }
    const R<L> r = t.result();
#pragma unroll
    for (int q = 0; q < L; q++) out[lane][warp * L + q] = r.x[q];
  }
}

// Shared memory of k_trsv_flow for nown owned blocks: residuals, x of two
// steps, the M blocks.
template <int L>
constexpr size_t trsv_flow_smem(int nown) {
  return (((size_t)nown + 2) * SOLVE_BS + (size_t)nown * SOLVE_BS * SOLVE_BS) * 2 * L * sizeof(double);
}

template <int L, bool LOWER, bool CONJT>
__global__ void __launch_bounds__(FLOW_T) k_trsv_flow(View A, int64_t n, const double *Winv, View R, View Y,
                                                      int *status) {
  constexpr int BS = SOLVE_BS;
  extern __shared__ double fsm[];
  const int G = (int)gridDim.x, g = (int)blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nblk = (int)((n + BS - 1) / BS);
  const int nown = (nblk - g + G - 1) / G;  // owned steps q = g + i G, i < nown
  double(*res)[BS][2 * L] = reinterpret_cast<double(*)[BS][2 * L]>(fsm);
  double(*xs)[BS][2 * L] = res + nown;  // [2][BS][2L], by step parity
  double(*Ms)[BS][BS][2 * L] = reinterpret_cast<double(*)[BS][BS][2 * L]>(xs + 2);  // [nown]
  __shared__ int s_ok;
  __shared__ double s_part[4 * SOLVE_BS * L];
  auto blk = [&](int q) -> int64_t { return LOWER ? q : nblk - 1 - q; };
  auto rows = [&](int q) -> int { return (int)min((int64_t)BS, n - blk(q) * BS); };
  auto wblk = [&](int q) -> const double * { return Winv + blk(q) * 2 * L * BS * BS; };
  auto yword = [&](int q, int t) -> unsigned long long * {  // word t = plane * rows + row of x_q in Y
    const int rq = rows(q);
    return reinterpret_cast<unsigned long long *>(Y.p + (int64_t)(t / rq) * Y.ps + blk(q) * BS + t % rq);
  };
  auto publish = [&](int q, const double (*x)[2 * L]) {  // warp 0: the words of x_q to Y
    const int rq = rows(q);
    for (int t = lane; t < rq * 2 * L; t += 32)
      st_relaxed_u64(yword(q, t), (unsigned long long)__double_as_longlong(x[t % rq][t / rq]));
  };
  auto fail_rest = [&](int qfrom) {  // NaN into every x this CTA still owed
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int i = 0; i < nown; i++) {
      const int q = g + i * G;
      if (q < qfrom) continue;
      for (int t = tid; t < rows(q) * 2 * L; t += FLOW_T)
        Y.p[(int64_t)(t / rows(q)) * Y.ps + blk(q) * BS + t % rows(q)] = nan;
    }
  };
  for (int t = tid; t < nown * BS; t += FLOW_T) {
    const int i = t / BS, r = t % BS, q = g + i * G;
    const int64_t row = blk(q) * BS + r;
    sts_z<L>(res[i][r], r < rows(q) ? ldz<L>(R, row, 0) : z_zero<L>());
  }
  // M_q = op(W_q) op(T)(b(q), b(q-1)) of every owned step q >= 1: thread t
  // forms part t & 1 (re, im) of entry (e >> 3, e & 7), e = t >> 1
  for (int i = 0; i < nown; i++) {
    const int q = g + i * G;
    if (q == 0) continue;
    const int br = rows(q), bc = rows(q - 1);
    const int e = tid >> 1, part = tid & 1, ei = e >> 3, ej = e & 7;
    const double *Wb = wblk(q);
    const int64_t r0 = blk(q) * BS, c0 = blk(q - 1) * BS;
    Acc<L> acc;
    acc.zero();
    if (ei < br && ej < bc) {
      for (int k = 0; k < br; k++) {
        if (LOWER ? k > ei : k < ei) continue;  // op(W) is triangular
        Z<L> w;
#pragma unroll
        for (int l = 0; l < L; l++) {
          if (CONJT) {
            w.re.x[l] = Wb[((size_t)l * BS + k) * BS + ei];
            w.im.x[l] = flip(Wb[((size_t)(L + l) * BS + k) * BS + ei]);
          } else {
            w.re.x[l] = Wb[((size_t)l * BS + ei) * BS + k];
            w.im.x[l] = Wb[((size_t)(L + l) * BS + ei) * BS + k];
          }
        }
        const Z<L> t = CONJT ? z_conj<L>(ldz<L>(A, c0 + ej, r0 + k)) : ldz<L>(A, r0 + k, c0 + ej);
        if (part == 0) {
          acc.template add_prod<false>(w.re, t.re);
          acc.template add_prod<true>(w.im, t.im);
        } else {
          acc.template add_prod<false>(w.re, t.im);
          acc.template add_prod<false>(w.im, t.re);
        }
      }
    }
    const auto v = acc.result();
#pragma unroll
    for (int l = 0; l < L; l++) Ms[i][ei][ej][part * L + l] = v.x[l];
  }
  __syncthreads();
  if (g == 0 && warp == 0) {  // step 0 needs no update
    InvRegs<L, LOWER, CONJT> w;
    w.load(wblk(0), rows(0), lane);
    warp_inv_apply<L>(w.w, res[0], xs[0], rows(0), lane);
    __syncwarp();
    publish(0, xs[0]);
  }
  __syncthreads();
  for (int q = 0; q < nblk; q++) {
    const int par = q & 1;
    const int qn = q + 1;
    const bool crit = qn < nblk && qn % G == g;
    const int ic = crit ? (qn - g) / G : 0;
    // 1. y = op(W) r of the next step's block, in place
    if (crit) {
      InvRegs<L, LOWER, CONJT> w;
      w.load(wblk(qn), rows(qn), lane);
      warp_part<L, true>(w.w, res[ic], s_part, warp, rows(qn), rows(qn), LOWER, true, lane);
      __syncthreads();
      combine_parts<L>(s_part, nullptr, res[ic], rows(qn), warp, lane);
      __syncthreads();
    }
    // 2. x_q
    if (q % G != g) {
      if (warp == 0) {
        const int nw = rows(q) * 2 * L;  // <= 64 words
        unsigned long long v0 = FLOW_SENT, v1 = FLOW_SENT;
        bool ok = true;
        const long long t0 = clock64();
        for (;;) {
          if (lane < nw && v0 == FLOW_SENT) v0 = ld_relaxed_u64(yword(q, lane));
          if (lane + 32 < nw && v1 == FLOW_SENT) v1 = ld_relaxed_u64(yword(q, lane + 32));
          const bool need = (lane < nw && v0 == FLOW_SENT) || (lane + 32 < nw && v1 == FLOW_SENT);
          if (!__any_sync(0xffffffffu, need)) break;
          if (__any_sync(0xffffffffu, clock64() - t0 > FLOW_WAIT)) {
            ok = false;
            break;
          }
        }
        const int rq = rows(q);
        if (lane < nw) xs[par][lane % rq][lane / rq] = __longlong_as_double((long long)v0);
        if (lane + 32 < nw) xs[par][(lane + 32) % rq][(lane + 32) / rq] = __longlong_as_double((long long)v1);
        if (lane == 0) {
          s_ok = ok ? 1 : 0;
          if (!ok) atomicOr(status, 1);
        }
      }
      __syncthreads();
      if (!s_ok) {
        fail_rest(q);
        return;
      }
    }
    // 3. x_{q+1} = y - M x_q, its products split over the four warps
    if (crit) {
      Z<L> mt[2];
      {
        const int i = lane >> 2, gq = lane & 3;
#pragma unroll
        for (int h = 0; h < 2; h++) mt[h] = lds_z<L>(Ms[ic][i][gq + 4 * h]);
      }
      warp_part<L, false>(mt, xs[par], s_part, warp, rows(qn), rows(q), false, false, lane);
      __syncthreads();
      combine_parts<L>(s_part, res[ic], xs[par ^ 1], rows(qn), warp, lane);
      __syncthreads();
      if (warp == 0) publish(qn, xs[par ^ 1]);
    }
    // 4. the other owned blocks of later steps
    {
      int k = 0;
      for (int i = 0; i < nown; i++) {
        const int q2 = g + i * G;
        if (q2 <= q || (crit && q2 == qn)) continue;
        const int wk = k % (FLOW_T / 32);
        k++;
        if (warp != wk) continue;
        TileRegs<L, CONJT> t;
        t.load(A, blk(q2) * BS, blk(q) * BS, rows(q2), rows(q), lane);
        warp_tile_apply<L>(t.t, xs[par], res[i], rows(q2), rows(q), lane);
      }
    }
    __syncthreads();
  }
}

// Plain complex multi-component GEMM on the FP64 pipe: C (m x n) = C - A B
// (BETA) or A B.  4M (Eq. 1): Re and Im accumulated directly.  3M (Eq. 3):
// T1 = ReA ReB, T2 = ImA ImB, T3 = (ReA+ImA)(ReB+ImB) accumulated separately,
// then Re = T1 - T2, Im = T3 - (T1 + T2); SA, SB hold the precomputed sums.
// One thread per output, k ascending (deterministic), 16 x 16 tile, k staged
// through shared memory 16 at a time.
template <int L, bool M3, bool BETA>
__global__ void __launch_bounds__(GEMM_T *GEMM_T)
    k_gemm(View A, View B, View C, View SA, View SB, int64_t m, int64_t n, int64_t k) {
  constexpr int T = GEMM_T;
  constexpr int NP = M3 ? 3 * L : 2 * L;  // planes staged per operand
  __shared__ double sA[T][T][NP];         // [k][row][plane]
  __shared__ double sB[T][T][NP];         // [k][col][plane]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * T + tx;
  const int64_t i0 = (int64_t)blockIdx.x * T, j0 = (int64_t)blockIdx.y * T;
  const int64_t i = i0 + tx, j = j0 + ty;
  const bool ok = i < m && j < n;
  Acc<L> a1, a2, a3;
  a1.zero();
  a2.zero();
  a3.zero();
  for (int64_t kk = 0; kk < k; kk += T) {
    {  // A tile: thread (tx, ty) loads A[i0+tx, kk+ty]
      const int64_t gi = i0 + tx, gk = kk + ty;
      const bool in = gi < m && gk < k;
#pragma unroll
      for (int pl = 0; pl < 2 * L; pl++) sA[ty][tx][pl] = in ? A.p[(int64_t)pl * A.ps + gk * A.ld + gi] : 0.0;
      if constexpr (M3) {
#pragma unroll
        for (int q = 0; q < L; q++) sA[ty][tx][2 * L + q] = in ? SA.p[(int64_t)q * SA.ps + gk * SA.ld + gi] : 0.0;
      }
    }
    {  // B tile: thread (tx, ty) loads B[kk+tx, j0+ty]
      const int64_t gk = kk + tx, gj = j0 + ty;
      const bool in = gk < k && gj < n;
#pragma unroll
      for (int pl = 0; pl < 2 * L; pl++) sB[tx][ty][pl] = in ? B.p[(int64_t)pl * B.ps + gj * B.ld + gk] : 0.0;
      if constexpr (M3) {
#pragma unroll
        for (int q = 0; q < L; q++) sB[tx][ty][2 * L + q] = in ? SB.p[(int64_t)q * SB.ps + gj * SB.ld + gk] : 0.0;
      }
    }
    __syncthreads();
    const int kmax = (int)min((int64_t)T, k - kk);
    for (int kq = 0; kq < kmax; kq++) {
      R<L> ar, ai, br, bi;
#pragma unroll
      for (int q = 0; q < L; q++) {
        ar.x[q] = sA[kq][tx][q];
        ai.x[q] = sA[kq][tx][L + q];
        br.x[q] = sB[kq][ty][q];
        bi.x[q] = sB[kq][ty][L + q];
      }
      if constexpr (!M3) {
        // a1 = Re, a2 = Im; BETA subtracts the product
        a1.template add_prod<BETA>(ar, br);
        a1.template add_prod<!BETA>(ai, bi);
        a2.template add_prod<BETA>(ar, bi);
        a2.template add_prod<BETA>(ai, br);
      } else {
        R<L> sa, sb;
#pragma unroll
        for (int q = 0; q < L; q++) {
          sa.x[q] = sA[kq][tx][2 * L + q];
          sb.x[q] = sB[kq][ty][2 * L + q];
        }
        a1.template add_prod<false>(ar, br);
        a2.template add_prod<false>(ai, bi);
        a3.template add_prod<false>(sa, sb);
      }
    }
    __syncthreads();
  }
  (void)tid;
  if (!ok) return;
  Z<L> out;
  if constexpr (!M3) {
    if (BETA) {
      Z<L> c0 = ldz<L>(C, i, j);
      a1.add(c0.re);
      a2.add(c0.im);
    }
    out.re = a1.result();
    out.im = a2.result();
  } else {
    // Re = [C] - T1 + T2 (BETA) or T1 - T2;  Im = [C] - T3 + T1 + T2 or T3 - (T1 + T2)
    Acc<L> re, im;
    if (BETA) {
      Z<L> c0 = ldz<L>(C, i, j);
      re.set(c0.re);
      im.set(c0.im);
    } else {
      re.zero();
      im.zero();
    }
    re.add_acc(a1, BETA);
    re.add_acc(a2, !BETA);
    im.add_acc(a3, BETA);
    im.add_acc(a1, !BETA);
    im.add_acc(a2, !BETA);
    out.re = re.result();
    out.im = im.result();
  }
  stz<L>(C, i, j, out);
}

// S = Re + Im for an m x k block (3M pre-sums of Eq. 3), L planes out.
template <int L>
__global__ void k_resum(View X, View S, int64_t m, int64_t k) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * k) return;
  const int64_t i = t % m, j = t / m;
  Z<L> z = ldz<L>(X, i, j);
  R<L> s = r_add<L>(z.re, z.im);
#pragma unroll
  for (int q = 0; q < L; q++) S.p[(int64_t)q * S.ps + j * S.ld + i] = s.x[q];
}

// Net permutation of a pivot sequence: perm[i] = source row of row i of P b.
// One thread in shared memory (n <= max_smem/4), else in global memory.
static __global__ void k_perm_build(const int32_t *ipiv, int64_t n, int32_t *perm, int use_smem) {
  extern __shared__ int32_t s_perm[];
  if (threadIdx.x != 0) return;
  int32_t *P = use_smem ? s_perm : perm;
  for (int64_t i = 0; i < n; i++) P[i] = (int32_t)i;
  for (int64_t k = 0; k < n; k++) {
    int64_t p = ipiv[k] - 1;
    int32_t a = P[k];
    P[k] = P[p];
    P[p] = a;
  }
  if (use_smem)
    for (int64_t i = 0; i < n; i++) perm[i] = P[i];
}

// Y[i] = X[perm[i]] (gather) or Y[perm[i]] = X[i] (scatter), all 2L planes.
template <int L>
__global__ void k_permute(View X, View Y, const int32_t *perm, int64_t n, int64_t ncols, int scatter) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ncols) return;
  const int64_t i = t % n, c = t / n;
  const int64_t s = perm[i];
#pragma unroll
  for (int pl = 0; pl < 2 * L; pl++) {
    if (scatter)
      Y.p[(int64_t)pl * Y.ps + c * Y.ld + s] = X.p[(int64_t)pl * X.ps + c * X.ld + i];
    else
      Y.p[(int64_t)pl * Y.ps + c * Y.ld + i] = X.p[(int64_t)pl * X.ps + c * X.ld + s];
  }
}

// Abar[i, j] = -lambda_i conj(x_j)
template <int L>
__global__ void k_rank1_adjoint(View lam, View x, View Ab, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n) return;
  Z<L> l = ldz<L>(lam, i, 0);
  Z<L> xj = z_conj<L>(ldz<L>(x, j, 0));
  stz<L>(Ab, i, j, z_neg<L>(z_mul<L>(l, xj)));
}

// Strassen-Winograd blocks (Sec. 2.3): Z = X + sgn Y for m x n complex
// blocks, each part an accurate L-limb addition (rounded to L limbs).
template <int L>
__global__ void k_madd(View X, View Y, View O, int64_t m, int64_t n, bool sub) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  const Z<L> x = ldz<L>(X, i, j), y = ldz<L>(Y, i, j);
  stz<L>(O, i, j, sub ? z_sub<L>(x, y) : z_add<L>(x, y));
}

// C = C - sum_q s_q P_q over up to four m x n product blocks (s_q = +1 or
// -1, bit q of neg set for -1), summed on the leveled accumulator with one
// rounding to L limbs: the combination steps of Winograd's variant.
template <int L>
__global__ void k_mcombine(View C, View P0, View P1, View P2, View P3, int np, unsigned neg, int64_t m, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  const Z<L> c = ldz<L>(C, i, j);
  Acc<L> re, im;
  re.set(c.re);
  im.set(c.im);
  const View P[4] = {P0, P1, P2, P3};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (q >= np) break;
    const Z<L> v = ldz<L>(P[q], i, j);
    const bool sgn = ((neg >> q) & 1u) == 0;  // subtract s_q P_q: negate when s_q = +1
    Acc<L> a, b;
    a.set(v.re);
    b.set(v.im);
    re.add_acc(a, sgn);
    im.add_acc(b, sgn);
  }
  Z<L> z;
  z.re = re.result();
  z.im = im.result();
  stz<L>(C, i, j, z);
}

// Z = -Z for an m x n complex block (exact: sign bits only).
template <int L>
__global__ void k_mneg(View O, int64_t m, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  stz<L>(O, i, j, z_neg<L>(ldz<L>(O, i, j)));
}

// Real L-limb matrices (L column-major planes, plane l at R + l ld_r cols)
// and the complex planes the factorisation runs on: to_complex copies the
// real planes into the real part of Z and zeroes its imaginary part; the
// reverse copies the real part of Z back.  One thread per element and plane.
template <int L>
__global__ void k_real_planes(double *R, int64_t ld_r, View Zc, int64_t rows, int64_t cols, bool to_complex) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int64_t i = t % rows, j = t / rows;
#pragma unroll
  for (int l = 0; l < L; l++) {
    double *r = R + (int64_t)l * ld_r * cols + j * ld_r + i;
    double *zr = Zc.p + (int64_t)l * Zc.ps + j * Zc.ld + i;
    if (to_complex) {
      *zr = *r;
      Zc.p[(int64_t)(L + l) * Zc.ps + j * Zc.ld + i] = 0.0;
    } else {
      *r = *zr;
    }
  }
}

// Reports a nonzero tensor-core pipeline status through info (< 0).
static __global__ void k_merge_status(const int *status, int *info) {
  if (*status) *info = -1000 - *status;
}

// Elementwise operations (mclu_vec_op).
template <int L>
__global__ void k_vec_op(int op, int64_t count, const double *x, const double *y, double *z) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  if (op < 10) {
    R<L> a, b;
#pragma unroll
    for (int q = 0; q < L; q++) {
      a.x[q] = x[q * count + e];
      b.x[q] = y[q * count + e];
    }
    R<L> r;
    switch (op) {
      case 0: r = r_add<L>(a, b); break;
      case 1: r = r_sub<L>(a, b); break;
      case 2: r = r_mul<L>(a, b); break;
      default: r = r_div<L>(a, b); break;
    }
#pragma unroll
    for (int q = 0; q < L; q++) z[q * count + e] = r.x[q];
    return;
  }
  View vx{const_cast<double *>(x), count, count};
  View vy{const_cast<double *>(y), count, count};
  View vz{z, count, count};
  Z<L> a = ldz<L>(vx, e, 0), b, r;
  if (op < 15) b = ldz<L>(vy, e, 0);
  switch (op) {
    case 10: r = z_add<L>(a, b); break;
    case 11: r = z_sub<L>(a, b); break;
    case 12: r = z_mul<L>(a, b); break;
    case 13: r = z_mul3m<L>(a, b); break;
    case 14: r = z_div<L>(a, b); break;
    case 15: r = z_inv<L>(a); break;
    case 17: r = z_inv_newton<L>(a); break;
    default:
      r.re = z_abs1<L>(a);
      r.im = r_zero<L>();
      break;
  }
  stz<L>(vz, e, 0, r);
}

}  // namespace mclu
