// lu_host.cuh - host-side orchestration of the complex multi-component LU,
// solve, ZGEMM and adjoint, templated on the limb count L.  Everything is
// enqueued on the caller's stream with no host synchronisation; workspace is
// allocated stream-ordered and freed at the end of each call.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "../../include/mclu.h"
#include "lu_kernels.cuh"
#include "ozaki.cuh"
#include "panel_coop.cuh"
#include "panel_team.cuh"

namespace mclu {

#define MCLU_TRY(expr)                         \
  do {                                         \
    cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) return (int)e_;     \
  } while (0)
// Every kernel launch is followed by MCLU_LAUNCHED(): it counts the launch
// (mclu_launch_count) and reports a failed launch as the CUDA error code.
void note_launch();
#define MCLU_LAUNCHED()            \
  do {                             \
    note_launch();                 \
    MCLU_TRY(cudaGetLastError());  \
  } while (0)

constexpr int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Raises a kernel's dynamic shared-memory limit to `bytes` once per device:
// the limit is a property of the function on one device, so bit d of `done`
// records device d (devices 64 and up set it on every call).  Concurrent
// first calls from several host threads may both set it (harmless).
template <class K>
inline cudaError_t smem_limit_once(K kern, int bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ULL << dev) : 0ULL;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Launch classes timed by mclu_profile_begin / mclu_profile_end.
enum ProfKind { PK_PANEL = 0, PK_LASWP = 1, PK_TRSM = 2, PK_GEMM = 3, PK_SOLVE = 4, PK_OTHER = 5, PK_COUNT = 6 };
bool prof_on(int kind);
void prof_push(int kind, cudaEvent_t e0, cudaEvent_t e1);

// Brackets the launches of one class with CUDA events on their stream when
// profiling of that class is enabled (no cost otherwise).
struct ProfScope {
  int kind;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfScope(int k, cudaStream_t st) : kind(k), s(st) {
    if (prof_on(kind) && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, s);
  }
  ~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e1, s);
      prof_push(kind, e0, e1);
    } else {
      cudaEventDestroy(e0);
    }
  }
};

// Stream-ordered workspace that is released on every exit path.
struct Workspace {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  ~Workspace() {
    if (p) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(size_t bytes, cudaStream_t st) {
    s = st;
    return cudaMallocAsync(&p, bytes < 256 ? 256 : bytes, st);
  }
};

// A second stream forked from the caller's stream s: work issued on it after
// fork() starts once everything issued on s before that call is done, and
// join() makes s wait for everything issued on it so far.  The destructor
// joins (the workspace is freed stream-ordered on s, so the side work must
// come first on every exit path) and releases the stream and the events.
struct SideStream {
  cudaStream_t main = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool open = false;  // work issued on side since the last join
  cudaError_t init(cudaStream_t s) {
    main = s;
    cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
    return e;
  }
  cudaError_t fork() {
    cudaError_t e = cudaEventRecord(ev_fork, main);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
    if (e == cudaSuccess) open = true;
    return e;
  }
  cudaError_t join() {
    if (!open) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ev_join, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, ev_join, 0);
    if (e == cudaSuccess) open = false;
    return e;
  }
  ~SideStream() {
    join();
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (side) cudaStreamDestroy(side);
  }
};

struct Carver {  // 256-byte aligned sub-allocations of one workspace block
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
    T *r = reinterpret_cast<T *>(base + off);
    off += bytes;
    return r;
  }
};

// Pivot-partial slots: one per CTA of the per-column panel launches, plus two
// per CTA of the cooperative panel (alternating by column parity).
constexpr size_t panel_nparts(int64_t n) {
  return (size_t)(((n > 1 ? n : 1) + PANEL_T - 1) / PANEL_T) + 1 + 2 * COOP_GMAX;
}

// Panel widths above this use the per-column panel launches.
constexpr int COOP_NB_MAX = 256;

// Workspace of getrf for order n and panel width nb (everything except the
// Ozaki engine's slices): header, pivot partials, multiplier buffer, the
// cooperative panel's row slots, and for 3M the pre-summed planes.
template <int L>
constexpr size_t getrf_ws_bytes(int64_t n, int nb, bool m3) {
  const size_t nparts = panel_nparts(n);
  const size_t nbc = (size_t)(nb < COOP_NB_MAX ? nb : COOP_NB_MAX);
  size_t b = 4 * 256;                                              // counter, info, zflag, recip, barrier
  b += ((nparts * L * sizeof(double)) + 255) & ~(size_t)255;      // part_key
  b += ((nparts * sizeof(int)) + 255) & ~(size_t)255;             // part_idx
  b += ((nparts * 2 * L * sizeof(double)) + 255) & ~(size_t)255;  // part_rcp
  b += ((2 * 2 * L * (size_t)n * sizeof(double)) + 255) & ~(size_t)255;              // lbuf
  b += ((2 * COOP_GMAX * 2 * L * nbc * sizeof(double)) + 255) & ~(size_t)255;        // prow
  b += ((2 * 2 * L * nbc * sizeof(double)) + 255) & ~(size_t)255;                    // srow
  b += ((2 * COOP_GMAX * sizeof(int)) + 255) & ~(size_t)255;                          // rcp_flag
  b += ((2 * COOP_GMAX * COOP_KS * sizeof(double)) + 255) & ~(size_t)255;              // kslot
  b += ((2 * COOP_GMAX * 2 * L * sizeof(double)) + 255) & ~(size_t)255;                // vnext
  b += ((2 * COOP_GMAX * sizeof(int)) + 255) & ~(size_t)255;                           // v_flag
  if (m3) b += 2 * ((((size_t)n * nb * L * sizeof(double)) + 255) & ~(size_t)255);  // 3M pre-sums
  return b + 1024;
}

// Launch a triangular block solve, staging the triangle in shared memory
// when it fits (raising the kernel's dynamic shared-memory limit once).
template <int L, bool LOWER, bool UNIT, bool CONJT>
int launch_tri_block(dim3 grid, dim3 block, cudaStream_t s, View A, int64_t k0, int bs, View X, int64_t ncols,
                     const double *rdiag, int64_t rld, int64_t xrow0) {
  const size_t staged = tri_block_smem<L>(bs, (int)block.y, true);
  if (staged <= 200 * 1024) {
    static std::atomic<unsigned long long> attr{0};
    MCLU_TRY(smem_limit_once(k_tri_block<L, LOWER, UNIT, CONJT, true>, 200 * 1024, attr));
    k_tri_block<L, LOWER, UNIT, CONJT, true><<<grid, block, staged, s>>>(A, k0, bs, X, ncols, rdiag, rld, xrow0);
  } else {
    k_tri_block<L, LOWER, UNIT, CONJT, false>
        <<<grid, block, tri_block_smem<L>(bs, (int)block.y, false), s>>>(A, k0, bs, X, ncols, rdiag, rld, xrow0);
  }
  MCLU_LAUNCHED();
  return 0;
}

// Unit lower block solve of the bs x bs block of A at (k0, k0) on ncols
// columns of X (rows xrow0 ..): the four-warp-group kernel where the step
// chain is latency bound (bs <= 64, or TD/QD up to 128: measured faster),
// else the one-thread-per-row block solve (DD at 128 rows is bound by each
// SMSP's FP64 throughput, where the extra barriers cost more).
// With ncols2 > 0 the same triangle also solves columns 0 .. ncols2-1 of X2
// (rows xrow2 ..), in the same launch where the four-warp-group kernel runs.
template <int L>
int launch_lsolve(cudaStream_t s, View A, int64_t k0, int bs, View X, int64_t ncols, int64_t xrow0,
                  View X2 = View{nullptr, 0, 0}, int64_t ncols2 = 0, int64_t xrow2 = 0) {
  if (ncols < 0 || ncols2 < 0) return (int)cudaErrorInvalidValue;
  if (ncols + ncols2 == 0) return 0;
  const int RT = (bs + 31) / 32 * 32;
  if (bs <= 64 || (L >= 3 && bs <= 128)) {
    k_lsolve4<L><<<(unsigned)(ncols + ncols2), dim3(RT, 4), lsolve4_smem<L>(RT), s>>>(A, k0, bs, X, xrow0, X2,
                                                                                      ncols, xrow2);
    MCLU_LAUNCHED();
    return 0;
  }
  if (ncols2 > 0) {
    int rc = launch_lsolve<L>(s, A, k0, bs, X2, ncols2, xrow2);
    if (rc) return rc;
  }
  if (ncols == 0) return 0;
  // one column per CTA: the solve is bound by each SM's FP64 unit, so the
  // columns go to as many SMs as possible
  return launch_tri_block<L, true, true, false>(dim3((unsigned)ncols), dim3(RT, 1), s, A, k0, bs, X, ncols, nullptr, 0,
                                                xrow0);
}

// Cooperative panel factorisation (k_panel_coop for DD, k_panel_team for TD
// and QD: measured faster for each).  Returns 0 (launched), 1 (the grid or
// its shared memory does not fit: caller falls back to per-column launches)
// or a CUDA error code.
template <int L>
int launch_panel_coop(View A, int64_t n, int64_t j0, int64_t jend, int32_t *ipiv, PanelWS<L> ws, CoopWS cw,
                      cudaStream_t s) {
  const int nb = (int)(jend - j0);
  const int64_t m = n - j0;
  const int sms = oz::sm_count();
  if (nb > COOP_NB_MAX) return 1;
  int G = (int)std::min<int64_t>({(int64_t)sms, cdiv(m, 8), (int64_t)COOP_GMAX});
  if (G < 1) G = 1;
  const int rpc = (int)cdiv(m, G);
  // owned rows + the pivot rows of two columns + the partial products of the
  // multipliers and of the next column (DD), of the multipliers (TD, QD)
  const size_t smem = (((size_t)rpc + 2) * nb * 2 * L + (size_t)(L == 2 ? 8 : 4) * rpc * L) * sizeof(double);
  if (smem > 200 * 1024) return 1;
  auto kern = L == 2 ? k_panel_coop<L> : k_panel_team<L>;
  static std::atomic<unsigned long long> attr{0};
  MCLU_TRY(smem_limit_once(kern, 200 * 1024, attr));
  int occ = 0;
  MCLU_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, COOP_T, smem));
  if ((int64_t)occ * sms < G) return 1;
  int64_t a_n = n, a_j0 = j0, a_jend = jend;
  int a_rpc = rpc;
  void *args[] = {&A, &a_n, &a_j0, &a_jend, &a_rpc, &ipiv, &ws, &cw};
  MCLU_TRY(cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(COOP_T), args, smem, s));
  note_launch();
  return 0;
}

template <int L>
int launch_gemm(int method, bool beta, View A, View B, View C, View SA, View SB, int64_t m, int64_t n, int64_t k,
                cudaStream_t s) {
  if (m <= 0 || n <= 0) return 0;
  dim3 grid((unsigned)cdiv(m, GEMM_T), (unsigned)cdiv(n, GEMM_T)), block(GEMM_T, GEMM_T);
  if (method == MCLU_METHOD_3M) {
    if (beta)
      k_gemm<L, true, true><<<grid, block, 0, s>>>(A, B, C, SA, SB, m, n, k);
    else
      k_gemm<L, true, false><<<grid, block, 0, s>>>(A, B, C, SA, SB, m, n, k);
  } else {
    if (beta)
      k_gemm<L, false, true><<<grid, block, 0, s>>>(A, B, C, SA, SB, m, n, k);
    else
      k_gemm<L, false, false><<<grid, block, 0, s>>>(A, B, C, SA, SB, m, n, k);
  }
  MCLU_LAUNCHED();
  return 0;
}

template <int L>
int launch_resum(View X, View S, int64_t m, int64_t k, cudaStream_t s) {
  int64_t tot = m * k;
  if (tot <= 0) return 0;
  k_resum<L><<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(X, S, m, k);
  MCLU_LAUNCHED();
  return 0;
}

// A plain block product C = C - A B (beta) or A B on the FP64 pipe with the
// 3M (Eq. 3, pre-sums into SA / SB, m x k and k x n L-limb planes) or the 4M
// (Eq. 1) kernel.
template <int L>
int block_product(bool m3, bool beta, View A, View B, View C, double *SA, double *SB, int64_t m, int64_t n,
                  int64_t k, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  View sa{nullptr, 0, 0}, sb{nullptr, 0, 0};
  if (m3) {
    sa = View{SA, m, m * k};
    sb = View{SB, k, k * n};
    int rc = launch_resum<L>(A, sa, m, k, s);
    if (rc) return rc;
    rc = launch_resum<L>(B, sb, k, n, s);
    if (rc) return rc;
  }
  return launch_gemm<L>(m3 ? MCLU_METHOD_3M : MCLU_METHOD_4M, beta, A, B, C, sa, sb, m, n, k, s);
}

template <int L>
int launch_madd(View X, View Y, View Z, int64_t m, int64_t n, bool sub, cudaStream_t s) {
  if (m <= 0 || n <= 0) return 0;
  k_madd<L><<<(unsigned)cdiv(m * n, 256), 256, 0, s>>>(X, Y, Z, m, n, sub);
  MCLU_LAUNCHED();
  return 0;
}

// C = C - A B (m x n, inner k) by one level of Winograd's variant of
// Strassen's algorithm (Sec. 2.3: the Strassen form of the complex matrix
// product): the even part of the three dimensions splits into 2 x 2 blocks,
//   S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2,
//   T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21,
//   P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4,
//   P5 = S1 T1, P6 = S2 T2, P7 = S3 T3,
//   C11 -= P1 + P2, C12 -= P1 + P6 + P5 + P3,
//   C21 -= P1 + P6 + P7 - P4, C22 -= P1 + P6 + P7 + P5,
// seven block products (3M or 4M kernel) instead of eight; the block sums
// are accurate L-limb additions and each C block takes its sum in one
// accumulator.  An odd last k index, row and column are peeled off as plain
// products.  Workspace: stream-ordered.
template <int L>
int strassen_update(bool m3, View A, View B, View C, int64_t m, int64_t n, int64_t k, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  const int64_t m2 = m / 2, n2 = n / 2, k2 = k / 2;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t zs = al((size_t)2 * L * m2 * k2 * 8), zt = al((size_t)2 * L * k2 * n2 * 8),
               zp = al((size_t)2 * L * m2 * n2 * 8);
  const size_t za = al((size_t)L * std::max<int64_t>(m, 1) * std::max<int64_t>(k, 1) * 8),
               zb = al((size_t)L * std::max<int64_t>(k, 1) * std::max<int64_t>(n, 1) * 8);
  Workspace w;
  const bool split = m2 > 0 && n2 > 0 && k2 > 0;
  MCLU_TRY(w.alloc((split ? 4 * zs + 4 * zt + 7 * zp : 0) + za + zb, s));
  char *cur = (char *)w.p;
  double *SA = (double *)cur;
  double *SB = (double *)(cur + za);
  cur += za + zb;
  if (split) {
    auto blk = [&](View X, int64_t r0, int64_t c0) { return View{X.p + c0 * X.ld + r0, X.ld, X.ps}; };
    const View A11 = blk(A, 0, 0), A12 = blk(A, 0, k2), A21 = blk(A, m2, 0), A22 = blk(A, m2, k2);
    const View B11 = blk(B, 0, 0), B12 = blk(B, 0, n2), B21 = blk(B, k2, 0), B22 = blk(B, k2, n2);
    const View C11 = blk(C, 0, 0), C12 = blk(C, 0, n2), C21 = blk(C, m2, 0), C22 = blk(C, m2, n2);
    View Sv[4], Tv[4], Pv[7];
    for (int q = 0; q < 4; q++, cur += zs) Sv[q] = View{(double *)cur, m2, m2 * k2};
    for (int q = 0; q < 4; q++, cur += zt) Tv[q] = View{(double *)cur, k2, k2 * n2};
    for (int q = 0; q < 7; q++, cur += zp) Pv[q] = View{(double *)cur, m2, m2 * n2};
    {
      ProfScope ps(PK_OTHER, s);
      int rc = launch_madd<L>(A21, A22, Sv[0], m2, k2, false, s);       // S1
      if (!rc) rc = launch_madd<L>(Sv[0], A11, Sv[1], m2, k2, true, s);  // S2
      if (!rc) rc = launch_madd<L>(A11, A21, Sv[2], m2, k2, true, s);    // S3
      if (!rc) rc = launch_madd<L>(A12, Sv[1], Sv[3], m2, k2, true, s);  // S4
      if (!rc) rc = launch_madd<L>(B12, B11, Tv[0], k2, n2, true, s);    // T1
      if (!rc) rc = launch_madd<L>(B22, Tv[0], Tv[1], k2, n2, true, s);  // T2
      if (!rc) rc = launch_madd<L>(B22, B12, Tv[2], k2, n2, true, s);    // T3
      if (!rc) rc = launch_madd<L>(Tv[1], B21, Tv[3], k2, n2, true, s);  // T4
      if (rc) return rc;
    }
    {
      ProfScope ps(PK_GEMM, s);
      const View X[7] = {A11, A12, Sv[3], A22, Sv[0], Sv[1], Sv[2]};
      const View Y[7] = {B11, B21, B22, Tv[3], Tv[0], Tv[1], Tv[2]};
      for (int q = 0; q < 7; q++) {
        const int rc = block_product<L>(m3, false, X[q], Y[q], Pv[q], SA, SB, m2, n2, k2, s);
        if (rc) return rc;
      }
    }
    {
      ProfScope ps(PK_OTHER, s);
      const unsigned g = (unsigned)cdiv(m2 * n2, 256);
      const View P1 = Pv[0], P2 = Pv[1], P3 = Pv[2], P4 = Pv[3], P5 = Pv[4], P6 = Pv[5], P7 = Pv[6];
      k_mcombine<L><<<g, 256, 0, s>>>(C11, P1, P2, P2, P2, 2, 0u, m2, n2);
      MCLU_LAUNCHED();
      k_mcombine<L><<<g, 256, 0, s>>>(C12, P1, P6, P5, P3, 4, 0u, m2, n2);
      MCLU_LAUNCHED();
      k_mcombine<L><<<g, 256, 0, s>>>(C21, P1, P6, P7, P4, 4, 8u, m2, n2);
      MCLU_LAUNCHED();
      k_mcombine<L><<<g, 256, 0, s>>>(C22, P1, P6, P7, P5, 4, 0u, m2, n2);
      MCLU_LAUNCHED();
    }
  }
  // peeled parts: the odd k index on the even block, the odd row, the odd column
  ProfScope ps(PK_GEMM, s);
  const int64_t me = 2 * m2, ne = 2 * n2, ke = 2 * k2;
  if (!split) return block_product<L>(m3, true, A, B, C, SA, SB, m, n, k, s);
  int rc = 0;
  if (k > ke)
    rc = block_product<L>(m3, true, View{A.p + ke * A.ld, A.ld, A.ps}, View{B.p + ke, B.ld, B.ps}, C, SA, SB, me,
                          ne, k - ke, s);
  if (!rc && m > me)
    rc = block_product<L>(m3, true, View{A.p + me, A.ld, A.ps}, B, View{C.p + me, C.ld, C.ps}, SA, SB, m - me, n, k,
                          s);
  if (!rc && n > ne)
    rc = block_product<L>(m3, true, A, View{B.p + ne * B.ld, B.ld, B.ps}, View{C.p + ne * C.ld, C.ld, C.ps}, SA, SB,
                          me, n - ne, k, s);
  return rc;
}

// Right-looking blocked LU (Sec. 3): for each panel of width nb: factor the
// panel (pivot search, swap, scale, rank-1 steps), swap the rows left and
// right of it, TRSM for U12, and the trailing update A22 <- A22 - L21 U12.
// ext_ws / ext_bytes: caller-provided workspace (no allocation in this call);
// nullptr = allocate stream-ordered workspace.
template <int L>
int getrf(int64_t n, double *Ap, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
          cudaStream_t s, void *ext_ws = nullptr, size_t ext_bytes = 0) {
  if (n < 0) return -1;
  if (n > 0 && Ap == nullptr) return -2;
  if (lda < std::max<int64_t>(1, n)) return -3;
  if (n > 0 && ipiv == nullptr) return -4;
  int nb = 64, method = MCLU_METHOD_4M;
  int Se = 0;  // Ozaki slices per operand (0: the precision's default)
  // Ozaki: sub-panel width; measured at n = 4096: 32 for DD (16: the panel
  // 43.8 -> 39.9 ms, the updates between sub-panels 10.8 -> 19.0 ms), 16 for
  // TD and QD (LU + solve +2% and +7.6% over 32); again with L11^-1 formed
  // on the side stream: DD 88.6 ms (16: 96.9, 24: 92.9), TD 223.9 ms (32:
  // 240.6), QD 392.9 ms (32: 450.0)
  int sbw = L == 2 ? oz::NB_MAX : oz::NB_MAX / 2;
  if (opts) {
    if (opts->nb < 0 || opts->nb > 256) return -6;
    if (opts->nb) nb = opts->nb;
    if (opts->method < MCLU_METHOD_4M || opts->method > MCLU_METHOD_STRASSEN) return -6;
    method = opts->method;
    if (opts->sub_nb < 0 || opts->sub_nb > oz::NB_MAX) return -6;
    if (opts->sub_nb != 0 && method != MCLU_METHOD_OZAKI) return -6;
    if (opts->sub_nb) sbw = opts->sub_nb;
    if (method == MCLU_METHOD_OZAKI) {
      if (opts->ozaki_slices < 0) return -6;
      if (opts->ozaki_slices > oz::Cfg<L>::S) return MCLU_ERR_UNSUPPORTED;
      Se = opts->ozaki_slices;
      if (opts->nb == 0) nb = 4 * oz::NB_MAX;  // 128: measured best at n = 4096 (64: -3%, 96: -1.3% DD)
    }
  }
  if (Se == 0) Se = oz::default_slices<L>();
  if (n > INT32_MAX - 1) return -1;
  if (n == 0) {
    if (info) MCLU_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
    return 0;
  }
  if (method == MCLU_METHOD_UNBLOCKED) nb = (int)std::min<int64_t>(n, INT32_MAX);
  const bool m3 = method == MCLU_METHOD_3M;
  const bool ozk = method == MCLU_METHOD_OZAKI;
  Workspace w;
  const size_t oz_need = ozk ? oz::ws_bytes<L>(n, n, nb) : 0;
  // L11^-1 formed with the sub-panels on a side stream, with an Ozaki
  // workspace of its own (its products overlap those of the main stream)
  const bool side_w = ozk && n > nb;
  const size_t oz_side_need = side_w ? ((oz::ws_bytes<L>(nb, nb, nb) + 255) & ~(size_t)255) +
                                           ((2 * L * (size_t)sbw * nb * sizeof(double) + 255) & ~(size_t)255)
                                     : 0;
  const size_t ws_need = getrf_ws_bytes<L>(n, nb, m3) + oz_need + oz_side_need +
                         (ozk ? (((size_t)2 * L * nb * nb * sizeof(double) + 255) & ~(size_t)255)
                              : 0);
  char *ws_base = nullptr;
  if (ext_ws) {
    if (ext_bytes < ws_need) return MCLU_ERR_SCRATCH_CAPACITY;
    ws_base = (char *)ext_ws;
  } else {
    MCLU_TRY(w.alloc(ws_need, s));
    ws_base = (char *)w.p;
  }
  Carver cv{ws_base};
  SideStream side;  // after w: the side stream is joined before w is freed
  if (side_w) MCLU_TRY(side.init(s));
  PanelWS<L> ws;
  char *hdr = cv.take<char>(4 * 256);
  ws.counter = (int *)hdr;
  ws.info = (int *)(hdr + 256);
  ws.zflag = (int *)(hdr + 512);
  ws.recip = (double *)(hdr + 768);
  const size_t nparts = panel_nparts(n);
  const size_t nbc = (size_t)std::min(nb, COOP_NB_MAX);
  ws.part_key = cv.take<double>(nparts * L);
  ws.part_idx = cv.take<int>(nparts);
  ws.part_rcp = cv.take<double>(nparts * 2 * L);
  ws.lbuf = cv.take<double>(2 * 2 * L * (size_t)n);
  ws.lbuf_ld = n;
  CoopWS cw;
  cw.status = (int *)(hdr + 648);
  cw.kslot = cv.take<double>((size_t)2 * COOP_GMAX * COOP_KS);
  cw.prow = cv.take<double>((size_t)2 * COOP_GMAX * 2 * L * nbc);
  cw.srow = cv.take<double>((size_t)2 * 2 * L * nbc);
  cw.rcp_flag = cv.take<int>((size_t)2 * COOP_GMAX);
  cw.vnext = cv.take<double>((size_t)2 * COOP_GMAX * 2 * L);
  cw.v_flag = cv.take<int>((size_t)2 * COOP_GMAX);
  double *sumL = nullptr, *sumU = nullptr;
  if (m3) {
    sumL = cv.take<double>((size_t)n * nb * L);
    sumU = cv.take<double>((size_t)n * nb * L);
  }
  void *oz_ws = ozk ? (void *)cv.take<char>(oz_need) : nullptr;
  void *oz_ws_side = side_w ? (void *)cv.take<char>(oz::ws_bytes<L>(nb, nb, nb)) : nullptr;
  double *tbuf = side_w ? cv.take<double>(2 * L * (size_t)sbw * nb) : nullptr;  // L11[R_s, ..) W of a sub-panel
  // L11^-1 of the current block
  double *winv = ozk ? cv.take<double>((size_t)2 * L * nb * nb) : nullptr;
  int *oz_status = ws.zflag + 1;  // spare word of the header block
  MCLU_TRY(cudaMemsetAsync(hdr, 0, 3 * 256, s));
  MCLU_TRY(cudaMemsetAsync(cw.rcp_flag, 0, (size_t)2 * COOP_GMAX * sizeof(int), s));
  MCLU_TRY(cudaMemsetAsync(cw.v_flag, 0, (size_t)2 * COOP_GMAX * sizeof(int), s));
  MCLU_TRY(cudaMemsetAsync(cw.kslot, 0, (size_t)2 * COOP_GMAX * COOP_KS * sizeof(double), s));
  View A{Ap, lda, lda * n};

  // panel on rows [p0, n), columns [p0, p1): one cooperative launch, or one
  // launch per column when the grid cannot be co-resident
  auto panel = [&](int64_t p0, int64_t p1) -> int {
    ProfScope ps(PK_PANEL, s);
    int rc = launch_panel_coop<L>(A, n, p0, p1, ipiv, ws, cw, s);
    if (rc == 1) {
      k_pivot_first<L><<<(unsigned)cdiv(n - p0, SEARCH_T), SEARCH_T, 0, s>>>(A, n, p0, p0, p1, ipiv, ws);
      MCLU_LAUNCHED();
      for (int64_t j = p0; j < p1; j++) {
        dim3 grid((unsigned)std::max<int64_t>(1, cdiv(n - j - 1, PANEL_T)), (unsigned)panel_colblocks(j, p1));
        k_panel_step<L><<<grid, dim3(PANEL_T, PANEL_T), 0, s>>>(A, n, j, p0, p1, ipiv, ws);
        MCLU_LAUNCHED();
      }
      return 0;
    }
    return rc;
  };
  // the swaps ipiv[k0..k1) applied to columns [c0, c1) other than [x0, x1)
  auto laswp = [&](int64_t k0, int64_t k1, int64_t c0, int64_t c1, int64_t x0, int64_t x1) -> int {
    const int64_t ncols = (c1 - c0) - (x1 - x0);
    if (ncols <= 0 || k1 <= k0) return 0;
    if (k1 - k0 > COOP_NB_MAX) return (int)cudaErrorInvalidValue;  // one pivot per thread of k_laswp_gather
    ProfScope ps(PK_LASWP, s);
    const size_t lsm = laswp_smem((int)(k1 - k0));
    if (lsm > 48 * 1024) {
      static std::atomic<unsigned long long> attr{0};
      MCLU_TRY(smem_limit_once(k_laswp_gather<L>, (int)laswp_smem(COOP_NB_MAX), attr));
    }
    k_laswp_gather<L><<<(unsigned)cdiv(ncols, LASWP_C), 256, lsm, s>>>(A, k0, k1, ipiv, c0, c1, x0, x1);
    MCLU_LAUNCHED();
    return 0;
  };

  for (int64_t j0 = 0; j0 < n; j0 += nb) {
    const int64_t jb = std::min<int64_t>(nb, n - j0), jend = j0 + jb;
    if (!ozk) {
      int rc = panel(j0, jend);
      if (rc) return rc;
    } else {
      // Ozaki: the block is factored as sub-panels of sbw <= 32 columns, each
      // followed by the update of the block's remaining columns (their swaps,
      // their U rows by the block solve, an Ozaki product for the rest), so
      // that the trailing update below takes all jb columns in one product
      // (K = 2 jb realified: several TMEM chunks, one exact C - P per element).
      //
      // When a trailing part follows, W = L11^{-1} is formed on the way, one
      // row block per sub-panel R_s: once R_s is factored and its swaps are
      // applied, its rows of L11 are final, and (W starts as I)
      //   W[R_s, R_s]   = L_ss^{-1}                       (block solve on I)
      //   T             = L11[R_s, ..s0) W[..s0, ..s0)    (Ozaki product)
      //   W[R_s, 0..s0) = -L_ss^{-1} T                    (Ozaki product)
      // L_ss^{-1} shares the launch of the block solve of the sub-panel's U
      // rows (the same triangle and chain).  The products read only rows R_s
      // of the block's columns (final once R_s's swaps are applied: later
      // swaps move rows below R_s) and W, and only U12 = W A12 below needs
      // W, so they run on a side stream: T forked after the swaps, beside the
      // block solve; the second product after the block solve, beside the
      // sub-panel's Ozaki product.  The next sub-panel's cooperative panel
      // joins the side stream first, so that its CTAs do not hold SMs the
      // panel's grid waits for; U12 joins the last row block.  Measured at
      // n = 4096 (DD), TRSM with the waits at the joins: 8.4 ms with W[R_s,
      // 0..s0) by one product and the row block's solve in the main stream;
      // 6.9 ms with those two on the side stream (a chain of 32 dependent
      // steps there, longer than the main stream's work beside it, so its
      // joins waited); joined at U12 only, TRSM 5.0 ms but the panel 37.6
      // -> 39.9 ms (its grid waited for the side stream's CTAs).  TD and QD
      // (16-column sub-panels) formed W after the block, from the 32 x 32
      // diagonal inverses by 2 x 2 block inversion (six Ozaki products on
      // the main stream); the row blocks on the side stream measured TRSM
      // TD 17.7 -> 8.3 ms, QD 27.4 -> 12.7 ms at n = 4096.
      const bool mkw = jend < n;
      View Wb{winv, jb, jb * jb};
      View Tv{tbuf, sbw, (int64_t)sbw * nb};
      if (mkw) {  // W = I (the previous block's U12 is done)
        k_identity<L><<<(unsigned)cdiv(jb * jb, 256), 256, 0, s>>>(Wb, jb);
        MCLU_LAUNCHED();
      }
      for (int64_t s0 = j0; s0 < jend; s0 += sbw) {
        const int64_t send = std::min<int64_t>(s0 + sbw, jend), sb = send - s0;
        const int64_t wc = s0 - j0;  // columns of W left of R_s
        if (mkw && wc > 0) {
          ProfScope ps(PK_TRSM, s);
          MCLU_TRY(side.join());
        }
        int rc = panel(s0, send);
        if (rc) return rc;
        rc = laswp(s0, send, j0, jend, s0, send);  // the block's other columns, in one launch
        if (rc) return rc;
        if (mkw && wc > 0) {  // T = L11[R_s, ..s0) W[..s0, ..s0)
          MCLU_TRY(side.fork());
          rc = oz::gemm<L>(false, View{Ap + j0 * lda + s0, lda, lda * n}, Wb, Tv, sb, wc, wc, oz_ws_side, oz_status,
                           side.side, note_launch, Se);
          if (rc) return rc;
        }
        {  // the U rows of the block's columns right of R_s, and W[R_s, R_s] = L_ss^{-1}
          ProfScope ps(send < jend ? PK_OTHER : PK_TRSM, s);
          View U{Ap + send * lda, lda, lda * n};  // rows s0.., columns send..jend
          rc = launch_lsolve<L>(s, A, s0, (int)sb, U, jend - send, s0, View{winv + wc * jb, jb, jb * jb},
                                mkw ? sb : 0, wc);
          if (rc) return rc;
        }
        if (mkw && wc > 0) {  // W[R_s, 0..s0) = -L_ss^{-1} T
          MCLU_TRY(side.fork());
          rc = oz::gemm<L>(true, View{winv + wc * jb + wc, jb, jb * jb}, Tv, View{winv + wc, jb, jb * jb}, sb, wc, sb,
                           oz_ws_side, oz_status, side.side, note_launch, Se);
          if (rc) return rc;
        }
        if (send < jend) {
          ProfScope ps(PK_OTHER, s);
          rc = oz::gemm<L>(true, View{Ap + s0 * lda + send, lda, lda * n}, View{Ap + send * lda + s0, lda, lda * n},
                           View{Ap + send * lda + send, lda, lda * n}, n - send, jend - send, sb, oz_ws, oz_status, s,
                           note_launch, Se);
          if (rc) return rc;
        }
      }
    }
    {  // apply the block's swaps to the columns left and right of it
      int rc = laswp(j0, jend, 0, n, j0, jend);
      if (rc) return rc;
    }
    if (jend < n) {
      const int64_t n2 = n - jend;
      {  // U12 = L11^{-1} A12
        ProfScope ps(PK_TRSM, s);
        View A12{Ap + jend * lda, lda, lda * n};
        if (!ozk) {
          int rc = launch_lsolve<L>(s, A, j0, (int)jb, A12, n2, j0);
          if (rc) return rc;
        } else {
          // U12 = W A12 with W = L11^{-1} (formed with the sub-panels above,
          // on the side stream), as an Ozaki product written in place (the
          // operands are sliced before the product is stored).
          View W{winv, jb, jb * jb};
          MCLU_TRY(side.join());
          int rc = oz::gemm<L>(false, W, View{Ap + jend * lda + j0, lda, lda * n}, View{Ap + jend * lda + j0, lda, lda * n},
                               jb, n2, jb, oz_ws, oz_status, s, note_launch, Se);
          if (rc) return rc;
        }
      }
      // A22 -= L21 U12
      View L21{Ap + j0 * lda + jend, lda, lda * n};
      View U12{Ap + jend * lda + j0, lda, lda * n};
      View A22{Ap + jend * lda + jend, lda, lda * n};
      View SL{nullptr, 0, 0}, SU{nullptr, 0, 0};
      if (m3) {
        ProfScope ps(PK_OTHER, s);
        SL = View{sumL, n2, n2 * jb};
        SU = View{sumU, jb, jb * n2};
        int rc = launch_resum<L>(L21, SL, n2, jb, s);
        if (rc) return rc;
        rc = launch_resum<L>(U12, SU, jb, n2, s);
        if (rc) return rc;
      }
      int rc;
      if (method == MCLU_METHOD_STRASSEN) {
        rc = strassen_update<L>(true, L21, U12, A22, n2, n2, jb, s);
      } else {
        ProfScope ps(PK_GEMM, s);
        rc = ozk ? oz::gemm<L>(true, L21, U12, A22, n2, n2, jb, oz_ws, oz_status, s, note_launch, Se)
                 : launch_gemm<L>(method, true, L21, U12, A22, SL, SU, n2, n2, jb, s);
      }
      if (rc) return rc;
    }
  }
  // a timed-out tensor-core pipeline or panel exchange is reported through info
  k_merge_status<<<1, 1, 0, s>>>(oz_status, ws.info);
  MCLU_LAUNCHED();
  k_merge_status<<<1, 1, 0, s>>>(cw.status, ws.info);
  MCLU_LAUNCHED();
  if (info) MCLU_TRY(cudaMemcpyAsync(info, ws.info, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return 0;
}

// Forward (LOWER) or backward substitution with op(T) over all diagonal
// blocks: R holds the right-hand sides on entry and is consumed as the
// residual; the solution goes to Y.  W: inverses of the diagonal blocks of
// T (k_blk_inv), applied as their conjugate transposes with CONJT.
template <int L, bool LOWER, bool CONJT>
int tri_solve(View A, int64_t n, const double *W, View R, View Y, int64_t nrhs, cudaStream_t s) {
  constexpr int BS = SOLVE_BS;
  constexpr size_t smem = blk_solve_smem<L>();
  if (smem > 48 * 1024) {
    static std::atomic<unsigned long long> attr{0};
    MCLU_TRY(smem_limit_once(k_blk_solve<L, LOWER, CONJT>, (int)smem, attr));
  }
  const int64_t nblk = cdiv(n, BS);
  for (int64_t c0 = 0; c0 < nrhs; c0 += 65535) {
    const int64_t nc = std::min<int64_t>(65535, nrhs - c0);
    const View Rc{R.p + c0 * R.ld, R.ld, R.ps}, Yc{Y.p + c0 * Y.ld, Y.ld, Y.ps};
    for (int64_t q = 0; q < nblk; q++) {
      const int64_t b = LOWER ? q : nblk - 1 - q;
      const int64_t k0 = b * BS;
      const int bs = (int)std::min<int64_t>(BS, n - k0);
      const int64_t r0 = LOWER ? k0 + bs : 0, r1 = LOWER ? n : k0;
      const dim3 grid((unsigned)std::max<int64_t>(1, cdiv(r1 - r0, 32)), (unsigned)nc);
      k_blk_solve<L, LOWER, CONJT><<<grid, 256, smem, s>>>(A, k0, bs, W + b * 2 * L * BS * BS, Rc, Yc, r0, r1);
      MCLU_LAUNCHED();
    }
  }
  return 0;
}

// The same substitution as one persistent cooperative launch per right-hand
// side (k_trsv_flow).  Y: packed planes (Y.ps = Y.ld nrhs); it is filled
// with FLOW_SENT first.  status: OR-ed with 1 if a wait ran out.  Returns 1
// when the grid cannot be co-resident (the caller falls back to tri_solve).
template <int L, bool LOWER, bool CONJT>
int tri_solve_flow(View A, int64_t n, const double *W, View R, View Y, int64_t nrhs, int *status, cudaStream_t s) {
  const int sms = oz::sm_count();
  const int64_t nblk = cdiv(n, SOLVE_BS);
  const int G = (int)std::min<int64_t>(sms, nblk);
  const int nown = (int)cdiv(nblk, G);
  const size_t smem = trsv_flow_smem<L>(nown);
  if (smem > 200 * 1024) return 1;
  if (smem > 48 * 1024) {
    static std::atomic<unsigned long long> attr{0};
    MCLU_TRY(smem_limit_once(k_trsv_flow<L, LOWER, CONJT>, 200 * 1024, attr));
  }
  int occ = 0;
  MCLU_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trsv_flow<L, LOWER, CONJT>, FLOW_T, smem));
  if ((int64_t)occ * sms < G) return 1;
  {  // every word of the solution starts as FLOW_SENT
    const int64_t words = 2 * L * Y.ps;
    k_fill_u64<<<(unsigned)cdiv(words, 256), 256, 0, s>>>(reinterpret_cast<unsigned long long *>(Y.p), words,
                                                           FLOW_SENT);
    MCLU_LAUNCHED();
  }
  for (int64_t c = 0; c < nrhs; c++) {
    View Rc{R.p + c * R.ld, R.ld, R.ps}, Yc{Y.p + c * Y.ld, Y.ld, Y.ps};
    int64_t a_n = n;
    const double *a_W = W;
    int *a_status = status;
    void *args[] = {&A, &a_n, &a_W, &Rc, &Yc, &a_status};
    MCLU_TRY(cudaLaunchCooperativeKernel((const void *)k_trsv_flow<L, LOWER, CONJT>, dim3(G), dim3(FLOW_T), args, smem,
                                         s));
    note_launch();
  }
  return 0;
}

template <int L>
int getrs(char trans, int64_t n, int64_t nrhs, const double *Ap, int64_t lda, const int32_t *ipiv, double *Bp,
          int64_t ldb, cudaStream_t s) {
  if (trans != 'N' && trans != 'n' && trans != 'C' && trans != 'c') return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (n > 0 && Ap == nullptr) return -4;
  if (lda < std::max<int64_t>(1, n)) return -5;
  if (n > 0 && ipiv == nullptr) return -6;
  if (n > 0 && nrhs > 0 && Bp == nullptr) return -7;
  if (ldb < std::max<int64_t>(1, n)) return -8;
  if (n == 0 || nrhs == 0) return 0;
  if (n > INT32_MAX - 1) return -2;
  const bool conj = (trans == 'C' || trans == 'c');
  ProfScope ps(PK_SOLVE, s);
  View A{const_cast<double *>(Ap), lda, lda * n};
  View B{Bp, ldb, ldb * nrhs};
  constexpr int BS = SOLVE_BS;
  const int64_t nblk = cdiv(n, BS);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t perm_bytes = al((size_t)n * sizeof(int32_t));
  const size_t rdiag_bytes = al((size_t)2 * L * n * sizeof(double));
  const size_t inv_bytes = al((size_t)nblk * 2 * L * BS * BS * sizeof(double));
  const size_t vec_bytes = al((size_t)2 * L * n * nrhs * sizeof(double));
  const size_t flag_bytes = al((size_t)(nblk + 1) * sizeof(int));
  if (2 * nrhs + 1 > INT32_MAX) return -3;
  Workspace w;
  MCLU_TRY(w.alloc(perm_bytes + rdiag_bytes + 2 * inv_bytes + 2 * vec_bytes + flag_bytes, s));
  char *cur = (char *)w.p;
  int *flags = (int *)cur;  // the status word of the dataflow substitutions at flags[nblk]
  cur += flag_bytes;
  MCLU_TRY(cudaMemsetAsync(flags, 0, (size_t)(nblk + 1) * sizeof(int), s));
  int32_t *perm = (int32_t *)cur;
  cur += perm_bytes;
  double *rdiag = (double *)cur;
  cur += rdiag_bytes;
  double *WL = (double *)cur;
  cur += inv_bytes;
  double *WU = (double *)cur;
  cur += inv_bytes;
  View X{(double *)cur, n, n * nrhs};
  cur += vec_bytes;
  View Y{(double *)cur, n, n * nrhs};
  // diagonal reciprocals, then the inverses of all diagonal blocks of L and U
  k_diag_recip<L><<<(unsigned)cdiv(n, 128), 128, 0, s>>>(A, n, rdiag, n);
  MCLU_LAUNCHED();
  k_blk_inv<L><<<dim3((unsigned)nblk, 2), BS, 0, s>>>(A, n, WL, WU, rdiag, n);
  MCLU_LAUNCHED();
  const size_t smem_perm = (size_t)n * sizeof(int32_t);
  const int use_smem = smem_perm <= 200 * 1024 ? 1 : 0;
  if (use_smem) MCLU_TRY(cudaFuncSetAttribute(k_perm_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  k_perm_build<<<1, 32, use_smem ? smem_perm : 0, s>>>(ipiv, n, perm, use_smem);
  MCLU_LAUNCHED();
  const unsigned pg = (unsigned)cdiv(n * nrhs, 256);
  if (!conj) {
    k_permute<L><<<pg, 256, 0, s>>>(B, X, perm, n, nrhs, 0);  // X = P B
    MCLU_LAUNCHED();
    int rc = tri_solve_flow<L, true, false>(A, n, WL, X, Y, nrhs, flags + nblk, s);  // L y = P b
    if (rc == 1) rc = tri_solve<L, true, false>(A, n, WL, X, Y, nrhs, s);
    if (rc) return rc;
    rc = tri_solve_flow<L, false, false>(A, n, WU, Y, X, nrhs, flags + nblk, s);  // U x = y
    if (rc == 1) rc = tri_solve<L, false, false>(A, n, WU, Y, X, nrhs, s);
    if (rc) return rc;
    MCLU_TRY(cudaMemcpy2DAsync(Bp, ldb * sizeof(double), X.p, n * sizeof(double), n * sizeof(double),
                               (size_t)2 * L * nrhs, cudaMemcpyDeviceToDevice, s));
  } else {
    MCLU_TRY(cudaMemcpy2DAsync(X.p, n * sizeof(double), Bp, ldb * sizeof(double), n * sizeof(double),
                               (size_t)2 * L * nrhs, cudaMemcpyDeviceToDevice, s));
    int rc = tri_solve_flow<L, true, true>(A, n, WU, X, Y, nrhs, flags + nblk, s);  // U^H w = b
    if (rc == 1) rc = tri_solve<L, true, true>(A, n, WU, X, Y, nrhs, s);
    if (rc) return rc;
    rc = tri_solve_flow<L, false, true>(A, n, WL, Y, X, nrhs, flags + nblk, s);  // L^H z = w
    if (rc == 1) rc = tri_solve<L, false, true>(A, n, WL, Y, X, nrhs, s);
    if (rc) return rc;
    k_permute<L><<<pg, 256, 0, s>>>(X, B, perm, n, nrhs, 1);  // B = P^T z
    MCLU_LAUNCHED();
  }
  return 0;
}

// Real (one-plane) factorisation and solve: the real L-limb planes enter the
// complex path as the real part of complex planes with a zero imaginary part
// (a complex workspace of 2L planes, stream-ordered).  The complex pivot key
// cabs1(a + 0i) = |a| is the real one, and every imaginary part stays exactly
// zero through the factorisation (each product with a zero factor is an exact
// zero, every sum of zeros is exact), so the factors are the real parts.
template <int L>
int dgetrf(int64_t n, double *Ap, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
           cudaStream_t s) {
  if (n < 0) return -1;
  if (n > 0 && Ap == nullptr) return -2;
  if (lda < std::max<int64_t>(1, n)) return -3;
  if (n > 0 && ipiv == nullptr) return -4;
  if (n == 0) return getrf<L>(0, Ap, lda, ipiv, info, opts, s);
  if (n > INT32_MAX - 1) return -1;
  Workspace w;
  MCLU_TRY(w.alloc((size_t)2 * L * n * n * sizeof(double), s));
  View Z{(double *)w.p, n, n * n};
  const unsigned grid = (unsigned)cdiv(n * n, 256);
  k_real_planes<L><<<grid, 256, 0, s>>>(Ap, lda, Z, n, n, true);
  MCLU_LAUNCHED();
  const int rc = getrf<L>(n, Z.p, n, ipiv, info, opts, s);
  if (rc) return rc;
  k_real_planes<L><<<grid, 256, 0, s>>>(Ap, lda, Z, n, n, false);
  MCLU_LAUNCHED();
  return 0;
}

// Solve with the factors of dgetrf: 'N' A X = B, 'T' A^T X = B (the complex
// 'C' solve on the zero-imaginary embedding).  B: L planes, n x nrhs,
// leading dimension ldb.
template <int L>
int dgetrs(char trans, int64_t n, int64_t nrhs, const double *Ap, int64_t lda, const int32_t *ipiv, double *Bp,
           int64_t ldb, cudaStream_t s) {
  if (trans != 'N' && trans != 'n' && trans != 'T' && trans != 't') return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (n > 0 && Ap == nullptr) return -4;
  if (lda < std::max<int64_t>(1, n)) return -5;
  if (n > 0 && ipiv == nullptr) return -6;
  if (n > 0 && nrhs > 0 && Bp == nullptr) return -7;
  if (ldb < std::max<int64_t>(1, n)) return -8;
  if (n == 0 || nrhs == 0) return 0;
  if (n > INT32_MAX - 1) return -2;
  Workspace w;
  const size_t za = (size_t)2 * L * n * n, zb = (size_t)2 * L * n * nrhs;
  MCLU_TRY(w.alloc((za + zb) * sizeof(double), s));
  View ZA{(double *)w.p, n, n * n}, ZB{(double *)w.p + za, n, n * nrhs};
  k_real_planes<L><<<(unsigned)cdiv(n * n, 256), 256, 0, s>>>(const_cast<double *>(Ap), lda, ZA, n, n, true);
  MCLU_LAUNCHED();
  k_real_planes<L><<<(unsigned)cdiv(n * nrhs, 256), 256, 0, s>>>(Bp, ldb, ZB, n, nrhs, true);
  MCLU_LAUNCHED();
  const char ct = (trans == 'N' || trans == 'n') ? 'N' : 'C';
  const int rc = getrs<L>(ct, n, nrhs, ZA.p, n, ipiv, ZB.p, n, s);
  if (rc) return rc;
  k_real_planes<L><<<(unsigned)cdiv(n * nrhs, 256), 256, 0, s>>>(Bp, ldb, ZB, n, nrhs, false);
  MCLU_LAUNCHED();
  return 0;
}

template <int L>
int gemm(int beta_mode, int method, int64_t m, int64_t n, int64_t k, const double *Ap, int64_t lda, const double *Bp,
         int64_t ldb, double *Cp, int64_t ldc, cudaStream_t s, int ozaki_slices = 0) {
  if (beta_mode != 0 && beta_mode != 1) return -1;
  if (method != MCLU_METHOD_4M && method != MCLU_METHOD_3M && method != MCLU_METHOD_OZAKI &&
      method != MCLU_METHOD_STRASSEN)
    return -2;
  // ozaki_slices: 0 (default) or 1 .. S, checked by the caller
  const int Se = ozaki_slices ? ozaki_slices : oz::default_slices<L>();
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  if (m > 0 && k > 0 && Ap == nullptr) return -6;
  if (lda < std::max<int64_t>(1, m)) return -7;
  if (k > 0 && n > 0 && Bp == nullptr) return -8;
  if (ldb < std::max<int64_t>(1, k)) return -9;
  if (m > 0 && n > 0 && Cp == nullptr) return -10;
  if (ldc < std::max<int64_t>(1, m)) return -11;
  if (m == 0 || n == 0) return 0;
  View A{const_cast<double *>(Ap), lda, lda * k}, B{const_cast<double *>(Bp), ldb, ldb * n}, C{Cp, ldc, ldc * n};
  View SA{nullptr, 0, 0}, SB{nullptr, 0, 0};
  Workspace w;
  if (method == MCLU_METHOD_OZAKI) {
    MCLU_TRY(w.alloc(oz::ws_bytes<L>(m, n, k) + 256, s));
    int *status = (int *)((char *)w.p + oz::ws_bytes<L>(m, n, k));
    MCLU_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    ProfScope ps(PK_GEMM, s);
    return oz::gemm<L>(beta_mode == 1, A, B, C, m, n, k, w.p, status, s, note_launch, Se);
  }
  if (method == MCLU_METHOD_STRASSEN) {
    if (beta_mode == 0) {  // C = A B: zero C, C -= A B, negate (exact)
      for (int pl = 0; pl < 2 * L; pl++)
        MCLU_TRY(cudaMemset2DAsync(C.p + (int64_t)pl * C.ps, C.ld * sizeof(double), 0, m * sizeof(double), n, s));
    }
    if (k == 0) return 0;
    int rc = strassen_update<L>(true, A, B, C, m, n, k, s);
    if (rc || beta_mode == 1) return rc;
    k_mneg<L><<<(unsigned)cdiv(m * n, 256), 256, 0, s>>>(C, m, n);
    MCLU_LAUNCHED();
    return 0;
  }
  if (method == MCLU_METHOD_3M && k > 0) {
    MCLU_TRY(w.alloc((size_t)(m * k + k * n) * L * sizeof(double) + 512, s));
    SA = View{(double *)w.p, m, m * k};
    SB = View{(double *)w.p + m * k * L, k, k * n};
    int rc = launch_resum<L>(A, SA, m, k, s);
    if (rc) return rc;
    rc = launch_resum<L>(B, SB, k, n, s);
    if (rc) return rc;
  }
  ProfScope ps(PK_GEMM, s);
  return launch_gemm<L>(method, beta_mode == 1, A, B, C, SA, SB, m, n, k, s);
}

template <int L>
int adjoint_rank1(int64_t n, const double *lam, const double *x, double *Ab, int64_t ldab, cudaStream_t s) {
  if (n < 0) return -1;
  if (n > 0 && (lam == nullptr)) return -2;
  if (n > 0 && (x == nullptr)) return -3;
  if (n > 0 && (Ab == nullptr)) return -4;
  if (ldab < std::max<int64_t>(1, n)) return -5;
  if (n == 0) return 0;
  if (n > 65535) return -1;
  View vl{const_cast<double *>(lam), n, n}, vx{const_cast<double *>(x), n, n}, vA{Ab, ldab, ldab * n};
  k_rank1_adjoint<L><<<dim3((unsigned)cdiv(n, 256), (unsigned)n), 256, 0, s>>>(vl, vx, vA, n);
  MCLU_LAUNCHED();
  return 0;
}

// Ozaki split of one operand (diagnostic): side 0 = row-scaled A (rows x cols),
// side 1 = column-scaled B (rows x cols); slices and exponents copied out.
template <int L>
int ozaki_split(int side, int64_t rows, int64_t cols, const double *X, int64_t ld, void *slices, int *E,
                cudaStream_t s) {
  if (side != 0 && side != 1) return -2;
  if (rows < 0) return -3;
  if (cols < 0) return -4;
  if (!X && rows > 0 && cols > 0) return -5;
  if (ld < std::max<int64_t>(1, rows)) return -6;
  if (!slices) return -7;
  if (!E) return -8;
  if (rows == 0 || cols == 0) return 0;
  View V{const_cast<double *>(X), ld, ld * cols};
  // reuse the two-operand split with a 1-element dummy on the other side
  const int64_t m = side == 0 ? rows : 1, n = side == 1 ? cols : 1, k = side == 0 ? cols : rows;
  const oz::Sizes<L> z = oz::sizes<L>(m, n, k);
  Workspace w;
  MCLU_TRY(w.alloc(z.total + 2 * L * 8 * (size_t)(k + 1), s));
  double *dummy = (double *)((char *)w.p + z.total);
  MCLU_TRY(cudaMemsetAsync(dummy, 0, 2 * L * 8 * (size_t)(k + 1), s));
  View D{dummy, side == 0 ? k : 1, side == 0 ? k : k};
  int rc = side == 0 ? oz::split<L>(V, View{dummy, k, k}, m, n, k, w.p, s, note_launch)
                     : oz::split<L>(View{dummy, 1, k}, V, m, n, k, w.p, s, note_launch);
  (void)D;
  if (rc) return rc;
  char *base = (char *)w.p;
  const size_t bytes = side == 0 ? z.a_bytes : z.b_bytes;
  MCLU_TRY(cudaMemcpyAsync(slices, base + (side == 0 ? 0 : z.a_bytes), bytes, cudaMemcpyDeviceToDevice, s));
  const int *Es = (const int *)(base + z.a_bytes + z.b_bytes) + (side == 0 ? 0 : z.Mpad);
  MCLU_TRY(cudaMemcpyAsync(E, Es, (side == 0 ? rows : cols) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  return 0;
}

template <int L>
int vec_op(int op, int64_t count, const double *x, const double *y, double *z, cudaStream_t s) {
  const bool real = op >= 0 && op <= 3;
  const bool cplx = op >= 10 && op <= 17;
  if (!real && !cplx) return -1;
  if (count < 0) return -3;
  if (count == 0) return 0;
  if (!x) return -4;
  if (!y && op < 15) return -5;
  if (!z) return -6;
  k_vec_op<L><<<(unsigned)cdiv(count, 128), 128, 0, s>>>(op, count, x, y, z);
  MCLU_LAUNCHED();
  return 0;
}

}  // namespace mclu

// One translation unit per precision defines the C entry points.
#define MCLU_DEFINE_PRECISION(SUF, LIMBS)                                                                        \
  extern "C" int zgetrf_##SUF##_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info,             \
                                   const mclu_opts *opts, void *stream) {                                       \
    return mclu::getrf<LIMBS>(n, A, lda, ipiv, info, opts, (cudaStream_t)stream);                               \
  }                                                                                                              \
  extern "C" int zgetrf_##SUF(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream) {                 \
    return mclu::getrf<LIMBS>(n, A, lda, ipiv, nullptr, nullptr, (cudaStream_t)stream);                         \
  }                                                                                                              \
  extern "C" int dgetrf_##SUF##_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info,             \
                                   const mclu_opts *opts, void *stream) {                                       \
    return mclu::dgetrf<LIMBS>(n, A, lda, ipiv, info, opts, (cudaStream_t)stream);                              \
  }                                                                                                              \
  extern "C" int dgetrf_##SUF(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream) {                 \
    return mclu::dgetrf<LIMBS>(n, A, lda, ipiv, nullptr, nullptr, (cudaStream_t)stream);                        \
  }                                                                                                              \
  extern "C" int dgetrs_##SUF(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda,                \
                              const int32_t *ipiv, double *B, int64_t ldb, void *stream) {                      \
    return mclu::dgetrs<LIMBS>(trans, n, nrhs, A, lda, ipiv, B, ldb, (cudaStream_t)stream);                     \
  }                                                                                                              \
  extern "C" int zgetrs_##SUF(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda,                \
                              const int32_t *ipiv, double *B, int64_t ldb, void *stream) {                      \
    return mclu::getrs<LIMBS>(trans, n, nrhs, A, lda, ipiv, B, ldb, (cudaStream_t)stream);                      \
  }                                                                                                              \
  extern "C" int zgemm_##SUF(int beta_mode, int method, int64_t m, int64_t n, int64_t k, const double *A,       \
                             int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, void *stream) { \
    return mclu::gemm<LIMBS>(beta_mode, method, m, n, k, A, lda, B, ldb, C, ldc, (cudaStream_t)stream);        \
  }                                                                                                              \
  extern "C" int zgemm_##SUF##_ex(int beta_mode, int method, int ozaki_slices, int64_t m, int64_t n, int64_t k,   \
                                 const double *A, int64_t lda, const double *B, int64_t ldb, double *C,          \
                                 int64_t ldc, void *stream) {                                                    \
    if (ozaki_slices < 0) return -3;                                                                             \
    if (ozaki_slices > mclu::oz::Cfg<LIMBS>::S) return MCLU_ERR_UNSUPPORTED;                                     \
    int rc = mclu::gemm<LIMBS>(beta_mode, method, m, n, k, A, lda, B, ldb, C, ldc, (cudaStream_t)stream,        \
                               ozaki_slices);                                                                    \
    return rc <= -3 ? rc - 1 : rc; /* the arguments after ozaki_slices are one place further */                 \
  }                                                                                                              \
  extern "C" int zadjoint_rank1_##SUF(int64_t n, const double *lambda, const double *x, double *Abar,           \
                                      int64_t ldab, void *stream) {                                             \
    return mclu::adjoint_rank1<LIMBS>(n, lambda, x, Abar, ldab, (cudaStream_t)stream);                          \
  }                                                                                                              \
  int mclu_vec_op_##SUF(int op, int64_t count, const double *x, const double *y, double *z, void *stream) {     \
    return mclu::vec_op<LIMBS>(op, count, x, y, z, (cudaStream_t)stream);                                       \
  }                                                                                                              \
  extern "C" int zozaki_split_##SUF(int side, int64_t rows, int64_t cols, const double *X, int64_t ld,          \
                                    void *slices, int32_t *E, void *stream) {                                   \
    return mclu::ozaki_split<LIMBS>(side, rows, cols, X, ld, slices, E, (cudaStream_t)stream);                  \
  }
