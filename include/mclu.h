/*
 * mclu.h - C ABI of the GB300 (sm_103a) complex multi-component LU library.
 *
 * The library factors and solves complex linear systems A x = b (Sec. 3,
 * Eq. (4) of Kouya, "Performance evaluation of accelerated complex
 * multiple-precision LU decomposition") in double-double (DD, 2 limbs),
 * triple-double (TD, 3 limbs) and quadruple-double (QD, 4 limbs) arithmetic:
 * a real value is the unevaluated sum of L binary64 limbs (Sec. 1).
 *
 * Storage ("separate arrays for the real and imaginary parts", Sec. 2.2):
 * a complex L-limb matrix with `rows` rows and `ncols` columns is 2*L
 * column-major binary64 planes.  Plane (c, l), c = 0 real / 1 imaginary,
 * l = 0..L-1 limb, starts at  base + (c*L + l) * ld * ncols, and element
 * (i, j) of a plane is at offset j*ld + i.  Limbs must be ordered and
 * nonoverlapping: |limb l+1| <= ulp(limb l).  Every result the library writes
 * satisfies this; inputs with |limb l+1| <= ulp(limb l)/2 are canonical.
 *
 * Pointers: every matrix / vector / pivot pointer is a DEVICE pointer owned by
 * the caller, unless a parameter says otherwise.  `stream` is a cudaStream_t
 * passed as void* (NULL = legacy default stream).  Calls are asynchronous and
 * stream-ordered: the return value only reports argument errors and launch
 * failures; results are valid after the stream has been synchronised.  The
 * library keeps no state between calls; workspace is allocated stream-ordered
 * (cudaMallocAsync) inside each call and released before it returns.
 *
 * Return status: 0 = enqueued; -i = argument i (1-based) invalid, nothing
 * enqueued; > 0 = a CUDA error code (cudaError_t) from a launch or allocation;
 * MCLU_ERR_UNSUPPORTED = a valid request this build does not implement.
 */
#ifndef MCLU_H
#define MCLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCLU_ERR_UNSUPPORTED 100000
#define MCLU_ERR_SCRATCH_CAPACITY 100001

/* Trailing-update methods (Sec. 2.1 and Sec. 3). */
enum {
  MCLU_METHOD_4M = 0,        /* complex product by Eq. (1): four real products per complex MAC   */
  MCLU_METHOD_3M = 1,        /* 3M matrix product by Eq. (3): T1, T2, T3 then Re = T1 - T2,      */
                             /*   Im = T3 - (T1 + T2)                                              */
  MCLU_METHOD_UNBLOCKED = 2, /* "Normal LU" of Sec. 3: right-looking row elimination, no GEMM    */
  MCLU_METHOD_OZAKI = 3,     /* Ozaki-scheme update (Sec. 2.3): exact bf16 slice products on the */
                             /*   tensor cores; block width nb <= 256 (default 128), factored as */
                             /*   sub-panels with Ozaki updates between them                     */
  MCLU_METHOD_STRASSEN = 4   /* Strassen form (Sec. 2.3): one level of Winograd's variant, seven */
                             /*   3M block products instead of eight on the FP64 pipe            */
};

/* Optional parameters of the *_ex factorisation calls (NULL = defaults). */
typedef struct mclu_opts {
  int32_t nb;           /* panel width K of Sec. 3 (block size NDIM); 0 = 64 (128 for Ozaki); */
                        /*   1..256                                                           */
  int32_t method;       /* MCLU_METHOD_*; default MCLU_METHOD_4M                             */
  int32_t ozaki_slices; /* MCLU_METHOD_OZAKI: slices kept per operand, 1..S (S = 16 DD, 24 TD, */
                        /*   32 QD; above S: MCLU_ERR_UNSUPPORTED); 0 = the precision's S     */
  int32_t sub_nb;       /* MCLU_METHOD_OZAKI: width of the sub-panels each block is factored  */
                        /*   in (the columns between them updated by Ozaki products), 1..32; */
                        /*   0 = 32 for DD, 16 for TD and QD.  Must be 0 for other methods    */
} mclu_opts;

/*
 * zgetrf_{dd,td,qd}: LU factorisation with partial pivoting, P A = L U
 * (Sec. 3: blocked right-looking LU with block size K, A22 <- A22 - L21 U12 by
 * complex matrix multiplication, partial pivoting).
 *   n     order of A (n >= 0)
 *   A     device, n x n planes with leading dimension lda (plane stride
 *         lda*n); overwritten by L (unit diagonal not stored) and U
 *   lda   >= max(1, n)
 *   ipiv  device int32[n]: 1-based pivot rows; row k was swapped with row
 *         ipiv[k]-1, applied for k = 0..n-1 (LAPACK convention)
 * Pivot key: cabs1(z) = |Re z| + |Im z| in L-limb arithmetic; ties go to the
 * lowest row index.  A zero pivot does not stop the factorisation (use the
 * _ex form to read info).  Default method: 4M, nb = 64.
 */
int zgetrf_dd(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream);
int zgetrf_td(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream);
int zgetrf_qd(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream);

/*
 * zgetrf_{dd,td,qd}_ex: as zgetrf_*, plus
 *   info  device int32[1] or NULL: 0, or k+1 for the first exactly-zero pivot
 *         U[k,k] (LAPACK convention); < 0 only if a tensor-core pipeline
 *         wait of MCLU_METHOD_OZAKI timed out (results invalid)
 *   opts  host pointer or NULL (defaults)
 * With MCLU_METHOD_OZAKI and n > nb, part of the work (the row blocks of
 * L11^-1, two small Ozaki products per sub-panel) runs on a stream the call
 * creates and destroys itself, forked from `stream` with events and joined
 * back to it before the call's last work on `stream`: to the caller the call
 * is ordered on `stream` like any other.
 */
int zgetrf_dd_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
                 void *stream);
int zgetrf_td_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
                 void *stream);
int zgetrf_qd_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
                 void *stream);

/*
 * zgetrf_dd_noalloc: zgetrf_dd_ex with the defaults (4M, nb = 64) that
 * allocates no memory.  The paper has no counterpart: this serves callers
 * that may not allocate device memory during the call (inside a CUDA graph
 * capture, real-time code that allows no allocator calls after start-up, or
 * a host that gives the library only its own buffers).  Its scratch is one
 * fixed device array in the library (about 1.6 MB, held on every GPU that
 * loads the library until the process exits), so:
 *   n     0 <= n <= zgetrf_dd_noalloc_max_n() (8192); larger n returns
 *         MCLU_ERR_SCRATCH_CAPACITY and enqueues nothing
 *   A, lda, ipiv, info, stream  as in zgetrf_dd_ex (info may be NULL)
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it: make that first call before any stream
 * capture.  The cache is never refreshed: after a cudaDeviceReset of a
 * device, the cached address is stale, so a process that resets a device must
 * not call this entry point on that device again.  All calls share the array: calls that can overlap on the GPU
 * (several streams or host threads) race and must be serialised by the
 * caller.  Counters that must start at zero are cleared by every call.
 */
int zgetrf_dd_noalloc(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, void *stream);
int64_t zgetrf_dd_noalloc_max_n(void);

/*
 * dgetrf_{dd,td,qd}, dgetrf_{dd,td,qd}_ex: LU factorisation with partial
 * pivoting of a REAL L-limb matrix, P A = L U (the real multi-component LU
 * of Secs. 1 and 3 that the complex one extends).
 *   A     device, L column-major planes (plane l at A + l*lda*n), n x n,
 *         leading dimension lda; overwritten by L (unit diagonal not
 *         stored) and U
 *   n, lda, ipiv, info, opts, stream  as in zgetrf_*_ex
 * Pivot key |a| in L-limb arithmetic, ties to the lowest row.  The real
 * planes run through the complex path as the real part of a complex matrix
 * with a zero imaginary part (cabs1(a + 0i) = |a|; every imaginary part
 * stays exactly zero): a workspace of 2 L n^2 doubles is allocated
 * stream-ordered, and the cost is that of the complex factorisation.
 */
int dgetrf_dd(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream);
int dgetrf_td(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream);
int dgetrf_qd(int64_t n, double *A, int64_t lda, int32_t *ipiv, void *stream);
int dgetrf_dd_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
                 void *stream);
int dgetrf_td_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
                 void *stream);
int dgetrf_qd_ex(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, const mclu_opts *opts,
                 void *stream);

/*
 * dgetrs_{dd,td,qd}: solve with the factors of dgetrf_* (Sec. 4).
 *   trans 'N': A X = B;  'T': A^T X = B
 *   B     device, L planes of n x nrhs, leading dimension ldb (plane stride
 *         ldb*nrhs); overwritten by X
 *   the other arguments as in zgetrs_*; a workspace of 2 L n (n + nrhs)
 *   doubles is allocated stream-ordered.
 */
int dgetrs_dd(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv, double *B,
              int64_t ldb, void *stream);
int dgetrs_td(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv, double *B,
              int64_t ldb, void *stream);
int dgetrs_qd(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv, double *B,
              int64_t ldb, void *stream);

/*
 * zgetrs_{dd,td,qd}: solve with the factors of zgetrf (Sec. 4: "forward and
 * backward substitutions").
 *   trans 'N': A X = B  (apply P, unit-lower forward, upper back substitution)
 *         'C': A^H X = B (U^H forward, unit L^H back substitution, then P^T)
 *   n, nrhs  >= 0
 *   A, lda, ipiv  as returned by zgetrf (device, read only)
 *   B     device, n x nrhs planes with leading dimension ldb (plane stride
 *         ldb*nrhs); overwritten by X
 */
int zgetrs_dd(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv, double *B,
              int64_t ldb, void *stream);
int zgetrs_td(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv, double *B,
              int64_t ldb, void *stream);
int zgetrs_qd(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv, double *B,
              int64_t ldb, void *stream);

/*
 * zgemm_{dd,td,qd}: complex multi-component matrix product (Sec. 2.1,
 * Eq. (1) for 4M and Eq. (3) for 3M; Sec. 2.3 for the Ozaki scheme).
 *   beta_mode 0: C = A B;  1: C = C - A B (the trailing-update form)
 *   method    MCLU_METHOD_4M, MCLU_METHOD_3M or MCLU_METHOD_OZAKI
 *   A  m x k planes (lda, plane stride lda*k);  B  k x n planes (ldb, ldb*n);
 *   C  m x n planes (ldc, ldc*n); all device.  C must not alias A or B.
 */
int zgemm_dd(int beta_mode, int method, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
             const double *B, int64_t ldb, double *C, int64_t ldc, void *stream);
int zgemm_td(int beta_mode, int method, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
             const double *B, int64_t ldb, double *C, int64_t ldc, void *stream);
int zgemm_qd(int beta_mode, int method, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
             const double *B, int64_t ldb, double *C, int64_t ldc, void *stream);

/*
 * zgemm_{dd,td,qd}_ex: zgemm_* with the number of Ozaki slices (Sec. 2.3:
 * the number of divisions of each operand, which sets the accuracy of the
 * Ozaki-scheme product).
 *   ozaki_slices  MCLU_METHOD_OZAKI: 1..S slices kept per operand (S = 16
 *                 DD, 24 TD, 32 QD), the digit pairs p + q <= ozaki_slices - 1
 *                 multiplied; 0 = S; above S: MCLU_ERR_UNSUPPORTED.  Ignored
 *                 by the other methods.
 *   the other arguments as in zgemm_* (argument errors are reported by
 *   their position in this signature).
 */
int zgemm_dd_ex(int beta_mode, int method, int ozaki_slices, int64_t m, int64_t n, int64_t k, const double *A,
                int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, void *stream);
int zgemm_td_ex(int beta_mode, int method, int ozaki_slices, int64_t m, int64_t n, int64_t k, const double *A,
                int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, void *stream);
int zgemm_qd_ex(int beta_mode, int method, int ozaki_slices, int64_t m, int64_t n, int64_t k, const double *A,
                int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, void *stream);

/*
 * zadjoint_rank1_{dd,td,qd}: Abar = -lambda x^H, the matrix part of the
 * adjoint of x = A^{-1} b (for lambda = A^{-H} xbar, computed by
 * zgetrs_*('C', ...); the right-hand-side part is bbar = lambda).
 *   lambda, x  device n x 1 planes (plane stride n)
 *   Abar       device n x n planes, leading dimension ldab (plane stride ldab*n)
 */
int zadjoint_rank1_dd(int64_t n, const double *lambda, const double *x, double *Abar, int64_t ldab, void *stream);
int zadjoint_rank1_td(int64_t n, const double *lambda, const double *x, double *Abar, int64_t ldab, void *stream);
int zadjoint_rank1_qd(int64_t n, const double *lambda, const double *x, double *Abar, int64_t ldab, void *stream);

/*
 * zozaki_split_{dd,td,qd}: the slicing step of the Ozaki-scheme product
 * (Sec. 2.3: split into slices whose products are exact), exposed for
 * inspection.  X: device rows x cols planes (leading dimension ld).
 *   side 0 (left operand A, one scale per row): slices = bf16
 *          [ceil(cols/32)][S][Mpad][64], Mpad = rows rounded up to 128; element
 *          (i, c) has its real digits at [c/32][p][i][c%32] and imaginary
 *          digits at [c/32][p][i][32 + c%32]; E int32[rows].
 *   side 1 (right operand B, one scale per column): slices = bf16
 *          [ceil(rows/32)][S][Npad][64], Npad = 2 cols rounded up to N
 *          (N = 32 DD, 16 TD/QD); element (r, j): row 2j holds [Re | -Im] and
 *          row 2j+1 [Im | Re] at K index r%32 | 32 + r%32; E int32[cols].
 * Digit p of x is a_p with x ~ 2^E sum_p a_p 2^(-beta (p+1)), beta = 7
 * and S = 16, 24, 32 for DD, TD, QD.  slices and E are caller-owned device
 * buffers of those sizes.
 */
int zozaki_split_dd(int side, int64_t rows, int64_t cols, const double *X, int64_t ld, void *slices, int32_t *E,
                    void *stream);
int zozaki_split_td(int side, int64_t rows, int64_t cols, const double *X, int64_t ld, void *slices, int32_t *E,
                    void *stream);
int zozaki_split_qd(int side, int64_t rows, int64_t cols, const double *X, int64_t ld, void *slices, int32_t *E,
                    void *stream);

/*
 * mclu_vec_op: elementwise multi-component arithmetic on device vectors (the
 * complex DD/TD/QD operations of Sec. 2.1-2.2: add, sub, mul, div, inv).
 *   L      2, 3 or 4
 *   op     real ops on limb-major arrays [L][count]:
 *            0 add, 1 sub, 2 mul, 3 div
 *          complex ops on plane arrays [2][L][count]:
 *            10 add, 11 sub, 12 mul (4M, Eq. 1), 13 mul (3M, Eq. 2),
 *            14 div, 15 inv (reciprocal), 16 cabs1 (result in the real part),
 *            17 inv by Newton's method from a binary64 seed (the panel's
 *            pivot reciprocal)
 *   x, y   device inputs (y ignored by 15, 16, 17); z device output
 */
int mclu_vec_op(int op, int L, int64_t count, const double *x, const double *y, double *z, void *stream);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices); a diagnostic for counting launches in a timed region. */
uint64_t mclu_launch_count(void);

/*
 * Launch-class timing (diagnostic).  mclu_profile_begin(mask) makes every
 * later call bracket its launches of the classes in `mask` (bit k = class k:
 * 0 panel factorisation, 1 row swaps, 2 TRSM, 3 trailing-update / ZGEMM,
 * 4 getrs, 5 other) with CUDA events recorded on the call's stream.
 * mclu_profile_end synchronises those events and writes, for k < nkinds, the
 * summed milliseconds ms[k] and the number of bracketed calls launches[k]
 * (host arrays, either may be NULL), then stops recording.  Returns 0 or a
 * CUDA error code.
 */
int mclu_profile_begin(uint32_t kind_mask);
int mclu_profile_end(double *ms, int64_t *launches, int nkinds);

/* Static description of a status code. */
const char *mclu_status_string(int status);

/* Library version as "major.minor.patch". */
const char *mclu_version(void);

/*
 * mclu_probe_fp64_rate: measures the current device's FP64 throughput (a
 * diagnostic for rooflines): 4 CTAs of 256 threads per SM, each thread 8
 * independent chains of 40000 fused multiply-adds, timed with CUDA events on
 * a stream of its own after a warm-up launch.  Writes to *ops_per_second
 * (host) the FP64 instructions per second, one DFMA counted as one operation
 * (the unit in which the library's kernels are costed: DADD, DMUL and DFMA
 * are one operation each).  Allocates and frees 8 bytes of device memory and
 * synchronises its stream (about 0.1 s on GB300).  Returns 0, -1 for a NULL
 * pointer, or a CUDA error code.
 */
int mclu_probe_fp64_rate(double *ops_per_second);

/*
 * mclu_selftest_wait_timeout: runs, on the current device, the bounded wait
 * that the cooperative panel kernels use between CTAs (a clock64 budget of
 * about one second) on a device flag that nothing sets, and writes to
 * *status (host) the status word the kernel left: 1 when the wait ran out
 * and the kernel recorded it and returned (what the panels then report
 * through info < 0), 0 otherwise.  Nothing faults or hangs; the context
 * stays usable.  Allocates and frees 8 bytes of device memory and
 * synchronises the device.  Returns 0, -1 for a NULL status, or a CUDA
 * error code.
 */
int mclu_selftest_wait_timeout(int32_t *status);

#ifdef __cplusplus
}
#endif

#endif /* MCLU_H */
