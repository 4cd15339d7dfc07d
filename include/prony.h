/*
 * prony.h -- C ABI of the GB300 (sm_103a) multivariate matrix-pencil Prony library.
 *
 * Method: N. Bosner, "Parallel Prony's method with multivariate matrix pencil
 * approach and its numerical aspect", arXiv 2012.11430.  The problem (Section 1,
 * Eq. 1): given samples of the exponential sum
 *     f(k) = sum_{j=1}^m c_j exp(-2 pi i <t_j, k>),   k in Z^d,
 * recover the nodes t_j in [0,1)^d and the coefficients c_j != 0.  The library
 * runs Algorithm 1 with the block power method for the SVD (Algorithm 3) on
 * the GPU: Toeplitz products T V, T^* U (T = [f(k-h)], k,h in I_n={0..n}^d),
 * S_l = U^* T_l V Sigma^{-1} (Eq. generateSl), the joint diagonalisation of a
 * random combination C_mu (Eq. diagonalizeSl), t from the principal logarithm,
 * and c from the Vandermonde least-squares problem (Eq. ls_probl).
 *
 * Conventions for every call:
 *   - Sample grid: complex128 values on {-n..n+1}^d, (2n+2)^d entries, row-major
 *     (last coordinate fastest); point x is at linear index
 *     sum_l (x_l + n) (2n+2)^(d-1-l).  Every matrix entry the method needs,
 *     f(k-h) and f(k-h+e_l) for k,h in I_n, lies on this grid.
 *   - Host-pointer calls are synchronous; the library copies inputs to the
 *     device and results back.  `*_dev` calls take device pointers and a CUDA
 *     stream (cudaStream_t passed as void*) and return when the results are
 *     written (they synchronise that stream).
 *   - All buffers are owned by the caller.  The context owns its device
 *     workspace (grown on demand and reused), its stream and its caches.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Return value: a prony_status.  Per-problem outcomes are in prony_info.
 *     PRONY_ERANK (detected rank below m) still fills every output.
 *   - No call ever aborts the process, traps on the GPU or falls back to a CPU
 *     implementation; every device loop is bounded and reports PRONY_ENOCONV.
 */
#ifndef PRONY_H
#define PRONY_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } prony_c128;     /* interleaved complex128 */
typedef struct prony_ctx prony_ctx;

typedef enum {
  PRONY_OK = 0,
  PRONY_EINVAL = -1,    /* bad argument (sizes, NULL pointer, unsupported precision) */
  PRONY_ERANK = -2,     /* detected numerical rank of T is below m (outputs still filled) */
  PRONY_ENOCONV = -3,   /* an iteration hit its cap (power method, eigen-QR, Jacobi) */
  PRONY_ENAN = -4,      /* non-finite input samples or intermediate results */
  PRONY_ECUDA = -5,     /* CUDA runtime error (message: prony_last_error) */
  PRONY_ENOMEM = -6     /* device allocation failed */
} prony_status;

/* Arithmetic of the Toeplitz block products (the small steps are FP64 always).
 *   PRONY_FP32   : complex64 operands, FP32 FMA on the CUDA cores.
 *   PRONY_BF16X3 : FP32 operands split into three BF16 parts, six tensor-core
 *                  products (tcgen05.mma kind::f16), FP32 accumulation.
 *   PRONY_TF32X3 : FP32 operands split into TF32 hi+lo, three tensor-core
 *                  products (tcgen05.mma kind::tf32), FP32 accumulation.
 *   PRONY_BF16X2 : BF16 hi+lo split, three tensor-core products.
 *   PRONY_FFT32  : no dense product: T embedded in a circulant of L^d points (L the power of
 *                  two >= 2n+2), FP32 FFTs in shared memory, O(L^d log L) per column instead
 *                  of O(N^2).  Needs d <= 3 and L^(d-1) (L+1) + L <= 128 * 130 for every
 *                  problem of the call (d = 1: n <= 4095; d = 2: n <= 63; d = 3: n <= 7), else
 *                  PRONY_EINVAL. */
typedef enum { PRONY_FP32 = 0, PRONY_BF16X3 = 1, PRONY_TF32X3 = 2, PRONY_BF16X2 = 3, PRONY_FFT32 = 4 } prony_precision;

typedef struct {
  int precision;            /* prony_precision */
  int oversample_p;         /* r0 = m + p columns in Algorithm 3; < 0: p = m (Section 5) */
  double tol_rank;          /* rank tolerance of the pivoted QR (Section 2.2); <= 0: default */
  double tol_power;         /* stop when ||R_k||_F <= tol_power ||T||_F (Algorithm 3); <= 0: default */
  int max_iter;             /* cap on power iterations; <= 0: default 30 */
  unsigned long long seed;  /* Philox4x64-10 key for mu, V_0 */
  int rank_mode;            /* 0: use the given m (rank detected and reported); 1: use the detected rank */
  int vandermonde;          /* matrix of the least-squares problem for c (Eq. ls_probl): 0 from t
                               (unit modulus, default); 1 from the raw eigenvalues z~ (the matrix
                               the Section 4 perturbation analysis works with) */
  int svd_method;           /* subspace of T: 0 block power method (Algorithm 3, default);
                               1 Lanczos bidiagonalisation with full reorthogonalisation
                               (Algorithm 2) up to the rank it reveals, then the block power
                               iteration from its right vectors with the pivoted-QR rank step */
} prony_opts;

typedef struct {
  int status;               /* prony_status of this problem */
  int rank_detected;        /* rank from the pivoted QR of the first T^* U block (Section 2.2) */
  int rank_used;            /* number of terms returned (m, or the detected rank with rank_mode 1) */
  int power_iters;          /* iterations k of Algorithm 3 */
  double power_resid;       /* ||R_k||_F / ||T||_F at exit */
  double ls_resid;          /* ||A^T c - f||_2 / ||f||_2 (Section 5 accuracy estimate) */
  double sigma_ratio;       /* sigma_m / sigma_1 */
  double normT;             /* ||T||_F (closed form from the grid) */
  int lanczos_steps;        /* left vectors u accepted by Algorithm 2 (svd_method 1), else 0 */
} prony_info;

/* Fill *opts with defaults: PRONY_BF16X3, p = m, tolerances and cap as documented above. */
void prony_default_opts(prony_opts* opts);
const char* prony_status_string(int status);
/* Message of the last PRONY_ECUDA / PRONY_ENOMEM on this host thread. */
const char* prony_last_error(void);

/* Create a context on CUDA device `device` (its own non-blocking stream). */
int prony_ctx_create(prony_ctx** ctx, int device);
int prony_ctx_destroy(prony_ctx* ctx);

/* Algorithm 1 for one problem.  samples: (2n+2)^d grid (see above).  d >= 1,
 * n >= 1, 1 <= m <= (n+1)^d, m <= 64, d m (n+1) <= 6144 (the phase tables of the right-hand
 * side), (n+1)^d <= 2e8, else PRONY_EINVAL.  opts may be NULL (defaults).
 * Outputs: t_out[m*d] (row j = t_j, components in [0,1)), c_out[m]; the pairs
 * are sorted lexicographically by t.  info may be NULL. */
int prony_solve(prony_ctx* ctx, const prony_c128* samples, int d, int n, int m,
                const prony_opts* opts, double* t_out, prony_c128* c_out, prony_info* info);

/* Steps 1-3 of Algorithm 1: the d matrices S_l = U^* T_l V Sigma^{-1} (Eq. generateSl)
 * in the phase-canonical basis (each singular pair u_i, v_i multiplied by
 * e^{-i theta_i}, theta_i = arg of the largest-modulus entry of v_i, lowest
 * index on ties).  S_out[d*m*m]: S_l row-major at offset l*m*m.
 * sigma_out[m]: leading singular values, descending.  U_out, V_out (nullable):
 * N x m column-major singular vectors in the same basis. */
int prony_build_S(prony_ctx* ctx, const prony_c128* samples, int d, int n, int m,
                  const prony_opts* opts, prony_c128* S_out, double* sigma_out,
                  prony_c128* U_out, prony_c128* V_out, prony_info* info);

/* The FP64 steps of Algorithm 1 after the Toeplitz products, on caller-given matrices, for
 * checking them in isolation: the SVD Q = U_Q Sigma V_Q^* of the projected block
 * Q = U^* T V (final step of Algorithm 3), S_l = U_Q^* M_l V_Q Sigma^{-1} with M_l = U^* T_l V
 * (Eq. generateSl), the eigenvectors W of C_mu = sum_l mu_l S_l (mu drawn from `seed`, as in
 * prony_solve), z_j(l) = (W^{-1} S_l W)_jj and t_j(l) = -arg z_j(l) / 2 pi mod 1
 * (Eq. diagonalizeSl).  These are the kernels prony_solve runs after its power loop.
 * Q: a x m row-major, M: d blocks of a x m row-major (m <= a <= 128, m <= 64, d <= 4), host
 * pointers.  Outputs (host): sigma_out[m] descending; S_out[d*m*m] row-major per l in the
 * basis of the computed singular vectors (unique up to a phase per vector); z_out[m*d],
 * t_out[m*d] row j for eigenvector j (unsorted); status_out (nullable): PRONY_OK or
 * PRONY_ENOCONV if an iteration reached its cap.  jacobi_cap / eigqr_cap (<= 0: defaults, 30
 * one-sided Jacobi sweeps and 30 m + 30 shifted-QR steps) lower the caps of the FP32
 * iterations whose results the FP64 steps refine. */
int prony_small_steps(prony_ctx* ctx, int d, int m, int a, const prony_c128* Q, const prony_c128* M,
                      unsigned long long seed, int jacobi_cap, int eigqr_cap, double* sigma_out,
                      prony_c128* S_out, prony_c128* z_out, double* t_out, int* status_out);

/* Eq. 1 at K integer points: f_out[q] = sum_j c_j exp(-2 pi i <t_j, k_q>).
 * t[m*d] row-major, c[m], k[K*d] row-major.  Phases reduced in FP64. */
int prony_eval(prony_ctx* ctx, const double* t, const prony_c128* c, int m, int d,
               const int* k, int K, prony_c128* f_out);

/* Many independent problems of uneven (d, n, m); P >= 1 (an empty batch is PRONY_EINVAL), each
 * problem within the limits of prony_solve.
 * sample_off[p]: offset (in prony_c128) of problem p's grid inside `samples`;
 * out_off[p]: offset (in terms) of its results: t_out[(out_off[p]+j)*dmax + l] for
 * l < d[p] (dmax = the largest d of the call; entries l >= d[p] are left untouched),
 * c_out[out_off[p]+j].  infos[P] nullable.  Returns the worst status. */
int prony_solve_batched(prony_ctx* ctx, int P, const int* d, const int* n, const int* m,
                        const long long* sample_off, const prony_c128* samples,
                        const long long* out_off, double* t_out, prony_c128* c_out,
                        prony_info* infos, const prony_opts* opts);

/* Device-pointer twin of prony_solve_batched: samples, t_out, c_out are device
 * pointers; d, n, m, sample_off, out_off, infos are host arrays. */
int prony_solve_batched_dev(prony_ctx* ctx, int P, const int* d, const int* n, const int* m,
                            const long long* sample_off, const prony_c128* samples_dev,
                            const long long* out_off, double* t_out_dev, prony_c128* c_out_dev,
                            prony_info* infos, const prony_opts* opts, void* stream);

/* Exponential-sum forward on device data (single precision results, FP64 phases):
 * f[q] = sum_j c_j exp(-2 pi i <t_j, k_q>) for the integer points of the box
 * {lo_l .. lo_l + len_l - 1}, row-major.  t_dev: m*d float64, c_dev: m complex64
 * (float2), f_dev: prod(len) complex64.  (Section 1, Eq. 1.) */
int prony_expsum_fwd_dev(prony_ctx* ctx, const double* t_dev, const void* c_dev, int m, int d,
                         const int* lo, const int* len, void* f_dev, void* stream);

/* Vector-Jacobian product of the exponential sum over the same box: given
 * g = dL/dRe f + i dL/dIm f as complex64 (L real; for L = sum |f - y|^2,
 * g = 2 (f - y)), writes grad_t[m*d] (float64) = dL/dt and grad_c[m]
 * (complex64) = dL/dRe c + i dL/dIm c, i.e. grad_c = sum_k g_k conj(e_jk) and
 * grad_t = 2 pi sum_k k Im(conj(g_k) c_j e_jk) with e_jk = exp(-2 pi i <t_j, k>).
 * The exponentials are recomputed, not stored. */
int prony_expsum_bwd_dev(prony_ctx* ctx, const double* t_dev, const void* c_dev, int m, int d,
                         const int* lo, const int* len, const void* g_dev,
                         double* grad_t_dev, void* grad_c_dev, void* stream);

/* Least-squares refinement of an exponential sum on device data by damped Gauss-Newton
 * (Levenberg-Marquardt) steps, starting from (t, c) -- typically the Prony estimate:
 *   minimise L(t, c) = sum_k |sum_j c_j exp(-2 pi i <t_j, k>) - y_k|^2
 * over the integer points k of the box {lo_l .. lo_l + len_l - 1} (row-major).  The model is
 * Eq. (1) of Section 1; the paper fits only c by least squares (Eq. ls_probl), this also moves t.
 * t_dev: m*d float64 (in/out, kept in [0,1)), c_dev: m complex128 (in/out),
 * y_dev: prod(len) complex64 samples, loss_dev: iters+1 float64 or NULL (the loss before each
 * step and after the last).  Each step: one pass over the points for J^* J and J^* r (FP32 per
 * block, FP64 accumulators), one FP32 Cholesky solve of the Jacobi-scaled damped system
 * (Marquardt damping lambda, initial value lambda0 > 0), one trial pass; the step is taken if
 * the loss decreased (lambda / 3), else refused (lambda * 4).  All steps run as one CUDA graph,
 * captured on the first call with a given argument set and reused while the set repeats.
 * m * (d + 2) <= 160, else PRONY_EINVAL.  Runs on `stream` (NULL: the context stream) and
 * returns when the refined (t, c) are written. */
int prony_refine_lm_dev(prony_ctx* ctx, double* t_dev, prony_c128* c_dev, int m, int d,
                        const int* lo, const int* len, const void* y_dev, int iters,
                        double lambda0, double* loss_dev, void* stream);

/* The Toeplitz block product used by the power iterations, exposed for testing:
 * Y[k, j] = sum_{h in I_n} F(k - h) X[h, j] for k in the box {0..L-1}^d
 * (L = n+1: T X; L = n+2: the rows of T, T_1..T_d at once), where F = f
 * (adjoint = 0) or F(x) = conj f(-x) (adjoint = 1, i.e. T^* X).
 * grid_dev: (2n+2)^d complex128 samples; X_dev: N x r complex64 column-major
 * (N = (n+1)^d, leading dimension N); Y_dev: L^d x r complex64 column-major
 * (leading dimension L^d).  precision: prony_precision. */
int prony_toeplitz_mm_dev(prony_ctx* ctx, const prony_c128* grid_dev, int d, int n,
                          const void* X_dev, int r, int L, int adjoint, int precision,
                          void* Y_dev, void* stream);

/* Allocation-free variant of prony_toeplitz_mm_dev (FP32 path).  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library allocate
 * device memory -- programs whose device memory is fixed up front by their own
 * allocator or budget, and latency-critical loops where cudaMalloc/cudaFree may
 * synchronise the device.  It takes no context and calls no cudaMalloc, cudaFree or
 * other allocating routine: its scratch (problem descriptor, job list, complex64
 * copies of the grid) lives in one fixed file-scope device array of
 * PRONY_STATIC_SCRATCH_BYTES that every GPU loading the library holds until exit.
 * Arguments and validation as prony_toeplitz_mm_dev (r <= (n+1)^d); it runs on the current
 * device, is asynchronous on `stream` (results are ready when the stream reaches that point)
 * and returns PRONY_EINVAL (message: prony_last_error) when (2n+2)^d > PRONY_STATIC_MAX_GRID.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress).  The first call on each device also loads the library's module
 * there and reserves the PRONY_STATIC_SCRATCH_BYTES, which may synchronise: make it once as
 * a warm-up, outside latency-critical loops and before any stream capture.  All calls share
 * the array and each rewrites what it reads; calls that overlap on the GPU (e.g. on two
 * streams at once) race on it.  The product runs without a K split (one CTA per row tile). */
#define PRONY_STATIC_MAX_GRID (1 << 20)
#define PRONY_STATIC_SCRATCH_BYTES (512 + 65536 * 16 + 16 * PRONY_STATIC_MAX_GRID)   /* 17 MiB */
int prony_toeplitz_mm_static(const prony_c128* grid_dev, int d, int n, const void* X_dev, int r, int L,
                             int adjoint, void* Y_dev, void* stream);

/* Measurement support (not part of the method).  With profiling on, every Toeplitz
 * block product launched by the solver is bracketed by CUDA events on the context
 * stream; its algorithmic work is accumulated: flops = 8 * rows * N * width per live
 * problem (one complex multiply-add = 8 real flops), bytes = samples read
 * (8 (2n+2)^d) + X read (8 N width) + Y written (8 rows width) at complex64.
 * launches counts every kernel the library launched (all kernels, all contexts)
 * since the last reset. */
typedef struct {
  long long launches;        /* all library kernel launches since reset */
  long long toeplitz_launches;
  double toeplitz_ms;        /* summed CUDA-event durations of the Toeplitz launches */
  double toeplitz_flops;     /* summed algorithmic flops of those launches */
  double toeplitz_bytes;     /* summed algorithmic bytes of those launches */
  int tc_ksplit;             /* tensor-core path of the last batch: K split of its products, as
                                chosen by the autotuner (0: not used) */
  int tc_bstages;            /* and its B' stages in shared memory (0: not used) */
} prony_stats;

/* Tuning overrides of the tensor-core products, read from the environment at every call:
 *   PRONY_TC_BSTAGES=s   exactly s B' stages in shared memory (default: the most stages, from
 *                        4 down to 2, that reach the smallest K split whose windows fit)
 *   PRONY_TC_KSPLIT=k    a K split of at least k (no autotuning)
 *   PRONY_TC_TUNE=0      no autotuning: the smallest K split
 *   PRONY_TC_APPLY=0     the X M products of the tall blocks (CholeskyQR2, the final U and V) on
 *                        the FP32 CUDA cores instead of the tensor cores (three BF16 planes)
 * The first three change launch configurations only, never the arithmetic beyond FP32 summation
 * order; the fourth changes how the X M products are rounded (both are FP32-accurate).
 * For a given launch configuration every product is deterministic: split-K partial sums are
 * added in the order of their K ranges, whatever order the CTAs finish in. */
int prony_set_profiling(prony_ctx* ctx, int enable);   /* also resets the statistics */
int prony_get_stats(prony_ctx* ctx, prony_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* PRONY_H */
