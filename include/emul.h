/*
 * emul.h -- C ABI of the GB300 (sm_103a) library for FP64 matrix products
 * emulated by split-integer arithmetic, used as the trailing-matrix update of
 * blocked LU (partial pivoting) and Cholesky factorizations.
 *
 * Method: arXiv 2509.23565, "Performance and Numerical Aspects of
 * Decompositional Factorizations with FP64 Floating-Point Emulation in INT8".
 *   Section 2, Eq. 1-2: split each FP64 operand into s INT8 pieces and sum the
 *     piece products, dropping those with i+j > t (threshold t = s+1 here).
 *   Section 2, Eq. 3-4: split pieces carry no exponent; each row of A and each
 *     column of B gets its own power-of-two scale.
 *   Section 4, Eq. 5-7: blocked LU; all third-order work is the Schur
 *     complement A22 <- A22 - L21 U12, computed by the emulated product.
 *   Section 4, Eq. 8: scaled residual, below 16 for a valid solve.
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major (LAPACK) with a leading dimension ld >= rows.
 *   - Matrix / vector pointers are DEVICE pointers owned by the caller.  The
 *     library owns only its workspace, held by the handle.
 *   - Work is enqueued on the handle's stream; calls return before the GPU is
 *     done unless stated.  Device faults surface at the caller's next sync.
 *   - ipiv is 1-based int32 on the device (LAPACK semantics).  info is int32
 *     on the device: 0 = success, k > 0 = zero pivot / non-SPD leading minor
 *     at 1-based index k.
 *   - `slices` is s, the number of signed 7-bit INT8 slices per operand
 *     (3..8; emul_dgetrf also accepts 0: chosen per step by the selector).  The slice products run on tcgen05 tensor cores as integer-valued
 *     BF16 with FP32 accumulation that is kept exact (|partial sums| < 2^24).
 *   - Return value: EMUL_OK or a negative status below.  On an error,
 *     emul_last_error(h) gives a one-line reason.  Nothing is enqueued when
 *     argument checking fails.
 */
#ifndef EMUL_H_
#define EMUL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMUL_OK 0
#define EMUL_INVALID_ARG (-1)    /* a size, pointer, ld or slice count is invalid */
#define EMUL_CUDA_ERROR (-2)     /* a CUDA runtime / driver call failed */
#define EMUL_NO_WORKSPACE (-3)   /* the workspace could not be allocated */
#define EMUL_TIMEOUT (-4)        /* a device-side wait gave up (kernel returned early) */
#define EMUL_NOT_SUPPORTED (-5)  /* this GPU / configuration is not supported */

typedef struct emul_handle_s* emul_handle_t;

/* Create a handle bound to `stream` (a cudaStream_t; NULL = the legacy default
 * stream) on the current device.  Requires compute capability 10.3. */
int emul_create(emul_handle_t* handle, void* stream);
/* Free the handle and its workspace (synchronises its stream first). */
int emul_destroy(emul_handle_t handle);
/* Re-bind the handle to another cudaStream_t. */
int emul_set_stream(emul_handle_t handle, void* stream);
/* One-line description of the last error on this handle ("" if none). */
const char* emul_last_error(emul_handle_t handle);
/* Synchronise the handle's stream and read the device status word: EMUL_OK,
 * or EMUL_TIMEOUT if any kernel since the last call gave up on a wait.  Clears it. */
int emul_sync_status(emul_handle_t handle);
/* Bytes of device workspace currently held by the handle. */
size_t emul_workspace_bytes(emul_handle_t handle);

/* Host-only introspection of the product kernel's schedule (the order in
 * which the level sums I_L of Sec. 2 are accumulated; the paper fixes only
 * their values, not this order): the sweeps and the TMEM slot plan the kernel
 * would use for `slices` slices and inner dimension k.  wide = 1 selects the
 * 64-column variant, level_sums = 1 the emul_level_sums mode; threshold is
 * the last level kept (0: slices + 1; else 2..2*slices).  Needs no GPU.
 *   sweeps     out, cap_sweeps rows of EMUL_SWEEP_INTS ints:
 *              k0c, k1c (K chunks of 32), L[2], pb[2], pe[2], flags[2],
 *              nplanes, kcs (L[1] = 0: one job; flags: 1 final, the job
 *              whose term completes the exact sum that is rounded)
 *   table      out, cap_table bytes: slot (bits 0-1) and barrier parity
 *              (bit 2) of job j in tile phase ph at ph * njobs + j
 *   meta       out, 5 ints: nsweeps, njobs, t0, period, table bytes
 * Returns EMUL_OK, EMUL_INVALID_ARG (no schedule for these arguments, or a
 * capacity too small; meta is still filled when a schedule exists). */
#define EMUL_SWEEP_INTS 12
int emul_schedule(int slices, int k, int wide, int level_sums, int threshold, int* sweeps, int cap_sweeps,
                  unsigned char* table, int cap_table, int* meta);

/* ---------------------------------------------------------------- steps --
 * Exposed individually so each step of the method can be checked bit for bit.
 */

/* Scale extraction and slicing of a GEMM operand (Section 2, Eq. 1-4).
 * The operand is `rows` x `k`: element (r, c) at X[r*rs + c*cs] with either
 * rs == 1 (rows contiguous, e.g. A in column-major: rs=1, cs=lda) or cs == 1
 * (k contiguous, e.g. the columns of B: rs=ldb, cs=1).
 *   exps[r] (int32, device): smallest e with max_c |x(r,c)| < 2^e; 0 for an
 *     all-zero row; 2147483647 if the row holds Inf or NaN.
 *   slices (device, bf16 bit patterns): plane p (0-based, most significant
 *     first) at slices[(p*rows + r)*ldk + c] holds the integer
 *     sign(x) * ((|N| >> 7(s-1-p)) & 127) with N = trunc(x * 2^(7s - e_r)).
 *   ldk >= k and ldk % 8 == 0.
 */
int emul_split(emul_handle_t h, int rows, int k, const double* X, long rs, long cs, int slices, int32_t* exps,
               uint16_t* slice_out, long ldk);

/* Level sums of the slice-pair products (Section 2, Eq. 2 with t = s+1):
 *   levels[(L-2)*ldl_plane + i + j*ldl] = sum_{p+q=L} sum_k SA_p(i,k) SB_q(j,k)
 * for L = 2..s+1, as exact int32, computed on the tensor cores from the slices
 * of A (m x k, lda) by rows and of B (k x n, ldb) by columns. */
int emul_level_sums(emul_handle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                    int slices, int32_t* levels, int ldl, long ldl_plane);

/* ---------------------------------------------------------------- BLAS --
 * C <- beta*C + alpha*(A B), A m x k (lda), B k x n (ldb), C m x n (ldc).
 * The kept slice-pair products are summed exactly and rounded once to FP64,
 * D = RN(sum), then C = RN(RN(alpha*D) + RN(beta*C)) (beta == 0: C is not read).
 * For alpha = -1, beta = 1 this is the Schur update of Eq. 7, C = RN(C - D).
 */
int emul_dgemm(emul_handle_t h, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
               int ldb, double beta, double* C, int ldc, int slices);

/* emul_dgemm with the truncation threshold as a parameter (Section 2, Eq. 2:
 * the slice pairs kept are those with p + q <= t).  threshold = 0 is the
 * method's t = s + 1 (identical to emul_dgemm); 2 <= threshold <= 2s keeps the
 * levels L = 2..threshold, threshold = 2s being the full s^2-pair product.
 * The result is D = RN(sum_{L<=t} I_L 2^(e + f - 7L)), exact sum, one rounding.
 * Returns EMUL_INVALID_ARG for a threshold outside that range and
 * EMUL_NOT_SUPPORTED when k is too large for the 128-bit exact sum at this
 * threshold (sum_L n_L 127^2 2^(7(t-L)) k >= 2^126). */
int emul_dgemm_threshold(emul_handle_t h, int m, int n, int k, double alpha, const double* A, int lda,
                         const double* B, int ldb, double beta, double* C, int ldc, int slices, int threshold);

/* emul_dgemm with unequal slice counts: slices_a slices of A and slices_b of B
 * (the paper's related work, Sec. 3, cites unequal split sizes among the
 * accuracy extensions of the method without defining them; this is the plain
 * reading).  Both operands are split with s = max(slices_a, slices_b) slices,
 * whose leading slices are exactly those of a shorter split, and only the
 * pairs p <= slices_a, q <= slices_b with p + q <= threshold are kept
 * (threshold = 0: s + 1; else 2..slices_a + slices_b; at slices_a + slices_b
 * the kept sum is the exact product of the operands truncated to 7 slices_a
 * and 7 slices_b bits).  Exact sum, one rounding, C update as emul_dgemm;
 * slices_a = slices_b = s is emul_dgemm_threshold.  Returns EMUL_INVALID_ARG
 * for counts outside 1..8 or a threshold outside that range. */
int emul_dgemm_unequal(emul_handle_t h, int m, int n, int k, double alpha, const double* A, int lda,
                       const double* B, int ldb, double beta, double* C, int ldc, int slices_a, int slices_b,
                       int threshold);

/* ------------------------------------------------------- factorizations --
 * Optional statistics of a factorization call (host memory, may be NULL).
 */
typedef struct emul_stats {
  int steps;          /* block steps taken */
  int slices_min;     /* smallest slice count used by a trailing update */
  int slices_max;     /* largest slice count used by a trailing update */
  int checks_failed;  /* a-posteriori checks that triggered a recomputation */
  double seconds;     /* host wall time of the call (set only when it synchronises) */
  double slices_mean; /* mean slice count over the trailing updates */
} emul_stats;

/* LU with partial pivoting of the n x n matrix A (lda), in place (Section 4,
 * Eq. 5-7): right-looking, block size nb (16..512, multiple of 16; 0 = default
 * 128; EMUL_NB_AUTO = tuned by emul_autotune_nb).  The panel is factored in FP64 (pivot search, swaps, scaling; a panel
 * wider than 256 columns as two halves, the right half updated through the
 * emulated product); the triangular solve for U12 and the trailing update use
 * the emulated product with `slices` slices.  ipiv: n int32 (device); info: 1
 * int32 (device). */
int emul_dgetrf(emul_handle_t h, int n, double* A, int lda, int32_t* ipiv, int nb, int slices, int32_t* info,
                emul_stats* stats);

/* Block-size tuner of emul_dgetrf (kind 0) and emul_dpotrf (kind 1), which
 * the large factorizations use with nb autotuned in {128, 256, 512}: one
 * factorization of a synthetic n x n matrix (seeded uniform(-1, 1) entries;
 * for kind 1 symmetric with diagonal n, hence positive definite) is timed at
 * each candidate with CUDA events on the handle's stream, after one untimed
 * run, and the fastest is written to *nb_out and kept in the handle for
 * (kind, n, slices).  nb = EMUL_NB_AUTO in emul_dgetrf / emul_dpotrf takes
 * the kept value, running this tuner first when there is none.  Allocates
 * n^2 doubles of device memory for the duration of the call (besides the
 * factorization's workspace); slices 1..8.  Synchronises the stream. */
#define EMUL_NB_AUTO (-1)
int emul_autotune_nb(emul_handle_t h, int kind, int n, int slices, int* nb_out);

/* LU without pivoting of the n x n matrix A (lda), in place, A = L U (L unit
 * lower, U upper): the Level-3-only factorization timed for blocking factors
 * 256 to 2048 (Section 8), right-looking with block size nb (16..4096; 0 =
 * 1024).  Every third-order step runs through the emulated product with
 * `slices` slices: the Schur update A22 <- A22 - L21 U12 (Eq. 7), and the
 * triangular solves through explicit inverses of the diagonal blocks (a
 * panel is halved recursively down to blocks of at most 64 columns, factored
 * in FP64).  No rows are exchanged, so the result is only as stable as
 * Gaussian elimination without pivoting on A (diagonally dominant or SPD
 * matrices need none).  A zero pivot sets *info to its 1-based index (the
 * first one) and leaves its column unscaled; the later entries are then not
 * meaningful.  info: 1 int32 (device).  emul_dgetrs solves with these factors
 * given ipiv[i] = i + 1. */
int emul_dgetrf_nopiv(emul_handle_t h, int n, double* A, int lda, int nb, int slices, int32_t* info,
                      emul_stats* stats);

/* Solve A X = B with the factors from emul_dgetrf (Section 4, Eq. 5: the
 * solution of A x = b through the triangular factors of the 2 x 2 blocked
 * partition of Eq. 6): the row interchanges, then forward substitution with
 * unit L and back substitution with U, in FP64.  B (n x nrhs, ldb) is
 * overwritten by X. */
int emul_dgetrs(emul_handle_t h, int n, int nrhs, const double* LU, int lda, const int32_t* ipiv, double* B,
                int ldb);

/* Lower Cholesky A = L L^T of the symmetric positive definite n x n matrix A
 * (lda), in place; only the lower triangle is read and written.  Section 4
 * notes that the method applies to symmetric positive definite matrices as
 * well: the Schur complement of Eq. 7 becomes A22 - L21 L21^T.  Block size
 * nb (16..512, multiple of 16; 0 = default 128; EMUL_NB_AUTO = tuned by
 * emul_autotune_nb).  Diagonal blocks in FP64;
 * L21 = A21 L11^-T and the trailing update (lower tiles only) use the
 * emulated product.  uplo must be 'L'. */
int emul_dpotrf(emul_handle_t h, char uplo, int n, double* A, int lda, int nb, int slices, int32_t* info,
                emul_stats* stats);

/* Solve A X = B from emul_dpotrf's factor (Section 4, Eq. 5, with A = L L^T):
 * forward substitution with L, back substitution with L^T, in FP64.  B (n x
 * nrhs, ldb) is overwritten by X. */
int emul_dpotrs(emul_handle_t h, char uplo, int n, int nrhs, const double* L, int lda, double* B, int ldb);

/* Residual measures of the solve (Section 4, Eq. 8), computed in FP64 on the
 * device.  out (device, 2 doubles):
 *   out[0] = ||Ax-b||_inf / ((||A||_inf ||x||_inf + ||b||_inf) n eps)   (Eq. 8)
 *   out[1] = ||Ax-b||_inf / (||A||_inf ||x||_inf n eps)
 * with eps = 2^-53. */
int emul_backward_error(emul_handle_t h, int n, const double* A, int lda, const double* x, const double* b,
                        double* out);

/* ------------------------------------------------------ batched solves --
 * Many independent systems A_i x_i = b_i of uneven sizes (1..4096) in one
 * persistent launch recorded in a CUDA graph: each block
 * takes whole systems from a work queue (largest first) and factors them in
 * reduced precision -- FP32 panel with partial pivoting, trailing updates by
 * the split-integer product (Sec. 2, Eq. 2) with `slices` INT8 slices as exact
 * INT8 x INT8 -> INT32 tensor-core products recombined in FP64 -- then refines
 * in FP64 (residual
 * b - A x with the original A) until the backward error
 * ||b - A x|| / (||A|| ||x|| n 2^-53) is at most 1 or max_iter is reached.
 * A system whose refinement has not converged after 8 steps is refactored
 * with 8 slices (the per-row scales of few slices drop entries far below
 * their row's largest, the range effect of Sec. 2, Eq. 3), then refined on.
 *   count        number of systems
 *   n_arr, lda_arr, A_arr, b_arr   HOST arrays: sizes, leading dimensions,
 *                device pointers of A_i (n_i x n_i, column-major, not modified)
 *                and of b_i (overwritten by x_i)
 *   info_arr, berr_arr, iters_arr  DEVICE arrays of count entries: zero pivot
 *                index of the FP32 factorization (0 = none), final backward
 *                error, refinement iterations
 *   slices       2..8 (first factorization), or 0 = per size bucket from the autotuned table
 *   nb           16, 32, 64, or 0 = autotuned
 * The workspace holds one FP32 copy of the largest system per SM. */
int emul_dgesv_batched_ir(emul_handle_t h, int count, const int* n_arr, double* const* A_arr, const int* lda_arr,
                          double* const* b_arr, int32_t* info_arr, double* berr_arr, int32_t* iters_arr, int max_iter,
                          int slices, int nb);
/* Autotuner of the batched solver: for each size bucket [0,128), [128,256),
 * [256,512), [512,4096] time every (nb, slices) in {16,32,64} x {3,4} on
 * synthetic systems and keep the fastest whose refinement passes; the table is
 * read from `cache_path` (JSON lines) if it exists, else tuned and written
 * there (NULL: tune, do not cache). */
int emul_autotune(emul_handle_t h, const char* cache_path);

/* ------------------------------------------------------ slice selector --
 * A small MLP predicts, per trailing update, the fewest slices that keep the
 * update within FP64 accuracy (the paper's Sec. 3 cites
 * a-posteriori validation of error-free products, which the check below
 * follows).  Features (64 floats): 32-bin histograms of each entry's exponent
 * offset from its row scale (A) and from its column scale (B), each divided
 * by its entry count; offsets >= 31 and zeros fall in bin 31.  Network:
 * 64 -> 128 -> 128 -> 128 -> 6 (ReLU; classes s = 3..8), BF16 weights for the
 * products, FP32 master weights, FP32 accumulation, softmax cross-entropy,
 * AdamW.  Parameters are one flat FP32 array of EMUL_SELECTOR_PARAMS values:
 * W0[128][64], b0[128], W1[128][128], b1[128], W2[128][128], b2[128], W3[6][128], b3[6].
 * emul_dgetrf with slices = 0 uses the loaded network per step and checks
 * each update with a Freivalds probe on sampled rows; an update that fails
 * the probe is redone with 8 slices (counted in emul_stats.checks_failed).
 */
#define EMUL_SELECTOR_FEATURES 64
#define EMUL_SELECTOR_CLASSES 6
#define EMUL_SELECTOR_PARAMS 42118

/* Features of the product block A (m x k, lda) times B (k x n, ldb); feat: 64 floats (device). */
int emul_selector_features(emul_handle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                           float* feat);
/* Training labels: err[s-3] = max_ij |D_s - D_8|_ij / (4 k 2^-53 (|A||B|)_ij) for s = 3..8 (device,
 * 6 doubles), D_s the emulated product with s slices, all from one INT32 level-sum pass. */
int emul_slice_errors(emul_handle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                      double* err);
/* Parameters from / to host memory (EMUL_SELECTOR_PARAMS floats); setting resets the optimizer state. */
int emul_selector_set_params(emul_handle_t h, const float* params);
int emul_selector_get_params(emul_handle_t h, float* params);
/* Gradients of the mean cross-entropy (device, EMUL_SELECTOR_PARAMS floats) and the loss (device, 1 float)
 * for a batch (<= 8192) of features X (batch x 64, row-major, device) and labels in 3..8 (device). */
int emul_selector_grad(emul_handle_t h, int batch, const float* X, const int32_t* labels, float* grad, float* loss);
/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch; loss (device, may be NULL). */
int emul_selector_train_step(emul_handle_t h, int batch, const float* X, const int32_t* labels, float lr,
                             float weight_decay, float* loss);
/* Predicted slice counts (3..8) for a batch of features (device in, device out). */
int emul_selector_predict(emul_handle_t h, int batch, const float* X, int32_t* slices);
/* Weight file: "SEL1", count, then the flat parameters (little-endian FP32). */
int emul_selector_save(emul_handle_t h, const char* path);
int emul_selector_load(emul_handle_t h, const char* path);

/* -------------------------------------------------------- no allocation --
 * emul_dgemm without any device allocation, for callers that cannot call
 * cudaMalloc: a host library whose device memory is owned by another
 * allocator (a framework's caching allocator, a memory pool sized at
 * start-up), or a latency-bound loop that must not call cudaMalloc or
 * cudaFree because either can synchronise the whole device.  The paper has no
 * counterpart to this entry point.
 *
 * Same arguments and results as emul_dgemm, but on `stream` (a cudaStream_t)
 * instead of a handle.  The scratch (slices, scales, schedule, status word)
 * lives in one 16 MiB static device array that every GPU which loads this
 * library holds until the process exits.  Limit: with kp = k rounded up to a
 * multiple of 8, 2 * slices * kp * (m + n) + 4 * (m + n) + about 17 KB must
 * fit in 16 MiB, else the call returns EMUL_NO_WORKSPACE and enqueues
 * nothing.  The first call on a device sets up that device (it looks up the
 * device address of the array); make that first call before any stream
 * capture.  Every call reuses the same array and keeps the previous call's
 * contents: calls that overlap on the GPU (other streams, other threads)
 * race and give unspecified results.  A device-side wait that gives up is
 * not reported by this entry point (C is then unspecified).
 */
int emul_dgemm_noalloc(void* stream, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                       int ldb, double beta, double* C, int ldc, int slices);

/* ------------------------------------------------------------ profiling --
 * Counters of the work this handle enqueued, for benchmarks (no paper
 * counterpart).  While enabled, every launch of the slice-pair product kernel
 * is bracketed by CUDA events on the handle's stream.
 */
typedef struct emul_profile {
  long long kernel_launches;    /* kernels launched by this handle since the last read */
  long long product_launches;   /* launches of the slice-pair product kernel */
  double product_ms;            /* their summed device time (CUDA events) */
  double product_tensor_flops;  /* sum of 2 m n k P, P the slice pairs kept: sum over the levels
                                   L = 2..t of their pairs (s(s+1)/2 at the default t = s + 1) */
  double product_bytes;         /* algorithmic bytes: C read + write (8 B each) and the slices read */
  double phase_ms[5];           /* device time of the factorization phases (CUDA events around each),
                                   indexed by EMUL_PHASE_* */
} emul_profile;

/* Phases of emul_dgetrf / emul_dgetrs timed when profiling is enabled:
 * PANEL  the panel factorization (leaves, inner products, small solves),
 * SWAP   the panel's row interchanges applied to the columns outside it,
 * U12    L11^-1 and U12 = L11^-1 A12,
 * UPDATE the trailing update A22 - L21 U12 (slicing, product, selector probe),
 * SOLVE  emul_dgetrs.
 * emul_dpotrf / emul_dpotrs use the same slots: PANEL the diagonal block
 * (L11 and L11^-1), U12 the product L21 = A21 L11^-T, UPDATE the lower
 * trailing update A22 - L21 L21^T, SOLVE emul_dpotrs. */
#define EMUL_PHASE_PANEL 0
#define EMUL_PHASE_SWAP 1
#define EMUL_PHASE_U12 2
#define EMUL_PHASE_UPDATE 3
#define EMUL_PHASE_SOLVE 4

/* Enable (1) or disable (0) event timing of the product kernel and of the
 * factorization phases. */
int emul_profile_enable(emul_handle_t h, int enable);
/* Synchronise the handle's stream, return the counters and reset them. */
int emul_profile_read(emul_handle_t h, emul_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* EMUL_H_ */
