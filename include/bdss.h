/*
 * bdss.h -- C ABI of the GB300 (sm_103a) block-tridiagonal SPD solver.
 *
 * Solves A X = B where A is symmetric positive definite and block-tridiagonal
 * (Eq. 1, Sec. 1): N diagonal blocks A_{i,i} of size n x n, N-1 sub-diagonal
 * blocks A_{i+1,i} (the block above the diagonal is A_{i+1,i}^T), and X, B of
 * size (N n) x d.  The method is the recursive Schur-complement reduction of
 * Sec. 3 (Eq. 2-5, Algorithms 1-7) with interior segments of length one,
 * i.e. odd-even block cyclic reduction: at every level the odd positions are
 * eliminated and the even positions are the separators of the next level.
 *
 * Data layout (all row-major, 0-based block indices, device memory unless a
 * parameter says "host"):
 *   A_diag : N x n x n doubles, A_diag[i] = A_{i,i}.  The operator reads
 *            sym(A_{i,i}) = (A_{i,i} + A_{i,i}^T) / 2.
 *   A_sub  : (N-1) x n x n doubles, A_sub[i] = A_{i+1,i}.  May be NULL iff N == 1.
 *   B, X   : N x n x d doubles, element (i, r, k) at ((i n + r) d + k).
 * Every pointer must be 16-byte aligned.
 *
 * Input location.  A_diag, A_sub and B may also be host memory that the GPU
 * can read: page-locked memory (cudaHostAlloc, cudaHostRegister) or, on a
 * system whose GPU reads pageable host memory (cudaDevAttrPageableMemoryAccess,
 * e.g. a coherent NVLink-C2C host link), any host memory.  The level-0
 * kernels then read the inputs in place, asking L2 for the next task's blocks
 * one task ahead, so that the transfer overlaps the factorisation; the FP64
 * path reads every input element once per bdss_factor_solve.  The mixed modes
 * read A again for every refinement residual, where device copies are
 * faster.  X must be device (or managed) memory.  A pointer the GPU cannot
 * read is rejected with BDSS_ERR_INVALID_ARG before any launch.
 *
 * Ownership.  The caller owns every input and output buffer; the library never
 * frees them.  A handle owns its workspace (factors of every level, the
 * level coupling blocks, a status word).  In the mixed-precision modes the
 * handle also remembers the A_diag / A_sub pointers given to bdss_factor and
 * reads them again in bdss_solve to form the FP64 residual: the caller must
 * keep them valid and unmodified until the next bdss_factor or bdss_destroy.
 *
 * Streams.  All work is enqueued on the CUDA stream given to bdss_create
 * (NULL = legacy default stream).  Each call that launches work synchronises
 * that stream before it returns, in order to read the device status word.
 *
 * Errors.  Functions return a bdss_status; they never abort or print.
 * Arguments are checked on the host before anything is launched.
 * Device-side failures (a non-positive or non-finite Cholesky pivot; a grid
 * barrier wait that exceeded its time limit) are reported through the status
 * word and leave the device usable.
 */
#ifndef BDSS_H
#define BDSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdss_ctx *bdss_handle;

typedef enum {
  BDSS_OK = 0,
  BDSS_ERR_INVALID_ARG = 1,     /* bad size, NULL or misaligned pointer, d > d_max, ... */
  BDSS_ERR_NOT_SPD = 2,         /* a Cholesky pivot was <= 0 or not finite; see bdss_info */
  BDSS_ERR_NOT_FACTORED = 3,    /* bdss_solve / bdss_logdet before a successful bdss_factor */
  BDSS_ERR_ALLOC = 4,           /* device or pinned-host allocation failed */
  BDSS_ERR_CUDA = 5,            /* a CUDA runtime call failed */
  BDSS_ERR_TIMEOUT = 6,         /* a device-side wait exceeded its time limit */
  BDSS_ERR_NO_CONVERGENCE = 7,  /* mixed precision: refinement did not reach the target */
  BDSS_ERR_UNSUPPORTED = 8,     /* a size or mode this build does not implement */
  BDSS_ERR_GUARD = 9            /* debug: a workspace guard band was overwritten */
} bdss_status;

typedef enum {
  BDSS_FP64 = 0,     /* every step in FP64 (DFMA) */
  BDSS_FP32_IR = 1,  /* factor/solve in FP32, FP64 residual + iterative refinement */
  BDSS_TF32_IR = 2   /* as FP32_IR; for 64 < n <= 256 (n % 4 == 0) the Schur-update
                        products run on tcgen05 tensor cores (3xTF32 split, FP32
                        accumulation); for n <= 64 it equals BDSS_FP32_IR */
} bdss_precision;

typedef struct {
  int64_t level;        /* NOT_SPD: reduction level of the failing pivot (-1: none) */
  int64_t block;        /* NOT_SPD: original 0-based block index of that pivot */
  int32_t iters;        /* mixed precision: refinement steps taken, plain corrections
                           plus CG iterations (0 in FP64) */
  int32_t reserved;
  double backward_err;  /* mixed precision: ||B-AX||_inf / (||A||_inf ||X||_inf) of
                           the returned X, FP64 residual; -1 when not computed */
} bdss_info;

/* Options for bdss_set_option. */
typedef enum {
  BDSS_OPT_TIMEOUT_MS = 0,      /* limit of every device-side wait (default 10000) */
  BDSS_OPT_PERSISTENT = 1,      /* 1 (default): one persistent launch with grid barriers
                                   per factor / solve; 0: one launch per level and phase
                                   (the per-level structure of Algorithms 4 and 7) */
  BDSS_OPT_MAX_REFINE = 2,      /* mixed precision: refinement step limit (default 10) */
  BDSS_OPT_TARGET_BERR_E18 = 3, /* mixed precision: target backward error x 1e18
                                   (default 10000 = 1e-14) */
  BDSS_OPT_DEBUG_SKIP_ARRIVE = 4, /* test hook: CTA 0 skips its arrival at the given
                                   grid barrier (1-based; 0 = off) so that the waits
                                   of the others run out and BDSS_ERR_TIMEOUT results */
  BDSS_OPT_DEBUG_GUARDS = 5,    /* 1: after every call, check the guard band (256 bytes
                                   of a fixed pattern) after each workspace buffer;
                                   an overwritten band gives BDSS_ERR_GUARD */
  BDSS_OPT_DEBUG_CORRUPT_GUARD = 6, /* test hook: overwrite, from the host, one byte of
                                   the guard band of workspace buffer `value` (1-based,
                                   allocation order) to exercise the check */
  BDSS_OPT_REFINE_KRYLOV = 7,   /* mixed precision: 0 = plain refinement only;
                                   1 (default) = when plain refinement stalls (kappa(A)
                                   near or above 1/u_32 ~ 1e7) or has used its
                                   BDSS_OPT_MAX_REFINE steps, cycles of FP64 conjugate
                                   gradients preconditioned by the FP32 factors;
                                   2 = those cycles from the first correction on.
                                   BDSS_OPT_MAX_REFINE = 0 allows no correction at all.
                                   The CG vectors (4 N n d_max doubles) are allocated on
                                   first use; at most 4 cycles, each restarted from the
                                   true FP64 residual */
  BDSS_OPT_MAX_KRYLOV_ITERS = 8, /* mixed precision: CG iterations per cycle (default 300) */
  BDSS_OPT_NSTAR = 12,          /* the crossover N_* of Sec. 3.3 (default 1): the reduction
                                   stops at the first level with at most N_* blocks, which
                                   one CTA then factors and solves by the serial block-
                                   Cholesky sweep (Algorithms 1 and 2 with K = 1), in FP64.
                                   1 <= N_* <= 64; values above 1 are offered for FP64
                                   handles with n <= 64 (else BDSS_ERR_UNSUPPORTED).
                                   Setting it discards the stored factors */
  BDSS_OPT_SHIFT = 11,          /* mixed precision: 1 (default) = when an FP32 pivot fails
                                   (kappa(A) beyond about 1/u_32), factor A + sigma diag(A)
                                   instead, sigma = 2^-20 growing 16x per failure up to
                                   2^-4 (bdss_factor_shift reports it), and refine with
                                   FP64 CG on the unshifted A from the first correction
                                   (unless BDSS_OPT_REFINE_KRYLOV = 0); the copy of A_diag
                                   (N n^2 doubles) is allocated on first use.
                                   0 = return BDSS_ERR_NOT_SPD */
  BDSS_OPT_SCHUR_EMU = 13,      /* FP64, N > 1, 32 <= n <= 256: 1 = the Schur products of the
                                   factorisation (the separator update of Algorithm 3,
                                   D - W^T W and -W^T W of Eq. 5's reduced system) on the
                                   tensor cores: each W row cut into ten BF16 digits below
                                   its maximum (59 bits), every digit product summed
                                   exactly in FP32, the rounds combined in FP64; one
                                   launch per level and phase even in persistent mode.
                                   0 = on the FP64 ALU (for n <= 64 the single persistent
                                   launch).  Default 1 for 64 < n <= 256, 0 for n <= 64.
                                   Setting 1 on a handle without it gives
                                   BDSS_ERR_UNSUPPORTED */
  BDSS_OPT_RESIDUAL_EMU = 10,   /* mixed precision, 64 < n <= 256 and d_max <= 16: 1 (default)
                                   = the FP64 residual of the refinement on the tensor cores
                                   (BF16 digit slices, exact FP32 accumulation: see
                                   bdss_residual); 0 = on the FP64 ALU.  Setting 1 on a
                                   handle without it gives BDSS_ERR_UNSUPPORTED */
  BDSS_OPT_SMALL_CLUSTER = 14,  /* FP64 handles with n <= 32 and d_max <= 16: the one-cluster
                                   path, which runs the whole factor and/or solve (the same
                                   recursion of Sec. 3, Algorithms 4 and 7, with the same
                                   arithmetic and factor storage as the persistent kernel) in
                                   one launch of a single thread-block cluster (up to 16 CTAs)
                                   with hardware cluster barriers between the phases instead
                                   of grid-wide barriers, and writes its status into page-locked
                                   memory itself (no status memset or copy).  -1 (default):
                                   used with BDSS_OPT_PERSISTENT = 1 when n <= 16,
                                   N <= 8 x the cluster's CTAs and N n <= 64 x the
                                   cluster's CTAs (where it measured faster than the
                                   grid kernel); 1: whenever the handle has it;
                                   0: never.  Setting 1 on a handle without it (another
                                   precision or size, or no cluster launch on the device)
                                   gives BDSS_ERR_UNSUPPORTED.  Its launches record no grid
                                   barriers and no trace */
  BDSS_OPT_KERNEL_TIMING = 9    /* 1: time every launch (group) of each following call with
                                   CUDA events recorded on the handle's stream, by kernel
                                   class (bdss_kernel_class); read with
                                   bdss_last_kernel_times.  0 (default): off.  The first
                                   switch-on creates 512 events. */
} bdss_option;

/* Kernel classes of bdss_last_kernel_times. */
typedef enum {
  BDSS_KT_FACTOR = 0,      /* factorisation passes (with the first solve when fused) on CUDA cores */
  BDSS_KT_SCHUR_TC = 1,    /* BDSS_TF32_IR, n > 64: the tensor-core Schur-update launches of a factorisation */
  BDSS_KT_SOLVE = 2,       /* the solve pass of bdss_solve on stored factors */
  BDSS_KT_CORRECTION = 3,  /* mixed precision: refinement corrections X += M^-1 (B - A X) */
  BDSS_KT_RESIDUAL = 4,    /* mixed precision: FP64 residuals B - A X (with the backward-error norms) */
  BDSS_KT_KRYLOV = 5,      /* mixed precision: CG refinement kernels and their preconditioner solves */
  BDSS_KT_SLICE = 6,       /* mixed precision: slicing the operator for the tensor-core residual */
  BDSS_KT_CLASSES = 7
} bdss_kernel_class;

/*
 * Create a solver for systems with N >= 1 blocks of size 1 <= n <= 256 and
 * 1 <= d_max <= 64 right-hand-side columns, allocating all device workspace
 * (the "Init" phase of the evaluation in Sec. 4.2).  Blocks up to n = 64 are
 * staged whole in one CTA's shared memory; 64 < n <= 256 runs the tiled path
 * (64 x 64 tiles).  `cuda_stream` is a cudaStream_t (NULL = default stream).
 * On success *h is a new handle; n > 256 gives BDSS_ERR_UNSUPPORTED.
 */
bdss_status bdss_create(bdss_handle *h, int64_t N, int32_t n, int32_t d_max,
                        bdss_precision prec, void *cuda_stream);

/* Set an option (see bdss_option).  Returns BDSS_ERR_INVALID_ARG for an
 * unknown key or a value out of range. */
bdss_status bdss_set_option(bdss_handle h, bdss_option key, int64_t value);

/*
 * Factor A (Algorithm 4, all levels): at level l, for every eliminated block
 * j: L_j = chol(A_jj) (Algorithm 1, potrf), W_L = L_j^{-1} A_{j,j-1} and
 * W_R = L_j^{-1} A_{j+1,j}^T (Sec. 3.3 stage 2, trsm); for every separator s:
 * S_ss = A_ss - W_R(s-1)^T W_R(s-1) - W_L(s+1)^T W_L(s+1) and
 * S_{s+2,s} = -W_R(s+1)^T W_L(s+1) (Algorithm 3 and Eq. 5, gemm + Assemble);
 * then the single remaining block is factored in FP64.  A_diag and A_sub are
 * not modified.  On BDSS_ERR_NOT_SPD, info->level / info->block name the
 * failing pivot (if info != NULL).
 */
bdss_status bdss_factor(bdss_handle h, const double *A_diag, const double *A_sub,
                        bdss_info *info);

/*
 * Solve with the stored factors (Algorithm 7): upward RHS reduction
 * y_j = L_j^{-1} b_j, b_s -= W^T y (Algorithm 5), the top solve, then the
 * downward back-substitution x_j = L_j^{-T}(y_j - W_L x_{j-1} - W_R x_{j+1})
 * (Algorithms 6 and 2).  1 <= d <= d_max.  In FP64, X may equal B (in
 * place); otherwise B is not modified.  In the mixed modes this runs the
 * refinement loop, which reads B again for every residual, so X must differ
 * from B (else BDSS_ERR_INVALID_ARG); it fills info->iters and
 * info->backward_err.
 */
bdss_status bdss_solve(bdss_handle h, const double *B, double *X, int32_t d, bdss_info *info);

/* bdss_factor followed by bdss_solve, with the upward RHS reduction riding
 * on the factor's levels (one fewer pass over the levels). */
bdss_status bdss_factor_solve(bdss_handle h, const double *A_diag, const double *A_sub,
                              const double *B, double *X, int32_t d, bdss_info *info);

/* log det A = sum over every eliminated block and the top block of
 * 2 sum_k log (L)_kk (det of the permuted matrix = det A_uu det S, Eq. 5),
 * from the stored factors.  `out` is a host pointer. */
bdss_status bdss_logdet(bdss_handle h, double *out);

/*
 * Gradients of a scalar loss L(X), X = A^{-1} B, for a hand-written adjoint
 * (reverse mode).  Given the adjoint Lambda = A^{-1} dL/dX -- obtained with
 * bdss_solve on the stored factors, since A is symmetric -- and X, writes
 *   dA_diag[i] = dL/dA_ii      = -sym(Lambda_i X_i^T)
 *   dA_sub[i]  = dL/dA_{i+1,i} = -(Lambda_{i+1} X_i^T + X_{i+1} Lambda_i^T)
 * (dL/dB = Lambda).  Lambda, X: N x n x d device doubles; dA_diag: N x n x n;
 * dA_sub: (N-1) x n x n (may be NULL iff N == 1).  The operator of Eq. 1 with
 * sym(A_ii) on the diagonal defines these derivatives; the paper has no
 * differentiation step.  Needs no factorisation; uses the handle's sizes and
 * stream.
 */
bdss_status bdss_adjoint_grads(bdss_handle h, const double *Lambda, const double *X, int32_t d,
                               double *dA_diag, double *dA_sub);

/*
 * Kalman-smoother normal equations (Sec. 4.2, the smoothing experiment),
 * assembled on the device from the model of N steps (0-based k):
 *   A_diag[k]  = Qinv[k] + G[k+1]^T Qinv[k+1] G[k+1] + H[k]^T Rinv[k] H[k]
 *   A_sub[k]   = -Qinv[k+1] G[k+1]                        (k < N-1)
 *   B[k]       = H[k]^T Rinv[k] z[k] + Qinv[k] zeta[k] - G[k+1]^T Qinv[k+1] zeta[k+1]
 * with the G[k+1] terms absent for k = N-1.  G[0] is not read (the prior mean
 * enters through zeta[0], the prior precision as Qinv[0]).  Layouts, all
 * row-major FP64 device memory, 16-byte aligned:
 *   G, Qinv: N x n x n;  H: N x m x n;  Rinv: N x m x m, or, with
 *   rinv_diagonal = 1, N x m holding the diagonals of diagonal R[k]^-1 (the
 *   R_k^-1 H_k product is then a row scaling);  z: N x m;
 *   zeta: N x n, or NULL for zero;  A_diag: N x n x n;  A_sub: (N-1) x n x n
 *   (may be NULL iff N == 1);  B: N x n x 1, or NULL to assemble the matrix
 *   only (z is then not read and may be NULL).
 * The outputs feed bdss_factor / bdss_solve directly.  Sizes: N, n, m >= 1
 * and rinv_diagonal 0 or 1 (else BDSS_ERR_INVALID_ARG); n <= 256, m <= 4096 and N (n/64 rounded up)
 * (n/64 + m/64 rounded up, + 1) < 2^31 (else BDSS_ERR_UNSUPPORTED).  The call
 * allocates N (m n + m + n) doubles of stream-ordered workspace on `cuda_stream`
 * (BDSS_ERR_ALLOC if that fails), runs two kernels and synchronises the stream
 * before it returns.  Outputs must not overlap inputs.
 */
bdss_status bdss_kalman_assemble(int64_t N, int32_t n, int32_t m, int32_t rinv_diagonal,
                                 const double *G, const double *H, const double *Qinv,
                                 const double *Rinv, const double *z, const double *zeta,
                                 double *A_diag, double *A_sub, double *B, void *cuda_stream);

/*
 * Partitioned solve of one system over several ranks (the separator /
 * interior partition of Sec. 3.1, Eq. 2-4, applied once at the top level):
 * the N blocks are cut into contiguous chunks, the last block of every chunk
 * but the last is a separator, and each rank eliminates the interior of its
 * chunk (the blocks between its left and right separators) with this handle.
 * The separators then form a block-tridiagonal reduced system (Eq. 5):
 *   S_ss    = A_ss - (S_RR of the interior on its left) - (S_LL of the one on its right)
 *   S_{s',s} = -(S_RL of the interior between s and the next separator s')
 *   b_hat_s = b_s - (b_R of the interior on its left) - (b_L of the one on its right)
 * which every rank solves after one exchange of the contributions, and
 * bdss_chunk_backsolve recovers the interior.
 *
 * bdss_chunk_reduce: factors the interior (A_diag: N x n x n, A_sub:
 * (N-1) x n x n, as bdss_factor; N and n are the handle's, FP64 handles only,
 * else BDSS_ERR_UNSUPPORTED) and returns its contribution to the reduced
 * system.  A_left = A_{first, sL}, the n x n coupling of the first interior
 * block to the left separator (the global sub-diagonal block above the
 * interior), or NULL if there is no left separator; A_right = A_{sR, last},
 * the coupling of the right separator to the last interior block (the global
 * sub-diagonal block below it), or NULL.  B: the interior's right-hand side,
 * N x n x d, 1 <= d <= d_max.  Outputs (device, row-major):
 *   S     = [S_LL, S_RR, S_RL], 3 x n x n:
 *           S_LL = A_left^T (A_I^{-1})_{first,first} A_left,
 *           S_RR = A_right (A_I^{-1})_{last,last} A_right^T,
 *           S_RL = A_right (A_I^{-1})_{last,first} A_left   (zero when absent);
 *   b_hat = [b_L, b_R], 2 x n x d: A_left^T (A_I^{-1} B)_first, A_right (A_I^{-1} B)_last.
 * The factors stay in the handle for bdss_chunk_backsolve.  Allocates
 * stream-ordered temporaries of 2 N n min(n, d_max) doubles (BDSS_ERR_ALLOC)
 * and synchronises the stream.
 *
 * bdss_chunk_backsolve: X = A_I^{-1} (B - E_first A_left x_left -
 * E_last A_right^T x_right) with the stored factors; x_left, x_right: the
 * separators' solution blocks (n x d, device), required where the matching
 * coupling is given.  X: N x n x d device memory.  Allocates N n d doubles
 * stream-ordered and synchronises.
 */
bdss_status bdss_chunk_reduce(bdss_handle h, const double *A_diag, const double *A_sub, const double *A_left,
                              const double *A_right, const double *B, int32_t d, double *S, double *b_hat,
                              bdss_info *info);
bdss_status bdss_chunk_backsolve(bdss_handle h, const double *B, const double *A_left, const double *A_right,
                                 const double *x_left, const double *x_right, int32_t d, double *X);

/* Number of grid barriers / kernel launches the last factor or solve issued
 * (host pointers, either may be NULL). */
bdss_status bdss_last_launch_stats(bdss_handle h, int64_t *kernel_launches, int64_t *grid_barriers);

/* Test hook: the k-th device or page-locked allocation of every following
 * bdss_create, bdss_kalman_assemble or first CG refinement of a handle
 * (counted per call, 1-based) fails as if the memory were exhausted; 0 turns
 * it off.  The call must then return BDSS_ERR_ALLOC; bdss_create frees what
 * it had allocated, a solve keeps its buffers for bdss_destroy. */
bdss_status bdss_debug_fail_alloc(int32_t k);

/* Relative diagonal shift sigma of the handle's stored factors (mixed
 * precision: the factors are those of A + sigma diag(A); 0 when the
 * unshifted FP32 factorisation succeeded).  Host pointer. */
bdss_status bdss_factor_shift(bdss_handle h, double *sigma);

/* Refinement steps of the handle's last mixed-precision solve (host pointers,
 * either may be NULL): plain corrections X += M^-1 r and preconditioned-CG
 * iterations (see BDSS_OPT_REFINE_KRYLOV).  bdss_info.iters is their sum. */
bdss_status bdss_last_refine_stats(bdss_handle h, int32_t *plain_steps, int32_t *cg_iters);

/* Launch configuration the handle chose at creation (host pointers, any may
 * be NULL): resident CTAs per SM of its persistent kernel (from the
 * occupancy calculator), the SM count, and the dynamic shared memory per CTA
 * in bytes.  A full persistent grid has ctas_per_sm * sm_count CTAs. */
bdss_status bdss_get_launch_config(bdss_handle h, int32_t *ctas_per_sm, int32_t *sm_count, int64_t *smem_bytes);

/* Phase trace of the last launch that ran grid barriers (a persistent factor
 * or solve pass): release_ns[i] = %globaltimer (ns) when grid barrier i was
 * released; barrier 0 is the start-up barrier, then for each level l the
 * barriers after its elimination (phase A) and separator (phase B) steps, then
 * one per downward level.  Differences of consecutive stamps are the time of
 * each step.  Writes min(*count, capacity) entries to the host array
 * release_ns and the number recorded (at most 256) to *count (may be NULL).
 * The paper reports wall-clock phases only; this is the per-level split. */
bdss_status bdss_last_trace(bdss_handle h, int64_t *release_ns, int32_t capacity, int32_t *count);

/* Self-check of the tensor-core Schur tile used by BDSS_TF32_IR for n > 64:
 * one 128 x 128 tile C = A B^T with K = 256 computed with TMA-fed
 * tcgen05.mma (3xTF32 split) and compared on the device with an FP64 product
 * of the same FP32 inputs.  *max_rel_err = max |C_tc - C_ref| / sum_k |a b|
 * (host pointer).  Allocates and frees its own small buffers. */
bdss_status bdss_tc_selftest(double *max_rel_err);

/*
 * R = B - A X for the A of the handle's last bdss_factor (or
 * bdss_factor_solve), 1 <= d <= d_max; B, X readable by the device, R device
 * memory, all N x n x d FP64.  The residual of the mixed-precision
 * refinement, exposed: with BDSS_OPT_RESIDUAL_EMU on (mixed
 * precision, 64 < n <= 256, d <= 16) it runs on the tensor cores -- every
 * operator row [A_{i,i-1}, sym(A_ii), A_{i,i+1}] and every column of X is
 * rounded to 59 bits below its maximum and cut into ten signed 6-bit digits
 * (exact in BF16); all digit products are summed exactly in the FP32
 * accumulators (no partial sum reaches 2^24) and combined in 64-bit integers
 * and FP64, so |R - R_exact| stays within a few units of 2^-59 times the row
 * maximum of A times the column maximum of X per term, FP64's own accuracy
 * for the backward error ||B - A X|| / (||A|| ||X||).  The operator is sliced
 * once per factorisation (about 30 n^2 bytes per block).  Otherwise R is
 * formed on the FP64 ALU.  Not in the paper, which takes residuals of its
 * final solutions only (Sec. 4); it is the residual of the refinement loop.
 */
bdss_status bdss_residual(bdss_handle h, const double *B, const double *X, int32_t d, double *R);

/* Device time of the handle's last bdss_factor, bdss_solve or
 * bdss_factor_solve by kernel class, with BDSS_OPT_KERNEL_TIMING on: ms[c]
 * (milliseconds between the CUDA events recorded on the handle's stream
 * before and after each launch or launch group of class c, summed) and
 * launches[c] (kernel launches in those groups; may be NULL), for
 * c < min(classes, BDSS_KT_CLASSES).  Zeros when timing is off.  Host
 * pointers.  The paper reports per-phase wall-clock times (factor, solve);
 * this is the same split per kernel, on the device. */
bdss_status bdss_last_kernel_times(bdss_handle h, double *ms, int64_t *launches, int32_t classes);

/* Description of the last CUDA runtime error that made a bdss_* call on this
 * host thread return BDSS_ERR_CUDA ("no error" if none).  Never NULL. */
const char *bdss_last_cuda_error(void);

/* ---------------------------------------------------------------------------
 * Batched solves: K independent systems of uneven N_k and n_k (FP64, d RHS
 * columns each) -- the batch {A^(k)} of Sec. 3.2 -- factored and solved in
 * ONE kernel launch.  A device work queue hands out (instance, stage, item
 * range) tasks; stage s of an instance (its levels' phase A and B, the top
 * block, the downward levels) starts when stage s-1 of the same instance is
 * complete, so instances overlap freely.  Per-instance results, status and
 * latency.  Pointer arrays are HOST arrays of K DEVICE pointers; A_sub_k[k]
 * may be NULL iff N_k[k] == 1.  1 <= n_k <= 64.
 * ------------------------------------------------------------------------- */
typedef struct bdss_batch_ctx *bdss_batch;

/* Allocate the workspace of all instances and build the task queue.  Uses
 * the autotuned (threads per CTA, items per task) for (max n_k, d) if
 * bdss_batch_autotune has run in this process, else a default. */
bdss_status bdss_batch_create(bdss_batch *b, int32_t K, const int64_t *N_k, const int32_t *n_k, int32_t d,
                              void *cuda_stream);
/* Bind the K systems' device buffers (X_k[k] may equal B_k[k]).  Synchronises. */
bdss_status bdss_batch_set_inputs(bdss_batch b, const double *const *A_diag_k, const double *const *A_sub_k,
                                  const double *const *B_k, double *const *X_k);
/* Enqueue one factor + solve of every instance on the batch's stream without
 * waiting.  use_graph != 0: the enqueue sequence (counter resets + the
 * kernel) is captured once into a CUDA graph and replayed. */
bdss_status bdss_batch_launch(bdss_batch b, int32_t use_graph);
/* Wait for the last launch; info_k[k] (K entries, may be NULL) gets the
 * instance's pivot failure (level/block) with its status code in `reserved`;
 * latency_us_k[k] (may be NULL) the time from the launch's first task start
 * to the instance's last task end, i.e. how long after the batch began the
 * instance's solution was complete.  Instances are queued in groups of
 * ascending work, each group stage by stage, so small instances complete
 * early.  Returns the first non-OK status. */
bdss_status bdss_batch_wait(bdss_batch b, bdss_info *info_k, double *latency_us_k);
/* Time every candidate (threads per CTA in {32,64,128,256} >= max n_k;
 * items per task in {1,2,4}) on the bound inputs, keep the fastest for this
 * batch and record it for (max n_k, d) in the process-wide table. */
bdss_status bdss_batch_autotune(bdss_batch b, int32_t reps, int32_t *threads, int32_t *items);
bdss_status bdss_batch_destroy(bdss_batch b);

/* One-shot: create + set_inputs + launch + wait + destroy.  info_k: host, K entries. */
bdss_status bdss_factor_solve_batched(int32_t K, const int64_t *N_k, const int32_t *n_k, int32_t d,
                                      const double *const *A_diag_k, const double *const *A_sub_k,
                                      const double *const *B_k, double *const *X_k, void *cuda_stream,
                                      bdss_info *info_k);

/*
 * No-allocation variant of bdss_factor_solve (FP64).  The paper has no
 * counterpart; this entry point exists for callers that may not allocate
 * device memory while they run: a real-time control or estimation loop in
 * which cudaMalloc / cudaFree could synchronise the device and take unbounded
 * time, or a plugin whose host application's allocator owns all device
 * memory.  It allocates nothing: its workspace is a fixed device array of
 * BDSS_NOALLOC_SCRATCH_BYTES inside this library, which every GPU that loads
 * the library holds from load until process exit.
 *
 * Arguments are those of bdss_create + bdss_factor_solve for one FP64 system
 * of blocks n <= 64 (same layouts; X may equal B; inputs in device memory or
 * memory the device can read in place); the result equals that of the
 * allocating entry point, with the same launch configuration.  The call
 * synchronises `cuda_stream` before it returns, to read the status word.
 * Returned before anything is launched: BDSS_ERR_INVALID_ARG for a bad size
 * or pointer, BDSS_ERR_UNSUPPORTED for n > 64 (the tiled path of larger
 * blocks is not offered here), for a shared-memory need beyond the device's
 * limit, and for systems whose workspace (about 3 N n^2 doubles) does not fit
 * the array.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress), the device's limits, and raises the kernels'
 * shared-memory limits; make that first call before any stream capture.
 * Later calls make no attribute calls.  All calls on a device share the one array
 * and it keeps the last call's contents (the status word is cleared at the
 * start of each call): calls that overlap on the GPU -- on different streams
 * or host threads -- race and must be serialised by the caller.
 */
#define BDSS_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
bdss_status bdss_factor_solve_noalloc(int64_t N, int32_t n, int32_t d, const double *A_diag,
                                      const double *A_sub, const double *B, double *X,
                                      void *cuda_stream, bdss_info *info);

/* Release the handle and its workspace.  NULL-safe. */
bdss_status bdss_destroy(bdss_handle h);

/* Static description of a status code (never NULL). */
const char *bdss_status_string(bdss_status s);

#ifdef __cplusplus
}
#endif

#endif /* BDSS_H */
