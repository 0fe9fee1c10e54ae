/*
 * admm.h -- C ABI of libadmm.so, a GB300 (sm_103a) implementation of the
 * norm-1 regularised ADMM of Heredia-Juesas, Molaei, Tirado and
 * Martinez-Lorenzo, "Consensus and Sectioning-based ADMM with Norm-1
 * Regularization for Imaging with a Compressive Reflector Antenna".
 *
 * The library solves   minimize 1/2 ||H u - g||_2^2 + lambda ||u||_1
 * over u in C^n (Section III, Eq. original; g = Hu + w of Eq. 2), with H in
 * C^{m x n} split into row_blocks x col_blocks contiguous blocks:
 *
 *   row_blocks = M, col_blocks = 1 : consensus ADMM       (Section III-A)
 *   row_blocks = 1, col_blocks = N : sectioning ADMM      (Section III-B)
 *   row_blocks = M, col_blocks = N : consensus and sectioning ADMM
 *                                                          (Section III-C)
 *   row_blocks = col_blocks = 1    : the unsplit lasso ADMM of Section III
 *
 * Conventions for every call:
 *  - Complex data is interleaved (re, im): complex64 = two floats,
 *    complex128 = two doubles, i.e. C99 float/double _Complex and the
 *    contiguous layout of torch.complex64 / numpy.complex64.
 *  - Matrices are row-major and contiguous.
 *  - A "buffer" argument may point to device memory or to host memory; the
 *    library copies with cudaMemcpyDefault (unified addressing).  Pinned host
 *    memory keeps the copy asynchronous; pageable host memory makes it
 *    synchronous.  The caller keeps ownership of every buffer it passes and
 *    the library never frees caller memory.  The library owns what it
 *    allocates in admm_setup (the packed H, the cached factors and the
 *    iteration state) until admm_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are asynchronous with respect to the host unless their
 *    comment says they synchronise.
 *  - Every function returns an admm status code (0 = ADMM_OK) unless noted;
 *    admm_last_error(h) then holds a one-line description.  A failed call
 *    leaves the handle usable unless it returned ADMM_ETIMEOUT or
 *    ADMM_ECUDA, after which only admm_reset, the getters and admm_destroy
 *    are accepted.
 *  - Blocks are contiguous and balanced: the first (m mod M) row blocks get
 *    one extra row, the first (n mod N) column blocks one extra column (the
 *    paper assumes exact division, Sections III-A..C).
 */
#ifndef ADMM_H
#define ADMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADMM_ABI_VERSION 5

/* status codes */
#define ADMM_OK            0  /* success */
#define ADMM_EINVAL        1  /* invalid argument: null pointer, size, split, lambda < 0, rho <= 0 */
#define ADMM_ENOMEM        2  /* a device allocation failed */
#define ADMM_ECUDA         3  /* a CUDA runtime call or launch failed */
#define ADMM_ENOTPD        4  /* a factor rho I + H_b H_b^H was not positive definite in FP64 */
#define ADMM_ENONFINITE    5  /* H or g holds NaN or Inf */
#define ADMM_ETIMEOUT      6  /* a bounded in-kernel wait expired; the iteration state is undefined */
#define ADMM_EUNSUPPORTED  7  /* a valid problem this library does not run (see admm_setup) */
#define ADMM_EDIVERGED     8  /* the iterates became NaN or Inf */

/* element type of H and g in admm_setup / admm_set_g */
#define ADMM_C64   0          /* complex64: two floats per element */
#define ADMM_C128  1          /* complex128: two doubles, rounded to complex64 on the device */

/* options for admm_set_option */
#define ADMM_OPT_TIMEOUT_NS    1  /* bound of every in-kernel wait, nanoseconds (default 5e9) */
#define ADMM_OPT_HIST_CAP      2  /* residual-history ring capacity, records (default 4096); resets the history */
#define ADMM_OPT_BARRIER_EXTRA 3  /* fault injection: make every grid barrier wait for this many
                                     CTAs that do not exist, so the bounded wait expires and the
                                     call ends with ADMM_ETIMEOUT (0 = off, the default) */
#define ADMM_OPT_TRACE_ITERS   4  /* record %globaltimer phase stamps of the first `value`
                                     iterations of each launch (0 = off, the default) */
#define ADMM_OPT_L2_KEEP_BYTES 5  /* bytes of H at the end of each pass over H that keep the
                                     normal L2 priority, so the next pass (which walks the
                                     rows in the opposite order) finds them in L2; the rest
                                     of H and the factors are loaded evict_first (default
                                     52 MiB; 0 = no L2 policy hints) */
#define ADMM_OPT_L2_PREFETCH_BYTES 7  /* bytes of H per pass prefetched into L2 (TMA
                                     prefetch, no shared memory) while the previous pass
                                     ends and the grid waits at its barriers: the rows the
                                     next pass reads right after its L2-resident head
                                     (default 0) */
#define ADMM_OPT_RECORD_ITERS  8  /* record the next `value` iterations for admm_backward
                                     (their shrinkage arguments a and factor solutions w);
                                     0 turns recording off.  Resets the state. */
#define ADMM_OPT_DIR_FACTOR_PASS 9  /* direct form: how u_b = L_b q_b reads the factors.  2: the
                                     lower triangle of the Hermitian L_b only, in 64 x 64 tiles
                                     (about half the bytes; blocks of 256 columns and more and at
                                     most 512 row blocks, else ADMM_EUNSUPPORTED): each tile adds
                                     L_IJ q_J to the rows of panel I and, below the diagonal,
                                     L_IJ^H q_I to those of panel J, summed per row in a fixed
                                     order; 1: full factor rows (plain loads, or bulk copies for
                                     blocks of 1024-2048 columns); 0 (the default): 2 for blocks
                                     of 1024 columns and more, else 1.  The lemma form ignores
                                     it. */
#define ADMM_OPT_H_FP16        6  /* 1: stream an FP16 copy of H (half the bytes per pass);
                                     0: stream the complex64 H (the default).  The first 1
                                     builds the copy: every 64-row group g of H gets the scale
                                     c_g = 2^(q-14), where max over the group of max(|Re|,|Im|)
                                     is f 2^q with f in [0.5, 1), and H16 = fp16_rn(H / c_g)
                                     (round to nearest even; |H / c_g| < 2^14).  The cached
                                     factors of that mode are those of the matrix H16 c_g
                                     encodes, so an FP16 run is exact ADMM on that matrix.
                                     The iteration state is shared: switching back to 0
                                     continues from the FP16 iterate on the complex64 H
                                     (polish iterations).  The copy takes m * ld * 4 bytes
                                     more device memory and is kept until admm_destroy;
                                     admm_set_rho refactors both.  Synchronises the device. */

/* factor form of the block update (admm_setup_form) */
#define ADMM_FORM_LEMMA   0   /* m_b x m_b factor K_b^{-1} = (rho I + H_b H_b^H)^{-1}, any block shape */
#define ADMM_FORM_DIRECT  1   /* n_b x n_b factor (H_b^H H_b + rho I)^{-1}, column blocks <= 12288 wide */
#define ADMM_FORM_AUTO    2   /* the paper's rule (Section III-B): DIRECT when every block has at
                                 least as many rows as columns (and fits), else LEMMA */

typedef struct admm_problem admm_t;

/* Sizes and plan of a handle (admm_get_info). */
typedef struct admm_info {
    int64_t m, n;             /* problem size */
    int64_t ld;               /* row pitch of the packed device copy of H, complex elements */
    int32_t row_blocks, col_blocks;
    double lambda, rho, kappa;  /* kappa = lambda / (row_blocks * rho), the shrinkage threshold */
    int64_t iterations;       /* iterations completed since setup / reset */
    int32_t ctas;             /* CTAs of the persistent iteration kernel (one per SM at most);
                                 direct form: CTAs of the factor pass */
    int32_t rows_per_stage;   /* rows of H per pipeline stage; direct form: factor rows per
                                 stage of the streamed factor pass (0: plain loads; 64: the
                                 tile pass over the lower triangles) */
    int32_t stages;           /* depth of the TMA pipeline (direct form: of the factor ring; the
                                 tile pass: slots of its ring of 16-row tile pieces) */
    int32_t slab_cols;        /* widest column slab owned by one CTA (0 in the direct form) */
    int32_t smem_bytes;       /* dynamic shared memory of the iteration kernel (direct form:
                                 of the streamed factor pass or the tile pass, 0 with plain
                                 loads) */
    int32_t num_sms;
    int64_t h_bytes;          /* bytes of H streamed by one pass (m * n * 8) */
    int64_t factor_bytes;     /* bytes of all cached factors (complex64); with the direct form's
                                 tile pass, of the lower-triangle tiles an iteration reads */
    int64_t state_bytes;      /* bytes of v, s, u, estimated data and scratch */
    double setup_gram_ms;     /* device time of the Gram products */
    double setup_factor_ms;   /* device time of the FP64 Cholesky and inverse */
    int32_t h_fp16;           /* 1 while the iterations stream the FP16 copy of H */
    int32_t h16_ready;        /* 1 once the FP16 copy and its factors exist */
    int64_t h16_bytes;        /* bytes of H streamed by one pass in FP16 (m * n * 4), 0 if none */
    int64_t l2_keep_bytes;    /* current ADMM_OPT_L2_KEEP_BYTES (admm_tune may change it) */
    int32_t factor_form;      /* ADMM_FORM_LEMMA or ADMM_FORM_DIRECT */
    int32_t reserved;         /* 0 */
} admm_info_t;

/* Launch plan of the iteration kernel, computed on the host (admm_plan). */
typedef struct admm_plan {
    int32_t ctas;             /* CTAs (column slabs) */
    int32_t slab_cols;        /* widest slab, columns (even) */
    int32_t chunks;           /* 32-pair chunks per lane (template width) */
    int32_t box_cols;         /* TMA box width, columns */
    int32_t boxes_per_row;    /* TMA boxes covering one slab row */
    int32_t rows_per_stage;   /* TMA box height */
    int32_t stages;           /* pipeline depth */
    int32_t smem_bytes;       /* dynamic shared memory */
    int32_t max_blocks_per_slab; /* most column blocks one slab intersects */
    int64_t ld;               /* padded row pitch, complex elements */
    int32_t groups;           /* column groups of consumer warps per CTA: 2 for slabs of more
                                 than 256 pairs (each group takes half the slab, so a lane
                                 holds chunks x 32 pairs of a half), else 1 */
    int32_t reserved;
} admm_plan_t;

/* ABI version of the loaded library (ADMM_ABI_VERSION at build time). */
int admm_abi_version(void);

/* Static text for a status code.  Never NULL. */
const char* admm_strerror(int status);

/* Description of the last failure on `h` (or of the last failed admm_setup
 * when h is NULL).  The string lives until the next call on the handle. */
const char* admm_last_error(const admm_t* h);

/* Contiguous balanced blocks (the partition used by every split): writes
 * parts+1 offsets, offsets[0] = 0, offsets[parts] = total, sizes differing by
 * at most one with the larger blocks first.  Host only, no GPU needed.
 * ADMM_EINVAL unless 1 <= parts <= total and offsets != NULL. */
int admm_partition(int64_t total, int32_t parts, int64_t* offsets);

/* Elements of C^1 one node exchanges per iteration when the split runs on
 * separate nodes (Section IV, Table I), for m measurements (N_m), n unknowns
 * (N_p), M = row_blocks and N = col_blocks: out[0] = 2 n (row split: the
 * replica out, the consensus image back), out[1] = N m (column split: the
 * estimated data of every block), out[2] = N m / M + 2 n / N (both; may be
 * fractional).  All three are written whatever the split, so callers can
 * compare them (Section IV-B).  Host only, no GPU needed.  ADMM_EINVAL unless
 * m, n >= 1, 1 <= row_blocks, 1 <= col_blocks and out != NULL.  The counts
 * are the paper's; a handle runs every block on one GPU and exchanges nothing
 * between nodes (the admm_shard_* calls exchange between ranks). */
int admm_comm_elements(int64_t m, int64_t n, int32_t row_blocks, int32_t col_blocks, double* out);

/* Plan of the persistent iteration kernel for an m x n problem split into
 * row_blocks x col_blocks on a GPU with `num_sms` SMs and `smem_limit` bytes of
 * opt-in shared memory per block.  Host only, no GPU needed.  When
 * cta_cols != NULL it receives 4*ctas entries, per CTA the [begin, end)
 * column range (even numbers) of its slab of H followed by the [first, last+1)
 * range of the columns whose state it owns; the buffer must hold 4*num_sms
 * entries.  Slabs are aligned to column blocks when col_blocks <= ctas, and
 * two neighbouring slabs then share the 16-byte column pair holding an odd
 * block boundary, each owning one of its columns.
 * ADMM_EINVAL for bad sizes, ADMM_EUNSUPPORTED when the slab or the shared
 * memory needs exceed what the kernel supports. */
int admm_plan(int64_t m, int64_t n, int32_t row_blocks, int32_t col_blocks,
              int32_t num_sms, int32_t smem_limit, admm_plan_t* plan, int32_t* cta_cols);

/* Create a solver for g = Hu + w (Eq. 2) under the split (row_blocks,
 * col_blocks), with regularisation weight `lambda` >= 0 and augmented
 * parameter `rho` > 0 (Section II).  Copies H (m x n) and g (m) -- host or
 * device buffers of element type h_dtype -- into library-owned device memory,
 * forms every Gram block H_b H_b^H with FP32 products accumulated in FP64,
 * and caches the inverse of K_b = rho I + H_b H_b^H computed from an FP64
 * Cholesky factorisation, stored as complex64.  K_b^{-1} is rho times the
 * (I + H_b H_b^H / rho)^{-1} of the inversion lemma, Eq. (inversion_lemma),
 * (inversion_lemma2) and (inversion_lemma3).  The iteration state starts at
 * v = s = u = 0 with zero estimated data.
 * Requires 1 <= row_blocks <= m, 1 <= col_blocks <= n and
 * row_blocks * col_blocks <= 256.  A block with at least as many rows as
 * columns, where the paper inverts the n_b x n_b matrix H_b^H H_b + rho I
 * directly (Section III-B), uses the same m_b x m_b factor: the identity
 * (H_b^H H_b + rho I)^{-1} (H_b^H x + rho z) = z + H_b^H K_b^{-1} (x - H_b z)
 * holds for every shape, so the result is the direct branch's; the cost is
 * m_b^2 cached factor elements per block instead of n_b^2 (ADMM_ENOMEM or
 * ADMM_EUNSUPPORTED when they do not fit).
 * Synchronises `stream`.  On success *out receives the handle; on failure
 * *out is NULL and admm_last_error(NULL) describes the error. */
int admm_setup(admm_t** out, const void* H, const void* g, int64_t m, int64_t n,
               int32_t row_blocks, int32_t col_blocks, double lambda, double rho,
               int32_t h_dtype, void* stream);

/* admm_setup with a choice of factor form.  ADMM_FORM_LEMMA is admm_setup.
 * ADMM_FORM_DIRECT caches, for every block, the n_b x n_b inverse
 *     L_b = (H_b^H H_b + rho I)^{-1}
 * (the original inversion of Eq. x_solution_columns, which Section III-B
 * prefers when N_m > N_p / N), formed with the same FP32-product / FP64-sum
 * Gram kernels and FP64 Cholesky inverse over the blocks of H^H, stored as
 * complex64.  Each iteration then computes
 *     q_b    = H_b^H gt_b + rho (v_j - s_j^i)     (one pass over H_b; with one
 *                                                  column block gt_b = g_i and
 *                                                  H_b^H g_i is computed once
 *                                                  per data vector, so H is not
 *                                                  read at all)
 *     u_b    = L_b q_b
 *     ghat_b = H_b u_b                            (one pass, col_blocks > 1)
 * and the same v, s update and residual record as the lemma form: the
 * iterates are the same algorithm's, so every getter, admm_set_g /
 * _lambda / _rho (which refactors L_b), checkpoints and admm_solve behave
 * as documented for admm_setup.  The persistent-kernel options
 * (ADMM_OPT_H_FP16, ADMM_OPT_RECORD_ITERS, ADMM_OPT_TRACE_ITERS,
 * ADMM_OPT_BARRIER_EXTRA) and admm_backward return ADMM_EUNSUPPORTED, the L2
 * options have no effect, admm_tune does nothing and admm_group_setup
 * refuses the handle.  Column blocks wider than 12288 columns return
 * ADMM_EUNSUPPORTED.  ADMM_FORM_AUTO picks DIRECT when every block has
 * m_b >= n_b and fits, else LEMMA; admm_get_info reports the choice. */
int admm_setup_form(admm_t** out, const void* H, const void* g, int64_t m, int64_t n,
                    int32_t row_blocks, int32_t col_blocks, double lambda, double rho,
                    int32_t h_dtype, int32_t form, void* stream);

/* Run `iters` >= 0 iterations, each the block update of Sections III-A..C:
 *   z_b   = v_b - s_b
 *   u_b   = (H_b^H H_b + rho I)^{-1} (H_b^H gt_b + rho z_b)
 *           with gt_b = g_i - sum_{q != j} H_iq u_q^i of the previous iterate
 *           (Eq. g_columns, g_rows_columns; gt_b = g_i for one column block),
 *   v_j   = S_kappa(mean_i u_j^i + mean_i s_j^i), kappa = lambda/(M rho)
 *           (Eq. v_variable, v_variable_columns, v_variable_rows_columns;
 *           S is the complex soft-threshold of Eq. softhresholding),
 *   s_b  += u_b - v_j,
 * plus the FP64 squared residual norms of each iteration (the norms below
 * Eq. inversion_lemma, inversion_lemma2 and inversion_lemma3).
 * One persistent cooperative kernel runs all `iters` iterations.
 * Asynchronous: errors of the in-kernel bounded waits (ADMM_ETIMEOUT) and
 * divergence (ADMM_EDIVERGED) surface at the next synchronising call. */
int admm_iterate(admm_t* h, int32_t iters, void* stream);

/* Iterate until the primal and dual residuals meet the tolerances of Boyd et
 * al. Section 3.3.1 (the reference the paper cites for its residuals):
 *   ||r_p|| <= sqrt(p) eps_abs + eps_rel max(||u||, ||v||),
 *   ||r_d|| <= sqrt(p) eps_abs + eps_rel rho ||s||,
 * with p = row_blocks * n the stacked length and u, v, s stacked over the
 * replicas, or until max_iter iterations.  The test runs on the device after
 * every iteration.  Synchronises `stream`.  *iters_done (may be NULL)
 * receives the iterations this call ran; the state is that after the last
 * of them. */
int admm_solve(admm_t* h, int32_t max_iter, double eps_abs, double eps_rel,
               int32_t* iters_done, void* stream);

/* Copy the image v (n complex64; Section III-C: v = [v_1; ...; v_N]) into `v`. */
int admm_get_v(admm_t* h, void* v, void* stream);

/* Copy the replicas u^i of the last iteration (row_blocks x n complex64,
 * replica-major) into `u`. */
int admm_get_u(admm_t* h, void* u, void* stream);

/* Copy up to `cap` per-iteration records into `out` (5 doubles each: ||r_p||^2,
 * ||r_d||^2, ||u||^2, ||v||^2, ||s||^2 with u, v, s stacked over the replicas),
 * oldest first, ending with the last completed iteration; *count receives the
 * number written.  Synchronises `stream` and returns the sticky device status
 * (ADMM_ETIMEOUT / ADMM_EDIVERGED) if one was raised. */
int admm_get_residuals(admm_t* h, double* out, int32_t cap, int32_t* count, void* stream);

/* Replace the data vector g (m elements of type h_dtype) -- a new scene for
 * the same H; no refactorisation.  The iteration state is kept (call
 * admm_reset for a cold start). */
int admm_set_g(admm_t* h, const void* g, int32_t h_dtype, void* stream);

/* Replace lambda >= 0 (no refactorisation; kappa = lambda/(M rho)). */
int admm_set_lambda(admm_t* h, double lambda);

/* Replace rho > 0: recomputes every cached factor rho I + H_b H_b^H and
 * rescales the scaled duals s by rho_old/rho_new so the unscaled duals are
 * unchanged.  Synchronises `stream`. */
int admm_set_rho(admm_t* h, double rho, void* stream);

/* Zero the iteration state (v = s = u = 0, estimated data 0), the
 * residual history and the iteration count; clears a sticky device error. */
int admm_reset(admm_t* h, void* stream);

/* Checkpoint: copy the iteration count and the state (v: n, s: row_blocks x
 * n, estimated data: col_blocks x m, all complex64) into caller buffers.
 * Any buffer may be NULL to skip it.  Synchronises `stream`. */
int admm_get_state(admm_t* h, int64_t* k, void* v, void* s, void* ghat, void* stream);

/* Restore a checkpoint written by admm_get_state (same layouts); the next
 * iteration continues exactly as the uninterrupted run would.  `ghat` may be
 * NULL only when col_blocks == 1. */
int admm_set_state(admm_t* h, int64_t k, const void* v, const void* s, const void* ghat,
                   void* stream);

/* Fill *info with the sizes and the kernel plan of `h`. */
int admm_get_info(const admm_t* h, admm_info_t* info);

/* Set an ADMM_OPT_* option. */
int admm_set_option(admm_t* h, int32_t option, int64_t value);

/* Autotune the L2 policy of the current mode (complex64 or FP16 H): time
 * single-iteration launches with candidate ADMM_OPT_L2_KEEP_BYTES values
 * (0 to 96 MiB, at most one pass of H) and keep the fastest.  Leaves the
 * handle reset (admm_reset).  Synchronises. */
int admm_tune(admm_t* h, void* stream);

/* Phase trace of the last launch (needs ADMM_OPT_TRACE_ITERS > 0): for CTA 0
 * and the last CTA, and for each of the first min(cap, trace length)
 * iterations, 8 %globaltimer stamps in nanoseconds: iteration start, first
 * pass over H done, first grid barrier passed, partial sums reduced, second
 * barrier passed, factors applied, third barrier passed, second pass over H
 * and state update done.  `out` holds 2 * cap * 8 int64 (CTA 0 first); *count
 * receives the iterations written per CTA.  Synchronises `stream`. */
int admm_get_trace(admm_t* h, int64_t* out, int32_t cap, int32_t* count, void* stream);

/* Gradient of a real loss L of the image v after the iterations run since the
 * last reset (all recorded: ADMM_OPT_RECORD_ITERS, with g, lambda, rho and the
 * H mode unchanged): given grad_v = dL/dv (n complex64, host or device, in the
 * convention x_bar = dL/dRe x + i dL/dIm x), write grad_g = dL/dg (m complex64)
 * and *grad_lambda, *grad_rho.  The reverse sweep is the adjoint of every
 * step of the iteration (see admm_batch_backward for the formulas), with the
 * products H sigma_bar, K^{-1} w_bar and H^H r_bar over the matrix the forward
 * streamed.  Synchronises.  ADMM_EINVAL when the iterations were not all
 * recorded.  The paper has no counterpart. */
int admm_backward(admm_t* h, const void* grad_v, void* grad_g, double* grad_lambda, double* grad_rho,
                  void* stream);

/* Synchronise `stream` and return the sticky device status of `h`. */
int admm_status(admm_t* h, void* stream);

/* Free everything the handle owns.  NULL is accepted. */
void admm_destroy(admm_t* h);

/* ---------------------------------------------------------------------------
 * Sharded iteration (Section IV, Table I): the blocks of one split spread
 * over several ranks, each rank holding a handle of its own blocks -- the
 * rows of its row blocks and the columns of its column blocks of H, set up
 * with those blocks' counts (admm_setup on the sub-matrix, lambda and rho of
 * the whole problem).  Per iteration the caller moves two sums between ranks
 * (with any collective library):
 *   1. column splits: t_local = admm_shard_ghat_sum (the handle's estimated
 *      data summed over its column blocks, per row); T = the sum of t_local
 *      over the ranks holding the same rows; admm_shard_set_exchange(T), so
 *      the handle's blocks fit g_i - sum_{q != j} ghat_iq over every column
 *      block q of the problem (Eq. g_columns, g_rows_columns);
 *   2. admm_shard_ustep: the u-step of every local block (the handle's one
 *      pass pair over its H), writing per column the sum over the local
 *      replicas of u^i + s^i; S = the sum over the ranks holding the same
 *      columns;
 *   3. admm_shard_vstep(S): v = S_kappa(S / row_blocks_total), kappa =
 *      lambda / (row_blocks_total rho) (Eq. v_variable, v_variable_rows_
 *      columns), and s^i += u^i - v for the local replicas; rec receives the
 *      local residual partials sum ||u^i - v||^2, ||v - v_old||^2,
 *      sum ||u^i||^2, ||v||^2, sum ||s^i||^2 (FP64).
 * Consensus exchanges only step 2's sums (n per rank), sectioning only step
 * 1's (m per rank), consensus and sectioning both over sub-groups.  The paper
 * has no code for this; it describes the node-to-node exchanges.
 * ------------------------------------------------------------------------- */

/* Put a lemma-form handle into sharded mode: row_blocks_total is the number
 * of row blocks (replicas) of the whole split.  Keeps the handle's g as the
 * data vector (admm_set_g and admm_reset keep using it).  Synchronises. */
int admm_shard_enable(admm_t* h, int32_t row_blocks_total, void* stream);

/* t_local (m complex64, host or device): per row, the sum of the handle's
 * current estimated data over its column blocks. */
int admm_shard_ghat_sum(admm_t* h, void* t_local, void* stream);

/* t_global (m complex64): the sum of t_local over the ranks sharing these
 * rows; the blocks then fit g - t_global + t_local - sum of the other local
 * blocks' estimated data. */
int admm_shard_set_exchange(admm_t* h, const void* t_global, void* stream);

/* One u-step of every local block (one launch of the persistent kernel);
 * sum_out (n complex64) receives sum over local replicas of u^i + s^i. */
int admm_shard_ustep(admm_t* h, void* sum_out, void* stream);

/* v and s update from sum_global (n complex64, the sum over all replicas);
 * rec: 5 doubles, the local residual partials.  Synchronises `stream`;
 * returns a device status (ADMM_ETIMEOUT, ADMM_EDIVERGED) raised meanwhile. */
int admm_shard_vstep(admm_t* h, const void* sum_global, double* rec, void* stream);

/* Allocation-free solve of a small problem.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * a framework whose own pool allocator owns all of the GPU's memory, or a
 * real-time loop that must not pay for (or risk failing) an allocation.
 * admm_setup allocates, so such callers use this call instead.
 * It computes what admm_setup + admm_iterate(iters) + admm_get_v compute
 * from the zero initial state (same kernels, same results), but takes all of
 * its working memory -- factors, FP64 factor workspace, iteration state and
 * products -- from one 8 MiB array in the library's device image, which every
 * GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   H      device pointer: m x n complex64, row-major, 16-byte aligned, with n
 *          a multiple of 32 in [32, 2^24] and 1 <= m <= 2^20 (used in place,
 *          not copied);
 *   g      device pointer: m complex64;
 *   v_out  device pointer: n complex64, receives the image v.
 * H, g and v_out must be memory of the current device (cudaMalloc'd on it,
 * or managed); host memory, pinned or not, returns ADMM_EINVAL before any
 * kernel runs.  Every block shape is accepted: like admm_setup, blocks with
 * m_b >= n_b use the m_b x m_b factor.  NaN or Inf in H or g returns
 * ADMM_ENONFINITE before any factor is formed.  A problem whose working
 * memory exceeds the 8 MiB (for example, 256 x 4096 with 4 row blocks needs
 * about 1.1 MiB) returns ADMM_EINVAL, as do other invalid arguments; the
 * reason is in admm_last_error(NULL).
 * The first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress) and keeps it; make that first call before any stream
 * capture.  Every call reuses the same array and clears what must start at
 * zero itself, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Synchronises `stream`
 * (after the input check and at the end). */
int admm_solve_small_noalloc(const void* H, const void* g, int64_t m, int64_t n,
                             int32_t row_blocks, int32_t col_blocks, double lambda, double rho,
                             int32_t iters, void* v_out, void* stream);

/* ---------------------------------------------------------------------------
 * Several independent problems in one persistent launch.  Each handle keeps
 * its state; the group re-plans every problem for a share of the SMs (in
 * proportion to its bytes of H and factors, at least what its column slabs
 * need) and runs all problems of a wave together in one cooperative launch,
 * each on its own CTAs with its own grid barriers.  Problems that do not fit
 * the SMs together go to further waves (launched one after another).  The
 * paper solves one problem at a time; this is the library's scheduler for
 * many uneven ones.  Up to 48 problems, all waves run in ONE cooperative
 * launch of the kernel instance every problem's plan shares.
 * ------------------------------------------------------------------------- */
typedef struct admm_group admm_group_t;

/* Build a group over `count` handles (which must outlive it).  Host planning
 * plus small allocations; synchronises the device.  On failure *out is NULL
 * and admm_group_last_error(NULL) says why. */
int admm_group_setup(admm_group_t** out, admm_t* const* handles, int32_t count, void* stream);

/* Run `iters` iterations of every problem (one launch per wave); each handle's
 * iteration count, history and state advance as under admm_iterate.  All
 * problems of a wave must share the H mode (complex64 or FP16).  Synchronises. */
int admm_group_iterate(admm_group_t* g, int32_t iters, void* stream);

/* Number of waves, and the CTAs each problem was given (cap entries). */
int admm_group_info(const admm_group_t* g, int32_t* waves, int32_t* ctas, int32_t cap);

/* Cooperative launches per admm_group_iterate: 1 when every wave runs in one
 * launch (groups of up to 48 problems: a CTA moves on to its next wave's
 * problem as soon as its current one is done), else the number of waves.
 * -1 for NULL. */
int admm_group_launches(const admm_group_t* g);

/* 1 when that one launch is replayed from a CUDA graph captured on the first
 * admm_group_iterate (per H mode; each call updates the graph node's
 * arguments), 0 when it is launched directly (before the first call, with
 * more than 48 problems, or where capture failed), -1 for NULL. */
int admm_group_uses_graph(const admm_group_t* g);

const char* admm_group_last_error(const admm_group_t* g);
void admm_group_destroy(admm_group_t* g);

/* ---------------------------------------------------------------------------
 * Batched shared-H solver.  `batch` independent scenes g_b (b = 0..batch-1)
 * with one sensing matrix H are iterated together under the same split: each
 * scene runs exactly the iteration of admm_iterate (Sections III-A..C, with
 * its own lambda_b), on the matrix the FP16 storage of H encodes
 * (ADMM_OPT_H_FP16: one power-of-two scale per 64-row group).  The products
 * H_ij z_j^i, K_ij^{-1} r_ij and H_ij^H w_ij of all scenes are GEMMs on the
 * tensor cores (tcgen05.mma, FP16 operands, FP32 accumulation): every
 * right-hand side is split into FP16 hi + lo parts after a power-of-two scale
 * per scene and block, so the products carry about 22 significant bits, and
 * the factors K^{-1} are split the same way.  The paper processes one scene;
 * the batch is this library's extension for many scenes with one H.
 * Vectors are scene-major complex64: G and Y batch x m, V and X batch x n.
 * ------------------------------------------------------------------------- */
typedef struct admm_batch admm_batch_t;

typedef struct admm_batch_info {
    int64_t m, n;
    int32_t batch, row_blocks, col_blocks;
    int32_t splits;           /* K splits of the forward product GEMM */
    int64_t iterations;
    double tensor_flops;      /* tensor-core FLOPs issued per iteration (tile padding included) */
    double method_flops;      /* 8 real FLOPs per complex multiply-add of the method, all scenes */
    double state_bytes;       /* bytes of state and packed operands moved per iteration */
} admm_batch_info_t;

/* Create a batched solver.  H (m x n, host or device, element type h_dtype)
 * is copied; lambda holds `batch` weights (host memory).  Requires m and every
 * block start to be multiples of 4 (16-byte TMA rows of the FP16 copy and of
 * its transpose), 1 <= batch <= 4096, and the shape limits of admm_setup.
 * The state starts at zero and G at zero (admm_batch_set_g).  Synchronises
 * `stream`.  On failure *out is NULL and admm_batch_last_error(NULL) says why. */
int admm_batch_setup(admm_batch_t** out, const void* H, int64_t m, int64_t n, int32_t row_blocks,
                     int32_t col_blocks, int32_t batch, const double* lambda, double rho, int32_t h_dtype,
                     void* stream);

/* Copy the batch x m measurements (complex64, host or device).  Synchronises. */
int admm_batch_set_g(admm_batch_t* h, const void* G, void* stream);

/* Run `iters` iterations for every scene (one CUDA graph launch each; the
 * graph is captured on the first call).  Asynchronous on `stream`. */
int admm_batch_iterate(admm_batch_t* h, int32_t iters, void* stream);

/* Copy the batch x n images v (complex64) into V (host or device). */
int admm_batch_get_v(admm_batch_t* h, void* V, void* stream);

/* ||r_p||^2 and ||r_d||^2 of the last iteration per scene (2 * batch doubles,
 * host), as in admm_get_residuals; synchronises and returns the device status. */
int admm_batch_get_residuals(admm_batch_t* h, double* out, void* stream);

/* Zero the state (v, s, estimated data) and the iteration count.  Synchronises. */
int admm_batch_reset(admm_batch_t* h, void* stream);

/* Y_b = Hq X_b for every scene with the tensor-core forward product, where Hq
 * is the matrix the FP16 storage encodes (the products of Eq. g_columns and of
 * the u-step); X is batch x n, Y batch x m.  Synchronises. */
int admm_batch_forward(admm_batch_t* h, const void* X, void* Y, void* stream);

/* X_b = Hq^H Y_b for every scene (the adjoint product of the u-step).  Synchronises. */
int admm_batch_adjoint(admm_batch_t* h, const void* Y, void* X, void* stream);

/* Autotune: time the forward product with every K split the partial-product
 * buffer allows (powers of two, at least 4 K blocks of 64 per split) on the
 * current state and keep the fastest for later iterations (the graph is
 * captured again).  The state is not changed.  Synchronises. */
int admm_batch_tune(admm_batch_t* h, void* stream);

/* Record the next `iters` iterations for admm_batch_backward: per iteration
 * the shrinkage arguments a = mean_i(u^i + s^i) (batch x n) and the factor
 * solutions w_ij = K_ij^{-1} r_ij (every block), all the reverse sweep needs,
 * since the soft-threshold is the iteration's only non-linear step.  0 turns
 * recording off.  Resets the state (admm_batch_reset) and synchronises. */
int admm_batch_record(admm_batch_t* h, int32_t iters);

/* Replace the per-scene weights lambda[b] >= 0 (`batch` doubles; no
 * refactorisation: kappa_b = lambda_b / (row_blocks rho)).  The iteration
 * state is kept; a recording made before is invalidated.  Synchronises the
 * device. */
int admm_batch_set_lambda(admm_batch_t* h, const double* lambda);

/* Replace rho > 0: refactors every block rho I + H_b H_b^H of the matrix the
 * FP16 copy encodes (as admm_set_rho does for a single handle), rescales the
 * scaled duals by rho_old / rho_new so the unscaled duals are kept, and
 * invalidates a recording.  Synchronises `stream`. */
int admm_batch_set_rho(admm_batch_t* h, double rho, void* stream);

/* Reverse sweep over the iterations run since the last reset (all recorded):
 * given dV = dL/dv (batch x n complex64, x_bar = dL/dRe x + i dL/dIm x) of a
 * real loss L of the image v after those iterations, write dG = dL/dg
 * (batch x m) and, per scene, dlambda = dL/dlambda_b and drho = dL/drho
 * (host doubles, batch each).  Every step is the adjoint of the iteration of
 * admm_batch_iterate: for |a| > kappa with a_hat = a/|a|, a_bar = t -
 * (kappa/|a|)(t - a_hat Re(conj(a_hat) t)) and kappa_bar = -Re(conj(a_hat) t)
 * (zero otherwise, Eq. softhresholding), and dw/drho = -K^{-1} w; the
 * products H sigma_bar, K^{-1} w_bar and H^H r_bar run on the tensor-core
 * GEMMs of the forward path.  Synchronises.  ADMM_EINVAL when the iterations
 * since the reset were not all recorded.  The paper has no counterpart. */
int admm_batch_backward(admm_batch_t* h, const void* dV, void* dG, double* dlambda, double* drho, void* stream);

/* Synchronise `stream` and return the sticky device status. */
int admm_batch_status(admm_batch_t* h, void* stream);

int admm_batch_get_info(const admm_batch_t* h, admm_batch_info_t* info);

/* Last failure on `h` (or of the last failed admm_batch_setup when h is NULL). */
const char* admm_batch_last_error(const admm_batch_t* h);

void admm_batch_destroy(admm_batch_t* h);

#ifdef __cplusplus
}
#endif

#endif /* ADMM_H */
