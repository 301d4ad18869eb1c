/*
 * mcinv.h -- C ABI of a GB300 (sm_103a) implementation of the correlated-chains
 * (CC) Monte Carlo inverse of Garcia-Cortes & Cabrillo, "A Monte Carlo
 * algorithm for efficient large matrix inversion".
 *
 * Method (Sec. 2): two vectors z and w are advanced by noisy Gauss-Seidel
 * sweeps that share their noise phi,
 *     Eq. 4:  z_i <- phi_i / sqrt(c_ii) - (1/c_ii)  sum_{j != i} c_ij  z_j
 *     Eq. 5:  w_i <- phi_i / sqrt(c*_ii) - (1/c*_ii) sum_{j != i} c*_ji w_j
 * with rows i ascending and in-place semantics (j < i sees the current
 * cycle, j > i the previous one).  After burn-in, the average of z w^dagger
 * estimates C^-1 (Eq. 1/C); its diagonal, a block of it, and tr(Q C^-1) for a
 * diagonal Q (Eq. tr) are the estimates this library returns.
 *
 * Conventions for every function below
 *  - Host pointers are plain host memory owned by the caller; the library
 *    copies what it needs and never keeps a caller pointer after returning.
 *  - Device memory is owned by the handle and freed by mcinv_destroy.
 *  - All GPU work is ordered on the stream given in mcinv_options.stream
 *    (NULL = the legacy default stream).  mcinv_burnin and mcinv_sample only
 *    enqueue work; mcinv_estimate, mcinv_get_state and mcinv_sync wait for it.
 *  - Every function returns an mcinv_status; nothing aborts or traps.  On
 *    error, mcinv_last_error(h) describes it.  After any error the handle can
 *    still be destroyed.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef MCINV_H
#define MCINV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcinv_ctx *mcinv_t;

typedef enum {
    MCINV_OK = 0,
    MCINV_E_ARG = 1,           /* invalid argument or malformed CSR */
    MCINV_E_SINGULAR_DIAG = 2, /* a c_ii is missing, zero or non-finite (D must be
                                  non-singular, Sec. 2.2) */
    MCINV_E_DIVERGED = 3,      /* a chain went non-finite or beyond 1e30: the sweep
                                  does not converge (sp(T) >= 1 or sp(S) >= 1, Sec. 2.2).
                                  The grid-wide and pool ring sweeps look at the last
                                  cycle of each launch (a diverging chain stays beyond
                                  the bound), the chain-sliced sweep at every cycle */
    MCINV_E_NOMEM = 4,         /* device memory could not be allocated */
    MCINV_E_CUDA = 5,          /* a CUDA runtime error; see mcinv_last_error */
    MCINV_E_TIMEOUT = 6,       /* a bounded device-side wait expired */
    MCINV_E_STATE = 7,         /* call not valid in the handle's current state */
    MCINV_E_UNSUPPORTED = 8    /* option not supported on this device/build */
} mcinv_status;

/* Value type of the host CSR given to mcinv_create. */
typedef enum {
    MCINV_REAL64 = 0,    /* val: double[nnz]; the sweep runs in FP32 */
    MCINV_COMPLEX128 = 1 /* val: double[2*nnz] interleaved re,im; the sweep runs in complex64 */
} mcinv_dtype;

/* How the block estimate accumulates z w^dagger. */
typedef enum {
    MCINV_ACC_FP32_SIMT = 0, /* FP32 CUDA-core contraction after every cycle */
    MCINV_ACC_BF16_TC = 1    /* BF16 operands on the tensor cores (tcgen05), FP32 accumulate,
                                over a batch of cycles at once */
} mcinv_acc;

typedef enum {
    MCINV_EST_BLOCK = 0, /* (C^-1)_{R[a], S[b]}: out [nR][nS] */
    MCINV_EST_DIAG = 1,  /* (C^-1)_{ii}: out [n] */
    MCINV_EST_TRACE = 2  /* tr(Q C^-1), Q = diag(q): out [1] */
} mcinv_kind;

typedef struct {
    int64_t K;              /* chains advanced in lockstep (>= 1) */
    uint64_t seed;          /* Philox key */
    int64_t chain_base;     /* global id of chain 0 (disjoint ranges shard work across GPUs) */
    uint32_t matrix_id;     /* Philox counter word 3; distinct per matrix in a batch */
    int32_t groups;         /* SE replicates G for diag/trace (chain groups); 0 = 32 */
    int32_t batch_cycles;   /* cycles per sweep launch / per block contraction; 0 = 8 */
    int32_t acc;            /* mcinv_acc for the block estimate */
    int32_t chains_per_cta; /* chain-slice width W per CTA: a power of two <= 128 (real) or
                               64 (complex); 0 = chosen by the library */
    int32_t threads_per_cta;/* 0 = chosen by the library (multiple of 32, <= 512) */
    int32_t flags;          /* MCINV_F_* bits */
    void *stream;           /* cudaStream_t; NULL = legacy default stream */
    const int64_t *block_rows; /* R (row indices of C^-1), may be NULL when n_block_rows = 0 */
    int64_t n_block_rows;
    const int64_t *block_cols; /* S (column indices of C^-1) */
    int64_t n_block_cols;
    int32_t ctas_per_slice; /* Q: CTAs of one thread-block cluster sharing a chain slice and
                               splitting each dependency level's rows (1..16); 0 = chosen by
                               the library */
    int32_t reserved;
} mcinv_options;

#define MCINV_F_NO_DIAG 1  /* do not accumulate the diagonal (and trace) */
#define MCINV_F_AUTOTUNE 2 /* when chains_per_cta, ctas_per_slice and threads_per_cta are all 0,
                              time the candidate slice shapes on this matrix for two cycles at
                              create time and keep the fastest (cached per n, nnz, K, type) */
#define MCINV_F_STAGED 8   /* real matrices: run the sweep whose producer warp stages the gathers in
                              shared memory (bulk copies on mbarriers) instead of the register
                              kernel; needs 16- or 32-chain slices and K a multiple of the slice
                              (MCINV_E_UNSUPPORTED otherwise).  MCINV_F_AUTOTUNE considers both. */
#define MCINV_F_GRID 16    /* run the sweep as one cooperative launch over every SM: a warp updates
                              one row for 32 x V chains (V = 4 real, 2 complex; a 512-byte segment
                              of z or w per gathered row), every CTA takes rows of every dependency
                              level, and a grid-wide barrier ends each level.  Same values, bit for
                              bit, as the chain-sliced kernel with 32 x V-chain slices.  Needs K a
                              multiple of V and one resident CTA per SM; threads_per_cta 384
                              (default) or 512, chains_per_cta and ctas_per_slice are ignored
                              (MCINV_E_UNSUPPORTED otherwise).  MCINV_F_AUTOTUNE without this flag
                              times it beside the chain-sliced shapes. */
#define MCINV_F_GRID_BULK 32 /* with MCINV_F_GRID: each warp stages its rows' gathered segments in a
                              ring of shared-memory slots with bulk asynchronous copies, up to three
                              rows in flight; a row longer than the ring runs in rounds.
                              threads_per_cta 384 (default: 12 warps of 32 slots), 192 or 96 (2 or
                              4 vectors a lane), or 512 (16 warps of 24 slots).  Same values, bit
                              for bit. */
#define MCINV_F_GRID_NOPAIR 64 /* with MCINV_F_GRID_BULK: keep z and w in separate buffers.  Without it,
                              for a structurally symmetric C (row i of C and of C^dagger name the
                              same columns) and threads_per_cta 0 the bulk sweep keeps the state
                              in the pair layout, a 32-vector chain block's z and w of a row side
                              by side, so one copy gathers both: 12 warps a CTA, each taking two
                              adjacent blocks (2 KB copies into 9 slots).  Readers of the state
                              (mcinv_get_state, the CUDA-core block accumulation) see the usual
                              layout.  Same values, bit for bit. */
#define MCINV_F_GRID_PAIR 128 /* with MCINV_F_GRID_BULK: the pair layout with the shape that
                              threads_per_cta names: 512 (16 warps, one block a warp, 12 slots of
                              1 KB), 384 (the default) or 256 (8 warps, two blocks a warp, 13 slots
                              of 2 KB).  MCINV_E_UNSUPPORTED when C is not structurally symmetric;
                              MCINV_E_ARG with MCINV_F_GRID_NOPAIR or another thread count. */
#define MCINV_F_GRID_TILE 256 /* with MCINV_F_GRID_BULK: the tile-staged sweep.  The positions of every
                              dependency level are cut into tiles of 64, 32, 16 or 8 consecutive
                              positions (the largest that fits); a CTA copies a tile's distinct
                              neighbours (at most 100 rows' 32-vector blocks of z and w, pair
                              layout) into shared memory once and its 16 warps update the tile's
                              rows from there, the next tile's copies in flight.  For lattices in
                              the colour order.  MCINV_E_UNSUPPORTED when C is not structurally
                              symmetric, a row is cut into pieces, or a tile would name more
                              neighbours; MCINV_E_ARG with MCINV_F_GRID_NOPAIR.  Same values, bit
                              for bit.  MCINV_F_AUTOTUNE times it where it applies. */
#define MCINV_F_GRID_WAVE 512 /* with MCINV_F_GRID_BULK: the wavefront sweep, for a C whose order has
                              two dependency levels of equal size (a lattice in the colour order:
                              red, then black) that cut into chunks of S consecutive positions
                              whose rows touch only the other level's chunks within B of their
                              own, cyclically.  Each CTA owns a slice of the chains (16, 8 or 4
                              vectors of 16 bytes) for whole cycles, with no grid barrier: it
                              updates red chunk t from black chunks t-B .. t+B copied into
                              shared memory once each, keeps the new red values there, then
                              updates black chunk t-B; the B black chunks at each end of the
                              cycle wait for its end.  A cycle reads the black half of the state
                              once and writes all of it once.  MCINV_E_UNSUPPORTED when C has no
                              such form (or its window does not fit a CTA's shared memory);
                              MCINV_E_ARG with MCINV_F_GRID_NOPAIR or MCINV_F_GRID_TILE.  Same
                              values, bit for bit, except the trace series' partial sums, which
                              are grouped by warp in another way.  MCINV_F_AUTOTUNE times it
                              where it applies. */
#define MCINV_F_TEST_EXPIRE_WAIT 1024 /* testing the bounded waits, with MCINV_F_GRID_WAVE only:
                              each launch's first stage is announced to its mbarrier but never
                              copied, so every CTA's wait for it expires (after 2 s), the CTAs
                              skip their rows and end the launch, and mcinv_sync reports
                              MCINV_E_TIMEOUT.  The state is then meaningless; the context and
                              other handles are unaffected.  MCINV_E_ARG without
                              MCINV_F_GRID_WAVE. */
#define MCINV_F_COLOR_ORDER 4 /* sweep the rows in the colour order of mcinv_color_order: the
                              handle samples C' = P C P^T (Sec. 4, reordering the rows and columns
                              of C), whose Gauss-Seidel sweep has one dependency level per colour.
                              E[z w^dagger] is then P C^-1 P^T; every row-indexed argument and
                              result (block rows and columns, q, the diagonal, the chain state)
                              stays in the rows of C as given.  The noise of C' row k is drawn
                              for row k, so the draws differ from the given order's.  Also a
                              pool flag (mcinv_pool_options.flags): every matrix of the pool. */

/*
 * The colour sweep order (Sec. 4: the paper's suggestion to reorder the rows and
 * columns of C).  Rows, in ascending index order, each take the smallest colour
 * not used by an already-coloured neighbour in the graph of C + C^T (off-diagonal
 * entries); order[k], k < n, lists colour 0's rows ascending, then colour 1's, and
 * so on, and *ncolors (may be NULL) receives the number of colours.  Host only: no
 * GPU is touched.  order is caller-owned, n entries.  Returns MCINV_E_ARG for a
 * malformed CSR or NULL order and MCINV_E_SINGULAR_DIAG for a missing diagonal.
 */
mcinv_status mcinv_color_order(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t *order,
                               int32_t *ncolors);

/* Fill *opt with defaults (K = 1024, seed = 0, everything else automatic). */
void mcinv_default_options(mcinv_options *opt);

/*
 * Create a sampler for the n x n sparse matrix C given in CSR form.
 *   row_ptr : int64[n+1], row_ptr[0] = 0, non-decreasing.
 *   col     : int32[nnz], strictly increasing within each row, in [0, n).
 *   val     : see mcinv_dtype.  Every row must hold its diagonal entry.
 * Validates the CSR on the host (MCINV_E_ARG), checks that D is non-singular
 * (MCINV_E_SINGULAR_DIAG), builds C^dagger and the Gauss-Seidel dependency
 * levels, uploads everything, and sets z = w = 0 for every chain (Algorithm 1,
 * step 1).  The per-row reciprocals 1/c_ii, 1/sqrt(c_ii) and 1/conj(sqrt(c_ii))
 * are formed on the GPU in FP64 and rounded once to the sweep precision.
 * On success *out is a new handle; on failure *out = NULL.
 */
mcinv_status mcinv_create(mcinv_t *out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const double *val, mcinv_dtype dt, const mcinv_options *opt);

/* Largest diagonal block of a partition (rows). */
#define MCINV_MAX_PARTITION_BLOCK 8

/*
 * Create a sampler that sweeps C block by block (Sec. 4: a partition of C into
 * small non-singular diagonal blocks, for matrices whose diagonal has zeros or
 * small entries).  block_ptr[0..nblocks] cuts the rows into contiguous blocks:
 * block b holds rows block_ptr[b] .. block_ptr[b+1]-1 (1 to
 * MCINV_MAX_PARTITION_BLOCK rows), block_ptr[0] = 0, block_ptr[nblocks] = n.
 * A block b of two or more rows is updated as a whole,
 *   z_b <- S_b^-1 phi_b - D_b^-1 sum_{c != b} C_bc z_c,
 *   w_b <- S_b^-H phi_b - D_b^-H sum_{c != b} (C^H)_bc w_c,
 * with S_b the principal square root of its diagonal block D_b, so that
 * S_b^-1 (S_b^-H)^H = D_b^-1, the block form of alpha_i conj(beta_i) = 1/c_ii in
 * Eqs. 4/5; a one-row block is a row of Eqs. 4/5.  Rows inside blocks of two or
 * more rows may lack a diagonal entry.  The block sweep is the row sweep of
 * C~ = S^-1 C S^-1 (S = blockdiag(S_b), 1 for one-row blocks) with z = S^-1 z~,
 * w = S^-H w~, which is how it runs on the GPU.  Options, estimates and the chain
 * state (mcinv_get_state returns the block sweep's z and w) are as for
 * mcinv_create, except that block_rows and block_cols may only name rows of
 * one-row blocks, the per-cycle trace series (mcinv_set_trace_weights,
 * mcinv_trace_series, mcinv_trace_mc_error, mcinv_sample_until) is
 * MCINV_E_UNSUPPORTED when a block has two or more rows, and
 * mcinv_burnin_coupled couples the paths of C~.  The arrays are the caller's.
 * Returns MCINV_E_ARG for a malformed partition and MCINV_E_SINGULAR_DIAG for a
 * block without a principal square root (singular, or an eigenvalue on the
 * closed negative real axis).
 */
mcinv_status mcinv_create_partitioned(mcinv_t *out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                      const double *val, mcinv_dtype dt, const mcinv_options *opt,
                                      int64_t nblocks, const int64_t *block_ptr);

/* Advance every chain `cycles` CC cycles (Eqs. 4, 5) without accumulating
 * (burn-in, Algorithm 1 steps 1-5 with a fixed count).  cycles >= 0. */
mcinv_status mcinv_burnin(mcinv_t h, int64_t cycles);

/*
 * Burn-in with the coupling test of Algorithm 1 (steps 1-5): the run length p
 * is the first cycle after which two paths started at z = w = 0 and at
 * z*_i = w*_i = i (1-based), sharing their noise, agree to max_i |z_i - z*_i| < tol
 * and max_i |w_i - w*_i| < tol (the paper's "z'z* < tol" read as this
 * sup-norm).  By Eq. 12 the difference follows noise-free Gauss-Seidel on C
 * (and on C^dagger), the same for every chain, so it is swept once as a
 * single chain; then every chain runs p burn-in cycles (as mcinv_burnin).
 * *cycles_out = p.  MCINV_E_DIVERGED if the paths still differ after
 * max_cycles cycles (sp(T) or sp(S) >= 1, or too tight a tol for FP32).
 */
mcinv_status mcinv_burnin_coupled(mcinv_t h, double tol, int64_t max_cycles, int64_t *cycles_out);

/* Advance every chain `cycles` cycles and accumulate each cycle's z w^dagger
 * into the diagonal / block estimates (Eq. 1/C; Algorithm 1 steps 6-9). */
mcinv_status mcinv_sample(mcinv_t h, int64_t cycles);

/*
 * Wait for queued work and return the current estimate and its Monte Carlo
 * standard error (Sec. 2.3) in FP64 host memory.
 *   DIAG : out[n]; TRACE: out[1] with q_diag = double[n] (Q = diag(q)).
 *   BLOCK: out[nR*nS] row-major over (R[a], S[b]).
 *   Complex matrices return interleaved re,im (twice the length); se_out has
 *   the same shape and holds the SE of the real and imaginary parts.
 *   se_out may be NULL.  DIAG/TRACE SE comes from independent chain groups,
 *   BLOCK SE from batch means over sampling batches.
 * MCINV_E_STATE if nothing was sampled or the estimate was not configured;
 * MCINV_E_DIVERGED if a chain diverged.
 */
mcinv_status mcinv_estimate(mcinv_t h, mcinv_kind kind, const double *q_diag, double *out,
                            double *se_out);

/*
 * Monte Carlo error of the trace by Geyer's effective length (Sec. 2.3, as the
 * paper's tables report it).  mcinv_set_trace_weights(h, q) (q[n], before any
 * sampling) makes every sampling cycle also record the realised value
 *     t_k = (1/K) sum_chains sum_i q_i Re(z_i conj(w_i))
 * (one FP64 value per cycle, reduced in a fixed order on the GPU).
 * mcinv_trace_mc_error returns its mean, variance gamma(0), Geyer's
 * initial-positive-sequence effective length and SE = sqrt(gamma(0) / ess).
 * mcinv_trace_series copies the series (up to capacity values).
 * mcinv_sample_until samples check_every cycles at a time until
 * SE < rel_tol * |mean| (the paper's stop rule, checked every 100 cycles there)
 * or max_cycles would be exceeded; *cycles_out = cycles sampled.
 */
mcinv_status mcinv_set_trace_weights(mcinv_t h, const double *q_diag);
mcinv_status mcinv_trace_mc_error(mcinv_t h, double *mean, double *var, double *ess, double *se);
mcinv_status mcinv_trace_series(mcinv_t h, double *out, int64_t capacity, int64_t *length);
mcinv_status mcinv_sample_until(mcinv_t h, double rel_tol, int64_t check_every, int64_t max_cycles,
                                int64_t *cycles_out);

/* Wait for queued work; report MCINV_E_DIVERGED / CUDA errors raised since the last check. */
mcinv_status mcinv_sync(mcinv_t h);

/*
 * Copy chains [chain0, chain0+nchains) of the current z and w to host memory
 * as double [n][nchains] (complex: interleaved, [n][nchains][2]); *cycle gets
 * the number of cycles run so far.  z, w, cycle may each be NULL.
 */
mcinv_status mcinv_get_state(mcinv_t h, int64_t chain0, int64_t nchains, double *z, double *w,
                             int64_t *cycle);

/* Overwrite all chains' z and w (same layout as mcinv_get_state with chain0 = 0,
 * nchains = K) and set the cycle counter; accumulated estimates are cleared.
 * Resuming from a saved state reproduces the uninterrupted run bit for bit. */
mcinv_status mcinv_set_state(mcinv_t h, const double *z, const double *w, int64_t cycle);

/* Clear the accumulated estimates (diagonal, trace, block) and the sample count. */
mcinv_status mcinv_reset_estimates(mcinv_t h);

typedef struct {
    int64_t n, nnz, K;
    int32_t is_complex;
    int32_t chains_per_cta;  /* W */
    int32_t threads_per_cta;
    int32_t slices;          /* chain slices = ceil(K / W) */
    int32_t ctas_per_slice;  /* Q: the sweep launches slices x Q CTAs */
    int32_t chains_per_lane; /* vector width of one lane's chains (1, 2 or 4) */
    int32_t groups;          /* G actually used (divides slices) */
    int32_t levels;          /* Gauss-Seidel dependency levels of C and C^dagger */
    int32_t batch_cycles;
    int32_t acc;
    int64_t cycle;           /* cycles run so far */
    int64_t samples;         /* cycles accumulated so far */
    int64_t block_batches;   /* batches folded into the block estimate */
    int64_t kernel_launches; /* kernels this handle has launched */
    int64_t device_bytes;    /* device memory held by the handle */
    int32_t sweep_kernel;    /* 0: chain-sliced (registers), 1: staged, 2: grid-wide (MCINV_F_GRID),
                                3: grid-wide with bulk-staged gathers (MCINV_F_GRID_BULK),
                                4: the same on the pair layout (structurally symmetric C),
                                5: the tile-staged sweep (MCINV_F_GRID_TILE),
                                6: the wavefront sweep (MCINV_F_GRID_WAVE) */
    int32_t grid_ctas;       /* CTAs of the grid-wide sweep, or of the wavefront sweep (one a chain
                                slice); 0 for the others */
} mcinv_info_t;

mcinv_status mcinv_info(mcinv_t h, mcinv_info_t *info);

/* Kernel classes for per-kernel timing. */
typedef enum {
    MCINV_KERNEL_NOISE = 0,    /* Philox noise plane */
    MCINV_KERNEL_SWEEP = 1,    /* coupled sweep of Eqs. 4/5 (with fused diagonal partials) */
    MCINV_KERNEL_BLOCK = 2,    /* block contraction z w^dagger (tensor-core or SIMT) */
    MCINV_KERNEL_FOLD = 3,     /* FP64 folds of the diagonal / block batches */
    MCINV_KERNEL_ESTIMATE = 4, /* mean / standard-error kernels */
    MCINV_KERNEL_CLASSES = 5
} mcinv_kernel;

/*
 * Per-kernel timing.  mcinv_profile(h, 1) starts bracketing every launch of
 * the handle with CUDA events on its stream (and clears earlier totals);
 * mcinv_profile(h, 0) stops.  mcinv_profile_read waits for the stream and
 * returns, for one kernel class, the launches recorded and the summed
 * event-to-event time in milliseconds.
 */
mcinv_status mcinv_profile(mcinv_t h, int enable);
mcinv_status mcinv_profile_read(mcinv_t h, mcinv_kernel kernel, int64_t *launches, double *ms);

/*
 * Diagnostic: run the tensor-core contraction used by the block estimate,
 * D = A B^T, on host data.  A: M x inner and B: N x inner, row-major BF16 bit
 * patterns; D: M x N row-major FP32.  Allocates and frees its own device
 * memory on the legacy default stream and waits for the result.
 * MCINV_E_UNSUPPORTED off sm_103a.
 */
mcinv_status mcinv_selftest_tc_gemm(int64_t M, int64_t N, int64_t inner, const uint16_t *A,
                                    const uint16_t *B, float *D);

/* ------------------------------------------------------------------------ */
/* Pool: many independent real matrices advanced together (the batched form) */
/* with continuous batching.                                                  */
/* ------------------------------------------------------------------------ */
typedef struct mcinv_pool_ctx *mcinv_pool_t;

typedef struct {
    int64_t K;              /* chains per matrix, a multiple of 4 */
    uint64_t seed;          /* Philox key shared by all matrices (each has its own matrix id) */
    int64_t chain_base;
    int64_t mem_budget;     /* bytes of device memory reserved for the pool (one arena) */
    int32_t max_slots;      /* matrices resident at once */
    int32_t batch_cycles;   /* B: cycles every matrix advances per step; 0 = 8 */
    int32_t groups;         /* SE groups of the diagonal; 0 = 32 */
    int32_t fold_steps;     /* F: sampling steps whose block products are summed in FP32 before
                               each FP64 fold, so a block batch (for the batch-means SE) is the
                               sampling cycles of F steps (fewer at a member's end); 0 = 8, at
                               most 1024 */
    int32_t chains_per_cta; /* 0 = the first steps time the candidate shapes; 4 x a power of two
                               <= 128 (a chain slice per CTA; 128 with 384 or 512 threads: the
                               bulk-staged ring form), or 256 (the ring form, two vectors a lane,
                               384 threads) */
    int32_t threads_per_cta;
    int32_t flags;
    void *stream;
} mcinv_pool_options;

typedef struct {
    int64_t K, steps, kernel_launches, arena_bytes, arena_used;
    int32_t chains_per_cta, threads_per_cta, groups, batch_cycles, active, tuned, fold_steps;
} mcinv_pool_info_t;

void mcinv_pool_default_options(mcinv_pool_options *opt);

/* Reserve the pool's device arena (mem_budget bytes, one allocation) and its
 * tables.  Every later device buffer of a member comes out of the arena. */
mcinv_status mcinv_pool_create(mcinv_pool_t *out, const mcinv_pool_options *opt);

/* Device bytes a real matrix with n rows and nnz entries would take (an upper
 * estimate before preparing it). */
mcinv_status mcinv_pool_footprint(mcinv_pool_t p, int64_t n, int64_t nnz, int32_t want_inverse, int64_t *bytes);

/*
 * Admit a real matrix (CSR as for mcinv_create) that will run `burnin` cycles
 * and then `samples` sampling cycles (Algorithm 1 with a fixed burn-in),
 * accumulating its diagonal and, if want_inverse, the full inverse (Eq. 1/C).
 * matrix_id keys its noise (Philox counter word 3).  Returns a ticket.
 * MCINV_E_NOMEM when no slot is free or the arena cannot hold it: the caller
 * keeps the request and submits it again after members are released.
 */
mcinv_status mcinv_pool_submit(mcinv_pool_t p, int64_t n, const int64_t *row_ptr, const int32_t *col,
                               const double *val, uint32_t matrix_id, int64_t burnin, int64_t samples,
                               int32_t want_inverse, int64_t *ticket);

/* Advance every admitted, unfinished matrix by one step of B cycles (their
 * own mix of burn-in and sampling).  Enqueues work on the pool's stream; a
 * step is a replay of one CUDA graph once the slice shape is chosen. */
mcinv_status mcinv_pool_step(mcinv_pool_t p);

/* *done = 1 once the ticket's matrix has run all its cycles. */
mcinv_status mcinv_pool_poll(mcinv_pool_t p, int64_t ticket, int32_t *done);

/* Estimates of one member, as mcinv_estimate (real only; BLOCK = the full
 * n x n inverse when want_inverse was set). */
mcinv_status mcinv_pool_estimate(mcinv_pool_t p, int64_t ticket, mcinv_kind kind, const double *q_diag,
                                 double *out, double *se_out);

/* Chain state of one member, as mcinv_get_state (test hook). */
mcinv_status mcinv_pool_get_state(mcinv_pool_t p, int64_t ticket, int64_t chain0, int64_t nchains, double *z,
                                  double *w, int64_t *cycle);

/* Free a member's slot and arena memory (waits for queued work first). */
mcinv_status mcinv_pool_release(mcinv_pool_t p, int64_t ticket);

mcinv_status mcinv_pool_info(mcinv_pool_t p, mcinv_pool_info_t *info);
mcinv_status mcinv_pool_sync(mcinv_pool_t p);
void mcinv_pool_destroy(mcinv_pool_t p);
const char *mcinv_pool_last_error(mcinv_pool_t p);

/* ------------------------------------------------------------------------ */
/* Server: estimate requests on a pool, admitted by device memory, run with  */
/* continuous batching by one engine thread.                                */
/* ------------------------------------------------------------------------ */
typedef struct mcinv_server_ctx *mcinv_server_t;

typedef struct {
    int64_t completed, queued, running, steps;
    double p50_ms, p99_ms, max_ms; /* submission-to-result latency of completed requests */
    double elapsed_s, busy_s;      /* since creation / last reset; time spent stepping */
} mcinv_server_stats_t;

/* Create a pool with these options and start its engine thread. */
mcinv_status mcinv_server_create(mcinv_server_t *out, const mcinv_pool_options *opt);

/*
 * Queue an estimate request (thread-safe; returns at once).  The CSR (real) is
 * copied.  kind: DIAG (out[n]), TRACE (out[1], q_diag[n] copied) or BLOCK (the
 * full n x n inverse).  The engine admits requests in arrival order while a
 * slot and arena memory are free, runs `burnin` + `samples` cycles of the
 * matrix alongside every other admitted request, then reads the estimate back
 * and releases the slot.
 */
mcinv_status mcinv_server_submit(mcinv_server_t s, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                 const double *val, uint32_t matrix_id, int64_t burnin, int64_t samples,
                                 mcinv_kind kind, const double *q_diag, int64_t *request);

/* Block until the request is done (MCINV_E_TIMEOUT after timeout_s seconds),
 * copy its estimate and SE (sized by its kind) and its latency in ms. */
mcinv_status mcinv_server_wait(mcinv_server_t s, int64_t request, double timeout_s, double *out, double *se_out,
                               double *latency_ms);

mcinv_status mcinv_server_stats(mcinv_server_t s, mcinv_server_stats_t *stats);
mcinv_status mcinv_server_reset_stats(mcinv_server_t s);
const char *mcinv_server_last_error(mcinv_server_t s);
/* Stop the engine (requests still queued or running are abandoned) and free everything. */
void mcinv_server_destroy(mcinv_server_t s);

/*
 * One batch of the block accumulation that allocates nothing.  The paper has
 * no counterpart: this exists for callers that cannot allocate device memory,
 * such as a serving process that reserves all device memory up front in its
 * own arena, or code that cannot take the device-wide synchronisation that
 * cudaMalloc and cudaFree imply in the middle of its work.
 *
 * On caller memory it computes D = A B^T on the tensor cores (BF16 operands,
 * FP32 accumulation) and folds it into FP64 accumulators:
 *     sum[e] += D[e],  sq[e] += D[e]^2 * scale_sq,   e < M*N (row-major M x N).
 *   A: M rows of `inner` BF16 bit patterns, row stride lda elements; B: N rows,
 *   stride ldb.  Device pointers owned by the caller; A and B start on 16-byte
 *   boundaries, lda and ldb are multiples of 8 and >= inner.  sum, sq: FP64,
 *   M*N each.  stream: cudaStream_t (NULL = legacy default stream).
 * The FP32 product D lives in a fixed 8 MiB array inside the library, so
 * M*N <= 2^21 (larger sizes return MCINV_E_ARG); every GPU that loads the
 * library holds that array until the process exits.  All calls share it and
 * it keeps the last call's product (the product is overwritten whole, so
 * nothing needs clearing): calls whose work overlaps on the GPU -- different
 * streams or host threads -- race; calls on one stream do not.  The first call
 * on a device looks up the array's device address with that device current.
 * The address is kept until the process exits, so do not use this entry
 * point across a cudaDeviceReset.
 * The call waits for its stream before returning.  No cudaMalloc, cudaFree or
 * other allocation.  On failure *error (when error is not NULL) points to a
 * static message.  MCINV_E_UNSUPPORTED off sm_103a; MCINV_E_TIMEOUT if a
 * bounded wait in the contraction expired, in which case sum and sq are left
 * unchanged (the fold is skipped).
 */
mcinv_status mcinv_block_accumulate_noalloc(int64_t M, int64_t N, int64_t inner, const uint16_t *A,
                                            int64_t lda, const uint16_t *B, int64_t ldb,
                                            double scale_sq, double *sum, double *sq, void *stream,
                                            const char **error);

/* Free everything the handle owns.  NULL is allowed. */
void mcinv_destroy(mcinv_t h);

/* Description of the last error on h (or of the last failed mcinv_create when
 * h is NULL, per host thread).  Never NULL. */
const char *mcinv_last_error(mcinv_t h);

#ifdef __cplusplus
}
#endif

#endif /* MCINV_H */
