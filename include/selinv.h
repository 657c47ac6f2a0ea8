/*
 * selinv.h -- C ABI of a GB300 (sm_103a) supernodal selected-inversion library.
 *
 * Problem (Alg. 1 and Alg. 2 of Jacquelin, Lin, Jia, Zhao, Yang,
 * "A left-looking selected inversion algorithm and task parallelism on shared
 * memory systems"): given a sparse symmetric or complex symmetric matrix A
 * (already symmetrically permuted) with supernodal factorization
 * A = L D L^T, compute the entries of A^{-1} on the pattern of L + L^T
 * ("selected elements of A^{-1} such that L_{I,J} is not an empty block",
 * output of Alg. 1), by the root-to-leaf elimination-tree recursion
 *     A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat_{C,K},   Lhat_{C,K} = L_{C,K} L_{K,K}^{-1}
 *     A^{-1}_{K,K} = L_KK^{-T} D_K^{-1} L_KK^{-1} - Lhat_{C,K}^T A^{-1}_{C,K}
 * with the diagonal block symmetrized (Sec. II-C).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Integers: column/row indices int32, offsets int64.
 *  - Supernode K has s_K columns super_ptr[K] .. super_ptr[K+1]-1 and a row
 *    list rows(K) = its own s_K columns followed by its c_K rows C below them,
 *    ascending (C = {I > K : L_{I,K} != 0} of Alg. 1 at the element level).
 *  - Panel layout ("panels"): supernode K owns a column-major (s+c) x s block
 *    with leading dimension s+c whose rows are rows(K); panels follow each
 *    other in supernode order; selinv_plan_panel_offset(K) gives the first
 *    element.  L, the cotangents and A^{-1} all use this layout.
 *      L: the diagonal block is unit lower triangular; its diagonal and
 *         strictly upper part are never read.
 *      A^{-1}: the diagonal block is written in full (symmetric), rows s..
 *         hold A^{-1}_{C,K}; together this is the lower part of A^{-1} on the
 *         pattern of L, the upper part being its transpose.
 *  - Transposes are plain for complex symmetric matrices (A = A^T), as the
 *    configured workloads are complex symmetric, not Hermitian.
 *  - Element types: SELINV_F64 = double, SELINV_C128 = two doubles (re, im)
 *    of a complex symmetric matrix (A = A^T), SELINV_C128H = the same storage
 *    for a complex Hermitian matrix (A = A^H, the variant of Sec. II-C with
 *    conjugate transposes: A = L D L^H with real D, Dinv_K = L_KK^{-H}
 *    D_K^{-1} L_KK^{-1}, A^{-1}_KK = Dinv_K - Lhat^H A^{-1}_{C,K}
 *    symmetrized as (X + X^H)/2, and the upper part of A^{-1} is the
 *    conjugate of the stored lower part).
 *  - Device pointers are caller-owned (the library never frees them) and must
 *    be 16-byte aligned.  Host arrays passed in are copied; the caller keeps
 *    ownership.
 *  - Numeric calls are asynchronous on the given cudaStream_t (passed as
 *    void*; NULL = legacy default stream).  Errors found on the device
 *    (timeouts of bounded waits, zero pivots, non-finite values) are latched
 *    in a per-plan status word read by selinv_status() after synchronizing.
 *  - Every call returns SELINV_OK (0) or a negative error code.
 */
#ifndef SELINV_H
#define SELINV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SELINV_OK 0
#define SELINV_ERR_INVALID_ARG (-1)
#define SELINV_ERR_BAD_ETREE (-2)    /* parent index not > child, or out of range   */
#define SELINV_ERR_BAD_PATTERN (-3)  /* rows not sorted / not closed under the tree */
#define SELINV_ERR_ZERO_PIVOT (-4)
#define SELINV_ERR_NONFINITE (-5)
#define SELINV_ERR_OOM (-6)
#define SELINV_ERR_CUDA (-7)
#define SELINV_ERR_TIMEOUT (-8)      /* a bounded device wait ran out              */
#define SELINV_ERR_UNSUPPORTED (-9)
#define SELINV_ERR_BAD_INDEX (-10)   /* a gather address fell outside the panels (debug_checks bit 2) */

typedef struct selinv_plan_s *selinv_plan;          /* opaque, owned by the library */
typedef struct selinv_analysis_s *selinv_analysis;  /* opaque, owned by the library */

typedef enum { SELINV_F64 = 0, SELINV_C128 = 1, SELINV_C128H = 2 } selinv_dtype;

typedef enum {
    SELINV_SCHED_PLAIN = 0,      /* one launch chain per supernode, K = N..1            */
    SELINV_SCHED_LEVEL = 1,      /* one grouped launch per elimination-tree level        */
    SELINV_SCHED_PERSISTENT = 2, /* one persistent launch, per-supernode completion flags;
                                    its traversal runs the FP64 / complex DFMA kernel
                                    whatever fast_contraction says                     */
    SELINV_SCHED_PUSH = 3        /* the left-looking form of Alg. 2, level by level from
                                    the root: each finished supernode pushes its outer-
                                    and inner-product updates into the descendants whose
                                    C meets its columns (DFMA, every fast_contraction) */
} selinv_schedule;

typedef struct {
    int symmetrize;        /* 1: A^{-1}_KK <- (X + X^T)/2 (Sec. II-C); default 1        */
    int schedule;          /* selinv_schedule; default SELINV_SCHED_LEVEL               */
    int autotune;          /* 1: the first selinv_numeric call per element type times the
                              tensor engine, split_target, split_min_steps and oz_min_s
                              candidates on the caller's data (synchronizing), keeps the
                              fastest for the plan (read back: selinv_plan_get_opts);
                              default 0                                                 */
    int debug_checks;      /* bit 0: scan inputs for non-finite values; bit 1: the
                              persistent schedule waits on a flag that is never set,
                              so every wait runs out (tests the timeout path); bit 2:
                              every address of the gather of A^{-1}_{C,C} is checked
                              against the panel array before the load: one outside it
                              is read as zero and latches SELINV_ERR_BAD_INDEX (no trap,
                              the results are then invalid); default 0                 */
    long long spin_limit;  /* polls (about 256 ns each) of every device spin-wait before
                              it gives up and latches SELINV_ERR_TIMEOUT; default 1<<22 */
    int use_graph;         /* 1: capture the level schedule in a CUDA graph; default 1  */
    int fast_contraction;  /* contraction of the supernodes with s >= oz_min_s: FP64-exact
                              on fp16 tensor cores (error-free slicing into 8-bit digits,
                              exact integer accumulation) -- 1: tcgen05 with tensor-memory
                              accumulators (default; real, complex symmetric and Hermitian
                              values), 2: mma.sync (real values only); 0: FP64 DFMA only */
    int split_target;      /* level schedule: k-splits of the contraction aim at this many
                              CTAs per SM on narrow levels (1..8); default 2           */
    int split_min_steps;   /* smallest k-range of a split item, in 16-row steps (8..64,
                              a multiple of 8); default 16                              */
    int oz_min_s;          /* narrowest supernode (columns) that uses the tensor-core
                              contraction (1..128); default 16                          */
} selinv_opts;

/* Fills *opts with the defaults listed above. */
void selinv_default_opts(selinv_opts *opts);

/* ---------------------------------------------------------------------------
 * Symbolic analysis (prerequisite; Sec. II-A supernodes, Sec. I/II-B tree).
 * From the lower triangle of the (already permuted) matrix, CSC with rows
 * ascending and row >= column: elimination tree, the column structure of L,
 * and the supernode partition.
 *   kind 0: fundamental supernodes of at most `cap` columns.
 *   kind 1: fundamental, then relaxed: the group ending at supernode K merges
 *           into K+1 when K+1 is its parent, the merged group has <= cap
 *           columns and explicit zeros <= fill x its stored lower entries.
 * Results are read with selinv_analysis_get:
 *   field 0 parent[n] (int32, column etree), 3 super_ptr[nsuper+1] (int32),
 *   4 sparent[nsuper] (int32), 5 rowptr[nsuper+1] (int64), 6 rows (int32),
 *   7 -> returns nsuper, 8 -> returns nnz of L without relaxation.
 * selinv_analysis_get returns the element count of the field (or the value
 * for 7/8) and copies it to dst when dst != NULL; <0 on a bad field.
 * Errors: INVALID_ARG (n < 0, cap < 1, null pointers), BAD_PATTERN (a row
 * index < its column or >= n, or unsorted), OOM.
 * ------------------------------------------------------------------------- */
int selinv_analyse(int32_t n, const int64_t *colptr, const int32_t *rowind, int kind,
                   int32_t cap, double fill, selinv_analysis *out);
int64_t selinv_analysis_get(selinv_analysis a, int field, void *dst);
void selinv_analysis_destroy(selinv_analysis a);

/* ---------------------------------------------------------------------------
 * selinv_symbolic: build the device-resident plan (Alg. 1 "find the
 * collection of indices C", made explicit once): elimination-tree level sets,
 * the split of every C into runs owned by one ancestor supernode, relative
 * row indices of C inside each owner's row list (the gather lists of
 * A^{-1}_{C,C}), work-item tables, and the scratch buffers of the numeric
 * phase.  Host arrays (copied):
 *   n, nsuper; super_ptr[nsuper+1] (super_ptr[0] = 0, increasing,
 *   super_ptr[nsuper] = n); sparent[nsuper] (supernodal etree parent, -1 =
 *   root, sparent[K] > K); rowptr[nsuper+1] (int64 offsets into rowind);
 *   rowind: rows(K) as described above.
 * opts may be NULL (defaults).  The plan lives on the current CUDA device.
 * Errors: INVALID_ARG, BAD_ETREE (sparent[K] <= K or >= nsuper, or the first
 * row below K not owned by sparent[K]), BAD_PATTERN (rows(K) not starting
 * with K's columns, not ascending, or some C entry of K missing from the row
 * list of its owner: the closure property the recursion relies on),
 * UNSUPPORTED (a supernode wider than SELINV_MAX_SUPERNODE columns), OOM, CUDA.
 * ------------------------------------------------------------------------- */
#define SELINV_MAX_SUPERNODE 128
int selinv_symbolic(int32_t n, int32_t nsuper, const int32_t *super_ptr, const int32_t *sparent,
                    const int64_t *rowptr, const int32_t *rowind, const selinv_opts *opts,
                    selinv_plan *out_plan);

/* Releases the plan and all device memory it owns.  NULL is ignored. */
void selinv_plan_destroy(selinv_plan plan);

/* Number of panel elements (= elements of L, of A^{-1}, of every cotangent). */
int64_t selinv_plan_nnz(selinv_plan plan);
/* First element of supernode K's panel; -1 if K is out of range. */
int64_t selinv_plan_panel_offset(selinv_plan plan, int32_t K);
/* Algorithmic work of one selected inversion: flops F = sum_K 2c^2s + 2cs^2 +
 * cs^2 + s^3 (real; complex work is 4x), bytes B = sum_K w (c(c+1)/2 +
 * 2(c+s)s + s) with w = 8 (f64) or 16 (c128).  Either pointer may be NULL. */
int selinv_plan_stats(selinv_plan plan, selinv_dtype dtype, double *flops, double *bytes);
/* Copies one host-side plan array (for inspection and tests):
 *   0 level[nsuper] int32 (root 0)   1 seg_ptr[nsuper+1] int64
 *   2 seg_owner int32   3 seg_start int32   4 seg_coloff int32
 *   5 rel_ptr[nseg+1] int64          6 relidx int32
 *   7 level_ptr[nlevels+1] int64     8 level_list[nsuper] int32
 *   9 panel_off[nsuper+1] int64
 *  10 active[nsuper] int32: 1 if the supernode runs under the current
 *     subset selection (selinv_plan_select), else 0
 *  11 colbase[rowptr[nsuper]] int64, 12 relbase[rowptr[nsuper]] int64: per
 *     row-list position rowptr[K]+s+q (q-th row of C_K), the panel element of
 *     column C_K[q] in its owner J's panel and the offset into relidx such
 *     that relidx[relbase + p] is the row of C_K[p] in rows(J), p >= q; zero
 *     at the positions of K's own columns
 * Returns the element count, or <0 on a bad field.  dst may be NULL. */
int64_t selinv_plan_get(selinv_plan plan, int field, void *dst);
/* The plan's current options (after autotuning: the chosen ones). */
int selinv_plan_get_opts(selinv_plan plan, selinv_opts *opts);

/* Changes the schedule / options of an existing plan. */
int selinv_plan_set_opts(selinv_plan plan, const selinv_opts *opts);

/* ---------------------------------------------------------------------------
 * selinv_numeric: the selected inversion itself (Alg. 1 with the
 * normalization of its first loop, symmetrization of Sec. II-C).
 *   L_dev   panels of L (unit-lower diagonal blocks), device
 *   D_dev   [n] diagonal of D, device
 *   Ainv_dev panels, device, caller-allocated (selinv_plan_nnz elements);
 *            every element is written.
 * Not reentrant per plan: calls on one plan must not overlap on the GPU
 * (they share the plan's scratch); use one plan per concurrent stream.
 * Errors: INVALID_ARG, CUDA; device-side errors via selinv_status.
 * ------------------------------------------------------------------------- */
int selinv_numeric(selinv_plan plan, selinv_dtype dtype, const void *L_dev, const void *D_dev,
                   void *Ainv_dev, void *cuda_stream);

/* The same selected inversion (Alg. 1) with host inputs and output: L and D
 * are copied in and A^{-1} out, the copies overlapped with the traversal.
 * The top levels' panels of L go first (the traversal starts on them while
 * the rest is copied; the lower levels' normalization waits for it), and the
 * panels of A^{-1} come back in groups of levels as soon as the traversal has
 * passed them (a panel is final once its level is done).
 *   L_host, D_host, Ainv_host  host buffers of selinv_plan_nnz / n /
 *            selinv_plan_nnz elements, same layouts as above; pinned memory
 *            for the copies to overlap (pageable memory works, serialized);
 *            caller-owned, not touched after the stream reaches the end of
 *            the call's work (Ainv_host is complete then).
 *   L_dev, D_dev, Ainv_dev  device staging buffers of the same sizes,
 *            caller-allocated (the call allocates nothing on the device
 *            beyond the plan's scratch).
 * Two copy streams of the plan run beside cuda_stream and are joined into it:
 * synchronizing cuda_stream covers the whole call.  A call that autotunes,
 * scans its inputs (debug_checks bit 0) or uses another schedule than the
 * level one copies everything in, inverts and copies everything out on
 * cuda_stream.  Not for a stream under capture (INVALID_ARG).
 * Errors: INVALID_ARG, CUDA; device-side errors via selinv_status. */
int selinv_numeric_host(selinv_plan plan, selinv_dtype dtype, const void *L_host, const void *D_host,
                        void *Ainv_host, void *L_dev, void *D_dev, void *Ainv_dev, void *cuda_stream);

/* Batched selected inversion: nitems independent problems (e.g. pole shifts
 * A - z_l S sharing one pattern, or different matrices), all tree levels of
 * all items merged into one level-scheduled (or persistent) launch sequence.
 * plans[i] may repeat.  Arrays are host arrays of device pointers.  The
 * batch's schedule comes from plans[0]'s options. */
int selinv_numeric_batched(int nitems, const selinv_plan *plans, const selinv_dtype *dtypes,
                           const void *const *L, const void *const *D, void *const *Ainv,
                           void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Prerequisite factorization A = L D L^T without pivoting (Sec. IV uses a
 * supernodal factorization with a symmetric permutation and no dynamic
 * pivoting).  The matrix pattern must first be attached to the plan:
 * selinv_plan_set_matrix(plan, n, colptr, rowind) with the same lower CSC
 * given to selinv_analyse (host arrays, copied).  A_vals_dev holds the values
 * of that CSC on the device.  Writes L (panels) and D.  A zero pivot latches
 * SELINV_ERR_ZERO_PIVOT in the status word (the factors are then invalid).
 * ------------------------------------------------------------------------- */
int selinv_plan_set_matrix(selinv_plan plan, int32_t n, const int64_t *colptr,
                           const int32_t *rowind);
int selinv_factor(selinv_plan plan, selinv_dtype dtype, const void *A_vals_dev, void *L_dev,
                  void *D_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Reverse mode (no counterpart in the paper; the chain rule through the
 * steps of Alg. 1 taken leaves-to-root, recomputing the gathers of
 * A^{-1}_{C,C}).  F64 only.
 *   selinv_adjoint: given the cotangent Ainv_bar of every panel slot that
 *     selinv_numeric writes (panels: the lower entries and the strictly upper
 *     part of the diagonal blocks, which holds the mirrored lower entries; a
 *     cotangent on an upper slot counts for its lower mirror, so a caller
 *     that differentiates only the lower entries passes zeros there),
 *     returns L_bar (panels, strictly lower entries) and D_bar [n].  Uses the
 *     forward outputs L, D, Ainv.  Ainv_bar is not modified (the plan keeps a
 *     working copy).
 *   selinv_factor_adjoint: given L_bar, D_bar, returns A_bar on the stored
 *     lower entries of A's CSC pattern (attached by selinv_plan_set_matrix):
 *     the derivative with respect to each stored lower entry a_ij (i >= j) of
 *     the symmetric matrix.
 * ------------------------------------------------------------------------- */
int selinv_adjoint(selinv_plan plan, selinv_dtype dtype, const void *L_dev, const void *D_dev,
                   const void *Ainv_dev, const void *Ainv_bar_dev, void *L_bar_dev,
                   void *D_bar_dev, void *cuda_stream);
int selinv_factor_adjoint(selinv_plan plan, selinv_dtype dtype, const void *L_dev,
                          const void *D_dev, const void *L_bar_dev, const void *D_bar_dev,
                          void *A_bar_vals_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * selinv_numeric_lu: Alg. 1 for nonsymmetric values on the symmetric pattern
 * (A = L U without pivoting, U kept separately, Sec. II-B; the factors come
 * from the caller, as the paper's come from an external sparse LU):
 *   Lhat_{C,K} = L_{C,K} L_KK^{-1},  Uhat_{K,C} = U_KK^{-1} U_{K,C},
 *   A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat_{C,K},  A^{-1}_{K,C} = -Uhat_{K,C} A^{-1}_{C,C},
 *   A^{-1}_{K,K} = U_KK^{-1} L_KK^{-1} - Uhat_{K,C} A^{-1}_{C,K}  (no symmetrization).
 *   L_dev   panels of L (unit lower diagonal blocks), as for selinv_numeric
 *   Ut_dev  U transposed in the same panel layout: the diagonal block holds
 *           U_KK^T (lower triangle with U's diagonal; the strict upper part is
 *           never read), rows s.. hold U_{K,C}^T
 *   Zl_dev  out: full diagonal blocks A^{-1}_KK and A^{-1}_{C,K} below them
 *   Zu_dev  out: (A^{-1}_KK)^T and A^{-1}_{K,C}^T below them
 * SELINV_F64 or SELINV_C128 (plain transposes), FP64 / complex FMA kernels,
 * level schedule (the plain one when the plan's options ask for it).  A zero
 * U_kk latches SELINV_ERR_ZERO_PIVOT.
 * ------------------------------------------------------------------------- */
int selinv_numeric_lu(selinv_plan plan, selinv_dtype dtype, const void *L_dev, const void *Ut_dev,
                      void *Zl_dev, void *Zu_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Subset selection (Sec. I: the selected elements may be all or only a
 * subset of the nonzero entries of the factors -- e.g. the diagonal of
 * A^{-1}, or the entries on A's own pattern).  Alg. 1 computes supernode K
 * from its ancestors' blocks only, so the supernodes that must run are the
 * owners of the selected columns and all their ancestors; the other
 * subtrees are skipped.
 *   selinv_plan_select: nsel entries (rows[e], cols[e]) of the permuted
 *     matrix (host arrays, copied; an upper entry is taken as its symmetric
 *     lower one).  Every entry must lie on the pattern of L + L^T, else
 *     BAD_PATTERN and the plan is unchanged; indices out of range give
 *     INVALID_ARG.  Later selinv_numeric / selinv_numeric_batched calls on
 *     this plan run only the needed supernodes: the panels of the others are
 *     not written.  nsel = 0 restores the full inversion.  pos_out (host,
 *     nsel entries, may be NULL) receives each entry's panel position.
 *     selinv_adjoint needs every block of A^{-1} and returns UNSUPPORTED
 *     while a selection is set.
 *   selinv_plan_selected: the number of selected entries; their panel
 *     positions to pos_out (host) when it is not NULL.
 *   selinv_gather: out_dev[e] = Ainv_dev[position of entry e] in the order
 *     given to selinv_plan_select (device arrays, element type dtype).
 * ------------------------------------------------------------------------- */
int selinv_plan_select(selinv_plan plan, int64_t nsel, const int32_t *rows, const int32_t *cols,
                       int64_t *pos_out);
int64_t selinv_plan_selected(selinv_plan plan, int64_t *pos_out);
int selinv_gather(selinv_plan plan, selinv_dtype dtype, const void *Ainv_dev, void *out_dev,
                  void *cuda_stream);

/* Pole-expansion sum (the use Sec. I names first, density functional
 * theory: a function of A, e.g. the Fermi function, as a weighted sum of the
 * selected inverses of shifted matrices A - z_l I on one pattern):
 *   out_dev[e] = sum_{l=0}^{nitems-1} w_l Ainv[l][pos_dev[e]]
 * in complex128 (w_l = weights[2l] + i weights[2l+1], host), terms added in
 * the order l = 0, 1, ... (deterministic).  Ainv: host array of nitems
 * device panel arrays of element type dtypes[l] (a real one counts as
 * complex with zero imaginary part); pos_dev: device int64[npos] panel
 * positions; out_dev: device complex128[npos]. */
int selinv_pole_sum(int nitems, const selinv_dtype *dtypes, const void *const *Ainv,
                    const double *weights, int64_t npos, const int64_t *pos_dev, void *out_dev,
                    void *cuda_stream);

/* Runs selinv_numeric once without graph capture, timing every kernel
 * launch with CUDA events on the stream, and synchronizes.  kernel_ms[k] and
 * kernel_launches[k] (arrays of SELINV_PROFILE_KINDS entries) receive the
 * summed device time in ms and the launch count of each kernel kind:
 *   0 L_KK^{-1} and Dinv (DFMA)        1 Lhat (DFMA)
 *   2 gather-GEMM + diagonal (DFMA)    3 digit planes of Lhat
 *   4 gather-GEMM on tensor cores      5 diagonal block after it
 *   6 digit planes of L_KK^{-1}        7 Lhat on tensor cores
 *   8 the persistent traversal          9 gather-GEMM on tcgen05
 *  10 split-k sums of the tcgen05 gather-GEMM
 *  11 diagonal block from the tensor-core sums (finisher)
 *  12 push schedule: diagonal block from the pushed A^{-1}_{C,K}
 *  13 push schedule: outer- and inner-product updates of the descendants
 *  14 Dinv_K of the supernodes wider than 32 columns (32 x 32 tiles)
 *  15 diagonal block on tcgen05 (exact sums of Lhat^T A^{-1}_{C,K})
 *  16 the whole step for supernodes of <= 8 columns and <= 64 rows, a warp each
 * For measurement only. */
#define SELINV_PROFILE_KINDS 17
int selinv_numeric_profile(selinv_plan plan, selinv_dtype dtype, const void *L_dev,
                           const void *D_dev, void *Ainv_dev, void *cuda_stream, double *kernel_ms,
                           int64_t *kernel_launches);

/* Device status word of the plan after asynchronous work (synchronizes the
 * plan's last stream, then returns and clears the latched code: SELINV_OK,
 * SELINV_ERR_TIMEOUT, SELINV_ERR_ZERO_PIVOT or SELINV_ERR_NONFINITE). */
int selinv_status(selinv_plan plan);

/* ---------------------------------------------------------------------------
 * selinv_dinv_noalloc: the diagonal-block step Dinv = L_KK^{-T} D_K^{-1}
 * L_KK^{-1} for one s x s unit-lower block, without allocating any memory.
 * There is no counterpart in the paper; it exists for callers that cannot
 * allocate device memory: code in a latency-critical loop (cudaMalloc and
 * cudaFree synchronize the whole device), code whose device memory is all
 * owned by another allocator (a framework's caching allocator or a fixed
 * arena), and code running where allocation is not permitted (a host
 * callback).
 *   s     block size, 0 <= s <= SELINV_NOALLOC_MAX_S (128); larger s returns
 *         SELINV_ERR_INVALID_ARG without doing anything.
 *   Lkk   device, column-major, leading dimension ld >= s; unit lower (its
 *         diagonal and strictly upper part are not read).
 *   D     device [s] pivots.
 *   Dinv  device output, column-major, leading dimension ldo >= s; every
 *         s x s entry is written.
 * The scratch block L_KK^{-1} lives in a file-scope static device array of
 * SELINV_NOALLOC_MAX_S^2 doubles (128 KB) that every GPU loading the library
 * holds until the process exits.  Its device address is looked up on the
 * first call on each device (with that device current), so make the first
 * call on a device before any stream capture.  The looked-up address is
 * kept for the life of the process; cudaDeviceReset invalidates it, so do
 * not call this entry point on a device after resetting that device.  All
 * calls share the array:
 * calls that overlap on the GPU (different streams, no ordering between
 * them) race on it.  Nothing in it needs clearing between calls.
 * Asynchronous on cuda_stream; no cudaMalloc, cudaFree or allocating library
 * call is made.
 * ------------------------------------------------------------------------- */
#define SELINV_NOALLOC_MAX_S 128
int selinv_dinv_noalloc(int32_t s, const double *Lkk, int64_t ld, const double *D, double *Dinv,
                        int64_t ldo, void *cuda_stream);

/* Static text for an error code. */
const char *selinv_error_string(int code);

/* Number of kernel launches the library issued since load (for accounting). */
int64_t selinv_launch_count(void);

/* Frees the device buffers that destroyed plans (and workspaces replaced by a
 * wider element type) left in the library's cache for reuse.  The cache
 * keeps released workspace buffers, keyed by exact size, up to 8 GB, so that
 * re-planning one pattern allocates and frees nothing; it is emptied by
 * itself when a device allocation fails.  Returns SELINV_OK; no device work
 * may be in flight on buffers of destroyed plans (destroying a plan already
 * synchronizes the device). */
int selinv_release_cached_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* SELINV_H */
