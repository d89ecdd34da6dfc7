/*
 * cdcc.h -- C ABI of the GB300 CD-CCSD gradient library.
 *
 * Closed-shell CCSD analytic gradients with Cholesky-decomposed integrals and
 * Abelian point-group symmetry (arXiv 2512.21909).  The library solves the
 * CCSD amplitude equations, the Lambda equations (Sec. 2.3), builds the
 * Cholesky-basis density Gamma^P_pq (Sec. 2.4 and 2.6) and contracts it with
 * derivative Cholesky vectors (Sec. 2.1, Eq. 2):
 *     dE/dx = sum_P sum_pq Gamma^P_pq dL^P_pq/dx .
 *
 * Conventions shared by every entry point
 *   - Irreps of the Abelian group are 0..h-1 (h = 1, 2, 4 or 8) in the Z2^k
 *     ordering; the direct product is bitwise XOR (Sec. 3.1).
 *   - Orbitals: n = nocc + nvir; the first nocc are occupied.  Within the
 *     occupied and within the virtual range the orbitals must be sorted by
 *     irrep (non-decreasing label).  Cholesky vectors must be sorted by
 *     irrep.  Violations return CDCC_EINVAL.
 *   - Packed Cholesky layout ("L-pattern") for L, dL and Gamma:
 *         for G_P in 0..h-1, for each vector P of irrep G_P,
 *           for G_p in 0..h-1 with G_q = G_p ^ G_P ^ G_x:
 *             the block L^P[p][q], p over the orbitals of irrep G_p and q over
 *             those of irrep G_q (ascending orbital order), row-major.
 *     G_x is the irrep of a displacement (0 for L and Gamma).  Its length is
 *     cdcc_packed_size(ctx, G_x) doubles.
 *   - Buffers: every pointer argument may be host memory or device memory of
 *     the context's device; the library detects which.  The caller owns all
 *     buffers; inputs are copied before the call returns (or, for device
 *     inputs, before the call's work is enqueued), outputs are written
 *     before the call returns.  The library never keeps a caller pointer.
 *   - Device memory: the context owns its device memory.  It is obtained
 *     through cdcc_options.dev_alloc / dev_free when set (a caching
 *     allocator such as PyTorch's), else with cudaMallocAsync.
 *   - Work runs on cdcc_options.stream (0 = the legacy default stream); every
 *     call synchronises that stream before returning a result to the host.
 *   - Errors: every call returns a cdcc_status; cdcc_last_error() gives a
 *     message.  After CDCC_ECUDA the context must be freed; after any other
 *     non-OK status the context stays usable.  Calls out of order return
 *     CDCC_ESTATE.  One context must not be used by two threads at once.
 */
#ifndef CDCC_H
#define CDCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CDCC_OK = 0,
    CDCC_EINVAL = 1,    /* invalid argument or input data                  */
    CDCC_ENOMEM = 2,    /* device or host allocation failed                */
    CDCC_ENOCONV = 3,   /* iterations did not converge within max_iter     */
    CDCC_ENUMERIC = 4,  /* NaN / Inf in a residual norm                    */
    CDCC_ECUDA = 5,     /* CUDA runtime error; the context is unusable     */
    CDCC_ESTATE = 6,    /* call out of order                               */
    CDCC_ETIMEOUT = 7   /* a bounded device wait gave up                   */
} cdcc_status;

/* Arithmetic of the dense contractions.                                   */
typedef enum {
    CDCC_PREC_FP64 = 0,   /* every contraction in FP64 (DFMA)              */
    CDCC_PREC_MIXED = 1,  /* split-precision tensor-core contractions with
                             an FP64 finish (see cdcc_options)             */
    CDCC_PREC_TC = 2      /* split-precision tensor-core contractions with
                             an exact-slice tensor-core finish: every
                             large contraction on the tensor cores         */
} cdcc_precision;

/* How the particle-particle ladder gets its (ac|bd) integrals.           */
typedef enum {
    CDCC_LADDER_AUTO = 0,   /* STORED when its estimated footprint is below
                               40 % (CDCC_PREC_TC) or 75 % (FP64 and MIXED,
                               whose on-the-fly build would run in FP64) of
                               the free device memory at init, else OTF    */
    CDCC_LADDER_STORED = 1, /* (ac|bd) of the undressed vectors built once
                               per gradient and kept in device memory      */
    CDCC_LADDER_OTF = 2     /* assembled from L^P_ab in row batches every
                               time the ladder is applied (Sec. 2.3); only
                               two batches are resident                    */
} cdcc_ladder;

/* Model Hamiltonian under a displacement (the MO basis is fixed, there is no
 * orbital relaxation):
 *   CDCC_FIXED_CORE   h = diag(eps) - G(L0) stays fixed while L moves; the
 *                     energy differentiated is E_ref + E_corr (default);
 *   CDCC_FROZEN_FOCK  the Fock matrix stays diag(eps) (h follows L) and the
 *                     energy differentiated is E_corr.
 * Both give the same amplitudes, multipliers and E_corr at the reference
 * geometry; only Gamma^P (and so the gradient) differs.                    */
typedef enum {
    CDCC_FIXED_CORE = 0,
    CDCC_FROZEN_FOCK = 1
} cdcc_fock_model;

typedef void *(*cdcc_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*cdcc_free_fn)(void *ptr, size_t bytes, void *stream,
                             void *user);

typedef struct {
    double conv_tol;        /* max |R/D| convergence (default 1e-10)        */
    double energy_tol;      /* |dE| convergence of CCSD (default 1e-12)     */
    int max_iter;           /* per solver (default 100)                     */
    int diis_dim;           /* DIIS vectors, 0 disables (default 8)         */
    int precision;          /* cdcc_precision (default CDCC_PREC_FP64)      */
    double switch_tol;      /* MIXED: max |R/D| below which the FP64
                               contractions take over (default 1e-6)        */
    int device;             /* CUDA device ordinal (default 0)              */
    void *stream;           /* cudaStream_t (default 0)                     */
    cdcc_alloc_fn dev_alloc;/* optional device allocator                    */
    cdcc_free_fn dev_free;
    void *alloc_user;
    int ladder;             /* cdcc_ladder (default CDCC_LADDER_AUTO)       */
    double ladder_batch_gb; /* OTF: GB of one (ab|cd) row batch (default 2) */
    int fock_model;         /* cdcc_fock_model (default CDCC_FIXED_CORE)    */
    int ladder_linearize;   /* MIXED / TC accurate phase: the ladder (linear
                               in its input) is evaluated accurately at an
                               anchor and corrected in BF16x3 around it;
                               convergence is accepted only on an iteration
                               with a fresh accurate anchor (default 1;
                               0 = every accurate iteration fully accurate) */
    double perm_cache_gb;   /* device GB for permuted copies of the
                               amplitude-independent tensors ((ia|jb),
                               (mc|bd), L blocks) in the layouts their
                               products need, made once per gradient and kept
                               with their tensor-core slices (about 2.5x this
                               in total); 0 = permute every time (default 32) */
    double ladder_slices_gb;/* ladder on the fly, float-slice arithmetic:
                               GB of the (ab|cd) batch rows' BF16 slices
                               kept from one ladder application to the next
                               within a gradient (they depend on L only;
                               kept while 8 GB stay free, freed before the
                               density sweep); 0 = rebuild every
                               application (default 48)                     */
    int ladder_pm;          /* ladder on the fly with symmetric /
                               antisymmetric (+/-) packing of the pairs ij,
                               ab and cd (Sec. 2.3): two products over the
                               canonical pairs, a quarter of the flops of
                               the plain map (default 1; 0 = plain map)     */
    int relaxed;            /* orbital relaxation (Sec. 2.5, Eq. z_vector):
                               the orbitals follow the closed-shell SCF
                               condition f_ai = 0 under a displacement;
                               build_density solves the Z-vector equations
                               and adds the relaxation term to Gamma^P, so
                               contract_dL returns the relaxed gradient
                               (CDCC_FIXED_CORE only; D stays the unrelaxed
                               dLag/dh).  Default 0.                        */
} cdcc_options;

typedef struct cdcc_ctx cdcc_ctx;

/* Fill *opt with the defaults above. */
void cdcc_default_options(cdcc_options *opt);

/*
 * Create a context from the model Hamiltonian (problem statement of
 * Sec. 2.1 / 2.2 for a synthetic MO basis).
 *   nirrep       1, 2, 4 or 8
 *   nocc, nvir   orbital counts (nocc >= 1, nvir >= 1)
 *   nchol        number of Cholesky vectors (>= 1)
 *   orb_irrep    [nocc+nvir] int32 irrep of each orbital (sorted, see above)
 *   eps          [nocc+nvir] double orbital energies; max eps_occ must be
 *                below min eps_vir
 *   chol_irrep   [nchol] int32 irrep of each vector (sorted)
 *   L            packed Cholesky vectors (L-pattern, G_x = 0), symmetric in
 *                pq: L^P_pq = L^P_qp within the stored blocks
 *   opt          NULL = defaults
 * The core Hamiltonian is fixed at h = diag(eps) - G(L) (the Fock matrix of
 * the closed-shell determinant is diag(eps)); displacements change L only.
 */
cdcc_status cd_ccsd_init(cdcc_ctx **out, int nirrep, int nocc, int nvir,
                         int nchol, const int32_t *orb_irrep,
                         const double *eps, const int32_t *chol_irrep,
                         const double *L, const cdcc_options *opt);

/* Number of doubles of a packed Cholesky-pattern tensor of irrep gx. */
size_t cdcc_packed_size(const cdcc_ctx *ctx, int gx);

/*
 * Solve the CCSD amplitude equations (T1/T2; the PPL of Sec. 2.3 is built
 * on the fly from L^P_ab).  Outputs (any may be NULL): correlation energy,
 * iteration count, final max |R/D|.
 */
cdcc_status ccsd_solve(cdcc_ctx *ctx, double *e_corr, int *iters,
                       double *resid);

/*
 * Solve the Lambda equations dLag/dt = 0 (Sec. 2.3).  Requires ccsd_solve.
 */
cdcc_status lambda_solve(cdcc_ctx *ctx, int *iters, double *resid);

/*
 * Build the densities (Sec. 2.4): Gamma^P_pq = dLag/dL^P_pq (symmetrised,
 * kept on the device in the packed L-pattern) and, if D1 != NULL, the
 * one-particle density D_pq = dLag/dh_pq as a dense [n][n] row-major array.
 * Requires lambda_solve.
 */
cdcc_status build_density(cdcc_ctx *ctx, double *D1);

/* Copy Gamma^P_pq (packed L-pattern, cdcc_packed_size(ctx,0) doubles). */
cdcc_status cdcc_get_gamma(cdcc_ctx *ctx, double *gamma);

/*
 * g[x] = sum_P sum_pq Gamma^P_pq dL_x^P_pq  (Sec. 2.1 Eq. 2, Sec. 2.6).
 *   nx        number of displacements
 *   x_irrep   [nx] irrep of each displacement (NULL = all totally
 *             symmetric).  Displacement x is stored with the L-pattern of
 *             irrep x_irrep[x]; for x_irrep[x] != 0 the gradient vanishes by
 *             symmetry (Sec. 3.1) and g[x] = 0 is returned without reading.
 *   dL        the nx packed tensors, back to back
 *   g         [nx] output
 * Requires build_density.
 */
cdcc_status contract_dL(cdcc_ctx *ctx, int nx, const int32_t *x_irrep,
                        const double *dL, double *g);

/*
 * Gradient in the density-fitting / Cholesky three-term form (Sec. 2.1 Eqs.
 * dfcd, cv_2ndstep and eri_cddf_der; Sec. 2.6 Eq. 2el_grad_cont), the
 * paper's own route: the Cholesky vectors are L^P = sum_R K^{-1}_PR B^R with
 * three-index integrals B^R_pq = (R|pq) and the metric M_PQ = (P|Q) =
 * (K K^T)_PQ (K lower triangular, M block diagonal by the irrep of P).  A
 * displacement changes B and M; with Jt = K^{-T} Gamma, Ltilde = K^{-T} L
 * and W_PQ = 1/2 sum_pq Ltilde^P_pq Jt^Q_pq,
 *     g[x] = sum_P <Jt^P, dB_x^P> - sum_PQ W_PQ dM_x,PQ .
 * It equals contract_dL with dL_x = d/dx [chol(M + x dM)^{-1} (B + x dB)].
 *   metric   M: for each irrep G, the nchol(G) x nchol(G) block, row-major,
 *            blocks back to back (cdcc_metric_size doubles); symmetric
 *            positive definite, else CDCC_EINVAL.  L given to cd_ccsd_init
 *            must be K^{-1} B for this M (K its Cholesky factor).
 *   nx       number of displacements (totally symmetric)
 *   dB       nx packed three-index derivatives (L-pattern, G_x = 0)
 *   dM       nx metric derivatives (packed as metric, symmetric blocks)
 *   g        [nx] output
 * The factorisation runs on the device in FP64, the transformations in the
 * accurate arithmetic of the schedule.  Requires build_density.
 */
size_t cdcc_metric_size(const cdcc_ctx *ctx);
cdcc_status contract_df(cdcc_ctx *ctx, const double *metric, int nx,
                        const double *dB, const double *dM, double *g);

/*
 * Symmetry-adapted two-step Cholesky decomposition of the ERI matrix
 * (Sec. 3.2, Algorithm 1; second step Eq. cv_2ndstep), context free.  The
 * pair-integral matrix is block diagonal by the irrep of the basis pair;
 * block G is given in factored form, (r|s) = sum_k B_G[r,k] B_G[s,k]
 * (positive semidefinite), and its integrals are evaluated from B.
 *   nirrep        1..8
 *   npair[G]      pairs of irrep G; naux[G] columns of B_G
 *   B             the blocks B_G (npair[G] x naux[G], row-major) back to
 *                 back; host or device memory of `device`
 *   tau           threshold: every residual |(r|s) - sum_P L_r L_s| ends
 *                 below tau (> 0)
 *   sigma         span factor of the qualified candidates (0 < sigma <= 1;
 *                 the paper uses 1e-2); qmax: candidates per macro
 *                 iteration (>= 1; the paper uses 1000)
 *   device, stream  CUDA device and stream (0: the default stream)
 *   ncv[G]        out (host): vectors (pivots) of irrep G
 *   piv           out (host or device): the pivots' pair indices within
 *                 their irrep, irrep blocks back to back, each in the
 *                 order taken; piv_cap entries
 *   L             out (host or device): the second-step vectors, for each
 *                 irrep ncv[G] x npair[G] row-major, blocks back to back;
 *                 L_cap doubles
 *   stats         out (host, may be null): [macro iterations, micro
 *                 iterations, first-step s, second-step s]
 *   msg           out (may be null): message of a failed call (msg_len
 *                 bytes, NUL terminated)
 * FP64 throughout.  Errors: CDCC_EINVAL (sizes, thresholds), CDCC_ENOMEM
 * (device memory, or piv_cap / L_cap too small: ncv is filled, retry with
 * the sizes it gives), CDCC_ENUMERIC (a non-finite diagonal, or the
 * pivots' metric not positive definite), CDCC_ECUDA.
 */
cdcc_status cdcc_cd_two_step(int nirrep, const int32_t *npair,
                             const int32_t *naux, const double *B,
                             double tau, double sigma, int qmax, int device,
                             void *stream, int32_t *ncv, int32_t *piv,
                             int64_t piv_cap, double *L, int64_t L_cap,
                             double *stats, char *msg, int msg_len);

/*
 * Error report of a result (the precision schedule of Sec. 2 / cdcc_options):
 * what the schedule's reduced-precision arithmetic changed, measured against
 * FP64 DFMA arithmetic at the same converged amplitudes t and multipliers
 * lambda.
 *   *dE    |E_FP64(t) - E(t)| + |<lambda, R_FP64(t)>|: the FP64 equations
 *          leave a residual R_FP64 at the schedule's t, and to first order the
 *          FP64 energy at its own solution differs from E_FP64(t) by
 *          -<lambda, R_FP64>;
 *   dg[x]  |<Gamma_FP64 - Gamma, dL_x>| with Gamma_FP64 from a density sweep
 *          in FP64 at (t, lambda) (the effect of the amplitude and multiplier
 *          errors on g is not included).
 * nx, x_irrep, dL as for contract_dL (nx may be 0, then dg is not touched).
 * Cost: one FP64 residual evaluation and one FP64 density sweep.  Gamma^P
 * and D of the context are left as they were.  Requires build_density; with
 * the FP64 schedule the numbers reflect the convergence threshold only.
 */
cdcc_status cdcc_error_estimate(cdcc_ctx *ctx, int nx, const int32_t *x_irrep,
                                const double *dL, double *dE, double *dg);

/* Everything that has not run yet, then contract_dL. */
cdcc_status gradient(cdcc_ctx *ctx, int nx, const int32_t *x_irrep,
                     const double *dL, double *e_corr, double *g);

/*
 * contract_dL without any memory allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * code embedded in a host framework or plugin whose device memory is owned
 * and budgeted by someone else, and serving loops that must not call
 * cudaMalloc because it synchronises the whole device.
 *
 * Computes g[x] = sum_e gamma[e] * dL[x*nnz + e] for x < nx, i.e. the same
 * contraction as contract_dL for totally symmetric displacements, where
 * gamma is the packed Gamma^P_pq (see cdcc_get_gamma) and dL holds nx packed
 * derivative tensors back to back.
 *   gamma, dL, g  DEVICE pointers of the current device (or managed
 *                 memory), owned by the caller; host pointers and memory of
 *                 another GPU return CDCC_EINVAL
 *   nx            1 .. CDCC_NOALLOC_MAX_NX, else CDCC_EINVAL
 *   nnz           elements per packed tensor (>= 1)
 *   stream        cudaStream_t of the current device (may be 0, a stream
 *                 of another device returns CDCC_EINVAL); the call only
 *                 enqueues work, g is valid once the stream reaches that point
 * No cudaMalloc / cudaFree or allocating library routine is called.  The
 * per-block partial sums live in a fixed device array of
 * 2048 x CDCC_NOALLOC_MAX_NX doubles (1 MiB) that every device loading the
 * library keeps until exit; a call uses min(8 x SM count, 2048) blocks of it.
 * The first call on a device looks that array's address up (with the device
 * current), so make it before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU race on it and must be
 * serialised.  A CUDA error already pending on the calling thread, or a
 * failed launch, returns CDCC_ECUDA (a pending error is left in place).
 */
#define CDCC_NOALLOC_MAX_NX 64
cdcc_status cdcc_contract_dL_noalloc(const double *gamma, const double *dL,
                                     int nx, size_t nnz, double *g,
                                     void *stream);

/* Amplitude / multiplier export for checks and warm starts:
 * which = 0: t1 [nocc][nvir], 1: t2 [nocc][nocc][nvir][nvir],
 *         2: lambda1, 3: lambda2 (same shapes; dense, zeros off-symmetry).
 * Index conventions of t2: amplitude of a+_{a,alpha} a+_{b,beta} a_{j,beta}
 * a_{i,alpha} at [i][j][a][b] (orbital indices relative to the occupied /
 * virtual range).                                                         */
cdcc_status cdcc_get_amplitudes(cdcc_ctx *ctx, int which, double *out);

/* Index tables of the +/- packed on-the-fly ladder (Sec. 2.3), for tests
 * and inspection: HOST ONLY, no device work, no context.  The doubles
 * amplitudes of nirrep irreps (1, 2, 4, 8) with nocc_irrep[g] occupied and
 * nvir_irrep[g] virtual orbitals per irrep are stored per pair irrep G as a
 * row-major block, rows (i,j) (i of irrep gi, sub-blocks by gi), columns
 * (c,d) likewise; batch_gb bounds the FP64 (ab|cd) rows of one batch.
 * Canonical pairs (p,q): irrep(p) > irrep(q), or the same irrep and p >= q.
 * For every G with canonical pairs, out receives
 *   G, uo, uv, nbatch, nrow(G), ncol(G),
 *   row of (i,j)[uo], row of (j,i)[uo]       canonical occupied pairs,
 *   column of (c,d)[uv], column of (d,c)[uv] canonical virtual pairs,
 * then per row batch (a in [a0,a1) of irrep ga >= gb = ga^G)
 *   ga, a0, a1, nv, row in the batch[nv], column of (a,b)[nv],
 *   column of (b,a) or -1 when a == b[nv]
 * (all int32, offsets inside the block).  *len = number of int32 written
 * (or needed, with out = NULL).  Errors: CDCC_EINVAL for bad arguments or
 * offsets beyond 32 bits, CDCC_ENOMEM when cap < *len.                    */
cdcc_status cdcc_ladder_pm_tables(int nirrep, const int32_t *nocc_irrep,
                                  const int32_t *nvir_irrep, double batch_gb,
                                  int32_t *out, int64_t cap, int64_t *len);

/* Wall-clock seconds of the last ccsd / lambda / density / contract_dL
 * phases (device time of the stream, CUDA events). */
cdcc_status cdcc_phase_times(cdcc_ctx *ctx, double *t4);

/* Per-kernel-class timing (CUDA events on the context's stream, around
 * every launch of the class while enabled).  Classes:
 *   0 FP64 GEMM (work = flops)          1 permutation / axpy (work = bytes)
 *   2 amplitude update (work = bytes)   3 contract_dL batched dot (bytes)
 *   4 other vector kernels (bytes)      5 tensor-core GEMM, BF16 float
 *   6 tensor-core GEMM, exact slices      slices (work = algorithmic
 *     (work = algorithmic flops 2MNK)     flops 2MNK)
 * cdcc_kernel_stats returns the accumulated device seconds, launches and
 * algorithmic work since the context was created. */
cdcc_status cdcc_profile(cdcc_ctx *ctx, int enable);
cdcc_status cdcc_kernel_stats(cdcc_ctx *ctx, int kind, double *seconds,
                              long long *launches, double *work);

/* Iterations of the last solves: info[0..3] = CCSD mixed-precision,
 * CCSD FP64, Lambda mixed-precision, Lambda FP64 iterations. */
cdcc_status cdcc_solver_info(cdcc_ctx *ctx, int *info);

/* The ladder mode the context chose (CDCC_LADDER_STORED or _OTF).         */
cdcc_status cdcc_ladder_mode(cdcc_ctx *ctx, int *mode);

/* Particle-particle ladder work since profiling was enabled (cdcc_profile):
 * device seconds, algorithmic flops (sum over the ladder products, their
 * adjoints, the (ac|bd) builds from L^P_ab and their adjoints) and calls.
 * Zero while profiling is off.                                            */
cdcc_status cdcc_ladder_stats(cdcc_ctx *ctx, double *seconds, double *flops,
                              long long *calls);

/*
 * C = beta*C + alpha * op(A) op(B) on device buffers, row-major, with the
 * library's contraction kernels (the building block of every contraction of
 * the path; exposed for testing and reuse).  op(A) is M x K (transA: A is
 * stored K x M), op(B) is K x N (transB: B is stored N x K).
 *   mode 0      FP64 DFMA GEMM
 *   mode 1..3   tensor-core GEMM with 1..3 BF16 slices per operand
 *               (products of slices i + j < mode, FP32 accumulation)
 *   mode 12..14 tensor-core GEMM with 2..4 exact integer slices per
 *               operand (row / column power-of-two scaling, exact FP32
 *               partial sums drained into double-float accumulators):
 *               8 + 7(s-1) bits of every element relative to its row or
 *               column maximum, FP64-class results for s = 4
 * Allocates its temporaries with cudaMallocAsync on `stream` and
 * synchronises the stream before returning.
 */
cdcc_status cdcc_dgemm(int transA, int transB, int M, int N, int K,
                       double alpha, const double *A, int lda,
                       const double *B, int ldb, double beta, double *C,
                       int ldc, int mode, void *stream);

/*
 * Self-test of the failure path of bounded device waits (no paper
 * counterpart): launches one kernel whose mbarrier wait can never complete;
 * the bounded spin gives up, the kernel records an error code and exits.
 * Returns CDCC_ETIMEOUT when that path works (the expected result), CDCC_OK
 * if the wait unexpectedly completed, CDCC_ECUDA / CDCC_ENOMEM on a runtime
 * error.  The device stays usable afterwards.
 */
cdcc_status cdcc_selftest_bounded_wait(void *stream);

/* ------------------------------------------------------------------------
 * Serving: a request loop on one GPU that admits gradient jobs of mixed
 * sizes and point groups as they arrive, by free slots and device memory,
 * keeps each admitted job's state (amplitudes, Lambda, DIIS histories,
 * intermediates) resident in its own context and runs the jobs concurrently
 * on their own CUDA streams (continuous batching: a job that arrives while
 * others run starts as soon as a slot and its memory are free).
 *
 * Admission: first come first served with a look-ahead of four jobs past
 * the head of the queue; a job is admitted when a slot is free and its
 * estimated peak device footprint (cdcc_job_footprint) fits the budget not
 * yet promised to running jobs, or when nothing else runs.  A job whose
 * device allocation fails anyway is put back at the head of the queue and
 * retried when it can run alone (at most three retries).  The ladder mode
 * of a job depends on its size only (stored when the stored integrals fit
 * stored_max_gb), so a job's result does not depend on the jobs it ran
 * beside.
 * Threads: one dispatcher and max_active workers inside the library; the
 * calls below may be made from any host thread.
 */
typedef struct cdcc_server cdcc_server;

/* One gradient job.  Arrays as for cd_ccsd_init / contract_dL; host or
 * device memory of the server's device; cdcc_submit copies them.        */
typedef struct {
    int nirrep, nocc, nvir, nchol;
    const int32_t *orb_irrep;   /* [nocc+nvir]                           */
    const double *eps;          /* [nocc+nvir]                           */
    const int32_t *chol_irrep;  /* [nchol]                               */
    const double *L;            /* packed L-pattern, G_x = 0             */
    int nx;                     /* displacements (>= 0)                  */
    const int32_t *x_irrep;     /* [nx] or NULL (all totally symmetric)  */
    const double *dL;           /* the nx packed tensors, back to back   */
} cdcc_job_desc;

typedef enum {
    CDCC_JOB_QUEUED = 0, CDCC_JOB_RUNNING = 1, CDCC_JOB_DONE = 2,
    CDCC_JOB_FAILED = 3
} cdcc_job_state;

typedef struct {
    int state;            /* cdcc_job_state                               */
    int status;           /* cdcc_status of a finished job (DONE: OK)     */
    int nx;               /* displacements of the job                     */
    int ladder;           /* ladder mode the job ran with                 */
    int retries;          /* allocation failures retried                  */
    double e_corr;        /* correlation energy (DONE)                    */
    double err_dE;        /* error report of e_corr (DONE; see
                             cdcc_energy_error)                           */
    double t_wait;        /* seconds from submission to admission         */
    double t_run;         /* seconds from admission to completion         */
    double *g;            /* in: caller buffer of >= nx doubles or NULL;
                             the gradient is written there once DONE      */
    char message[160];    /* reason of a FAILED job                       */
} cdcc_result;

/* Host-side stand-in for the gradient of a job (tests of the scheduling
 * logic without a GPU, or embedding a different executor): fills *e_corr,
 * g[nx], *err_dE and returns a cdcc_status (CDCC_ENOMEM = allocation failed,
 * the job is retried).                                                    */
typedef int (*cdcc_executor_fn)(uint64_t ticket, const cdcc_job_desc *job,
                                int slot, double *e_corr, double *g,
                                double *err_dE, void *user);

typedef struct {
    int max_active;         /* slots: jobs in flight (default 4)           */
    double budget_gb;       /* device memory the jobs may use; 0 = the free
                               memory at creation minus reserve_gb          */
    double reserve_gb;      /* kept free when budget_gb = 0 (default 8)    */
    double stored_max_gb;   /* stored ladder when its integrals need at most
                               this much (default 24), else on the fly     */
    int error_report;       /* attach cdcc_energy_error to every result
                               (default 1)                                  */
    cdcc_executor_fn executor;  /* NULL = the library's gradient          */
    void *executor_user;
} cdcc_server_options;

void cdcc_server_default_options(cdcc_server_options *sopt);

/* Create a server on opt->device (opt: options of every job; NULL =
 * defaults; its stream, allocator and ladder fields are ignored: every slot
 * has its own stream and jobs allocate with cudaMallocAsync on it).       */
cdcc_status cdcc_server_create(cdcc_server **out, const cdcc_options *opt,
                               const cdcc_server_options *sopt);

/* Queue a job (inputs copied before returning); *ticket identifies it.
 * CDCC_EINVAL for inconsistent sizes, CDCC_ESTATE after shutdown began.   */
cdcc_status cdcc_submit(cdcc_server *srv, const cdcc_job_desc *job,
                        uint64_t *ticket);

/* Non-blocking state of a job; res->g (if set) receives the gradient once
 * the job is DONE.  CDCC_EINVAL for an unknown ticket.                    */
cdcc_status cdcc_poll(cdcc_server *srv, uint64_t ticket, cdcc_result *res);

/* Block until the job finishes or timeout_s passes (then CDCC_ETIMEOUT),
 * then as cdcc_poll.                                                      */
cdcc_status cdcc_wait(cdcc_server *srv, uint64_t ticket, double timeout_s,
                      cdcc_result *res);

/* Largest number of jobs that ran at once so far.                         */
int cdcc_server_max_active_seen(const cdcc_server *srv);

/* Estimated peak device bytes of a job with the given precision and ladder
 * mode (the admission estimate; on-the-fly batches of batch_gb).          */
size_t cdcc_job_footprint(const cdcc_job_desc *job, int precision,
                          int ladder, double batch_gb);

/* Stop accepting jobs, let running jobs finish, fail queued ones, free. */
void cdcc_server_destroy(cdcc_server *srv);

/*
 * Error report of the correlation energy (Sec. 2 precision schedule; cheap
 * enough to attach to every result): what the accurate arithmetic of the
 * schedule leaves in E_corr.
 *   CDCC_PREC_TC     the exact-slice arithmetic with s = 4 slices keeps 7
 *                    more bits per operand than s = 3; one residual with
 *                    s = 3 at the converged amplitudes t gives
 *                      dE_3 = |E_3(t) - E_4(t)| + |<lambda, R_3(t) - R_4(t)>|
 *                    and the report is dE_3 / 2^7 plus the convergence
 *                    term |<lambda, R_4(t)>|;
 *   FP64 / MIXED     the convergence term |<lambda, R(t)>| (FP64 rounding is
 *                    far below it).
 * Requires lambda_solve.  Cost: one residual in the 3-slice arithmetic (TC)
 * or none.  The recorded intermediates are re-evaluated when next needed.
 */
cdcc_status cdcc_energy_error(cdcc_ctx *ctx, double *dE);

/* Number of kernels this context has launched so far. */
long long cdcc_kernel_launches(const cdcc_ctx *ctx);

const char *cdcc_last_error(const cdcc_ctx *ctx);
void cd_ccsd_free(cdcc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CDCC_H */
