/*
 * fame.h -- C ABI of the GB300 library for the null-space-free reduced Maxwell
 * eigenproblem of Huang, Li, Li, Lin, Lin and Tian, "Eigenvalue problems of
 * discrete curl operators on various lattices for simulating three
 * dimensional photonic crystals" (arXiv:1806.10284).
 *
 * The library applies A_r = Sigma_r Q_r^* B^{-1} Q_r Sigma_r (eq. NFSEP,
 * Section 5.2) with hand-written sm_103a FFT kernels, finds its smallest
 * eigenvalues with a block LOBPCG on the GPU (complex64 or complex128
 * applies, FP64 Rayleigh-Ritz), and returns the eps-gradient of eigenvalues.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  * n = n1 n2 n3.  Grid arrays are in vec order: index i + n1 (j + n2 k),
 *    x index fastest (Section 1.3, Section 3).
 *  * A vector of A_r has 2n complex entries laid out [2][n]: the Pi_1
 *    coordinate block, then the Pi_2 coordinate block; within a block the
 *    frequency index (p, q, r) is ordered p + n1 (q + n2 r).  This is a fixed
 *    permutation of the column order of T in eq. (T).  A block of m vectors is
 *    [m][2][n], vector-major.
 *  * Complex numbers are interleaved (re, im): complex64 = two float,
 *    complex128 = two double (the layout of float2 / double2).
 *  * "device" pointers are CUDA device memory of the current device; "host"
 *    pointers are ordinary host memory.  The caller owns every buffer it
 *    passes; the library owns everything inside a context.
 *  * stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued on it.  Calls that return host values
 *    synchronise that stream before returning.
 *  * Every call returns a fame_status; nothing aborts.  After a non-OK
 *    status, fame_last_error(ctx) describes it (a thread-local copy is kept
 *    for failures of fame_create, readable with fame_last_error(NULL)).
 *  * A context is not thread safe: one host thread at a time.
 */
#ifndef FAME_H
#define FAME_H

#if defined(__GNUC__)
#define FAME_API __attribute__((visibility("default")))
#else
#define FAME_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fame_ctx fame_ctx;

typedef enum {
    FAME_OK = 0,
    FAME_E_ARG = 1,      /* bad argument (null pointer, size out of range)              */
    FAME_E_LATTICE = 2,  /* no ordering of a1..a3 meets the Section 2.2 conditions,     */
                         /* or the vectors are linearly dependent                       */
    FAME_E_RADIX = 3,    /* a grid size has a prime factor other than 2, 3, 5, or is   */
                         /* outside [2, 1024]                                           */
    FAME_E_CUDA = 4,     /* a CUDA runtime call failed (message holds its name/error)   */
    FAME_E_NOMEM = 5,    /* device or host allocation failed                           */
    FAME_E_STATE = 6,    /* call out of order (e.g. gradient before eigs, no eps set)   */
    FAME_E_NOCONV = 7,   /* eigensolver hit max_iter before the residual tolerance      */
    FAME_E_TIMEOUT = 8   /* a bounded device wait of a tensor-core kernel gave up       */
                         /* (limit: environment FAME_WAIT_TIMEOUT_MS, default 1000)      */
} fame_status;

/* dtype of vectors passed to fame_apply_Ar / fame_lift.  FAME_C128_DF: complex128
 * vectors (the same memory layout as FAME_C128), transformed in double-float
 * arithmetic -- pairs of floats, about 48 significant bits -- on the FP32 units,
 * which on GB300 run FP64 work at 1/64 of their rate; results agree with FAME_C128
 * to about 1e-14 of the largest entry.  Grids whose z length has no two-level
 * pass take the FAME_C128 path instead.
 * The eigensolver uses this form for its complex128 applies when the requested
 * residual is at least 1e-10 (environment FAME_FP64_NATIVE=1: never). */
enum { FAME_C64 = 0, FAME_C128 = 1, FAME_C128_DF = 2 };

/* flags of fame_eigs */
enum {
    FAME_FP64 = 1,          /* complex128 applies throughout                          */
    FAME_MIXED = 2,         /* complex64 applies, then complex128 refinement          */
    FAME_DETERMINISTIC = 4, /* fixed reduction order (always true in this build)      */
    FAME_WARM_START = 8,    /* start from the context's last eigenvectors if present  */
    FAME_INV_LANCZOS = 16   /* the paper's solver: Lanczos on A_r^{-1}, inner CG       */
};

/* Geometry chosen by fame_create (Section 2.2), for sampling eps on the Yee points. */
typedef struct {
    int n[3];          /* n1, n2, n3 along the canonical a1, a2, a3                   */
    int perm[3];       /* input vector index used as canonical a1, a2, a3             */
    int m[3];          /* grid offsets m1, m2, m3 after rounding                      */
    int rho[3];        /* rho1, rho2, rho3 (obtuse-case indicators)                    */
    int s[3];          /* index shifts: a2 <-> (s1, n2, 0), a3 <-> (s2, s3, n3)        */
    double delta[3];   /* mesh sizes delta_x, delta_y, delta_z                         */
    double a[9];       /* corrected vectors of eq. (transvec), column-major: a1, a2, a3 */
    double kappa[3];   /* Bloch fractions kappa_l = k . a_l (eq. quasi_periodic)        */
} fame_plan_info;

/* Counters of the last fame_eigs call. */
typedef struct {
    int iters_mixed;        /* LOBPCG iterations with complex64 applies               */
    int iters_fp64;         /* LOBPCG iterations with complex128 applies               */
    long long applies_c64;  /* single-vector A_r applies, complex64                    */
    long long applies_c128; /* single-vector A_r applies, complex128                   */
    double max_residual;    /* max_j ||A_r y_j - lambda_j y_j|| / lambda_j (FP64 apply) */
    double rr_host_ms;      /* host time spent in the small dense Rayleigh-Ritz solves  */
} fame_solve_stats;

/*
 * fame_create -- plan one lattice and Bloch vector (Section 2.2, eq. transvec).
 *   out      : receives the new context (host pointer to a pointer).
 *   lattice  : Bravais lattice id 0..13, or 14 = generic; informational only.
 *   a1,a2,a3 : primitive vectors (host, 3 doubles each), any Cartesian frame.
 *   n1,n2,n3 : grid sizes along the canonical a1, a2, a3 (the vectors after
 *              the ordering of Section 2.2: a1 the longest, the sin(gamma)
 *              condition met); each in [2, 1024] with prime factors 2, 3, 5.
 *   bloch    : the Bloch vector 2*pi*k (host, 3 doubles), same frame as a_l.
 * The vectors are reordered, rotated to the upper-triangular form, the grid
 * offsets m1, m2, m3 rounded (floor below 1/2, ceiling otherwise) and the
 * angles corrected so that a2 and a3 end on grid points.  Uses the current
 * CUDA device.  Errors: FAME_E_ARG, FAME_E_LATTICE, FAME_E_RADIX,
 * FAME_E_CUDA, FAME_E_NOMEM; *out is NULL on failure.
 */
FAME_API fame_status fame_create(fame_ctx** out, int lattice, const double a1[3], const double a2[3],
                        const double a3[3], int n1, int n2, int n3, const double bloch[3]);

/*
 * fame_plan_lattice -- host only, no GPU needed: the geometry fame_create
 * would choose for these arguments (same meaning as fame_create), written to
 * *info.  Errors: FAME_E_ARG, FAME_E_LATTICE, FAME_E_RADIX (message via
 * fame_last_error(NULL)).
 */
FAME_API fame_status fame_plan_lattice(const double a1[3], const double a2[3], const double a3[3],
                                       int n1, int n2, int n3, const double bloch[3],
                                       fame_plan_info* info);

/* fame_get_plan -- copy the chosen geometry (host struct). */
FAME_API fame_status fame_get_plan(const fame_ctx* ctx, fame_plan_info* info);

/*
 * fame_set_k -- change the Bloch vector 2*pi*k (host, 3 doubles) of a context:
 * rebuilds only the twist-phase tables (Section 4.2, eq. diagonal_matrix).
 * Invalidates stored eigenvectors' warm start only if the grid changes (it
 * does not).  Errors: FAME_E_ARG, FAME_E_CUDA.
 */
FAME_API fame_status fame_set_k(fame_ctx* ctx, const double bloch[3]);

/*
 * fame_set_eps -- set B = diag(vec B1, vec B2, vec B3) (Section 3): the
 * permittivity sampled at the E1, E2, E3 Yee points (i+1/2, j, k),
 * (i, j+1/2, k), (i, j, k+1/2) of the canonical grid.
 *   B1,B2,B3 : host arrays of n doubles each, vec order, every value > 0.
 * The library keeps 1/B in float and double on the device.  Errors:
 * FAME_E_ARG (null, non-positive or non-finite value), FAME_E_CUDA.
 */
FAME_API fame_status fame_set_eps(fame_ctx* ctx, const double* B1, const double* B2, const double* B3,
                         void* stream);

/* fame_set_eps_device -- as fame_set_eps with B a device array [3][n] of doubles. */
FAME_API fame_status fame_set_eps_device(fame_ctx* ctx, const double* B, void* stream);

/*
 * fame_apply_Ar -- Ay = A_r y = Sigma_r Q_r^* B^{-1} Q_r Sigma_r y (eq. NFSEP),
 * Q_r = (I_3 (x) T)[Pi_1 Pi_2] with T applied by twisted FFTs (Algorithms
 * 5.1 and 5.2) and Pi_1, Pi_2, Sigma_r of eqs. (range_basis1), (range_basis2),
 * (SVD).
 *   y, Ay : device, [m][2][n] complex of type dtype; may not overlap.
 *   m     : number of vectors, 1 <= m <= 4096.
 *   dtype : FAME_C64, FAME_C128 or FAME_C128_DF.
 * Asynchronous on stream.  Errors: FAME_E_ARG, FAME_E_STATE (no eps set),
 * FAME_E_NOMEM (workspace), FAME_E_CUDA.
 */
FAME_API fame_status fame_apply_Ar(fame_ctx* ctx, const void* y, void* Ay, int m, int dtype, void* stream);

/*
 * fame_apply_Ar_static -- the same A_r y as fame_apply_Ar, computed in a
 * workspace the library reserves statically in device memory, so that the
 * call allocates no device memory (the paper has no counterpart: it is an
 * interface for callers that may not allocate -- code running under a
 * memory budget fixed by a framework's caching allocator, or latency-bound
 * loops where a cudaMalloc, which can synchronise the device, is not
 * acceptable).
 *   The workspace holds 3 m n complex entries of type dtype and is limited to
 *   FAME_STATIC_WORKSPACE_BYTES (32 MiB: e.g. m <= 5 complex64 vectors at
 *   64^3); larger requests fail with FAME_E_ARG and allocate nothing.
 *   The first call on a device looks up the workspace address (set-up, once
 *   per device, with that device current); make it before any stream capture.
 *   The workspace is shared by all contexts of the process on a device:
 *   calls that overlap in time race on it.  Its contents need no
 *   initialisation.  Arguments, layout and other errors as fame_apply_Ar.
 */
#define FAME_STATIC_WORKSPACE_BYTES (32u << 20)
FAME_API fame_status fame_apply_Ar_static(fame_ctx* ctx, const void* y, void* Ay, int m, int dtype,
                                          void* stream);

/*
 * Apply plans -- the launch choices of fame_apply_Ar / fame_lift for one dtype
 * (no counterpart in the paper; they change speed, not results beyond rounding).
 *   z_kernel          : Z-in / Z-out family: 0 automatic, 1 fixed-length (complex64,
 *                       n3 in {16,32,48,64,80,96}; each block issues the loads of its
 *                       next vector while it transforms the current one), 2 two-level
 *                       radix, 3 Stockham, 4 fixed-length without that prefetch.
 *   xy_kernel         : XY family: 0 automatic, 1 fixed-length (complex64, square
 *                       16..96 or 80x96 planes), 2 two-level plane, 3 Stockham plane,
 *                       4 split y / x / y passes (any plane), 5 fixed-length with 512
 *                       threads per plane (complex64, 64x64, 96x96, 80x96).
 *   vectors_per_block : vectors each Z-pass thread block takes; 0 automatic.
 * fame_set_apply_plan: FAME_E_ARG if a family is not available for the grid and
 * dtype.  fame_autotune: times every available Z family and block size, then every
 * XY family, on m scratch vectors (allocates 2 m 2n complex temporarily), keeps the
 * fastest plan in the context and returns its time (ms per apply of m vectors) in
 * *best_ms (may be NULL).  Synchronises stream.  Errors: FAME_E_ARG, FAME_E_STATE
 * (no eps), FAME_E_NOMEM, FAME_E_CUDA.
 */
typedef struct fame_apply_plan {
    int z_kernel;
    int xy_kernel;
    int vectors_per_block;
} fame_apply_plan;
FAME_API fame_status fame_set_apply_plan(fame_ctx* ctx, int dtype, const fame_apply_plan* plan);
FAME_API fame_status fame_get_apply_plan(const fame_ctx* ctx, int dtype, fame_apply_plan* plan);
FAME_API fame_status fame_autotune(fame_ctx* ctx, int m, int dtype, double* best_ms, void* stream);

/*
 * fame_lift -- x = B^{-1} Q_r Sigma_r y, the GEP eigenvector for an A_r
 * eigenvector y (below Theorem invariant_space).
 *   y : device [m][2][n]; x : device [m][3][n] (E1, E2, E3 on the Yee grid);
 *   complex of type dtype.  Asynchronous.  Errors as fame_apply_Ar.
 */
FAME_API fame_status fame_lift(fame_ctx* ctx, const void* y, void* x, int m, int dtype, void* stream);

/*
 * fame_fields -- the electric and magnetic fields of eigenpairs (lambda_j, y_j) of A_r
 * on the Yee grid: E_j = B^{-1} Q_r Sigma_r y_j (the GEP eigenvector, as fame_lift) and
 * H_j = C E_j / (i omega_j) = -i omega_j P_r y_j, omega_j = sqrt(lambda_j) (mu_0 = 1),
 * with P_r = (I_3 (x) T)[P_1 P_2] the left singular vectors of C = P_r Sigma_r Q_r^*
 * (eq. SVD, Section 5.1): per frequency P_r = C^ Pi_r / Sigma_r, C^ the curl symbol
 * of C_l T = T Lambda_l.  Then C^* H_j = -i omega_j B E_j (Section 3).
 *   y      : device [m][2][n] complex128 eigenvectors of A_r.
 *   lambda : host, m eigenvalues (needed for H).
 *   E, H   : device [m][3][n] complex128 each, or NULL for a field not wanted.
 *   dtype  : FAME_C128.  Synchronises stream.
 * Errors: FAME_E_ARG, FAME_E_STATE (no eps set), FAME_E_NOMEM, FAME_E_CUDA.
 */
FAME_API fame_status fame_fields(fame_ctx* ctx, const void* y, const double* lambda, void* E, void* H, int m,
                                 int dtype, void* stream);

/*
 * fame_eigs -- the nev smallest (nonzero) eigenvalues of A_r, which are the
 * nev smallest nonzero eigenvalues of C^*C e = lambda B e (eq. GEP; Theorem
 * invariant_space).  Block LOBPCG with the preconditioner S P_K(M) S
 * (S = Sigma_r^{-1}, M = Q_r^* B^{-1} Q_r, P_K the degree-K Chebyshev
 * approximation of M^{-1} on [min 1/B, max 1/B]; K from the environment
 * variable FAME_CHEB_DEGREE, default 3, K = 1 the diagonal Sigma_r^{-2} /
 * mean(B^{-1})); Gram matrices accumulated in FP64 and the Rayleigh-Ritz
 * problem solved in FP64.  With FAME_MIXED the iteration runs
 * on complex64 applies and is then refined with complex128 applies; with
 * FAME_FP64 it runs on complex128 throughout.  Converged when
 * ||A_r y_j - lambda_j y_j|| <= tol * lambda_j (||y_j|| = 1, complex128
 * apply) for every j < nev.  At 2*pi*k = 0 the two zero eigenvalues of the
 * zero-frequency coordinates are excluded.
 *   nev        : 1 <= nev <= 64.
 *   tol        : residual tolerance (e.g. 1e-8), > 0.
 *   max_iter   : iteration cap for the whole solve (both phases).
 *   flags      : FAME_MIXED or FAME_FP64, optionally | FAME_WARM_START.
 *   lambda_out : host, nev doubles, ascending.
 *   Y_out      : device [nev][2][n] complex128 unit eigenvectors, or NULL.
 *   iters_out  : host int (total iterations), or NULL.
 * The eigenpairs are also kept in the context for fame_grad_eps.
 * FAME_INV_LANCZOS (instead of FAME_MIXED / FAME_FP64) runs the paper's solver
 * (Section 5.2; settings of Section 6): Lanczos on A_r^{-1} with full
 * reorthogonalisation, each A_r^{-1} q = S M^{-1} S q (S = Sigma_r^{-1},
 * M = Q_r^* B^{-1} Q_r) by an unpreconditioned complex128 CG to relative residual
 * min(tol, 1e-13); converged when the Ritz estimates of the nev largest eigenvalues
 * theta of A_r^{-1} are <= tol theta (the paper uses tol = 1e-12); at most
 * min(max_iter, 160) Lanczos steps.  The explicit residuals ||A_r y - lambda y|| /
 * lambda are then measured (complex128 apply) and reported in max_residual;
 * iters_out is the number of Lanczos steps, stats.iters_mixed the inner CG
 * iterations in all.
 * Synchronises stream.  Errors: FAME_E_ARG, FAME_E_STATE, FAME_E_NOCONV
 * (lambda_out still holds the best values), FAME_E_NOMEM, FAME_E_CUDA,
 * FAME_E_TIMEOUT (a tensor-core wait gave up).
 */
FAME_API fame_status fame_eigs(fame_ctx* ctx, int nev, double tol, int max_iter, int flags,
                      double* lambda_out, void* Y_out, int* iters_out, void* stream);

/* fame_get_stats -- counters of the last fame_eigs (host struct). */
FAME_API fame_status fame_get_stats(const fame_ctx* ctx, fame_solve_stats* stats);

/*
 * fame_grad_eps -- dB = sum_j dobj_dlambda[j] * d lambda_j / d B, with
 * d lambda_j / d B_l(v) = -|x_{j,l}(v)|^2, x_j = B^{-1} Q_r Sigma_r y_j
 * (Hellmann-Feynman on eq. NFSEP; A_r depends on B only through B^{-1}),
 * using the eigenpairs of the last fame_eigs call.  Bands whose eigenvalues
 * differ by at most rel_cluster * lambda form a cluster; every member gets
 * the cluster mean of -|x_j|^2.
 *   nev          : number of leading bands used, <= the last solve's nev.
 *   dobj_dlambda : host, nev doubles.
 *   rel_cluster  : degeneracy threshold (e.g. 1e-8 after FP64 refinement).
 *   dB_out       : device [3][n] doubles (overwritten).
 * Synchronises stream.  Errors: FAME_E_ARG, FAME_E_STATE (no solve yet),
 * FAME_E_CUDA.
 */
FAME_API fame_status fame_grad_eps(fame_ctx* ctx, int nev, const double* dobj_dlambda, double rel_cluster,
                          double* dB_out, void* stream);

/*
 * fame_block_gram -- G = U^H V, the block inner products from which the eigensolver
 * forms its Rayleigh-Ritz projections of eq. NFSEP (no counterpart in the paper,
 * whose inverse Lanczos needs only vector inner products; exposed for callers that
 * build their own projections, and for testing).
 *   U : device [ku][2n] complex of type dtype (ku vectors of A_r length, vector-major).
 *   V : device [kv][2n] complex of type dtype.
 *   G : device [kv][ku] complex128, column-major: G[j ku + i] = sum_r conj(U_i[r]) V_j[r].
 *   ku, kv in [1, 4096]; dtype FAME_C64 or FAME_C128.
 * Complex64 blocks with at most 128 vectors on each side are multiplied on the tensor
 * cores (tcgen05, TF32 operands split into high and low parts: about 2^-21 relative
 * accuracy per product, FP32 sums within a row block, FP64 across row blocks); other
 * shapes use FP32 (complex64) or FP64 (complex128) products.  Asynchronous on stream.
 * Errors: FAME_E_ARG, FAME_E_NOMEM, FAME_E_CUDA.  If a bounded device wait of the
 * tensor-core kernel gives up, G is filled with NaN.
 */
FAME_API fame_status fame_block_gram(fame_ctx* ctx, const void* U, int ku, const void* V, int kv, int dtype,
                                     void* G, void* stream);

/*
 * fame_eigs_batched -- solve several contexts (lattices and Bloch vectors along
 * band paths, grids may differ), several problems in flight at once: four
 * host worker threads with their own streams take problems in order, so the
 * GPU runs one problem's kernels while another waits for its host
 * Rayleigh-Ritz step.  Each worker lends one transform/solver workspace to the
 * problems it solves (device memory grows with the workers, not the batch);
 * every context keeps its eigenvectors as after fame_eigs.  The work starts
 * after the work already queued on stream.
 *   ctxs       : host array of nprob distinct context pointers (eps set on each).
 *   nev, tol, max_iter, flags : as fame_eigs (FAME_MIXED or FAME_FP64).  With
 *                FAME_WARM_START the batch is read as band paths (Section 6): runs of
 *                consecutive contexts on the same grid are cut into segments of at most
 *                ceil(nprob / 8) problems, and inside a segment each problem starts from
 *                the eigenvectors of the one before it (the first from random vectors);
 *                segments run concurrently.
 *   lambda_out : host [nprob][nev] doubles.
 *   iters_out  : host [nprob] ints, or NULL.
 * Returns when every problem is done.  Errors: as fame_eigs (the first failing
 * problem's status; its context holds the message); FAME_E_ARG for a repeated
 * context; FAME_E_NOCONV if any problem did not converge.
 */
FAME_API fame_status fame_eigs_batched(fame_ctx* const* ctxs, int nprob, int nev, double tol,
                              int max_iter, int flags, double* lambda_out, int* iters_out,
                              void* stream);

/*
 * Per-kernel timing.  fame_profile(1) clears the records and starts timing:
 * every kernel launch is then bracketed by two CUDA events recorded on the
 * stream it is launched on, with the algorithmic bytes (compulsory reads and
 * writes of that launch) and flops attached.  fame_profile(0) stops.
 * fame_profile_read synchronises the device and writes up to max entries,
 * one per kernel kind that launched, returning how many it wrote.
 */
typedef struct {
    char name[32];        /* kernel kind, e.g. "xy_c64"                          */
    long long launches;
    double total_ms;      /* sum of event-timed durations                        */
    double bytes;         /* sum of algorithmic bytes over the launches          */
    double flops;         /* sum of algorithmic flops over the launches          */
} fame_kernel_stat;
FAME_API fame_status fame_profile(int enable);
FAME_API int fame_profile_read(fame_kernel_stat* out, int max);

/* fame_last_error -- message of the last failure on ctx (or of fame_create if ctx is NULL). */
FAME_API const char* fame_last_error(const fame_ctx* ctx);

/* fame_destroy -- free a context and its device memory; NULL is ignored. */
FAME_API void fame_destroy(fame_ctx* ctx);

/* fame_launch_count -- kernels this library has launched in this process (monotone). */
FAME_API unsigned long long fame_launch_count(void);

/* fame_version -- library version string. */
FAME_API const char* fame_version(void);

/*
 * fame_bounds_violations -- for the bounds-checked debug build of the library
 * (libfame_check.so, compiled with -DFAME_CHECK_BOUNDS; no counterpart in the
 * paper).  In that build the kernels check the indices of their TMA boxes, of the
 * FFT passes' global loads and stores and of the staged block copies before each
 * access, skip an access that fails and record it.  Returns the number of failed
 * checks since the previous call (and clears them); *code (may be NULL) receives
 * the kind of the first (1 TMA coordinate, 2 tensor-core Gram output, 3 / 4 Z-pass
 * load / store, 5 staged 16-byte copy, 6 refinement row, 7 two-level Z-pass store)
 * and *index (may be NULL) its index.  Synchronous.  In the normal build: -1.
 */
FAME_API int fame_bounds_violations(int* code, long long* index);

#ifdef __cplusplus
}
#endif
#endif /* FAME_H */
