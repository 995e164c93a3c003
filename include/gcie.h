/*
 * gcie: contour-integral generalized eigensolver for GB300 (sm_103a), C ABI.
 *
 * Problem (paper arXiv 2511.01927, Eq. GEP in Section 3.1 and the REQUIRE/ENSURE lines of
 * Algorithm 1): given a real symmetric sparse K (the paper's A) and a symmetric positive
 * definite sparse M (the paper's B) and a target range [lo, hi], return every eigenpair
 * (lambda, x) of K x = lambda M x with lambda in [lo, hi].
 *
 * Method: the contour-integral pipeline of Algorithm 1 with the moment method and FEAST
 * subspace iteration of Appendix A.3.3 (Sakurai-Sugiura moments, U_{i+1} = orth(P_k U_i)),
 * trapezoid quadrature on circles (Section 4.2), shifted systems (z_j M - K) X_j = M V at every
 * node (Eq. quadrature_appendix), moments S_k, M-orthonormal basis, Rayleigh-Ritz, keep
 * lambda in I_k, merge/de-duplicate.  The shifted solves run as batched COCG (conjugate
 * orthogonal CG for complex symmetric systems) in FP32 complex with FP64 residual refinement,
 * or in FP64 throughout; everything after the solves is FP64.
 *
 * Conventions for every call:
 *   - return value 0 (GCIE_OK) on success, otherwise one of the GCIE_E* codes below; no call
 *     throws or aborts; gcie_strerror() names a code and gcie_last_error() gives a message
 *     for the calling thread's most recent failure.
 *   - pointers named h_* / taking gcie_csr are HOST memory, borrowed for the duration of the
 *     call (the library copies what it needs).  Pointers named d_* are DEVICE memory on the
 *     context's device, owned by the caller, and must stay valid until the call returns.
 *   - complex arrays are interleaved (re, im) pairs.
 *   - a context is used by one host thread at a time; calls on it are ordered on its stream.
 */
#ifndef GCIE_H
#define GCIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
enum {
    GCIE_OK = 0,
    GCIE_EINVAL = 1,      /* bad argument: CSR structure, sizes, lo >= hi, option out of range */
    GCIE_ENOTSYM = 2,     /* K or M not symmetric (checked on every stored entry) */
    GCIE_ENOTSPD = 3,     /* M has a non-positive diagonal entry, or a Gram matrix lost rank */
    GCIE_ENOMEM = 4,      /* device or host allocation failed, or the budget is too small */
    GCIE_ENOCONV = 5,     /* some contour did not reach the tolerance; converged pairs returned */
    GCIE_EBREAKDOWN = 6,  /* COCG breakdown (p^T A p = 0) that refinement could not recover */
    GCIE_ETIMEOUT = 7,    /* a bounded device-side wait expired (about one second of SM clock); the
                             waiting CTAs let their copies in flight land and returned, and the
                             context stays usable (see GCIE_ECONTEXT for when it does not) */
    GCIE_ECOUNT = 8,      /* returned count differs from a caller-supplied expected count */
    GCIE_ECUDA = 9,       /* CUDA runtime error */
    GCIE_ECONTEXT = 10    /* the context is unusable: after a bounded wait gave up, a bulk copy into
                             shared memory could not be confirmed complete before its CTA exited
                             (a second bounded wait ran out too); every later call on the context
                             returns this code: destroy it and create a new one */
};

enum { GCIE_MIXED = 0, GCIE_FP64 = 1 };   /* precision of the shifted solves */
/* preconditioner of the shifted solves */
enum { GCIE_PREC_NONE = 0, GCIE_PREC_AUTO = 1, GCIE_PREC_AMG = 2, GCIE_PREC_BAND = 3 };

/* Sparse matrix in CSR form, host memory: 0-based, column indices sorted and unique within a
 * row, both triangles stored, n >= 1, rowptr[0] = 0, rowptr[n] = nnz. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *rowptr;   /* n + 1 */
    const int32_t *col;      /* nnz */
    const double *val;       /* nnz */
} gcie_csr;

/* One contour: the circle |z - c| = r and the interval [lo, hi] whose eigenvalues it keeps
 * (Algorithm 1: "keep lambda in I_k").  Section 4.2: c = (lo+hi)/2, r = (1+alpha)(hi-lo)/2. */
typedef struct {
    double c, r;
    double lo, hi;
} gcie_contour;

typedef struct {
    int32_t nodes;          /* trapezoid nodes N per circle, even, 2..64 (default 16) */
    int32_t L;              /* columns of the random starting block V (default 32) */
    int32_t moments;        /* moments m: basis [S_0 .. S_{m-1}] (default 2) */
    int32_t max_outer;      /* FEAST iterations cap (default 8) */
    int32_t max_iters;      /* COCG iteration cap per shifted solve (default 5000) */
    int32_t precision;      /* GCIE_MIXED (default) or GCIE_FP64 */
    double tol;             /* eigenpair tolerance on ||Kx - lambda Mx||_2 / (||K||_1 ||x||_2) (1e-10) */
    double lin_tol;         /* shifted-solve target on the diagonally scaled residual (default 1e-11) */
    int32_t ncontours;      /* > 0: use contours[0..ncontours-1]; 0: nuniform equal-width pieces */
    int32_t nuniform;       /* number of equal-width contours when ncontours == 0 (default 1) */
    const gcie_contour *contours;   /* host, borrowed */
    double alpha;           /* radius inflation for uniform contours (default 0) */
    const double *h_V0;     /* host n x L row-major starting block, or NULL: library draws N(0,1) */
    uint64_t seed;          /* seed for the library's own draw when h_V0 == NULL */
    size_t hbm_budget_bytes;/* device memory the solve may use (0: 90% of free memory) */
    int32_t expected_count; /* >= 0: return GCIE_ECOUNT if the merged count differs; -1: off */
    int32_t profile;        /* 1: time every kernel launch with CUDA events (see gcie_stats) */
    int32_t precond;        /* GCIE_PREC_AUTO (default): banded LDL^T factors (FP32) when the
                               bandwidth allows, else the multigrid cycle; or a GCIE_PREC_* */
    int32_t judge;          /* 1: count check of every finished contour (see gcie_count_miss): a
                               contour that misses eigenvalues is replaced by the two halves of
                               gcie_resplit (w = 10) and they are solved; 0 (default): off */
    int32_t max_resplit;    /* levels of re-splitting below an input contour, 0..16 (default 4); a
                               contour that still fails at the last level keeps its pairs and
                               reports GCIE_ENOCONV */
    int32_t batch_streams;  /* gcie_solve_batch: pencils solved at the same time, each by its own host
                               thread on its own stream (1..16; default 4) */
    double lin_tol_first;   /* looser inner tolerance in the first FEAST iteration (Appendix A.3.3: the
                               subspace iteration needs the filtered basis, not converged solves): 0
                               (default) = lin_tol in every iteration; otherwise >= lin_tol, the
                               shifted-solve target of every contour's first iteration, the later ones
                               using lin_tol.  A contour whose pairs do not meet tol after the first
                               iteration is iterated again, so results keep tol either way. */
} gcie_opts;

/* Results: library-allocated host arrays, released by gcie_result_free. */
typedef struct {
    int64_t n;
    int32_t count;              /* eigenpairs returned (converged, inside [lo, hi], de-duplicated) */
    double *evals;              /* count, ascending */
    double *evecs;              /* n x count, column j at evecs[j*n .. j*n+n), M-normalised, the
                                   entry of largest magnitude positive */
    double *resid;              /* count: ||Kx - lambda Mx||_2 / (||K||_1 ||x||_2) */
    int32_t *contour_of;        /* count: index of the contour that produced the pair */
    int32_t ncontours;
    int32_t *status_per_contour;/* ncontours: GCIE_OK or GCIE_ENOCONV */
    int32_t *iters_per_contour; /* ncontours: FEAST iterations used */
    int32_t outer_iters;        /* max over contours */
    int64_t cocg_iters;         /* COCG iterations summed over solve batches */
    double norm_k1;             /* ||K||_1 used in the residual */
    gcie_contour *contours;     /* ncontours: the final contours, each re-split one replaced in place
                                   by its two halves (ascending when the input was) */
    double *count_estimate;     /* ncontours: stochastic trace estimate of the enclosed eigenvalue
                                   count, from the contour's first FEAST iteration (formed whether or
                                   not judge is on: a contour that stops on the stall rule is checked
                                   against it) */
    int32_t resplits;           /* contours replaced by their halves */
} gcie_result;

/* Per-kernel-class accounting since the last gcie_reset_stats (profile = 1 fills times). */
enum { GCIE_K_SPMM_DIR = 0, GCIE_K_SPMM_UPD = 1, GCIE_K_REFINE = 2, GCIE_K_MOMENT = 3,
       GCIE_K_DENSE = 4, GCIE_K_OTHER = 5, GCIE_K_PREC = 6, GCIE_K_FACTOR = 7, GCIE_K_NCLASS = 8 };
typedef struct {
    int64_t launches[GCIE_K_NCLASS];
    double ms[GCIE_K_NCLASS];          /* summed CUDA-event durations of those launches */
    double bytes[GCIE_K_NCLASS];       /* algorithmic DRAM bytes of those launches */
    double flops[GCIE_K_NCLASS];
    int64_t total_launches;            /* every kernel the library launched */
} gcie_stats;

typedef struct gcie_ctx gcie_ctx;
typedef struct gcie_pencil gcie_pencil;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  stream: a cudaStream_t to order work on, or NULL
 * for a stream the context creates and owns.  Errors: GCIE_EINVAL (bad device), GCIE_ECUDA. */
int gcie_create(gcie_ctx **out, int device, void *stream);
/* Release the context and everything it allocated (pencils must be destroyed first). */
void gcie_destroy(gcie_ctx *ctx);

/* Default options (the values in the comments above). */
void gcie_default_opts(gcie_opts *o);
const char *gcie_strerror(int code);
/* Message of the calling thread's last failure ("" if none). */
const char *gcie_last_error(void);
int gcie_get_stats(gcie_ctx *ctx, gcie_stats *out);
void gcie_reset_stats(gcie_ctx *ctx);
/* Time every subsequent kernel launch of this context with CUDA events (on = 1) or not (0);
 * gcie_solve_pencil also sets it from opts.profile. */
void gcie_set_profile(gcie_ctx *ctx, int on);

/* ------------------------------------------------------------------ pencil ingest (step a1)
 * Validate K and M (structure, symmetry of every stored entry, positive diagonal of M), build
 * the union sparsity pattern and upload FP64 and FP32 copies of both value arrays to the
 * device.  The pencil stays resident until gcie_pencil_destroy.
 * Errors: GCIE_EINVAL, GCIE_ENOTSYM, GCIE_ENOTSPD, GCIE_ENOMEM, GCIE_ECUDA. */
int gcie_pencil_create(gcie_ctx *ctx, const gcie_csr *K, const gcie_csr *M, gcie_pencil **out);
void gcie_pencil_destroy(gcie_pencil *p);
int64_t gcie_pencil_n(const gcie_pencil *p);
int64_t gcie_pencil_nnz(const gcie_pencil *p);   /* of the union pattern */

/* ------------------------------------------------------------------ whole solve
 * All eigenpairs of K x = lambda M x in [lo, hi] (Algorithm 1 ENSURE).  gcie_solve ingests K, M
 * from the host, solves, and frees the device copy; gcie_solve_pencil reuses a resident pencil.
 * On GCIE_ENOCONV the result still holds every pair that met the tolerance.
 * Errors: those of gcie_pencil_create plus GCIE_ENOCONV, GCIE_EBREAKDOWN, GCIE_ECOUNT. */
int gcie_solve(gcie_ctx *ctx, const gcie_csr *K, const gcie_csr *M, double lo, double hi,
               const gcie_opts *opts, gcie_result *out);
int gcie_solve_pencil(gcie_ctx *ctx, gcie_pencil *p, double lo, double hi, const gcie_opts *opts,
                      gcie_result *out);
/* Independent pencils (the serving case; Algorithm 1 treats contours, and so pencils, as independent):
 * pencil i is K[i], M[i] with the interval [lo[i], hi[i]], solved into out[i] with the same options.
 * opts.batch_streams pencils are solved at the same time: a scheduler hands the pencils, largest first,
 * to that many host threads, each driving its own context (stream, memory pool) on the context's device
 * (the first one is ctx itself), so the small pencils' latency-bound kernels overlap on the GPU.  Each
 * solve may use 1/batch_streams of the device-memory budget.  K, M, lo, hi, out: host arrays of
 * npencils >= 1; each out[i] is released with gcie_result_free.  A pencil that ends with GCIE_ENOCONV
 * does not stop the batch; any other error stops the scheduler from starting further pencils (those
 * results stay zeroed).  Kernel statistics of all workers are added to ctx's.
 * Returns GCIE_OK when every solve did, else the status of the lowest-numbered pencil that failed. */
int gcie_solve_batch(gcie_ctx *ctx, int32_t npencils, const gcie_csr *K, const gcie_csr *M, const double *lo,
                     const double *hi, const gcie_opts *opts, gcie_result *out);
void gcie_result_free(gcie_result *r);
/* Frees one array of a gcie_result that the caller took out of the struct (and set to NULL there,
 * so that gcie_result_free skips it), e.g. to hand the eigenvectors to another owner without a
 * copy.  NULL is ignored. */
void gcie_buffer_free(void *p);

/* ------------------------------------------------------------------ contours from a predicted spectrum
 * Algorithm 2 (adaptive contour construction via KDE; Section 4.2): the range of the predictions,
 * widened by eps = beta (max - min) on both sides, is split recursively at the minimiser of the
 * interval sparsity function G_k(t) = sum_j exp(-w (t - lam_j)^2 / (b - a)^2) until no interval
 * holds more than nmax predictions; intervals with fewer than nmin are then joined to their
 * nearer neighbour (a joined interval above nmax is split between its two middle predictions).
 * Contour k: c = (lo + hi)/2, r = (1 + alpha)(hi - lo)/2, lo/hi the interval (a prediction belongs
 * to [lo, hi); the last interval also takes hi).  Host only, no device work.
 *   pred: host, npred >= 1 finite predicted eigenvalues, any order (the paper's Lambda-hat).
 *   nmin, nmax: per-contour count range (paper: 10, 50); w: gap sensitivity (paper: 10).
 *   out, counts: host arrays of cap entries: the contours in ascending order and the number of
 *   predictions each holds.  *nout: number of contours (also set when cap is too small).
 * Errors: GCIE_EINVAL for bad arguments or cap < *nout (nothing written then). */
int gcie_kde_contours(const double *pred, int32_t npred, int32_t nmin, int32_t nmax, double w, double alpha,
                      double beta, gcie_contour *out, int32_t *counts, int32_t cap, int32_t *nout);

/* Contours for a fixed budget: [lo, hi] is cut in gaps of the predicted spectrum until it has
 * max_contours pieces (fewer when no piece can be cut).  While the budget is not reached, the piece
 * with the most predictions in its closed interval [a, b] (leftmost on ties) is cut at the middle of
 * the widest gap between consecutive sorted predictions of ranks k/4 .. k-1-k/4 (k in the piece;
 * first such gap on ties), so each half keeps a quarter of them; a piece whose widest such gap is
 * empty stops the planning.  This keeps the number of shifted systems fixed (the solve runs them all
 * in one wave when it fits) and puts every boundary in a gap, where the quadrature filter converges
 * fastest; Algorithm 2 instead fixes N_max per contour and lets the count follow.
 * Contour i: c = (lo_i + hi_i)/2, r = (1 + alpha)(hi_i - lo_i)/2 (Section 4.2).  Host only.
 *   pred: host, npred >= 0 finite predicted eigenvalues, any order (those outside [lo, hi] are ignored).
 *   out, counts: host arrays of cap entries: the contours in ascending order and the predictions in
 *   each closed interval.  *nout: number of contours (also set when cap is too small).
 * Errors: GCIE_EINVAL for bad arguments or cap < *nout (nothing written then). */
int gcie_plan_contours(const double *pred, int32_t npred, double lo, double hi, int32_t max_contours, double alpha,
                       gcie_contour *out, int32_t *counts, int32_t cap, int32_t *nout);

/* Count check of a finished contour (the judge of gcie_opts).  est is the stochastic trace estimate
 * of the number of eigenvalues the contour encloses, mean_l v_l^T (S_0)_l over the L columns of the
 * Gaussian starting block V (Section 2, CI eigensolvers: eigenvalue counts by stochastic trace
 * estimation; E[v^T S_0] = trace of the quadrature filter), se its standard error std_l / sqrt(L).
 * theta, res: host, the q Ritz values and residuals of the contour's last iteration; rank: the
 * dimension of its basis.  *miss = 1 when every Ritz value lies on the diameter [c - r, c + r]
 * (on >= rank: the basis has no spare direction) or est exceeds the converged ones there
 * (res <= tol) by more than max(1.5, 3 se); else 0.  Host only.  Errors: GCIE_EINVAL. */
int gcie_count_miss(double est, double se, const double *theta, const double *res, int32_t q, double c,
                    double r, int32_t rank, double tol, int32_t *miss);

/* The two contours that replace one that failed the count check: [lo, t] and [t, hi], t the
 * minimiser of the KDE sparsity function G_k (Algorithm 2) of the Ritz values in [lo, hi], searched
 * between their quartiles (the (k/4)-th and (k-1-k/4)-th of k sorted) so that the cut lies in a gap
 * and each half keeps a quarter of them; the midpoint when fewer than two distinct values lie
 * between the quartiles or the cut is not strictly inside.  Both halves keep the parent's ratio
 * r / ((hi - lo)/2).  theta: host, q values; out: host, 2 contours.  Host only.
 * Errors: GCIE_EINVAL unless lo < hi, r > 0, w > 0. */
int gcie_resplit(const double *theta, int32_t q, const gcie_contour *parent, double w, gcie_contour *out);

/* ------------------------------------------------------------------ steps of the path
 * Device-pointer entry points for the individual steps, used by the parity tests and by
 * callers that drive the pipeline themselves.  Each runs the same kernels as gcie_solve. */

/* Nodes and weights of the N-point trapezoid rule on |z - c| = r, upper half only
 * (Section 4.2; Eq. quadrature_appendix): theta_j = 2 pi (j - 1/2)/N, z_j = c + r e^{i theta_j},
 * w_j = r e^{i theta_j} / N, j = 1..N/2.  h_z, h_w: host, N/2 complex each. */
int gcie_trapezoid_nodes(double c, double r, int32_t N, double *h_z, double *h_w);

/* Step a4 (fused multi-shift SpMM): for each shift s and column l,
 *   Q[s][i][l] = z_s (M P[s])[i][l] - (K P[s])[i][l].
 * d_P, d_Q: FP32 complex, nshift blocks of n x ncol row-major.  h_z: host, nshift complex. */
int gcie_shifted_spmm_f32(gcie_ctx *ctx, gcie_pencil *p, int32_t nshift, const double *h_z,
                          int32_t ncol, const float *d_P, float *d_Q);
/* The same operator in FP64 (used by the refinement residual): d_P, d_Q FP64 complex. */
int gcie_shifted_spmm_f64(gcie_ctx *ctx, gcie_pencil *p, int32_t nshift, const double *h_z,
                          int32_t ncol, const double *d_P, double *d_Q);

/* Steps a4-a6 (shifted block solves): X[s] = (z_s M - K)^{-1} B for every shift s, by batched
 * COCG (FP32 with FP64 refinement for GCIE_MIXED, FP64 for GCIE_FP64) on the symmetrically
 * scaled system D^-1/2 (z_s M - K) D^-1/2 (D = diag K, or diag M if some K_ii <= 0), to
 * ||D^-1/2 (B - A X[s])||_2 / ||D^-1/2 B||_2 <= lin_tol per column.
 * d_B: FP64 real n x ncol row-major (shared by all shifts); d_X: FP64 complex, nshift blocks of
 * n x ncol row-major; if x0 != 0, d_X holds the initial guess on entry.  precond: a GCIE_PREC_*
 * value; GCIE_PREC_BAND factors every shifted matrix as a complex-symmetric band L D L^T in FP32 and
 * uses the factors as the COCG preconditioner (bandwidth limited by shared memory; in GCIE_FP64 mode the
 * factors stay FP32: the residual is rounded to FP32 for their sweeps and the result widened back,
 * while the COCG recurrences, the SpMM and the residual checks run in FP64),
 * GCIE_PREC_AMG applies the multigrid V-cycle (hierarchy built on the first call for this pencil and
 * kept with it), GCIE_PREC_AUTO picks the band factors when possible, GCIE_PREC_NONE runs plain COCG.
 * h_iters (host, may be NULL) receives the COCG iterations used.  Errors: GCIE_ENOCONV if a column missed lin_tol
 * within max_iters, or its true residual stopped decreasing (no 4x drop over 4 refinements); d_X then
 * holds the last iterate. */
int gcie_shifted_solve(gcie_ctx *ctx, gcie_pencil *p, int32_t nshift, const double *h_z,
                       int32_t ncol, const double *d_B, double *d_X, int32_t x0, double lin_tol,
                       int32_t max_iters, int32_t precision, int32_t precond, int64_t *h_iters);

/* Step a7 (moments): S_k += 2 Re( w_s ((z_s - c)/r)^k X[s] ), k = 0..m-1, summed over the nshift
 * upper-half nodes.  d_X as in gcie_shifted_solve; d_S: FP64 n x (m*ncol) row-major, column
 * k*ncol + l holds S_k[:, l]; accumulated into (zero it first for a fresh sum). */
int gcie_moments(gcie_ctx *ctx, int64_t n, int32_t nshift, const double *h_z, const double *h_w,
                 double c, double r, int32_t m, int32_t ncol, const double *d_X, double *d_S);

/* Step a8 (M-orthonormal basis of span Y): G = Y^T M Y, G = U diag(s) U^T (Jacobi), keep
 * s_i > drop * max s, Q = Y U_k diag(s_k)^-1/2; applied twice (the second pass restores
 * orthonormality lost to rounding).  d_Y: FP64 n x p row-major; d_Q: FP64 n x p row-major
 * (columns >= *h_rank are zero).  Errors: GCIE_ENOTSPD if the rank is 0. */
int gcie_m_orthonormalize(gcie_ctx *ctx, gcie_pencil *p, int32_t ncolY, const double *d_Y,
                          double drop, double *d_Q, int32_t *h_rank);

/* Steps a9-a11 (Rayleigh-Ritz): Khat = Q^T K Q, Jacobi Khat = W diag(theta) W^T, Z = Q W,
 * residual_i = ||K z_i - theta_i M z_i||_2 / (||K||_1 ||z_i||_2).  d_Q: FP64 n x q row-major,
 * M-orthonormal; d_Z: FP64 n x q row-major; h_theta, h_res: host, q (theta ascending). */
int gcie_rayleigh_ritz(gcie_ctx *ctx, gcie_pencil *p, int32_t q, const double *d_Q, double *d_Z,
                       double *h_theta, double *h_res);

/* Cyclic Jacobi on a dense symmetric p x p FP64 matrix on the device (the small-eigensolve
 * kernel of steps a8 and a10).  d_A: row-major, destroyed; d_w: p eigenvalues ascending;
 * d_V: p x p row-major, column j = eigenvector j. */
int gcie_jacobi_eig(gcie_ctx *ctx, int32_t p, double *d_A, double *d_w, double *d_V);

/* ------------------------------------------------------------------ tensor-core products (tcgen05)
 * D = A B^T on the fifth-generation tensor cores, A row-major M x K (leading dimension lda), B row-major
 * N x K (ldb), D row-major M x N (ldd), all device memory on the context's device, caller-owned; the
 * call returns when D is written (synchronous on the context's stream).  M, N, K >= 1 (0 does nothing).
 * Errors: GCIE_EINVAL (sizes, leading dimensions, null pointers), GCIE_ETIMEOUT (a bounded wait for the
 * tensor cores expired), GCIE_ECUDA.
 *
 * gcie_gemm_tf32x3: FP32 operands; each is split into a TF32 head and tail (x = hi + lo) and
 *   D = Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T is accumulated in FP32, close to an FP32 product (per element
 *   within a few 2^-22 of sum_k |A_ik| |B_jk|).  The dense contractions of the shifted solves' band
 *   factors (Algorithm 1, "solve (z_j B - A) X_j = B V"; Eq. quadrature_appendix) are of this kind.
 * gcie_gemm_bf16: BF16 operands (uint16 bit patterns), FP32 accumulation, epilogue
 *   D = act(A B^T + bias), bias (N, FP32, may be NULL) and act = ReLU when relu != 0, else identity: the
 *   layers of the density predictor that stands in for the paper's spectrum predictor (Section 4.1). */
int gcie_gemm_tf32x3(gcie_ctx *ctx, int32_t M, int32_t N, int32_t K, const float *d_A, int32_t lda,
                     const float *d_B, int32_t ldb, float *d_D, int32_t ldd);
int gcie_gemm_bf16(gcie_ctx *ctx, int32_t M, int32_t N, int32_t K, const uint16_t *d_A, int32_t lda,
                   const uint16_t *d_B, int32_t ldb, const float *d_bias, int32_t relu, float *d_D, int32_t ldd);

/* ------------------------------------------------------------------ density predictor (learned contours)
 * A small network that predicts the eigenvalue density of a pencil of the 2D log-normal family from its
 * coefficient fields: the stand-in for the paper's spectrum predictor (Section 4.1: a neural operator
 * maps the PDE coefficients to the spectrum) whose prediction places the contours (Section 4.2,
 * Algorithm 3: predict, construct contours, solve).  Inference runs on the GPU: BF16 weights and
 * activations, FP32 accumulation on the tensor cores (gcie_gemm_bf16's kernel).
 *
 * Input: kappa and rho (the coefficients in K and M) on a G x G cell grid, G a multiple of 64; channel
 * c of the 64 x 64 input is the mean of log(kappa) (c = 0) or log(rho) (c = 1) over (G/64)^2 cells.
 * Bounds: the target interval [lo, hi] (0 < lo < hi) enters as u = (log lo - 6.5, log hi - 6.5).
 * Network (NHWC activations): four 3 x 3 convolutions, stride 2, zero padding 1, ReLU, channels
 * 2 -> 16 -> 32 -> 64 -> 64 (64 x 64 -> 4 x 4); the 4 x 4 x 64 features flattened in (y, x, channel)
 * order and followed by u (1026 values); fc1 1026 -> 512, ReLU; fc2 512 -> 256, softplus.  Output: the
 * expected number of eigenvalues in each of 256 equal bins of [lo, hi].
 * Weights: one FP32 array, in this order, each weight tensor followed by its bias:
 *   conv l (l = 1..4): W[Cout][3][3][Cin] (ky, kx, input channel), b[Cout];
 *   fc1: W[512][1026], b[512];  fc2: W[256][512], b[256]   (GCIE_DENSITY_NWEIGHTS values in all).
 * The weights are rounded to BF16 on upload; each layer's input is rounded to BF16. */
#define GCIE_DENSITY_NWEIGHTS 717520
#define GCIE_DENSITY_BINS 256
typedef struct gcie_density_net gcie_density_net;
/* Upload the weights (host, nweights == GCIE_DENSITY_NWEIGHTS, finite) to the context's device.
 * Errors: GCIE_EINVAL, GCIE_ENOMEM, GCIE_ECUDA. */
int gcie_density_net_create(gcie_ctx *ctx, const float *h_weights, int64_t nweights, gcie_density_net **out);
void gcie_density_net_destroy(gcie_density_net *net);
/* Predict the histograms of `batch` pencils.  h_kappa, h_rho: host, batch x G x G FP32 (cell (y, x) of
 * member i at i G^2 + y G + x), positive; h_bounds: host, batch x 2 (lo, hi); h_hist: host, batch x 256,
 * written.  Errors: GCIE_EINVAL (G not a positive multiple of 64, batch < 1, bad bounds), GCIE_ENOMEM,
 * GCIE_ETIMEOUT, GCIE_ECUDA. */
int gcie_density_predict(gcie_ctx *ctx, gcie_density_net *net, int32_t batch, int32_t grid, const float *h_kappa,
                         const float *h_rho, const double *h_bounds, double *h_hist);
/* Pseudo-eigenvalues from a predicted histogram: with N = round(sum of the counts) (at most cap), the
 * k-th value (k = 1..N) is where the piecewise-linear cumulative count of the histogram over
 * [lo, hi] (counts spread evenly inside each bin) reaches k - 1/2; the spectrum the contour planners
 * (gcie_plan_contours, gcie_kde_contours) take as their prediction (Algorithm 3).  Host only.
 * hist: host, nbins >= 1 non-negative counts; out: host, cap values, ascending; *nout = N.
 * Errors: GCIE_EINVAL (bad arguments, or N > cap: nothing written then). */
int gcie_hist_quantiles(const double *hist, int32_t nbins, double lo, double hi, double *out, int32_t cap,
                        int32_t *nout);

/* FP64 throughput of the context's GPU on its two FP64 paths, measured by two short kernels (about a
 * millisecond each): CUDA-core FMAs and FP64 tensor MMAs (mma.sync m8n8k4; tcgen05 has no FP64 kind), in
 * TFLOP/s.  The dense products of the basis and of the projection (Algorithm 1, "orth", "project") and the
 * refinement residual run in FP64; the probe shows which path is faster on this part and is the FP64 peak
 * of their roofline.  Errors: GCIE_EINVAL, GCIE_ECUDA. */
int gcie_fp64_rates(gcie_ctx *ctx, double *h_fma_tflops, double *h_mma_tflops);

/* The same eigensolve for callers that must not allocate device memory.  (The paper has no
 * counterpart; this entry point exists for integration only.)  Some callers cannot call cudaMalloc:
 * a process that reserves all device memory for its own pool up front has none left to give, and a
 * thread driving a latency-critical stream cannot accept the device-wide synchronisation that
 * cudaMalloc/cudaFree may cause.  This variant takes no context and allocates nothing: its p x p
 * workspace is a fixed array in the library's device memory (512 KB per GPU, held until exit).
 *   stream: a cudaStream_t (NULL = legacy default stream); the call only enqueues the kernel, results
 *           are ready when the stream has passed it.
 *   p: 1..256; larger p returns GCIE_EINVAL ("exceeds the fixed workspace").
 *   d_A, d_w, d_V: as in gcie_jacobi_eig (device, caller-owned).
 * The first call on a device looks up the workspace's device address (once, with that device
 * current); make that first call before any stream capture.  The looked-up address is kept for the
 * life of the process and is not refreshed after a device reset (cudaDeviceReset): do not call this
 * entry point on a device that was reset after its first call.  All calls on a device share the
 * workspace, so calls that overlap on the GPU (other streams, other threads) race and must be
 * ordered by the caller. */
int gcie_jacobi_eig_noalloc(void *stream, int32_t p, double *d_A, double *d_w, double *d_V);

#ifdef __cplusplus
}
#endif
#endif /* GCIE_H */
