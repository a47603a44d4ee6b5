/*
 * feast_nl.h -- C ABI of a GB300 (sm_103a) library for the contour-quadrature
 * filter of nonlinear FEAST (Gavin, Miedlar, Polizzi, "FEAST Eigensolver for
 * Nonlinear Eigenvalue Problems", arXiv 1801.09794).
 *
 * Problem (Sec. 2, Eq. NLEVP and the matrix polynomial P(lambda) = sum_i lambda^i A_i):
 *     find lambda inside a closed contour C and x != 0 with T(lambda) x = 0,
 *     T(lambda) = sum_t scale_t * f_t(lambda) * A_t,
 *     f_t(lambda) = lambda^p            (FEAST_NL_POW), or
 *     f_t(lambda) = exp(-tau*lambda)    (FEAST_NL_EXP, the non-polynomial case of Sec. 6).
 *
 * Method (Algorithm 1): node matrices T(z_j) are factored once per contour; each
 * iteration projects T onto the subspace Q (Step 1), keeps the m0 Ritz pairs
 * closest to the interior of C (Step 2), tests the residuals (Step 3), applies
 * the quadrature filter
 *     Q = sum_j omega_j (X - T(z_j)^{-1} T(X, Lambda)) (z_j I - Lambda)^{-1}   (Step 4)
 * and orthonormalises Q (Step 5).  All of it runs on the GPU.
 *
 * Conventions for every entry point:
 *   - Matrices crossing the ABI are complex128 (interleaved re, im doubles),
 *     row-major ("C order", as numpy / torch store them).
 *   - A pointer may be host or device memory; the library asks the CUDA driver
 *     which one it is (terms say it explicitly with on_device).  The caller
 *     keeps ownership of every buffer it passes; the library copies inputs
 *     before returning and never keeps a caller pointer.
 *   - Every function returns a status (FEAST_NL_OK == 0 on success); no C++
 *     exception, abort or exit crosses the ABI.  feast_nl_last_error() gives a
 *     one-line reason for the last failure on the calling thread.
 *   - A handle is not thread-safe: use one handle per host thread.  Each handle
 *     works on its own CUDA stream (created by the library, or the caller's).
 *   - Device memory is owned by the handle and freed by feast_nl_destroy().
 */
#ifndef FEAST_NL_H
#define FEAST_NL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FEAST_NL_OK              0
#define FEAST_NL_EINVAL          1  /* bad argument (size, pointer, enum, order of calls) */
#define FEAST_NL_ESINGULAR_NODE  2  /* T(z_j) singular, or a Ritz value equal to a node z_j */
#define FEAST_NL_ENOT_CONVERGED  3  /* maxit reached; results of the last iterate are readable */
#define FEAST_NL_ETOO_MANY       4  /* all m0 kept Ritz values are inside C: m0 is too small
                                       (Algorithm 1 needs fewer than m0 eigenvalues inside) */
#define FEAST_NL_ENOMEM          5  /* device or host allocation failed */
#define FEAST_NL_EDEVICE         6  /* CUDA error, or a device-side iteration limit was hit */
#define FEAST_NL_EUNSUPPORTED    7  /* valid request this build does not implement */

/* ---- enums --------------------------------------------------------------- */
enum feast_nl_fkind { FEAST_NL_POW = 0, FEAST_NL_EXP = 1 };

/* Arithmetic of the node factorisations and solves (Step 4).  In every mode the
 * block residual T(X, Lambda) and the projections Q^H A_t Q are FP64-accurate,
 * and so are the kept Ritz pairs: the reduced problem's eigenvalues are located
 * in FP32 (Hessenberg reduction and QR of the companion matrix), then every kept
 * pair is refined by Newton's method with FP64 residuals until it is an
 * eigenpair of the FP64 projected problem (with an FP64 factor, or the whole
 * stage in FP64, when the FP32 start does not converge).  The
 * orthonormalisation (Steps 0, 5) is two Cholesky-QR passes with the Gram
 * matrix and its Cholesky factor in FP32 and Q R^{-1} formed FP64-accurately:
 * Step 1 depends only on span(Q), which this keeps to FP64 rounding.
 *   FEAST_NL_FP64  : LU and solves in FP64.
 *   FEAST_NL_FP32  : LU and solves in FP32 (complex64).  The filter is a
 *                    residual inverse iteration (Sec. 4.2), so solve errors scale
 *                    with ||T(X, Lambda)|| and vanish as the pairs converge.
 *   FEAST_NL_FP32_I8 : as FP32, and the products A_t Q (block residual and
 *                    projections) run on the BF16 tensor cores through an
 *                    error-free split into seven 7-bit integer digit slices with
 *                    power-of-two row / column scales (exact integer sums,
 *                    recombined in FP64; relative error about 1e-14 of |A||Q|).
 *                    Needs n <= 22000; larger n falls back to FP64 products. */
enum feast_nl_precision { FEAST_NL_FP64 = 0, FEAST_NL_FP32 = 1, FEAST_NL_FP32_I8 = 2 };

/* Quadrature rule on the parametrised contour z(theta) = c + ra cos(theta) + i rb sin(theta),
 * omega_j = w_j z'(theta_j) / (2 pi i):
 *   FEAST_NL_GL        : Gauss-Legendre, nc points on theta in [0, 2 pi]
 *   FEAST_NL_TRAPEZOID : theta_j = 2 pi (j + 1/2) / nc, w_j = 2 pi / nc
 *   FEAST_NL_GL_HALVES : Gauss-Legendre, nc/2 points on each half [0, pi], [pi, 2 pi] */
enum feast_nl_rule { FEAST_NL_GL = 0, FEAST_NL_TRAPEZOID = 1, FEAST_NL_GL_HALVES = 2 };

/* ---- types --------------------------------------------------------------- */
typedef struct feast_nl_handle feast_nl_handle;   /* opaque */

/* One term scale * f(lambda) * A of T(lambda).
 *   kind, p, tau : f(lambda) = lambda^p (kind POW, 0 <= p <= 8) or exp(-tau lambda) (kind EXP).
 *   scale        : complex multiplier (scale_re + i scale_im).
 *   A            : n x n complex128, row-major with row stride lda (>= n) elements;
 *                  NULL means the identity matrix.
 *   on_device    : nonzero if A is device memory of the current CUDA device. */
typedef struct {
    int32_t kind;
    int32_t p;
    double tau;
    double scale_re;
    double scale_im;
    const void* A;
    int64_t lda;
    int32_t on_device;
    int32_t reserved;
} feast_nl_term;

/* Summary of a solve (filled by feast_nl_solve). */
typedef struct {
    int32_t iters;        /* executions of Step 1 */
    int32_t n_inside;     /* kept Ritz values strictly inside C */
    int32_t n_converged;  /* inside pairs with relative residual <= tol */
    int32_t status;       /* same value feast_nl_solve returned */
    double max_relres;    /* max relative residual over the inside pairs (0 if none) */
    double ms_factor;     /* device time of node assembly + LU (0 when reused) */
    double ms_iterate;    /* device time of all iterations */
} feast_nl_info;

/* ---- entry points ---------------------------------------------------------- */

/* Create a solver for T(lambda) = sum_t scale_t f_t(lambda) A_t of size n.
 * Copies every A_t to the device (transposed to the library's column-major
 * layout) and estimates ||A_t||_2 by 30 power iterations on A^H A from the
 * normalised all-ones vector (identity terms: 1); these norms scale the
 * relative residual of Step 3.
 *   h         : out, the new handle (NULL on failure).
 *   n         : 1 <= n <= 65536.
 *   nterms    : 1 <= nterms <= 16.
 *   precision : enum feast_nl_precision.
 *   stream    : cudaStream_t to run on, or NULL for a library-owned stream.
 * Errors: EINVAL, ENOMEM, EDEVICE. */
int feast_nl_create(feast_nl_handle** h, int64_t n, int32_t nterms,
                    const feast_nl_term* terms, int32_t precision, void* stream);

/* Set the contour C and its quadrature (Algorithm 1 inputs), assemble every
 * T(z_j) on the device and LU-factor it with partial pivoting (the shifts are
 * fixed, so this is done once per contour and reused by every iteration).
 *   c_re, c_im : center; ra, rb > 0 : semi-axes along the real and imaginary
 *   axes (a circle when equal); 1 <= nc <= 1024 nodes; rule : enum feast_nl_rule.
 * Errors: EINVAL, ENOMEM, ESINGULAR_NODE (a zero pivot: a node sits on an
 * eigenvalue), EDEVICE. */
int feast_nl_set_contour(feast_nl_handle* h, double c_re, double c_im, double ra,
                         double rb, int32_t nc, int32_t rule);

/* Run Algorithm 1 with a subspace of m0 columns until every kept Ritz pair
 * strictly inside C has relative residual
 *     ||T(lambda_i) x_i||_2 / sum_t |scale_t f_t(lambda_i)| ||A_t||_2 <= tol,  ||x_i||_2 = 1,
 * (tested after at least one filter application) or maxit executions of Step 1.
 *   m0   : 1 <= m0 <= min(n, 112).
 *   X0   : n x m0 complex128 row-major start block (host or device), or NULL to
 *          draw one on the device from `seed` (complex normal, counter-based).
 *   info : optional out summary.
 * Step 1-2 for polynomial T (POW terms only): the first companion
 * linearisation of the projected polynomial (Sec. 2).  With any EXP term
 * (e.g. the delay problem T = -lambda I + A0 + A1 e^{-tau lambda}), the paper
 * names no reduced solver: the projected problem is solved by the first two
 * contour moments of its inverse (Beyn's method) on the contour scaled by 1.5
 * (256 trapezoid nodes; FP32 node LUs, moments summed in FP64 in a fixed order,
 * FP32 SVD with the rank cut at 1e-5 sigma_1, above FP32 noise), then Newton per
 * pair with FP64 residuals (FP64 factor when the FP32 one does not converge),
 * which makes each kept pair FP64-accurate; slots the moments leave
 * empty hold lambda = c + 1.5 ra (outside C) and are never tested.  There
 * m0 <= 64.
 * Returns OK, ENOT_CONVERGED, ETOO_MANY, ESINGULAR_NODE, EINVAL, ENOMEM,
 * EDEVICE.  After OK, ENOT_CONVERGED or ETOO_MANY the last iterate is
 * readable with feast_nl_get_eigpairs. */
int feast_nl_solve(feast_nl_handle* h, int32_t m0, double tol, int32_t maxit,
                   uint64_t seed, const void* X0, feast_nl_info* info);

/* Copy out the kept Ritz pairs of the last solve, in the order of Step 2
 * (increasing normalised radius).
 *   capacity    : number of pairs the buffers hold.
 *   m_out       : out, number of pairs written (<= capacity).
 *   lambda      : 2*capacity doubles (re, im), host or device; may be NULL.
 *   X           : n x capacity complex128 row-major (column i = x_i, unit 2-norm),
 *                 host or device; may be NULL.
 *   relres      : capacity doubles, host or device; may be NULL.
 *   inside_only : nonzero to return only the pairs strictly inside C.
 * Errors: EINVAL (no solve yet, bad capacity), EDEVICE. */
int feast_nl_get_eigpairs(feast_nl_handle* h, int32_t capacity, int32_t* m_out,
                          double* lambda, void* X, double* relres, int32_t inside_only);

/* Quadrature nodes and weights in use (2*nc doubles each, host memory). */
int feast_nl_get_nodes(feast_nl_handle* h, double* z, double* omega);

/* Apply T(z_j)^{-1} with the stored factors of node j to an n x m block
 * (complex128 row-major, host or device), in the handle's LU precision.
 * Exposes the node solves of Step 4 for testing. */
int feast_nl_node_solve(feast_nl_handle* h, int32_t j, int32_t m, const void* R, void* Y);

/* One filter application (Step 4) without orthonormalisation: given unit
 * Ritz vectors X (n x m) and values lambda (2*m doubles), compute
 * T(X, Lambda) and Q = sum_j omega_j (X - T(z_j)^{-1} T(X, Lambda)) (z_j I - Lambda)^{-1}.
 * X, Q: complex128 row-major, host or device; 1 <= m <= min(n, 112). */
int feast_nl_filter_apply(feast_nl_handle* h, int32_t m, const void* X,
                          const double* lambda, void* Q);

/* Projected coefficients of Step 1 for an n x m block Q (complex128 row-major):
 * Ahat_p = sum_{t: f_t = lambda^p} scale_t Q^H A_t Q for p = 0..k, written as
 * (k+1) consecutive m x m complex128 row-major matrices.  kmax_out receives k. */
int feast_nl_project(feast_nl_handle* h, int32_t m, const void* Q, void* Ahat,
                     int32_t* kmax_out);

/* Grouped factorisation: sets the contour of each of count handles (arrays of
 * count entries, as for feast_nl_set_contour, one rule for all) and factors
 * the node matrices of all of them, whatever their orders, in one launch
 * sequence per panel (Sec. 4.2: the nodes' linear systems are the independent
 * parallel work of the method; here nodes of different problems share each
 * launch).  Every handle needs complex64 factors (FP32 or FP32_I8) and
 * n <= 4096; at most 65535 nodes in all.  stream: where the assembly and the
 * factorisation run (NULL: a temporary stream); the call returns when they are
 * done, after which each handle solves on its own stream as usual.
 * Errors: EINVAL, ESINGULAR_NODE (an exact zero pivot), ENOMEM, EDEVICE; after
 * an error none of the group's handles has a contour. */
int feast_nl_set_contour_group(int32_t count, feast_nl_handle* const* hs, const double* c_re,
                               const double* c_im, const double* ra, const double* rb,
                               const int32_t* nc, int32_t rule, void* stream);

/* ---- serving: continuous batching of independent requests ------------------ */
/* No counterpart in the paper (its parallelism is over nodes and regions on
 * CPUs).  A request is one whole run of Algorithm 1 (create + contour +
 * solve) on its own handle and stream.  The server keeps up to max_active
 * requests in flight, admitting them in submission order while the summed
 * device-memory footprint (feast_nl_request_footprint) stays within
 * hbm_budget bytes (a request larger than the budget runs when nothing else
 * does).  The requests admitted together have their node matrices factored in
 * one grouped launch sequence (feast_nl_set_contour_group; complex128 factors
 * and n > 4096 one by one), then each is solved by a worker thread.  Requests
 * in flight overlap on the GPU; each one's results are the same bits as when
 * it runs alone.  The caller keeps the term buffers of a request alive until
 * the request is done.  All calls are thread-safe. */
typedef struct feast_nl_server feast_nl_server;
typedef struct {
    int64_t n;
    int32_t nterms;
    const feast_nl_term* terms;   /* as for feast_nl_create */
    int32_t precision;
    double c_re, c_im, ra, rb;    /* contour, as for feast_nl_set_contour */
    int32_t nc, rule;
    int32_t m0;                   /* as for feast_nl_solve (start block drawn from seed) */
    double tol;
    int32_t maxit;
    uint64_t seed;
} feast_nl_request;

/* Estimated device bytes of one request (coefficients, node factors, digit
 * slices, subspace blocks); host-only; -1 for an invalid request. */
int64_t feast_nl_request_footprint(const feast_nl_request* r);
/* 1 <= max_active <= 64 worker threads; hbm_budget > 0 bytes. */
int feast_nl_server_create(feast_nl_server** s, int32_t max_active, int64_t hbm_budget);
/* Queues a request; *ticket identifies it.  Errors: EINVAL. */
int feast_nl_server_submit(feast_nl_server* s, const feast_nl_request* r, uint64_t* ticket);
/* *state: 0 queued, 1 running, 2 done.  Errors: EINVAL (unknown ticket). */
int feast_nl_server_poll(feast_nl_server* s, uint64_t ticket, int32_t* state);
/* Blocks until the request is done; returns the status of its run (as
 * feast_nl_solve), fills info and the time from submission to completion. */
int feast_nl_server_wait(feast_nl_server* s, uint64_t ticket, feast_nl_info* info,
                         double* latency_ms);
/* Copies the kept Ritz pairs of a done request into host buffers (layouts as
 * feast_nl_get_eigpairs) and releases the ticket; returns the run's status.
 * EINVAL for an unknown, unfinished or already fetched ticket, and while
 * another thread is still inside feast_nl_server_wait on the same ticket (the
 * ticket is released only once no thread waits on it). */
int feast_nl_server_fetch(feast_nl_server* s, uint64_t ticket, int32_t capacity, int32_t* m_out,
                          double* lambda, void* X, double* relres, int32_t inside_only);
/* At most `limit` requests admitted together are factored as one group (1:
 * every request factored on its own); default 64.  Errors: EINVAL. */
int feast_nl_server_set_group_limit(feast_nl_server* s, int32_t limit);
/* Largest number of requests seen in flight at once, requests completed, and
 * the largest group admitted (and factored) together (any pointer may be NULL). */
int feast_nl_server_stats(feast_nl_server* s, int32_t* max_concurrent, int64_t* completed,
                          int32_t* max_group);
/* Finishes every submitted request, then stops the workers. */
void feast_nl_server_destroy(feast_nl_server* s);

/* ---- spectrum slicing: many contours of one problem ------------------------- */
/* Sec. 1 and Sec. 3: disjoint regions of the complex plane are solved
 * independently of one another.  A slicing set holds ndisc such contours of the
 * problem of a handle, each with nc nodes of the given rule; it assembles and
 * factors all ndisc * nc node matrices in one batch (create), then runs
 * Algorithm 1 for every contour at once (solve): each iteration forms A_t Q for
 * all contours in one product and solves all node systems in one batch, and
 * the per-contour steps run side by side.  Every contour keeps its pairs from
 * the iteration at which it passed Step 3 (or from maxit).  The handle must
 * outlive the set and is only read by it; the set owns its own stream and
 * device memory (node factors: ndisc * nc * n * n elements in the handle's LU
 * precision). */
typedef struct feast_nl_slices feast_nl_slices;
/* Contour d: center c_re[d] + i c_im[d], semi-axes ra[d], rb[d] (host arrays of
 * ndisc doubles).  1 <= ndisc <= 4096, 1 <= nc <= 1024, ndisc * nc <= 65535.
 * stream: cudaStream_t the set's work is ordered on (its per-contour steps fork
 * from and join back into it), or NULL for a stream of its own.
 * Errors: EINVAL, ESINGULAR_NODE (an exact zero pivot), ENOMEM, EDEVICE. */
int feast_nl_slices_create(feast_nl_slices** s, feast_nl_handle* h, int32_t ndisc,
                           const double* c_re, const double* c_im, const double* ra,
                           const double* rb, int32_t nc, int32_t rule, void* stream);
/* Solve flags. */
#define FEAST_NL_SLICES_NO_GRAPH 1   /* launch every iteration's kernels one by one */
/* Algorithm 1 on every contour with m0 columns each (arguments as for
 * feast_nl_solve; the start blocks of all contours are one n x (ndisc m0)
 * block drawn from seed, contour d taking columns d m0 .. d m0 + m0 - 1).
 * Unless flags has FEAST_NL_SLICES_NO_GRAPH, the iteration after the first is
 * captured once as a CUDA graph and replayed.  infos: host array of ndisc
 * (may be NULL).  Returns OK when every contour converged, else the status of
 * the first contour that did not (EDEVICE first). */
int feast_nl_slices_solve(feast_nl_slices* s, int32_t m0, double tol, int32_t maxit,
                          uint64_t seed, int32_t flags, feast_nl_info* infos);
/* Contour d's kept pairs, layouts and ordering as feast_nl_get_eigpairs. */
int feast_nl_slices_get_eigpairs(feast_nl_slices* s, int32_t disc, int32_t capacity,
                                 int32_t* m_out, double* lambda, void* X, double* relres,
                                 int32_t inside_only);
/* Kernel launches in one replay of the last solve's iteration graph (0 when
 * it ran without a graph). */
int64_t feast_nl_slices_graph_launches(feast_nl_slices* s);
void feast_nl_slices_destroy(feast_nl_slices* s);

/* ---- environment ------------------------------------------------------------ */
/* Read by the library at the calls named; none changes a result's bits except
 * where stated.
 *   FEAST_NL_TRACE=1                : every iteration's kept Ritz values, residuals
 *                                     and status on stderr (solve runs eagerly).
 *   FEAST_NL_PANEL_ROWS_PER_CTA=r   : complex64 LU panels taller than r rows are
 *                                     factored by a cluster of up to 8 CTAs, one per
 *                                     r rows (default 1024; 0 = one CTA per panel).
 *                                     Same factors for every r.
 *   FEAST_NL_LU_PERSISTENT=1        : the complex64 factorisation of set_contour,
 *                                     feast_nl_set_contour_group and the slicing
 *                                     set (orders <= 4096) runs as one persistent
 *                                     launch over all nodes instead of launches per
 *                                     panel step.  Same factors; slower on the
 *                                     measured workloads, so off by default. */

/* ---- measurement ------------------------------------------------------------ */
/* Phases of the path, for feast_nl_get_profile. */
enum feast_nl_phase {
    FEAST_NL_PH_ASSEMBLE = 0,  /* T(z_j) for all nodes                          */
    FEAST_NL_PH_LU = 1,        /* node LU factorisations                          */
    FEAST_NL_PH_APPLY = 2,     /* W_t = A_t Q (FP64)                              */
    FEAST_NL_PH_PROJECT = 3,   /* Q^H W_t and the projected coefficients          */
    FEAST_NL_PH_REDUCED = 4,   /* reduced eigenproblem, selection, Ritz vectors y */
    FEAST_NL_PH_RITZ = 5,      /* X = Q Y, T(X, Lambda), residual test            */
    FEAST_NL_PH_SOLVE = 6,     /* node solves T(z_j)^{-1} T(X, Lambda)            */
    FEAST_NL_PH_ACCUM = 7,     /* quadrature weights and accumulation into Q      */
    FEAST_NL_PH_ORTH = 8,      /* orthonormalisation (Steps 0 and 5)              */
    FEAST_NL_PH_IO = 9,        /* start-block upload                              */
    FEAST_NL_NPHASES = 10
};

/* Turn per-phase device timing on (nonzero) or off, and reset its totals.
 * When on, every phase of set_contour and solve is bracketed by CUDA events
 * on the handle's stream. */
int feast_nl_set_profiling(feast_nl_handle* h, int32_t on);

/* Iteration graph of feast_nl_solve (on by default): from the second
 * iteration on, Steps 4, 5 and 1-3 of Algorithm 1 (node solves, accumulation,
 * orthonormalisation, A_t Q, Rayleigh-Ritz, residual test) are captured once
 * per solve as one CUDA graph and replayed; the host reads only the residual
 * summary between replays.  Results are bit-identical with and without the
 * graph.  Per-phase profiling (feast_nl_set_profiling) and the trace output
 * run the iteration eagerly.  on: nonzero = use the graph. */
int feast_nl_set_iteration_graph(feast_nl_handle* h, int32_t on);

/* Totals since the last feast_nl_set_profiling: device milliseconds and kernel
 * launches per phase (arrays of nphases entries, host memory, may be NULL). */
int feast_nl_get_profile(feast_nl_handle* h, int32_t nphases, double* ms, int64_t* launches);

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t feast_nl_launch_count(void);

/* Failure-path self-test (no counterpart in the paper).  Every wait of the
 * tensor-core kernels on an mbarrier gives up after a bounded number of
 * cycles, sets bit 4 of the call's status (reported as EDEVICE) and lets the
 * kernel finish normally, so a lost arrival never hangs the GPU.  This runs
 * that wait, with a limit of `cycles` (1 .. 2^32), on a barrier that nothing
 * signals, and returns the status bits it left in *flags_out (16 when the
 * wait ran out, as it must).  The context stays usable afterwards. */
int feast_nl_selftest_bounded_wait(int64_t cycles, int32_t* flags_out);

/* ---- allocation-free Gram product --------------------------------------------
 * G = Q^H Q for a device-resident n x m block Q.  The paper has no counterpart:
 * this serves callers that must not touch the CUDA allocator (their device
 * memory belongs to another framework's pool, or they run where cudaMalloc /
 * cudaFree would stall or synchronise the device).  It allocates nothing and
 * needs no handle.
 *   Q      : device, complex128, COLUMN-major n x m with leading dimension ldq >= n.
 *   G      : device, complex128, COLUMN-major m x m (leading dimension m), written
 *            in full (G is Hermitian).
 *   stream : cudaStream_t or NULL; the call is asynchronous on that stream.
 * Limits: 1 <= n <= 2^30, n <= ldq <= 2^40, 1 <= m, m*m <= 262144 (m <= 512);
 * other sizes return EINVAL without touching the GPU.  Q and G must be device
 * memory of the current device, or managed memory (else EINVAL: the kernel runs
 * on the current device and must not reach into another GPU's memory).
 * The split-K partial sums live in one static 4 MiB device array that every GPU
 * loading this library holds until the process exits; every call overwrites the
 * partials it reads, so nothing needs clearing, but all calls share that array:
 * calls that overlap on the GPU (different streams, or other host threads) race.
 * The first call on each device looks up the array's device address with that
 * device current; make that first call before any stream capture. */
int feast_nl_gram_noalloc(int64_t n, int32_t m, const void* Q, int64_t ldq, void* G,
                          void* stream);

/* Free the handle and all its device memory.  NULL is ignored. */
void feast_nl_destroy(feast_nl_handle* h);

/* Static text for a status code. */
const char* feast_nl_strerror(int status);

/* One-line detail of the last failure on the calling thread ("" if none). */
const char* feast_nl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FEAST_NL_H */
