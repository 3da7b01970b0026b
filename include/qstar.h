/* qstar: the Pfaffian-sign hot path for QCD+QED with C* boundary conditions
 * (arXiv:2108.11989, Sec. 3), as a C-ABI library for one NVIDIA GB300 GPU.
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Lattice.  The physical lattice is T x L^3 with C* boundary conditions in the
 *   spatial directions and periodic (or antiperiodic) time.  The quark/antiquark
 *   doublet on which D acts (a 24V x 24V matrix, Sec. 3) is stored on the
 *   orientifold-doubled lattice T x L x L x 2L: sites with x in [0, L) hold psi,
 *   sites with x in [L, 2L) hold psi^C.  Moving across the y (or z) boundary moves
 *   x by L; x itself is periodic with period 2L.  N_s = 2 L^3 T doubled sites.
 * Directions.  mu = 0 (t), 1 (x), 2 (y), 3 (z).
 * Dirac basis.  Chiral basis, gamma_5 = diag(1, 1, -1, -1), C = i gamma_0 gamma_2.
 * Spinor layout ("canonical").  [rhs][t][z][y][x in 0..2L-1][spin 4][colour 3][re, im],
 *   double for QS_F64, float for QS_F32.  Buffers given to the apply calls are
 *   DEVICE pointers owned by the caller; in and out must not overlap.
 * Gauge layout (host input).  su3 [t][z][y][x in 0..L-1][mu 4][a 3][b 3][re, im]
 *   (physical lattice only, double); u1_theta [t][z][y][x][mu] (double) or NULL.
 *   The mirror half is derived inside (charge conjugate links).
 * Operator (Sec. 2: O(a)-improved Wilson quarks with SU(3) and U(1) SW terms;
 *   Sec. 3: Q = gamma_5 D):
 *     D psi(x) = (4 + m0) psi(x) + A(x) psi(x)
 *                - 1/2 sum_mu [ V(x,mu)(1 - gamma_mu) psi(x+mu) + V(x-mu,mu)^+ (1 + gamma_mu) psi(x-mu) ]
 *     V = U exp(i theta),  A = (i/4) sum_{mu,nu} sigma_{mu nu} (c_sw F^SU3 + c_sw,U1 F^U1),
 *     F = clover field strength (Q_{mu nu} - Q_{nu mu}) / 8.
 *
 * Errors.  Every call returns 0 (QS_OK) or a negative code below; none aborts the
 *   process.  On error the contents of output buffers are unspecified.
 *   qs_strerror() gives a static message.
 * Streams.  All GPU work of a lattice handle runs on the stream given at creation
 *   (NULL = the legacy default stream).  Calls on one handle must not overlap; calls on
 *   different handles may run in different host threads.
 * No CPU fallback: a call that cannot run on the GPU returns QS_ECUDA.
 */
#ifndef QSTAR_H
#define QSTAR_H

#include <stdint.h>

#if defined(__GNUC__)
#define QS_API __attribute__((visibility("default")))
#else
#define QS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum qs_status {
    QS_OK = 0,
    QS_EINVAL = -1,      /* bad argument (size, pointer, precision, call order) */
    QS_ENOMEM = -2,      /* device allocation failed */
    QS_ECUDA = -3,       /* CUDA runtime error (message in qs_last_cuda_error) */
    QS_ENOCONV = -4,     /* an iteration hit its cap before reaching its tolerance */
    QS_ETIMEOUT = -5,    /* a bounded device wait gave up */
    QS_ENUMERIC = -6,    /* NaN / Inf met in a reduction */
    QS_EUNDECIDED = -7   /* |lambda| at the target mass is below its certified accuracy */
};

/* Precision of the spinors given to the operator calls.  QS_F64: double, FP64
 * arithmetic.  QS_F32: float, FP32 arithmetic.  QS_F16 / QS_BF16: 16-bit storage with
 * FP32 arithmetic, in the tiled layout only (OR QS_LAYOUT_TILED into prec): tiles of 16
 * sites, each 12 x 16 words of two 16-bit reals (re, im of component c of site
 * 16 t + j at word 16 c + j) followed by 16 FP32 scales, 832 bytes per tile; site j's 24
 * reals are stored divided by its scale (the largest of their magnitudes), so a
 * vector takes 52 bytes per site.  Outputs are written in the same format. */
enum qs_prec { QS_F64 = 0, QS_F32 = 1, QS_F16 = 2, QS_BF16 = 3 };

/* OR into the prec argument of qs_apply_Dw / qs_apply_Q to pass spinors in the
 * solver's site-tiled layout [rhs][site / 16][spin-colour 12][site % 16][re, im]
 * (site = canonical site index) instead of the canonical one. */
#define QS_LAYOUT_TILED 16

typedef struct qs_lattice qs_lattice;

typedef struct {
    int L, T;            /* physical extents; L even, L >= 2, T >= 2, 2 L^3 T < 2^30 */
    int cstar_mask;      /* bit k-1: C* in spatial direction k (bit 0 = x, required) */
    int t_antiperiodic;  /* 0: periodic in time (Sec. 2), 1: antiperiodic for fermions */
    int device;          /* CUDA device ordinal */
} qs_geom;

/* Create a lattice handle (Sec. 3 geometry).  stream: a cudaStream_t or NULL.
 * Allocates nothing large until qs_load_gauge.  *out receives the handle. */
QS_API int qs_create_lattice(const qs_geom *geom, void *stream, qs_lattice **out);

/* Release every device buffer of the handle.  NULL is accepted. */
QS_API int qs_destroy_lattice(qs_lattice *lat);

/* Number of doubled sites N_s = 2 L^3 T (0 for a NULL handle). */
QS_API int64_t qs_n_sites(const qs_lattice *lat);

/* Load a gauge configuration (Sec. 2: SU(3) x U(1) links, c_sw's) from HOST arrays
 * (layouts above; copied, the caller keeps ownership), build the doubled links and
 * the SW term A(x) on the GPU in FP64, and keep FP64 and FP32 copies resident.
 * Replaces any earlier configuration of the handle.  Synchronises the stream.
 * Returns QS_ENUMERIC (and leaves no field loaded) if a link, an angle or the SW
 * term built from them is NaN or infinite. */
QS_API int qs_load_gauge(qs_lattice *lat, const double *su3, const double *u1_theta,
                  double csw_su3, double csw_u1);

/* out = D(m0) in for nrhs <= 64 vectors (Sec. 2 operator on the doubled lattice, Sec. 3).
 * in, out: device buffers of nrhs vectors, canonical layout (or the tiled one with
 * QS_LAYOUT_TILED), in precision prec (QS_F64: double, arithmetic in FP64; QS_F32:
 * float, arithmetic in FP32; QS_F16 / QS_BF16: tiled 16-bit storage, arithmetic in
 * FP32, see enum qs_prec).  Vectors are contiguous: N_s * 24 reals each, or N_s * 52
 * bytes in 16-bit storage; 16-byte aligned.  Asynchronous on the handle's stream.
 * The first call for a (precision, layout, nrhs) on a lattice shape times the launch
 * variants of the kernel once on the stream (writing only `out`); if the environment
 * variable QS_TUNE_CACHE names a file, choices are read from it and new ones appended,
 * so later processes on the same GPU model skip the timing. */
QS_API int qs_apply_Dw(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, int prec);

/* out = Q(m0) in = gamma_5 D(m0) in (Sec. 3).  Same arguments as qs_apply_Dw. */
QS_API int qs_apply_Q(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, int prec);

/* out = P in = C T gamma_5 in^* for nrhs FP64 spinors (prec = QS_F64, optionally with
 * QS_LAYOUT_TILED): the antiunitary symmetry of Sec. 3 -- if Q v = lambda v then P v is
 * an eigenvector with the same eigenvalue, orthogonal to v (the double degeneracy of
 * the spectrum of Q).  T is the translation by L along x, C = i gamma_0 gamma_2; P
 * commutes with Q and P^2 = -1.  DEVICE buffers, not overlapping.  Asynchronous. */
QS_API int qs_cstar_partner(qs_lattice *lat, const void *in, void *out, int nrhs, int prec);

/* Convert nrhs spinors between precisions, both in the tiled layout (in_prec, out_prec:
 * QS_F64, QS_F32, QS_F16, QS_BF16, different; QS_LAYOUT_TILED may be ORed in).  Into 16
 * bits each site is scaled by its largest component; out of 16 bits the values are
 * expanded exactly.  DEVICE buffers, not overlapping, 16-byte aligned.  Asynchronous
 * on the handle's stream.  (Storage conversion; no counterpart in the paper.) */
QS_API int qs_convert_spinors(qs_lattice *lat, const void *in, int in_prec, void *out, int out_prec, int nrhs);

/* Several configurations in ONE launch (the batched form of the hot path: many
 * masses, several gauge configurations of uneven volume, blocks of vectors).
 * items[i].out = Q(m0_r) items[i].in for every right-hand side r < items[i].nrhs,
 * m0_r = items[i].m0[r] (host array).  Up to 8 items, up to 16 right-hand sides
 * each, all lattices on one device with their gauge fields loaded; buffers as for
 * qs_apply_Q (prec may carry QS_LAYOUT_TILED).  Runs on `stream` (a cudaStream_t or
 * NULL).  Returns QS_EINVAL for more items / right-hand sides, mixed devices,
 * overlapping in/out of an item. */
#define QS_BATCH_MAX_ITEMS 8
#define QS_BATCH_MAX_RHS 16
typedef struct {
    qs_lattice *lat;
    const void *in;
    void *out;
    int nrhs;
    const double *m0;   /* host, nrhs masses */
} qs_batch_item;

QS_API int qs_apply_Q_batch(const qs_batch_item *items, int n, int prec, void *stream);

/* ---------------------------------------------------------------------------
 * Step-proposal network (learned form of the flow; the paper steps with the fixed
 * rule m <- m + c lambda_bar of Sec. 3).  A 3-layer FP32 perceptron
 * in -> hidden -> hidden -> out with ReLU, trained on the GPU by the library's own
 * forward, backward and Adam kernels.  Parameters (host layout, row-major FP32):
 * [W1 (hidden x in), b1, W2 (hidden x hidden), b2, W3 (out x hidden), b3].
 * Loss over B rows with targets T (column 0 regression, columns 1.. labels in [0, 1]):
 *   L = (1/B) sum_b [ (Y_b0 - T_b0)^2 / 2 + sum_{j>=1} (softplus(Y_bj) - T_bj Y_bj) ].
 * Adam with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.  X, T, Y are DEVICE arrays.
 * ------------------------------------------------------------------------- */
typedef struct qs_mlp qs_mlp;
/* on the current device; stream: cudaStream_t or NULL; parameters start at zero */
QS_API int qs_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, void *stream, qs_mlp **out);
QS_API int qs_mlp_destroy(qs_mlp *net);
QS_API int64_t qs_mlp_n_params(const qs_mlp *net);
/* copy parameters in / out (host arrays of qs_mlp_n_params floats); set resets Adam */
QS_API int qs_mlp_set_params(qs_mlp *net, const float *host);
QS_API int qs_mlp_get_params(qs_mlp *net, float *host);
/* gradients of the last qs_mlp_train_step (host array of qs_mlp_n_params floats) */
QS_API int qs_mlp_get_grads(qs_mlp *net, float *host);
/* Y [B][out] = network(X [B][in]), B <= max_batch */
QS_API int qs_mlp_forward(qs_mlp *net, const float *X, int B, float *Y);
/* one Adam step on the batch (X [B][in], T [B][out]); *loss (host, may be NULL) = L
 * before the step */
QS_API int qs_mlp_train_step(qs_mlp *net, const float *X, const float *T, int B, float lr, float *loss);

/* ---------------------------------------------------------------------------
 * Low modes of Q(m0) (Sec. 3: lambda_bar = min_n |lambda_n| "by the power method
 * plus Chebyshev acceleration"; the eigenvalues closest to zero are what the
 * sign algorithm follows across masses).
 *
 * Method: block subspace iteration with Rayleigh-Ritz of Q in FP64.  While the
 * relative residuals are large, each pass applies a Chebyshev filter in Q^2 (FP32
 * storage and arithmetic) that damps the interval [theta_k^2, lambda_max^2];
 * near convergence, passes are power steps with Q^-2, each solve a CG on Q^2 with
 * FP32 inner iterations and FP64 defect correction.  Every eigenvalue returned is
 * a Ritz value of the FP64 Q with its residual r = ||Q v - theta v||, so some
 * eigenvalue of Q lies in [theta - r, theta + r].
 * ------------------------------------------------------------------------- */
typedef struct {
    int k;             /* block size = eigenpairs returned, even, 2..64 */
    int nwant;         /* the nwant smallest |theta| must meet tol (1..k) */
    double tol;        /* target: r_i <= tol * |theta_i| for i < nwant, or r_i <= 1e-13 qn
                          (qn = |4 + m0| + max ||A(x)|| + 4 >= ||Q||), so that an exact zero
                          mode also ends the iteration (with |theta_i| - r_i <= 0) */
    int max_iter;      /* cap on subspace passes (filter + refinement) */
    int cheb_degree;   /* degree of the Q^2 Chebyshev filter (>= 2) */
    int warm_start;    /* 1: start from the subspace the handle kept from its last call */
    uint64_t seed;     /* seed of the random start block */
    int precision;     /* QS_F32: mixed form (FP32 filter, FP32-inner CG refinement, FP64
                          Rayleigh-Ritz); QS_F16 / QS_BF16: the mixed form with the filter's
                          vectors stored in 16 bits (per-site scale, FP32 arithmetic);
                          QS_F64: plain FP64 form (FP64 filter passes and FP64 Rayleigh-Ritz
                          only) */
    int pairing;       /* 1: in the mixed forms, filter and Q^-2 steps act on k / 2 vectors and
                          their C* partners C T gamma_5 v^* (qs_cstar_partner) complete the
                          block -- the spectrum is doubly degenerate (Sec. 3), so half the
                          operator work spans the same subspace; 0: all k vectors */
} qs_eig_opts;

typedef struct {
    int iterations;          /* subspace passes done */
    int filter_passes, refine_passes;
    int64_t dslash_f32, dslash_f64;   /* single-vector operator applications */
    int64_t cg_iterations;   /* inner FP32 CG iterations (per block) */
    double seconds;          /* wall time of the call */
} qs_eig_stats;

/* Fill *opts with defaults (k = 16, nwant = 4, tol = 1e-8, max_iter = 200,
 * cheb_degree = 24, warm_start = 1, seed = 1, precision = QS_F32, pairing = 1). */
QS_API void qs_eig_default_opts(qs_eig_opts *opts);

/* Lowest-|lambda| eigenpairs of Q(m0) on the handle's gauge field.
 * evals, resid: HOST arrays of k doubles, sorted by increasing |theta| (signed
 *   Ritz values and residual norms ||Q v - theta v||).
 * evecs: NULL, or a DEVICE buffer of k * N_s * 24 doubles (canonical layout) that
 *   receives the orthonormal Ritz vectors.
 * stats: NULL or receives counters.  Returns QS_ENOCONV (with the best values so
 * far written) if max_iter passes do not reach tol.  Synchronises the stream. */
QS_API int qs_lowmodes_at_mass(qs_lattice *lat, double m0, const qs_eig_opts *opts, double *evals,
                               double *resid, void *evecs, qs_eig_stats *stats);

/* ---------------------------------------------------------------------------
 * Sign of the Pfaffian (Sec. 3, eq. power1/4 and the enumerated algorithm).
 * W_sgn(m0) = (-1)^(number of zero crossings of eigenvalues of Q between m0 and
 * large mass), counted along the mass flow:
 *  step A (Sec. 3, steps 1-5): m <- m + c lambda_bar while lambda_bar does not
 *    decrease; stop with the sign found so far once m > m0_max.  lambda_bar is the
 *    smallest |theta| of the block and lo = min (|theta_j| - r_j) its certified lower
 *    bound.  Each step is certified by |lambda'| <= 1 (eq. derivativebound):
 *    lo_n + lo_{n+1} >= m_{n+1} - m_n; a step that fails it hands over to step B
 *    from m_n (or, with the retreat option, is shortened to m_n + 0.95 lo_n).
 *  step B (the paper defers it to other work; our reading): from the last
 *    certified mass, step by dm inside a spectral gap (a - dm, a + dm) of the
 *    tracked window and add the change of the number of eigenvalues in (-a, 0);
 *    return to step A when lambda_bar grows again.
 * ------------------------------------------------------------------------- */
#define QS_TRACE_MAX 1024

#define QS_WINDOW 24   /* eigenvalues per mass in the step model's features / traces */

struct qs_mlp;
typedef struct {
    double c;          /* step factor of step A, slightly below 2 */
    double m0_max;     /* step A stops above it; <= 0 selects 3 (c_sw + c_sw,U(1)) */
    int max_steps;     /* cap on masses visited */
    qs_eig_opts eig;   /* low-mode solver options (warm starts between masses) */
    /* optional learned step (NULL: the fixed rule).  Network with 8 * QS_WINDOW inputs:
     * the windows of the last 8 step-A masses (newest first, QS_WINDOW signed Ritz
     * values each in the solver's order, divided by the newest lambda_bar, zero where
     * missing); output 0 = log(dm / lambda_bar).  The proposal, clamped to
     * [c lambda_bar, 8 lambda_bar] so that it can only lengthen the plain step, replaces
     * c lambda_bar; the step is then certified exactly as a plain one. */
    struct qs_mlp *step_model;
    /* optional HOST buffer of max_steps * QS_WINDOW doubles: the window of every mass
     * visited, in visiting order (training data for the step model), or NULL */
    double *window_trace;
    /* 0 (default): the paper's order -- a step-A step that is not certified counts as
     * step 3 and step B starts from the last certified mass.  1: such a step is first
     * shortened to m + 0.95 lo (the edge of the crossing-free interval around m). */
    int retreat;
    /* optional path of a JSON-lines log: one line appended per mass visited (step, mass,
     * phase, lambda_bar, its lower bound, eigensolver work, seconds since the start), or NULL */
    const char *log_path;
    /* optional checkpoint file, or NULL.  After every certified mass (the start, each step-A
     * step, each counted step-B step) the flow state -- target mass, the certified mass, the
     * crossings counted up to it, steps taken, the lattice's extents, C* mask and c_sw's --
     * is written as one JSON object, atomically (temporary file, then rename). */
    const char *checkpoint_path;
    /* 1: if checkpoint_path exists and was written for the same target mass and lattice,
     * continue the flow from its certified mass with its crossing count (the window there
     * is solved again); otherwise start from the target.  0: always start from the target. */
    int resume;
} qs_sign_opts;

typedef struct {
    int n;                              /* masses visited */
    double mass[QS_TRACE_MAX];
    double lambda_bar[QS_TRACE_MAX];    /* min |theta| at that mass (block values with
                                           r <= |theta| / 2, and the converged ones) */
    double resid[QS_TRACE_MAX];         /* lambda_bar minus its certified lower bound
                                           min (|theta_j| - r_j) over the same values */
    char phase[QS_TRACE_MAX];           /* 'A' or 'B' */
    int crossings;                      /* zero crossings counted by step B */
    int steps_a, steps_b;
    int64_t dslash_f32, dslash_f64;
    int64_t cg_iterations;
    double seconds;
    int learned_accepted, learned_rejected;   /* step-model proposals certified / not */
    int fail_reason;   /* 0 ok; 1 an eigensolve missed its tolerance; 2 step B found no
                          spectral gap; 3 a step-B count was not certified (bounds straddle
                          the gap, or the window does not reach above it); 4 odd change of
                          the negative count; 5 max_steps reached; 6 lambda_bar - r <= 0 */
    int checkpoint_errors;   /* checkpoints that could not be written (the flow goes on) */
    double resumed_from;     /* the certified mass a resumed flow started from (else m0_target) */
} qs_sign_report;

/* Mass reweighting (Sec. 4).
 *
 * qs_ratapprox: the order-(n, n) rational function R(y) = A prod_i (y + nu_i^2) / (y + mu_i^2)
 * with the least uniform relative error |R(y) y^(1/4) - 1| for y in [ra^2, rb^2] (eq.
 * ratapprox; R(Q_hat^2) replaces (Q_hat^2)^(-1/4) in eq. detQ2, [ra, rb] the range of the
 * spectrum of |Q_hat|).  Host computation (no GPU work).  0 <= n <= 32, 0 < ra < rb.
 * nu, mu: HOST arrays of n values, returned in increasing order; *delta the maximal
 * relative error.  QS_ENOCONV if the Remez iteration does not level the error (orders far
 * beyond what double precision resolves). */
QS_API int qs_ratapprox(int n, double ra, double rb, double *A, double *nu, double *mu, double *delta);

/* qs_w_mass: the stochastic estimate of W_mass = det[R(Q_hat_m^2) R^-1(Q_hat_m'^2)] (eq. Wmass)
 * from the factors j = 1..n, each estimated with the nsrc sources eta as in Sec. 4:
 *   q[j * nsrc + l] = (eta_l, R_j eta_l),  R_j = X^+ + X + X^+ X,  X = (D_hat(m') - D_hat(m)) S_j,
 *   *log_w = sum_j log( (1/nsrc) sum_l exp(-q[j * nsrc + l]) ).
 * The mean of exp(-(eta, R_j eta)) over sources with density ~ exp(-(eta, eta)) estimates
 * 1/det(1 + R_j), whose product over j is W_mass exactly.  The normalisation A cancels.
 * nu, mu: HOST arrays of n > 0 values (from qs_ratapprox or any other choice).
 * eta: DEVICE buffer of nsrc <= 64 FP64 spinors in the canonical layout (complex Gaussian
 * entries of unit variance; the caller draws them).  Odd-site entries are ignored.
 * Shifted inverses: FP64 conjugate gradients on Q_hat^2 + shift^2, each to
 * ||r|| <= tol ||b||, at most max_iter iterations (QS_ENOCONV beyond).  q: HOST array of
 * n * nsrc; log_w, cg_iterations (total over all solves): HOST, may be NULL.  Allocates
 * 12 nsrc vectors of work and the odd-site block inverses at m and m' (2 x 1152 bytes per
 * odd physical site); synchronises the lattice's stream.  QS_EINVAL for odd T or L. */
QS_API int qs_w_mass(qs_lattice *lat, double m, double mp, int n, const double *nu, const double *mu,
                     const void *eta, int nsrc, double tol, int max_iter, double *q, double *log_w,
                     int *cg_iterations);

/* qs_solve_D: x = D(m0)^-1 b in FP64.  even_odd = 1: the even-odd preconditioned solve of
 * Sec. 4 -- b'_e = b_e - D_eo (D_oo)^-1 b_o, D_hat x_e = b'_e by conjugate gradients on
 * Q_hat^2 (half the sites, better conditioned), x_o = (D_oo)^-1 (b_o - D_oe x_e); requires even
 * T and L.  even_odd = 0: conjugate gradients on the full-lattice Q^2 (for comparison).
 * b, x: DEVICE buffers of nrhs <= 64 FP64 spinors, canonical layout, not overlapping.  The CG
 * stops at ||r|| <= tol ||rhs|| for every right-hand side (QS_ENOCONV after max_iter);
 * *iterations (may be NULL) gets the count.  Allocates 11 nrhs vectors of work (plus the
 * odd-site inverses, 1152 bytes per odd physical site); synchronises the stream. */
QS_API int qs_solve_D(qs_lattice *lat, double m0, const void *b, void *x, int nrhs, int even_odd, double tol,
                      int max_iter, int *iterations);

/* The bounds step A takes from one block of Ritz pairs (host arithmetic, no GPU work):
 * *lambda_bar = min |theta_j| and *lo = min (|theta_j| - res_j) over the values that carry
 * information: the first nwant (the converged ones) and every other one with
 * res_j <= |theta_j| / 2 (k <= 64).  The block is ordered by theta^2 + res^2, so the smallest lower
 * bound need not be the first value's.  theta, res: HOST arrays of k values.  Sec. 3 (the
 * derivative bound: no eigenvalue of Q crosses zero within lo of the mass). */
QS_API int qs_block_bounds(const double *theta, const double *res, int k, int nwant, double *lambda_bar,
                           double *lo);

/* Fill *opts with defaults (c = 1.9, m0_max = 0 (auto), max_steps = 400, eig defaults
 * with tol = 1e-5).  Step A also stops as soon as m + (lambda_bar - r) > m0_max. */
QS_API void qs_sign_default_opts(qs_sign_opts *opts);

/* *sign = W_sgn(m0_target) in {+1, -1}.  report may be NULL.  Returns
 * QS_EUNDECIDED if lambda_bar at the target is not certified > 0, QS_ENOCONV if
 * the flow exceeds max_steps or an eigensolve does not converge. */
QS_API int qs_pfaffian_sign(qs_lattice *lat, double m0_target, const qs_sign_opts *opts, int *sign,
                            qs_sign_report *report);

/* ---------------------------------------------------------------------------
 * Even-odd factor of the mass reweighting (Sec. 4).  With even-odd preconditioning the
 * reweighting factor from bare mass m to m' carries the exact factor
 *   W_eo = |det[D^oo_m' (D^oo_m)^-1]|^(1/2),
 * D^oo the operator restricted to the odd sites of the doubled lattice (parity
 * (t + z + y + x) mod 2).  No hopping term connects two odd sites, so D^oo is the
 * site-diagonal 4 + m0 + A(x) and its log-determinant is a sum of 6 x 6 block terms.
 * ------------------------------------------------------------------------- */

/* logdet[i] = sum over odd doubled sites x of log|det(4 + m0[i] + A(x))| (FP64) for
 * nmass <= 16 masses (host arrays).  Synchronises the stream.  QS_ENUMERIC if a block
 * is singular (log of zero) or the field is not finite. */
QS_API int qs_log_det_oo(qs_lattice *lat, int nmass, const double *m0, double *logdet);

/* *w_eo = W_eo(m -> mp) and *log_w_eo its logarithm (either may be NULL, not both). */
QS_API int qs_w_eo(qs_lattice *lat, double m, double mp, double *w_eo, double *log_w_eo);

/* The even-odd preconditioned operator of Sec. 4: out = D_hat(m0) in, with
 * D_hat = D_ee - D_eo (D_oo)^-1 D_oe on the even sites (gamma5 = 1: Q_hat = gamma_5 D_hat).
 * in, out: DEVICE buffers of nrhs <= 64 FP64 spinors in the canonical layout of the full
 * doubled lattice; the odd-site entries of in are ignored and those of out set to zero.
 * FP64 arithmetic (two operator applications and a site-local 6 x 6 solve per odd site);
 * allocates three work vectors per call; synchronises the stream.  QS_EINVAL for an odd T
 * or L (then a hop can join two sites of one parity), overlapping or unaligned buffers.  det D = det D_oo det D_hat,
 * which is why W_eo carries the D_oo part of a mass reweighting. */
QS_API int qs_apply_Dhat(qs_lattice *lat, double m0, const void *in, void *out, int nrhs, int gamma5);

/* W_sgn for n configurations at once (the batched form; Sec. 3 runs the algorithm on
 * each configuration independently).  lats: n distinct handles with gauge fields
 * loaded; m0_targets, signs, status: HOST arrays of n; reports: NULL or n reports.
 * The flows run concurrently, one host thread each on its handle's stream, so the GPU
 * overlaps their work -- give every handle its own stream (handles on one stream
 * serialise).  status[i] receives qs_pfaffian_sign's status for configuration i; the
 * return value is QS_OK if all succeeded, else the first failing status.  Synchronises
 * every stream. */
QS_API int qs_pfaffian_sign_batch(qs_lattice *const *lats, int n, const double *m0_targets,
                                  const qs_sign_opts *opts, int *signs, int *status, qs_sign_report *reports);

/* ---------------------------------------------------------------------------
 * Kernel profiling (measurement support, no counterpart in the paper).  While on,
 * every operator launch of the handle is bracketed by CUDA events on the handle's
 * stream; qs_get_profile synchronises the stream and reports per precision the
 * launches, their summed device time and their algorithmic bytes (per doubled site:
 * every right-hand side's spinor in and out -- plus two more spinors for the fused
 * Chebyshev step of the filter -- and once per launch 36 link + 36 SW-term reals, in
 * the operator's arithmetic precision).
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t launches;
    double ms;        /* summed event time of the launches */
    double bytes;     /* summed algorithmic bytes */
} qs_kernel_prof;

typedef struct {
    qs_kernel_prof dslash[4];   /* by spinor precision [QS_F64], [QS_F32], [QS_F16], [QS_BF16] */
} qs_profile;

/* on = 1 starts (and zeroes) the counters, on = 0 stops recording. */
QS_API int qs_set_profiling(qs_lattice *lat, int on);

/* Resolve the recorded events into *prof (synchronises the stream). */
QS_API int qs_get_profile(qs_lattice *lat, qs_profile *prof);

/* Number of CUDA kernels this library has launched in this process (all handles). */
QS_API int64_t qs_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Allocation-free operator application (the paper has no counterpart: this is
 * for callers that cannot allocate device memory when they apply the operator,
 * such as code running while a CUDA graph is captured, host callbacks, or
 * frameworks that own every allocation).
 *
 * out = Q(m0) in (as qs_apply_Q) and norm2[r] = ||out_r||^2 for r < nrhs.
 * in, out: DEVICE buffers as for qs_apply_Q; norm2: DEVICE array of nrhs doubles.
 * nrhs must be <= 64: the norm reduction keeps its partial sums in one static
 * device array of 608 x 64 doubles (311 KB, held by every device that loads the
 * library until the process exits); larger nrhs returns QS_EINVAL.  The call
 * allocates nothing (no cudaMalloc, no events; the operator uses the variant the
 * handle's autotuner chose earlier, else a fixed one).  Its first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current: make that first call before any stream capture.  Every call shares the
 * array, so calls whose work overlaps on the GPU (other streams, other handles of
 * the same device) race; calls on one stream are ordered and safe.  Asynchronous
 * on the handle's stream. */
QS_API int qs_apply_Q_norm2_noalloc(qs_lattice *lat, double m0, const void *in, void *out, int nrhs,
                                    int prec, double *norm2);

/* Static description of a status code. */
QS_API const char *qs_strerror(int status);

/* Text of the last CUDA error the library saw in the calling thread ("" if none). */
QS_API const char *qs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QSTAR_H */
