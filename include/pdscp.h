/*
 * pdscp.h — C ABI of the GB300 library for the primal-dual symmetric-cone MWU
 * framework (Zheng, Varvitsiotis, Tan, Lin, arXiv 2405.09157), specialised to
 * its two applications: the Smallest Enclosing Sphere (SES, Sec. 4.1) and the
 * hard-margin SVM / polytope distance (Sec. 4.2).
 *
 * Conventions for every entry point
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or framework
 *     tensors on the current device); *_host are host pointers. The caller
 *     owns every buffer. The library allocates no device memory and keeps no
 *     state between calls other than the thread-local error message.
 *   - Points are row-major n x d, element type selected by `dtype`
 *     (PDSCP_F32 = float32, PDSCP_BF16 = bfloat16), rows contiguous (pitch d).
 *     Vectorised 16-byte loads are used when the base address is 16-byte
 *     aligned and d * sizeof(element) is a multiple of 16; other inputs take a
 *     scalar-load path with identical results.
 *   - All device work is enqueued on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) in call order. Entry points that return a host
 *     value synchronise the stream; the doc comment says so.
 *   - Errors are returned as pdscp_status and never thrown or aborted across
 *     the ABI; pdscp_last_error() gives a message for the calling thread.
 *     Numeric and device-side problems are reported in the status word of the
 *     step record / state header written on the device.
 */
#ifndef PDSCP_H
#define PDSCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pdscp_stream; /* == cudaStream_t */

typedef enum pdscp_status {
  PDSCP_OK = 0,
  PDSCP_ERR_INVALID_ARG = 1,     /* bad size, pointer, alignment or option */
  PDSCP_ERR_CUDA = 2,            /* a CUDA runtime call failed */
  PDSCP_ERR_TIMEOUT = 3,         /* a bounded device wait gave up */
  PDSCP_ERR_NOT_SEPARABLE = 4,   /* SVM: certificate shows margin 0 */
  PDSCP_ERR_NOT_CONVERGED = 5,   /* iteration budget spent before the target */
  PDSCP_ERR_NUMERIC = 6,         /* NaN/Inf or an underflowed normaliser */
  PDSCP_ERR_NOT_IMPLEMENTED = 7, /* unsupported d / dtype combination */
  PDSCP_ERR_WORKSPACE = 8        /* workspace too small */
} pdscp_status;

/* problem kinds */
#define PDSCP_SES 0 /* Smallest Enclosing Sphere, K = prod_{i>=2} Q^{d+1} */
#define PDSCP_SVM 1 /* hard-margin SVM (min variant), K = R^n_+ */

/* point storage */
#define PDSCP_F32 0
#define PDSCP_BF16 1

/* alpha-FTP stopping rules (Sec. 3 Theorems 2/3, Sec. 5) */
#define PDSCP_RULES_NONE 0      /* stop only when the ORACLE separates */
#define PDSCP_RULES_PRACTICAL 1 /* also: f beats alpha; |df|/f < delta `patience` times */

/* solve modes */
#define PDSCP_MODE_PRACTICAL 0  /* Sec. 5 rules inside each alpha-FTP */
#define PDSCP_MODE_THEORY 1     /* T_i iterations of Theorem 2/3 per FTP */
#define PDSCP_MODE_CERTIFIED 2  /* proven conclusions only; ends on the certificates (see ses_solve) */
#define PDSCP_MODE_CORESET 3    /* CERTIFIED plus core-set certificates (see ses_solve, svm_solve) */

/* Largest supported dimension d. */
#define PDSCP_MAX_D 1024

/*
 * Per-step record written on the device by mwu_step (Sec. 3 alpha-FTP
 * iteration t -> t+1; Sec. 5 objective). 72 bytes.
 *   oracle_value  value of the ORACLE program at p^{t+1}: Eq. (ses_oracle) /
 *                 Eq. (svm_oracle). Negative = separated.
 *   objective     f at the mean read by this step (ubar^t or wbar^t), Sec. 5:
 *                 SES radius max_i ||ubar - v_i|| + gamma_i; SVM margin.
 *   lower_bound   SES: value of the primal solution of Eq. (primal_construction)
 *                 built from p^{t+1} (<= OPT). SVM: the margin f (<= OPT).
 *   upper_bound   SES: f (>= OPT). SVM: Claim 8 PD value (>= OPT).
 *   t             completed ORACLE calls after the step.
 *   failed        1 if the ORACLE separated (alpha < OPT for SES; OPT < alpha
 *                 for SVM).
 *   stopped       1 if the alpha-FTP has ended (separation or a rule).
 *   status        pdscp_status of the device computation.
 *   outcome       PDSCP_OUT_* of the alpha-FTP after the step.
 *   k             eta t / rho used by the step.
 *   dual_bound    certificate from the dual weights averaged over the
 *                 alpha-FTP so far (iterate t weighted by t^2, t >= 1). SES
 *                 (points; 0 for spheres or before the first update): lower
 *                 bound sqrt(Abar - |Bbar|^2) from the QP of Sec. 5 (Eq.
 *                 ses_qp), where mu_i = c_i / sum_j c_j are the weights of the
 *                 points in the ORACLE's g (w_i = c_i (v_i - ubar) / (sqrt2 S)),
 *                 A = sum mu_i |v_i - v_1|^2 and B = sum mu_i (v_i - v_1): any
 *                 simplex weights give OPT^2 >= A - |B|^2. SVM: upper bound
 *                 |zbar|, zbar the average of the Claim 8 vectors
 *                 P mu/Tr mu - Q gamma/Tr gamma (inf before the first update).
 *                 Both enter the state's best bounds (lower_bound /
 *                 upper_bound of the solves).
 */
typedef struct pdscp_step_out {
  double oracle_value;
  double objective;
  double lower_bound;
  double upper_bound;
  int64_t t;
  int32_t failed;
  int32_t stopped;
  int32_t status;
  int32_t outcome;
  double k;
  double dual_bound;
} pdscp_step_out;

/* Outcome codes in pdscp_step_out.outcome / pdscp_state header. */
#define PDSCP_OUT_RUNNING 0
#define PDSCP_OUT_SEPARATED 1  /* ORACLE value < 0 */
#define PDSCP_OUT_BEAT_ALPHA 2 /* SES f < alpha / SVM f > alpha (Sec. 5) */
#define PDSCP_OUT_STALLED 3    /* Sec. 5 delta/patience rule */

typedef struct pdscp_options {
  double eps;         /* target (1+eps) accuracy of the search, > 0 */
  double delta;       /* Sec. 5 stability threshold (paper: 1e-4) */
  int32_t patience;   /* Sec. 5 consecutive iterations (paper: 10) */
  int32_t mode;       /* PDSCP_MODE_* */
  int64_t max_iters;  /* MWU iterations over the whole search */
  int32_t poll_every; /* host polls the device state every k iterations */
  int32_t max_steps;  /* search steps (alpha values) at most */
  double eta;         /* 0: eta_i = sqrt(ln r / T_i) (Theorems 2/3); else fixed */
} pdscp_options;

typedef struct pdscp_report {
  double value;       /* SES: radius of the returned ball; SVM: its margin */
  double lower_bound; /* certificate: OPT >= lower_bound */
  double upper_bound; /* certificate: OPT <= upper_bound */
  double D;           /* bound of Sec. 4.1 (SES) / Lemma 6 (SVM) */
  double search_L;    /* final search range [L, U] of Sec. 3 */
  double search_U;
  int64_t iters;      /* MWU iterations run */
  int32_t search_steps;
  int32_t status;
} pdscp_report;

/* Library version (major*10000 + minor*100 + patch). */
int32_t pdscp_version(void);

/* Message describing the last failing call on this thread ("" if none). */
const char* pdscp_last_error(void);

/*
 * Exact polytope distance (Eq. PD, Sec. 4.2) of two small point sets on the
 * host: min ||P^T mu - Q^T gamma|| over mu, gamma in the simplices, P_host
 * nP x d and Q_host nQ x d row-major doubles (caller-owned). The solver of the
 * core-set certificates of svm_solve (PDSCP_MODE_CORESET): a primal
 * active-set method (the affine least-distance problem on the support solved
 * exactly, the most violating point added, points whose weight reaches zero
 * dropped) until z.z - (min_i p_i.z - max_j q_j.z) <= tol z.z or max_iter
 * additions. Writes the weights (mu_host: nP, gamma_host: nQ, in the
 * simplices) and *dist_host = ||P^T mu - Q^T gamma||, an upper bound on the
 * distance whatever the convergence. Synchronous, host only, no device work.
 * PDSCP_ERR_INVALID_ARG for null pointers, empty sets, d < 1, tol < 0 or
 * max_iter < 1.
 */
pdscp_status pdscp_polytope_distance(const double* P_host, int32_t nP, const double* Q_host, int32_t nQ,
                                     int32_t d, double tol, int32_t max_iter, double* mu_host,
                                     double* gamma_host, double* dist_host);

/*
 * Dual bound of the minimum enclosing ball of a small point set on the host
 * (the solver of the SES core-set certificates, ses_solve's
 * PDSCP_MODE_CORESET): weights mu on the simplex over the m rows of P_host
 * (m x d row-major doubles, caller-owned) maximising phi(mu) =
 * sum_i mu_i |p_i|^2 - |sum_i mu_i p_i|^2 (Sec. 4.1's dual pair for points:
 * phi(mu) <= OPT^2 for any such mu) by Frank-Wolfe steps toward the farthest
 * row and away steps from the nearest row of the support, each with its exact
 * line search, until the farthest row lies within (1 + tol) sqrt(phi) of the
 * barycentre c = sum_i mu_i p_i, or max_iter steps. Writes mu_host (m),
 * center_host (d) = c, *lb_host = sqrt(phi(mu)) (a lower bound on the ball's
 * radius whatever the convergence) and *far_host = max_i |p_i - c| (the
 * radius of an enclosing ball, an upper bound). Best conditioned with the
 * rows near the origin (the ball is translation invariant). Synchronous,
 * host only. PDSCP_ERR_INVALID_ARG for null pointers, m < 1, d < 1, tol < 0
 * or max_iter < 1.
 */
pdscp_status pdscp_meb_dual(const double* P_host, int32_t m, int32_t d, double tol, int32_t max_iter,
                            double* mu_host, double* center_host, double* lb_host, double* far_host);

/*
 * Bytes of device workspace needed by pdscp_bounds / mwu_step / the solves for
 * a problem of this kind and size on the current device. The workspace holds
 * per-CTA partial sums and a completion counter; it must be zeroed once before
 * first use (mwu_state_init and the solves do this) and may be reused by
 * consecutive calls on one stream. Calls that share a workspace must not
 * overlap on the GPU. The size includes the region of the core-set
 * certificates (PDSCP_MODE_CORESET of ses_solve / svm_solve); the other
 * calls need only its first part and accept the larger size.
 */
pdscp_status pdscp_workspace_size(int32_t problem, int64_t n, int32_t d, size_t* bytes_host);

/* Bytes of device state for mwu_step (a header plus O(d) doubles/floats). */
pdscp_status pdscp_state_size(int32_t problem, int32_t d, size_t* bytes_host);

/*
 * Bounds pre-pass (Sec. 4.1 / Lemma 6). Writes D to *D_dev (one double):
 *   SES: D = max_{i>=2} ||v_1 - v_i|| + gamma_1 + gamma_i  (OPT in [D/2, D])
 *   SVM: D = max_i ||x_i||                                  (s_1, s_2 <= D)
 * radii_dev (SES, may be NULL = all zero) holds n float radii.
 * Asynchronous. Requires n >= 2, 1 <= d <= PDSCP_MAX_D.
 */
pdscp_status pdscp_bounds(int32_t problem, const void* pts_dev, int32_t dtype,
                          const float* radii_dev, int64_t n, int32_t d,
                          void* ws_dev, size_t ws_bytes, pdscp_stream stream,
                          double* D_dev);

/*
 * Start an alpha-FTP (Sec. 3): t = 0, the running mean set to v_1 (SES; any
 * value works because the exponent is 0 at t = 0) or to (w, s1, s2) = 0
 * (SVM), no best point yet, stop rules `rules` (PDSCP_RULES_*) with the Sec. 5
 * parameters delta and patience. Also zeroes the workspace's counter.
 * Asynchronous.
 */
pdscp_status mwu_state_init(int32_t problem, const void* pts_dev, int32_t dtype,
                            int64_t n, int32_t d, int32_t rules, double delta,
                            int32_t patience, void* state_dev, void* ws_dev,
                            size_t ws_bytes, pdscp_stream stream);

/*
 * One iteration t -> t+1 of the alpha-FTP (Sec. 3; Eq. implement for SES,
 * Eq. min_implement for SVM), as one kernel launch over the n points:
 *   SES (Sec. 4.1): per cone i >= 2 the exponent -(eta t/rho)(ubar - v_i;
 *     alpha - gamma_i), its closed-form SOC exponential (Sec. 2.1), the trace
 *     normaliser, g = sum w_i, the ORACLE u = v_1 + (alpha - gamma_1) g/||g||,
 *     its value, the primal bound of Eq. (primal_construction), f^t, and the
 *     running-mean update ubar^{t+1}.
 *   SVM (Sec. 4.2): per point the exponent -(eta t/rho)(y_i x_i^T wbar -
 *     sbar_{class i}), the normaliser, z = P mu - Q gamma, the ORACLE
 *     (w, s1, s2) of Eq. (svm_oracle), its value, the Claim 8 bound, f^t,
 *     and the running means.
 * eta_over_rho = eta/rho (> 0); k = eta_over_rho * t is formed on the device.
 * alpha > 0. D (SVM) must be >= the largest point norm (pdscp_bounds); it is
 * ignored for SES. labels_dev (SVM): n int8 in {+1,-1}. radii_dev (SES) may be
 * NULL. out_dev (may be NULL) receives one pdscp_step_out. If the state's
 * alpha-FTP has stopped, the launch returns at once and writes nothing.
 * eval_only != 0 evaluates f at the current mean (and the best-point
 * bookkeeping) without an ORACLE step. Asynchronous; no host sync.
 */
pdscp_status mwu_step(int32_t problem, const void* pts_dev, int32_t dtype,
                      const float* radii_dev, const int8_t* labels_dev,
                      int64_t n, int32_t d, double alpha, double eta_over_rho,
                      double D, int32_t eval_only, void* state_dev,
                      void* ws_dev, size_t ws_bytes, pdscp_stream stream,
                      pdscp_step_out* out_dev);

/*
 * Resume an alpha-FTP from a checkpoint (t, running mean): sets t and the
 * mean from mean_dev (device doubles; SES: ubar, d values; SVM: wbar, then
 * s1bar and s2bar, d+2 values), clears the stop flags and best-point records
 * (rules PDSCP_RULES_NONE), then runs one evaluation pass over the points at
 * that mean to recompute the exponent-shift bound. D as for mwu_step (SVM
 * only). Asynchronous.
 */
pdscp_status mwu_state_set(int32_t problem, const void* pts_dev, int32_t dtype,
                           const float* radii_dev, const int8_t* labels_dev,
                           int64_t n, int32_t d, int64_t t, const double* mean_dev,
                           double D, void* state_dev, void* ws_dev, size_t ws_bytes,
                           pdscp_stream stream);

/*
 * mwu_step without a workspace argument, for callers that cannot allocate
 * device memory: code running inside a host program that owns all GPU memory
 * through its own pool, or that must not risk the implicit device
 * synchronisation an allocation can bring. The paper has no counterpart; it
 * is a deployment convenience. Same arguments and results as mwu_step minus
 * ws_dev/ws_bytes: the per-CTA partial sums and completion counters live in a
 * 2 MiB array built into the library, which every GPU that loads the library
 * reserves until the process exits. Problems whose scratch does not fit
 * (d > 380 for SES and d > 188 for SVM on a 152-SM GPU) are rejected with
 * PDSCP_ERR_WORKSPACE and a message; use mwu_step for them.
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, host-side; nothing is cached, so a device reset
 * leaves no stale address); the first call on a device may load the
 * library's device code there, so make that first call before any stream
 * capture.
 * Each call clears the counters on `stream` (cudaMemsetAsync) and allocates
 * nothing. All calls on a device share the one array: calls that overlap on
 * the GPU (different streams, or several threads) race and give wrong
 * results; serialise them on one stream.
 */
pdscp_status mwu_step_noalloc(int32_t problem, const void* pts_dev, int32_t dtype,
                              const float* radii_dev, const int8_t* labels_dev,
                              int64_t n, int32_t d, double alpha, double eta_over_rho,
                              double D, int32_t eval_only, void* state_dev,
                              pdscp_stream stream, pdscp_step_out* out_dev);

/*
 * k iterations of mwu_step (same arguments and meaning, eval_only = 0) enqueued
 * back to back on `stream`, consecutive launches overlapping by programmatic
 * dependent launch: each launch's CTAs issue their first point loads while
 * the previous launch finishes and wait for it (a hardware dependency)
 * before reading the state. The results are those of k mwu_step calls, bit
 * for bit. out_dev (may be NULL) receives k pdscp_step_out, one per
 * iteration (an iteration after the alpha-FTP stopped writes nothing). k = 0
 * does nothing. Asynchronous; no host sync.
 */
pdscp_status mwu_run(int32_t problem, const void* pts_dev, int32_t dtype,
                     const float* radii_dev, const int8_t* labels_dev,
                     int64_t n, int32_t d, double alpha, double eta_over_rho,
                     double D, int64_t k, void* state_dev, void* ws_dev,
                     size_t ws_bytes, pdscp_stream stream, pdscp_step_out* out_dev);

/*
 * Read the running mean (SES: ubar, d floats; SVM: wbar then s1bar, s2bar:
 * d+2 floats) and the best point seen (SES: centre with the smallest f; SVM:
 * direction with the largest margin; d floats) of a state into device
 * buffers (either may be NULL). Asynchronous.
 */
pdscp_status mwu_state_read(int32_t problem, int32_t d, const void* state_dev,
                            float* mean_dev, float* best_dev, pdscp_stream stream);

/*
 * (1+eps)-approximate Smallest Enclosing Sphere (Sec. 4.1) by the search of
 * Sec. 3 over alpha in [D/2, D], each alpha-FTP run on the device with the
 * host polling every opts->poll_every iterations (this synchronises the
 * stream). Writes the best centre (d floats) to center_dev and fills
 * *report_host: radius of an actual enclosing ball (upper bound), the best
 * lower bound (Eq. (primal_construction) or, for points, the averaged QP
 * bound of pdscp_step_out.dual_bound), the search range.
 * Returns PDSCP_ERR_NOT_CONVERGED (with a valid report) when opts->max_iters
 * ran out before the range or the certificate gap closed.
 * Modes: PRACTICAL runs the Sec. 5 rules in each alpha-FTP and reads a stall
 * as the affirmative answer (U moves), so the range may close below OPT while
 * the certificates stay wide; THEORY runs T_i iterations of Theorem 2.
 * CERTIFIED draws only proven conclusions: separation gives L = alpha_i,
 * f < alpha_i gives U = f; each FTP also ends at a poll where the
 * certificates close (ub <= (1+eps) max(lb, L)) or, as stuck, at the first
 * poll with t >= c, 2c, 4c, ... (c = 1024/eta) where the FTP's own gap (best
 * f over its lower bound, minus 1) has not shrunk by the factor 0.8 since the
 * previous such poll, after which eta is halved (not below 1/64, where the
 * test stops); the solve ends only on the certificates (or the budget) and
 * report.lower_bound is max(lb, L). eta 0 means 1 in this mode.
 * PDSCP_MODE_CORESET (points, radii_dev NULL; with radii it is CERTIFIED) is
 * CERTIFIED plus core-set certificates (not in the paper; built on the dual
 * pair of Sec. 4.1): at the polls where the search's iteration count first
 * reaches 256, 512, 1024, ..., the points farthest from the running mean
 * (between 512 and 1024, by a threshold found on the device) form a core set;
 * Frank-Wolfe steps with away steps on the host give weights mu on it whose
 * dual value sqrt(sum_i mu_i |v_i|^2 - |sum_i mu_i v_i|^2) is a lower bound on
 * OPT (weak duality), and the radius of the ball at sum_i mu_i v_i over every
 * point (one pass on the device) an upper bound; up to four rounds add the
 * points farthest from each new centre. The bounds join the FTP's own; the
 * returned centre is the one of the smallest ball found. The workspace then
 * also holds the n distances and the core set's rows (pdscp_workspace_size
 * counts them).
 */
pdscp_status ses_solve(const void* pts_dev, int32_t dtype, const float* radii_dev,
                       int64_t n, int32_t d, const pdscp_options* opts,
                       void* ws_dev, size_t ws_bytes, pdscp_stream stream,
                       float* center_dev, pdscp_report* report_host);

/*
 * (1-eps)-approximate hard-margin SVM / (1+eps) polytope distance (Sec. 4.2)
 * by the minimisation search over alpha in (0, 2D]. Writes the best
 * direction w (d floats, unit norm) to w_dev and its margin and Claim 8
 * upper bound (per iteration or averaged, pdscp_step_out.dual_bound) to
 * *report_host. Synchronises like ses_solve. Modes as in ses_solve, with the
 * roles mirrored: in CERTIFIED mode separation gives U = alpha_i, a margin
 * f > alpha_i gives L = f, the FTP's own gap is its Claim 8 bound over its
 * best margin, and report.upper_bound is min(ub, U).
 * PDSCP_MODE_CORESET is CERTIFIED plus core-set certificates (not in the
 * paper; built on Eq. PD): at the polls where the search's iteration count
 * first reaches 256, 512, 1024, ..., the 512 points of each class nearest
 * the hyperplane of the running FTP's best direction form a core set whose
 * exact polytope distance (solved on the host, pdscp_polytope_distance) is
 * an upper bound on OPT, and whose solution direction, projected on every
 * point on the device, gives a margin, a lower bound; up to four rounds add
 * the core set of each new direction. The bounds join the FTP's own; the
 * returned direction is the one of the best margin. The workspace then also
 * holds the projections of the n points and the core set's rows (see
 * pdscp_workspace_size, which counts them).
 */
pdscp_status svm_solve(const void* X_dev, int32_t dtype, const int8_t* labels_dev,
                       int64_t n, int32_t d, const pdscp_options* opts,
                       void* ws_dev, size_t ws_bytes, pdscp_stream stream,
                       float* w_dev, pdscp_report* report_host);

/*
 * Batched SES (many independent instances, one launch per iteration for all).
 * Instance i has n_i >= 2 points of dimension 1 <= d_i <= 64, stored row-major
 * in one buffer of pts_len elements of type dtype (PDSCP_F32 or PDSCP_BF16;
 * bfloat16 rows are widened to float32 on load, the arithmetic is that of
 * float32 rows), starting at element offset_i (a start aligned to 4 elements
 * enables 16-byte (float32) or 8-byte (bfloat16) loads when d_i % 4 == 0;
 * pts_dev must be aligned to its element). Each
 * instance runs its own alpha-FTP (Sec. 3 with the SES data of Sec. 4.1)
 * with its own state, kept in the workspace. Rows are cut into tiles of
 * tile_rows (>= 32); a persistent grid takes tiles from a counter and the
 * CTA that completes an instance's last tile finishes that instance.
 *   ses_batch_workspace_size: bytes of the workspace (host sizes).
 *   ses_batch_init: builds the tile tables (host -> workspace, synchronises
 *     the stream), records dtype and starts every instance's alpha-FTP (t = 0,
 *     mean = v_1). An unknown dtype, an instance past pts_len or a misaligned
 *     pointer returns PDSCP_ERR_INVALID_ARG before any device work.
 *   ses_batch_step: one MWU iteration of every instance (asynchronous);
 *     pts_dev and dtype must be those given to ses_batch_init (not checked
 *     against the workspace: the call does not synchronise); alpha_dev and
 *     eta_over_rho_dev hold one double per instance; out_dev (may be NULL)
 *     receives one pdscp_step_out per instance.
 *   ses_batch_read: each instance's running mean and best centre, packed one
 *     after another (instance i's d_i values after those of instances < i).
 */
pdscp_status ses_batch_workspace_size(int32_t num, const int64_t* n_host, const int32_t* d_host,
                                      int32_t tile_rows, size_t* bytes_host);
pdscp_status ses_batch_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                            const int64_t* offset_host, const int64_t* n_host,
                            const int32_t* d_host, int32_t tile_rows, void* ws_dev,
                            size_t ws_bytes, pdscp_stream stream);
pdscp_status ses_batch_step(int32_t num, const void* pts_dev, int32_t dtype, const double* alpha_dev,
                            const double* eta_over_rho_dev, void* ws_dev, size_t ws_bytes,
                            pdscp_stream stream, pdscp_step_out* out_dev);
pdscp_status ses_batch_read(int32_t num, const void* ws_dev, float* mean_dev, float* best_dev,
                            pdscp_stream stream);

/*
 * Batched search: every instance runs the whole search of Sec. 3 (alpha in
 * [D/2, D], alpha_i = L + (U-L)/3, eps_i and T_i of Theorem 2 with the Sec.
 * 4.1 constants, the Sec. 5 rules when opts->mode is PDSCP_MODE_PRACTICAL;
 * PDSCP_MODE_CERTIFIED as in ses_solve, its certificate and progress tests
 * made every opts->poll_every iterations of an instance's FTP),
 * with the decisions of ses_solve, on the device: the CTA that finishes an
 * instance's iteration also updates its search and starts its next
 * alpha-FTP. An instance's first launch is an evaluation pass at v_1 (which
 * gives D); a finished instance's tiles are skipped.
 *   ses_batch_solve_init: as ses_batch_init, plus the search records and
 *     options (opts->poll_every is used by the CERTIFIED mode only;
 *     opts->max_iters counts MWU iterations per instance). Synchronises the
 *     stream.
 *   ses_batch_solve_run: (pts_dev as given to ses_batch_solve_init, whose
 *     dtype the workspace records) replays a CUDA graph of launches_per_poll launches
 *     on `stream` until every instance is done or max_launches launches ran
 *     (host polls a device counter after each replay); reports the launches
 *     run and the instances done (host pointers, may be NULL).
 *   ses_batch_solve_read: one pdscp_report per instance (value = upper_bound
 *     = radius of the returned centre, lower_bound = best lower bound (Eq.
 *     primal_construction, the averaged QP bound; CERTIFIED: also the search's
 *     L), search_L/U, iters, search_steps, status: OK when
 *     U <= (1+eps) L or ub <= (1+eps) lb, PDSCP_ERR_NOT_CONVERGED otherwise)
 *     to reports_dev and the centres, packed as in ses_batch_read, to
 *     centers_dev (either may be NULL).
 *   ses_batch_autotune: times the search launch on this batch for every
 *     tile_rows in {512, ..., 32768} whose workspace fits ws_bytes, with 1, 2
 *     and 3 CTAs per SM in the persistent grid and both lane-layout policies
 *     (0: 4-element chunk loads for instances with d % 4 == 0 whose rows
 *     start on a 4-element boundary, scalar layouts otherwise; 1: scalar
 *     layouts only), and returns the fastest (tile_rows_host, and, where not
 *     NULL, its time, CTAs per SM and layout); leaves the workspace set up
 *     for the last candidate tried, so ses_batch_solve_init must follow.
 *   ses_batch_set_launch: after ses_batch_init or ses_batch_solve_init,
 *     records the CTAs per SM of ses_batch_solve_run's persistent grid
 *     (0: as many as fit, else 1..3) and applies a layout policy (0 or 1)
 *     to every instance (pts_dev as given to the init); ses_batch_step keeps
 *     the grid of as many CTAs as fit. Synchronises the stream.
 *     PDSCP_ERR_INVALID_ARG for values out of range or another batch's
 *     instance count.
 */
pdscp_status ses_batch_solve_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                                  const int64_t* offset_host, const int64_t* n_host,
                                  const int32_t* d_host, int32_t tile_rows,
                                  const pdscp_options* opts, void* ws_dev, size_t ws_bytes,
                                  pdscp_stream stream);
pdscp_status ses_batch_solve_run(int32_t num, const void* pts_dev, void* ws_dev, size_t ws_bytes,
                                 int32_t launches_per_poll, int64_t max_launches,
                                 pdscp_stream stream, int64_t* launches_host, int32_t* done_host);
pdscp_status ses_batch_solve_read(int32_t num, const void* ws_dev, double eps,
                                  pdscp_report* reports_dev, float* centers_dev,
                                  pdscp_stream stream);
pdscp_status ses_batch_autotune(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                                const int64_t* offset_host, const int64_t* n_host,
                                const int32_t* d_host, const pdscp_options* opts, void* ws_dev,
                                size_t ws_bytes, pdscp_stream stream, int32_t* tile_rows_host,
                                float* ms_per_launch_host, int32_t* ctas_per_sm_host,
                                int32_t* layout_host);
pdscp_status ses_batch_set_launch(int32_t num, const void* pts_dev, void* ws_dev, int32_t ctas_per_sm,
                                  int32_t layout, pdscp_stream stream);

/*
 * Batched SVM (many independent hard-margin SVM instances, one launch per
 * iteration for all): instance i has n_i >= 2 points of dimension
 * 1 <= d_i <= 64, stored as for the batched SES (offset_i, dtype, pts_len),
 * and n_i int8 labels (+1: class P, -1: class Q, Sec. 4.2) starting at
 * element label_offset_i of labels_dev (labels_len elements). Each instance
 * runs its own minimisation alpha-FTP (Sec. 3, Eq. min_implement, the SVM
 * data of Sec. 4.2) with its own state; the tiles, the persistent grid and
 * the completion are those of the batched SES.
 *   svm_batch_workspace_size: bytes of the workspace (host sizes).
 *   svm_batch_init: builds the tables (host -> workspace), computes each
 *     instance's D = max_i ||x_i|| on the device (FP64 norms of the stored
 *     values) and starts every alpha-FTP (t = 0, means 0); synchronises the
 *     stream. Bad pointers, an unknown dtype, or an instance past pts_len or
 *     labels_len return PDSCP_ERR_INVALID_ARG before any device work.
 *   svm_batch_step: one MWU iteration of every instance (asynchronous);
 *     pts_dev, dtype and labels_dev must be those given to svm_batch_init;
 *     alpha_dev and eta_over_rho_dev hold one double per instance; out_dev
 *     (may be NULL) receives one pdscp_step_out per instance.
 *   svm_batch_read: each instance's running mean wbar and best-margin
 *     direction (packed as in ses_batch_read) and its D (one double each);
 *     any output may be NULL.
 *   svm_batch_solve_init / _run / _read: the search of svm_solve for every
 *     instance on the device (alpha in (0, 2D], alpha_i = U - (U-L)/3; the
 *     PRACTICAL and THEORY modes with T_i of Theorem 3 and the Sec. 5 rules,
 *     CERTIFIED with the certificate and progress tests of svm_solve every
 *     opts->poll_every iterations); the CUDA-graph replay and polling of
 *     ses_batch_solve_run. The reports carry value = lower_bound = the margin
 *     of the returned direction, upper_bound = the best Claim 8 value (with
 *     CERTIFIED: min(ub, U)); the directions are packed as in ses_batch_read.
 */
pdscp_status svm_batch_workspace_size(int32_t num, const int64_t* n_host, const int32_t* d_host,
                                      int32_t tile_rows, size_t* bytes_host);
pdscp_status svm_batch_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                            const int64_t* offset_host, const int64_t* n_host,
                            const int32_t* d_host, const int8_t* labels_dev, int64_t labels_len,
                            const int64_t* label_offset_host, int32_t tile_rows, void* ws_dev,
                            size_t ws_bytes, pdscp_stream stream);
pdscp_status svm_batch_step(int32_t num, const void* pts_dev, int32_t dtype, const int8_t* labels_dev,
                            const double* alpha_dev, const double* eta_over_rho_dev, void* ws_dev,
                            size_t ws_bytes, pdscp_stream stream, pdscp_step_out* out_dev);
pdscp_status svm_batch_read(int32_t num, const void* ws_dev, float* mean_dev, float* best_dev,
                            double* D_dev, pdscp_stream stream);
pdscp_status svm_batch_solve_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                                  const int64_t* offset_host, const int64_t* n_host,
                                  const int32_t* d_host, const int8_t* labels_dev, int64_t labels_len,
                                  const int64_t* label_offset_host, int32_t tile_rows,
                                  const pdscp_options* opts, void* ws_dev, size_t ws_bytes,
                                  pdscp_stream stream);
pdscp_status svm_batch_solve_run(int32_t num, const void* pts_dev, const int8_t* labels_dev, void* ws_dev,
                                 size_t ws_bytes, int32_t launches_per_poll, int64_t max_launches,
                                 pdscp_stream stream, int64_t* launches_host, int32_t* done_host);
pdscp_status svm_batch_solve_read(int32_t num, const void* ws_dev, double eps,
                                  pdscp_report* reports_dev, float* w_dev, pdscp_stream stream);

/*
 * Row-sharded iteration: the rows (cones) split across G GPUs, one shard per
 * GPU. An MWU iteration over a product of cones (Sec. 3, Eq. implement /
 * min_implement) needs, besides the replicated O(d) state, only column sums
 * and extrema over the points (Sec. 4.1: S, G', Wt, max dist; Sec. 4.2: S_P,
 * S_Q, Z_P, Z_Q, min/max margins), so each GPU streams its shard into one
 * row of column totals, the caller exchanges the G rows (an all-gather of
 * width x 8 bytes per GPU, e.g. NCCL), and every GPU runs the same O(d)
 * finish on the rows in rank order, which keeps the replicated states
 * identical. Sums are compensated FP32 pairs; the rank order fixes the result.
 *   mwu_shard_row_width: the row width in (float, float) pairs (host int).
 *   mwu_shard_init: starts the alpha-FTP on this GPU's replica of the state;
 *     first_dev = v_1 (SES: the easy cone's centre, d elements of dtype,
 *     replicated on every GPU; SVM: unused, may be NULL); clears the
 *     workspace counters. ws as for mwu_step with this shard's n.
 *   mwu_shard_partial: one pass over this GPU's shard (n >= 1 rows, layout as
 *     mwu_step); holds_first = 1 on the GPU whose shard starts with v_1 (that
 *     row is the easy cone and is skipped), else 0; state_dev is read only;
 *     writes 2 * width floats to row_dev (8-byte aligned, caller-owned).
 *     Writes nothing when the FTP has stopped (as mwu_step).
 *   mwu_shard_finish: reduces rows_dev (ranks rows of 2 * width floats, rank
 *     order) and finishes the iteration exactly as mwu_step does: state
 *     update, step record to out_dev (may be NULL). first_dev / dtype /
 *     first_radius_dev (may be NULL: 0) give v_1 and gamma_1 for SES.
 * alpha, eta_over_rho, D and eval_only have mwu_step's meaning and must be the
 * same in the partial calls and the finish. Asynchronous on `stream`; errors
 * as mwu_step.
 */
pdscp_status mwu_shard_row_width(int32_t problem, int32_t d, int32_t* width_host);
pdscp_status mwu_shard_init(int32_t problem, const void* first_dev, int32_t dtype, int32_t d,
                            int32_t rules, double delta, int32_t patience, void* state_dev,
                            void* ws_dev, size_t ws_bytes, pdscp_stream stream);
pdscp_status mwu_shard_partial(int32_t problem, const void* pts_dev, int32_t dtype,
                               const float* radii_dev, const int8_t* labels_dev, int64_t n,
                               int32_t d, int32_t holds_first, double alpha, double eta_over_rho,
                               double D, int32_t eval_only, const void* state_dev, void* ws_dev,
                               size_t ws_bytes, pdscp_stream stream, float* row_dev);
pdscp_status mwu_shard_finish(int32_t problem, const float* rows_dev, int32_t ranks,
                              const void* first_dev, int32_t dtype, const float* first_radius_dev,
                              int32_t d, double alpha, double eta_over_rho, double D,
                              int32_t eval_only, void* state_dev, pdscp_stream stream,
                              pdscp_step_out* out_dev);

/*
 * Multi-candidate SES iteration: one streaming pass over the points advances
 * k in {1, 2, 4, 8, 16} independent alpha-FTPs of the same instance (Sec. 3
 * with the SES data of Sec. 4.1), each with its own alpha_j, eta_j/rho and
 * state: the candidates of a k-ary search over alpha share every byte read.
 * Float32 points, d <= 64; k = 16 needs d = 32 and a 16-byte aligned pts_dev
 * and runs on the tensor cores (the squared distances' cross terms and the
 * weighted sums as tf32 MMAs on three-part operand splits, accumulators in
 * tensor memory, point tiles loaded by TMA).
 * Per candidate the result is that of mwu_step with the same alpha_j,
 * eta_j/rho and state (up to the order and splitting of the FP32 sums).
 *   ses_multi_state_stride: bytes between consecutive candidate states in
 *     states_dev (a multiple of 256); each state is started with
 *     mwu_state_init (PDSCP_SES, the same points) at states_dev + j * stride.
 *   ses_multi_workspace_size: bytes of ws_dev for (d, k); ws_dev must be
 *     zero-filled before its first use (the kernels leave their counters at 0).
 *   ses_multi_step: alpha_dev, eta_over_rho_dev: k doubles (device); out_dev:
 *     k records or NULL. A stopped candidate keeps its state. Asynchronous.
 */
pdscp_status ses_multi_state_stride(int32_t d, size_t* bytes_host);
pdscp_status ses_multi_workspace_size(int32_t d, int32_t k, size_t* bytes_host);
pdscp_status ses_multi_step(const float* pts_dev, const float* radii_dev, int64_t n, int32_t d,
                            int32_t k, const double* alpha_dev, const double* eta_over_rho_dev,
                            void* states_dev, void* ws_dev, size_t ws_bytes, pdscp_stream stream,
                            pdscp_step_out* out_dev);

/*
 * Reverse-mode sweep through T unrolled iterations of the alpha-FTP at fixed
 * alpha and eta/rho (Sec. 3, Eq. implement / min_implement, ORACLE Eq.
 * ses_oracle / svm_oracle): the gradient, with respect to the points, of
 *   SES: L = seed * f(ubar^T), f(c) = max_i ||c - v_i|| + gamma_i (the radius of Sec. 5);
 *   SVM: L = seed * f(wbar^T), f(w) = max{(min_P x^T w - max_Q x^T w)/||w||, 0} (the margin of Sec. 5).
 * The sweep first runs the T forward iterations from t = 0 (as mwu_state_init
 * + T mwu_step calls with rules PDSCP_RULES_NONE), recording O(d) values per
 * iteration in the workspace (SES: the mean, g, the normaliser, |g|, the
 * exponent scale and shift; SVM: the mean, z, the normaliser, |z|, k, the
 * shift, s1bar, s2bar), then one streaming pass per iteration in reverse
 * order, each adding that iteration's dL/dx_i to grad_dev and summing the
 * adjoint of the mean. If the ORACLE separates at step t_f < T, the sweep
 * differentiates the t_f iterations taken. f is a maximum (SES) or a margin
 * between a minimum and a maximum (SVM): the rows attaining them (smallest
 * index on ties) receive the subgradient; a clipped SVM margin has gradient 0.
 * Radii, D and alpha are constants; for SVM, s_1 and s_2 are piecewise
 * constant in the points and pass no gradient.
 *   problem: PDSCP_SES or PDSCP_SVM; dtype: PDSCP_F32 or PDSCP_BF16 (bfloat16
 *     rows are widened to float32 on load: the result is the gradient at the
 *     bfloat16 values, in float32); radii_dev (SES, may be NULL), labels_dev
 *     and D (SVM) as for mwu_step.
 *   seed_dev: dL/df, one device double (NULL: 1).
 *   ws_dev: mwu_backward_workspace_size bytes (256-byte aligned); on return
 *     it holds the forward's final state and tape (caller-owned).
 *   grad_dev: n x d float32, row-major, overwritten (d % 4 == 0 with grad_dev
 *     16-byte aligned and pts_dev aligned to 4 elements takes the vector path).
 *   out_dev (may be NULL): one pdscp_step_out: objective = f at the final
 *     mean, t = iterations taken, oracle_value/outcome of the forward,
 *     k = the index of the row attaining f (SES) or the minimum over P (SVM;
 *     -1 when the margin is clipped).
 * Asynchronous on `stream` (2T + 3 launches); errors as mwu_step.
 */
pdscp_status mwu_backward_workspace_size(int32_t problem, int64_t n, int32_t d, int64_t T,
                                         size_t* bytes_host);
pdscp_status mwu_backward(int32_t problem, const void* pts_dev, int32_t dtype,
                          const float* radii_dev, const int8_t* labels_dev, int64_t n,
                          int32_t d, double alpha, double eta_over_rho, double D, int64_t T,
                          const double* seed_dev, void* ws_dev, size_t ws_bytes,
                          pdscp_stream stream, float* grad_dev, pdscp_step_out* out_dev);

#ifdef __cplusplus
}
#endif

#endif /* PDSCP_H */
