/*
 * qmc.h -- C ABI of the GB300 reduced QMC matrix-vector product library
 * (libqmc_gb300.so).
 *
 * The library evaluates QMC rules Q_N(f) = N^-1 sum_{k<N} f(x_k^T A)
 * (eq. (2) of Dick, Ebert, Herrmann, Kritzer, Longo, "The fast reduced QMC
 * matrix-vector product") over N = 2^m points of a reduced rank-1 lattice or a
 * reduced polynomial lattice (Sec. 1.3), of a reduced digital net (Sec. 4) or
 * of a reduced Monte Carlo point set (Sec. 5), exploiting that coordinate j of
 * x_k depends only on k mod 2^(m-w_j) (Sec. 3): every weight block of A's rows
 * is multiplied only against its distinct point rows (Algorithm 2) and the
 * partial products are summed back periodically over the N outputs.
 *
 * Conventions shared by every entry point
 *  - Columns are 0-based: j = 0..s-1 is the paper's j+1.
 *  - Points are held as 32-bit fixed point X32 = x * 2^32 (x in [0,1)).
 *    A random shift Delta_j is D_j * 2^-32 with D_j a uint32: lattices add it
 *    mod 2^32 ({x + Delta}, Sec. 2.3), nets and polynomial lattices XOR it
 *    (digital shift).  Reduced Monte Carlo takes no shift.
 *  - A is s x tau row-major (row j is a_j, Sec. 3.1).  Its element type is
 *    fixed by the precision: QMC_FP64 -> double; QMC_FP32, QMC_SPLIT and
 *    QMC_BF16 -> float.
 *  - "HOST" pointers are read during the call only; "DEVICE" pointers must be
 *    device memory of the current CUDA device, and are read or written by
 *    work enqueued on `stream` (the call returns before that work finishes).
 *    The caller owns all memory.  The library allocates no device memory: all
 *    scratch space comes from the caller's workspace (see qmc_workspace_size).
 *  - Every function returns a qmc_status and never aborts or throws.
 *    qmc_last_error() gives a message for the last failure on this thread.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 */
#ifndef QMC_GB300_H
#define QMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qmc_status;
#define QMC_OK                0
#define QMC_ERR_INVALID_ARG   1   /* argument violates the paper's definitions or the sizes */
#define QMC_ERR_UNSUPPORTED   2   /* valid in the paper, not built here (b != 2, ...) */
#define QMC_ERR_NO_MEMORY     3   /* workspace smaller than qmc_workspace_size() */
#define QMC_ERR_CUDA          4   /* a CUDA runtime call failed (message has the CUDA error string) */
#define QMC_ERR_DEVICE        5   /* a kernel reported an inconsistent state through its error word */
#define QMC_ERR_TIMEOUT       6   /* a bounded device-side wait ran out */

/* point-set kinds */
#define QMC_LATTICE      0        /* reduced rank-1 lattice, Sec. 1.3 */
#define QMC_DIGITAL_NET  1        /* reduced digital net, Sec. 4, eq. reduced_genmat_net2 */
#define QMC_REDUCED_MC   2        /* reduced Monte Carlo, Sec. 5, eq. randpts: coordinate j of point n is
                                     the i.i.d. sample y_{j, n mod N_j}, N_j = 2^(m-min(w_j,m)) */
#define QMC_POLY_LATTICE 3        /* reduced polynomial lattice, Sec. 1.3: x_{k,j} = nu(k(x) g_j(x) / x^m) with
                                     g_j = x^{w_j} gt_j over F_2 (a digital net; digital shifts) */

/* coordinate transforms phi_j applied to the (shifted) points, Sec. 2.3 */
#define QMC_T_IDENTITY   0        /* x */
#define QMC_T_CENTER     1        /* x - 1/2 */
#define QMC_T_INV_NORMAL 2        /* Phi^-1(x), standard normal quantile (Sec. 1, Gaussian change of variables) */
#define QMC_T_TENT       3        /* 1 - |1 - 2x|, Sec. 1.2 */

/* arithmetic precision of the product and of the integrand */
#define QMC_FP64  0               /* double A, double arithmetic */
#define QMC_FP32  1               /* float A, float arithmetic; estimates reduced in double */
#define QMC_SPLIT 2               /* float A and data; the coarse block products X_I A_I (Algorithm 2)
                                     and block gradients X_I^T F_I on tensor cores with three bf16
                                     pieces per operand and six piece products (bf16x6), FP32
                                     accumulation: FP32-level accuracy; the rest as QMC_FP32 */
#define QMC_BF16  3               /* as QMC_SPLIT with one bf16 piece per operand (one product):
                                     relative error ~2^-8 in the block products */

/* row-separable integrands f(y) = g(sum_t h(y_t)), y = x^T A in R^tau */
#define QMC_F_NONE          0     /* no integrand (qmc_reduced_matmul only) */
#define QMC_F_LINEAR_MEAN   1     /* f = tau^-1 sum_t y_t */
#define QMC_F_MEAN_COS      2     /* f = tau^-1 sum_t cos(y_t) */
#define QMC_F_CALL_MEAN_EXP 3     /* f = max(tau^-1 sum_t exp(c y_t) - K, 0); params = {c, K} */
#define QMC_F_GAUSS_NORM2   4     /* f = exp(-sum_t y_t^2 / (2 tau)) */
#define QMC_F_PDE_INV_SQ    5     /* f = tau^-1 sum_t (1 + c y_t)^-2; params = {c} */
#define QMC_F_LOGSUMEXP     6     /* f = log sum_t exp(y_t) */

/* gen_points layouts */
#define QMC_LAYOUT_FULL     0     /* N x s row-major uint32: X32 of x_{k,j} for every k */
#define QMC_LAYOUT_DISTINCT 1     /* column j's 2^(m-min(w_j,m)) distinct rows, columns concatenated in order */

/* operations for qmc_workspace_size */
#define QMC_OP_GEN_POINTS     0
#define QMC_OP_REDUCED_MATMUL 1
#define QMC_OP_INTEGRATE      2
#define QMC_OP_INTEGRATE_BWD  3

/* flags for qmc_integrate_backward */
#define QMC_BWD_REUSE_FORWARD 1u  /* d_ws still holds the state of a qmc_integrate call with the same
                                     rules, A, f and precision, enqueued earlier on the same stream with
                                     the same workspace: the forward pass is not recomputed */

/*
 * A reduced QMC rule (the point set).
 *  kind       QMC_LATTICE, QMC_DIGITAL_NET, QMC_REDUCED_MC or QMC_POLY_LATTICE.
 *  b          base, a prime.  b = 2: every kind (the tensor-core block products and the binary fine band
 *             of Sec. 3.2).  b > 2: QMC_LATTICE and QMC_REDUCED_MC (Sec. 1.3 lattices with N = b^m, and
 *             Sec. 5; the other kinds return QMC_ERR_UNSUPPORTED), computed by the generic top-down
 *             levels on the CUDA cores in every tier (FP32 in the tensor-core tiers).  A b > 2 lattice
 *             point is u / b^q_j in double (u = k z_j mod b^q_j), shifted as {x + D 2^-32}, then
 *             transformed; z_j must lie in U_{b^q_j} (not divisible by b, < b^q_j).
 *  m          N = b^m points, 1 <= m <= 30 (b = 2), b^m <= 2^31 (b > 2; larger: QMC_ERR_UNSUPPORTED).
 *  s          dimension (rows of A), 1 <= s <= 65536.
 *  w          HOST uint32[s]: reduction indices, nondecreasing (Sec. 1.3: 0 = w_1 <= w_2 <= ...;
 *             any nondecreasing sequence is accepted).  Values >= m make column j constant.
 *  z          HOST uint32[s] (lattice): reduced generating vector, z_j in U_{b^(m-w_j)}, i.e. odd and
 *             < 2^(m-w_j) if w_j < m, else exactly 1 (Sec. 1.3).  The lattice's generating vector is
 *             (2^{w_1} z_1, ..., 2^{w_s} z_s).
 *  z          HOST uint32[s] (polynomial lattice): the reduced generating polynomials gt_j, coefficient
 *             of x^i at bit i, with gt_j(0) = 1 and deg gt_j < m - w_j (odd and < 2^(m-w_j)), or exactly 1
 *             if w_j >= m: the analogue of z_j (then y = (k(x) gt_j(x) mod x^(m-w_j)) read with the
 *             coefficient of x^i as the digit of 2^(i-(m-w_j))).
 *  C          HOST uint32[s*m] (net): generating matrices as column masks.  Word C[j*m + q] is column q+1
 *             of C^(j); row p (1-based, the digit of 2^-p) is bit m-p of the word (Sec. 4, eq.
 *             def:digital, digits of n least significant first).  The library zeroes the last
 *             min(w_j,m) rows (eq. reduced_genmat_net2); the first m-w_j rows that remain must be
 *             linearly independent over GF(2), so that each value repeats exactly 2^{w_j} times
 *             (otherwise QMC_ERR_INVALID_ARG).  If every reduced C^(j) is zero beyond its column
 *             m-w_j, the net is periodic (column j depends on n mod 2^(m-w_j)) and takes the reduced
 *             product of Algorithm 2.  Otherwise it is a non-periodic reduced net (Sec. 4, Algorithm 4's
 *             case): no column repeats periodically, every column has N distinct rows, the product is
 *             formed densely over all N points, and the workspace grows with N*s.
 *  z          HOST uint32[R_eff * T] (reduced MC): the samples y_{j,i} as X32 = y 2^32, drawn by the
 *             caller (i.i.d. uniform words give i.i.d. U[0,1) samples on the 2^-32 grid).  Replica r
 *             holds, for j = 0..s-1 in order, the N_j = 2^(m-min(w_j,m)) samples y_{j,0..N_j-1} of
 *             column j (the QMC_LAYOUT_DISTINCT layout); T = sum_j N_j.  C, shift and d_shift must be NULL.
 *  R          number of random shifts (0 = unshifted rule); results are produced for R_eff = max(R,1).
 *             Reduced MC: the number of independent replicas (each its own samples in z).
 *  shift      HOST uint32[R*s]: shift r of column j is shift[r*s + j] (units of 2^-32).
 *  transform  QMC_T_*; QMC_T_INV_NORMAL requires R >= 1 for lattices and nets (the unshifted point 0
 *             maps to -inf) and every shift word D_j with a nonzero bit among its low 32 - q_j bits,
 *             q_j = m - min(w_j, m) (otherwise some shifted point of column j is exactly 0, because
 *             the column takes every value u 2^(32-q_j), u < 2^q_j, over a period); reduced MC
 *             requires no zero sample word.  All of this is checked on the host.
 *  d_gen      DEVICE copy of z (s words; reduced MC: R_eff * T words) or C (s*m words), or NULL: then
 *             the host array is copied into the workspace on every call (a pageable copy, which also
 *             prevents CUDA graph capture).  It must hold exactly the host values.
 *  d_shift    DEVICE copy of shift (R*s words) or NULL (uploaded per call like d_gen).
 */
typedef struct {
    int kind;
    uint32_t b, m, s;
    const uint32_t* w;
    const uint32_t* z;
    const uint32_t* C;
    uint32_t R;
    const uint32_t* shift;
    int transform;
    const uint32_t* d_gen;
    const uint32_t* d_shift;
} qmc_rule;

/* An integrand (eq. (2)'s f) from the QMC_F_* family with its parameters. */
typedef struct {
    int kind;
    double params[4];
} qmc_integrand;

/* Library version string and the message of the last failed call on this thread. */
const char* qmc_version(void);
const char* qmc_last_error(void);

/*
 * qmc_validate_rule: host-only check of a rule against the definitions above (no CUDA call).
 */
qmc_status qmc_validate_rule(const qmc_rule* rule);

/*
 * qmc_device_status: synchronises the current device and reads its sticky device error word.
 *  Returns QMC_ERR_TIMEOUT if a tensor-core kernel (QMC_SPLIT / QMC_BF16) gave up a bounded
 *  wait on its MMA completion since the word was last cleared (its outputs were then written
 *  as NaN), or qmc_selftest_wait_timeout ran, QMC_OK otherwise.  clear != 0 resets the word.
 *  Not callable during stream capture.
 */
qmc_status qmc_device_status(int clear);

/*
 * qmc_selftest_wait_timeout: exercises the failure path of the bounded device-side waits without a
 *  fault.  Enqueues one CTA whose single thread polls, at most `polls` times (1 <= polls <= 2^20),
 *  an mbarrier that nothing arrives at, then sets bit 31 of the sticky error word and returns; a
 *  following qmc_device_status reports QMC_ERR_TIMEOUT, and the context stays usable.
 */
qmc_status qmc_selftest_wait_timeout(uint32_t polls, void* stream);

/*
 * qmc_workspace_size: bytes of device workspace `op` needs for these arguments (written to *bytes).
 *  rules/tau/f are arrays of nprob entries (nprob = 1 for GEN_POINTS and REDUCED_MATMUL; f may be
 *  NULL there).  The workspace must be 256-byte aligned.
 */
qmc_status qmc_workspace_size(int op, const qmc_rule* rules, const uint32_t* tau, uint32_t nprob,
                              const qmc_integrand* f, int precision, size_t* bytes);

/*
 * qmc_gen_points: the point set (Sec. 1.3 lattice / Algorithm 3 net, Sec. 2.3 shift), bit-exact.
 *  shift_idx  which shift to apply (ignored when R = 0); reduced MC: which replica.
 *  layout     QMC_LAYOUT_FULL: d_out is N*s uint32, d_out[k*s + j] = X32 of x_{k,j}.
 *             QMC_LAYOUT_DISTINCT: d_out holds, for j = 0..s-1 in order, the 2^(m-min(w_j,m)) values
 *             x_{k,j}, k < 2^(m-min(w_j,m)) (one period of the column); for a non-periodic net, all N
 *             values of every column.
 *  out_words  capacity of d_out in uint32 words (checked).
 *  d_ws       DEVICE workspace (may be NULL when d_gen and d_shift are given).
 */
qmc_status qmc_gen_points(const qmc_rule* rule, uint32_t shift_idx, int layout, uint32_t* d_out,
                          size_t out_words, void* d_ws, size_t ws_bytes, void* stream);

/*
 * qmc_reduced_matmul: the materialised product P = X A of Algorithms 1/2 ("Return P = XA"),
 *  with the shift and transform of the rule applied to X (Sec. 2.3).
 *  d_A   DEVICE s x tau row-major (double for QMC_FP64, float otherwise).
 *  d_P   DEVICE R_eff x N x tau row-major, same element type: d_P[(r*N + k)*tau + t] = (x_k^T A)_t
 *        for shift r.  16-byte aligned (QMC_ERR_INVALID_ARG otherwise, before any CUDA call).
 */
qmc_status qmc_reduced_matmul(const qmc_rule* rule, const void* d_A, uint32_t tau, int precision,
                              void* d_P, void* d_ws, size_t ws_bytes, void* stream);

/*
 * qmc_integrate: QMC estimates Q_N(f) (eq. (2)) for nprob independent problems.
 *  rules[p], d_A[p] (DEVICE s_p x tau[p]), f[p]: problem p.
 *  d_est   DEVICE double; problem p writes R_eff(p)+1 values at offset sum_{p'<p} (R_eff(p')+1):
 *          the per-shift estimates Q_r followed by their mean (the randomised QMC estimate).
 *  d_rowf  NULL, or an array of nprob DEVICE pointers (entries may be NULL): problem p writes the
 *          per-point values f(x_k^T A) for every shift, R_eff x N elements of the precision's type.
 *  The N x tau product itself is never written to memory.  Results are deterministic (fixed
 *  reduction order).
 */
qmc_status qmc_integrate(const qmc_rule* rules, const void* const* d_A, const uint32_t* tau,
                         uint32_t nprob, const qmc_integrand* f, int precision, double* d_est,
                         void* const* d_rowf, void* d_ws, size_t ws_bytes, void* stream);

/*
 * qmc_integrate_backward: gradient of the shift-averaged estimate with respect to A,
 *  dL/dA = upstream_p * (R_eff N)^-1 sum_r X_r^T grad f(X_r A), for every problem p.
 *  d_upstream  DEVICE double[nprob]: dL/dQ for each problem's mean estimate.
 *  d_gradA     array of nprob DEVICE pointers, each s_p x tau[p] of the precision's type (overwritten).
 *  flags       0 or QMC_BWD_REUSE_FORWARD.
 */
qmc_status qmc_integrate_backward(const qmc_rule* rules, const void* const* d_A, const uint32_t* tau,
                                  uint32_t nprob, const qmc_integrand* f, int precision,
                                  const double* d_upstream, void* const* d_gradA, uint32_t flags,
                                  void* d_ws, size_t ws_bytes, void* stream);

/*
 * Schedule autotuning (the paper has no counterpart: it picks launch shapes of this library's
 * kernels, never the arithmetic).  For a problem shape (m, the column counts per weight level,
 * tau, shifts, precision, integrand) the planner uses a cached schedule when one exists, else its
 * cost models: the fine band's forward columns per CTA and adjoint roots per CTA, and in the
 * the fine forward's level-3 nodes per thread and the fine adjoint's column pairs per lane
 * (autotuned only), in the
 * tensor-core tiers the coarse forward's path (1 level passes, 2 block products and chain sum)
 * and the coarse adjoint's path (1 one fold of the root gradients and the cp.async block-gradient
 * kernel, 2 the fused fold-gradient kernel and the TMA block-gradient kernel).
 *  qmc_autotune  times, with CUDA events on `stream`, the forward and the forward + backward of this
 *                problem under the cost model's schedule and a ladder of others, and caches the
 *                fastest.  d_est (R_eff + 1 doubles), d_gradA (s x tau) and d_ws are scratch: the
 *                timed runs overwrite them.  Candidates whose workspace exceeds ws_bytes are skipped;
 *                a tuned schedule can change qmc_workspace_size, so size workspaces after tuning.
 *                Synchronises the stream (not callable during stream capture).  *n_timed (may be
 *                NULL) receives the number of candidates timed.
 *  qmc_tune_set  caches the given schedule for this problem's shape (host only, no CUDA call):
 *                fwd_qpg (columns per CTA / 4, <= 128), bwd_rpc (roots per CTA), coarse (0-2) and
 *                bwd_path (0-2); 0 keeps the cost model's choice of that value.  QMC_ERR_INVALID_ARG
 *                for values out of range or an invalid rule; QMC_ERR_UNSUPPORTED for rules in a base
 *                b > 2, whose plan takes no schedule.
 *  qmc_tune_save / qmc_tune_load   write / merge the cache as a text file, one line per shape
 *                ("key|columns per CTA / 4|roots per CTA|coarse path|adjoint path|forward level-3
 *                nodes per thread (1 or 2)|adjoint column pairs per lane (1 or 2)"; the last four are
 *                optional when loading; 0 keeps the cost model's choice).
 *  qmc_tune_clear  empties the cache.
 */
qmc_status qmc_autotune(const qmc_rule* rule, const void* d_A, uint32_t tau, const qmc_integrand* f, int precision,
                        double* d_est, void* d_gradA, void* d_ws, size_t ws_bytes, void* stream, uint32_t* n_timed);
qmc_status qmc_tune_set(const qmc_rule* rule, uint32_t tau, const qmc_integrand* f, int precision, int fwd_qpg,
                        int bwd_rpc, int coarse, int bwd_path);
qmc_status qmc_tune_save(const char* path);
qmc_status qmc_tune_load(const char* path, uint32_t* n_entries);
qmc_status qmc_tune_clear(void);

/*
 * qmc_integrate_noalloc: qmc_integrate for one problem without a caller workspace and without
 *  allocating any device memory.  The paper has no counterpart; this entry point serves callers
 *  that cannot allocate device memory when they call the library (a framework that forbids
 *  cudaMalloc while it captures a stream, a real-time or embedded host that reserves all device
 *  memory up front, a foreign-function caller with no device allocator of its own).
 *  Scratch space is a static 64 MiB array inside the library (present on every GPU that loads
 *  the library, until the process exits).  Problems whose qmc_workspace_size(QMC_OP_INTEGRATE)
 *  exceeds it are rejected with QMC_ERR_NO_MEMORY before any work is enqueued.
 *  Arguments are those of qmc_integrate for nprob = 1, without d_rowf: d_A DEVICE s x tau,
 *  d_est DEVICE double[R_eff + 1].  The first call on each device looks up the array's device
 *  address (cudaGetSymbolAddress); make that first call before any stream capture.  All calls
 *  share the one array: calls whose work overlaps on the GPU (other streams, other host threads)
 *  race on it and must be serialised by the caller.  The array keeps the last call's contents;
 *  every value a call reads from it is written earlier in the same call.
 */
qmc_status qmc_integrate_noalloc(const qmc_rule* rule, const void* d_A, uint32_t tau,
                                 const qmc_integrand* f, int precision, double* d_est, void* stream);

/*
 * Kernel tracing (library instrumentation; the paper has no counterpart).
 *  qmc_trace_enable(1) clears earlier records and brackets every kernel the library launches from
 *  then on with two CUDA events recorded on the launch stream; qmc_trace_enable(0) stops recording.
 *  qmc_trace_collect waits for the recorded events and aggregates them per kernel name (*n_kernels
 *  distinct names); qmc_trace_entry(i, ...) returns name i (valid until the next collect or enable),
 *  its launch count and its summed device time in milliseconds.  Tracing adds two event records per
 *  launch and must not be enabled while a stream is being captured into a CUDA graph.
 */
qmc_status qmc_trace_enable(int on);
qmc_status qmc_trace_collect(uint32_t* n_kernels);
qmc_status qmc_trace_entry(uint32_t i, const char** name, uint64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* QMC_GB300_H */
