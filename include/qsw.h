/*
 * qsw.h -- C ABI of the GB300 L-QSW time-series library (libqsw.so).
 *
 * The library computes the time series of a locally-interacting quantum
 * stochastic walk (L-QSW) on a weighted digraph,
 *
 *     rho~(t_k) = exp(t_k L~) rho~(0),   t_k = t0 + k dt,  k = 0..steps,
 *
 * where L~ is the N~^2 x N~^2 vectorised superoperator of the master equation
 * (paper: QSW_MPI, arXiv:2003.02450, Section 2.5, Eqs. qsw, qsw_ss,
 * vec_mappings, qsw_vec_sol), computed by Al-Mohy & Higham's truncated-Taylor
 * scaling-and-squaring algorithms (paper Section 3.1: Algorithm 3.2 `step`,
 * Algorithm 5.2 `series`, parameters from the 1-norm series of L~ that is
 * precomputed at construction, Section 4 footnote).
 *
 * Conventions used by every call
 * ------------------------------
 * - Graphs: CSR with row = destination vertex i, column = source vertex j, so
 *   that G[i][j] = w(v_i, v_j) is the weight of the arc j -> i
 *   (Eq. adjacency_graph; the printed omega = 1 example of Section 4 fixes this
 *   orientation).  Columns strictly increasing within a row, no self-loops
 *   (simple graphs, Tr G = 0), weights finite and > 0.  Graph arrays are HOST
 *   pointers; the library copies them.
 * - Vectorisation is column-major: rho~[i + N~ j] = rho[i][j] (Section 2.5.3).
 *   Sources, then sinks, are appended after the N graph vertices, in argument
 *   order, so N~ = N + n_sources + n_sinks (Section 2.5.1).
 * - Complex numbers are interleaved (re, im) pairs of doubles: a state vector
 *   of n = N~^2 entries occupies 2n doubles (16 n bytes).
 * - "d_" arguments are DEVICE pointers on the context's device, owned by the
 *   caller; "h_" arguments are host pointers.  Every call is ordered on the
 *   context's CUDA stream; calls that return results or statistics to the host
 *   synchronise that stream before returning.
 * - A context, and the operators built on it, serve one host thread at a
 *   time; separate contexts (each with its own stream) may run concurrently.
 *   The qsw_server_* calls are safe from any thread.
 * - No exception crosses this boundary: every call returns a qsw_status and,
 *   on failure, a message retrievable with qsw_last_error().  Failed calls
 *   leave caller buffers in an unspecified state and leak nothing.
 * - Index limits: N~^2 and nnz(L~) must each be < 2^31 (32-bit CSR indices,
 *   as in the paper's Section 3.2); larger problems return QSW_ERR_TOO_LARGE.
 */
#ifndef QSW_H
#define QSW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QSW_OK = 0,
  QSW_ERR_INVALID_ARG = 1,    /* bad pointer, size, CSR structure, time grid */
  QSW_ERR_NOT_SIMPLE = 2,     /* self-loop or non-positive weight (Section 2.1: simple graphs) */
  QSW_ERR_OMEGA_RANGE = 3,    /* omega outside [0, 1] (Eq. qsw) */
  QSW_ERR_OOM = 4,            /* device allocation failed */
  QSW_ERR_NOT_CONVERGED = 5,  /* a device loop hit its iteration or wait limit */
  QSW_ERR_CUDA = 6,           /* any other CUDA runtime error */
  QSW_ERR_TOO_LARGE = 7,      /* N~^2 or nnz(L~) does not fit 32-bit indices */
  QSW_ERR_NOT_HERMITIAN = 8   /* caller-supplied H is not symmetric */
} qsw_status;

/* Arithmetic of the Taylor loop.
 * QSW_C128: complex128 superoperator and vectors, tolerance 2^-53 (Section 5).
 * QSW_C64_BULK: complex64 superoperator values and Taylor terms with FP32
 *   accumulation of every matrix-vector product; the running Taylor sum, the
 *   stop test's norms, the 1-norm estimates and the (m, s) choice stay FP64;
 *   tolerance 2^-24 with its own theta table.  Not in the paper. */
typedef enum { QSW_C128 = 0, QSW_C64_BULK = 1 } qsw_precision;

/* How the series applies L~.
 * QSW_OPERATOR_MATRIX_FREE (default): from H and the jump lists directly
 *   (Eq. vec_mappings applied to Eq. qsw_ss), no stored superoperator; every
 *   term is a real coefficient times a complex entry.  Same operator as the CSR
 *   entry by entry; only the summation order differs.
 * QSW_OPERATOR_CSR: the assembled CSR superoperator (Section 3.2-3.3). */
typedef enum { QSW_OPERATOR_MATRIX_FREE = 0, QSW_OPERATOR_CSR = 1 } qsw_operator;

/* OR-ed into operator_kind: skip the 1-norm series at construction.  The
 * norms are then computed when the operator is first used (by
 * qsw_expmv_series, or on the device by qsw_batch_series). */
#define QSW_BUILD_DEFER_NORMS 0x100

/* OR-ed into operator_kind: do not autotune this operator's schedule (a
 * QSW_OPERATOR_CSR operator then keeps the row-length heuristic's lanes per
 * row instead of the tuned value; see qsw_op_schedule). */
#define QSW_BUILD_FIXED_SCHEDULE 0x200

/* OR-ed into operator_kind: take every product of the 1-norm estimator in
 * complex128.  By default the matrix-free L-QSW operator runs the adjoint
 * step Z = (L~^H)^p sign(Y) of Higham & Tisseur's Algorithm 2.4 in complex64:
 * Z only ranks rows (which unit vectors to try next, and the stop test on the
 * best one), while every estimate is the complex128 1-norm of L~^p x for a
 * column x the algorithm tried.  Both forms return estimates the algorithm
 * can return; they may follow different branches where two row maxima are
 * within complex64 rounding of each other. */
#define QSW_BUILD_FP64_RANKING 0x400

typedef struct qsw_ctx qsw_ctx;   /* device + stream + workspace cache */
typedef struct qsw_op qsw_op;     /* one assembled superoperator L~ */

/* Weighted digraph / Hamiltonian in CSR (host arrays, see conventions). */
typedef struct {
  int32_t n;               /* vertices */
  int32_t nnz;             /* stored entries */
  const int32_t* rowptr;   /* [n + 1], rowptr[0] = 0, rowptr[n] = nnz */
  const int32_t* col;      /* [nnz], strictly increasing within a row */
  const double* w;         /* [nnz] */
} qsw_csr;

/* A source (feeding `vertex`) or a sink (draining `vertex`) with its rate
 * Gamma or Theta (Section 2.5.1, Eq. qsw_ss).  The rate multiplies a unit
 * jump operator and is not scaled by omega. */
typedef struct {
  int32_t vertex;
  double rate;
} qsw_port;

/* Statistics of one qsw_expmv_series call (filled when non-null). */
typedef struct {
  int32_t m0, s0;            /* (m*, s) used for the first state, exp(t0 L~) rho0 */
  int32_t m_star, s;         /* (m*, s) for the whole interval (steps * dt) L~ */
  int32_t step_m, step_s;    /* (m*, s) of each dt step when steps <= s (else 0) */
  int32_t outputs_per_block; /* d of Algorithm 5.2 (0 when steps <= s) */
  int32_t jobs;              /* Taylor blocks executed */
  int64_t matvecs;           /* applications of L~ performed */
  double bytes_per_matvec;   /* algorithmic bytes of one application of L~ */
  double kernel_ms;          /* device time of the series kernel (CUDA events) */
  int64_t fupdates;          /* sum over Taylor terms of the outputs updated */
  double algorithmic_bytes;  /* bytes the series kernel must move: matvecs x
                                bytes_per_matvec + 32 n fupdates + block inits */
  double algorithmic_flops;  /* FP64 (QSW_C128) or FP32 + FP64 (QSW_C64_BULK)
                                flops of the series: per application of L~,
                                4 per real x complex off-diagonal term, 8 per
                                diagonal term, 4 per jump term, 2 per scaling,
                                3 per squared modulus; per updated output
                                element 4 + 3 */
  int32_t hermitian;         /* 1: rho0 was Hermitian and the matrix-free form
                                computed upper triangles only (every Taylor
                                term of a Hermitian matrix is Hermitian) */
} qsw_series_stats;

/* A complex sparse matrix in CSR (host arrays): row i holds columns
 * col[rowptr[i] .. rowptr[i+1]-1], strictly increasing, values re + i im
 * (im may be NULL for a real matrix). */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* re;
  const double* im;
} qsw_zcsr;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL selects the legacy default stream).  The stream is
 * borrowed, not owned.  Errors: INVALID_ARG (null ctx / bad device), CUDA. */
qsw_status qsw_create(qsw_ctx** ctx, int device, void* cuda_stream);

/* Destroy a context and its workspace (ops must be destroyed first). */
void qsw_destroy(qsw_ctx* ctx);

/* Message of the last failed call on `ctx` ("" if none).  Owned by ctx. */
const char* qsw_last_error(const qsw_ctx* ctx);

/* ---------------------------------------------------------- construction */

/* Build L~ for an L-QSW (paper Section 2.5, Eq. qsw_ss; condensed
 * construction of Section 3.3, Eq. condensed_lindblads).
 *   G        : the digraph (host CSR).  One jump operator sqrt(G_ij)|i><j| per
 *              arc j -> i (Eq. lindblad), weighted by omega.
 *   H        : the Hamiltonian (host CSR, real symmetric, N x N), used exactly
 *              as given; NULL selects trans(1, G^u), the Laplacian of the
 *              undirected companion G^u = max(G, G^T) (Eq. generator_matrix).
 *   omega    : decoherence parameter in [0, 1] (Eq. qsw).
 *   sources, n_sources, sinks, n_sinks : ports (may be NULL when the count is 0).
 *   precision: a qsw_precision.
 *   operator_kind: a qsw_operator.  With QSW_OPERATOR_CSR the CSR is assembled
 *              here; with QSW_OPERATOR_MATRIX_FREE it is assembled only if
 *              qsw_op_export_csr asks for it.
 * On success *out receives a library-owned operator (free with
 * qsw_op_destroy).  Construction also precomputes ||L~||_1 exactly and
 * estimates ||L~^p||_1 for p = 2..9 (Section 4 footnote) on the device.
 * Errors: INVALID_ARG, NOT_SIMPLE, OMEGA_RANGE, NOT_HERMITIAN, TOO_LARGE, OOM,
 * CUDA.  Synchronises the stream. */
qsw_status qsw_build_superoperator(qsw_ctx* ctx, const qsw_csr* G, const qsw_csr* H,
                                   double omega, const qsw_port* sources, int32_t n_sources,
                                   const qsw_port* sinks, int32_t n_sinks,
                                   int32_t precision, int32_t operator_kind, qsw_op** out);

/* Rebuild the values and the 1-norm series of `op` at a new omega, keeping
 * its graph, Hamiltonian and ports (the package's set_omega, Section 4). */
qsw_status qsw_set_omega(qsw_op* op, double omega);

/* Sizes and norms of an operator.  norms[0] = ||L~||_1 (exact; for a global
 * walk exact when it has one Lindblad operator without diagonal entries, else
 * estimated), norms[p-1] = estimate of ||L~^p||_1 for p = 2..9.  n_tilde is the
 * state dimension N~ (the vertex copies for an NM-G-QSW), n = N~^2.  Any
 * output pointer may be NULL; asking for the norms of an operator built with
 * QSW_BUILD_DEFER_NORMS computes them. */
qsw_status qsw_op_info(const qsw_op* op, int64_t* n_tilde, int64_t* n, int64_t* nnz,
                       double* norms9);
/* nnz is the number of stored entries of the CSR form of L~ (computed from the
 * structure without assembling it); 0 for global-interaction walks, which have
 * no CSR form. */

/* Copy the CSR of L~ (assembled on first use for a matrix-free operator) into
 * caller device buffers: d_rowptr[n + 1],
 * d_col[nnz], d_val[2 nnz] (complex128; for a QSW_C64_BULK operator its
 * complex64 values are widened).  Any pointer may be NULL to skip that array.
 * Used by tests and tools.  Errors: INVALID_ARG for global-interaction walks. */
qsw_status qsw_op_export_csr(const qsw_op* op, int32_t* d_rowptr, int32_t* d_col,
                             double* d_val);

void qsw_op_destroy(qsw_op* op);

/* ------------------------------------------------------------- evolution */

/* d_state[n] (complex128) <- vec(rho0).  Exactly one of h_rho0 (N~ x N~
 * complex128, column-major, interleaved) or h_populations (N~ doubles: a
 * diagonal rho0, off-diagonals zero; Section 4 `initial_state`) is non-NULL.
 * Errors: INVALID_ARG (both/neither given, trace not 1 within 1e-12). */
qsw_status qsw_initial_state(const qsw_op* op, const double* h_rho0,
                             const double* h_populations, double* d_state);

/* One application y = L~ x (complex128 in and out; a QSW_C64_BULK operator
 * computes in complex64 with FP32 accumulation and widens).  d_x, d_y: n
 * complex128, must not overlap. */
qsw_status qsw_apply(const qsw_op* op, const double* d_x, double* d_y);

/* The L-QSW time series (Algorithm 5.2 `series`; steps = 0 gives Algorithm 3.2
 * `step` at t0):
 *   d_rho0 : n complex128 (device), vec(rho(0)).
 *   t0, dt : start time and spacing, finite and >= 0.
 *   steps  : q >= 0 intervals; the series has steps + 1 states, state k at
 *            t0 + k dt (state 0 at t0).
 *   d_out  : (steps+1) x n complex128 (device, state k at offset 2 n k
 *            doubles) or NULL.
 *   d_pops : (steps+1) x N~ doubles (device), p_i(t_k) = Re rho_ii(t_k), or NULL.
 *   stats  : host struct or NULL.
 * At least one of d_out / d_pops must be non-NULL.  Synchronises the stream.
 * Any number of output times: an Algorithm 5.2 block of d > 128 outputs runs
 * as ceil(d / 128) jobs that each start from the block's input and form its
 * Taylor powers again (each output gets exactly the arithmetic of the whole
 * block; the extra cost is the repeated operator applications).  With d_out
 * NULL the outputs of one block are kept in a device ring of d + 1 states.
 * Errors: INVALID_ARG, OOM, NOT_CONVERGED (a device wait exceeded its limit),
 * CUDA. */
qsw_status qsw_expmv_series(qsw_op* op, const double* d_rho0, double t0, double dt,
                            int32_t steps, double* d_out, double* d_pops,
                            qsw_series_stats* stats);

/* Size of the fixed device scratch behind qsw_expmv_series_noalloc. */
#define QSW_NOALLOC_SCRATCH_BYTES (16u << 20)

/* qsw_expmv_series without any device allocation.  The paper has no
 * counterpart: this is a property of the library, not of the method.
 *
 * Same arguments, results, errors and synchronisation as qsw_expmv_series,
 * but the call's workspace (control words, the Taylor block plan, the two
 * Taylor-term vectors and, when d_out is NULL, the ring of output slots)
 * lives in one array of QSW_NOALLOC_SCRATCH_BYTES per device, reserved when
 * the library's module loads.  Nothing in the call asks cudaMalloc,
 * cudaMallocAsync or any other allocator for memory.  It is for callers that
 * cannot allocate: a serving process whose device memory has been handed in
 * full to another allocator's pool (an allocation would fail or evict that
 * pool's cache), and latency-bound loops where an allocation or free may
 * wait on other work on the device.
 *
 * - The operator must already hold its 1-norm series: one built without
 *   QSW_BUILD_DEFER_NORMS, or used once by qsw_expmv_series.  Otherwise
 *   INVALID_ARG (computing the norms needs workspace).
 * - A series whose workspace exceeds QSW_NOALLOC_SCRATCH_BYTES is rejected
 *   with TOO_LARGE before any work is issued.  The workspace is
 *   (2 n + ring n) complex values plus the plan: with d_out given (no
 *   ring) about 2 n x 16 bytes for QSW_C128, i.e. N~ up to ~700.
 * - The call clears the parts that must start at zero itself (the control
 *   words and the Hermiticity-check accumulators).
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, checked; CUDA error otherwise); make that first
 *   call before any stream capture.  The address is kept for the life of
 *   the process, so the device's primary context must live as long: do not
 *   call cudaDeviceReset between calls.
 * - Every call on a device shares the array: calls in flight at the same time
 *   on one device (other threads, contexts or streams) race.
 * - stats->kernel_ms is 0 (no timing events are created). */
qsw_status qsw_expmv_series_noalloc(qsw_op* op, const double* d_rho0, double t0, double dt,
                                    int32_t steps, double* d_out, double* d_pops,
                                    qsw_series_stats* stats);

/* Same computation with HOST buffers: h_rho0 (n complex128), h_out / h_pops
 * as d_out / d_pops above but in host memory (pinned memory is fastest).  The
 * host<->device copies are part of the call: outputs are copied to h_out on a
 * second stream owned by the context as soon as the Taylor block that computes
 * them has finished (the series kernel reports its progress through a
 * host-mapped counter owned by the context), overlapping the copies with the
 * later blocks; populations are copied after the kernel.  Results are the
 * same bits as qsw_expmv_series with device buffers.  One call at a time per
 * context. */
qsw_status qsw_expmv_series_host(qsw_op* op, const double* h_rho0, double t0, double dt,
                                 int32_t steps, double* h_out, double* h_pops,
                                 qsw_series_stats* stats);

/* Populations of `count` consecutive states: d_pops[c N~ + i] =
 * Re d_rho_series[c n + i (N~ + 1)] (Section 2.4; `gather_populations`). */
qsw_status qsw_populations(const qsw_op* op, const double* d_rho_series, int32_t count,
                           double* d_pops);

/* ------------------------------------------------------------ batching */

/* Statistics of one qsw_batch_series call. */
typedef struct {
  int32_t walks;        /* walks in the batch */
  int32_t clusters;     /* thread-block clusters (cluster_size CTAs each)
                           launched for the series phase (0: every walk was
                           small) */
  double norms_ms;      /* device time of the 1-norm phase */
  double series_ms;     /* device time of the series phase */
  int64_t matvecs;      /* applications of the walks' L~ to an n x n0 block */
  int64_t fupdates;     /* sum over terms of the outputs updated */
  int32_t small_walks;  /* walks whose two n x n0 Taylor-term blocks fit in
                           small_limit bytes: run by one thread block each
                           with the terms in shared memory, alongside the
                           clusters */
  double algorithmic_flops;  /* series phase, all walks: the operator's flops
                                on every right-hand side (FP32 for complex64
                                bulk walks, FP64 otherwise) plus the FP64 output
                                updates, counted as in qsw_series_stats */
  double algorithmic_bytes;  /* series phase, all walks: operator data, term
                                read and written, output updates per
                                application, as in qsw_series_stats */
  int32_t cluster_size;      /* the series phase's schedule: CTAs per cluster */
  int32_t small_limit;       /* ... and the largest pair of Taylor-term blocks
                                (bytes) run by one CTA (0: none) */
  int32_t tuned;             /* 1: this call timed the candidate schedules */
} qsw_batch_stats;

/* Many independent walks in one launch (not in the paper): walk w is `ops[w]`
 * (built with QSW_OPERATOR_MATRIX_FREE, any precision), evolved from the n0
 * right-hand sides d_rho0[w] (n0 x n_w complex128, device, column c at offset
 * 2 n_w c doubles; 1 <= n0 <= 4, treated as one n_w x n0 block as in
 * Algorithm 3.2/5.2) over its own grid t0[w], dt[w], steps[w] (host arrays).
 * d_pops[w] receives (steps[w]+1) x n0 x N~_w populations (device; entry
 * [(k n0 + c) N~_w + i]).  Each walk is handled by one cluster of thread
 * blocks; walks with Hermitian right-hand sides are computed on upper
 * triangles.  The 1-norm estimates are computed on the device only when Code
 * Fragment 3.1 needs them for the walk's time span.  Any number of output
 * times: Taylor blocks of more than 64 outputs run as several jobs from the
 * block's input, as in qsw_expmv_series.  Synchronises the stream.
 * Errors: INVALID_ARG, OOM, CUDA. */
qsw_status qsw_batch_series(qsw_ctx* ctx, int32_t count, qsw_op* const* ops,
                            const double* const* d_rho0, int32_t n0, const double* t0,
                            const double* dt, const int32_t* steps, double* const* d_pops,
                            qsw_batch_stats* stats);

/* The series phase's schedule for this context's batched calls.  By default
 * (cluster_size 0, small_limit -1) it is autotuned: the first batch of a kind
 * (n0, the precisions present, the largest N~ and the walk count, each by
 * power of two) with at least 16 walks times its own series phase under every
 * candidate (clusters of 4, 8 or 16 CTAs x one-CTA limit 0, 32 or 64 KB),
 * keeps the fastest for the process and counts one measurement
 * (qsw_tune_measurements); smaller batches run clusters of 8 and a 64 KB
 * limit.  A walk's populations do not depend on the schedule (same
 * per-element arithmetic; the phase's cluster reductions are maxima).
 * cluster_size: 0 (tuned) or 2, 4, 8, 16; small_limit: -1 (tuned) or 0 ..
 * 65536 bytes (walks whose two Taylor-term blocks, 2 n0 n_w values of the
 * walk's precision, fit run on one thread block with the terms in shared
 * memory).  A fixed value replaces only its own half of the pair: the other
 * half is the tuned one when this kind of batch has been tuned, else the
 * default; no call tunes while either half is fixed.  Errors: INVALID_ARG. */
qsw_status qsw_batch_set_schedule(qsw_ctx* ctx, int32_t cluster_size, int32_t small_limit);

/* ------------------------------------------ global-interaction walks */

/* A global-interaction walk (G-QSW, Section 2.5.2, Eq. L_global; the
 * non-moralising NM-G-QSW of Eq. nm_gqsw): on n_vertices vertices plus the
 * ports,
 *   d rho/dt = -i(1-omega)[H, rho] + omega sum_k (L_k rho L_k^dag - 1/2 {L_k^dag L_k, rho})
 *              + i omega [H_rot, rho] + (source / sink terms as for the L-QSW),
 * with H (Hermitian, required), n_L <= 8 Lindblad operators L_k (any complex
 * n_vertices x n_vertices matrices) and an optional Hermitian H_rot (NULL:
 * none).  The operator is matrix-free (no CSR form: qsw_op_info reports
 * nnz = 0 and qsw_op_export_csr is refused); qsw_expmv_series,
 * qsw_survival_time, qsw_apply, qsw_populations, qsw_initial_state and
 * qsw_set_omega accept it; the batched and no-allocation entry points do not.
 * ||L~||_1 is exact for one L_k without diagonal entries, estimated
 * otherwise.  flags: 0 or QSW_BUILD_DEFER_NORMS.
 * Errors: INVALID_ARG, OMEGA_RANGE, NOT_HERMITIAN, TOO_LARGE, OOM, CUDA. */
qsw_status qsw_build_global(qsw_ctx* ctx, int32_t n_vertices, const qsw_zcsr* H,
                            const qsw_zcsr* Ls, int32_t n_L, const qsw_zcsr* H_rot, double omega,
                            const qsw_port* sources, int32_t n_sources, const qsw_port* sinks,
                            int32_t n_sinks, int32_t precision, int32_t flags, qsw_op** op);

/* The G-QSW of digraph G (Section 2.5.2): one Lindblad operator
 * L_global = sum_ij G_ij |v_i><v_j| (G itself, row = destination) and H as
 * passed, or trans(1, G^u) (the Laplacian of the undirected companion) when H
 * is NULL.  Errors as qsw_build_superoperator. */
qsw_status qsw_build_gqsw(qsw_ctx* ctx, const qsw_csr* G, const qsw_csr* H, double omega,
                          const qsw_port* sources, int32_t n_sources, const qsw_port* sinks,
                          int32_t n_sinks, int32_t precision, qsw_op** op);

/* The non-moralising G-QSW of digraph G (Section 2.5.2 "Graph
 * Demoralisation", Eq. nm_gqsw): vertex v becomes d_v = max(1, deg_{G^u}(v))
 * copies; H^D = trans(1, G^{uD}) with G^{uD} weights w / sqrt(d_v d_u); one
 * Lindblad operator L^D that sends each copy of u, for an arc u -> v, to the
 * Fourier column F_{d_v}[., c_v(u)] (F_d[j, c] = exp(2 pi i j c / d), c_v(u)
 * the position of u among v's sorted G^u neighbours) with amplitude
 * w / sqrt(d_v d_u); the rotating Hamiltonian <v^{k+1}|H_rot|v^k> = i.  The
 * operator lives on the N^D = sum_v d_v copies (qsw_op_info: N~ = N^D); use
 * qsw_nm_initial_state and qsw_nm_populations for vertex populations.
 * Errors as qsw_build_superoperator. */
qsw_status qsw_build_nm_gqsw(qsw_ctx* ctx, const qsw_csr* G, double omega, int32_t precision,
                             qsw_op** op);

/* offsets[v] .. offsets[v+1]-1 index vertex v's copies (host array of N+1).
 * Errors: INVALID_ARG (not an NM-G-QSW operator). */
qsw_status qsw_nm_vsets(const qsw_op* op, int32_t* offsets);

/* Eq. nm_rho_map for `count` population vectors: d_pops[c N + v] = sum over
 * v's copies k of d_pops_expanded[c N^D + k] (device arrays).  Synchronises. */
qsw_status qsw_nm_populations(const qsw_op* op, const double* d_pops_expanded, int32_t count,
                              double* d_pops);

/* rho^D(0) with vertex populations h_pops (host, N values summing to 1)
 * spread uniformly over each vertex's copies (diagonal), into d_state
 * (N^D x N^D complex128, device).  Synchronises. */
qsw_status qsw_nm_initial_state(const qsw_op* op, const double* h_pops, double* d_state);

/* ------------------------------------------- expected survival time */

/* Expected survival time of a walk with a sink (Section 4.1.4, transport
 * through a disordered network):
 *   eta = integral over [0, t_end] of (1 - p_sink(t)),
 * evaluated as the paper does: the series of populations at t_k = k h,
 * h = t_end / q, k = 0..q (qsw_expmv_series from t0 = 0), then Simpson's rule
 * h/3 (y_0 + 4 y_1 + 2 y_2 + ... + 4 y_{q-1} + y_q) on y_k = 1 - p_sink(t_k).
 * `sink` is the vertex index of the sink (sinks follow the N graph vertices
 * and the sources).  q must be even and >= 2; t_end finite and > 0.  *eta is
 * a host double.  d_pops, when non-NULL, receives the (q+1) x N~ populations
 * (device); otherwise the call uses its own workspace.  Synchronises the
 * stream.  Errors: INVALID_ARG (odd q, bad sink, ...), OOM, NOT_CONVERGED,
 * CUDA. */
qsw_status qsw_survival_time(qsw_op* op, const double* d_rho0, double t_end, int32_t q,
                             int32_t sink, double* eta, double* d_pops, qsw_series_stats* stats);

/* The same for `count` walks in one batched launch (qsw_batch_series with
 * n0 = 1, t0 = 0, dt = t_end[w] / q[w], steps = q[w]), e.g. a sweep of eta over
 * omega.  t_end, q, sink and eta are host arrays of `count` entries; the
 * populations live in the call's workspace.  Errors as qsw_batch_series, plus
 * those of qsw_survival_time. */
qsw_status qsw_batch_survival_time(qsw_ctx* ctx, int32_t count, qsw_op* const* ops,
                                   const double* const* d_rho0, const double* t_end,
                                   const int32_t* q, const int32_t* sink, double* eta,
                                   qsw_batch_stats* stats);

/* --------------------------------------------------------- diagnostics */

/* Exercise the bounded wait of the series kernel's grid barrier (not in the
 * paper): a cooperative launch in which one block never arrives, so the
 * others give up after about a second of polling and record the timeout, as a
 * series would (QSW_ERR_NOT_CONVERGED).  Returns QSW_OK when the timeout was
 * reported; *seconds (optional) receives the time the launch took.  The
 * context stays usable.  Errors: INVALID_ARG, CUDA (the timeout was not
 * reported). */
qsw_status qsw_probe_wait_limit(qsw_ctx* ctx, double* seconds);

/* ------------------------------------------------------------- serving */

/* A request server (not in the paper): walks of any size, omega, time grid and
 * precision are submitted from any host thread and evolved as they arrive.
 * `workers` threads each own a CUDA stream; a free worker takes every queued
 * request that fits the device-memory budget (oldest first, up to max_batch),
 * builds their operators, runs them as one batched launch (qsw_batch_series,
 * one thread-block cluster per walk) and copies the populations to the
 * request's host buffer.  Requests arriving while batches run are launched by
 * another worker on its own stream, so their work overlaps on the device.  A
 * request's populations do not depend on which other requests share its
 * batch.  A worker's batches take the series-phase schedule tuned for their
 * kind by earlier qsw_batch_series calls in the process (the default when
 * there is none): a worker never stalls a batch to time candidates.
 * memory_budget_bytes = 0 selects half of the free device memory; a request
 * larger than the budget runs alone. */
typedef struct {
  int32_t workers;             /* concurrent batches (streams), >= 1; 0 -> 2 */
  int32_t max_batch;           /* requests per batched launch; 0 -> 64 */
  double memory_budget_bytes;  /* admission limit on the summed footprints */
} qsw_server_config;

typedef struct qsw_server qsw_server;

typedef struct {
  qsw_csr graph;               /* host digraph (copied at submit); H = Laplacian of G^u */
  double omega;
  int32_t precision;           /* qsw_precision */
  const double* rho0;          /* host N x N complex128 column-major, or NULL */
  const double* populations;   /* host N doubles (diagonal rho0), or NULL */
  double t0, dt;
  int32_t steps;
  double* pops_out;            /* host (steps+1) x N doubles, written on completion;
                                  must stay valid until qsw_server_wait returns */
} qsw_request;

typedef struct {
  qsw_status status;
  double latency_ms;           /* submit -> populations on the host */
  double queue_ms;             /* submit -> taken by a worker */
  char error[256];
} qsw_request_result;

qsw_status qsw_server_create(int device, const qsw_server_config* config, qsw_server** out);
/* Enqueue a request; *id identifies it.  The graph and rho0 are copied. */
qsw_status qsw_server_submit(qsw_server* server, const qsw_request* request, int64_t* id);
/* Wait up to timeout_s seconds for request `id`; returns its status
 * (QSW_ERR_NOT_CONVERGED on timeout, the request stays pending).  A completed
 * request is forgotten after this call. */
qsw_status qsw_server_wait(qsw_server* server, int64_t id, double timeout_s,
                           qsw_request_result* result);
qsw_status qsw_server_stats(qsw_server* server, int64_t* queued, int64_t* batches,
                            double* bytes_in_use);
/* Finish every queued request, stop the workers and free everything. */
void qsw_server_destroy(qsw_server* server);

/* ----------------------------------------------------- host-side helpers */

/* Number of CUDA kernels this library has launched in the calling process
 * (all contexts), for launch accounting.  Pure host call. */
int64_t qsw_kernel_launches(void);

/* Number of device-memory allocations (stream-ordered cudaMallocAsync) the
 * library has made in the calling process, all contexts.  Pure host call; a
 * caller can read it around a call to see whether that call allocated. */
int64_t qsw_device_allocations(void);

/* ------------------------------------------------------------ autotuning
 *
 * Not in the paper (a schedule choice of this library).  The CSR sweep of
 * the series kernel runs TPR lanes per row of L~ (1, 2, 4, 8, 16 or 32), which
 * sets the cost of its shuffle reductions and how the operator stream is
 * coalesced, or the sliced form (qsw_op_schedule), and keeps 2 or 4 entries
 * per lane in flight (unroll depth).
 * The first qsw_expmv_series on a QSW_OPERATOR_CSR operator
 * (without QSW_BUILD_FIXED_SCHEDULE) looks up the device's choice for its
 * (precision, row-length bucket, size bucket); when there is none it times
 * every candidate pair with the series kernel on that operator (eight Taylor
 * terms from a fixed vector, 42 short launches, plus two Taylor-term vectors
 * of workspace and the sliced copy of the operator, which is kept only when
 * the sliced form wins), keeps the fastest for the life of the process and
 * uses it for every later operator in that bucket.  Results depend on the
 * choice only through the summation order within a row (well inside the
 * 1e-10 parity bound).  The no-allocation entry point never tunes: it uses
 * the operator's current value, and the sliced form only when its copy is
 * already built (after qsw_set_omega, the first qsw_expmv_series rebuilds
 * it; until then the no-allocation call runs the lanes-per-row form). */

/* Number of schedule measurements (one per tuned CSR bucket, and one per
 * tuned kind of batch: qsw_batch_set_schedule) made in this process.  Pure
 * host call. */
int64_t qsw_tune_measurements(void);
/* Forget every tuned schedule (the next CSR operator of each bucket, and the
 * next batch of each kind, is measured again).  Pure host call; not safe
 * against concurrent series. */
void qsw_tune_reset(void);
/* The operator's CSR schedule (0 and 0 for a matrix-free operator): lanes
 * per row and the row loop's unroll depth (2 or 4 entries per lane in flight;
 * csr_unroll may be NULL).  lanes per row -1: the sliced form (one lane per
 * row, the operator copied into 32-row slices sorted by row length within
 * windows of 4096 rows, so that a warp's loads of the operator are
 * contiguous; it holds a second copy of the operator's entries, padded).
 * The heuristic values until its first series, the tuned values after it. */
qsw_status qsw_op_schedule(const qsw_op* op, int32_t* csr_lanes_per_row, int32_t* csr_unroll);
/* Fix a QSW_OPERATOR_CSR operator's schedule (no tuning for it afterwards):
 * csr_lanes_per_row 1, 2, 4, 8, 16, 32 or -1 (the sliced form, built by the
 * next qsw_expmv_series), csr_unroll 2 or 4.  Pure host call.
 * Errors: INVALID_ARG (a matrix-free operator, or another value). */
qsw_status qsw_op_set_csr_schedule(qsw_op* op, int32_t csr_lanes_per_row, int32_t csr_unroll);

/* theta_m for m = 1..55 of the given precision (tol 2^-53 or 2^-24): the
 * largest theta with sum_{k>m} |c_k| theta^(k-1) <= tol, c_k the Taylor
 * coefficients of log(exp(-x) T_m(x)) (Al-Mohy & Higham, Section 3).  Pure
 * host computation; no GPU needed. */
qsw_status qsw_theta_table(int32_t precision, double* theta55);

/* Code Fragment 3.1 of Al-Mohy & Higham for the matrix t L~, from norms9 as
 * returned by qsw_op_info, n0 right-hand sides: *m_star, *s.  The same code
 * runs on the device inside qsw_expmv_series.  Pure host computation. */
qsw_status qsw_select_params(const double* norms9, double t, int32_t n0, int32_t precision,
                             int32_t* m_star, int32_t* s);

#ifdef __cplusplus
}
#endif

#endif /* QSW_H */
