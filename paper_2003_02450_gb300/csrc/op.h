// Context and operator objects behind the opaque handles of qsw.h.
#pragma once

#include <complex>
#include <functional>

#include "qsw_internal.h"

struct qsw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;   // owned: the batched small-walk kernel's stream
  cudaStream_t copy = nullptr;   // owned: device-to-host copies of finished outputs
  int* count_h = nullptr;        // owned, host-mapped: final-output counter of a series
  int* count_d = nullptr;        // its device address
  int num_sms = 0;
  int batch_cs = 0;        // qsw_batch_set_schedule: CTAs per cluster (0: tuned)
  int batch_small = -1;    // ... and the one-CTA limit in bytes (-1: tuned)
  bool batch_no_tune = false;   // use tuned schedules, never time candidates (server workers)
  std::string last_error;
};

namespace qsw {

// Device-side graph data of one walk (Section 2.1-2.5 normalisation).
struct GraphDev {
  int N = 0;        // graph vertices
  int Nt = 0;       // N~ = N + sources + sinks
  int nnz_g = 0;
  DevBuf g_rowptr, g_col, g_w;       // G (row = destination)
  DevBuf gt_rowptr, gt_col, gt_w;    // G^T (row = source)
  DevBuf hdiag;                      // [Nt] diagonal of H (0 beyond N)
  DevBuf hoff_rowptr, hoff_col, hoff_val;  // off-diagonal H, N rows
  int nnz_hoff = 0;
  std::vector<int> hlen;             // host: entries of each off-diagonal H row
  DevBuf src_v, src_r, snk_v, snk_r;       // ports
  int n_src = 0, n_snk = 0;
  // jump lists (coefficient included, omega-scaled for graph arcs)
  DevBuf j_rowptr, j_col, j_val;     // rows = destination i (for L)
  DevBuf jt_rowptr, jt_col, jt_val;  // rows = source q (for L^H)
  DevBuf dtot;                       // [Nt] total jump rate leaving each vertex
  int n_jumps = 0;                   // entries of J (= entries of J^T)
  DevBuf scratch;                    // small integer scratch
};

struct Csr {
  DevBuf rowptr, col, val;   // val: double2 (c128) or float2 (c64)
  int64_t nnz = 0;
  bool fp32 = false;
};

// The CSR operator in 32-row slices (sliced ELLPACK, SELL-32-sigma): rows
// sorted by length, longest first, within windows of kSellSigma rows; slice s
// holds rows perm[32 s .. 32 s + 31] column-major (entry k of the slice's
// lane l at off[s] + 32 k + l), each row padded to the slice's width with
// zero values (column: the row itself).  One lane per row, and a warp's
// loads of the operator stream are contiguous.
struct Sell {
  DevBuf col, val;          // [entries]: int, and the CSR's value type
  DevBuf perm;              // [32 slices]: row of each lane, -1 past n
  DevBuf off;               // [slices]: int64 offset of each slice
  DevBuf width;             // [slices]: entries per lane
  long long entries = 0;    // padded
  int slices = 0;
};

// Coefficients of the matrix-free operator (matfree.cuh), FP64 and FP32 copies.
struct MfData {
  DevBuf hval64, hval32;   // (1 - omega) H_offdiag
  DevBuf ad64, ad32;       // -dtot / 2
  DevBuf hw64, hw32;       // (1 - omega) H_vv
  DevBuf jval32, jtval32;  // jump rates (FP64 copies live in GraphDev)
  DevBuf habs;             // [Nt] sum_m |(1 - omega) H_vm|, for the exact 1-norm
  DevBuf prow;             // [64 ceil(Nt / 64)] lane order of each 64-row window
  DevBuf pwin;             // [ceil(Nt / 64)] 1 where that order pairs the rows
  DevBuf pmax;             // [ceil(Nt / 64)] longest merged part-A list of each paired window
  DevBuf paoff;            // [ceil(Nt / 64) + 1] paired windows' list offsets (in rows of 32)
  DevBuf pacol, paval64, paval32;   // their lane-interleaved merged part-A lists
  bool pa_ready = false;   // built (ensure_pair_lists) for the current values
};

// A complex matrix in CSR on the host (columns increasing within a row).
struct ZMat {
  int n = 0;
  std::vector<int> rowptr, col;
  std::vector<std::complex<double>> val;
};

// Global-interaction walk (G-QSW / NM-G-QSW): host operators and the device
// form of gqsw.cuh (rebuilt for every omega).
struct GlobalData {
  bool active = false;
  ZMat H, Hrot;               // N x N; Hrot.n == 0: no rotating Hamiltonian
  std::vector<ZMat> Ls;       // N x N Lindblad operators
  int nl = 0;                 // operators in the sandwich (0 at omega = 0)
  bool exact_norm = false;    // ||L~||_1 in closed form (one operator, no diagonal)
  long long nnz_q = 0, nnz_l = 0;
  DevBuf q_rowptr, q_col, q_val64, q_val32;       // Q
  DevBuf qh_rowptr, qh_col, qh_val64, qh_val32;   // Q^dag
  DevBuf l_rowptr[kMaxGlobalOps], l_col[kMaxGlobalOps], l_val64[kMaxGlobalOps],
      l_val32[kMaxGlobalOps];                      // L'_k = sqrt(omega) L_k
  DevBuf lh_rowptr[kMaxGlobalOps], lh_col[kMaxGlobalOps], lh_val64[kMaxGlobalOps],
      lh_val32[kMaxGlobalOps];                     // L'_k^dag
  DevBuf j_rowptr, j_col, j_val64, j_val32;       // port jumps (rows = target)
  DevBuf jt_rowptr, jt_col, jt_val64, jt_val32;   // transposed
  DevBuf cq, qdiag, cl, jout;                     // exact 1-norm ingredients
  DevBuf west;                                    // pass-A scratch of the estimator
  std::vector<int> vset_off;  // NM-G-QSW: copies of vertex v are vset_off[v] .. vset_off[v+1]-1
  DevBuf vset_dev;
};

struct Op {
  qsw_ctx* ctx = nullptr;
  int precision = QSW_C128;
  int opkind = QSW_OPERATOR_MATRIX_FREE;
  long long nnz_csr = 0;   // entries of the CSR form (closed form)
  double omega = 0.0;
  int N = 0, Nt = 0;
  int64_t n = 0;
  // host copies kept for set_omega
  std::vector<int> g_rowptr, g_col;
  std::vector<double> g_w;
  bool h_given = false;
  std::vector<int> h_rowptr, h_col;
  std::vector<double> h_w;
  std::vector<int> src_v, snk_v;
  std::vector<double> src_r, snk_r;

  GraphDev g;
  MfData mf;
  GlobalData gq;   // global-interaction walks only
  Csr L;           // the superoperator in CSR (assembled for QSW_OPERATOR_CSR or on export)
  double norms[kNormPowers] = {0};   // ||L||_1, est ||L^p||_1
  double dp[kNormPowers + 1] = {0};  // dp[0] = ||L||_1, dp[p-1] = ||L^p||^(1/p)
  DevBuf dp_dev;
  int tpr = 8;     // SpMV threads per row
  int csr_unroll = 2;       // CSR sweep: entries per lane in flight (2 or 4)
  bool tpr_fixed = false;   // set: keep tpr and csr_unroll (tuned, or QSW_BUILD_FIXED_SCHEDULE)
  bool csr_sell = false;    // the tuned CSR schedule is the sliced form (sell), not TPR lanes
  Sell sell;                // built when csr_sell (values follow set_omega: rebuilt on use)
  bool norms_ready = false;
  bool rank64 = false;      // QSW_BUILD_FP64_RANKING: the estimator's adjoint step in FP64

  // series workspace
  DevBuf kbuf, ring, jobs, ctrl, scratch;
  DevBuf scratch_w;   // global walks: pass-A products
};

// graph.cu
void build_graph(Op& op);           // uploads host graph, builds G^T, G^u, H, ports
void build_jumps(Op& op);           // J, J^T, dtot for op.omega
// assemble.cu
void assemble(Op& op, bool adjoint, Csr& out);   // L (adjoint = false) or L^H, FP64 values
void to_fp32(Op& op, Csr& m);                    // replace FP64 values by FP32
void prep_matfree(Op& op);         // MfData for op.omega
void ensure_pair_lists(Op& op);    // the interleaved part-A lists the estimator's products read
// gqsw.cu
void build_global(Op& op);                        // device form for op.omega
template <class R> struct GqOp;
template <class R> GqOp<R> make_gq(const Op& op, bool adjoint);
void gq_apply64(const Op& op, bool adjoint, int cols, const double* x, double* y, double scale);
void gq_apply_herm64(const Op& op, bool adjoint, const double* x, double* y);   // Hermitian x
bool global_exact_norm(const Op& op, double* one);
void nm_construct(int N, const int* rowptr, const int* col, const double* w, std::vector<int>& off,
                  ZMat& Hd, ZMat& Ld, ZMat& Hrot);
void nm_populations(const Op& op, const double* d_pe, int count, double* d_p);
void nm_initial_state(const Op& op, const double* d_p, double* d_state);
// norms.cu
void compute_norms(Op& op, const Csr* L, const Csr* LH);   // null: matrix-free
// series.cu
void upload_theta(int device);
// Receiver of caller outputs as they become final: the series kernel stores
// the count of final outputs in a host-mapped int (h_count / d_count, zero on
// entry) and run_series calls ready(count) while it waits for the kernel.
struct OutputSink {
  int* h_count;
  int* d_count;
  std::function<void(int)> ready;
};
void run_series(Op& op, const double* d_rho0, double t0, double dt, int steps, double* d_out,
                double* d_pops, qsw_series_stats* stats, const OutputSink* sink = nullptr);
void run_series_noalloc(Op& op, const double* d_rho0, double t0, double dt, int steps,
                        double* d_out, double* d_pops, qsw_series_stats* stats);
double probe_wait_limit(qsw_ctx* ctx);   // seconds until the bounded wait gave up
void apply(const Op& op, const double* d_x, double* d_y);
void populations(const Op& op, const double* d_rho, int count, double* d_pops);
void initial_state_from_pops(const Op& op, const double* d_pops, double* d_state);
void widen_values(const Op& op, double* d_val);
double op_bytes(const Op& op);
template <class R> struct MfOp;
template <class R> MfOp<R> make_mf(const Op& op, bool adjoint);
void mf_apply64(const Op& op, bool adjoint, int cols, const double* x, double* y, double scale);
void mf_apply32(const Op& op, bool adjoint, int cols, const float* x, float* y, double scale);
int choose_tpr(double avg_row);
void tune_csr_schedule(Op& op);  // autotuned lanes per row and unroll (cached per bucket)
void build_sell(Op& op);         // op.sell from op.L (allocates)
long long tune_measurements();   // schedule measurements made in this process
void tune_reset();               // forget every tuned schedule
// batch.cu
// Receiver of walks as they finish inside one batched call: the kernel that
// runs walk w stores 1 into the host-mapped int h_done[w] (device address
// d_done + w, zero on entry) once the walk's populations are final, and
// run_batch calls ready(w) while it waits for the kernels.
struct WalkSink {
  int* h_done;
  int* d_done;
  std::function<void(int)> ready;
};
void run_batch(qsw_ctx* ctx, int count, Op* const* ops, const double* const* d_rho0, int n0,
               const double* t0s, const double* dts, const int* steps, double* const* d_pops,
               qsw_batch_stats* stats, const WalkSink* sink = nullptr);
long long batch_tune_measurements();   // series-phase schedules measured in this process
void batch_tune_reset();               // forget every tuned series-phase schedule
// est.cu
void run_survival(Op& op, const double* d_rho0, double t_end, int q, int sink, double* eta,
                  double* d_pops, qsw_series_stats* stats);
void run_batch_survival(qsw_ctx* ctx, int count, Op* const* ops, const double* const* d_rho0,
                        const double* t_end, const int* q, const int* sink, double* eta,
                        qsw_batch_stats* stats);

inline unsigned grid_for(int64_t items, int block, int max_blocks = 1 << 20) {
  int64_t b = (items + block - 1) / block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned)b;
}

}  // namespace qsw
