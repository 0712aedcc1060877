// Expected survival time of walks with a sink (Section 4.1.4, the transport
// example): eta = integral over [0, t_end] of (1 - p_sink(t)), evaluated as the
// paper does from the series output at q + 1 equally spaced times by
// Simpson's rule,
//
//   eta = h/3 (y_0 + 4 y_1 + 2 y_2 + ... + 4 y_{q-1} + y_q),  y_k = 1 - p_sink(k h),
//
// h = t_end / q, q even.  The populations come from the series kernel (one
// walk) or the batched kernel (many walks, e.g. a sweep over omega); the rule
// is one warp per walk over its sink column, summed in a fixed order.
#include <math.h>

#include <vector>

#include "op.h"

namespace qsw {
namespace {

struct EstWalk {
  const double* pops;   // (q + 1) x N~, row k = populations at t_k
  int nt;
  int q;
  int sink;
  double h;
};

__global__ void simpson_kernel(const EstWalk* __restrict__ walks, int count,
                               double* __restrict__ eta) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= count) return;   // whole warp
  const EstWalk W = walks[w];
  double acc = 0.0;
  for (int k = lane; k <= W.q; k += 32) {
    const double c = (k == 0 || k == W.q) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
    acc = fma(c, 1.0 - W.pops[(long long)k * W.nt + W.sink], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) eta[w] = W.h / 3.0 * acc;
}

void check_est(int nt, double t_end, int q, int sink) {
  QSW_CHECK_ARG(q >= 2 && q % 2 == 0, QSW_ERR_INVALID_ARG,
                "Simpson's rule needs an even number q >= 2 of intervals");
  QSW_CHECK_ARG(isfinite(t_end) && t_end > 0.0, QSW_ERR_INVALID_ARG, "t_end must be finite and > 0");
  QSW_CHECK_ARG(sink >= 0 && sink < nt, QSW_ERR_INVALID_ARG, "sink vertex out of range");
}

// Simpson over the walks' sink columns; eta (host) receives `count` values.
void simpson_many(cudaStream_t st, const std::vector<EstWalk>& walks, double* eta) {
  const int count = (int)walks.size();
  DevBuf desc, out;
  desc.alloc(sizeof(EstWalk) * count);
  out.alloc(sizeof(double) * count);
  QSW_CUDA_TRY(cudaMemcpyAsync(desc.p, walks.data(), sizeof(EstWalk) * count,
                               cudaMemcpyHostToDevice, st));
  const int warps_per_block = 8;
  QSW_LAUNCH simpson_kernel<<<(count + warps_per_block - 1) / warps_per_block, 32 * warps_per_block,
                              0, st>>>(desc.as<EstWalk>(), count, out.as<double>());
  QSW_CUDA_TRY(cudaGetLastError());
  QSW_CUDA_TRY(cudaMemcpyAsync(eta, out.p, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));   // walks[] and eta[] are host memory
}

}  // namespace

void run_survival(Op& op, const double* d_rho0, double t_end, int q, int sink, double* eta,
                  double* d_pops, qsw_series_stats* stats) {
  check_est(op.Nt, t_end, q, sink);
  DevBuf own;
  double* pops = d_pops;
  if (!pops) {
    own.alloc(sizeof(double) * (size_t)op.Nt * ((size_t)q + 1));
    pops = own.as<double>();
  }
  const double h = t_end / q;
  run_series(op, d_rho0, 0.0, h, q, nullptr, pops, stats);
  simpson_many(op.ctx->stream, {EstWalk{pops, op.Nt, q, sink, h}}, eta);
}

void run_batch_survival(qsw_ctx* ctx, int count, Op* const* ops, const double* const* d_rho0,
                        const double* t_end, const int* q, const int* sink, double* eta,
                        qsw_batch_stats* stats) {
  std::vector<size_t> off(count + 1, 0);
  for (int w = 0; w < count; ++w) {
    check_est(ops[w]->Nt, t_end[w], q[w], sink[w]);
    off[w + 1] = off[w] + (size_t)ops[w]->Nt * ((size_t)q[w] + 1);
  }
  DevBuf pops;
  pops.alloc(sizeof(double) * off[count]);
  std::vector<double> t0(count, 0.0), dt(count);
  std::vector<double*> pp(count);
  std::vector<EstWalk> walks(count);
  for (int w = 0; w < count; ++w) {
    dt[w] = t_end[w] / q[w];
    pp[w] = pops.as<double>() + off[w];
    walks[w] = EstWalk{pp[w], ops[w]->Nt, q[w], sink[w], dt[w]};
  }
  run_batch(ctx, count, ops, d_rho0, 1, t0.data(), dt.data(), q, pp.data(), stats);
  simpson_many(ctx->stream, walks, eta);
}

}  // namespace qsw
