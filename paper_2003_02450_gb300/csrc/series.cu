// The Taylor-series engine: Algorithms 3.2 (`step`) and 5.2 (`series`) of
// Al-Mohy & Higham as used by the paper (Section 3.1), run as ONE persistent
// cooperative kernel per call.
//
// The host-independent plan (params.cuh) turns the call into a list of Taylor
// blocks.  A block with input Z, span hspan = d h and outputs k = 1..d computes
//     Khat_0 = Z,   Khat_p = (hspan / p) L Khat_{p-1},
//     F_k = Z + sum_{p=1}^{p_k} (k/d)^p Khat_p,
// which is Algorithm 5.2's  F_k = sum_p k^p K_p  with K_p = (hA)^p Z / p!
// (Khat_p = d^p K_p), and with d = 1 one stage of Algorithm 3.2.  Output k stops
// after the first p with  c1 + c2 <= tol ||F_k||_inf,  c2 = (k/d)^p ||Khat_p||_inf,
// c1 the previous term's norm (||Z||_inf at p = 1).  The powers are formed once
// per block and every active output is updated in the same pass, so the block
// costs max_k p_k applications of L~, as in the paper's `series` (Section 5:
// one time series for about the cost of one `step`).
//
// One term = one pass over the rows: the complex SpMV (TPR lanes per row,
// coalesced column/value streams, vector gathers through L2), the scaled store
// of Khat_p, the FP64 update of every active F_k, and the inf-norm partial
// maxima (warp shuffles, then one atomicMax per block).  A grid barrier with a
// bounded wait separates terms; after it every block reads the same maxima and
// takes the same stop decisions, so no host round trip is needed.
//
// Precision: VT = double2 (complex128) or float2 (complex64 bulk: FP32 matrix
// values, FP32 Taylor terms and FP32 accumulation of each product).  The F_k
// accumulators, the norms and the stop test are FP64 in both cases.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>

#include "op.h"
#include "params.cuh"

namespace qsw {

__constant__ double c_theta[2][kMMax];

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kKpl = 4;                 // outputs owned per lane
constexpr int kDMax = kKpl * 32;        // max outputs per job at TPR = 32
constexpr unsigned kSpinLimit = 1u << 24;  // bounded barrier wait (~seconds)

enum : int { kErrNone = 0, kErrBarrier = 1, kErrPlan = 2 };

struct Ctrl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int error;
  int njobs;
  unsigned long long matvecs;
  unsigned long long gmax[3][1 + kDMax];
};

struct SeriesArgs {
  int n, nt;
  const int* rowptr;
  const int* col;
  const void* val;
  void* k0;
  void* k1;
  const double2* rho0;
  double2* slots;
  int ring;              // 0: series index k -> slot k; else k % ring
  double* pops;          // (steps+1) x nt or null
  const Job* jobs;
  int njobs;
  Ctrl* ctrl;
  double tol;
};

template <class VT> struct Cplx;
template <> struct Cplx<double2> {
  using R = double;
  __device__ static double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct Cplx<float2> {
  using R = float;
  __device__ static float2 make(float a, float b) { return make_float2(a, b); }
};

__device__ __forceinline__ double2 ld_cg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }

__device__ __forceinline__ double2* slot_ptr(const SeriesArgs& a, int idx) {
  const long long s = a.ring ? (idx % a.ring) : idx;
  return a.slots + s * (long long)a.n;
}

__device__ __forceinline__ unsigned long long as_bits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ double from_bits(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// Grid barrier for a cooperative launch (all blocks co-resident).  The wait is
// bounded: on timeout the block records kErrBarrier and returns false, and so
// does every later barrier, so all blocks leave the kernel.
__device__ bool grid_barrier(Ctrl* c) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = *((volatile unsigned*)&c->bar_gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      unsigned spins = 0;
      while (*((volatile unsigned*)&c->bar_gen) == gen) {
        if (*((volatile int*)&c->error) != kErrNone || ++spins > kSpinLimit) {
          atomicCAS(&c->error, kErrNone, kErrBarrier);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (*((volatile int*)&c->error) != kErrNone) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class VT, int TPR>
__global__ void __launch_bounds__(kBlock)
series_kernel(SeriesArgs a) {
  using R = typename Cplx<VT>::R;
  __shared__ double s_red[kWarps][1 + kDMax];
  __shared__ double s_c1[kDMax];
  __shared__ double s_coef[kDMax];
  __shared__ double s_step[kDMax];
  __shared__ int s_active[kDMax];
  __shared__ int s_any;
  __shared__ double s_normk;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int glane = lane % TPR;
  constexpr int kGpw = 32 / TPR;   // row groups per warp
  const long long wglobal = ((long long)blockIdx.x * kBlock + tid) / 32;
  const long long rstride = (long long)gridDim.x * kWarps * kGpw;
  const long long gthread = (long long)blockIdx.x * kBlock + tid;
  const long long nthreads = (long long)gridDim.x * kBlock;
  Ctrl* ctrl = a.ctrl;
  const VT* __restrict__ val = static_cast<const VT*>(a.val);
  const int* __restrict__ col = a.col;
  const int* __restrict__ rowptr = a.rowptr;
  unsigned term = 0;

  for (int jb = 0; jb < a.njobs; ++jb) {
    const Job J = a.jobs[jb];
    const double2* Z = J.z_slot < 0 ? a.rho0 : slot_ptr(a, J.z_slot);
    VT* kcur = static_cast<VT*>(a.k0);
    VT* knext = static_cast<VT*>(a.k1);

    // ---- init: Khat_0 = Z, F_k = Z, ||Z||_inf
    double zmax = 0.0;
    for (long long r = gthread; r < a.n; r += nthreads) {
      const double2 z = ld_cg(Z + r);
      kcur[r] = Cplx<VT>::make((R)z.x, (R)z.y);
      for (int k = 0; k < J.d; ++k) slot_ptr(a, J.out_index0 + k)[r] = z;
      zmax = fmax(zmax, z.x * z.x + z.y * z.y);
    }
    for (int o = 16; o > 0; o >>= 1) zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    if (lane == 0) s_red[warp][0] = zmax;
    __syncthreads();
    unsigned slot3 = term % 3;
    if (tid == 0) {
      double m = 0.0;
      for (int w = 0; w < kWarps; ++w) m = fmax(m, s_red[w][0]);
      atomicMax(&ctrl->gmax[slot3][0], as_bits(m));
    }
    if (blockIdx.x == 0) {
      const unsigned nx = (term + 1) % 3;
      for (int q = tid; q <= J.d; q += kBlock) ctrl->gmax[nx][q] = 0ULL;
    }
    if (!grid_barrier(ctrl)) return;
    const double normz = sqrt(from_bits(__ldcg(&ctrl->gmax[slot3][0])));
    ++term;
    for (int k = tid; k < J.d; k += kBlock) {
      s_c1[k] = normz;
      s_coef[k] = 1.0;
      s_step[k] = (double)(k + 1) / (double)J.d;
      s_active[k] = 1;
    }
    __syncthreads();

    for (int p = 1; p <= J.m; ++p) {
      const double scale = J.hspan / p;
      const R rscale = (R)scale;
      for (int k = tid; k < J.d; k += kBlock) s_coef[k] *= s_step[k];
      __syncthreads();
      double coef[kKpl];
      int own[kKpl];
#pragma unroll
      for (int u = 0; u < kKpl; ++u) {
        const int k = glane + u * TPR;
        own[u] = (k < J.d) ? s_active[k] : 0;
        coef[u] = own[u] ? s_coef[k] : 0.0;
      }
      double kmax = 0.0;
      double fmaxv[kKpl];
#pragma unroll
      for (int u = 0; u < kKpl; ++u) fmaxv[u] = 0.0;

      // warp-uniform row loop: every lane takes part in the group shuffles
      for (long long rb = wglobal * kGpw; rb < a.n; rb += rstride) {
        const long long r = rb + lane / TPR;
        const bool valid = r < a.n;
        const int e0 = valid ? rowptr[r] : 0;
        const int e1 = valid ? rowptr[r + 1] : 0;
        R ax = 0, ay = 0;
        int e = e0 + glane;
        for (; e + TPR < e1; e += 2 * TPR) {
          const int c0 = __ldcs(col + e);
          const int c1 = __ldcs(col + e + TPR);
          const VT v0 = __ldcs(val + e);
          const VT v1 = __ldcs(val + e + TPR);
          const VT x0 = ld_cg(kcur + c0);
          const VT x1 = ld_cg(kcur + c1);
          ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
          ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
          ax = fma(v1.x, x1.x, fma(-v1.y, x1.y, ax));
          ay = fma(v1.x, x1.y, fma(v1.y, x1.x, ay));
        }
        if (e < e1) {
          const int c0 = __ldcs(col + e);
          const VT v0 = __ldcs(val + e);
          const VT x0 = ld_cg(kcur + c0);
          ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
          ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) {
          ax += __shfl_xor_sync(0xffffffffu, ax, o, TPR);
          ay += __shfl_xor_sync(0xffffffffu, ay, o, TPR);
        }
        if (!valid) continue;
        const R yx = ax * rscale, yy = ay * rscale;
        if (glane == 0) knext[r] = Cplx<VT>::make(yx, yy);
        const double dyx = (double)yx, dyy = (double)yy;
        kmax = fmax(kmax, dyx * dyx + dyy * dyy);
#pragma unroll
        for (int u = 0; u < kKpl; ++u) {
          if (own[u]) {
            double2* F = slot_ptr(a, J.out_index0 + glane + u * TPR) + r;
            double2 f = ld_cg(F);
            f.x = fma(coef[u], dyx, f.x);
            f.y = fma(coef[u], dyy, f.y);
            *F = f;
            fmaxv[u] = fmax(fmaxv[u], f.x * f.x + f.y * f.y);
          }
        }
      }
      // ---- block reduction of ||Khat_p||^2 and ||F_k||^2 partial maxima
      for (int o = 16; o > 0; o >>= 1) kmax = fmax(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
#pragma unroll
      for (int u = 0; u < kKpl; ++u)
        for (int o = TPR; o < 32; o <<= 1)
          fmaxv[u] = fmax(fmaxv[u], __shfl_xor_sync(0xffffffffu, fmaxv[u], o));
      if (lane == 0) s_red[warp][0] = kmax;
      if (lane < TPR) {
#pragma unroll
        for (int u = 0; u < kKpl; ++u) {
          const int k = lane + u * TPR;
          if (k < J.d) s_red[warp][1 + k] = fmaxv[u];
        }
      }
      __syncthreads();
      slot3 = term % 3;
      for (int q = tid; q <= J.d; q += kBlock) {
        if (q > 0 && !s_active[q - 1]) continue;
        double m = 0.0;
        for (int w = 0; w < kWarps; ++w) m = fmax(m, s_red[w][q]);
        atomicMax(&ctrl->gmax[slot3][q], as_bits(m));
      }
      if (blockIdx.x == 0) {
        const unsigned nx = (term + 1) % 3;
        for (int q = tid; q <= J.d; q += kBlock) ctrl->gmax[nx][q] = 0ULL;
        if (tid == 0) atomicAdd(&ctrl->matvecs, 1ULL);
      }
      if (!grid_barrier(ctrl)) return;
      ++term;
      if (tid == 0) {
        s_normk = sqrt(from_bits(__ldcg(&ctrl->gmax[slot3][0])));
        s_any = 0;
      }
      __syncthreads();
      // ---- stop test (identical in every block)
      for (int k = tid; k < J.d; k += kBlock) {
        if (!s_active[k]) continue;
        const double c2 = s_coef[k] * s_normk;
        const double nf = sqrt(from_bits(__ldcg(&ctrl->gmax[slot3][1 + k])));
        if (s_c1[k] + c2 <= a.tol * nf) s_active[k] = 0;
        else atomicOr(&s_any, 1);
        s_c1[k] = c2;
      }
      __syncthreads();
      VT* t = kcur;
      kcur = knext;
      knext = t;
      if (!s_any) break;
    }

    // ---- populations of the finished outputs
    if (J.final_outputs && a.pops) {
      const long long tot = (long long)J.d * a.nt;
      for (long long q = gthread; q < tot; q += nthreads) {
        const int k = (int)(q / a.nt);
        const int v = (int)(q % a.nt);
        const double2 z = ld_cg(slot_ptr(a, J.out_index0 + k) + (long long)v * (a.nt + 1));
        a.pops[(long long)(J.out_index0 + k) * a.nt + v] = z.x;
      }
      if (a.ring) {
        if (!grid_barrier(ctrl)) return;   // ring slots are reused by the next job
      }
    }
  }
}

__global__ void plan_kernel(const double* __restrict__ dp, int prec, double t0, double dt,
                            int steps, int n0, int ring, Job* jobs, int max_jobs, int expect,
                            Ctrl* ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const PlanInfo info = plan_series(dp, c_theta[prec], t0, dt, steps, n0, ring, jobs, max_jobs);
    ctrl->njobs = info.njobs;
    if (info.njobs != expect) ctrl->error = kErrPlan;
  }
}

template <class VT>
__global__ void apply_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const VT* __restrict__ val, const double2* __restrict__ x,
                             double2* __restrict__ y) {
  using R = typename Cplx<VT>::R;
  constexpr int G = 8;
  const int lane = threadIdx.x % G;
  const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const long long stride = (long long)gridDim.x * blockDim.x / G;
  for (long long rb = wg * (32 / G); rb < n; rb += stride) {
    const long long r = rb + (threadIdx.x % 32) / G;
    const bool valid = r < n;
    const int e0 = valid ? rowptr[r] : 0, e1 = valid ? rowptr[r + 1] : 0;
    R ax = 0, ay = 0;
    for (int e = e0 + lane; e < e1; e += G) {
      const VT v = val[e];
      const double2 xd = x[col[e]];
      const R xx = (R)xd.x, xy = (R)xd.y;
      ax = fma(v.x, xx, fma(-v.y, xy, ax));
      ay = fma(v.x, xy, fma(v.y, xx, ay));
    }
    for (int o = G / 2; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o, G);
      ay += __shfl_xor_sync(0xffffffffu, ay, o, G);
    }
    if (valid && lane == 0) y[r] = make_double2((double)ax, (double)ay);
  }
}

__global__ void pops_kernel(int count, int nt, long long n, const double2* __restrict__ rho,
                            double* __restrict__ pops) {
  const long long tot = (long long)count * nt;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = q / nt;
    const long long v = q % nt;
    pops[q] = rho[c * n + v * (nt + 1)].x;
  }
}

__global__ void widen_kernel(long long nnz, const float2* __restrict__ in, double2* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 v = in[e];
    out[e] = make_double2((double)v.x, (double)v.y);
  }
}

__global__ void diag_state_kernel(int nt, long long n, const double* __restrict__ p,
                                  double2* __restrict__ state) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q % nt, j = q / nt;
    state[q] = make_double2(i == j ? p[i] : 0.0, 0.0);
  }
}

template <class VT, int TPR>
cudaError_t launch_series(const SeriesArgs& a, int sms, cudaStream_t st, int* grid_out) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, series_kernel<VT, TPR>,
                                                                kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  long long want = ((long long)a.n * TPR + kBlock - 1) / kBlock;
  long long maxg = (long long)per_sm * sms;
  int grid = (int)std::max<long long>(1, std::min(want, maxg));
  *grid_out = grid;
  SeriesArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)series_kernel<VT, TPR>, dim3(grid), dim3(kBlock),
                                     params, 0, st);
}

template <class VT>
cudaError_t launch_series_tpr(int tpr, const SeriesArgs& a, int sms, cudaStream_t st, int* g) {
  switch (tpr) {
    case 4: return launch_series<VT, 4>(a, sms, st, g);
    case 8: return launch_series<VT, 8>(a, sms, st, g);
    case 16: return launch_series<VT, 16>(a, sms, st, g);
    default: return launch_series<VT, 32>(a, sms, st, g);
  }
}

}  // namespace

int choose_tpr(double avg_row) {
  if (avg_row <= 12) return 4;
  if (avg_row <= 24) return 8;
  if (avg_row <= 56) return 16;
  return 32;
}

void upload_theta(int device) {
  (void)device;
  QSW_CUDA_TRY(cudaMemcpyToSymbol(c_theta, theta_table(QSW_C128), sizeof(double) * kMMax, 0));
  QSW_CUDA_TRY(cudaMemcpyToSymbol(c_theta, theta_table(QSW_C64_BULK), sizeof(double) * kMMax,
                                  sizeof(double) * kMMax));
}

void run_series(Op& op, const double* d_rho0, double t0, double dt, int steps, double* d_out,
                double* d_pops, qsw_series_stats* stats) {
  cudaStream_t st = op.ctx->stream;
  const int prec = op.precision == QSW_C64_BULK ? 1 : 0;
  const double* theta = theta_table(op.precision);
  // Host copy of the plan: sizes only (the device plans for itself below).
  const PlanInfo info = plan_series(op.dp, theta, t0, dt, steps, 1, 0, nullptr, 0);
  QSW_CHECK_ARG(info.max_d <= kDMax, QSW_ERR_INVALID_ARG,
                "more than " + std::to_string(kDMax) + " outputs per Taylor block (steps/s too large)");
  int tpr = op.tpr;
  while (tpr < 32 && kKpl * tpr < info.max_d) tpr *= 2;
  const int ring = d_out ? 0 : info.max_d + 1;
  const size_t vbytes = op.precision == QSW_C64_BULK ? sizeof(float2) : sizeof(double2);
  op.kbuf.alloc(2 * vbytes * (size_t)op.n);
  if (!d_out) op.ring.alloc(sizeof(double2) * (size_t)op.n * ring);
  op.jobs.alloc(sizeof(Job) * std::max(1, info.njobs));
  op.ctrl.alloc(sizeof(Ctrl));
  QSW_CUDA_TRY(cudaMemsetAsync(op.ctrl.p, 0, sizeof(Ctrl), st));
  plan_kernel<<<1, 32, 0, st>>>(op.dp_dev.as<double>(), prec, t0, dt, steps, 1, ring,
                                op.jobs.as<Job>(), info.njobs, info.njobs, op.ctrl.as<Ctrl>());
  QSW_CUDA_TRY(cudaGetLastError());

  SeriesArgs a{};
  a.n = (int)op.n;
  a.nt = op.Nt;
  a.rowptr = op.L.rowptr.as<int>();
  a.col = op.L.col.as<int>();
  a.val = op.L.val.p;
  a.k0 = op.kbuf.p;
  a.k1 = static_cast<char*>(op.kbuf.p) + vbytes * (size_t)op.n;
  a.rho0 = reinterpret_cast<const double2*>(d_rho0);
  a.slots = d_out ? reinterpret_cast<double2*>(d_out) : op.ring.as<double2>();
  a.ring = ring;
  a.pops = d_pops;
  a.jobs = op.jobs.as<Job>();
  a.njobs = info.njobs;
  a.ctrl = op.ctrl.as<Ctrl>();
  a.tol = tolerance(op.precision);

  cudaEvent_t ev0, ev1;
  QSW_CUDA_TRY(cudaEventCreate(&ev0));
  QSW_CUDA_TRY(cudaEventCreate(&ev1));
  QSW_CUDA_TRY(cudaEventRecord(ev0, st));
  int grid = 0;
  cudaError_t e = op.precision == QSW_C64_BULK
                      ? launch_series_tpr<float2>(tpr, a, op.ctx->num_sms, st, &grid)
                      : launch_series_tpr<double2>(tpr, a, op.ctx->num_sms, st, &grid);
  QSW_CUDA_TRY(e);
  QSW_CUDA_TRY(cudaEventRecord(ev1, st));
  Ctrl h{};
  QSW_CUDA_TRY(cudaMemcpyAsync(&h, op.ctrl.p, offsetof(Ctrl, gmax), cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (h.error == kErrBarrier)
    throw Error{QSW_ERR_NOT_CONVERGED, "series kernel: grid barrier wait exceeded its limit"};
  if (h.error == kErrPlan)
    throw Error{QSW_ERR_CUDA, "series kernel: device plan differs from host plan"};
  if (stats) {
    stats->m0 = info.m0;
    stats->s0 = info.s0;
    stats->m_star = info.m_star;
    stats->s = info.s;
    stats->step_m = info.step_m;
    stats->step_s = info.step_s;
    stats->outputs_per_block = info.d;
    stats->jobs = info.njobs;
    stats->matvecs = (int64_t)h.matvecs;
    stats->bytes_per_matvec = (double)op.L.nnz * (vbytes + 4) + (double)(op.n + 1) * 4 +
                              2.0 * (double)op.n * vbytes;
    stats->kernel_ms = ms;
  }
}

void apply(const Op& op, const double* d_x, double* d_y) {
  cudaStream_t st = op.ctx->stream;
  const int n = (int)op.n;
  const unsigned grid = grid_for((long long)n * 8, 256, 152 * 16);
  if (op.L.fp32)
    apply_kernel<float2><<<grid, 256, 0, st>>>(n, op.L.rowptr.as<int>(), op.L.col.as<int>(),
                                               op.L.val.as<float2>(),
                                               reinterpret_cast<const double2*>(d_x),
                                               reinterpret_cast<double2*>(d_y));
  else
    apply_kernel<double2><<<grid, 256, 0, st>>>(n, op.L.rowptr.as<int>(), op.L.col.as<int>(),
                                                op.L.val.as<double2>(),
                                                reinterpret_cast<const double2*>(d_x),
                                                reinterpret_cast<double2*>(d_y));
  QSW_CUDA_TRY(cudaGetLastError());
}

void populations(const Op& op, const double* d_rho, int count, double* d_pops) {
  cudaStream_t st = op.ctx->stream;
  pops_kernel<<<grid_for((long long)count * op.Nt, 256, 4096), 256, 0, st>>>(
      count, op.Nt, op.n, reinterpret_cast<const double2*>(d_rho), d_pops);
  QSW_CUDA_TRY(cudaGetLastError());
}

void widen_values(const Op& op, double* d_val) {
  widen_kernel<<<grid_for(op.L.nnz, 256, 4096), 256, 0, op.ctx->stream>>>(
      op.L.nnz, op.L.val.as<float2>(), reinterpret_cast<double2*>(d_val));
  QSW_CUDA_TRY(cudaGetLastError());
}

void initial_state_from_pops(const Op& op, const double* d_pops, double* d_state) {
  cudaStream_t st = op.ctx->stream;
  diag_state_kernel<<<grid_for(op.n, 256, 4096), 256, 0, st>>>(
      op.Nt, op.n, d_pops, reinterpret_cast<double2*>(d_state));
  QSW_CUDA_TRY(cudaGetLastError());
}

}  // namespace qsw
