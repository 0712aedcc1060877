// Batched L-QSW series: many independent walks of uneven size in one launch.
//
// Each walk is handled by one thread-block cluster (kCl CTAs in phase 1; in
// phase 2 the cluster size of the tuned schedule, 4, 8 or 16); clusters take
// walks from a queue ordered by decreasing size (largest first), so big and
// small walks pack onto the GPU together.  Inside a cluster every pass over the
// walk's elements is split over the cluster's warps, and passes are separated
// by hardware cluster barriers (barrier.cluster: no spin loop).  Reductions go
// through distributed shared memory: each CTA reduces its part, then every CTA
// reads the cluster's partials in rank order, so all CTAs hold the same value
// and take the same decisions.
//
// Phase 1 (norms): the exact ||L||_1 and, only when Code Fragment 3.1 needs
// them for the walk's time span (condition (3.13) fails), the Higham--Tisseur
// estimates of ||L^p||_1, p = 2..9 -- the same algorithm as norms.cu, with its
// branches taken on the device.
// Phase 2 (series): the walk's plan (params.cuh) and its Taylor blocks on a
// block of n0 <= 4 right-hand sides (A-H treat B = [b_1 .. b_n0] as one matrix:
// ||B||_inf is the largest row sum of moduli), populations of every output.
// Hermitian right-hand sides are computed on upper triangles as in series.cu.
//
// Small walks (their two Taylor-term blocks fit in the schedule's one-CTA
// limit, at most 64 KB) take phase 2 on ONE CTA instead, with the Taylor terms in shared memory: for such walks each term
// is a few hundred nanoseconds of work, and a cluster's barriers and its
// gathers of terms written by other SMs (L2 round trips) would dominate.  The
// small-walk kernel runs on a second stream alongside the cluster kernel.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <chrono>
#include <type_traits>

#include "matfree.cuh"
#include "op.h"
#include "params.cuh"

namespace cg = cooperative_groups;

namespace qsw {

// theta tables for this translation unit (uploaded with the series tables)
__constant__ double c_theta_b[2][kMMax];

void upload_theta_batch() {
  QSW_CUDA_TRY(cudaMemcpyToSymbol(c_theta_b, theta_table(QSW_C128), sizeof(double) * kMMax, 0));
  QSW_CUDA_TRY(cudaMemcpyToSymbol(c_theta_b, theta_table(QSW_C64_BULK), sizeof(double) * kMMax,
                                  sizeof(double) * kMMax));
}

namespace {

constexpr int kCl = 8;        // CTAs per cluster
constexpr int kBT = 256;      // threads per CTA
constexpr int kBW = kBT / 32;
constexpr int kMaxRhs = 4;
constexpr int kItMax = 5;
constexpr int kMaxHist = 2 * (kItMax + 1);
constexpr int kBDMax = 64;    // outputs per Taylor job in the batched kernel (larger
                              // blocks are split into jobs that recompute the powers)
constexpr unsigned long long kSeed = 0x51535700ULL;

struct BWalk {
  MfOp<double> mf64;   // L
  MfOp<double> mfh64;  // L^H
  MfOp<float> mf32;    // L, FP32 coefficients
  int Nt;
  long long n;
  int n0;
  int f32;             // complex64 bulk
  int herm;            // every right-hand side Hermitian
  const double2* rho0; // n0 x n
  double* pops;        // (steps+1) x n0 x Nt
  double t0, dt;
  int steps;
  double norm_span;    // max(t0, steps dt): decides whether estimates are needed
  // phase 1 outputs / phase 2 inputs
  double* dp;          // [kNormPowers + 1]
  double2* est;        // phase 1 workspace: X, Y, W (2 n each), h (n doubles)
  // phase 2 workspace
  void* kbuf;          // 2 x n0 x n of VT
  double2* fring;      // ring x n0 x n
  int ring;
  int fsmem;           // small walks: the ring lives in shared memory after the terms
  Job* jobs;
  int njobs;
  long long* counters; // [0] matvecs, [1] fupdates, [2] plan mismatch
  int* done;           // host-mapped completion flag, or null
};

struct BArgs {
  BWalk* walks;
  const int* order;    // phase 1: every walk, largest first
  int count;
  const int* big;      // phase 2 on clusters: walks too large for one CTA, largest first
  int nbig;
  const int* small;    // phase 2 on one CTA each, largest first
  int nsmall;
  unsigned int* queue; // [0] phase 1, [1] cluster phase 2, [2] small-walk phase 2
  double tol[2];
};

constexpr size_t kSmallTotalBytes = 96 * 1024;   // a small walk's two Taylor-term blocks plus
                                                 // its output ring, when both fit on chip

__device__ __forceinline__ unsigned long long bits_of(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ double of_bits(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long i) {
  unsigned long long z = seed + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// --------------------------------------------------------- cluster reductions
struct Red {
  double v[kBW][2];
  int idx[kBW][2];
  double blk[2];
  int blki[2];
  double out[2];
  int outi[2];
};

// The CTAs that share one walk in phase 2: a thread-block cluster (hardware
// barrier, partial results read through distributed shared memory) or one CTA.
struct ClusterG {
  cg::cluster_group cl;
  int sz;   // CTAs in the cluster (phase 1: kCl; phase 2: the launch's cluster size)
  __device__ int size() const { return sz; }
  __device__ int rank() const { return (int)cl.block_rank(); }
  __device__ void sync() { cl.sync(); }
  __device__ const Red* peer(Red& R, int r) { return cl.map_shared_rank(&R, r); }
};
struct CtaG {
  __device__ int size() const { return 1; }
  __device__ int rank() const { return 0; }
  __device__ void sync() { __syncthreads(); }
  __device__ const Red* peer(Red& R, int) { return &R; }
};

__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
  if (ib < 0) return ia >= 0;
  if (ia < 0) return false;
  return va > vb || (va == vb && ia < ib);
}

// Sum of (a, b) over the cluster, fixed order (deterministic).
__device__ void cl_sum2(cg::cluster_group& cl, Red& R, double a, double b, double& oa, double& ob) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) { R.v[warp][0] = a; R.v[warp][1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < kBW; ++w) { s0 += R.v[w][0]; s1 += R.v[w][1]; }
    R.blk[0] = s0;
    R.blk[1] = s1;
  }
  cl.sync();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int r = 0; r < kCl; ++r) {
      const Red* p = cl.map_shared_rank(&R, r);
      s0 += p->blk[0];
      s1 += p->blk[1];
    }
    R.out[0] = s0;
    R.out[1] = s1;
  }
  cl.sync();
  oa = R.out[0];
  ob = R.out[1];
}

// Max of two non-negative values over the group's CTAs.  Non-negative doubles
// order like their bit patterns, so the maxima are integer operations (the
// FP64 pipe is 1/64 of FP32 on this part and is kept for the arithmetic).
__device__ __forceinline__ double dmax_bits(double a, double b) {
  return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}

template <class G>
__device__ void grp_max2(G& g, Red& R, double a, double b, double& oa, double& ob) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a = dmax_bits(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = dmax_bits(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if (lane == 0) { R.v[warp][0] = a; R.v[warp][1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < kBW; ++w) { s0 = dmax_bits(s0, R.v[w][0]); s1 = dmax_bits(s1, R.v[w][1]); }
    R.blk[0] = s0;
    R.blk[1] = s1;
  }
  g.sync();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int r = 0; r < g.size(); ++r) {
      const Red* p = g.peer(R, r);
      s0 = dmax_bits(s0, p->blk[0]);
      s1 = dmax_bits(s1, p->blk[1]);
    }
    R.out[0] = s0;
    R.out[1] = s1;
  }
  g.sync();
  oa = R.out[0];
  ob = R.out[1];
}

__device__ __forceinline__ void cl_max2(cg::cluster_group& cl, Red& R, double a, double b,
                                        double& oa, double& ob) {
  ClusterG g{cl, kCl};
  grp_max2(g, R, a, b, oa, ob);
}

// argmax over the cluster: larger value first, ties to the smaller index.
__device__ void cl_argmax(cg::cluster_group& cl, Red& R, double v, int i, double& ov, int& oi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(v2, i2, v, i)) { v = v2; i = i2; }
  }
  if (lane == 0) { R.v[warp][0] = v; R.idx[warp][0] = i; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = 0;
    int bi = -1;
    for (int w = 0; w < kBW; ++w)
      if (better(R.v[w][0], R.idx[w][0], bv, bi)) { bv = R.v[w][0]; bi = R.idx[w][0]; }
    R.blk[0] = bv;
    R.blki[0] = bi;
  }
  cl.sync();
  if (threadIdx.x == 0) {
    double bv = 0;
    int bi = -1;
    for (int r = 0; r < kCl; ++r) {
      const Red* p = cl.map_shared_rank(&R, r);
      if (better(p->blk[0], p->blki[0], bv, bi)) { bv = p->blk[0]; bi = p->blki[0]; }
    }
    R.out[0] = bv;
    R.outi[0] = bi;
  }
  cl.sync();
  ov = R.out[0];
  oi = R.outi[0];
}

// Next walk from the queue (cluster rank 0 takes it, everyone reads it).
__device__ int next_walk(cg::cluster_group& cl, unsigned int* counter, int* s_w,
                          const int* list, int count) {
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    const unsigned k = atomicAdd(counter, 1u);
    *s_w = k < (unsigned)count ? list[k] : -1;
  }
  cl.sync();
  const int w = *cl.map_shared_rank(s_w, 0);
  cl.sync();
  return w;
}

// y_c = scale * M x_c for `cols` vectors (general elements), FP64, over the
// cluster's warps; M = L or L^H.
template <bool ADJ>
__device__ void cl_apply64(const MfOp<double>& op, int cols, const double2* x, double2* y,
                           long long n) {
  const int gw = (int)(cg::this_cluster().block_rank() * kBW + (threadIdx.x >> 5));
  const int lane = threadIdx.x & 31;
  const long long nitems = mf_item_count(op.Nt, false);
  for (long long k = gw; k < nitems; k += kCl * kBW) {
    int j, i0;
    mf_item(k, op.Nt, false, j, i0);
    int irow[2];
    for (int u = 0; u < 2; ++u) {
      const int i = i0 + lane + 32 * u;
      irow[u] = i < op.Nt ? i : -1;
    }
    for (int c = 0; c < cols; ++c) {
      const double2* xc = x + c * n;
      double cx[2], cy[2];
      mf_partB<double, double2, 2>(op, xc, j, irow, cx, cy);
      for (int u = 0; u < 2; ++u) {
        if (irow[u] < 0) continue;
        double yx, yy;
        mf_finish<double, double2, ADJ>(op, xc, irow[u], j, cx[u], cy[u], yx, yy);
        y[c * n + irow[u] + (long long)op.Nt * j] = make_double2(yx, yy);
      }
    }
  }
}

// --------------------------------------------------------------- phase 1
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kBT)
batch_norms_kernel(BArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ Red R;
  __shared__ int s_w;
  const int crank = (int)cl.block_rank();
  const long long ct = (long long)crank * kBT + threadIdx.x;   // thread index in the cluster
  const long long cstride = (long long)kCl * kBT;
  for (;;) {
    const int wi = next_walk(cl, &a.queue[0], &s_w, a.order, a.count);
    if (wi < 0) break;
    BWalk& W = a.walks[wi];
    const int Nt = W.Nt;
    const long long n = W.n;
    const MfOp<double>& L = W.mf64;
    // exact ||L||_1: column (i, j) sums |c| over H rows i and j, |D_ij|, and
    // the rates leaving i when i = j (= dtot_i = -2 ad_i)
    double best = 0.0;
    for (long long r = ct; r < n; r += cstride) {
      const int i = (int)(r % Nt), j = (int)(r / Nt);
      double s = 0.0;
      if (i < L.N) for (int e = L.hrow[i]; e < L.hrow[i + 1]; ++e) s += fabs(L.hval[e]);
      if (j < L.N) for (int e = L.hrow[j]; e < L.hrow[j + 1]; ++e) s += fabs(L.hval[e]);
      s += hypot(L.ad[i] + L.ad[j], L.hw[j] - L.hw[i]);
      if (i == j) s += -2.0 * L.ad[i];
      best = fmax(best, s);
    }
    double one, dummy;
    cl_max2(cl, R, best, 0.0, one, dummy);
    double norms[kNormPowers] = {0};
    norms[0] = one;
    const int prec = W.f32 ? 1 : 0;
    const bool need = one > 0.0 &&
                      !small_norm_condition(W.norm_span * one, c_theta_b[prec], W.n0);
    if (need) {
      // Higham--Tisseur Algorithm 2.4 for A^p, p = 2..9 (t = 2 columns)
      double2* X = W.est;
      double2* Y = X + 2 * n;
      double2* Wb = Y + 2 * n;
      double* h = reinterpret_cast<double*>(Wb + 2 * n);
      const int t = n >= 2 ? 2 : 1;
      for (int p = 2; p <= kNormPowers; ++p) {
        // X = [1, +-1] / n
        for (long long r = ct; r < n; r += cstride) {
          X[r] = make_double2(1.0 / n, 0.0);
          if (t > 1) {   // signs symmetric under the transposed index (a Hermitian column)
            const long long rt = (r / Nt) + (long long)Nt * (r % Nt);
            const bool neg = (splitmix64(kSeed, (unsigned long long)(rt < r ? rt : r)) >> 63) != 0;
            X[n + r] = make_double2(neg ? -1.0 / n : 1.0 / n, 0.0);
          }
        }
        cl.sync();
        int hist[kMaxHist];
        int nhist = 0;
        double est_old = 0.0, est = 0.0;
        int ind[2] = {0, 0};
        int ind_best = 0;
        for (int k = 1;; ++k) {
          // Y = A^p X (ping-pong through Wb)
          const double2* src = X;
          for (int q = 0; q < p; ++q) {
            double2* dst = ((p - q) % 2 == 1) ? Y : Wb;
            cl_apply64<false>(L, t, src, dst, n);
            cl.sync();
            src = dst;
          }
          double c0 = 0, c1 = 0;
          for (long long r = ct; r < n; r += cstride) {
            const double2 y0 = __ldcg(Y + r);
            c0 += hypot(y0.x, y0.y);
            if (t > 1) {
              const double2 y1 = __ldcg(Y + n + r);
              c1 += hypot(y1.x, y1.y);
            }
          }
          double cn0, cn1;
          cl_sum2(cl, R, c0, c1, cn0, cn1);
          const int jbest = (t > 1 && cn1 > cn0) ? 1 : 0;
          est = jbest ? cn1 : cn0;
          if (est > est_old || k == 2) ind_best = ind[jbest];
          if (k >= 2 && est <= est_old) { est = est_old; break; }
          est_old = est;
          if (k > kItMax) break;
          // S = sign(Y) into X, Z = (A^H)^p S into Y
          for (long long r = ct; r < (long long)t * n; r += cstride) {
            const double2 y = __ldcg(Y + r);
            const double m = hypot(y.x, y.y);
            X[r] = m == 0.0 ? make_double2(1.0, 0.0) : make_double2(y.x / m, y.y / m);
          }
          cl.sync();
          src = X;
          for (int q = 0; q < p; ++q) {
            double2* dst = ((p - q) % 2 == 1) ? Y : Wb;
            cl_apply64<true>(W.mfh64, t, src, dst, n);
            cl.sync();
            src = dst;
          }
          // h_i = max_c |Z_ic|, argmax (ties to the smaller index)
          double bv = 0;
          int bi = -1;
          for (long long r = ct; r < n; r += cstride) {
            const double2 z0 = __ldcg(Y + r);
            double v = hypot(z0.x, z0.y);
            if (t > 1) {
              const double2 z1 = __ldcg(Y + n + r);
              v = fmax(v, hypot(z1.x, z1.y));
            }
            h[r] = v;
            if (better(v, (int)r, bv, bi)) { bv = v; bi = (int)r; }
          }
          double hmax;
          int imax;
          cl_argmax(cl, R, bv, bi, hmax, imax);   // (syncs make h visible)
          if (k >= 2 && hmax == __ldcg(h + ind_best)) break;
          // top-2 overall, then the first t indices not used before
          auto argmax_excl = [&](const int* ex, int nex, double& ov, int& oi) {
            double v2 = 0;
            int i2 = -1;
            for (long long r = ct; r < n; r += cstride) {
              bool skip = false;
              for (int q = 0; q < nex; ++q) skip |= ex[q] == (int)r;
              if (skip) continue;
              if (better(h[r], (int)r, v2, i2)) { v2 = h[r]; i2 = (int)r; }
            }
            cl_argmax(cl, R, v2, i2, ov, oi);
          };
          int fresh[2] = {imax, -1};
          if (t > 1) {
            double v2;
            int i2;
            argmax_excl(&imax, 1, v2, i2);
            bool in0 = false, in1 = false;
            for (int q = 0; q < nhist; ++q) { in0 |= hist[q] == imax; in1 |= hist[q] == i2; }
            if (in0 && in1) break;
            int ex[kMaxHist + 1];
            for (int q = 0; q < nhist; ++q) ex[q] = hist[q];
            double fv;
            argmax_excl(ex, nhist, fv, fresh[0]);
            ex[nhist] = fresh[0];
            argmax_excl(ex, nhist + 1, fv, fresh[1]);
            if (fresh[0] < 0 || fresh[1] < 0) break;
          }
          ind[0] = fresh[0];
          ind[1] = fresh[1];
          for (long long r = ct; r < (long long)t * n; r += cstride) X[r] = make_double2(0.0, 0.0);
          cl.sync();
          if (crank == 0 && threadIdx.x == 0) {
            X[ind[0]] = make_double2(1.0, 0.0);
            if (t > 1) X[n + ind[1]] = make_double2(1.0, 0.0);
          }
          cl.sync();
          if (nhist + t <= kMaxHist) {
            hist[nhist++] = ind[0];
            if (t > 1) hist[nhist++] = ind[1];
          }
        }
        norms[p - 1] = est;
      }
    }
    if (crank == 0 && threadIdx.x == 0) {
      W.dp[0] = norms[0];
      for (int p = 2; p <= kNormPowers; ++p) W.dp[p - 1] = need ? pow(norms[p - 1], 1.0 / p) : 0.0;
      W.dp[kNormPowers] = 0.0;
    }
    cl.sync();
  }
}

// --------------------------------------------------------------- phase 2
template <class VT> struct BC;
template <> struct BC<double2> {
  using R = double;
  __device__ static double2 mk(double a, double b) { return make_double2(a, b); }
  __device__ static const MfOp<double>& mf(const BWalk& w) { return w.mf64; }
};
template <> struct BC<float2> {
  using R = float;
  __device__ static float2 mk(float a, float b) { return make_float2(a, b); }
  __device__ static const MfOp<float>& mf(const BWalk& w) { return w.mf32; }
};

// Truncating double -> float with integer operations only (no FP64 pipe
// instruction); exact to 2^-23 relative, tiny values flush to zero.  Used for
// the norms of the complex64-bulk stop test, whose tolerance is 2^-24.
__device__ __forceinline__ float f32_trunc(double v) {
  const long long b = __double_as_longlong(v);
  const int hi = (int)(b >> 32);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  const int m = (int)((b >> 29) & 0x7fffff);
  const int bits = (hi & (int)0x80000000) | (e << 23) | m;
  return e <= 0 ? 0.0f : __int_as_float(e >= 255 ? ((hi & (int)0x80000000) | 0x7f800000) : bits);
}

// |z| contribution of one entry to a row sum (n0 > 1) or |z|^2 (n0 = 1), in
// the precision the stop test needs: FP32 for complex64 bulk, FP64 otherwise.
template <bool F32, int N0> struct NormAcc;
template <int N0> struct NormAcc<true, N0> {
  using T = float;
  __device__ static float of(double x, double y) {
    const float a = f32_trunc(x), b = f32_trunc(y);
    return N0 == 1 ? a * a + b * b : sqrtf(a * a + b * b);
  }
  __device__ static float of_f(float a, float b) { return N0 == 1 ? a * a + b * b : sqrtf(a * a + b * b); }
  __device__ static float vmax(float a, float b) {   // non-negative: integer compare
    return __int_as_float(max(__float_as_int(a), __float_as_int(b)));
  }
};
template <int N0> struct NormAcc<false, N0> {
  using T = double;
  __device__ static double of(double x, double y) {
    return N0 == 1 ? x * x + y * y : sqrt(x * x + y * y);
  }
  __device__ static double of_f(double a, double b) { return of(a, b); }
  __device__ static double vmax(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
  }
};

constexpr int kBKReg = 4;   // outputs whose running maxima live in registers

// Reads of the output ring and of Z: global-memory reads that bypass L1 on a
// cluster (other CTAs wrote them), generic reads in one-CTA mode (the ring may
// be in shared memory; in global memory this CTA wrote it itself).
template <bool SK> __device__ __forceinline__ double2 ldf(const double2* p) {
  if (SK) return *p;
  return __ldcg(p);
}

// All n0 right-hand sides of a walk in one pass over the operator's lists
// (an SpMM): part B of C for the two rows of a lane, then part A, the
// diagonal and the jumps for one row, every column at once, so the gathers
// of the n0 columns are in flight together.  Per (row, column) the terms are
// added in the same order as mf_partB / mf_finish / mf_tail.
template <class R, class VT, int N0, class LD>
__device__ __forceinline__ void bmf_partB(const MfOp<R>& op, const VT* __restrict__ x, long long n,
                                          int j, const int* irow, R (*cx)[N0], R (*cy)[N0]) {
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int c = 0; c < N0; ++c) { cx[u][c] = 0; cy[u][c] = 0; }
  if (j >= op.N) return;
  const int e0 = op.hrow[j], e1 = op.hrow[j + 1];
  for (int e = e0; e < e1; ++e) {
    const long long off = (long long)op.Nt * op.hcol[e];
    const R h = op.hval[e];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (irow[u] < 0) continue;
      VT v[N0];
#pragma unroll
      for (int c = 0; c < N0; ++c) v[c] = LD::ld(x + c * n + off + irow[u]);
#pragma unroll
      for (int c = 0; c < N0; ++c) {
        cx[u][c] = fma(-h, v[c].x, cx[u][c]);
        cy[u][c] = fma(-h, v[c].y, cy[u][c]);
      }
    }
  }
}

template <class R, class VT, int N0, class LD>
__device__ __forceinline__ void bmf_finish(const MfOp<R>& op, const VT* __restrict__ x, long long n,
                                           int i, int j, R* cx, R* cy) {
  const long long base = (long long)op.Nt * j;
  if (i < op.N) {
    const int e0 = op.hrow[i], e1 = op.hrow[i + 1];
    for (int e = e0; e < e1; ++e) {
      const long long a = base + op.hcol[e];
      const R h = op.hval[e];
      VT v[N0];
#pragma unroll
      for (int c = 0; c < N0; ++c) v[c] = LD::ld(x + c * n + a);
#pragma unroll
      for (int c = 0; c < N0; ++c) {
        cx[c] = fma(h, v[c].x, cx[c]);
        cy[c] = fma(h, v[c].y, cy[c]);
      }
    }
  }
  VT xs[N0];
#pragma unroll
  for (int c = 0; c < N0; ++c) xs[c] = LD::ld(x + c * n + base + i);
  const R dx = op.ad[i] + op.ad[j];
  const R dy = op.hw[j] - op.hw[i];
#pragma unroll
  for (int c = 0; c < N0; ++c) {   // -i C + D x
    const R rx = fma(dx, xs[c].x, fma(-dy, xs[c].y, cy[c]));
    const R ry = fma(dx, xs[c].y, fma(dy, xs[c].x, -cx[c]));
    cx[c] = rx;
    cy[c] = ry;
  }
  if (i == j) {
    const int e0 = op.jrow[i], e1 = op.jrow[i + 1];
    for (int e = e0; e < e1; ++e) {
      const long long a = (long long)op.jcol[e] * (op.Nt + 1);
      const R r = op.jval[e];
#pragma unroll
      for (int c = 0; c < N0; ++c) {
        const VT v = LD::ld(x + c * n + a);
        cx[c] = fma(r, v.x, cx[c]);
        cy[c] = fma(r, v.y, cy[c]);
      }
    }
  }
}

// Phase 2 of one walk on group g.  SK: the Taylor-term blocks live in shared
// memory at `sk` (one-CTA groups); otherwise in the walk's workspace.
template <class G, class VT, int N0, bool SK>
__device__ __noinline__ void run_walk(G g, Red& R, const BWalk& W, double tol, double* s_coef,
                                      double* s_step, double* s_c1, int* s_active, VT* sk) {
  using Rt = typename BC<VT>::R;
  constexpr bool kF32 = sizeof(Rt) == sizeof(float);
  using NA = NormAcc<kF32, N0>;
  using NT = typename NA::T;
  using LDP = typename std::conditional<SK, LdGeneric, LdGlobal>::type;
  const int crank = g.rank();
  const long long ct = (long long)crank * kBT + threadIdx.x;
  const long long cstride = (long long)g.size() * kBT;
  const int Nt = W.Nt;
  const long long n = W.n;
  const bool herm = W.herm != 0;
  const MfOp<Rt>& op = BC<VT>::mf(W);
  const int lane = threadIdx.x & 31;
  const int gw = crank * kBW + (threadIdx.x >> 5);
  // outputs: the walk's ring in global memory, or (small walks whose ring fits)
  // in shared memory right after the two Taylor-term blocks
  double2* const fring =
      (SK && W.fsmem) ? reinterpret_cast<double2*>(sk + 2 * (long long)N0 * n) : W.fring;
  const int ring = W.ring;
  auto fslot = [&](int idx) { return fring + (long long)(idx % ring) * N0 * n; };
  // per-block maxima of outputs k >= kBKReg (shared, as bit patterns)
  unsigned long long* s_extra = reinterpret_cast<unsigned long long*>(s_c1 + kBDMax);
  long long matvecs = 0, fupd = 0;

  for (int jb = 0; jb < W.njobs; ++jb) {
    const Job J = W.jobs[jb];
    const double2* Z = J.z_slot < 0 ? W.rho0 : fslot(J.z_slot);
    VT* kc = SK ? sk : static_cast<VT*>(W.kbuf);
    VT* kn = kc + (long long)N0 * n;
    // init: Khat_0 = Z, F_k = Z, ||Z||_inf
    NT zn = 0;
    for (long long r = ct; r < n; r += cstride) {
      const int i = (int)(r % Nt), j = (int)(r / Nt);
      NT rs = 0;
#pragma unroll
      for (int c = 0; c < N0; ++c) {
        double2 z;
        if (herm && i > j) {
          z = ldf<SK>(Z + c * n + j + (long long)Nt * i);
          z.y = -z.y;
        } else {
          z = ldf<SK>(Z + c * n + r);
        }
        kc[c * n + r] = BC<VT>::mk((Rt)z.x, (Rt)z.y);
        for (int k = 0; k < J.d; ++k) fslot(J.out_index0 + k)[c * n + r] = z;
        rs += NA::of(z.x, z.y);
      }
      zn = NA::vmax(zn, rs);
    }
    double znorm, dmy;
    grp_max2(g, R, (double)zn, 0.0, znorm, dmy);
    if (N0 == 1) znorm = sqrt(znorm);
    for (int k = threadIdx.x; k < J.d; k += kBT) {
      s_c1[k] = znorm;
      s_coef[k] = 1.0;
      s_step[k] = (double)(J.k_off + k + 1) / J.d_block;
      s_active[k] = 1;
      s_extra[k] = 0ULL;
    }
    __syncthreads();
    for (int p = 1; p <= J.m; ++p) {
      // h/p once per CTA (an FP64 division is a long FP64-pipe sequence)
      __shared__ double s_scale;
      if (threadIdx.x == 0) s_scale = J.hspan / p;
      for (int k = threadIdx.x; k < J.d; k += kBT) s_coef[k] *= s_step[k];
      __syncthreads();
      const Rt scale = (Rt)s_scale;
      double coef[kBKReg];
      bool own[kBKReg];
#pragma unroll
      for (int u = 0; u < kBKReg; ++u) {
        own[u] = u < J.d && s_active[u];
        coef[u] = own[u] ? s_coef[u] : 0.0;
      }
      NT kmax = 0;
      NT fmx[kBKReg];
#pragma unroll
      for (int u = 0; u < kBKReg; ++u) fmx[u] = 0;
      // the new term at element (i, j) (all n0 columns): store it (and its
      // mirror), fold it into the running maxima and the active outputs
      // The output updates are read-modify-writes of the ring (L2); the
      // compiler cannot move a read above a store to the same array, so the
      // n0 reads of one accumulator are issued together before its stores
      // (one round trip per output instead of one per right-hand side).
      auto element = [&](int i, int j, const Rt* yx, const Rt* yy) {
        const long long r = i + (long long)Nt * j;
        NT rs = 0;
        double dx[N0], dy[N0];
#pragma unroll
        for (int c = 0; c < N0; ++c) {
          const Rt ax = yx[c] * scale, ay = yy[c] * scale;
          kn[c * n + r] = BC<VT>::mk(ax, ay);
          if (herm && i != j) kn[c * n + j + (long long)Nt * i] = BC<VT>::mk(ax, -ay);
          rs += NA::of_f((NT)ax, (NT)ay);
          dx[c] = (double)ax;
          dy[c] = (double)ay;
        }
        kmax = NA::vmax(kmax, rs);
        auto update = [&](int k, double ck) -> NT {
          double2* F = fslot(J.out_index0 + k);
          double2 f[N0];
#pragma unroll
          for (int c = 0; c < N0; ++c) f[c] = ldf<SK>(F + c * n + r);
          NT fs = 0;
#pragma unroll
          for (int c = 0; c < N0; ++c) {
            f[c].x = fma(ck, dx[c], f[c].x);
            f[c].y = fma(ck, dy[c], f[c].y);
            fs += NA::of(f[c].x, f[c].y);
          }
#pragma unroll
          for (int c = 0; c < N0; ++c) F[c * n + r] = f[c];
          return fs;
        };
#pragma unroll
        for (int u2 = 0; u2 < kBKReg; ++u2)
          if (own[u2]) fmx[u2] = NA::vmax(fmx[u2], update(u2, coef[u2]));
        for (int k = kBKReg; k < J.d; ++k)
          if (s_active[k]) atomicMax(&s_extra[k], bits_of((double)update(k, s_coef[k])));
      };
      if (SK) {
        // one CTA, terms on chip: one thread per element (upper triangle in
        // the Hermitian form), so a small walk's rows fill the warps
        const long long nel = herm ? (long long)Nt * (Nt + 1) / 2 : n;
        for (long long q = threadIdx.x; q < nel; q += kBT) {
          int i, j;
          if (herm) {
            j = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
            while ((long long)j * (j + 1) / 2 > q) --j;
            while ((long long)(j + 1) * (j + 2) / 2 <= q) ++j;
            i = (int)(q - (long long)j * (j + 1) / 2);
          } else {
            i = (int)(q % Nt);
            j = (int)(q / Nt);
          }
          Rt yx[N0], yy[N0];
#pragma unroll
          for (int c = 0; c < N0; ++c) {
            Rt cx, cy;
            mf_partB<Rt, VT, 1, LDP>(op, kc + c * n, j, &i, &cx, &cy);
            mf_finish<Rt, VT, false, LDP>(op, kc + c * n, i, j, cx, cy, yx[c], yy[c]);
          }
          element(i, j, yx, yy);
        }
      } else {
        const long long nitems = mf_item_count(Nt, herm);
        for (long long it = gw; it < nitems; it += (long long)g.size() * kBW) {
          int j, i0;
          mf_item(it, Nt, herm, j, i0);
          int irow[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int i = i0 + lane + 32 * u;
            irow[u] = (i < Nt && (!herm || i <= j)) ? i : -1;
          }
          Rt yx[2][N0], yy[2][N0];
          bmf_partB<Rt, VT, N0, LDP>(op, kc, n, j, irow, yx, yy);
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (irow[u] >= 0) bmf_finish<Rt, VT, N0, LDP>(op, kc, n, irow[u], j, yx[u], yy[u]);
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (irow[u] >= 0) element(irow[u], j, yx[u], yy[u]);
        }
      }
      // cluster maxima: K and the register outputs in pairs, the rest from s_extra
      double fn[kBDMax];
      double gk;
      grp_max2(g, R, (double)kmax, (double)fmx[0], gk, fn[0]);
#pragma unroll
      for (int u = 1; u < kBKReg; u += 2) {
        if (u >= J.d) break;
        double a0, a1;
        grp_max2(g, R, (double)fmx[u], u + 1 < kBKReg ? (double)fmx[u + 1] : 0.0, a0, a1);
        fn[u] = a0;
        if (u + 1 < kBKReg) fn[u + 1] = a1;
      }
      for (int k = kBKReg; k < J.d; k += 2) {
        double a0, a1;
        grp_max2(g, R, of_bits(s_extra[k]), k + 1 < J.d ? of_bits(s_extra[k + 1]) : 0.0, a0, a1);
        fn[k] = a0;
        if (k + 1 < J.d) fn[k + 1] = a1;
      }
      ++matvecs;
      for (int k = 0; k < J.d; ++k) fupd += s_active[k];
      // stop test, identical in every CTA of the cluster (only the threads
      // that own an output take the square roots)
      int any = 0;
      __syncthreads();
      for (int k = threadIdx.x; k < J.d; k += kBT) {
        s_extra[k] = 0ULL;
        if (!s_active[k]) continue;
        const double normk = N0 == 1 ? sqrt(gk) : gk;
        const double c2 = s_coef[k] * normk;
        const double nf = N0 == 1 ? sqrt(fn[k]) : fn[k];
        if (s_c1[k] + c2 <= tol * nf) s_active[k] = 0;
        s_c1[k] = c2;
      }
      __syncthreads();
      for (int k = 0; k < J.d; ++k) any |= s_active[k];
      VT* t = kc;
      kc = kn;
      kn = t;
      if (!any) break;
    }
    // populations of the finished outputs
    if (J.final_outputs && W.pops) {
      const long long tot = (long long)J.d * N0 * Nt;
      for (long long q = ct; q < tot; q += cstride) {
        const int k = (int)(q / ((long long)N0 * Nt));
        const int rem = (int)(q % ((long long)N0 * Nt));
        const int c = rem / Nt, v = rem % Nt;
        const double2 z = ldf<SK>(fslot(J.out_index0 + k) + c * n + (long long)v * (Nt + 1));
        W.pops[((long long)(J.out_index0 + k) * N0 + c) * Nt + v] = z.x;
      }
    }
    g.sync();   // outputs complete before the next block reads them
  }
  if (crank == 0 && threadIdx.x == 0) {
    W.counters[0] = matvecs;
    W.counters[1] = fupd;
    // every CTA of the group is past the sync that ended the last job: the
    // walk's populations are final; tell a host that hands walks out early
    if (W.done) {
      __threadfence_system();
      *(volatile int*)W.done = 1;
    }
  }
}

template <class G, bool SK>
__device__ void dispatch_walk(G g, Red& R, const BWalk& W, double tol, double* s_coef,
                              double* s_step, double* s_c1, int* s_active, unsigned char* sk) {
  double2* kd = reinterpret_cast<double2*>(sk);
  float2* kf = reinterpret_cast<float2*>(sk);
  switch (W.n0 * 2 + W.f32) {
    case 2: run_walk<G, double2, 1, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kd); break;
    case 3: run_walk<G, float2, 1, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kf); break;
    case 4: run_walk<G, double2, 2, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kd); break;
    case 5: run_walk<G, float2, 2, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kf); break;
    case 6: run_walk<G, double2, 3, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kd); break;
    case 7: run_walk<G, float2, 3, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kf); break;
    case 8: run_walk<G, double2, 4, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kd); break;
    default: run_walk<G, float2, 4, SK>(g, R, W, tol, s_coef, s_step, s_c1, s_active, kf); break;
  }
}

// 4 blocks per SM (64 registers): the walks' phase 2 is latency-bound on
// gathers from L2, and twice the resident clusters outweigh the register
// spills (batch256: 214 -> 180 ms for the series phase).  The cluster size is
// the launch's (2, 4, 8 or 16 CTAs, chosen by the schedule tuner); a walk's
// results do not depend on it (per-element arithmetic is the same, and the
// cluster reductions of this phase are maxima).
__global__ void __launch_bounds__(kBT, 4)
batch_series_kernel(BArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ Red R;
  __shared__ int s_w;
  __shared__ double s_coef[kBDMax];
  __shared__ double s_step[kBDMax];
  __shared__ double s_c1[2 * kBDMax];
  __shared__ int s_active[kBDMax];
  for (int k = threadIdx.x; k < 2 * kBDMax; k += kBT) s_c1[k] = 0.0;
  __syncthreads();
  for (;;) {
    const int wi = next_walk(cl, &a.queue[1], &s_w, a.big, a.nbig);
    if (wi < 0) break;
    BWalk& W = a.walks[wi];
    // plan on the device from the walk's own norms
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      const PlanInfo info = plan_series(W.dp, c_theta_b[W.f32 ? 1 : 0], W.t0, W.dt, W.steps, W.n0,
                                        W.ring, W.jobs, W.njobs, kBDMax);
      if (info.njobs != W.njobs || info.max_job_d > kBDMax) W.counters[2] = 1;
    }
    cl.sync();
    if (__ldcg(&W.counters[2])) continue;   // L2 read: every CTA sees rank 0's flag
    const double tol = a.tol[W.f32 ? 1 : 0];
    dispatch_walk<ClusterG, false>(ClusterG{cl, (int)cl.num_blocks()}, R, W, tol, s_coef, s_step,
                                   s_c1, s_active, nullptr);
  }
}

// Phase 2 for small walks: one CTA per walk, Taylor terms in dynamic shared
// memory (2 n0 n values of the walk's precision, at most the schedule's
// one-CTA limit).  CTAs of 128 threads measured the same on the EST sweep
// and 64 or 32 threads slower (a walk's term then runs on fewer warps).
__global__ void __launch_bounds__(kBT) batch_small_kernel(BArgs a) {
  extern __shared__ __align__(16) unsigned char s_k[];
  __shared__ Red R;
  __shared__ int s_w;
  __shared__ double s_coef[kBDMax];
  __shared__ double s_step[kBDMax];
  __shared__ double s_c1[2 * kBDMax];
  __shared__ int s_active[kBDMax];
  for (int k = threadIdx.x; k < 2 * kBDMax; k += kBT) s_c1[k] = 0.0;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned k = atomicAdd(&a.queue[2], 1u);
      s_w = k < (unsigned)a.nsmall ? a.small[k] : -1;
    }
    __syncthreads();
    const int wi = s_w;
    __syncthreads();
    if (wi < 0) break;
    BWalk& W = a.walks[wi];
    if (threadIdx.x == 0) {
      const PlanInfo info = plan_series(W.dp, c_theta_b[W.f32 ? 1 : 0], W.t0, W.dt, W.steps, W.n0,
                                        W.ring, W.jobs, W.njobs, kBDMax);
      if (info.njobs != W.njobs || info.max_job_d > kBDMax) W.counters[2] = 1;
    }
    __syncthreads();
    if (*((volatile long long*)&W.counters[2])) continue;
    const double tol = a.tol[W.f32 ? 1 : 0];
    dispatch_walk<CtaG, true>(CtaG{}, R, W, tol, s_coef, s_step, s_c1, s_active, s_k);
  }
}

__global__ void herm_check_many(int Nt, long long n, int cols, const double2* __restrict__ x,
                                unsigned long long* __restrict__ out) {
  unsigned long long da = 0, xa = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * cols;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = q / n, r = q % n;
    const int i = (int)(r % Nt), j = (int)(r / Nt);
    const double2 u = x[c * n + r];
    const double2 v = x[c * n + j + (long long)Nt * i];
    const double ex = u.x - v.x, ey = u.y + v.y;
    da = max(da, bits_of(ex * ex + ey * ey));
    xa = max(xa, bits_of(u.x * u.x + u.y * u.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    da = max(da, __shfl_xor_sync(0xffffffffu, da, o));
    xa = max(xa, __shfl_xor_sync(0xffffffffu, xa, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], da);
    atomicMax(&out[1], xa);
  }
}

// The small-walk kernel's dynamic shared-memory limit is a property of the
// function on a device, shared by every thread and stream: it is raised once
// per device to the largest size any batch uses (kSmallTotalBytes), never
// lowered, so that concurrent batches (the server's workers) cannot undercut
// each other's launches.
void allow_small_smem(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  QSW_CHECK_ARG(device >= 0 && device < 64, QSW_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (done[device]) return;
  QSW_CUDA_TRY(cudaFuncSetAttribute(batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmallTotalBytes));
  done[device] = true;
}

// ------------------------------------------------ series-phase schedule
// The series phase's schedule: CTAs per cluster (cs) and the largest pair of
// Taylor-term blocks (bytes) with which a walk runs on ONE CTA with its terms
// in shared memory (small_limit; 0: every walk on a cluster).  A walk's
// results do not depend on it (same per-element arithmetic; the phase's
// cluster reductions are maxima), so the schedule is free to tune.  The first
// batch of a kind (n0, precisions, largest N~ and walk count, each by power
// of two) with at least kTuneMinWalks walks times its own series phase under
// every candidate and keeps the fastest for the process; smaller batches take
// kDefaultSched.
struct BSched {
  int cs;
  int small_limit;
};
constexpr BSched kDefaultSched{8, 64 * 1024};
constexpr int kCsCandidates[] = {4, 8, 16};
constexpr int kSmallCandidates[] = {0, 32 * 1024, 64 * 1024};
constexpr int kTuneMinWalks = 16;

struct BTuneKey {
  int device, n0, precs, nbucket, cbucket;
  bool operator<(const BTuneKey& o) const {
    if (device != o.device) return device < o.device;
    if (n0 != o.n0) return n0 < o.n0;
    if (precs != o.precs) return precs < o.precs;
    if (nbucket != o.nbucket) return nbucket < o.nbucket;
    return cbucket < o.cbucket;
  }
};

std::mutex g_btune_mu;
std::map<BTuneKey, BSched> g_btune;
std::atomic<long long> g_btune_measurements{0};

int ilog2(int v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b;
}

bool btune_lookup(const BTuneKey& k, BSched* out) {
  std::lock_guard<std::mutex> lock(g_btune_mu);
  auto it = g_btune.find(k);
  if (it == g_btune.end()) return false;
  *out = it->second;
  return true;
}

BSched btune_store(const BTuneKey& k, const BSched& s) {
  g_btune_measurements.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lock(g_btune_mu);
  return g_btune.emplace(k, s).first->second;   // a concurrent tuner may have won
}

// Resident clusters of cs CTAs of the series-phase kernel (0: cannot run);
// clusters of more than 8 CTAs are opted into on first use.
int series_clusters(int device, int cs) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({device, cs});
  if (it != cache.end()) return it->second;
  if (cs > 8)
    QSW_CUDA_TRY(cudaFuncSetAttribute(batch_series_kernel,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(cs * 4096));
  cfg.blockDim = dim3(kBT);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, batch_series_kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    n = 0;
  }
  cache[{device, cs}] = n;
  return n;
}

}  // namespace

long long batch_tune_measurements() { return g_btune_measurements.load(); }

void batch_tune_reset() {
  std::lock_guard<std::mutex> lock(g_btune_mu);
  g_btune.clear();
}

void run_batch(qsw_ctx* ctx, int count, Op* const* ops, const double* const* d_rho0, int n0,
               const double* t0s, const double* dts, const int* steps, double* const* d_pops,
               qsw_batch_stats* stats, const WalkSink* sink) {
  cudaStream_t st = ctx->stream;
  QSW_CHECK_ARG(n0 >= 1 && n0 <= kMaxRhs, QSW_ERR_INVALID_ARG, "n0 must be 1..4");
  std::vector<BWalk> hw(count);
  std::vector<DevBuf> bufs;
  bufs.reserve(4 * count + 4);
  // Hermitian check of every walk's right-hand sides (one readback)
  DevBuf hb;
  hb.alloc(sizeof(unsigned long long) * 2 * count);
  QSW_CUDA_TRY(cudaMemsetAsync(hb.p, 0, hb.bytes, st));
  for (int w = 0; w < count; ++w) {
    const Op& op = *ops[w];
    QSW_CHECK_ARG(op.opkind == QSW_OPERATOR_MATRIX_FREE && !op.gq.active, QSW_ERR_INVALID_ARG,
                  "batched series needs matrix-free L-QSW operators");
    QSW_LAUNCH herm_check_many<<<grid_for(op.n * n0, 256, 1024), 256, 0, st>>>(
        op.Nt, op.n, n0, reinterpret_cast<const double2*>(d_rho0[w]),
        hb.as<unsigned long long>() + 2 * w);
  }
  QSW_CUDA_TRY(cudaGetLastError());
  std::vector<unsigned long long> hbits(2 * count);
  QSW_CUDA_TRY(cudaMemcpyAsync(hbits.data(), hb.p, hb.bytes, cudaMemcpyDeviceToHost, st));
  // per-walk descriptors, phase-1 workspace
  DevBuf dpbuf, cnt;
  dpbuf.alloc(sizeof(double) * (kNormPowers + 1) * count);
  cnt.alloc(sizeof(long long) * 4 * count);
  QSW_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, cnt.bytes, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  for (int w = 0; w < count; ++w) {
    const Op& op = *ops[w];
    BWalk& W = hw[w];
    memset(&W, 0, sizeof(W));
    W.mf64 = make_mf<double>(op, false);
    W.mfh64 = make_mf<double>(op, true);
    W.mf32 = make_mf<float>(op, false);
    W.Nt = op.Nt;
    W.n = op.n;
    W.n0 = n0;
    W.f32 = op.precision == QSW_C64_BULK;
    double a2, m2;
    memcpy(&a2, &hbits[2 * w], 8);
    memcpy(&m2, &hbits[2 * w + 1], 8);
    W.herm = sqrt(a2) <= 1e-13 * std::max(1.0, sqrt(m2));
    W.rho0 = reinterpret_cast<const double2*>(d_rho0[w]);
    W.pops = d_pops[w];
    W.t0 = t0s[w];
    W.dt = dts[w];
    W.steps = steps[w];
    W.norm_span = std::max(t0s[w], steps[w] * dts[w]);
    W.dp = dpbuf.as<double>() + (kNormPowers + 1) * w;
    W.counters = cnt.as<long long>() + 4 * w;
    W.done = sink ? sink->d_done + w : nullptr;
    bufs.emplace_back();
    bufs.back().alloc(sizeof(double2) * 6 * op.n + sizeof(double) * op.n);
    W.est = bufs.back().as<double2>();
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hw[x].n > hw[y].n; });
  DevBuf dwalks, dorder, dq;
  dwalks.alloc(sizeof(BWalk) * count);
  dorder.alloc(sizeof(int) * 3 * count);   // phase-1 order, cluster list, small list
  dq.alloc(sizeof(unsigned) * 3);
  QSW_CUDA_TRY(cudaMemcpyAsync(dwalks.p, hw.data(), sizeof(BWalk) * count, cudaMemcpyHostToDevice, st));
  QSW_CUDA_TRY(cudaMemcpyAsync(dorder.p, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  QSW_CUDA_TRY(cudaMemsetAsync(dq.p, 0, sizeof(unsigned) * 3, st));
  BArgs args{};
  args.walks = dwalks.as<BWalk>();
  args.order = dorder.as<int>();
  args.count = count;
  args.queue = dq.as<unsigned>();
  args.tol[0] = tolerance(QSW_C128);
  args.tol[1] = tolerance(QSW_C64_BULK);
  int max_clusters = 0;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl * 4096);
    cfg.blockDim = dim3(kBT);
    cfg.numAttrs = 0;   // the kernel declares its cluster shape
    QSW_CUDA_TRY(cudaOccupancyMaxActiveClusters(&max_clusters, batch_norms_kernel, &cfg));
  }
  const int clusters = std::max(1, std::min(max_clusters, count));
  cudaEvent_t e0, e1, e1b, e2;
  QSW_CUDA_TRY(cudaEventCreate(&e0));
  QSW_CUDA_TRY(cudaEventCreate(&e1));
  QSW_CUDA_TRY(cudaEventCreate(&e1b));
  QSW_CUDA_TRY(cudaEventCreate(&e2));
  QSW_CUDA_TRY(cudaEventRecord(e0, st));
  QSW_LAUNCH batch_norms_kernel<<<clusters * kCl, kBT, 0, st>>>(args);
  QSW_CUDA_TRY(cudaGetLastError());
  QSW_CUDA_TRY(cudaEventRecord(e1, st));
  // plans (host copy, same code as the device) size the phase-2 workspace
  std::vector<double> dps((kNormPowers + 1) * count);
  QSW_CUDA_TRY(cudaMemcpyAsync(dps.data(), dpbuf.p, sizeof(double) * dps.size(),
                               cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  // Every walk gets Taylor-term blocks and an output ring in global memory,
  // whichever schedule runs it (a walk small enough for one CTA needs a few KB).
  std::vector<size_t> kbw(count), rbw(count);
  int maxN = 0, precs = 0;
  for (int w = 0; w < count; ++w) {
    BWalk& W = hw[w];
    const double* theta = theta_table(W.f32 ? QSW_C64_BULK : QSW_C128);
    const PlanInfo info = plan_series(&dps[(kNormPowers + 1) * w], theta, W.t0, W.dt, W.steps,
                                      n0, 0, nullptr, 0, kBDMax);
    W.njobs = info.njobs;
    W.ring = info.max_d + 1;
    const size_t vb = W.f32 ? sizeof(float2) : sizeof(double2);
    kbw[w] = 2 * vb * n0 * (size_t)W.n;
    rbw[w] = sizeof(double2) * (size_t)W.ring * n0 * W.n;
    bufs.emplace_back();
    bufs.back().alloc(kbw[w]);
    W.kbuf = bufs.back().p;
    bufs.emplace_back();
    bufs.back().alloc(rbw[w]);
    W.fring = bufs.back().as<double2>();
    bufs.emplace_back();
    bufs.back().alloc(sizeof(Job) * std::max(1, W.njobs));
    W.jobs = bufs.back().as<Job>();
    maxN = std::max(maxN, W.Nt);
    precs |= W.f32 ? 2 : 1;
  }
  // One series phase under schedule sc: walks whose two Taylor-term blocks fit
  // in sc.small_limit bytes run on one CTA each (terms in shared memory, and
  // the ring too when both fit in kSmallTotalBytes) on the side stream; the
  // others on clusters of sc.cs CTAs.  Returns the clusters launched.
  std::vector<int> big, small, lists;
  cudaEvent_t fork = nullptr, join = nullptr;
  auto phase2 = [&](const BSched& sc, bool with_sink) -> int {
    big.clear();
    small.clear();
    size_t small_bytes = 0;
    for (int w : order) {
      BWalk& W = hw[w];
      const bool sm = kbw[w] <= (size_t)sc.small_limit;
      W.fsmem = sm && kbw[w] + rbw[w] <= kSmallTotalBytes;
      W.done = (with_sink && sink) ? sink->d_done + w : nullptr;
      if (sm) {
        small.push_back(w);
        small_bytes = std::max(small_bytes, kbw[w] + (W.fsmem ? rbw[w] : 0));
      } else {
        big.push_back(w);
      }
    }
    QSW_CUDA_TRY(cudaMemcpyAsync(dwalks.p, hw.data(), sizeof(BWalk) * count, cudaMemcpyHostToDevice,
                                 st));
    lists = big;
    lists.insert(lists.end(), small.begin(), small.end());
    if (!lists.empty())
      QSW_CUDA_TRY(cudaMemcpyAsync(dorder.as<int>() + count, lists.data(), sizeof(int) * lists.size(),
                                   cudaMemcpyHostToDevice, st));
    QSW_CUDA_TRY(cudaMemsetAsync(dq.as<unsigned>() + 1, 0, 2 * sizeof(unsigned), st));
    args.big = dorder.as<int>() + count;
    args.nbig = (int)big.size();
    args.small = args.big + big.size();
    args.nsmall = (int)small.size();
    if (!small.empty()) {
      const int dyn = (int)small_bytes;
      allow_small_smem(ctx->device);
      int per_sm = 0;
      QSW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_small_kernel, kBT, dyn));
      const int grid = std::max(1, std::min((int)small.size(), std::max(1, per_sm) * ctx->num_sms));
      cudaStream_t ss = st;
      if (!big.empty()) {
        if (!ctx->side) QSW_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        if (!fork) QSW_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        if (!join) QSW_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        QSW_CUDA_TRY(cudaEventRecord(fork, st));
        QSW_CUDA_TRY(cudaStreamWaitEvent(ctx->side, fork, 0));
        ss = ctx->side;
      }
      QSW_LAUNCH batch_small_kernel<<<grid, kBT, dyn, ss>>>(args);
      QSW_CUDA_TRY(cudaGetLastError());
      if (ss != st) QSW_CUDA_TRY(cudaEventRecord(join, ss));
    }
    int launched = 0;
    if (!big.empty()) {
      launched = std::max(1, std::min(series_clusters(ctx->device, sc.cs), (int)big.size()));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)sc.cs;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(launched * sc.cs));
      cfg.blockDim = dim3(kBT);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      QSW_CUDA_TRY((QSW_LAUNCH cudaLaunchKernelEx(&cfg, batch_series_kernel, args)));
      // the small walks' kernel (side stream) runs alongside; the call's
      // stream waits for both
      if (!small.empty()) QSW_CUDA_TRY(cudaStreamWaitEvent(st, join, 0));
    }
    return launched;
  };
  // the schedule: the context's fixed one, the tuned one for this batch's
  // kind, or (first batch of its kind) every candidate timed on this batch
  BSched sc = kDefaultSched;
  bool tuned = false;
  const BTuneKey key{ctx->device, n0, precs, ilog2(maxN), ilog2(count)};
  if (ctx->batch_cs > 0 || ctx->batch_small >= 0) {
    if (count >= kTuneMinWalks) btune_lookup(key, &sc);   // the other half, when tuned
    if (ctx->batch_cs > 0) sc.cs = ctx->batch_cs;
    if (ctx->batch_small >= 0) sc.small_limit = ctx->batch_small;
  } else if (count >= kTuneMinWalks) {
    if (!btune_lookup(key, &sc) && !ctx->batch_no_tune) {
      cudaEvent_t ta, tb;
      QSW_CUDA_TRY(cudaEventCreate(&ta));
      QSW_CUDA_TRY(cudaEventCreate(&tb));
      float best_ms = 0.f;
      for (int cs : kCsCandidates) {
        if (series_clusters(ctx->device, cs) < 1) continue;
        for (int sl : kSmallCandidates) {
          const BSched cand{cs, sl};
          QSW_CUDA_TRY(cudaEventRecord(ta, st));
          phase2(cand, false);
          QSW_CUDA_TRY(cudaEventRecord(tb, st));
          QSW_CUDA_TRY(cudaEventSynchronize(tb));
          float ms = 0.f;
          QSW_CUDA_TRY(cudaEventElapsedTime(&ms, ta, tb));
          if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            sc = cand;
          }
        }
      }
      cudaEventDestroy(ta);
      cudaEventDestroy(tb);
      sc = btune_store(key, sc);
      tuned = true;
    }
  }
  QSW_CUDA_TRY(cudaEventRecord(e1b, st));
  const int clusters2 = phase2(sc, true);
  QSW_CUDA_TRY(cudaEventRecord(e2, st));
  if (sink) {
    // hand finished walks out while the kernels run; the loop ends when both
    // kernels have (their waits are cluster barriers, which always complete).
    // The thread yields between polls: a timed sleep can overshoot by
    // milliseconds on a loaded host, and each overshoot delays a walk's result.
    std::vector<char> seen(count, 0);
    for (;;) {
      const bool done = cudaEventQuery(e2) != cudaErrorNotReady;
      for (int w = 0; w < count; ++w)
        if (!seen[w] && ((volatile int*)sink->h_done)[w]) {
          seen[w] = 1;
          sink->ready(w);
        }
      if (done) break;
      std::this_thread::yield();
    }
  }
  std::vector<long long> hc(4 * count);
  QSW_CUDA_TRY(cudaMemcpyAsync(hc.data(), cnt.p, cnt.bytes, cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  float ms1 = 0, ms2 = 0;
  cudaEventElapsedTime(&ms1, e0, e1);
  cudaEventElapsedTime(&ms2, e1b, e2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e1b);
  cudaEventDestroy(e2);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  for (int w = 0; w < count; ++w)
    QSW_CHECK_ARG(hc[4 * w + 2] == 0, QSW_ERR_CUDA, "batched series: device plan mismatch");
  if (stats) {
    stats->walks = count;
    stats->clusters = big.empty() ? 0 : clusters2;
    stats->cluster_size = sc.cs;
    stats->small_limit = sc.small_limit;
    stats->tuned = tuned ? 1 : 0;
    stats->small_walks = (int)small.size();
    stats->norms_ms = ms1;
    stats->series_ms = ms2;
    long long mv = 0, fu = 0;
    double flops = 0.0, bytes = 0.0;
    for (int w = 0; w < count; ++w) {
      mv += hc[4 * w];
      fu += hc[4 * w + 1];
      // per walk, as for one series: the Hermitian form computes the upper
      // triangle; every application acts on the walk's n0 right-hand sides
      const Op& op = *ops[w];
      const BWalk& W = hw[w];
      const double frac = W.herm ? (op.Nt + 1.0) / (2.0 * op.Nt) : 1.0;
      const double elems = frac * (double)op.n * n0;
      const double offdiag = frac * (double)(op.nnz_csr - op.n - op.g.n_jumps) * n0;
      const double per_app = 4.0 * offdiag + 13.0 * elems + 4.0 * op.g.n_jumps * n0;
      const double vb = W.f32 ? sizeof(float2) : sizeof(double2);
      flops += (double)hc[4 * w] * per_app + 7.0 * (elems / n0) * (double)hc[4 * w + 1] * n0;
      bytes += (double)hc[4 * w] * (op_bytes(op) + 2.0 * elems * vb) +
               32.0 * elems * (double)hc[4 * w + 1];
    }
    stats->matvecs = mv;
    stats->fupdates = fu;
    stats->algorithmic_flops = flops;
    stats->algorithmic_bytes = bytes;
  }
}

}  // namespace qsw
