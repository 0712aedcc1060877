// The Taylor-series engine: Algorithms 3.2 (`step`) and 5.2 (`series`) of
// Al-Mohy & Higham as used by the paper (Section 3.1), run as ONE persistent
// cooperative kernel per call.
//
// The plan (params.cuh, built on the device by plan_kernel) turns the call into
// a list of Taylor blocks.  A block with input Z, span hspan = d h and outputs
// k = 1..d computes
//     Khat_0 = Z,   Khat_p = (hspan / p) L Khat_{p-1},
//     F_k = Z + sum_{p=1}^{p_k} (k/d)^p Khat_p,
// which is Algorithm 5.2's  F_k = sum_p k^p K_p  with K_p = (hA)^p Z / p!
// (Khat_p = d^p K_p), and with d = 1 one stage of Algorithm 3.2.  Output k stops
// after the first p with  c1 + c2 <= tol ||F_k||_inf,  c2 = (k/d)^p ||Khat_p||_inf,
// c1 the previous term's norm (||Z||_inf at p = 1).  The powers are formed once
// per block and every active output is updated in the same pass, so a block
// costs max_k p_k applications of L~ (paper Section 5: a whole time series for
// about the cost of one `step`).
//
// One term = one pass over the n elements: apply L~ (matrix-free, or CSR), scale,
// store Khat_p, update every active F_k in FP64, and keep running inf-norm
// maxima (squared moduli compared as integer bit patterns, which keeps them
// off the FP64 pipe).  A grid barrier with a bounded wait separates terms;
// after it every block reads the same maxima and takes the same stop decisions,
// so the host is never consulted inside the series.
//
// Precision: VT = double2 (complex128) or float2 (complex64 bulk: FP32 operator
// coefficients, FP32 Taylor terms, FP32 accumulation of every product).  The
// F_k accumulators, the norms and the stop test are FP64 in both cases.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <thread>

#include "gqsw.cuh"
#include "matfree.cuh"
#include "op.h"
#include "params.cuh"

namespace qsw {

__constant__ double c_theta[2][kMMax];

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kDMax = 128;              // outputs per Taylor job (a larger Algorithm 5.2
                                        // block becomes several jobs from the same Z)
constexpr int kKReg = 2;                // outputs whose running max lives in registers (the
                                        // rest use shared memory): 2 keeps the kernel at 64
                                        // registers, 4 blocks (32 warps) per SM
constexpr int kRpt = 2;                 // rows per thread in one matrix-free pass
constexpr unsigned kSpinLimit = 1u << 24;  // bounded barrier wait (~seconds)

enum : int { kErrNone = 0, kErrBarrier = 1, kErrPlan = 2 };
enum : int { kOpCsr = 0, kOpMatfree = 1, kOpMatfreeHerm = 2, kOpGlobal = 3, kOpGlobalHerm = 4,
             kOpSell = 5 };
static_assert(kItemRows == 32 * kRpt, "a work item is one row per lane per kRpt");

// Each group of words that the grid hits at once sits in its own 256-byte
// block: the barrier's arrival counter, the word it spins on, the item
// counters and the norm maxima (sharing lines made the atomics and the spin
// reads of one barrier queue behind each other: 1 % of the ER-1000 series).
struct Ctrl {
  alignas(256) unsigned int bar_count;
  alignas(256) unsigned int bar_gen;
  alignas(256) int error;
  int njobs;
  unsigned long long matvecs;
  unsigned long long fupdates;   // sum over terms of the outputs updated
  alignas(256) unsigned int work[3];    // matrix-free column counters, one per term slot
  alignas(256) unsigned int work2[3];   // global walks: pass-A counters
  alignas(256) unsigned long long gmax[3][1 + kDMax];
};

struct SeriesArgs {
  int n, nt;
  const int* rowptr;     // CSR operator (col and val: its slices, for the sliced form)
  const int* col;
  const void* val;
  const int* sperm;      // sliced form: row of each lane, slice offsets and widths
  const long long* soff;
  const int* swidth;
  int slices;
  MfOp<double> mf64;     // matrix-free operator (one of the two is used)
  MfOp<float> mf32;
  GqOp<double> gq64;     // global-interaction walk (one of the two is used)
  GqOp<float> gq32;
  void* wbuf;            // its pass-A products, nl x n
  void* k0;
  void* k1;
  const double2* rho0;
  double2* slots;
  int ring;              // 0: series index k -> slot k; else k % ring
  int mirror;            // Hermitian form with caller outputs: fill lower triangles
  double* pops;          // (steps+1) x nt or null
  const Job* jobs;
  int njobs;
  Ctrl* ctrl;
  double tol;
  int* progress;         // host-mapped count of final caller outputs, or null
};

template <class VT> struct Cplx;
template <> struct Cplx<double2> {
  using R = double;
  __device__ static double2 make(double a, double b) { return make_double2(a, b); }
  __device__ static double2 conj_of(double a, double b) {
    return make_double2(a, __longlong_as_double(__double_as_longlong(b) ^ (1LL << 63)));
  }
  __device__ static const MfOp<double>& mf(const SeriesArgs& a) { return a.mf64; }
  __device__ static const GqOp<double>& gq(const SeriesArgs& a) { return a.gq64; }
};
template <> struct Cplx<float2> {
  using R = float;
  __device__ static float2 make(float a, float b) { return make_float2(a, b); }
  __device__ static float2 conj_of(float a, float b) {
    return make_float2(a, __int_as_float(__float_as_int(b) ^ (int)0x80000000));
  }
  __device__ static const MfOp<float>& mf(const SeriesArgs& a) { return a.mf32; }
  __device__ static const GqOp<float>& gq(const SeriesArgs& a) { return a.gq32; }
};

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
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Grid barrier for a cooperative launch (all blocks co-resident).  The wait is
// bounded: on timeout the block records kErrBarrier and returns false, and so
// does every later barrier, so all blocks leave the kernel.
__device__ bool grid_barrier(Ctrl* c, unsigned limit = kSpinLimit) {
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
        if (*((volatile int*)&c->error) != kErrNone || ++spins > limit) {
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

// Keys of the running inf-norm maxima: squared moduli as integer bit patterns
// (non-negative numbers order like their bits), so the max never touches the
// FP64 pipe.  complex128 keeps FP64 moduli; complex64 bulk takes them in FP32
// (the F accumulators through an integer-only truncation to float), which is
// ample for its 2^-24 stop test.
__device__ __forceinline__ float f32_trunc(double v) {
  const long long b = __double_as_longlong(v);
  const int hi = (int)(b >> 32);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  const int m = (int)((b >> 29) & 0x7fffff);
  const int bits = (hi & (int)0x80000000) | (e << 23) | m;
  return e <= 0 ? 0.0f : __int_as_float(e >= 255 ? ((hi & (int)0x80000000) | 0x7f800000) : bits);
}

template <class VT> struct NormKey;
template <> struct NormKey<double2> {
  __device__ static unsigned long long y(double a, double b) { return as_bits(a * a + b * b); }
  __device__ static unsigned long long f(double a, double b) { return as_bits(a * a + b * b); }
  __device__ static double value(unsigned long long k) { return from_bits(k); }
};
template <> struct NormKey<float2> {
  __device__ static unsigned long long y(float a, float b) { return __float_as_uint(a * a + b * b); }
  __device__ static unsigned long long f(double a, double b) {
    const float x = f32_trunc(a), z = f32_trunc(b);
    return __float_as_uint(x * x + z * z);
  }
  __device__ static double value(unsigned long long k) { return (double)__uint_as_float((unsigned)k); }
};

// Per-thread epilogue state of one Taylor term.
template <class VT> struct Epilogue {
  using R = typename Cplx<VT>::R;
  double2* slots;       // the outputs (caller's array or ring) and their layout
  int ring;
  long long n;
  VT* knext;
  int out0, d;
  unsigned long long kmax;
  unsigned long long fmax[kKReg];
  const double* s_coef;
  const int* s_active;
  unsigned long long* s_fmax_extra;   // outputs k >= kKReg (shared, block-level keys)

  __device__ __forceinline__ double2* slot(int idx) const {
    return slots + (long long)(ring ? idx % ring : idx) * n;
  }

  __device__ void consume(long long r, R yx, R yy) {
    knext[r] = Cplx<VT>::make(yx, yy);
    kmax = umax64(kmax, NormKey<VT>::y(yx, yy));
    const double dx = (double)yx, dy = (double)yy;
#pragma unroll
    for (int u = 0; u < kKReg; ++u) {
      // coefficients and activity come from shared memory (broadcast reads):
      // keeping copies in registers measured slower at this register budget
      if (u < d && s_active[u]) {
        double2* F = slot(out0 + u) + r;
        double2 f = __ldcg(F);
        f.x = fma(s_coef[u], dx, f.x);
        f.y = fma(s_coef[u], dy, f.y);
        *F = f;
        fmax[u] = umax64(fmax[u], NormKey<VT>::f(f.x, f.y));
      }
    }
    for (int k = kKReg; k < d; ++k) {
      if (!s_active[k]) continue;
      double2* F = slot(out0 + k) + r;
      double2 f = __ldcg(F);
      f.x = fma(s_coef[k], dx, f.x);
      f.y = fma(s_coef[k], dy, f.y);
      *F = f;
      atomicMax(&s_fmax_extra[k], NormKey<VT>::f(f.x, f.y));
    }
  }
};

// UNR: entries per lane in flight in the CSR sweep's row loop (2 or 4; the
// matrix-free and global sweeps ignore it).
template <class VT, int OPK, int TPR, int UNR = 2>
__global__ void __launch_bounds__(kBlock, 4)
series_kernel(SeriesArgs a) {
  using R = typename Cplx<VT>::R;
  __shared__ unsigned long long s_red[kWarps][1 + kKReg];
  __shared__ unsigned long long s_fmax_extra[kDMax];
  __shared__ double s_c1[kDMax];
  __shared__ double s_coef[kDMax];
  __shared__ double s_step[kDMax];
  __shared__ int s_active[kDMax];
  __shared__ int s_any;
  __shared__ double s_normk;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const long long gthread = (long long)blockIdx.x * kBlock + tid;
  const long long nthreads = (long long)gridDim.x * kBlock;
  Ctrl* ctrl = a.ctrl;
  unsigned term = 0;

  for (int jb = 0; jb < a.njobs; ++jb) {
    const Job J = a.jobs[jb];
    const double2* Z = J.z_slot < 0 ? a.rho0 : slot_ptr(a, J.z_slot);
    VT* kcur = static_cast<VT*>(a.k0);
    VT* knext = static_cast<VT*>(a.k1);

    // ---- init: Khat_0 = Z, F_k = Z, ||Z||_inf
    unsigned long long zmax = 0;
    for (long long r = gthread; r < a.n; r += nthreads) {
      double2 z;
      if (OPK == kOpMatfreeHerm || OPK == kOpGlobalHerm) {
        // only upper triangles are maintained: read (i, j), i > j, as conj(Z(j, i))
        const int i = (int)(r % a.nt), j = (int)(r / a.nt);
        if (i > j) {
          z = __ldcg(Z + j + (long long)a.nt * i);
          z.y = -z.y;
        } else {
          z = __ldcg(Z + r);
        }
        // a global walk's Hermitian form needs exactly Hermitian terms
        // (gq_element_herm): the input's diagonal is taken as real
        if (OPK == kOpGlobalHerm && i == j) z.y = 0.0;
      } else {
        z = __ldcg(Z + r);
      }
      kcur[r] = Cplx<VT>::make((R)z.x, (R)z.y);
      for (int k = 0; k < J.d; ++k) slot_ptr(a, J.out_index0 + k)[r] = z;
      zmax = umax64(zmax, as_bits(z.x * z.x + z.y * z.y));
    }
    zmax = warp_umax(zmax);
    if (lane == 0) s_red[warp][0] = zmax;
    __syncthreads();
    unsigned slot3 = term % 3;
    if (tid == 0) {
      unsigned long long m = 0;
      for (int w = 0; w < kWarps; ++w) m = umax64(m, s_red[w][0]);
      atomicMax(&ctrl->gmax[slot3][0], m);
    }
    if (blockIdx.x == 0) {
      const unsigned nx = (term + 1) % 3;
      for (int q = tid; q <= J.d; q += kBlock) ctrl->gmax[nx][q] = 0ULL;
      if (tid == 0) {
        ctrl->work[nx] = 0u;
        ctrl->work2[nx] = 0u;
      }
    }
    if (!grid_barrier(ctrl)) return;
    const double normz = sqrt(from_bits(__ldcg(&ctrl->gmax[slot3][0])));
    ++term;
    for (int k = tid; k < J.d; k += kBlock) {
      s_c1[k] = normz;
      s_coef[k] = 1.0;
      s_step[k] = (double)(J.k_off + k + 1) / (double)J.d_block;
      s_active[k] = 1;
    }
    __syncthreads();

    for (int p = 1; p <= J.m; ++p) {
      const double scale = J.hspan / p;
      const R rscale = (R)scale;
      slot3 = term % 3;
      for (int k = tid; k < J.d; k += kBlock) {
        s_coef[k] *= s_step[k];
        s_fmax_extra[k] = 0ULL;
      }
      __syncthreads();
      Epilogue<VT> ep;
      ep.slots = a.slots;
      ep.ring = a.ring;
      ep.n = a.n;
      ep.knext = knext;
      ep.out0 = J.out_index0;
      ep.d = J.d;
      ep.s_coef = s_coef;
      ep.s_active = s_active;
      ep.s_fmax_extra = s_fmax_extra;
      ep.kmax = 0;
#pragma unroll
      for (int u = 0; u < kKReg; ++u) ep.fmax[u] = 0;

      if (OPK == kOpGlobal || OPK == kOpGlobalHerm) {
        // ---- global walk: pass A (W_k = K L'_k^dag, every element), a grid
        // barrier, then pass B (the term, upper triangle for Hermitian input)
        constexpr bool kHerm = OPK == kOpGlobalHerm;
        const GqOp<R>& op = Cplx<VT>::gq(a);
        VT* w = static_cast<VT*>(a.wbuf);
        const int nt = a.nt;
        if (op.nl || kHerm) {
          const long long nall = mf_item_count(nt, false);
          for (;;) {
            unsigned int k = 0;
            if (lane == 0) k = atomicAdd(&ctrl->work2[slot3], 1u);
            k = __shfl_sync(0xffffffffu, k, 0);
            if ((long long)k >= nall) break;
            int j, a0;
            mf_item(k, nt, false, j, a0);
            int arow[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int r = a0 + lane + 32 * u;
              arow[u] = r < nt ? r : -1;
            }
            gq_pass_a<R, VT>(op, kcur, w, j, arow);
            if (kHerm) gq_pass_a_r<R, VT>(op, kcur, w, j, arow);
          }
          if (!grid_barrier(ctrl)) return;
        }
        const long long nitems = mf_item_count(nt, kHerm);
        for (;;) {
          unsigned int k = 0;
          if (lane == 0) k = atomicAdd(&ctrl->work[slot3], 1u);
          k = __shfl_sync(0xffffffffu, k, 0);
          if ((long long)k >= nitems) break;
          int j, i0;
          mf_item(k, nt, kHerm, j, i0);
#pragma unroll
          for (int u = 0; u < kRpt; ++u) {
            const int i = i0 + lane + 32 * u;
            if (i >= nt || (kHerm && i > j)) continue;
            R yx, yy;
            if (kHerm) gq_element_herm<R, VT>(op, kcur, w, i, j, yx, yy);
            else gq_element<R, VT>(op, kcur, w, i, j, yx, yy);
            yx *= rscale;
            yy *= rscale;
            ep.consume(i + (long long)nt * j, yx, yy);
            if (kHerm && i != j) knext[j + (long long)nt * i] = Cplx<VT>::conj_of(yx, yy);
          }
        }
      } else if (OPK == kOpMatfree || OPK == kOpMatfreeHerm) {
        // ---- matrix-free sweep: warps take 64-row chunks of columns from a
        // counter (no block-level synchronisation inside the pass)
        constexpr bool kHerm = OPK == kOpMatfreeHerm;
        const MfOp<R>& op = Cplx<VT>::mf(a);
        const int nt = a.nt;
        const long long nitems = mf_item_count(nt, kHerm);
        for (;;) {
          unsigned int k = 0;
          if (lane == 0) k = atomicAdd(&ctrl->work[slot3], 1u);
          k = __shfl_sync(0xffffffffu, k, 0);
          if ((long long)k >= nitems) break;
          int j, i0;
          mf_item(k, nt, kHerm, j, i0);
          int irow[kRpt];
          mf_window_rows(op.prow, i0, lane, kHerm ? j : nt - 1, irow);
          R ox[kRpt], oy[kRpt];
          mf_window_apply<R, VT, false>(op, kcur, j, i0, irow, ox, oy);
#pragma unroll
          for (int u = 0; u < kRpt; ++u) {
            if (irow[u] < 0) continue;
            const R yx = ox[u] * rscale;
            const R yy = oy[u] * rscale;
            ep.consume(irow[u] + (long long)nt * j, yx, yy);
            // Hermitian form: the term is stored in full, its lower triangle
            // as the conjugate (sign flip on the bit pattern, no FP64 op)
            if (kHerm && irow[u] != j)
              knext[j + (long long)nt * irow[u]] = Cplx<VT>::conj_of(yx, yy);
          }
        }
      } else if (OPK == kOpSell) {
        // ---- sliced CSR sweep: one lane per row, a warp per 32-row slice;
        // entry k of every lane of a slice is one contiguous 32-entry load
        const VT* __restrict__ val = static_cast<const VT*>(a.val);
        const int* __restrict__ col = a.col;
        const long long wglobal = gthread / 32;
        const long long wstride = (long long)gridDim.x * kWarps;
        for (long long sl = wglobal; sl < a.slices; sl += wstride) {
          const int r = a.sperm[sl * 32 + lane];
          const long long base = a.soff[sl] + lane;
          const int w = a.swidth[sl];
          R ax = 0, ay = 0, bx = 0, by = 0;
          int k = 0;
          if (UNR == 4) {
            R cx = 0, cy = 0, dx = 0, dy = 0;
            for (; k + 3 < w; k += 4) {
              const long long e = base + 32LL * k;
              const int c0 = __ldcs(col + e), c1 = __ldcs(col + e + 32);
              const int c2 = __ldcs(col + e + 64), c3 = __ldcs(col + e + 96);
              const VT v0 = __ldcs(val + e), v1 = __ldcs(val + e + 32);
              const VT v2 = __ldcs(val + e + 64), v3 = __ldcs(val + e + 96);
              const VT x0 = __ldcg(kcur + c0), x1 = __ldcg(kcur + c1);
              const VT x2 = __ldcg(kcur + c2), x3 = __ldcg(kcur + c3);
              ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
              ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
              bx = fma(v1.x, x1.x, fma(-v1.y, x1.y, bx));
              by = fma(v1.x, x1.y, fma(v1.y, x1.x, by));
              cx = fma(v2.x, x2.x, fma(-v2.y, x2.y, cx));
              cy = fma(v2.x, x2.y, fma(v2.y, x2.x, cy));
              dx = fma(v3.x, x3.x, fma(-v3.y, x3.y, dx));
              dy = fma(v3.x, x3.y, fma(v3.y, x3.x, dy));
            }
            ax += cx;
            ay += cy;
            bx += dx;
            by += dy;
          }
          for (; k + 1 < w; k += 2) {
            const long long e = base + 32LL * k;
            const int c0 = __ldcs(col + e), c1 = __ldcs(col + e + 32);
            const VT v0 = __ldcs(val + e), v1 = __ldcs(val + e + 32);
            const VT x0 = __ldcg(kcur + c0), x1 = __ldcg(kcur + c1);
            ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
            ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
            bx = fma(v1.x, x1.x, fma(-v1.y, x1.y, bx));
            by = fma(v1.x, x1.y, fma(v1.y, x1.x, by));
          }
          if (k < w) {
            const long long e = base + 32LL * k;
            const int c0 = __ldcs(col + e);
            const VT v0 = __ldcs(val + e);
            const VT x0 = __ldcg(kcur + c0);
            ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
            ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
          }
          if (r >= 0) ep.consume(r, (ax + bx) * rscale, (ay + by) * rscale);
        }
      } else {
        // ---- CSR sweep: TPR lanes per row.  A warp owns 32 consecutive rows and
        // covers them in TPR rounds of 32 / TPR rows; after each round's
        // reduction, row rb + L's sum moves to lane L, so the epilogue (FP64
        // output updates and norms) runs on all 32 lanes instead of one lane
        // per row.
        const VT* __restrict__ val = static_cast<const VT*>(a.val);
        const int* __restrict__ col = a.col;
        const int* __restrict__ rowptr = a.rowptr;
        const int glane = lane % TPR;
        constexpr int kGpw = 32 / TPR;
        const long long wglobal = gthread / 32;
        const long long rstride = (long long)gridDim.x * kWarps * 32;
        for (long long rb = wglobal * 32; rb < a.n; rb += rstride) {
          R mx = 0, my = 0;   // the sums of row rb + lane
#pragma unroll
          for (int q = 0; q < TPR; ++q) {
            const long long r = rb + q * kGpw + lane / TPR;
            const bool valid = r < a.n;
            const int e0 = valid ? rowptr[r] : 0;
            const int e1 = valid ? rowptr[r + 1] : 0;
            R ax = 0, ay = 0;
            int e = e0 + glane;
            if (UNR == 4) {   // four entries in flight, two accumulator pairs
              R bx = 0, by = 0;
              for (; e + 3 * TPR < e1; e += 4 * TPR) {
                const int c0 = __ldcs(col + e);
                const int c1 = __ldcs(col + e + TPR);
                const int c2 = __ldcs(col + e + 2 * TPR);
                const int c3 = __ldcs(col + e + 3 * TPR);
                const VT v0 = __ldcs(val + e);
                const VT v1 = __ldcs(val + e + TPR);
                const VT v2 = __ldcs(val + e + 2 * TPR);
                const VT v3 = __ldcs(val + e + 3 * TPR);
                const VT x0 = __ldcg(kcur + c0);
                const VT x1 = __ldcg(kcur + c1);
                const VT x2 = __ldcg(kcur + c2);
                const VT x3 = __ldcg(kcur + c3);
                ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
                ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
                bx = fma(v1.x, x1.x, fma(-v1.y, x1.y, bx));
                by = fma(v1.x, x1.y, fma(v1.y, x1.x, by));
                ax = fma(v2.x, x2.x, fma(-v2.y, x2.y, ax));
                ay = fma(v2.x, x2.y, fma(v2.y, x2.x, ay));
                bx = fma(v3.x, x3.x, fma(-v3.y, x3.y, bx));
                by = fma(v3.x, x3.y, fma(v3.y, x3.x, by));
              }
              ax += bx;
              ay += by;
            }
            for (; e + TPR < e1; e += 2 * TPR) {
              const int c0 = __ldcs(col + e);
              const int c1 = __ldcs(col + e + TPR);
              const VT v0 = __ldcs(val + e);
              const VT v1 = __ldcs(val + e + TPR);
              const VT x0 = __ldcg(kcur + c0);
              const VT x1 = __ldcg(kcur + c1);
              ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
              ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
              ax = fma(v1.x, x1.x, fma(-v1.y, x1.y, ax));
              ay = fma(v1.x, x1.y, fma(v1.y, x1.x, ay));
            }
            if (e < e1) {
              const int c0 = __ldcs(col + e);
              const VT v0 = __ldcs(val + e);
              const VT x0 = __ldcg(kcur + c0);
              ax = fma(v0.x, x0.x, fma(-v0.y, x0.y, ax));
              ay = fma(v0.x, x0.y, fma(v0.y, x0.x, ay));
            }
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) {
              ax += __shfl_xor_sync(0xffffffffu, ax, o, TPR);
              ay += __shfl_xor_sync(0xffffffffu, ay, o, TPR);
            }
            // every lane of a group holds its row's sum; lane L of this round's
            // range takes row rb + L from group L - q kGpw
            const int src = ((lane - q * kGpw) & (kGpw - 1)) * TPR;
            const R sx = __shfl_sync(0xffffffffu, ax, src);
            const R sy = __shfl_sync(0xffffffffu, ay, src);
            if (lane / kGpw == q) {
              mx = sx;
              my = sy;
            }
          }
          const long long r = rb + lane;
          if (r < a.n) ep.consume(r, mx * rscale, my * rscale);
        }
      }

      // ---- block reduction of the squared-norm maxima, one atomic per value
      unsigned long long km = warp_umax(ep.kmax);
      if (lane == 0) s_red[warp][0] = km;
#pragma unroll
      for (int u = 0; u < kKReg; ++u) {
        const unsigned long long fm = warp_umax(ep.fmax[u]);
        if (lane == 0) s_red[warp][1 + u] = fm;
      }
      __syncthreads();
      for (int q = tid; q <= J.d; q += kBlock) {
        if (q > 0 && !s_active[q - 1]) continue;
        unsigned long long m = 0;
        if (q <= kKReg) {
          for (int w = 0; w < kWarps; ++w) m = umax64(m, s_red[w][q]);
        } else {
          m = s_fmax_extra[q - 1];
        }
        atomicMax(&ctrl->gmax[slot3][q], as_bits(NormKey<VT>::value(m)));
      }
      if (blockIdx.x == 0) {
        const unsigned nx = (term + 1) % 3;
        for (int q = tid; q <= J.d; q += kBlock) ctrl->gmax[nx][q] = 0ULL;
        if (tid == 0) {
          ctrl->work[nx] = 0u;
          ctrl->work2[nx] = 0u;
          int act = 0;
          for (int k = 0; k < J.d; ++k) act += s_active[k];
          atomicAdd(&ctrl->matvecs, 1ULL);
          atomicAdd(&ctrl->fupdates, (unsigned long long)act);
        }
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

    // ---- Hermitian form: complete the caller's outputs from their upper triangles
    if ((OPK == kOpMatfreeHerm || OPK == kOpGlobalHerm) && a.mirror && J.final_outputs) {
      const long long tot = (long long)J.d * a.n;
      for (long long q = gthread; q < tot; q += nthreads) {
        const int k = (int)(q / a.n);
        const long long r = q % a.n;
        const int i = (int)(r % a.nt), j = (int)(r / a.nt);
        if (i <= j) continue;
        double2* F = slot_ptr(a, J.out_index0 + k);
        double2 z = __ldcg(F + j + (long long)a.nt * i);
        F[r] = make_double2(z.x, -z.y);
      }
      // the next block reads its input Z (this block's last output) in full
      if (!grid_barrier(ctrl)) return;
    }

    // ---- this block's outputs are final (every block is past the barrier
    // that ended the last term or the mirror pass): tell a host that copies
    // finished outputs out while the series runs
    if (a.progress && J.final_outputs && blockIdx.x == 0 && tid == 0) {
      __threadfence_system();
      *(volatile int*)a.progress = J.out_index0 + J.d;
    }

    // ---- populations of the finished outputs
    if (J.final_outputs && a.pops) {
      const long long tot = (long long)J.d * a.nt;
      for (long long q = gthread; q < tot; q += nthreads) {
        const int k = (int)(q / a.nt);
        const int v = (int)(q % a.nt);
        const double2 z = __ldcg(slot_ptr(a, J.out_index0 + k) + (long long)v * (a.nt + 1));
        a.pops[(long long)(J.out_index0 + k) * a.nt + v] = z.x;
      }
      if (a.ring) {
        if (!grid_barrier(ctrl)) return;   // ring slots are reused by the next job
      }
    }
  }
}

// The bounded wait of grid_barrier, exercised: block `absent` never arrives,
// so every other block gives up after `limit` polls and records kErrBarrier.
__global__ void __launch_bounds__(kBlock) barrier_probe_kernel(Ctrl* ctrl, int absent,
                                                               unsigned limit) {
  if ((int)blockIdx.x == absent) return;
  grid_barrier(ctrl, limit);
}

__global__ void plan_kernel(const double* __restrict__ dp, int prec, double t0, double dt,
                            int steps, int n0, int ring, Job* jobs, int max_jobs, int expect,
                            Ctrl* ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const PlanInfo info =
        plan_series(dp, c_theta[prec], t0, dt, steps, n0, ring, jobs, max_jobs, kDMax);
    ctrl->njobs = info.njobs;
    if (info.njobs != expect) ctrl->error = kErrPlan;
  }
}

// y = scale L x (or scale L^H x) for `cols` vectors stored one after another
// (n apart), matrix-free.  Blocks stride over the columns j of the density
// matrix.  PA: part A through the lane-interleaved lists (built for the
// operator's current values: MfData::pa_ready).
template <class R, class VT, bool ADJ, bool PA = false>
__global__ void __launch_bounds__(kBlock)
mf_apply_kernel(MfOp<R> op, int cols, const VT* __restrict__ x, VT* __restrict__ y, double scale) {
  const long long n = (long long)op.Nt * op.Nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = blockIdx.x; j < op.Nt; j += gridDim.x) {
    for (int i0 = warp * kItemRows; i0 < op.Nt; i0 += kWarps * kItemRows) {
      int irow[kRpt];
      mf_window_rows(op.prow, i0, lane, op.Nt - 1, irow);
      for (int c = 0; c < cols; ++c) {
        const VT* xc = x + c * n;
        R ox[kRpt], oy[kRpt];
        mf_window_apply<R, VT, ADJ, LdGlobal, PA>(op, xc, j, i0, irow, ox, oy);
#pragma unroll
        for (int u = 0; u < kRpt; ++u) {
          if (irow[u] < 0) continue;
          y[c * n + irow[u] + (long long)op.Nt * j] =
              Cplx<VT>::make(ox[u] * (R)scale, oy[u] * (R)scale);
        }
      }
    }
  }
}

template <class VT>
__global__ void apply_csr_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
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

// max |x_ij - conj(x_ji)|^2 and max |x_ij|^2 as bit patterns (one atomic per warp)
__global__ void herm_check_kernel(int nt, const double2* __restrict__ x,
                                  unsigned long long* __restrict__ out) {
  const long long n = (long long)nt * nt;
  unsigned long long da = 0, xa = 0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(r % nt), j = (int)(r / nt);
    const double2 u = x[r];
    const double2 v = x[j + (long long)nt * i];
    const double ex = u.x - v.x, ey = u.y + v.y;
    da = umax64(da, as_bits(ex * ex + ey * ey));
    xa = umax64(xa, as_bits(u.x * u.x + u.y * u.y));
  }
  da = warp_umax(da);
  xa = warp_umax(xa);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], da);
    atomicMax(&out[1], xa);
  }
}

__global__ void narrow_vec_kernel(long long n, const double2* __restrict__ in, float2* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

__global__ void widen_vec_kernel(long long n, const float2* __restrict__ in, double2* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = make_double2((double)in[e].x, (double)in[e].y);
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

__global__ void diag_state_kernel(int nt, long long n, const double* __restrict__ p,
                                  double2* __restrict__ state) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q % nt, j = q / nt;
    state[q] = make_double2(i == j ? p[i] : 0.0, 0.0);
  }
}

template <class VT, int OPK, int TPR, int UNR = 2>
cudaError_t launch_series(const SeriesArgs& a, int sms, cudaStream_t st, int* grid_out) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, series_kernel<VT, OPK, TPR, UNR>, kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const long long want =
      OPK == kOpCsr    ? ((long long)a.n + 32 * kWarps - 1) / (32 * kWarps)   // 32 rows per warp
      : OPK == kOpSell ? ((long long)a.slices + kWarps - 1) / kWarps           // a slice per warp
                       : (mf_item_count(a.nt, OPK == kOpMatfreeHerm) + kWarps - 1) / kWarps;
  const long long maxg = (long long)per_sm * sms;
  const int grid = (int)std::max<long long>(1, std::min(want, maxg));
  *grid_out = grid;
  SeriesArgs args = a;
  void* params[] = {&args};
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaLaunchCooperativeKernel((const void*)series_kernel<VT, OPK, TPR, UNR>, dim3(grid),
                                     dim3(kBlock), params, 0, st);
}

template <class VT>
cudaError_t launch_series_op(const Op& op, int tpr, int unr, bool herm, const SeriesArgs& a,
                             int sms, cudaStream_t st, int* g) {
  if (op.gq.active)
    return herm ? launch_series<VT, kOpGlobalHerm, 1>(a, sms, st, g)
                : launch_series<VT, kOpGlobal, 1>(a, sms, st, g);
  if (op.opkind == QSW_OPERATOR_MATRIX_FREE)
    return herm ? launch_series<VT, kOpMatfreeHerm, 1>(a, sms, st, g)
                : launch_series<VT, kOpMatfree, 1>(a, sms, st, g);
  if (tpr < 0)   // the sliced form (a.col, a.val and the slice arrays set by the caller)
    return unr == 4 ? launch_series<VT, kOpSell, 1, 4>(a, sms, st, g)
                    : launch_series<VT, kOpSell, 1, 2>(a, sms, st, g);
#define QSW_CSR_CASE(T)                                                        \
  case T:                                                                      \
    return unr == 4 ? launch_series<VT, kOpCsr, T, 4>(a, sms, st, g)           \
                    : launch_series<VT, kOpCsr, T, 2>(a, sms, st, g);
  switch (tpr) {
    QSW_CSR_CASE(1)
    QSW_CSR_CASE(2)
    QSW_CSR_CASE(4)
    QSW_CSR_CASE(8)
    QSW_CSR_CASE(16)
    default:
      return unr == 4 ? launch_series<VT, kOpCsr, 32, 4>(a, sms, st, g)
                      : launch_series<VT, kOpCsr, 32, 2>(a, sms, st, g);
  }
#undef QSW_CSR_CASE
}

}  // namespace

// Lanes per row without tuning: 2 was fastest on both measured superoperators
// (the 45 x 45 lattice, ~9 entries per row, complex64; the ER-1000 walk, ~40
// entries per row, complex128); very long rows get 4.
int choose_tpr(double avg_row) { return avg_row <= 96 ? 2 : 4; }

// ------------------------------------------------ autotuned CSR lanes per row
// The CSR sweep's lanes per row (TPR) set the cost of the shuffle reduction and
// how the operator stream is coalesced, its unroll depth (2 or 4 entries per
// lane in flight) how many loads each lane keeps waiting; the best pair depends
// on the row lengths, the precision and the size, and on the part.  The first CSR series
// on a device for a (precision, row-length bucket, size bucket) times every
// candidate pair with the series kernel itself on that operator (one job of
// kTuneTerms Taylor terms from a fixed vector, tolerance 0 so that every
// candidate runs the same terms, a warm-up launch then two timed launches) and
// keeps the fastest for the life of the process.  Results depend on the pair
// only through the summation order of each row.
namespace {

constexpr int kTuneTerms = 8;
constexpr int kTprCandidates[] = {1, 2, 4, 8, 16, 32};
constexpr int kUnrollCandidates[] = {2, 4};

struct TuneKey {
  int device, precision, row_bucket, n_bucket;
  bool operator<(const TuneKey& o) const {
    if (device != o.device) return device < o.device;
    if (precision != o.precision) return precision < o.precision;
    if (row_bucket != o.row_bucket) return row_bucket < o.row_bucket;
    return n_bucket < o.n_bucket;
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_tpr;   // (lanes per row, unroll)
std::atomic<long long> g_tune_measurements{0};

__global__ void tune_fill_kernel(long long n, double2* __restrict__ x) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = make_double2(1.0 / (1.0 + (double)(e % 97)), 1.0 / (2.0 + (double)(e % 89)));
}

TuneKey csr_tune_key(const Op& op) {
  const double avg = op.n > 0 ? (double)op.L.nnz / (double)op.n : 1.0;
  return TuneKey{op.ctx->device, (int)op.precision, (int)floor(2.0 * log2(avg > 1.0 ? avg : 1.0)),
                 (int)floor(log2((double)(op.n > 1 ? op.n : 1)))};
}

}  // namespace

long long tune_measurements() { return g_tune_measurements.load(); }

void tune_reset() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_tpr.clear();
}

// ------------------------------------------------------- sliced CSR form
namespace {

constexpr int kSellSigma = 4096;   // rows sorted by length within windows of this many

// Slice s, lane l: row perm[32 s + l] (-1: none), its CSR entries in order,
// then zero entries pointing at the row itself up to the slice's width.
template <class VT>
__global__ void sell_fill_kernel(int slices, const int* __restrict__ perm,
                                 const long long* __restrict__ off, const int* __restrict__ width,
                                 const int* __restrict__ rowptr, const int* __restrict__ ccol,
                                 const VT* __restrict__ cval, int* __restrict__ scol,
                                 VT* __restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long ws = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long sl = w0; sl < slices; sl += ws) {
    const int r = perm[sl * 32 + lane];
    const int e0 = r >= 0 ? rowptr[r] : 0;
    const int len = r >= 0 ? rowptr[r + 1] - e0 : 0;
    const int w = width[sl];
    VT zero;
    zero.x = 0;
    zero.y = 0;
    for (int k = 0; k < w; ++k) {
      const long long e = off[sl] + 32LL * k + lane;
      if (k < len) {
        scol[e] = ccol[e0 + k];
        sval[e] = cval[e0 + k];
      } else {
        scol[e] = r >= 0 ? r : 0;
        sval[e] = zero;
      }
    }
  }
}

}  // namespace

void build_sell(Op& op) {
  cudaStream_t st = op.ctx->stream;
  const long long n = op.n;
  std::vector<int> rp((size_t)n + 1);
  QSW_CUDA_TRY(cudaMemcpyAsync(rp.data(), op.L.rowptr.p, sizeof(int) * (n + 1),
                               cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  Sell& S = op.sell;
  S.slices = (int)((n + 31) / 32);
  std::vector<int> perm((size_t)S.slices * 32, -1);
  for (long long w0 = 0; w0 < n; w0 += kSellSigma) {
    const long long w1 = std::min(n, w0 + kSellSigma);
    for (long long r = w0; r < w1; ++r) perm[r] = (int)r;
    std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int x, int y) {
      return rp[x + 1] - rp[x] > rp[y + 1] - rp[y];
    });
  }
  std::vector<long long> off(S.slices);
  std::vector<int> width(S.slices);
  long long tot = 0;
  for (int sl = 0; sl < S.slices; ++sl) {
    int w = 0;
    for (int l = 0; l < 32; ++l) {
      const int r = perm[(size_t)sl * 32 + l];
      if (r >= 0) w = std::max(w, rp[r + 1] - rp[r]);
    }
    off[sl] = tot;
    width[sl] = w;
    tot += 32LL * w;
  }
  S.entries = tot;
  const size_t vb = op.L.fp32 ? sizeof(float2) : sizeof(double2);
  S.perm.alloc(sizeof(int) * perm.size());
  S.off.alloc(sizeof(long long) * off.size());
  S.width.alloc(sizeof(int) * width.size());
  S.col.alloc(sizeof(int) * (size_t)std::max(1LL, tot));
  S.val.alloc(vb * (size_t)std::max(1LL, tot));
  QSW_CUDA_TRY(cudaMemcpyAsync(S.perm.p, perm.data(), sizeof(int) * perm.size(),
                               cudaMemcpyHostToDevice, st));
  QSW_CUDA_TRY(cudaMemcpyAsync(S.off.p, off.data(), sizeof(long long) * off.size(),
                               cudaMemcpyHostToDevice, st));
  QSW_CUDA_TRY(cudaMemcpyAsync(S.width.p, width.data(), sizeof(int) * width.size(),
                               cudaMemcpyHostToDevice, st));
  const unsigned grid = grid_for((long long)S.slices * 32, 256, 152 * 16);
  if (op.L.fp32)
    QSW_LAUNCH sell_fill_kernel<float2><<<grid, 256, 0, st>>>(
        S.slices, S.perm.as<int>(), S.off.as<long long>(), S.width.as<int>(),
        op.L.rowptr.as<int>(), op.L.col.as<int>(), op.L.val.as<float2>(), S.col.as<int>(),
        S.val.as<float2>());
  else
    QSW_LAUNCH sell_fill_kernel<double2><<<grid, 256, 0, st>>>(
        S.slices, S.perm.as<int>(), S.off.as<long long>(), S.width.as<int>(),
        op.L.rowptr.as<int>(), op.L.col.as<int>(), op.L.val.as<double2>(), S.col.as<int>(),
        S.val.as<double2>());
  QSW_CUDA_TRY(cudaGetLastError());
  QSW_CUDA_TRY(cudaStreamSynchronize(st));   // the host arrays above are released on return
}

namespace {
// Points a series' operator arguments at the sliced form.
void set_sell_args(const Op& op, SeriesArgs& a) {
  a.col = op.sell.col.as<int>();
  a.val = op.sell.val.p;
  a.sperm = op.sell.perm.as<int>();
  a.soff = op.sell.off.as<long long>();
  a.swidth = op.sell.width.as<int>();
  a.slices = op.sell.slices;
}
}  // namespace

void tune_csr_schedule(Op& op) {
  const TuneKey key = csr_tune_key(op);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_tpr.find(key);
    if (it != g_tune_tpr.end()) {
      op.csr_sell = it->second.first < 0;
      if (!op.csr_sell) op.tpr = it->second.first;
      op.csr_unroll = it->second.second;
      return;
    }
  }
  cudaStream_t st = op.ctx->stream;
  const bool f32 = op.precision == QSW_C64_BULK;
  const size_t vbytes = f32 ? sizeof(float2) : sizeof(double2);
  DevBuf x, kbuf, slot, ctrl, job;
  x.alloc(sizeof(double2) * (size_t)op.n);
  kbuf.alloc(2 * vbytes * (size_t)op.n);
  slot.alloc(sizeof(double2) * (size_t)op.n);
  ctrl.alloc(sizeof(Ctrl));
  job.alloc(sizeof(Job));
  QSW_LAUNCH tune_fill_kernel<<<grid_for(op.n, 256, 4096), 256, 0, st>>>(op.n, x.as<double2>());
  QSW_CUDA_TRY(cudaGetLastError());
  Job j{};
  j.z_slot = -1;
  j.d = 1;
  j.m = kTuneTerms;
  j.d_block = 1;
  j.hspan = op.dp[0] > 0.0 ? 1.0 / op.dp[0] : 1.0;   // terms shrink: no overflow
  QSW_CUDA_TRY(cudaMemcpyAsync(job.p, &j, sizeof(Job), cudaMemcpyHostToDevice, st));
  SeriesArgs a{};
  a.n = (int)op.n;
  a.nt = op.Nt;
  a.rowptr = op.L.rowptr.as<int>();
  a.col = op.L.col.as<int>();
  a.val = op.L.val.p;
  a.k0 = kbuf.p;
  a.k1 = static_cast<char*>(kbuf.p) + vbytes * (size_t)op.n;
  a.rho0 = x.as<double2>();
  a.slots = slot.as<double2>();
  a.jobs = job.as<Job>();
  a.njobs = 1;
  a.ctrl = ctrl.as<Ctrl>();
  a.tol = 0.0;
  cudaEvent_t e0, e1;
  QSW_CUDA_TRY(cudaEventCreate(&e0));
  QSW_CUDA_TRY(cudaEventCreate(&e1));
  std::pair<int, int> best{op.tpr, op.csr_unroll};
  float best_ms = 0.f;
  // the candidates: TPR lanes per row on the CSR arrays, and the sliced form
  // (lanes per row -1), each with both unroll depths
  std::vector<int> tprs(std::begin(kTprCandidates), std::end(kTprCandidates));
  tprs.push_back(-1);
  if (op.sell.slices == 0) build_sell(op);
  SeriesArgs as = a;
  set_sell_args(op, as);
  for (int tpr : tprs)
  for (int unr : kUnrollCandidates) {
    const SeriesArgs& aa = tpr < 0 ? as : a;
    float tmin = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      QSW_CUDA_TRY(cudaMemsetAsync(ctrl.p, 0, sizeof(Ctrl), st));
      QSW_CUDA_TRY(cudaEventRecord(e0, st));
      int grid = 0;
      QSW_CUDA_TRY(f32 ? launch_series_op<float2>(op, tpr, unr, false, aa, op.ctx->num_sms, st, &grid)
                       : launch_series_op<double2>(op, tpr, unr, false, aa, op.ctx->num_sms, st, &grid));
      QSW_CUDA_TRY(cudaEventRecord(e1, st));
      QSW_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      QSW_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1 || (rep > 1 && ms < tmin)) tmin = ms;
    }
    Ctrl h{};
    QSW_CUDA_TRY(cudaMemcpyAsync(&h, ctrl.p, offsetof(Ctrl, gmax), cudaMemcpyDeviceToHost, st));
    QSW_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.error != kErrNone)
      throw Error{QSW_ERR_NOT_CONVERGED, "CSR schedule tuning: grid barrier wait exceeded its limit"};
    if (best_ms == 0.f || tmin < best_ms) {
      best_ms = tmin;
      best = {tpr, unr};
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_tune_measurements.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const auto chosen = g_tune_tpr.emplace(key, best).first->second;   // a concurrent tuner may have won
  op.csr_sell = chosen.first < 0;
  if (!op.csr_sell) {
    op.tpr = chosen.first;
    op.sell = Sell{};   // the sliced copy of the operator is not kept
  }
  op.csr_unroll = chosen.second;
}

void upload_theta_batch();

// The theta tables live in __constant__ memory, one copy per device: they are
// written once per device (the first context on it), so that contexts created
// later (e.g. a server's workers) never rewrite them under running kernels.
void upload_theta(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  QSW_CHECK_ARG(device >= 0 && device < 64, QSW_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (done[device]) return;
  upload_theta_batch();
  QSW_CUDA_TRY(cudaMemcpyToSymbol(c_theta, theta_table(QSW_C128), sizeof(double) * kMMax, 0));
  QSW_CUDA_TRY(cudaMemcpyToSymbol(c_theta, theta_table(QSW_C64_BULK), sizeof(double) * kMMax,
                                  sizeof(double) * kMMax));
  QSW_CUDA_TRY(cudaDeviceSynchronize());   // the tables are in place before any launch
  done[device] = true;
}

template <class R> MfOp<R> make_mf(const Op& op, bool adjoint) {
  const MfData& m = op.mf;
  const bool f = sizeof(R) == sizeof(float);
  MfOp<R> o;
  o.N = op.omega < 1.0 ? op.N : 0;   // the commutator vanishes at omega = 1
  o.Nt = op.Nt;
  o.hrow = op.g.hoff_rowptr.as<int>();
  o.hcol = op.g.hoff_col.as<int>();
  o.hval = static_cast<const R*>(f ? m.hval32.p : m.hval64.p);
  o.ad = static_cast<const R*>(f ? m.ad32.p : m.ad64.p);
  o.hw = static_cast<const R*>(f ? m.hw32.p : m.hw64.p);
  o.jrow = adjoint ? op.g.jt_rowptr.as<int>() : op.g.j_rowptr.as<int>();
  o.jcol = adjoint ? op.g.jt_col.as<int>() : op.g.j_col.as<int>();
  o.jval = static_cast<const R*>(adjoint ? (f ? m.jtval32.p : op.g.jt_val.p)
                                         : (f ? m.jval32.p : op.g.j_val.p));
  o.prow = m.prow.as<int>();
  o.pwin = m.pwin.as<int>();
  o.paoff = m.paoff.as<int>();
  o.pacol = m.pacol.as<int>();
  o.paval = static_cast<const R*>(f ? m.paval32.p : m.paval64.p);
  return o;
}
template MfOp<double> make_mf<double>(const Op&, bool);
template MfOp<float> make_mf<float>(const Op&, bool);

void mf_apply64(const Op& op, bool adjoint, int cols, const double* x, double* y, double scale) {
  const MfOp<double> m = make_mf<double>(op, adjoint);
  const unsigned grid = (unsigned)std::min(op.Nt, 152 * 8);
  const double2* xv = reinterpret_cast<const double2*>(x);
  double2* yv = reinterpret_cast<double2*>(y);
  cudaStream_t st = op.ctx->stream;
  if (op.mf.pa_ready) {
    if (adjoint)
      QSW_LAUNCH mf_apply_kernel<double, double2, true, true><<<grid, kBlock, 0, st>>>(m, cols, xv, yv, scale);
    else
      QSW_LAUNCH mf_apply_kernel<double, double2, false, true><<<grid, kBlock, 0, st>>>(m, cols, xv, yv, scale);
  } else {
    if (adjoint)
      QSW_LAUNCH mf_apply_kernel<double, double2, true><<<grid, kBlock, 0, st>>>(m, cols, xv, yv, scale);
    else
      QSW_LAUNCH mf_apply_kernel<double, double2, false><<<grid, kBlock, 0, st>>>(m, cols, xv, yv, scale);
  }
  QSW_CUDA_TRY(cudaGetLastError());
}

// The same in complex64 with the FP32 coefficients (the 1-norm estimator's
// ranking products).
void mf_apply32(const Op& op, bool adjoint, int cols, const float* x, float* y, double scale) {
  QSW_CHECK_ARG(op.mf.pa_ready, QSW_ERR_CUDA, "estimator products before the part-A lists");
  const MfOp<float> m = make_mf<float>(op, adjoint);
  const unsigned grid = (unsigned)std::min(op.Nt, 152 * 8);
  const float2* xv = reinterpret_cast<const float2*>(x);
  float2* yv = reinterpret_cast<float2*>(y);
  if (adjoint)
    QSW_LAUNCH mf_apply_kernel<float, float2, true, true><<<grid, kBlock, 0, op.ctx->stream>>>(
        m, cols, xv, yv, scale);
  else
    QSW_LAUNCH mf_apply_kernel<float, float2, false, true><<<grid, kBlock, 0, op.ctx->stream>>>(
        m, cols, xv, yv, scale);
  QSW_CUDA_TRY(cudaGetLastError());
}

double op_bytes(const Op& op) {
  const bool f32 = op.precision == QSW_C64_BULK;
  if (op.gq.active)   // Q and L' rows: column index + complex value
    return (double)(op.gq.nnz_q + op.gq.nnz_l) * (4.0 + (f32 ? sizeof(float2) : sizeof(double2)));
  if (op.opkind == QSW_OPERATOR_CSR)
    return (double)op.L.nnz * ((f32 ? sizeof(float2) : sizeof(double2)) + 4) +
           (double)(op.n + 1) * 4;
  // matrix-free: H off-diagonal (col + value) and the per-vertex coefficients
  const double rb = f32 ? 4.0 : 8.0;
  return (double)op.g.nnz_hoff * (4 + rb) + (double)op.Nt * 2 * rb;
}

// Plan figures and the algorithmic byte / flop counts of one series call, from
// the plan and the kernel's counters (every series entry point reports these).
void fill_series_stats(const Op& op, const PlanInfo& info, unsigned long long matvecs,
                       unsigned long long fupdates, bool herm, qsw_series_stats* stats) {
  const bool f32 = op.precision == QSW_C64_BULK;
  const double vbytes = f32 ? sizeof(float2) : sizeof(double2);
  stats->m0 = info.m0;
  stats->s0 = info.s0;
  stats->m_star = info.m_star;
  stats->s = info.s;
  stats->step_m = info.step_m;
  stats->step_s = info.step_s;
  stats->outputs_per_block = info.d;
  stats->jobs = info.njobs;
  stats->matvecs = (int64_t)matvecs;
  stats->fupdates = (int64_t)fupdates;
  // per job: read Z and write Khat_0; per output: one copy of Z
  const double init_bytes =
      (16.0 + vbytes) * (double)op.n * info.njobs + 16.0 * (double)op.n * info.outputs;
  // the Hermitian form computes the upper triangle: (N~+1)/(2N~) of the
  // off-diagonal terms and N~(N~+1)/2 elements
  const double frac = herm ? (op.Nt + 1.0) / (2.0 * op.Nt) : 1.0;
  const double elems = frac * (double)op.n;
  double flops_per_matvec;
  double wbytes = 0.0;   // global walks: pass A writes and pass B reads the W products
  if (op.gq.active) {
    // pass A: 8 flops per (element, entry of row j of L'); pass B: 8 per
    // entry of rows i and j of Q and of row i of L' (complex products)
    const double nt = op.Nt;
    flops_per_matvec = 8.0 * nt * (double)op.gq.nnz_l +
                       frac * 8.0 * nt * (2.0 * (double)op.gq.nnz_q + (double)op.gq.nnz_l) +
                       5.0 * elems;
    wbytes = 2.0 * vbytes * (double)op.gq.nl * (double)op.n;
  } else {
    const double offdiag_terms = frac * (double)(op.nnz_csr - op.n - op.g.n_jumps);
    flops_per_matvec = 4.0 * offdiag_terms + 8.0 * elems + 4.0 * op.g.n_jumps + 5.0 * elems;
  }
  // one application: the operator's own data, reading the input once and
  // writing the output once (the elements computed)
  stats->bytes_per_matvec = op_bytes(op) + 2.0 * elems * vbytes + wbytes;
  stats->algorithmic_bytes = (double)matvecs * stats->bytes_per_matvec +
                             32.0 * elems * (double)fupdates + init_bytes;
  stats->algorithmic_flops = (double)matvecs * flops_per_matvec + 7.0 * elems * fupdates;
  stats->hermitian = herm ? 1 : 0;
  stats->kernel_ms = 0.0;
}

void run_series(Op& op, const double* d_rho0, double t0, double dt, int steps, double* d_out,
                double* d_pops, qsw_series_stats* stats, const OutputSink* sink) {
  cudaStream_t st = op.ctx->stream;
  const int prec = op.precision == QSW_C64_BULK ? 1 : 0;
  const double* theta = theta_table(op.precision);
  // Host copy of the plan: sizes only (the device plans for itself below).
  const PlanInfo info = plan_series(op.dp, theta, t0, dt, steps, 1, 0, nullptr, 0, kDMax);
  const int ring = d_out ? 0 : info.max_d + 1;
  const bool f32 = op.precision == QSW_C64_BULK;
  const size_t vbytes = f32 ? sizeof(float2) : sizeof(double2);
  if (op.opkind == QSW_OPERATOR_CSR && !op.tpr_fixed) {   // first CSR series: tuned schedule
    tune_csr_schedule(op);
    op.tpr_fixed = true;
  }
  if (op.opkind == QSW_OPERATOR_CSR && op.csr_sell && op.sell.slices == 0) build_sell(op);
  op.kbuf.alloc(2 * vbytes * (size_t)op.n);
  if (!d_out) op.ring.alloc(sizeof(double2) * (size_t)op.n * ring);
  op.jobs.alloc(sizeof(Job) * std::max(1, info.njobs));
  op.ctrl.alloc(sizeof(Ctrl));
  QSW_CUDA_TRY(cudaMemsetAsync(op.ctrl.p, 0, sizeof(Ctrl), st));
  QSW_LAUNCH plan_kernel<<<1, 32, 0, st>>>(op.dp_dev.as<double>(), prec, t0, dt, steps, 1, ring,
                                           op.jobs.as<Job>(), info.njobs, info.njobs,
                                           op.ctrl.as<Ctrl>());
  QSW_CUDA_TRY(cudaGetLastError());

  // Hermitian input (every density matrix): L~ maps Hermitian matrices to
  // Hermitian matrices, so every Taylor term and output is Hermitian and the
  // matrix-free form computes only the upper triangle.
  bool herm = false;
  if (op.opkind == QSW_OPERATOR_MATRIX_FREE) {
    op.scratch.alloc(2 * sizeof(unsigned long long));
    QSW_CUDA_TRY(cudaMemsetAsync(op.scratch.p, 0, 2 * sizeof(unsigned long long), st));
    QSW_LAUNCH herm_check_kernel<<<grid_for(op.n, 256, 152 * 8), 256, 0, st>>>(
        op.Nt, reinterpret_cast<const double2*>(d_rho0), op.scratch.as<unsigned long long>());
    QSW_CUDA_TRY(cudaGetLastError());
    unsigned long long hb[2] = {0, 0};
    QSW_CUDA_TRY(cudaMemcpyAsync(hb, op.scratch.p, sizeof(hb), cudaMemcpyDeviceToHost, st));
    QSW_CUDA_TRY(cudaStreamSynchronize(st));
    double asym2, max2;
    memcpy(&asym2, &hb[0], sizeof(double));
    memcpy(&max2, &hb[1], sizeof(double));
    herm = sqrt(asym2) <= 1e-13 * (sqrt(max2) > 1.0 ? sqrt(max2) : 1.0);
  }

  SeriesArgs a{};
  a.n = (int)op.n;
  a.nt = op.Nt;
  a.mirror = herm && d_out != nullptr;
  const bool sell = op.opkind == QSW_OPERATOR_CSR && op.csr_sell && op.sell.slices > 0;
  if (op.opkind == QSW_OPERATOR_CSR) {
    a.rowptr = op.L.rowptr.as<int>();
    a.col = op.L.col.as<int>();
    a.val = op.L.val.p;
    if (sell) set_sell_args(op, a);
  } else if (op.gq.active) {
    a.gq64 = make_gq<double>(op, false);
    a.gq32 = make_gq<float>(op, false);
    op.scratch_w.alloc(vbytes * (size_t)(op.gq.nl + 1) * (size_t)op.n);   // W_k, then R
    a.wbuf = op.scratch_w.p;
  } else {
    a.mf64 = make_mf<double>(op, false);
    a.mf32 = make_mf<float>(op, false);
  }
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
  a.progress = (sink && d_out) ? sink->d_count : nullptr;

  cudaEvent_t ev0, ev1;
  QSW_CUDA_TRY(cudaEventCreate(&ev0));
  QSW_CUDA_TRY(cudaEventCreate(&ev1));
  QSW_CUDA_TRY(cudaEventRecord(ev0, st));
  int grid = 0;
  const int tpr = sell ? -1 : op.tpr;
  cudaError_t e = f32 ? launch_series_op<float2>(op, tpr, op.csr_unroll, herm, a, op.ctx->num_sms, st, &grid)
                      : launch_series_op<double2>(op, tpr, op.csr_unroll, herm, a, op.ctx->num_sms, st, &grid);
  QSW_CUDA_TRY(e);
  QSW_CUDA_TRY(cudaEventRecord(ev1, st));
  Ctrl h{};
  QSW_CUDA_TRY(cudaMemcpyAsync(&h, op.ctrl.p, offsetof(Ctrl, gmax), cudaMemcpyDeviceToHost, st));
  if (a.progress) {
    // hand finished outputs to the sink while the kernel runs; the loop ends
    // when the kernel has (its grid barriers bound every wait inside it).  The
    // thread yields between polls instead of sleeping: on a loaded host a
    // timed sleep overslept by up to ~15 ms now and then, which delayed the
    // last copies by as much.
    int seen = 0;
    for (;;) {
      const bool done = cudaEventQuery(ev1) != cudaErrorNotReady;
      const int k = *(volatile int*)sink->h_count;
      if (k > seen) {
        sink->ready(k);
        seen = k;
      }
      if (done) break;
      std::this_thread::yield();
    }
  }
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
    fill_series_stats(op, info, h.matvecs, h.fupdates, herm, stats);
    stats->kernel_ms = ms;
  }
}

// ----------------------------------------------- series without allocation
// Scratch of qsw_expmv_series_noalloc: one fixed array per device, reserved
// when the module loads, so the call itself never asks the allocator for
// memory.  Layout per call (each part starts on a 256-byte boundary):
//   Ctrl | Hermiticity-check words | Job[njobs] | K0 K1 | output ring
// Ctrl and the check words must start at zero and are cleared by every call;
// the rest is written before it is read.  Every call on a device uses the
// same array: two calls in flight at the same time on one device race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QSW_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kNoAllocDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the first call on a device does this set-up).  The address is
// kept for the life of the process: it assumes the device's primary context
// lives as long (a cudaDeviceReset would leave a stale address behind).
unsigned char* noalloc_base(int device) {
  QSW_CHECK_ARG(device >= 0 && device < kNoAllocDevices, QSW_ERR_INVALID_ARG,
                "device index beyond the no-allocation scratch table");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error{QSW_ERR_CUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                                    cudaGetErrorString(e)};
    g_noalloc_base[device] = p;
  }
  return static_cast<unsigned char*>(g_noalloc_base[device]);
}

}  // namespace

void run_series_noalloc(Op& op, const double* d_rho0, double t0, double dt, int steps,
                        double* d_out, double* d_pops, qsw_series_stats* stats) {
  cudaStream_t st = op.ctx->stream;
  const int prec = op.precision == QSW_C64_BULK ? 1 : 0;
  const double* theta = theta_table(op.precision);
  const PlanInfo info = plan_series(op.dp, theta, t0, dt, steps, 1, 0, nullptr, 0, kDMax);
  const int ring = d_out ? 0 : info.max_d + 1;
  const bool f32 = op.precision == QSW_C64_BULK;
  const size_t vbytes = f32 ? sizeof(float2) : sizeof(double2);

  const size_t off_herm = align256(sizeof(Ctrl));
  const size_t off_jobs = off_herm + align256(2 * sizeof(unsigned long long));
  const size_t off_k = off_jobs + align256(sizeof(Job) * (size_t)std::max(1, info.njobs));
  const size_t off_ring = off_k + align256(2 * vbytes * (size_t)op.n);
  const size_t need = off_ring + sizeof(double2) * (size_t)op.n * (size_t)ring;
  if (need > (size_t)QSW_NOALLOC_SCRATCH_BYTES)
    throw Error{QSW_ERR_TOO_LARGE,
                "series needs " + std::to_string(need) + " bytes of scratch; the no-allocation "
                "entry point has " + std::to_string((size_t)QSW_NOALLOC_SCRATCH_BYTES) +
                " (use qsw_expmv_series, or pass d_out to drop the output ring)"};

  unsigned char* base = noalloc_base(op.ctx->device);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(base);
  unsigned long long* hwords = reinterpret_cast<unsigned long long*>(base + off_herm);
  Job* jobs = reinterpret_cast<Job*>(base + off_jobs);
  void* kbuf = base + off_k;
  double2* ringbuf = reinterpret_cast<double2*>(base + off_ring);

  QSW_CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
  QSW_LAUNCH plan_kernel<<<1, 32, 0, st>>>(op.dp_dev.as<double>(), prec, t0, dt, steps, 1, ring,
                                           jobs, info.njobs, info.njobs, ctrl);
  QSW_CUDA_TRY(cudaGetLastError());

  bool herm = false;
  if (op.opkind == QSW_OPERATOR_MATRIX_FREE) {
    QSW_CUDA_TRY(cudaMemsetAsync(hwords, 0, 2 * sizeof(unsigned long long), st));
    QSW_LAUNCH herm_check_kernel<<<grid_for(op.n, 256, 152 * 8), 256, 0, st>>>(
        op.Nt, reinterpret_cast<const double2*>(d_rho0), hwords);
    QSW_CUDA_TRY(cudaGetLastError());
    unsigned long long hb[2] = {0, 0};
    QSW_CUDA_TRY(cudaMemcpyAsync(hb, hwords, sizeof(hb), cudaMemcpyDeviceToHost, st));
    QSW_CUDA_TRY(cudaStreamSynchronize(st));
    double asym2, max2;
    memcpy(&asym2, &hb[0], sizeof(double));
    memcpy(&max2, &hb[1], sizeof(double));
    herm = sqrt(asym2) <= 1e-13 * (sqrt(max2) > 1.0 ? sqrt(max2) : 1.0);
  }

  SeriesArgs a{};
  a.n = (int)op.n;
  a.nt = op.Nt;
  a.mirror = herm && d_out != nullptr;
  // the sliced form only when it is already built (this path allocates nothing)
  const bool sell = op.opkind == QSW_OPERATOR_CSR && op.csr_sell && op.sell.slices > 0;
  if (op.opkind == QSW_OPERATOR_CSR) {
    a.rowptr = op.L.rowptr.as<int>();
    a.col = op.L.col.as<int>();
    a.val = op.L.val.p;
    if (sell) set_sell_args(op, a);
  } else {
    a.mf64 = make_mf<double>(op, false);
    a.mf32 = make_mf<float>(op, false);
  }
  a.k0 = kbuf;
  a.k1 = static_cast<char*>(kbuf) + vbytes * (size_t)op.n;
  a.rho0 = reinterpret_cast<const double2*>(d_rho0);
  a.slots = d_out ? reinterpret_cast<double2*>(d_out) : ringbuf;
  a.ring = ring;
  a.pops = d_pops;
  a.jobs = jobs;
  a.njobs = info.njobs;
  a.ctrl = ctrl;
  a.tol = tolerance(op.precision);

  int grid = 0;
  const int tpr = sell ? -1 : op.tpr;
  cudaError_t e = f32 ? launch_series_op<float2>(op, tpr, op.csr_unroll, herm, a, op.ctx->num_sms, st, &grid)
                      : launch_series_op<double2>(op, tpr, op.csr_unroll, herm, a, op.ctx->num_sms, st, &grid);
  QSW_CUDA_TRY(e);
  Ctrl h{};
  QSW_CUDA_TRY(cudaMemcpyAsync(&h, ctrl, offsetof(Ctrl, gmax), cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.error == kErrBarrier)
    throw Error{QSW_ERR_NOT_CONVERGED, "series kernel: grid barrier wait exceeded its limit"};
  if (h.error == kErrPlan)
    throw Error{QSW_ERR_CUDA, "series kernel: device plan differs from host plan"};
  // the same figures as qsw_expmv_series, except kernel_ms (no timing events)
  if (stats) fill_series_stats(op, info, h.matvecs, h.fupdates, herm, stats);
}

double probe_wait_limit(qsw_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  DevBuf ctrl;
  ctrl.alloc(sizeof(Ctrl));
  QSW_CUDA_TRY(cudaMemsetAsync(ctrl.p, 0, sizeof(Ctrl), st));
  int per_sm = 0;
  QSW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_probe_kernel, kBlock, 0));
  const int grid = std::max(2, std::min(per_sm, 1) * ctx->num_sms);
  Ctrl* c = ctrl.as<Ctrl>();
  int absent = 0;
  unsigned limit = 1u << 20;   // ~1 s of polling
  void* params[] = {&c, &absent, &limit};
  cudaEvent_t e0, e1;
  QSW_CUDA_TRY(cudaEventCreate(&e0));
  QSW_CUDA_TRY(cudaEventCreate(&e1));
  QSW_CUDA_TRY(cudaEventRecord(e0, st));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  QSW_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)barrier_probe_kernel, dim3(grid),
                                           dim3(kBlock), params, 0, st));
  QSW_CUDA_TRY(cudaEventRecord(e1, st));
  Ctrl h{};
  QSW_CUDA_TRY(cudaMemcpyAsync(&h, ctrl.p, offsetof(Ctrl, gmax), cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (h.error != kErrBarrier)
    throw Error{QSW_ERR_CUDA, "barrier probe: the bounded wait did not report its timeout"};
  return ms * 1e-3;
}

void apply(const Op& op, const double* d_x, double* d_y) {
  if (op.gq.active) {
    gq_apply64(op, false, 1, d_x, d_y, 1.0);
    return;
  }
  cudaStream_t st = op.ctx->stream;
  const int n = (int)op.n;
  if (op.opkind == QSW_OPERATOR_MATRIX_FREE) {
    if (op.precision == QSW_C64_BULK) {
      DevBuf xs, ys;
      xs.alloc(sizeof(float2) * op.n);
      ys.alloc(sizeof(float2) * op.n);
      QSW_LAUNCH narrow_vec_kernel<<<grid_for(op.n, 256, 4096), 256, 0, st>>>(
          op.n, reinterpret_cast<const double2*>(d_x), xs.as<float2>());
      const MfOp<float> m = make_mf<float>(op, false);
      QSW_LAUNCH mf_apply_kernel<float, float2, false><<<std::min(op.Nt, 152 * 8), kBlock, 0, st>>>(
          m, 1, xs.as<float2>(), ys.as<float2>(), 1.0);
      QSW_LAUNCH widen_vec_kernel<<<grid_for(op.n, 256, 4096), 256, 0, st>>>(
          op.n, ys.as<float2>(), reinterpret_cast<double2*>(d_y));
      QSW_CUDA_TRY(cudaGetLastError());
      QSW_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      mf_apply64(op, false, 1, d_x, d_y, 1.0);
    }
    return;
  }
  const unsigned grid = grid_for((long long)n * 8, 256, 152 * 16);
  if (op.L.fp32)
    QSW_LAUNCH apply_csr_kernel<float2><<<grid, 256, 0, st>>>(
        n, op.L.rowptr.as<int>(), op.L.col.as<int>(), op.L.val.as<float2>(),
        reinterpret_cast<const double2*>(d_x), reinterpret_cast<double2*>(d_y));
  else
    QSW_LAUNCH apply_csr_kernel<double2><<<grid, 256, 0, st>>>(
        n, op.L.rowptr.as<int>(), op.L.col.as<int>(), op.L.val.as<double2>(),
        reinterpret_cast<const double2*>(d_x), reinterpret_cast<double2*>(d_y));
  QSW_CUDA_TRY(cudaGetLastError());
}

void populations(const Op& op, const double* d_rho, int count, double* d_pops) {
  cudaStream_t st = op.ctx->stream;
  QSW_LAUNCH pops_kernel<<<grid_for((long long)count * op.Nt, 256, 4096), 256, 0, st>>>(
      count, op.Nt, op.n, reinterpret_cast<const double2*>(d_rho), d_pops);
  QSW_CUDA_TRY(cudaGetLastError());
}

void widen_values(const Op& op, double* d_val) {
  QSW_LAUNCH widen_vec_kernel<<<grid_for(op.L.nnz, 256, 4096), 256, 0, op.ctx->stream>>>(
      op.L.nnz, op.L.val.as<float2>(), reinterpret_cast<double2*>(d_val));
  QSW_CUDA_TRY(cudaGetLastError());
}

void initial_state_from_pops(const Op& op, const double* d_pops, double* d_state) {
  cudaStream_t st = op.ctx->stream;
  QSW_LAUNCH diag_state_kernel<<<grid_for(op.n, 256, 4096), 256, 0, st>>>(
      op.Nt, op.n, d_pops, reinterpret_cast<double2*>(d_state));
  QSW_CUDA_TRY(cudaGetLastError());
}

}  // namespace qsw
