// The 1-norm series of L~ (paper Section 4 footnote: {||L~^p||_1, p = 1..9},
// computed once per operator and reused for every t at the same omega).
//
//   ||L~||_1 exactly: the largest row sum of moduli of L~^H (= largest column
//   sum of L~), a max-reduction, hence deterministic.
//   ||L~^p||_1, p = 2..9: the block 1-norm estimator of Higham & Tisseur
//   (2000, Algorithm 2.4), complex form (sign(z) = z/|z|, sign(0) = 1, products
//   with (L~^H)^p, no parallel-column tests), t = 2 columns, itmax = 5.  The
//   starting block is [1, x] / n with x_i = +-1 from the counter-based
//   SplitMix64 generator (Steele, Lea & Flood 2014) at a fixed seed; ties in
//   the row-norm ranking go to the smaller index.
//
// The products that give the estimates (Y = A^p X and its column norms) run in
// FP64 on the device, so every estimate is the FP64 1-norm of A^p x for a
// column x the algorithm tried.  The adjoint step Z = (A^H)^p sign(Y) only
// ranks the rows of Z by their largest modulus (which unit vectors to try
// next, and the stop test on the best one); for the matrix-free L-QSW
// operator it runs in complex64 with FP32 coefficients, scaled by 1/||A||_1
// per product.  Where rounding at that precision reorders two nearly equal
// row maxima, the estimator follows another branch Algorithm 2.4 allows; the
// GB300's FP32 pipe issues 64 times the FP64 rate, which takes the adjoint
// products off the FP64 pipe that bounds every other product.  The host only
// follows the algorithm's branches on the few scalars each iteration returns
// (one read-back for the column norms, one for the row ranking).
// All reductions use a fixed grid and a fixed summation order, so repeated
// builds give bit-identical estimates.
//
// Work shared between the estimates (same values up to rounding, fewer
// products):
//   * the first iteration of every estimate starts from the same block X0, so
//     A^p X0 for p = 1..9 is one chain;
//   * later iterations start from unit vectors e_c, and the estimates for
//     successive p often pick the same c: A^k e_c is kept per c and extended,
//     so A^p e_c costs p - k products instead of p;
//   * for the matrix-free L-QSW operator A^k e_c is zero outside a box of rows
//     x columns that grows by one H-neighbourhood per product; the products
//     visit only that box (the elements they compute are the ones the full
//     product computes, in the same order);
//   * on graphs where that box stays small (lattices), the adjoint step takes
//     (A^H)^p sign(Y) = (A^H)^p 1 + (A^H)^p (sign(Y) - 1): the first term is one
//     chain shared by every estimate, the second is supported on the box of Y;
//   * L~ and L~^H map X^dag to (L X)^dag: both columns of the starting block
//     (all ones, and random signs drawn symmetric under the transpose of the
//     density-matrix index) are Hermitian, so their products are taken on the
//     upper triangle and mirrored, and a unit-vector pair e_(a,b), e_(b,a) (the
//     row ranking ties them) costs one column, the other being its mirror.
// The last two change the rounding of some products, not their values.
#include <math.h>
#include <stddef.h>

#include <algorithm>

#include "matfree.cuh"
#include "op.h"

namespace qsw {
namespace {

constexpr int kRedBlock = 256;
constexpr int kRedGrid = 512;
constexpr unsigned long long kSeed = 0x51535700ULL;
constexpr int kItMax = 5;
constexpr int kMaxExcl = 16;

__device__ __forceinline__ double cabs(double2 z) { return hypot(z.x, z.y); }

// |z| for the estimator's vector passes: sqrt(x^2 + y^2) where the sum of
// squares neither overflows nor underflows, hypot otherwise.  On this FP64-lean
// part hypot's scaling costs several times the issue slots of the plain form,
// and these passes run over every element of every block the estimator forms.
__device__ __forceinline__ double cabs_fast(double2 z) {
  const double s = fma(z.x, z.x, z.y * z.y);
  if (s < 1e300 && (s > 1e-300 || (z.x == 0.0 && z.y == 0.0))) return sqrt(s);
  return hypot(z.x, z.y);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long i) {
  unsigned long long z = seed + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Y = A X for t column vectors stored n apart (CSR operator), 8 lanes per row.
__global__ void spmm_kernel(int n, int t, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double2* __restrict__ val, const double2* __restrict__ X,
                            double2* __restrict__ Y) {
  constexpr int G = 8;
  const int lane = threadIdx.x % G;
  const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const long long stride = (long long)gridDim.x * blockDim.x / G;
  // warp-uniform row loop: every lane takes part in the group shuffles
  for (long long rb = wg * (32 / G); rb < n; rb += stride) {
    const long long r = rb + (threadIdx.x % 32) / G;
    const bool valid = r < n;
    const int e0 = valid ? rowptr[r] : 0, e1 = valid ? rowptr[r + 1] : 0;
    double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
    for (int e = e0 + lane; e < e1; e += G) {
      const double2 v = val[e];
      const long long c = col[e];
      const double2 x0 = X[c];
      acc0.x = fma(v.x, x0.x, fma(-v.y, x0.y, acc0.x));
      acc0.y = fma(v.x, x0.y, fma(v.y, x0.x, acc0.y));
      if (t > 1) {
        const double2 x1 = X[n + c];
        acc1.x = fma(v.x, x1.x, fma(-v.y, x1.y, acc1.x));
        acc1.y = fma(v.x, x1.y, fma(v.y, x1.x, acc1.y));
      }
    }
    for (int o = G / 2; o > 0; o >>= 1) {
      acc0.x += __shfl_xor_sync(0xffffffffu, acc0.x, o);
      acc0.y += __shfl_xor_sync(0xffffffffu, acc0.y, o);
      acc1.x += __shfl_xor_sync(0xffffffffu, acc1.x, o);
      acc1.y += __shfl_xor_sync(0xffffffffu, acc1.y, o);
    }
    if (valid && lane == 0) {
      Y[r] = acc0;
      if (t > 1) Y[n + r] = acc1;
    }
  }
}

// Per-block sums of |Y(:, c)|, c < t; partials[b * 2 + c].
__global__ void colabs_partial_kernel(int n, int t, const double2* __restrict__ Y,
                                      double* __restrict__ partials) {
  __shared__ double s0[kRedBlock], s1[kRedBlock];
  double a0 = 0, a1 = 0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    a0 += cabs_fast(Y[r]);
    if (t > 1) a1 += cabs_fast(Y[n + r]);
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2] = s0[0];
    partials[blockIdx.x * 2 + 1] = s1[0];
  }
}

// Deterministic sum of per-block partials: fixed tree over one block.
__global__ void sum_partials_kernel(int nparts, const double* __restrict__ partials,
                                    double* __restrict__ out) {
  __shared__ double s0[kRedGrid], s1[kRedGrid];
  for (int b = threadIdx.x; b < kRedGrid; b += blockDim.x) {
    s0[b] = b < nparts ? partials[b * 2] : 0.0;
    s1[b] = b < nparts ? partials[b * 2 + 1] : 0.0;
  }
  __syncthreads();
  for (int o = kRedGrid / 2; o > 0; o >>= 1) {
    for (int b = threadIdx.x; b < o; b += blockDim.x) {
      s0[b] += s0[b + o];
      s1[b] += s1[b + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

__global__ void sign_kernel(long long m, const double2* __restrict__ Y, double2* __restrict__ S) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 y = Y[e];
    const double a = cabs_fast(y);
    if (a == 0.0) {
      S[e] = make_double2(1.0, 0.0);
    } else {
      const double r = 1.0 / a;
      S[e] = make_double2(y.x * r, y.y * r);
    }
  }
}

__global__ void rowmax_kernel(int n, int t, const double2* __restrict__ Z, double* __restrict__ h) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    double v = cabs_fast(Z[r]);
    if (t > 1) v = fmax(v, cabs_fast(Z[n + r]));
    h[r] = v;
  }
}

// The adjoint step's ranking products run in complex64 (below, Estimator::
// rank32): S = sign(Y) rounded to complex64.  Y is scaled by the power of two
// that brings its larger component into [1, 2) (exact), so the rounding loses
// neither range nor the direction; sign(0) = 1.  The map commutes with complex
// conjugation (a Hermitian Y gives an exactly Hermitian S).
__device__ __forceinline__ float2 sign32(double2 y) {
  const double m = fmax(fabs(y.x), fabs(y.y));
  if (m == 0.0) return make_float2(1.0f, 0.0f);
  const int ex = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
  if (ex == 0 || ex > 2045) {   // subnormal, near overflow or not finite: the FP64 form
    const double a = cabs_fast(y);
    return make_float2((float)(y.x / a), (float)(y.y / a));
  }
  const double f = __longlong_as_double((long long)(2046 - ex) << 52);   // 2^(1023 - ex)
  const float a = (float)(y.x * f), b = (float)(y.y * f);
  const float r = rsqrtf(fmaf(a, a, b * b));
  return make_float2(a * r, b * r);
}

__global__ void sign32_kernel(long long m, const double2* __restrict__ Y, float2* __restrict__ S) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x)
    S[e] = sign32(Y[e]);
}

__global__ void rowmax32_kernel(int n, int t, const float2* __restrict__ Z, double* __restrict__ h) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    float v = hypotf(Z[r].x, Z[r].y);
    if (t > 1) v = fmaxf(v, hypotf(Z[n + r].x, Z[n + r].y));
    h[r] = (double)v;
  }
}

struct Excl {
  int n;
  int idx[kMaxExcl];
};

__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
  // larger value first, ties to the smaller index; ia < 0 means "none"
  if (ib < 0) return ia >= 0;
  if (ia < 0) return false;
  return va > vb || (va == vb && ia < ib);
}

// argmax over indices not in ex (host list) nor in dex[0 .. ndex - 1] (indices
// found by an earlier launch, read on the device: no read-back in between).
__global__ void argmax_partial_kernel(int n, const double* __restrict__ h, Excl ex,
                                      const int* __restrict__ dex, int ndex,
                                      double* __restrict__ pv, int* __restrict__ pi) {
  __shared__ double sv[kRedBlock];
  __shared__ int si[kRedBlock];
  const int d0 = ndex > 0 ? dex[0] : -1;
  double bv = 0;
  int bi = -1;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    bool skip = (int)r == d0;
    for (int q = 0; q < ex.n; ++q) skip |= ex.idx[q] == (int)r;
    if (skip) continue;
    const double v = h[r];
    if (better(v, (int)r, bv, bi)) { bv = v; bi = (int)r; }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      if (better(sv[threadIdx.x + o], si[threadIdx.x + o], sv[threadIdx.x], si[threadIdx.x])) {
        sv[threadIdx.x] = sv[threadIdx.x + o];
        si[threadIdx.x] = si[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

// The row ranking one iteration needs, computed without read-backs in between:
// the largest h (and h at the current best index), the second largest, and the
// two largest outside the history.
struct Select {
  double hmax, hbest;
  int idx[4];   // argmax, argmax without it, argmax outside hist, next outside hist
};

__global__ void argmax_final_kernel(int nparts, const double* __restrict__ pv,
                                    const int* __restrict__ pi, const double* __restrict__ h,
                                    int probe, Select* __restrict__ out, int slot) {
  __shared__ double sv[kRedGrid];
  __shared__ int si[kRedGrid];
  for (int b = threadIdx.x; b < kRedGrid; b += blockDim.x) {
    sv[b] = b < nparts ? pv[b] : 0.0;
    si[b] = b < nparts ? pi[b] : -1;
  }
  __syncthreads();
  for (int o = kRedGrid / 2; o > 0; o >>= 1) {
    for (int b = threadIdx.x; b < o; b += blockDim.x)
      if (better(sv[b + o], si[b + o], sv[b], si[b])) {
        sv[b] = sv[b + o];
        si[b] = si[b + o];
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out->idx[slot] = si[0];
    if (slot == 0) {
      out->hmax = sv[0];
      out->hbest = probe >= 0 ? h[probe] : 0.0;
    }
  }
}

// X = [1, x] / n; x_r = +-1 from SplitMix64 output min(r, r^T), r^T the index
// of the transposed density-matrix entry, so that x is a Hermitian (real
// symmetric) N~ x N~ matrix like the first column.
__global__ void init_block_kernel(int n, int Nt, int t, double2* __restrict__ X) {
  const double inv = 1.0 / n;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    X[r] = make_double2(inv, 0.0);
    if (t > 1) {
      const long long rt = (r / Nt) + (long long)Nt * (r % Nt);
      const bool neg = (splitmix64(kSeed, (unsigned long long)(rt < r ? rt : r)) >> 63) != 0;
      X[n + r] = make_double2(neg ? -inv : inv, 0.0);
    }
  }
}

__global__ void set_units_kernel(int n, int t, double2* __restrict__ X, int i0, int i1) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    X[i0] = make_double2(1.0, 0.0);
    if (t > 1) X[(long long)n + i1] = make_double2(1.0, 0.0);
  }
}

// ||L||_1 = max over rows of L^H of sum |entry|
__global__ void rowabs_max_kernel(int n, const int* __restrict__ rowptr,
                                  const double2* __restrict__ val,
                                  unsigned long long* __restrict__ out_bits) {
  double best = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) s += cabs(val[e]);
    best = fmax(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(best));
}

// ||L||_1 matrix-free: column (i, j) of L holds |(1-omega) H| entries of rows
// i and j of H, the diagonal D_ij and, when i = j, the rates of the jumps out
// of i (which sum to dtot_i).
__global__ void mf_colabs_max_kernel(int Nt, const double* __restrict__ habs,
                                     const double* __restrict__ ad, const double* __restrict__ hw,
                                     const double* __restrict__ dtot,
                                     unsigned long long* __restrict__ out_bits) {
  const long long n = (long long)Nt * Nt;
  double best = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(r % Nt), j = (int)(r / Nt);
    double s = habs[i] + habs[j] + hypot(ad[i] + ad[j], hw[j] - hw[i]);
    if (i == j) s += dtot[i];
    best = fmax(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(best));
}

__global__ void roots_kernel(const double* __restrict__ norms, double* __restrict__ dp) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    dp[0] = norms[0];
    for (int p = 2; p <= kNormPowers; ++p) dp[p - 1] = pow(norms[p - 1], 1.0 / p);
    dp[kNormPowers] = 0.0;
  }
}

// ---------------------------------------------- supports of unit-vector chains
// A vector supported on rows I x columns J of the N~ x N~ density matrix maps
// under L~ (or L~^H) to one supported on I' x J':
//   I' = I + {i : row i of H meets I} + T,   J' = J + {j : row j of H meets J} + T,
// T = {v : a jump into (v, v) starts at some q in I and J}: part A of C at (i, j)
// reads x(m, j) for m in row i of H, part B reads x(i, m) for m in row j, the
// diagonal term reads x(i, j), and the jump sum at (v, v) reads x(q, q).
// Masks hold [2 Nt] bytes (rows, then columns); lists hold [2 Nt] ints (rows,
// then columns, ascending) and count[0] = |I|, count[1] = |J|.
__global__ void box_grow_kernel(MfOp<double> op, const unsigned char* __restrict__ in,
                                unsigned char* __restrict__ out) {
  const int Nt = op.Nt;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nt; v += gridDim.x * blockDim.x) {
    bool r = in[v] != 0, c = in[Nt + v] != 0;
    if (v < op.N)
      for (int e = op.hrow[v]; e < op.hrow[v + 1]; ++e) {
        const int m = op.hcol[e];
        r = r || in[m] != 0;
        c = c || in[Nt + m] != 0;
      }
    for (int e = op.jrow[v]; e < op.jrow[v + 1]; ++e) {
      const int q = op.jcol[e];
      if (in[q] && in[Nt + q]) r = c = true;
    }
    out[v] = r;
    out[Nt + v] = c;
  }
}

constexpr int kListThreads = 1024;

// Both masks to ascending index lists (one block, chunks of kListThreads).
__global__ void __launch_bounds__(kListThreads)
box_list_kernel(int Nt, const unsigned char* __restrict__ mask, int* __restrict__ list,
                int* __restrict__ count) {
  __shared__ int warp_tot[kListThreads / 32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int s = 0; s < 2; ++s) {
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < Nt; c0 += kListThreads) {
      const int v = c0 + threadIdx.x;
      const bool f = v < Nt && mask[s * Nt + v] != 0;
      const unsigned b = __ballot_sync(0xffffffffu, f);
      if (lane == 0) warp_tot[w] = __popc(b);
      __syncthreads();
      int off = base;
      for (int q = 0; q < w; ++q) off += warp_tot[q];
      if (f) list[s * Nt + off + __popc(b & ((1u << lane) - 1u))] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        int tot = 0;
        for (int q = 0; q < kListThreads / 32; ++q) tot += warp_tot[q];
        base += tot;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) count[s] = base;
    __syncthreads();
  }
}

// Start of a chain: e_idx, idx = a + Nt b (row a, column b).  The masks and
// the vector are zero on entry.
__global__ void box_init_kernel(int Nt, int a, int b, unsigned char* __restrict__ mask,
                                int* __restrict__ list, int* __restrict__ count,
                                double2* __restrict__ v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    mask[a] = 1;
    mask[Nt + b] = 1;
    list[0] = a;
    list[Nt] = b;
    count[0] = 1;
    count[1] = 1;
    v[a + (long long)Nt * b] = make_double2(1.0, 0.0);
  }
}

constexpr int kBoxBlock = 256;
constexpr int kBoxWarps = kBoxBlock / 32;

// y = L~ x (or L~^H x) on the box (list, count) of the output; y is left as it
// is outside the box.  Blocks take the box's columns, warps 64-row chunks of
// its rows.  Every element is computed by the same helpers, in the same order,
// as in the full product: with all rows in the box the chunks are the
// operator's paired 64-row windows, otherwise the rows run through part B and
// then their own part-A loops.
template <bool ADJ>
__global__ void __launch_bounds__(kBoxBlock)
mf_box_kernel(MfOp<double> op, const int* __restrict__ list, const int* __restrict__ count,
              const double2* __restrict__ x, double2* __restrict__ y) {
  const int nI = count[0], nJ = count[1];
  const int* rows = list;
  const int* cols = list + op.Nt;
  const bool all_rows = nI == op.Nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jj = blockIdx.x; jj < nJ; jj += gridDim.x) {
    const int j = cols[jj];
    for (int i0 = warp * kItemRows; i0 < nI; i0 += kBoxWarps * kItemRows) {
      int irow[2];
      double ox[2], oy[2];
      if (all_rows) {
        mf_window_rows(op.prow, i0, lane, op.Nt - 1, irow);
        mf_window_apply<double, double2, ADJ, LdGlobal, true>(op, x, j, i0, irow, ox, oy);
      } else {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k = i0 + lane + 32 * u;
          irow[u] = k < nI ? rows[k] : -1;
        }
        double cx[2], cy[2];
        mf_partB<double, double2, 2>(op, x, j, irow, cx, cy);
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (irow[u] >= 0)
            mf_finish<double, double2, ADJ>(op, x, irow[u], j, cx[u], cy[u], ox[u], oy[u]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (irow[u] >= 0) y[irow[u] + (long long)op.Nt * j] = make_double2(ox[u], oy[u]);
    }
  }
}

__device__ __forceinline__ double2 cmake(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 cmake(float x, float y) { return make_float2(x, y); }

// y_c = L~ x_c (or L~^H x_c) for `cols` Hermitian vectors stored n apart; both
// maps preserve Hermiticity, so only the upper triangle is computed (the same
// per-element helpers and order as the full product) and mirrored.  The
// diagonal's imaginary part, zero in exact arithmetic, is stored as zero,
// which keeps y exactly Hermitian.  Warps stride over the upper triangle's
// 64-row windows (nearly equal work each); every window is applied to all
// columns while its rows and neighbour lists are at hand.  The complex64 form
// (the ranking products of the adjoint step) multiplies by `scale`; the
// complex128 form ignores it.
template <class R, class VT, bool ADJ>
__global__ void __launch_bounds__(kBoxBlock)
mf_herm_kernel(MfOp<R> op, int cols, long long n, R scale, const VT* __restrict__ x,
               VT* __restrict__ y) {
  constexpr bool kScaled = sizeof(R) == sizeof(float);
  const int Nt = op.Nt;
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nitems = mf_item_count(Nt, true);
  for (long long k = gw; k < nitems; k += nw) {
    int j, i0;
    mf_item(k, Nt, true, j, i0);
    int irow[2];
    mf_window_rows(op.prow, i0, lane, j, irow);
    for (int c = 0; c < cols; ++c) {
      const VT* xc = x + c * n;
      VT* yc = y + c * n;
      R ox[2], oy[2];
      mf_window_apply<R, VT, ADJ, LdGlobal, true>(op, xc, j, i0, irow, ox, oy);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = irow[u];
        if (i < 0) continue;
        if (kScaled) {
          ox[u] *= scale;
          oy[u] *= scale;
        }
        if (i == j) {
          yc[i + (long long)Nt * j] = cmake(ox[u], R(0));
        } else {
          yc[i + (long long)Nt * j] = cmake(ox[u], oy[u]);
          yc[j + (long long)Nt * i] = cmake(ox[u], -oy[u]);
        }
      }
    }
  }
}

// D = sign(Y) - 1 on the box of Y (0 where Y = 0); D is zero outside the box.
__global__ void sign_minus_one_kernel(int Nt, const int* __restrict__ list,
                                      const int* __restrict__ count, const double2* __restrict__ Y,
                                      double2* __restrict__ D) {
  const int nI = count[0];
  const long long tot = (long long)nI * count[1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = list[e % nI] + (long long)Nt * list[Nt + e / nI];
    const double2 y = Y[k];
    const double a = cabs_fast(y);
    if (a == 0.0) {
      D[k] = make_double2(0.0, 0.0);
    } else {
      const double r = 1.0 / a;
      D[k] = make_double2(y.x * r - 1.0, y.y * r);
    }
  }
}

// out = in^dag for N~ x N~ matrices (column-major), through 32 x 32 tiles.
template <class VT>
__global__ void conj_transpose_kernel(int Nt, const VT* __restrict__ in, VT* __restrict__ out) {
  __shared__ VT tile[32][33];
  const int tiles = (Nt + 31) / 32;
  for (long long b = blockIdx.x; b < (long long)tiles * tiles; b += gridDim.x) {
    const int bi = (int)(b % tiles) * 32, bj = (int)(b / tiles) * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int i = bi + threadIdx.x, j = bj + r;
      if (i < Nt && j < Nt) tile[r][threadIdx.x] = in[i + (long long)Nt * j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int i = bj + threadIdx.x, j = bi + r;   // out(i, j) = conj(in(j, i))
      if (i < Nt && j < Nt) {
        const VT v = tile[threadIdx.x][r];
        out[i + (long long)Nt * j] = cmake(v.x, -v.y);
      }
    }
    __syncthreads();
  }
}

__global__ void fill_ones_kernel(long long n, double2* __restrict__ v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    v[e] = make_double2(1.0, 0.0);
}

// z = a + b
__global__ void add_kernel(long long n, const double2* __restrict__ a, const double2* __restrict__ b,
                           double2* __restrict__ z) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 u = a[e], v = b[e];
    z[e] = make_double2(u.x + v.x, u.y + v.y);
  }
}

// A^pow e_idx (or, for the adjoint step, (A^H)^pow D), with a spare vector;
// both are zero outside the current box.  Each product writes a box that
// contains the previous two, so the spare needs no clearing between products.
struct Chain {
  int idx = -1;
  int pow = 0;
  long long used = 0;
  bool box = false;         // support tracked (matrix-free L-QSW operator)
  bool full = false;        // the box is the whole matrix (known on the host)
  long long box_elems = 0;  // |I| |J| at the last host read
  int* pending = nullptr;   // pinned words of a box size in flight to the host
  DevBuf v, w, mask, mask2, list, count;
};

constexpr int kChainsMax = 8;

// Small pinned host array per thread (box sizes in flight to the host), kept
// for the thread's lifetime; portable across devices.
int* pinned_words() {
  static thread_local int* words = nullptr;
  if (!words)
    QSW_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&words), sizeof(int) * 2 * kChainsMax,
                               cudaHostAllocPortable));
  return words;
}
constexpr size_t kChainBytes = size_t(1) << 30;   // device memory for cached chains
constexpr size_t kOnesChainBytes = size_t(4) << 30;

struct Estimator {
  cudaStream_t st;
  int n, t;
  int Nt = 0;
  const Op* op;
  const Csr* A;    // CSR operator, or null for matrix-free
  const Csr* AH;
  DevBuf X, Y, W, h, partials, pv, pi, out, sel;
  DevBuf S32, Z32, T32;     // complex64 ranking products of the adjoint step
  double inv_one = 1.0;     // 1 / ||L||_1: their per-product scale
  bool box_ok = false;      // matrix-free L-QSW: unit chains track their box
  bool rank32 = false;      // ... and the adjoint step ranks rows in complex64
  bool split_ok = false;    // ... and the adjoint step may split off (A^H)^p 1
  Chain chains[kChainsMax];
  int n_chains = 2;
  long long tick = 0;
  Chain dchain;             // (A^H)^q D of the split adjoint step
  DevBuf ones;              // [(kNormPowers + 1) n]: (A^H)^k 1, k = 0..ones_pow
  int ones_pow = -1;

  void sync() { QSW_CUDA_TRY(cudaStreamSynchronize(st)); }

  // out = M^p in (M = L or L^H) for `cols` columns, ping-ponging through tmp.
  // herm_cols: the first herm_cols columns are Hermitian (matrix-free operators:
  // upper-triangle products).
  void mult(bool adjoint, int p, const double2* in, double2* out_, double2* tmp, int cols,
            int herm_cols = 0) {
    if (herm_cols > 0 && box_ok) {
      // every Hermitian column in one launch per power
      const int hc = std::min(herm_cols, cols);
      const long long items = mf_item_count(Nt, true);
      const unsigned grid =
          (unsigned)std::max<long long>(1, std::min<long long>((items + kBoxWarps - 1) / kBoxWarps,
                                                               152 * 8));
      const MfOp<double> m = make_mf<double>(*op, adjoint);
      const double2* src = in;
      for (int k = 0; k < p; ++k) {
        double2* dst = ((p - k) % 2 == 1) ? out_ : tmp;
        if (adjoint)
          QSW_LAUNCH mf_herm_kernel<double, double2, true><<<grid, kBoxBlock, 0, st>>>(
              m, hc, (long long)n, 1.0, src, dst);
        else
          QSW_LAUNCH mf_herm_kernel<double, double2, false><<<grid, kBoxBlock, 0, st>>>(
              m, hc, (long long)n, 1.0, src, dst);
        src = dst;
      }
      QSW_CUDA_TRY(cudaGetLastError());
      if (cols > hc) mult(adjoint, p, in + (size_t)n * hc, out_ + (size_t)n * hc,
                          tmp ? tmp + (size_t)n * hc : nullptr, cols - hc, 0);
      return;
    }
    if (herm_cols > 0 && op->gq.active) {
      const double2* src = in;
      for (int k = 0; k < p; ++k) {
        double2* dst = ((p - k) % 2 == 1) ? out_ : tmp;
        gq_apply_herm64(*op, adjoint, reinterpret_cast<const double*>(src),
                        reinterpret_cast<double*>(dst));
        src = dst;
      }
      QSW_CUDA_TRY(cudaGetLastError());
      if (cols > 1) mult(adjoint, p, in + n, out_ + n, tmp ? tmp + n : nullptr, cols - 1, herm_cols - 1);
      return;
    }
    const double2* src = in;
    for (int k = 0; k < p; ++k) {
      double2* dst = ((p - k) % 2 == 1) ? out_ : tmp;
      if (A) {
        const Csr& M = adjoint ? *AH : *A;
        QSW_LAUNCH spmm_kernel<<<grid_for((long long)n * 8, 256, 152 * 16), 256, 0, st>>>(
            n, cols, M.rowptr.as<int>(), M.col.as<int>(), M.val.as<double2>(), src, dst);
      } else if (op->gq.active) {
        gq_apply64(*op, adjoint, cols, reinterpret_cast<const double*>(src),
                   reinterpret_cast<double*>(dst), 1.0);
      } else {
        mf_apply64(*op, adjoint, cols, reinterpret_cast<const double*>(src),
                   reinterpret_cast<double*>(dst), 1.0);
      }
      src = dst;
    }
    QSW_CUDA_TRY(cudaGetLastError());
  }

  // One product of a chain: on its box (grown first), or the full product.
  void chain_step(Chain& ch, bool adjoint) {
    if (ch.box && !ch.full) {
      const MfOp<double> m = make_mf<double>(*op, adjoint);
      QSW_LAUNCH box_grow_kernel<<<grid_for(Nt, 256, 1024), 256, 0, st>>>(
          m, ch.mask.as<unsigned char>(), ch.mask2.as<unsigned char>());
      QSW_LAUNCH box_list_kernel<<<1, kListThreads, 0, st>>>(Nt, ch.mask2.as<unsigned char>(),
                                                             ch.list.as<int>(), ch.count.as<int>());
      const unsigned grid = (unsigned)std::min(Nt, 152 * 8);
      if (adjoint)
        QSW_LAUNCH mf_box_kernel<true><<<grid, kBoxBlock, 0, st>>>(
            m, ch.list.as<int>(), ch.count.as<int>(), ch.v.as<double2>(), ch.w.as<double2>());
      else
        QSW_LAUNCH mf_box_kernel<false><<<grid, kBoxBlock, 0, st>>>(
            m, ch.list.as<int>(), ch.count.as<int>(), ch.v.as<double2>(), ch.w.as<double2>());
      QSW_CUDA_TRY(cudaGetLastError());
      std::swap(ch.mask, ch.mask2);
    } else {
      mult(adjoint, 1, ch.v.as<double2>(), ch.w.as<double2>(), nullptr, 1);
    }
    std::swap(ch.v, ch.w);
    ++ch.pow;
  }

  // The box size of a chain reaches the host with the next read-back the
  // iteration makes anyway (a copy into pinned words queued now, settled after
  // that sync); until then the chain keeps its box products, which are exact
  // for a full box too.
  void read_box(Chain& ch) {
    int* w = pinned_words() + 2 * (&ch - chains);
    QSW_CUDA_TRY(cudaMemcpyAsync(w, ch.count.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ch.pending = w;
  }

  void settle() {
    for (int q = 0; q < n_chains; ++q) {
      Chain& ch = chains[q];
      if (!ch.pending) continue;
      ch.box_elems = (long long)ch.pending[0] * ch.pending[1];
      ch.full = ch.pending[0] == Nt && ch.pending[1] == Nt;
      ch.pending = nullptr;
    }
  }

  // Both vectors (and the masks) cleared; the box, when tracked, still empty.
  void chain_reset(Chain& ch, bool with_box) {
    const size_t vb = sizeof(double2) * (size_t)n;
    ch.v.alloc(vb);
    ch.w.alloc(vb);
    QSW_CUDA_TRY(cudaMemsetAsync(ch.v.p, 0, vb, st));
    QSW_CUDA_TRY(cudaMemsetAsync(ch.w.p, 0, vb, st));
    ch.box = with_box;
    ch.full = false;
    ch.pow = 0;
    ch.box_elems = 0;
    ch.pending = nullptr;
    if (with_box) {
      ch.mask.alloc(2 * (size_t)Nt);
      ch.mask2.alloc(2 * (size_t)Nt);
      ch.list.alloc(sizeof(int) * 2 * (size_t)Nt);
      ch.count.alloc(sizeof(int) * 2);
      QSW_CUDA_TRY(cudaMemsetAsync(ch.mask.p, 0, 2 * (size_t)Nt, st));
    }
  }

  // dst = A^p e_idx, from the chain kept for idx (extended as needed); the
  // chain is returned (its box describes the support of dst).
  Chain* unit_power(int idx, int p, double2* dst) {
    Chain* ch = nullptr;
    for (int q = 0; q < n_chains; ++q)
      if (chains[q].idx == idx) ch = &chains[q];
    if (ch && ch->pow > p) ch->idx = -1;   // cannot go back: restart it
    if (!ch || ch->idx != idx) {
      if (!ch) {   // an unused slot, else the least recently used
        ch = &chains[0];
        for (int q = 1; q < n_chains; ++q)
          if ((chains[q].idx < 0) != (ch->idx < 0) ? chains[q].idx < 0 : chains[q].used < ch->used)
            ch = &chains[q];
      }
      ch->idx = idx;
      chain_reset(*ch, box_ok);
      if (box_ok)
        QSW_LAUNCH box_init_kernel<<<1, 32, 0, st>>>(Nt, idx % Nt, idx / Nt,
                                                     ch->mask.as<unsigned char>(),
                                                     ch->list.as<int>(), ch->count.as<int>(),
                                                     ch->v.as<double2>());
      else
        QSW_LAUNCH set_units_kernel<<<1, 32, 0, st>>>(n, 1, ch->v.as<double2>(), idx, 0);
      QSW_CUDA_TRY(cudaGetLastError());
    }
    ch->used = ++tick;
    const bool advanced = ch->pow < p;
    while (ch->pow < p) chain_step(*ch, false);
    QSW_CUDA_TRY(cudaMemcpyAsync(dst, ch->v.p, sizeof(double2) * (size_t)n,
                                 cudaMemcpyDeviceToDevice, st));
    if (ch->box && !ch->full && advanced) read_box(*ch);
    return ch;
  }

  // column 1 of a block = column 0 ^dag
  void mirror_column(bool z32 = false) {
    const int tiles = (Nt + 31) / 32;
    const unsigned grid = (unsigned)std::min<long long>((long long)tiles * tiles, 4096);
    if (z32)
      QSW_LAUNCH conj_transpose_kernel<float2><<<grid, dim3(32, 8), 0, st>>>(
          Nt, Z32.as<float2>(), Z32.as<float2>() + (size_t)n);
    else
      QSW_LAUNCH conj_transpose_kernel<double2><<<grid, dim3(32, 8), 0, st>>>(
          Nt, Y.as<double2>(), Y.as<double2>() + (size_t)n);
    QSW_CUDA_TRY(cudaGetLastError());
  }

  // Z32 = ((A^H / ||A||_1)^p S32) for `cols` columns of S32 (the first
  // herm_cols Hermitian: upper-triangle products), in complex64.  Only the
  // ranking of the rows of Z by their largest modulus is used, which the
  // positive scale leaves as it is; with it |Z| <= 1 (||A^H||_inf = ||A||_1,
  // |sign| = 1), so no power overflows the FP32 range.
  void mult32_adjoint(int p, int cols, int herm_cols) {
    const float scale = (float)inv_one;
    const float2* src = S32.as<float2>();
    for (int k = 0; k < p; ++k) {
      float2* dst = ((p - k) % 2 == 1) ? Z32.as<float2>() : T32.as<float2>();
      if (herm_cols > 0) {
        const long long items = mf_item_count(Nt, true);
        const unsigned grid = (unsigned)std::max<long long>(
            1, std::min<long long>((items + kBoxWarps - 1) / kBoxWarps, 152 * 8));
        const MfOp<float> m = make_mf<float>(*op, true);
        QSW_LAUNCH mf_herm_kernel<float, float2, true><<<grid, kBoxBlock, 0, st>>>(
            m, cols, (long long)n, scale, src, dst);
      } else {
        mf_apply32(*op, true, cols, reinterpret_cast<const float*>(src),
                   reinterpret_cast<float*>(dst), scale);
      }
      src = dst;
    }
    QSW_CUDA_TRY(cudaGetLastError());
  }

  // ones[k n ..] = (A^H)^k 1 for k = 0..p (the all-ones vector and its chain).
  void ensure_ones(int p) {
    const size_t nn = (size_t)n;
    if (ones_pow < 0) {
      ones.alloc(sizeof(double2) * nn * (kNormPowers + 1));
      QSW_LAUNCH fill_ones_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(n, ones.as<double2>());
      QSW_CUDA_TRY(cudaGetLastError());
      ones_pow = 0;
    }
    for (; ones_pow < p; ++ones_pow)   // Hermitian: upper-triangle products
      mult(true, 1, ones.as<double2>() + nn * ones_pow, ones.as<double2>() + nn * (ones_pow + 1),
           nullptr, 1, 1);
  }

  // Y(:, c) <- (A^H)^p sign(Y(:, c)) = (A^H)^p 1 + (A^H)^p D_c, D_c = sign(Y(:, c)) - 1
  // supported on the box of the chain that produced Y(:, c); columns c < cols.
  void adjoint_split(int p, Chain* const* src, int cols) {
    ensure_ones(p);
    double2* Yp = Y.as<double2>();
    const size_t nn = (size_t)n;
    for (int c = 0; c < cols; ++c) {
      Chain& d = dchain;
      chain_reset(d, true);
      QSW_CUDA_TRY(cudaMemcpyAsync(d.mask.p, src[c]->mask.p, 2 * (size_t)Nt,
                                   cudaMemcpyDeviceToDevice, st));
      QSW_CUDA_TRY(cudaMemcpyAsync(d.list.p, src[c]->list.p, sizeof(int) * 2 * (size_t)Nt,
                                   cudaMemcpyDeviceToDevice, st));
      QSW_CUDA_TRY(cudaMemcpyAsync(d.count.p, src[c]->count.p, sizeof(int) * 2,
                                   cudaMemcpyDeviceToDevice, st));
      QSW_LAUNCH sign_minus_one_kernel<<<grid_for(src[c]->box_elems, 256, 4096), 256, 0, st>>>(
          Nt, d.list.as<int>(), d.count.as<int>(), Yp + nn * c, d.v.as<double2>());
      QSW_CUDA_TRY(cudaGetLastError());
      for (int q = 0; q < p; ++q) chain_step(d, true);
      QSW_LAUNCH add_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(
          n, ones.as<double2>() + nn * p, d.v.as<double2>(), Yp + nn * c);
      QSW_CUDA_TRY(cudaGetLastError());
    }
  }

  void colnorms(const double2* Yp, double* host2) {
    QSW_LAUNCH colabs_partial_kernel<<<kRedGrid, kRedBlock, 0, st>>>(n, t, Yp, partials.as<double>());
    QSW_LAUNCH sum_partials_kernel<<<1, 256, 0, st>>>(kRedGrid, partials.as<double>(), out.as<double>());
    QSW_CUDA_TRY(cudaMemcpyAsync(host2, out.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    settle();
  }

  // The iteration's ranking of h (Select), one read-back: four argmax passes
  // queued back to back, the later ones excluding earlier results on the device.
  void select(const std::vector<int>& hist, int probe, Select* res) {
    Excl none{};
    Excl eh{};
    eh.n = (int)std::min<size_t>(hist.size(), kMaxExcl);
    for (int q = 0; q < eh.n; ++q) eh.idx[q] = hist[q];
    Select* d = sel.as<Select>();
    const int* didx = reinterpret_cast<const int*>(reinterpret_cast<const char*>(d) + offsetof(Select, idx));
    struct Pass {
      const Excl* ex;
      const int* dex;
      int slot;
    } passes[4] = {{&none, nullptr, 0}, {&none, didx + 0, 1}, {&eh, nullptr, 2}, {&eh, didx + 2, 3}};
    const int np = t > 1 ? 4 : 1;
    for (int q = 0; q < np; ++q) {
      QSW_LAUNCH argmax_partial_kernel<<<kRedGrid, kRedBlock, 0, st>>>(
          n, h.as<double>(), *passes[q].ex, passes[q].dex, passes[q].dex ? 1 : 0, pv.as<double>(),
          pi.as<int>());
      QSW_LAUNCH argmax_final_kernel<<<1, 256, 0, st>>>(kRedGrid, pv.as<double>(), pi.as<int>(),
                                                        h.as<double>(), q == 0 ? probe : -1, d,
                                                        passes[q].slot);
    }
    QSW_CUDA_TRY(cudaGetLastError());
    QSW_CUDA_TRY(cudaMemcpyAsync(res, d, sizeof(Select), cudaMemcpyDeviceToHost, st));
    sync();
    settle();
  }

  // A^p X0 for the common starting block X0: every estimate's first product
  // comes from this one chain.  The estimates run in increasing p, so only the
  // current power is kept (and advanced in place), not all nine.
  DevBuf chain, chain_tmp;
  int chain_pow = -1;
  void start_chain() {
    const size_t blk = (size_t)n * t;
    chain.alloc(sizeof(double2) * blk);
    chain_tmp.alloc(sizeof(double2) * blk);
    QSW_LAUNCH init_block_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(n, Nt, t,
                                                                          chain.as<double2>());
    QSW_CUDA_TRY(cudaGetLastError());
    chain_pow = 0;
  }
  const double2* chain_power(int p) {
    QSW_CHECK_ARG(chain_pow >= 0 && chain_pow <= p, QSW_ERR_CUDA, "estimator chain out of order");
    // both columns (all ones, and the transpose-symmetric signs) are
    // Hermitian, and so are their powers
    for (; chain_pow < p; ++chain_pow) {
      mult(false, 1, chain.as<double2>(), chain_tmp.as<double2>(), nullptr, t, t);
      std::swap(chain, chain_tmp);
    }
    return chain.as<double2>();
  }

  double estimate(int p) {
    double2* Xp = X.as<double2>();
    double2* Yp = Y.as<double2>();
    double2* Wp = W.as<double2>();
    std::vector<int> hist;
    double est_old = 0.0, est = 0.0;
    int ind[2] = {0, 0};
    int ind_best = 0;
    Chain* ych[2] = {nullptr, nullptr};   // chains behind the columns of Y (k >= 2)
    for (int k = 1;; ++k) {
      // L~ maps X^dag to (L~ X)^dag (and so does L~^H): when the two unit vectors
      // are e_(a,b) and e_(b,a), the second column of Y, and of Z below, is the
      // first one ^dag.
      bool mirror = false;
      if (k == 1) {
        QSW_CUDA_TRY(cudaMemcpyAsync(Yp, chain_power(p), sizeof(double2) * (size_t)n * t,
                                     cudaMemcpyDeviceToDevice, st));
      } else {   // Y = A^p [e_ind0, e_ind1]
        mirror = t > 1 && ind[1] == (ind[0] / Nt) + Nt * (ind[0] % Nt);
        ych[0] = unit_power(ind[0], p, Yp);
        if (mirror) {
          mirror_column();
          ych[1] = ych[0];
        } else {
          for (int c = 1; c < t; ++c) ych[c] = unit_power(ind[c], p, Yp + (size_t)n * c);
        }
      }
      double cn[2] = {0, 0};
      colnorms(Yp, cn);
      const int jbest = (t > 1 && cn[1] > cn[0]) ? 1 : 0;
      est = cn[jbest];
      if (est > est_old || k == 2) ind_best = ind[jbest];
      if (k >= 2 && est <= est_old) {
        est = est_old;
        break;
      }
      est_old = est;
      if (k > kItMax) break;
      // Z = (A^H)^p S, S = sign(Y), in Y
      const int tz = mirror ? 1 : t;   // columns computed (the mirrored one follows)
      bool split = k >= 2 && split_ok;
      for (int c = 0; c < tz && split; ++c)
        split = ych[c]->box && !ych[c]->full && ych[c]->box_elems * 16 <= (long long)n;
      bool z32 = false;
      if (split) {
        adjoint_split(p, ych, tz);
      } else if (rank32) {
        QSW_LAUNCH sign32_kernel<<<grid_for((long long)n * tz, 256, 4096), 256, 0, st>>>(
            (long long)n * tz, Yp, S32.as<float2>());
        mult32_adjoint(p, tz, k == 1 ? tz : 0);   // k = 1: sign(Y) is Hermitian
        z32 = true;
      } else {
        QSW_LAUNCH sign_kernel<<<grid_for((long long)n * tz, 256, 4096), 256, 0, st>>>(
            (long long)n * tz, Yp, Xp);
        mult(true, p, Xp, Yp, Wp, tz, k == 1 ? tz : 0);   // k = 1: sign(Y) is Hermitian
      }
      if (mirror) mirror_column(z32);
      if (z32)
        QSW_LAUNCH rowmax32_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(n, t, Z32.as<float2>(),
                                                                           h.as<double>());
      else
        QSW_LAUNCH rowmax_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(n, t, Yp, h.as<double>());
      QSW_CUDA_TRY(cudaGetLastError());
      Select pick;
      select(hist, ind_best, &pick);
      if (k >= 2 && pick.hmax == pick.hbest) break;
      int fresh[2] = {-1, -1};
      if (t > 1) {
        const bool in0 = std::find(hist.begin(), hist.end(), pick.idx[0]) != hist.end();
        const bool in1 = std::find(hist.begin(), hist.end(), pick.idx[1]) != hist.end();
        if (in0 && in1) break;
        fresh[0] = pick.idx[2];
        fresh[1] = pick.idx[3];
        if (fresh[0] < 0 || fresh[1] < 0) break;   // fewer than t unused unit vectors
      } else {
        fresh[0] = pick.idx[0];
      }
      ind[0] = fresh[0];
      ind[1] = fresh[1];
      hist.push_back(ind[0]);
      if (t > 1) hist.push_back(ind[1]);
    }
    return est;
  }
};

}  // namespace

void compute_norms(Op& op, const Csr* L, const Csr* LH) {
  cudaStream_t st = op.ctx->stream;
  if (!L && !op.gq.active) ensure_pair_lists(op);   // the products below read part A through them
  const int n = (int)op.n;
  // exact ||L||_1 (global walks: closed form when it applies, else estimated below)
  bool one_estimated = false;
  double one = 0.0;
  DevBuf bits;
  bits.alloc(sizeof(unsigned long long));
  QSW_CUDA_TRY(cudaMemsetAsync(bits.p, 0, sizeof(unsigned long long), st));
  if (op.gq.active) {
    one_estimated = !global_exact_norm(op, &one);
  } else if (LH) {
    QSW_LAUNCH rowabs_max_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(
        n, LH->rowptr.as<int>(), LH->val.as<double2>(), bits.as<unsigned long long>());
  } else {
    QSW_LAUNCH mf_colabs_max_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(
        op.Nt, op.mf.habs.as<double>(), op.mf.ad64.as<double>(), op.mf.hw64.as<double>(),
        op.g.dtot.as<double>(), bits.as<unsigned long long>());
  }
  if (!op.gq.active) {
    QSW_CUDA_TRY(cudaGetLastError());
    unsigned long long b = 0;
    QSW_CUDA_TRY(cudaMemcpyAsync(&b, bits.p, sizeof(b), cudaMemcpyDeviceToHost, st));
    QSW_CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(&one, &b, sizeof(one));
  }

  Estimator E;
  E.st = st;
  E.n = n;
  E.t = n >= 2 ? kEll : 1;
  E.op = &op;
  E.A = L;
  E.AH = LH;
  E.X.alloc(sizeof(double2) * (size_t)n * E.t);
  E.Y.alloc(sizeof(double2) * (size_t)n * E.t);
  E.W.alloc(sizeof(double2) * (size_t)n * E.t);
  E.h.alloc(sizeof(double) * n);
  E.partials.alloc(sizeof(double) * 2 * kRedGrid);
  E.pv.alloc(sizeof(double) * kRedGrid);
  E.pi.alloc(sizeof(int) * kRedGrid);
  E.out.alloc(sizeof(double) * 4);
  E.sel.alloc(sizeof(Select));
  E.Nt = op.Nt;
  E.box_ok = !L && !op.gq.active;
  E.rank32 = E.box_ok && !op.rank64;
  if (E.rank32) {
    E.S32.alloc(sizeof(float2) * (size_t)n * E.t);
    E.Z32.alloc(sizeof(float2) * (size_t)n * E.t);
    E.T32.alloc(sizeof(float2) * (size_t)n * E.t);
  }
  E.split_ok = E.box_ok &&
               sizeof(double2) * (size_t)n * (kNormPowers + 1) <= kOnesChainBytes;
  E.n_chains = (int)std::min<size_t>(
      kChainsMax, std::max<size_t>(2, kChainBytes / (2 * sizeof(double2) * (size_t)n)));
  if (one_estimated) {   // several sandwich operators (or diagonal entries): estimate p = 1 too
    E.start_chain();
    one = E.estimate(1);
  } else if (one != 0.0) {
    E.start_chain();
  }
  op.norms[0] = one;
  E.inv_one = one > 0.0 ? 1.0 / one : 1.0;
  for (int p = 2; p <= kNormPowers; ++p) op.norms[p - 1] = one == 0.0 ? 0.0 : E.estimate(p);

  // d_p = ||L^p||_1^(1/p), taken on the device; the host keeps a copy for sizing.
  DevBuf nd;
  nd.alloc(sizeof(double) * kNormPowers);
  QSW_CUDA_TRY(cudaMemcpyAsync(nd.p, op.norms, sizeof(double) * kNormPowers,
                               cudaMemcpyHostToDevice, st));
  op.dp_dev.alloc(sizeof(double) * (kNormPowers + 1));
  QSW_LAUNCH roots_kernel<<<1, 32, 0, st>>>(nd.as<double>(), op.dp_dev.as<double>());
  QSW_CUDA_TRY(cudaGetLastError());
  QSW_CUDA_TRY(cudaMemcpyAsync(op.dp, op.dp_dev.p, sizeof(double) * (kNormPowers + 1),
                               cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace qsw
