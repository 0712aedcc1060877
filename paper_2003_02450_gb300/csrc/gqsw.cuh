// Matrix-free application of a global-interaction walk (G-QSW, Section 2.5.2
// Eq. L_global; NM-G-QSW, Eq. nm_gqsw).  With Q = -i H_tot - 1/2 sum_k
// L'_k^dag L'_k - 1/2 (port terms), L'_k = sqrt(omega) L_k and
// H_tot = (1 - omega) H - omega H_rot, the master equation is
//
//   L~ x = Q x + x Q^dag + sum_k L'_k x L'_k^dag + (port jumps on the diagonal),
//
// and its adjoint (the 1-norm estimator's L~^H) is the same expression with
// Q -> Q^dag, L'_k -> L'_k^dag and the port jumps transposed.  The sandwich is
// taken in two passes: W_k = x L'_k^dag over every element (pass A), then
// (L'_k W_k)_ij (pass B, with the Q terms).  A Hermitian x gives a Hermitian
// result, so pass B may run on the upper triangle; W_k is not Hermitian and
// pass A always covers the whole matrix.
//
// The gather loops are unrolled four ways: a row of Q holds ~100 entries for
// the G-QSW of a sparse digraph (L'^dag L' couples every pair of in-neighbours),
// and at a few hundred vertices a term gives each warp less than one item, so
// the passes are latency-bound; four iterations' loads in flight measured
// 13 % faster on ER N = 400.
#pragma once

#include "matfree.cuh"

namespace qsw {

template <class R> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };

template <class R> struct GqOp {
  using VT = typename V2<R>::T;
  int Nt;
  const int* qrow;     // [Nt + 1]  Q (or Q^dag), complex
  const int* qcol;
  const VT* qval;
  int nl;              // operators in the sandwich (0 when omega = 0)
  const int* lrow[kMaxGlobalOps];   // L'_k (or L'_k^dag), complex
  const int* lcol[kMaxGlobalOps];
  const VT* lval[kMaxGlobalOps];
  const int* jrow;     // [Nt + 1] port jumps into i (or out of i for the adjoint)
  const int* jcol;
  const VT* jval;      // rates in .x
};

// acc += a b
template <class VT, class R>
__device__ __forceinline__ void cmad(R& ax, R& ay, const VT a, const VT b) {
  ax = fma(a.x, b.x, fma(-a.y, b.y, ax));
  ay = fma(a.x, b.y, fma(a.y, b.x, ay));
}
// acc += x conj(q)
template <class VT, class R>
__device__ __forceinline__ void cmad_conj(R& ax, R& ay, const VT x, const VT q) {
  ax = fma(x.x, q.x, fma(x.y, q.y, ax));
  ay = fma(x.y, q.x, fma(-x.x, q.y, ay));
}

// Pass A for the lane's rows a (2 per lane, -1 = none) of column j:
// W_k(a, j) = sum_{b in row j of L'_k} x(a, b) conj(L'_k(j, b)); the list is
// the same for every lane and the reads of x run down column b (coalesced).
template <class R, class VT, class LD = LdGlobal>
__device__ __forceinline__ void gq_pass_a(const GqOp<R>& op, const VT* __restrict__ x, VT* w, int j,
                                          const int* arow) {
  const long long n = (long long)op.Nt * op.Nt;
  for (int k = 0; k < op.nl; ++k) {
    R ax[2] = {0, 0}, ay[2] = {0, 0};
    const int e0 = op.lrow[k][j], e1 = op.lrow[k][j + 1];
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
      const long long off = (long long)op.Nt * op.lcol[k][e];
      const VT l = op.lval[k][e];
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (arow[u] >= 0) cmad_conj<VT, R>(ax[u], ay[u], LD::ld(x + off + arow[u]), l);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (arow[u] >= 0) {
        VT v;
        v.x = ax[u];
        v.y = ay[u];
        w[k * n + arow[u] + (long long)op.Nt * j] = v;
      }
  }
}

// Hermitian x: Q x = (x Q^dag)^dag, so with R = x Q^dag the two Q terms of
// element (i, j) are R(i, j) + conj(R(j, i)).  R is formed in pass A next to
// the W_k (stored after them, at w + nl n) by the same row-j loop: the list is
// shared by the warp and the reads of x run down columns, instead of every
// lane walking its own row of Q.
template <class R, class VT, class LD = LdGlobal>
__device__ __forceinline__ void gq_pass_a_r(const GqOp<R>& op, const VT* __restrict__ x, VT* w,
                                            int j, const int* arow) {
  const long long n = (long long)op.Nt * op.Nt;
  R ax[2] = {0, 0}, ay[2] = {0, 0};
#pragma unroll 4
  for (int e = op.qrow[j]; e < op.qrow[j + 1]; ++e) {
    const long long off = (long long)op.Nt * op.qcol[e];
    const VT q = op.qval[e];
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (arow[u] >= 0) cmad_conj<VT, R>(ax[u], ay[u], LD::ld(x + off + arow[u]), q);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
    if (arow[u] >= 0) {
      VT v;
      v.x = ax[u];
      v.y = ay[u];
      w[op.nl * n + arow[u] + (long long)op.Nt * j] = v;
    }
}

// Pass B at element (i, j) of a Hermitian x, from the pass-A products.  The
// Q terms come from R = x Q^dag alone, which is right only while x is exactly
// Hermitian: for an anti-Hermitian part A of x this form gives -Q A in place of
// Q A, and -Q = i H_tot + 1/2 sum L'^dag L' + ... amplifies A like exp(+t ||L'^dag L'||/2).
// A diagonal element is real in exact arithmetic but the L'_k W_k sum leaves a
// rounding-level imaginary part, so it is stored as zero here (and the series
// kernel takes real diagonals from its input), keeping every term exactly
// Hermitian.
template <class R, class VT, class LD = LdGlobal>
__device__ __forceinline__ void gq_element_herm(const GqOp<R>& op, const VT* __restrict__ x,
                                                const VT* __restrict__ w, int i, int j, R& yx,
                                                R& yy) {
  const long long n = (long long)op.Nt * op.Nt;
  const long long cj = (long long)op.Nt * j;
  const VT rij = LD::ld(w + op.nl * n + cj + i);
  const VT rji = LD::ld(w + op.nl * n + (long long)op.Nt * i + j);
  R ax = rij.x + rji.x, ay = rij.y - rji.y;
  for (int k = 0; k < op.nl; ++k)
#pragma unroll 4
    for (int e = op.lrow[k][i]; e < op.lrow[k][i + 1]; ++e)
      cmad<VT, R>(ax, ay, op.lval[k][e], LD::ld(w + k * n + cj + op.lcol[k][e]));
  if (i == j) {
    for (int e = op.jrow[i]; e < op.jrow[i + 1]; ++e) {
      const VT v = LD::ld(x + (long long)op.jcol[e] * (op.Nt + 1));
      const R r = op.jval[e].x;
      ax = fma(r, v.x, ax);
    }
    ay = 0;
  }
  yx = ax;
  yy = ay;
}

// Pass B at element (i, j): (L~ x)_(i,j) from x and the pass-A products w.
template <class R, class VT, class LD = LdGlobal>
__device__ __forceinline__ void gq_element(const GqOp<R>& op, const VT* __restrict__ x,
                                           const VT* __restrict__ w, int i, int j, R& yx, R& yy) {
  const long long n = (long long)op.Nt * op.Nt;
  const long long cj = (long long)op.Nt * j;
  R ax = 0, ay = 0;
  // sum_m Q(i, m) x(m, j): row i of Q, reads gathered in column j
#pragma unroll 4
  for (int e = op.qrow[i]; e < op.qrow[i + 1]; ++e)
    cmad<VT, R>(ax, ay, op.qval[e], LD::ld(x + cj + op.qcol[e]));
  // sum_m x(i, m) conj(Q(j, m)): row j of Q (the same for a warp's lanes)
#pragma unroll 4
  for (int e = op.qrow[j]; e < op.qrow[j + 1]; ++e)
    cmad_conj<VT, R>(ax, ay, LD::ld(x + i + (long long)op.Nt * op.qcol[e]), op.qval[e]);
  // sum_k sum_a L'_k(i, a) W_k(a, j)
  for (int k = 0; k < op.nl; ++k)
#pragma unroll 4
    for (int e = op.lrow[k][i]; e < op.lrow[k][i + 1]; ++e)
      cmad<VT, R>(ax, ay, op.lval[k][e], LD::ld(w + k * n + cj + op.lcol[k][e]));
  if (i == j) {
    for (int e = op.jrow[i]; e < op.jrow[i + 1]; ++e) {
      const VT v = LD::ld(x + (long long)op.jcol[e] * (op.Nt + 1));
      const R r = op.jval[e].x;
      ax = fma(r, v.x, ax);
      ay = fma(r, v.y, ay);
    }
  }
  yx = ax;
  yy = ay;
}

}  // namespace qsw
