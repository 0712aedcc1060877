// Matrix-free application of the L-QSW superoperator (no CSR): the action of
// Eq. qsw_ss on a vectorised rho, written with the identities of
// Eq. vec_mappings so that every term is a product of a REAL coefficient and a
// complex entry of rho:
//
//   (L~ x)_(i,j) = -i C_ij + D_ij x_ij + [i = j] sum_q r_iq x_(q,q)
//   C_ij  = sum_{m != i} c_im x_(m,j)  -  sum_{m != j} x_(i,m) c_mj,   c = (1 - omega) H
//   D_ij  = -(dtot_i + dtot_j)/2 - i (1 - omega)(H_ii - H_jj)
//
// (r_iq the jump rates, dtot_v the total rate leaving v).  The adjoint L~^H
// (used by the 1-norm estimator) is  +i C_ij + conj(D_ij) x_ij + jumps of the
// transposed list.  This is the same operator the CSR assembly stores, entry by
// entry; only the summation order differs.
//
// On GB300 the FP64 pipe issues 2 FMA per SM per clock, so the complex128 form
// is bound by FP64 issue, not by HBM: each off-diagonal term costs the minimum
// of 2 FMA (real x complex), there are no cross-lane FP64 reductions (one thread
// owns one element), and no matrix is streamed from memory.
#pragma once

#include "qsw_internal.h"

namespace qsw {

template <class R> struct MfOp {
  int N, Nt;           // N: vertices that have Hamiltonian rows (0 when omega = 1)
  const int* hrow;     // [N + 1] off-diagonal H, rows of the graph vertices
  const int* hcol;
  const R* hval;       // (1 - omega) H_im
  const R* ad;         // [Nt] -dtot_v / 2
  const R* hw;         // [Nt] (1 - omega) H_vv
  const int* jrow;     // [Nt + 1] jumps into i (L) or out of i (L^H)
  const int* jcol;
  const R* jval;
  const int* prow;     // [64 ceil(Nt / 64)] rows of each 64-row window in lane
                       // order (see mf_window_rows); -1 pads the last window
  const int* pwin;     // [ceil(Nt / 64)] 1: the window's rows are paired (part A
                       // by mf_partA2), 0: natural order (part A row by row)
  const int* paoff;    // [ceil(Nt / 64) + 1] paired windows: first row of each
                       // window's lists in pacol / paval (32 entries per row)
  const int* pacol;    // paired windows, lane-interleaved: entry t of lane l's
  const R* paval;      // merged list (row a's entries, then row b's) at
                       // 32 (paoff[w] + t) + l, so a warp's loads are contiguous
};

constexpr int kWindowRows = 64;   // rows of one window (two per lane)

// Reads of the operand x.  Inside the persistent series kernel x was written
// by other SMs before the last grid (or cluster) barrier, whose fences form a
// gpu-scope (cluster-scope) release/acquire pair with those writes; a weak
// load ordered after that acquire must return the new values, so x may be
// cached in L1 (ld.global.ca).  The non-coherent read-only path (ld.global.nc)
// would not be covered and is not used.  Part A of C reads one column of x
// about 20 times per element, which L1 serves instead of L2.
template <class VT> __device__ __forceinline__ VT ldx(const VT* p) { return __ldca(p); }

// Load policies of the helpers below: x in global memory (ldx), or x at a
// generic address that may be shared memory (the small-walk batched kernel
// keeps a walk's Taylor terms on chip).
struct LdGlobal {
  template <class VT> __device__ __forceinline__ static VT ld(const VT* p) { return ldx(p); }
};
struct LdGeneric {
  template <class VT> __device__ __forceinline__ static VT ld(const VT* p) { return *p; }
};

// Part B of C for RPT rows of one column, accumulated with a minus sign:
// c = -sum_{m in H row j} c_mj x_(i,m)  (the uniform list, coalesced over i).
template <class R, class VT, int RPT, class LD = LdGlobal>
__device__ __forceinline__ void mf_partB(const MfOp<R>& op, const VT* __restrict__ x, int j,
                                         const int* irow, R* cx, R* cy) {
#pragma unroll
  for (int u = 0; u < RPT; ++u) { cx[u] = 0; cy[u] = 0; }
  if (j >= op.N) return;
  const int e0 = op.hrow[j], e1 = op.hrow[j + 1];
#pragma unroll 2
  for (int e = e0; e < e1; ++e) {
    const long long off = (long long)op.Nt * op.hcol[e];
    const R h = op.hval[e];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (irow[u] >= 0) {
        const VT v = LD::ld(x + off + irow[u]);
        cx[u] = fma(-h, v.x, cx[u]);
        cy[u] = fma(-h, v.y, cy[u]);
      }
    }
  }
}

// Part A of C for the two rows a = irow[0], b = irow[1] of one lane (same
// column j): c += sum_{m in H row i} c_im x_(m,j).  The rows' entries run as one
// list (a's, then b's) with the accumulator picked by a select, so a lane's
// trip count is len(a) + len(b); the windows pair short rows with long ones
// (mf_window_rows) to make that sum nearly equal across a warp.  Each row's
// terms are added in the same order as a loop over that row alone.  PA: the
// merged lists are read from the window's lane-interleaved copy (pacol,
// paval), so entry t of all 32 lanes is one contiguous load where the rows'
// own lists cost a cache sector per lane.  Same terms, same order, same
// results; the 1-norm estimator's products use it (1.1 ms less per ER-1000
// build), the series kernel does not (its FP64 work hides the list reads,
// and the extra index loads made it 0.8 % slower).
template <class R, class VT, class LD = LdGlobal, bool PA = false>
__device__ __forceinline__ void mf_partA2(const MfOp<R>& op, const VT* __restrict__ x, int j,
                                          int w0, const int* irow, R* cx, R* cy) {
  const long long base = (long long)op.Nt * j;
  if (!PA) {   // the rows' own lists
    const int a = irow[0], b = irow[1];
    const int ea = (a >= 0 && a < op.N) ? op.hrow[a] : 0;
    const int la = (a >= 0 && a < op.N) ? op.hrow[a + 1] - ea : 0;
    const int eb = (b >= 0 && b < op.N) ? op.hrow[b] : 0;
    const int lb = (b >= 0 && b < op.N) ? op.hrow[b + 1] - eb : 0;
    R ax = cx[0], ay = cy[0], bx = cx[1], by = cy[1];
    const int tot = la + lb;
    for (int t = 0; t < tot; ++t) {
      const bool second = t >= la;
      const int e = second ? eb + (t - la) : ea + t;
      const VT v = LD::ld(x + base + op.hcol[e]);
      const R h = op.hval[e];
      const R tx = fma(h, v.x, second ? bx : ax);
      const R ty = fma(h, v.y, second ? by : ay);
      ax = second ? ax : tx;
      ay = second ? ay : ty;
      bx = second ? tx : bx;
      by = second ? ty : by;
    }
    cx[0] = ax;
    cy[0] = ay;
    cx[1] = bx;
    cy[1] = by;
    return;
  }
  const int lane = threadIdx.x & 31;
  // the lane's two rows before any masking (a Hermitian chunk masks rows past
  // its column): their full list lengths place row b's entries in the list
  const int ra = op.prow[w0 + lane], rb = op.prow[w0 + 32 + lane];
  const int la = (ra >= 0 && ra < op.N) ? op.hrow[ra + 1] - op.hrow[ra] : 0;
  const int lb = (rb >= 0 && rb < op.N) ? op.hrow[rb + 1] - op.hrow[rb] : 0;
  const int t0 = irow[0] >= 0 ? 0 : la;
  const int t1 = irow[1] >= 0 ? la + lb : la;
  const long long p0 = 32LL * op.paoff[w0 / kWindowRows] + lane;
  R ax = cx[0], ay = cy[0], bx = cx[1], by = cy[1];
  for (int t = t0; t < t1; ++t) {
    const bool second = t >= la;
    const long long e = p0 + 32LL * t;
    const VT v = LD::ld(x + base + op.pacol[e]);
    const R h = op.paval[e];
    const R tx = fma(h, v.x, second ? bx : ax);
    const R ty = fma(h, v.y, second ? by : ay);
    ax = second ? ax : tx;
    ay = second ? ay : ty;
    bx = second ? tx : bx;
    by = second ? ty : by;
  }
  cx[0] = ax;
  cy[0] = ay;
  cx[1] = bx;
  cy[1] = by;
}

// Element (i, j) once C is complete: the diagonal and the jumps; returns
// (L x)_(i,j) or (L^H x)_(i,j).
template <class R, class VT, bool ADJ, class LD = LdGlobal>
__device__ __forceinline__ void mf_tail(const MfOp<R>& op, const VT* __restrict__ x, int i, int j,
                                        R cx, R cy, R& yx, R& yy) {
  const long long base = (long long)op.Nt * j;
  const VT xs = LD::ld(x + base + i);
  const R dx = op.ad[i] + op.ad[j];
  const R dy = op.hw[j] - op.hw[i];
  R rx, ry;
  if (!ADJ) {   // -i C + D x
    rx = fma(dx, xs.x, fma(-dy, xs.y, cy));
    ry = fma(dx, xs.y, fma(dy, xs.x, -cx));
  } else {      // +i C + conj(D) x
    rx = fma(dx, xs.x, fma(dy, xs.y, -cy));
    ry = fma(dx, xs.y, fma(-dy, xs.x, cx));
  }
  if (i == j) {
    const int e0 = op.jrow[i], e1 = op.jrow[i + 1];
    for (int e = e0; e < e1; ++e) {
      const VT v = LD::ld(x + (long long)op.jcol[e] * (op.Nt + 1));
      const R r = op.jval[e];
      rx = fma(r, v.x, rx);
      ry = fma(r, v.y, ry);
    }
  }
  yx = rx;
  yy = ry;
}

// The rest of element (i, j): part A (added to the same accumulators), the
// diagonal and the jumps; returns (L x)_(i,j) or (L^H x)_(i,j).
template <class R, class VT, bool ADJ, class LD = LdGlobal>
__device__ __forceinline__ void mf_finish(const MfOp<R>& op, const VT* __restrict__ x, int i, int j,
                                          R cx, R cy, R& yx, R& yy) {
  const long long base = (long long)op.Nt * j;
  if (i < op.N) {
    const int e0 = op.hrow[i], e1 = op.hrow[i + 1];
    for (int e = e0; e < e1; ++e) {
      const VT v = LD::ld(x + base + op.hcol[e]);
      const R h = op.hval[e];
      cx = fma(h, v.x, cx);
      cy = fma(h, v.y, cy);
    }
  }
  mf_tail<R, VT, ADJ, LD>(op, x, i, j, cx, cy, yx, yy);
}

// Rows of one 64-row window for a lane: (prow[w0 + lane], prow[w0 + 32 + lane]),
// -1 where there is no row (past Nt, or past `last` in a Hermitian chunk).
// Paired windows list the rows so that lane l holds ranks l and 63 - l by H
// row length; the others list them in natural order (lane l: rows w0 + l and
// w0 + 32 + l).
__device__ __forceinline__ void mf_window_rows(const int* prow, int w0, int lane, int last,
                                               int* irow) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int i = prow[w0 + lane + 32 * u];
    irow[u] = (i >= 0 && i <= last) ? i : -1;
  }
}

// Work items of one matrix-free pass: 64-row chunks of the columns j.  In the
// Hermitian form only rows i <= j are computed, so column j has
// floor(j / 64) + 1 chunks and the items before column j number
// P(j) = j + 64 a(a-1)/2 + a b  (j = 64 a + b).
constexpr int kItemRows = 64;

// C for the two rows of one lane in window w0 of column j, then the element
// values y = (L x) or (L^H x) (scaled by the caller): part B (uniform), part A
// (merged over the pair when the window is paired), the diagonal and jumps.
template <class R, class VT, bool ADJ, class LD = LdGlobal, bool PA = false>
__device__ __forceinline__ void mf_window_apply(const MfOp<R>& op, const VT* __restrict__ x, int j,
                                                int w0, const int* irow, R* yx, R* yy) {
  R cx[2], cy[2];
  mf_partB<R, VT, 2, LD>(op, x, j, irow, cx, cy);
  if (op.pwin[w0 / kItemRows]) {
    mf_partA2<R, VT, LD, PA>(op, x, j, w0, irow, cx, cy);
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (irow[u] >= 0) mf_tail<R, VT, ADJ, LD>(op, x, irow[u], j, cx[u], cy[u], yx[u], yy[u]);
  } else {
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (irow[u] >= 0) mf_finish<R, VT, ADJ, LD>(op, x, irow[u], j, cx[u], cy[u], yx[u], yy[u]);
  }
}

__device__ __forceinline__ long long herm_items_before(int j) {
  const long long a = j / kItemRows, b = j % kItemRows;
  return j + kItemRows * a * (a - 1) / 2 + a * b;
}

__host__ __device__ inline long long mf_item_count(int Nt, bool herm) {
  if (!herm) return (long long)Nt * ((Nt + kItemRows - 1) / kItemRows);
  const long long a = Nt / kItemRows, b = Nt % kItemRows;
  return Nt + kItemRows * a * (a - 1) / 2 + a * b;
}

// item -> (column j, first row i0)
__device__ __forceinline__ void mf_item(long long k, int Nt, bool herm, int& j, int& i0) {
  if (!herm) {
    const int cpc = (Nt + kItemRows - 1) / kItemRows;
    j = (int)(k / cpc);
    i0 = (int)(k % cpc) * kItemRows;
    return;
  }
  int lo = 0, hi = Nt - 1;   // largest j with herm_items_before(j) <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (herm_items_before(mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  j = lo;
  i0 = (int)(k - herm_items_before(lo)) * kItemRows;
}

}  // namespace qsw
