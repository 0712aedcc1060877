// Global-interaction walks (G-QSW, Section 2.5.2; NM-G-QSW, Eq. nm_gqsw):
// construction of the matrix-free operator of gqsw.cuh for one omega, its
// application outside the series kernel (two passes, for the 1-norm estimator
// and qsw_apply), and the exact 1-norm.
//
// Construction is host work on N x N operators (the walk's vertex space, not
// the N~^2 superoperator): Q = -i H_tot - 1/2 sum_k L'_k^dag L'_k - 1/2 (ports),
// with H_tot = (1 - omega) H - omega H_rot and L'_k = sqrt(omega) L_k; the
// sparse product L'^dag L' is formed row by row with a dense accumulator.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>

#include "gqsw.cuh"
#include "op.h"

namespace qsw {
namespace {

using cd = std::complex<double>;

ZMat embed(const ZMat& a, int nt) {
  ZMat m = a;
  m.n = nt;
  m.rowptr.resize(nt + 1, a.rowptr.empty() ? 0 : a.rowptr.back());
  if (a.rowptr.empty()) m.rowptr.assign(nt + 1, 0);
  return m;
}

// conjugate transpose
ZMat adjoint(const ZMat& a) {
  ZMat t;
  t.n = a.n;
  t.rowptr.assign(a.n + 1, 0);
  for (int c : a.col) ++t.rowptr[c + 1];
  for (int i = 0; i < a.n; ++i) t.rowptr[i + 1] += t.rowptr[i];
  t.col.resize(a.col.size());
  t.val.resize(a.val.size());
  std::vector<int> fill(t.rowptr.begin(), t.rowptr.end() - 1);
  for (int i = 0; i < a.n; ++i)
    for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
      const int k = fill[a.col[e]]++;
      t.col[k] = i;
      t.val[k] = std::conj(a.val[e]);
    }
  return t;   // rows visited in order, so columns increase within a row
}

// alpha a + beta b (same dimension)
ZMat axpby(cd alpha, const ZMat& a, cd beta, const ZMat& b) {
  ZMat c;
  c.n = a.n;
  c.rowptr.assign(a.n + 1, 0);
  for (int i = 0; i < a.n; ++i) {
    int p = a.rowptr[i], q = b.rowptr[i];
    const int pe = a.rowptr[i + 1], qe = b.rowptr[i + 1];
    while (p < pe || q < qe) {
      int col;
      cd v;
      if (q >= qe || (p < pe && a.col[p] < b.col[q])) {
        col = a.col[p];
        v = alpha * a.val[p++];
      } else if (p >= pe || b.col[q] < a.col[p]) {
        col = b.col[q];
        v = beta * b.val[q++];
      } else {
        col = a.col[p];
        v = alpha * a.val[p++] + beta * b.val[q++];
      }
      c.col.push_back(col);
      c.val.push_back(v);
    }
    c.rowptr[i + 1] = (int)c.col.size();
  }
  return c;
}

// a^dag a.  An entry whose computed magnitude is within its own rounding
// error (16 eps times the sum of its terms' magnitudes) is dropped: such sums
// cancel exactly in exact arithmetic (the demoralised operator's Fourier
// columns of different in-neighbours are orthogonal) and would only fill Q
// with rounding residue.
ZMat gram(const ZMat& a) {
  const ZMat ah = adjoint(a);
  ZMat g;
  g.n = a.n;
  g.rowptr.assign(a.n + 1, 0);
  std::vector<cd> acc(a.n);
  std::vector<double> mag(a.n);
  std::vector<char> hit(a.n, 0);
  std::vector<int> touched;
  const double eps = 2.220446049250313e-16;
  for (int i = 0; i < a.n; ++i) {
    touched.clear();
    for (int e = ah.rowptr[i]; e < ah.rowptr[i + 1]; ++e) {   // (a^dag)_{i r} = conj(a_{r i})
      const int r = ah.col[e];
      for (int f = a.rowptr[r]; f < a.rowptr[r + 1]; ++f) {
        const int m = a.col[f];
        if (!hit[m]) {
          hit[m] = 1;
          acc[m] = 0.0;
          mag[m] = 0.0;
          touched.push_back(m);
        }
        acc[m] += ah.val[e] * a.val[f];
        mag[m] += std::abs(ah.val[e]) * std::abs(a.val[f]);
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int m : touched) {
      if (std::abs(acc[m]) > 16.0 * eps * mag[m]) {
        g.col.push_back(m);
        g.val.push_back(acc[m]);
      }
      hit[m] = 0;
    }
    g.rowptr[i + 1] = (int)g.col.size();
  }
  return g;
}

ZMat diagonal(int n, const std::vector<cd>& d) {
  ZMat m;
  m.n = n;
  m.rowptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    if (d[i] != 0.0) {
      m.col.push_back(i);
      m.val.push_back(d[i]);
    }
    m.rowptr[i + 1] = (int)m.col.size();
  }
  return m;
}

void upload_z(const ZMat& m, DevBuf& rowptr, DevBuf& col, DevBuf& v64, DevBuf& v32,
              cudaStream_t st) {
  const size_t nz = std::max<size_t>(1, m.col.size());
  rowptr.alloc(sizeof(int) * (m.n + 1));
  col.alloc(sizeof(int) * nz);
  v64.alloc(sizeof(double2) * nz);
  v32.alloc(sizeof(float2) * nz);
  std::vector<double2> d(m.val.size());
  std::vector<float2> f(m.val.size());
  for (size_t e = 0; e < m.val.size(); ++e) {
    d[e] = make_double2(m.val[e].real(), m.val[e].imag());
    f[e] = make_float2((float)m.val[e].real(), (float)m.val[e].imag());
  }
  QSW_CUDA_TRY(cudaMemcpyAsync(rowptr.p, m.rowptr.data(), sizeof(int) * (m.n + 1),
                               cudaMemcpyHostToDevice, st));
  if (!m.col.empty()) {
    QSW_CUDA_TRY(cudaMemcpyAsync(col.p, m.col.data(), sizeof(int) * m.col.size(),
                                 cudaMemcpyHostToDevice, st));
    QSW_CUDA_TRY(cudaMemcpyAsync(v64.p, d.data(), sizeof(double2) * d.size(),
                                 cudaMemcpyHostToDevice, st));
    QSW_CUDA_TRY(cudaMemcpyAsync(v32.p, f.data(), sizeof(float2) * f.size(),
                                 cudaMemcpyHostToDevice, st));
  }
  QSW_CUDA_TRY(cudaStreamSynchronize(st));   // host staging vectors go out of scope
}

void upload_d(const std::vector<double>& h, DevBuf& b, cudaStream_t st) {
  b.alloc(sizeof(double) * std::max<size_t>(1, h.size()));
  if (!h.empty())
    QSW_CUDA_TRY(cudaMemcpyAsync(b.p, h.data(), sizeof(double) * h.size(),
                                 cudaMemcpyHostToDevice, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
}

// ----------------------------------------------------------------- kernels
constexpr int kGB = 256;
constexpr int kGW = kGB / 32;

// Pass A over every element: blocks take columns j, warps 64-row windows.
template <class R>
__global__ void __launch_bounds__(kGB)
gq_pass_a_kernel(GqOp<R> op, const typename V2<R>::T* __restrict__ x, typename V2<R>::T* w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = blockIdx.x; j < op.Nt; j += gridDim.x)
    for (int a0 = warp * kItemRows; a0 < op.Nt; a0 += kGW * kItemRows) {
      int arow[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int a = a0 + lane + 32 * u;
        arow[u] = a < op.Nt ? a : -1;
      }
      gq_pass_a<R>(op, x, w, j, arow);
    }
}

// Pass B over every element: y = scale L~ x.
template <class R>
__global__ void __launch_bounds__(kGB)
gq_pass_b_kernel(GqOp<R> op, const typename V2<R>::T* __restrict__ x,
                 const typename V2<R>::T* __restrict__ w, typename V2<R>::T* __restrict__ y,
                 double scale) {
  const long long n = (long long)op.Nt * op.Nt;
  for (long long r = blockIdx.x * (long long)kGB + threadIdx.x; r < n;
       r += (long long)gridDim.x * kGB) {
    const int i = (int)(r % op.Nt), j = (int)(r / op.Nt);
    R yx, yy;
    gq_element<R>(op, x, w, i, j, yx, yy);
    typename V2<R>::T v;
    v.x = yx * (R)scale;
    v.y = yy * (R)scale;
    y[r] = v;
  }
}

// Hermitian input (the 1-norm estimator's Hermitian column): pass A forms the
// W_k and R = x Q^dag over every element, pass B the upper triangle, mirrored,
// with the diagonal's imaginary part (zero in exact arithmetic) stored as zero.
template <class R>
__global__ void __launch_bounds__(kGB)
gq_pass_ar_kernel(GqOp<R> op, const typename V2<R>::T* __restrict__ x, typename V2<R>::T* w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = blockIdx.x; j < op.Nt; j += gridDim.x)
    for (int a0 = warp * kItemRows; a0 < op.Nt; a0 += kGW * kItemRows) {
      int arow[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int a = a0 + lane + 32 * u;
        arow[u] = a < op.Nt ? a : -1;
      }
      gq_pass_a<R>(op, x, w, j, arow);
      gq_pass_a_r<R>(op, x, w, j, arow);
    }
}

template <class R>
__global__ void __launch_bounds__(kGB)
gq_pass_bh_kernel(GqOp<R> op, const typename V2<R>::T* __restrict__ x,
                  const typename V2<R>::T* __restrict__ w, typename V2<R>::T* __restrict__ y) {
  const long long n = (long long)op.Nt * op.Nt;
  for (long long r = blockIdx.x * (long long)kGB + threadIdx.x; r < n;
       r += (long long)gridDim.x * kGB) {
    const int i = (int)(r % op.Nt), j = (int)(r / op.Nt);
    if (i > j) continue;
    R yx, yy;
    gq_element_herm<R>(op, x, w, i, j, yx, yy);
    typename V2<R>::T v;
    v.x = yx;
    v.y = i == j ? (R)0 : yy;
    y[r] = v;
    if (i != j) {
      v.y = -yy;
      y[j + (long long)op.Nt * i] = v;
    }
  }
}

// ||L~||_1 for one sandwich operator without diagonal entries: column (a, b) of
// L~ is L~(|a><b|) = Q|a><b| + |a><b|Q^dag + L'|a><b|L'^dag + ports; its entries
// sit at (i, b), (a, j) and (i, j) with i, j != a, b except the shared (a, b)
// entry Q_aa + conj(Q_bb), so its 1-norm is
//   cq(a) + cq(b) + |Q_aa + conj(Q_bb)| + cl(a) cl(b) + [a = b] jout(a).
__global__ void global_colabs_kernel(int Nt, const double* __restrict__ cq,
                                     const double2* __restrict__ qdiag,
                                     const double* __restrict__ cl,
                                     const double* __restrict__ jout,
                                     unsigned long long* out_bits) {
  const long long n = (long long)Nt * Nt;
  double best = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(r % Nt), b = (int)(r / Nt);
    double s = cq[a] + cq[b] + hypot(qdiag[a].x + qdiag[b].x, qdiag[a].y - qdiag[b].y) +
               cl[a] * cl[b];
    if (a == b) s += jout[a];
    best = fmax(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(best));
}

}  // namespace

void build_global(Op& op) {
  cudaStream_t st = op.ctx->stream;
  GlobalData& G = op.gq;
  const int N = op.N, Nt = op.Nt;
  const double omega = op.omega;
  // Q = -i H_tot - 1/2 sum_k L'^dag L' - 1/2 (ports)
  ZMat Htot = embed(G.H, Nt);
  if (G.Hrot.n) Htot = axpby(1.0 - omega, Htot, -omega, embed(G.Hrot, Nt));
  else Htot = axpby(1.0 - omega, Htot, 0.0, Htot);
  ZMat Q = axpby(cd(0.0, -1.0), Htot, 0.0, Htot);
  std::vector<ZMat> Lp;
  if (omega > 0.0)
    for (const ZMat& L : G.Ls) Lp.push_back(axpby(sqrt(omega), embed(L, Nt), 0.0, embed(L, Nt)));
  for (const ZMat& L : Lp) Q = axpby(1.0, Q, -0.5, gram(L));
  std::vector<cd> pd(Nt, 0.0);
  // port jumps: source s feeds v (y_vv += rate x_ss), sink z drains v (y_zz += rate x_vv)
  std::vector<std::vector<std::pair<int, double>>> jr(Nt), jt(Nt);
  for (size_t s = 0; s < op.src_v.size(); ++s) {
    const int v = op.src_v[s], sv = N + (int)s;
    pd[sv] -= 0.5 * op.src_r[s];
    jr[v].push_back({sv, op.src_r[s]});
    jt[sv].push_back({v, op.src_r[s]});
  }
  for (size_t z = 0; z < op.snk_v.size(); ++z) {
    const int v = op.snk_v[z], zv = N + (int)op.src_v.size() + (int)z;
    pd[v] -= 0.5 * op.snk_r[z];
    jr[zv].push_back({v, op.snk_r[z]});
    jt[v].push_back({zv, op.snk_r[z]});
  }
  Q = axpby(1.0, Q, 1.0, diagonal(Nt, pd));
  const ZMat Qh = adjoint(Q);
  G.nl = (int)Lp.size();
  QSW_CHECK_ARG(G.nl <= kMaxGlobalOps, QSW_ERR_INVALID_ARG,
                "at most " + std::to_string(kMaxGlobalOps) + " Lindblad operators");
  upload_z(Q, G.q_rowptr, G.q_col, G.q_val64, G.q_val32, st);
  upload_z(Qh, G.qh_rowptr, G.qh_col, G.qh_val64, G.qh_val32, st);
  G.nnz_q = (long long)Q.col.size();
  G.nnz_l = 0;
  bool diag_free = true;
  for (int k = 0; k < G.nl; ++k) {
    upload_z(Lp[k], G.l_rowptr[k], G.l_col[k], G.l_val64[k], G.l_val32[k], st);
    upload_z(adjoint(Lp[k]), G.lh_rowptr[k], G.lh_col[k], G.lh_val64[k], G.lh_val32[k], st);
    G.nnz_l += (long long)Lp[k].col.size();
    for (int i = 0; i < Nt; ++i)
      for (int e = Lp[k].rowptr[i]; e < Lp[k].rowptr[i + 1]; ++e)
        if (Lp[k].col[e] == i && Lp[k].val[e] != 0.0) diag_free = false;
  }
  auto jumps = [&](const std::vector<std::vector<std::pair<int, double>>>& rows, DevBuf& rp,
                   DevBuf& cc, DevBuf& v64, DevBuf& v32) {
    ZMat m;
    m.n = Nt;
    m.rowptr.assign(Nt + 1, 0);
    for (int i = 0; i < Nt; ++i) {
      auto r = rows[i];
      std::sort(r.begin(), r.end());
      for (auto& e : r) {
        m.col.push_back(e.first);
        m.val.push_back(e.second);
      }
      m.rowptr[i + 1] = (int)m.col.size();
    }
    upload_z(m, rp, cc, v64, v32, st);
  };
  jumps(jr, G.j_rowptr, G.j_col, G.j_val64, G.j_val32);
  jumps(jt, G.jt_rowptr, G.jt_col, G.jt_val64, G.jt_val32);
  // exact 1-norm ingredients (one sandwich operator without diagonal entries)
  G.exact_norm = G.nl <= 1 && diag_free;
  if (G.exact_norm) {
    std::vector<double> cq(Nt, 0.0), qd(2 * Nt, 0.0), cl(Nt, 0.0), jo(Nt, 0.0);
    for (int v = 0; v < Nt; ++v) {
      for (int e = Qh.rowptr[v]; e < Qh.rowptr[v + 1]; ++e) {   // column v of Q
        if (Qh.col[e] == v) {
          const cd q = std::conj(Qh.val[e]);   // Q_vv
          qd[2 * v] = q.real();
          qd[2 * v + 1] = q.imag();
        } else {
          cq[v] += std::abs(Qh.val[e]);
        }
      }
      for (auto& e : jt[v]) jo[v] += e.second;
    }
    if (G.nl == 1) {
      const ZMat Lh = adjoint(Lp[0]);
      for (int v = 0; v < Nt; ++v)
        for (int e = Lh.rowptr[v]; e < Lh.rowptr[v + 1]; ++e) cl[v] += std::abs(Lh.val[e]);
    }
    upload_d(cq, G.cq, st);
    upload_d(qd, G.qdiag, st);
    upload_d(cl, G.cl, st);
    upload_d(jo, G.jout, st);
  }
  op.nnz_csr = 0;   // global walks are matrix-free only
}

template <class R> GqOp<R> make_gq(const Op& op, bool adjoint) {
  const GlobalData& G = op.gq;
  const bool f = sizeof(R) == sizeof(float);
  using VT = typename V2<R>::T;
  GqOp<R> o{};
  o.Nt = op.Nt;
  o.qrow = (adjoint ? G.qh_rowptr : G.q_rowptr).as<int>();
  o.qcol = (adjoint ? G.qh_col : G.q_col).as<int>();
  o.qval = static_cast<const VT*>(adjoint ? (f ? G.qh_val32.p : G.qh_val64.p)
                                          : (f ? G.q_val32.p : G.q_val64.p));
  o.nl = G.nl;
  for (int k = 0; k < G.nl; ++k) {
    o.lrow[k] = (adjoint ? G.lh_rowptr[k] : G.l_rowptr[k]).as<int>();
    o.lcol[k] = (adjoint ? G.lh_col[k] : G.l_col[k]).as<int>();
    o.lval[k] = static_cast<const VT*>(adjoint ? (f ? G.lh_val32[k].p : G.lh_val64[k].p)
                                               : (f ? G.l_val32[k].p : G.l_val64[k].p));
  }
  o.jrow = (adjoint ? G.jt_rowptr : G.j_rowptr).as<int>();
  o.jcol = (adjoint ? G.jt_col : G.j_col).as<int>();
  o.jval = static_cast<const VT*>(adjoint ? (f ? G.jt_val32.p : G.jt_val64.p)
                                          : (f ? G.j_val32.p : G.j_val64.p));
  return o;
}
template GqOp<double> make_gq<double>(const Op&, bool);
template GqOp<float> make_gq<float>(const Op&, bool);

void gq_apply64(const Op& op, bool adjoint, int cols, const double* x, double* y, double scale) {
  cudaStream_t st = op.ctx->stream;
  const GqOp<double> g = make_gq<double>(op, adjoint);
  const long long n = op.n;
  DevBuf& west = const_cast<Op&>(op).gq.west;
  west.alloc(sizeof(double2) * std::max(1, g.nl) * (size_t)n);
  const unsigned grid_a = (unsigned)std::min(op.Nt, 152 * 8);
  const unsigned grid_b = grid_for(n, kGB, 152 * 16);
  for (int c = 0; c < cols; ++c) {
    const double2* xc = reinterpret_cast<const double2*>(x) + c * n;
    double2* yc = reinterpret_cast<double2*>(y) + c * n;
    if (g.nl)
      QSW_LAUNCH gq_pass_a_kernel<double><<<grid_a, kGB, 0, st>>>(g, xc, west.as<double2>());
    QSW_LAUNCH gq_pass_b_kernel<double><<<grid_b, kGB, 0, st>>>(g, xc, west.as<double2>(), yc, scale);
  }
  QSW_CUDA_TRY(cudaGetLastError());
}

void gq_apply_herm64(const Op& op, bool adjoint, const double* x, double* y) {
  cudaStream_t st = op.ctx->stream;
  const GqOp<double> g = make_gq<double>(op, adjoint);
  const long long n = op.n;
  DevBuf& west = const_cast<Op&>(op).gq.west;
  west.alloc(sizeof(double2) * (size_t)(g.nl + 1) * (size_t)n);
  const unsigned grid_a = (unsigned)std::min(op.Nt, 152 * 8);
  const unsigned grid_b = grid_for(n, kGB, 152 * 16);
  QSW_LAUNCH gq_pass_ar_kernel<double><<<grid_a, kGB, 0, st>>>(
      g, reinterpret_cast<const double2*>(x), west.as<double2>());
  QSW_LAUNCH gq_pass_bh_kernel<double><<<grid_b, kGB, 0, st>>>(
      g, reinterpret_cast<const double2*>(x), west.as<double2>(), reinterpret_cast<double2*>(y));
  QSW_CUDA_TRY(cudaGetLastError());
}

bool global_exact_norm(const Op& op, double* one) {
  if (!op.gq.exact_norm) return false;
  cudaStream_t st = op.ctx->stream;
  DevBuf bits;
  bits.alloc(sizeof(unsigned long long));
  QSW_CUDA_TRY(cudaMemsetAsync(bits.p, 0, sizeof(unsigned long long), st));
  QSW_LAUNCH global_colabs_kernel<<<grid_for(op.n, 256, 152 * 16), 256, 0, st>>>(
      op.Nt, op.gq.cq.as<double>(), op.gq.qdiag.as<double2>(), op.gq.cl.as<double>(),
      op.gq.jout.as<double>(), bits.as<unsigned long long>());
  QSW_CUDA_TRY(cudaGetLastError());
  unsigned long long b = 0;
  QSW_CUDA_TRY(cudaMemcpyAsync(&b, bits.p, sizeof(b), cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  memcpy(one, &b, sizeof(double));
  return true;
}

// ------------------------------------------------------- NM-G-QSW (demoralised)
// Section 2.5.2 "Graph Demoralisation", in these readings: vertex v becomes
// d_v = max(1, deg_{G^u}(v)) copies; G^{uD} joins every copy of v to every copy
// of each G^u neighbour u with weight w^u / sqrt(d_v d_u); H^D = trans(1, G^{uD});
// an arc u -> v of weight w sends each copy of u to the Fourier column
// F_{d_v}[., c_v(u)] (c_v(u) = u's position among v's sorted G^u neighbours,
// F_d[j, c] = exp(2 pi i j c / d)) with amplitude w / sqrt(d_v d_u); H_rot has
// <v^{k+1}|H_rot|v^k> = i within each subspace (one pair when d = 2).
void nm_construct(int N, const int* rowptr, const int* col, const double* w, std::vector<int>& off,
                  ZMat& Hd, ZMat& Ld, ZMat& Hrot) {
  // G^u neighbours with weights max(G_vu, G_uv), sorted
  std::vector<std::vector<std::pair<int, double>>> nb(N);
  for (int v = 0; v < N; ++v)
    for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      nb[v].push_back({col[e], w[e]});
      nb[col[e]].push_back({v, w[e]});
    }
  for (auto& r : nb) {
    std::sort(r.begin(), r.end());
    std::vector<std::pair<int, double>> u;
    for (auto& e : r) {
      if (!u.empty() && u.back().first == e.first) u.back().second = std::max(u.back().second, e.second);
      else u.push_back(e);
    }
    r.swap(u);
  }
  off.assign(N + 1, 0);
  for (int v = 0; v < N; ++v) off[v + 1] = off[v] + std::max<int>(1, (int)nb[v].size());
  const int ND = off[N];
  auto dim = [&](int v) { return off[v + 1] - off[v]; };
  // H^D
  Hd = ZMat{};
  Hd.n = ND;
  Hd.rowptr.assign(ND + 1, 0);
  for (int v = 0; v < N; ++v) {
    const int dv = dim(v);
    double deg = 0.0;
    for (auto& e : nb[v]) deg += dim(e.first) * e.second / sqrt((double)dv * dim(e.first));
    for (int j = 0; j < dv; ++j) {
      const int row = off[v] + j;
      bool placed = false;
      for (auto& e : nb[v]) {
        const int u = e.first, du = dim(u);
        if (!placed && u > v) {
          Hd.col.push_back(row);
          Hd.val.push_back(deg);
          placed = true;
        }
        const double h = -e.second / sqrt((double)dv * du);
        for (int l = 0; l < du; ++l) {
          Hd.col.push_back(off[u] + l);
          Hd.val.push_back(h);
        }
      }
      if (!placed) {
        Hd.col.push_back(row);
        Hd.val.push_back(deg);
      }
      Hd.rowptr[row + 1] = (int)Hd.col.size();
    }
  }
  // L^D: rows are copies of the arc's target v, columns copies of its source u
  Ld = ZMat{};
  Ld.n = ND;
  Ld.rowptr.assign(ND + 1, 0);
  const double two_pi = 6.283185307179586476925286766559;
  for (int v = 0; v < N; ++v) {
    const int dv = dim(v);
    for (int j = 0; j < dv; ++j) {
      const int row = off[v] + j;
      for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {   // arcs u -> v, u increasing
        const int u = col[e], du = dim(u);
        int c = 0;
        while (nb[v][c].first != u) ++c;
        const std::complex<double> f = std::polar(1.0, two_pi * (double)((long long)j * c % dv) / dv);
        const std::complex<double> a = f * (w[e] / sqrt((double)dv * du));
        for (int l = 0; l < du; ++l) {
          Ld.col.push_back(off[u] + l);
          Ld.val.push_back(a);
        }
      }
      Ld.rowptr[row + 1] = (int)Ld.col.size();
    }
  }
  // H_rot
  std::vector<std::vector<std::pair<int, std::complex<double>>>> rr(ND);
  for (int v = 0; v < N; ++v) {
    const int d = dim(v), b = off[v];
    const std::complex<double> I(0.0, 1.0);
    if (d == 2) {
      rr[b + 1].push_back({b, I});
      rr[b].push_back({b + 1, -I});
    } else if (d >= 3) {
      for (int k = 0; k < d; ++k) {
        const int k1 = (k + 1) % d;
        rr[b + k1].push_back({b + k, I});
        rr[b + k].push_back({b + k1, -I});
      }
    }
  }
  Hrot = ZMat{};
  Hrot.n = ND;
  Hrot.rowptr.assign(ND + 1, 0);
  for (int i = 0; i < ND; ++i) {
    std::sort(rr[i].begin(), rr[i].end(),
              [](const std::pair<int, std::complex<double>>& x,
                 const std::pair<int, std::complex<double>>& y) { return x.first < y.first; });
    for (auto& e : rr[i]) {
      Hrot.col.push_back(e.first);
      Hrot.val.push_back(e.second);
    }
    Hrot.rowptr[i + 1] = (int)Hrot.col.size();
  }
}

namespace {

__global__ void nm_pops_kernel(int count, int N, int ND, const int* __restrict__ off,
                               const double* __restrict__ pe, double* __restrict__ p) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)count * N;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = q / N;
    const int v = (int)(q % N);
    double s = 0.0;
    for (int k = off[v]; k < off[v + 1]; ++k) s += pe[c * ND + k];
    p[q] = s;
  }
}

__global__ void nm_init_kernel(int N, int ND, const int* __restrict__ off,
                               const double* __restrict__ p, double2* __restrict__ state) {
  const long long n = (long long)ND * ND;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(r % ND), j = (int)(r / ND);
    double v = 0.0;
    if (i == j) {
      int lo = 0, hi = N - 1;   // vertex whose copies hold i
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
      }
      v = p[lo] / (double)(off[lo + 1] - off[lo]);
    }
    state[r] = make_double2(v, 0.0);
  }
}

}  // namespace

void nm_populations(const Op& op, const double* d_pe, int count, double* d_p) {
  const int N = (int)op.gq.vset_off.size() - 1;
  QSW_LAUNCH nm_pops_kernel<<<grid_for((long long)count * N, 256, 4096), 256, 0, op.ctx->stream>>>(
      count, N, op.Nt, op.gq.vset_dev.as<int>(), d_pe, d_p);
  QSW_CUDA_TRY(cudaGetLastError());
}

void nm_initial_state(const Op& op, const double* d_p, double* d_state) {
  const int N = (int)op.gq.vset_off.size() - 1;
  QSW_LAUNCH nm_init_kernel<<<grid_for(op.n, 256, 4096), 256, 0, op.ctx->stream>>>(
      N, op.Nt, op.gq.vset_dev.as<int>(), d_p, reinterpret_cast<double2*>(d_state));
  QSW_CUDA_TRY(cudaGetLastError());
}

}  // namespace qsw
