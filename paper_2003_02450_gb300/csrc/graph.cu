// Digraph normalisation on the device (paper Section 2.1-2.5).
//
//   G^T            : transpose of the adjacency (rows = source vertex).
//   OutDeg(j)      : sum_i G_ij (Eq. out_degree) -- part of the jump rates.
//   G^u            : max(G, G^T) (Section 2.1).
//   H              : trans(1, G^u) = diag(OutDeg_{G^u}) - G^u (Eq. generator_matrix),
//                    or the caller's symmetric H split into diagonal + off-diagonal.
//   J, J^T         : the jump operators as weighted arc lists.  Row i of J
//                    lists every jump |i><q| with its rate: omega * G_iq for the
//                    graph's arcs (Eq. lindblad, weighted by omega in Eq. qsw),
//                    Gamma for a source feeding i, Theta for the sink i
//                    (Eq. qsw_ss, not omega-scaled).  J^T lists them by q.
//   dtot(q)        : sum of the rates of the jumps leaving q, i.e. the diagonal
//                    of sum_k tau_k L_k^dag L_k that enters the anticommutator.
//
// All lists come out sorted by column, and every floating-point sum is taken
// in ascending index order, so the results are deterministic.
#include <algorithm>

#include "op.h"

namespace qsw {
namespace {

__global__ void count_cols_kernel(int nnz, const int* __restrict__ col, int* __restrict__ cnt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[e]], 1);
}

// Exclusive scan of cnt[0..n) into out[0..n], out[n] = total.  One block.
__global__ void scan_small_kernel(const int* __restrict__ cnt, int* __restrict__ out, int n) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int chunk = (n + blockDim.x - 1) / blockDim.x;
  const int lo = t * chunk;
  const int hi = min(n, lo + chunk);
  long long s = 0;
  for (int i = lo; i < hi; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long long acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const long long v = part[i];
      part[i] = acc;
      acc += v;
    }
    out[n] = (int)acc;
  }
  __syncthreads();
  long long acc = part[t];
  for (int i = lo; i < hi; ++i) {
    out[i] = (int)acc;
    acc += cnt[i];
  }
}

__global__ void scatter_transpose_kernel(int N, const int* __restrict__ rowptr,
                                         const int* __restrict__ col, const double* __restrict__ w,
                                         int* __restrict__ cursor, int* __restrict__ tcol,
                                         double* __restrict__ tw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int pos = atomicAdd(&cursor[col[e]], 1);
      tcol[pos] = i;
      tw[pos] = w[e];
    }
  }
}

// Insertion sort of every row segment by column (segments are short).
__global__ void sort_segments_kernel(int N, const int* __restrict__ rowptr, int* __restrict__ col,
                                     double* __restrict__ val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int lo = rowptr[i], hi = rowptr[i + 1];
    for (int a = lo + 1; a < hi; ++a) {
      const int c = col[a];
      const double v = val[a];
      int b = a - 1;
      while (b >= lo && col[b] > c) {
        col[b + 1] = col[b];
        val[b + 1] = val[b];
        --b;
      }
      col[b + 1] = c;
      val[b + 1] = v;
    }
  }
}

// |row i of G  union  row i of G^T|
__global__ void union_count_kernel(int N, const int* __restrict__ ar, const int* __restrict__ ac,
                                   const int* __restrict__ br, const int* __restrict__ bc,
                                   int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int a = ar[i], ae = ar[i + 1], b = br[i], be = br[i + 1], c = 0;
    while (a < ae || b < be) {
      const int ca = a < ae ? ac[a] : INT_MAX;
      const int cb = b < be ? bc[b] : INT_MAX;
      if (ca <= cb) ++a;
      if (cb <= ca) ++b;
      ++c;
    }
    cnt[i] = c;
  }
}

// G^u row i = max over the union; H off-diagonal = -G^u, H_ii = sum_j G^u_ij.
__global__ void laplacian_fill_kernel(int N, const int* __restrict__ ar, const int* __restrict__ ac,
                                      const double* __restrict__ aw, const int* __restrict__ br,
                                      const int* __restrict__ bc, const double* __restrict__ bw,
                                      const int* __restrict__ urow, int* __restrict__ hcol,
                                      double* __restrict__ hval, double* __restrict__ hdiag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int a = ar[i], ae = ar[i + 1], b = br[i], be = br[i + 1], pos = urow[i];
    double deg = 0.0;
    while (a < ae || b < be) {
      const int ca = a < ae ? ac[a] : INT_MAX;
      const int cb = b < be ? bc[b] : INT_MAX;
      double wa = 0.0, wb = 0.0;
      int c;
      if (ca <= cb) { wa = aw[a]; c = ca; }
      if (cb <= ca) { wb = bw[b]; c = cb; }
      if (ca <= cb) ++a;
      if (cb <= ca) ++b;
      const double wu = wa > wb ? wa : wb;
      hcol[pos] = c;
      hval[pos] = -wu;
      ++pos;
      deg += wu;
    }
    hdiag[i] = deg;
  }
}

__global__ void h_offcount_kernel(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                                  int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int c = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) c += col[e] != i;
    cnt[i] = c;
  }
}

__global__ void h_split_kernel(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ w, const int* __restrict__ orow,
                               int* __restrict__ ocol, double* __restrict__ oval,
                               double* __restrict__ hdiag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int pos = orow[i];
    double dgl = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (col[e] == i) {
        dgl = w[e];
      } else {
        ocol[pos] = col[e];
        oval[pos] = w[e];
        ++pos;
      }
    }
    hdiag[i] = dgl;
  }
}

struct PortArgs {
  int N, Nt, n_src, n_snk;
  const int* src_v;
  const double* src_r;
  const int* snk_v;
  const double* snk_r;
};

// Row lengths of J (adjoint = 0, rows = destination) or J^T (rows = source).
__global__ void jump_count_kernel(PortArgs pa, int graph_on, const int* __restrict__ grow,
                                  int* __restrict__ cnt, int adjoint) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < pa.Nt; v += gridDim.x * blockDim.x) {
    int c = 0;
    if (v < pa.N) {
      if (graph_on) c += grow[v + 1] - grow[v];
      if (!adjoint) {
        for (int s = 0; s < pa.n_src; ++s) c += pa.src_v[s] == v;
      } else {
        for (int z = 0; z < pa.n_snk; ++z) c += pa.snk_v[z] == v;
      }
    } else if (!adjoint && v >= pa.N + pa.n_src) {
      c = 1;   // sink vertex: fed by the vertex it drains
    } else if (adjoint && v < pa.N + pa.n_src) {
      c = 1;   // source vertex: feeds its vertex
    }
    cnt[v] = c;
  }
}

__global__ void jump_fill_kernel(PortArgs pa, int graph_on, double omega,
                                 const int* __restrict__ grow, const int* __restrict__ gcol,
                                 const double* __restrict__ gw, const int* __restrict__ jrow,
                                 int* __restrict__ jcol, double* __restrict__ jval, int adjoint) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < pa.Nt; v += gridDim.x * blockDim.x) {
    int pos = jrow[v];
    if (v < pa.N) {
      if (graph_on) {
        for (int e = grow[v]; e < grow[v + 1]; ++e) {
          jcol[pos] = gcol[e];
          jval[pos] = omega * gw[e];
          ++pos;
        }
      }
      if (!adjoint) {
        for (int s = 0; s < pa.n_src; ++s)
          if (pa.src_v[s] == v) { jcol[pos] = pa.N + s; jval[pos] = pa.src_r[s]; ++pos; }
      } else {
        for (int z = 0; z < pa.n_snk; ++z)
          if (pa.snk_v[z] == v) { jcol[pos] = pa.N + pa.n_src + z; jval[pos] = pa.snk_r[z]; ++pos; }
      }
    } else if (!adjoint && v >= pa.N + pa.n_src) {
      const int z = v - pa.N - pa.n_src;
      jcol[pos] = pa.snk_v[z];
      jval[pos] = pa.snk_r[z];
    } else if (adjoint && v < pa.N + pa.n_src) {
      const int s = v - pa.N;
      jcol[pos] = pa.src_v[s];
      jval[pos] = pa.src_r[s];
    }
  }
}

__global__ void row_sum_kernel(int n, const int* __restrict__ rowptr, const double* __restrict__ val,
                               double* __restrict__ out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) s += val[e];
    out[v] = s;
  }
}

__global__ void prep_mf_kernel(int N, int Nt, double omw, const int* __restrict__ hrow,
                               const double* __restrict__ hval, int nnz_h, double* hval64,
                               float* hval32, const double* __restrict__ hdiag,
                               const double* __restrict__ dtot, double* ad64, float* ad32,
                               double* hw64, float* hw32, double* habs,
                               const double* __restrict__ jval, float* jval32, int nj,
                               const double* __restrict__ jtval, float* jtval32, int njt) {
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int e = t0; e < nnz_h; e += nth) {
    const double v = omw * hval[e];
    hval64[e] = v;
    hval32[e] = (float)v;
  }
  for (int v = t0; v < Nt; v += nth) {
    const double a = -0.5 * dtot[v];
    const double h = omw * hdiag[v];
    ad64[v] = a;
    ad32[v] = (float)a;
    hw64[v] = h;
    hw32[v] = (float)h;
    double s = 0.0;
    if (v < N)
      for (int e = hrow[v]; e < hrow[v + 1]; ++e) s += fabs(omw * hval[e]);
    habs[v] = s;
  }
  for (int e = t0; e < nj; e += nth) jval32[e] = (float)jval[e];
  for (int e = t0; e < njt; e += nth) jtval32[e] = (float)jtval[e];
}

// Lane order of each 64-row window of the matrix-free sweep.  Part A of C
// costs a lane the H row lengths of its two rows.  In natural order (lane l:
// rows l and 32 + l) a warp runs max_l len(l) + max_l len(32 + l) iterations;
// with the rows ranked by length (ties by index; rows past Nt rank first with
// length -1) and lane l taking ranks l and 63 - l as one merged list, it runs
// max_l (len(rank l) + len(rank 63 - l)).  The window is paired when that is
// at most 85 % of the natural cost (the merged list costs a few selects per
// term; uniform-degree windows keep the natural order).  One block of 64
// threads per window.
__global__ void window_rows_kernel(int N, int Nt, const int* __restrict__ hrow, int* prow,
                                   int* pwin, int* pmax) {
  __shared__ int len[64];
  __shared__ int by_rank[64];
  __shared__ int cost_nat[2], cost_pair;
  const int k = threadIdx.x, w0 = blockIdx.x * 64;
  const int i = w0 + k;
  len[k] = i < Nt ? (i < N ? hrow[i + 1] - hrow[i] : 0) : -1;
  if (k < 2) cost_nat[k] = 0;
  if (k == 0) cost_pair = 0;
  __syncthreads();
  int rank = 0;
  for (int q = 0; q < 64; ++q)
    rank += (len[q] < len[k]) || (len[q] == len[k] && q < k);
  by_rank[rank] = k;
  atomicMax(&cost_nat[k >> 5], len[k] > 0 ? len[k] : 0);
  __syncthreads();
  if (k < 32) {
    const int la = len[by_rank[k]], lb = len[by_rank[63 - k]];
    atomicMax(&cost_pair, (la > 0 ? la : 0) + (lb > 0 ? lb : 0));
  }
  __syncthreads();
  const bool paired = 100 * cost_pair <= 85 * (cost_nat[0] + cost_nat[1]);
  const int slot = paired ? (rank < 32 ? rank : 32 + (63 - rank)) : k;
  prow[w0 + slot] = i < Nt ? i : -1;
  if (k == 0) {
    pwin[blockIdx.x] = paired ? 1 : 0;
    pmax[blockIdx.x] = paired ? cost_pair : 0;   // longest merged list of the window
  }
}

// Paired windows' merged part-A lists, lane-interleaved: entry t of lane l
// (row a = prow[w0 + l]'s entries, then row b = prow[w0 + 32 + l]'s) at
// 32 (paoff[w] + t) + l; entries past a lane's list are zero (never read).
__global__ void pair_lists_kernel(int N, const int* __restrict__ hrow, const int* __restrict__ hcol,
                                  const double* __restrict__ hval64,
                                  const float* __restrict__ hval32, const int* __restrict__ prow,
                                  const int* __restrict__ pwin, const int* __restrict__ paoff,
                                  int* __restrict__ pacol, double* __restrict__ paval64,
                                  float* __restrict__ paval32) {
  const int w = blockIdx.x, l = threadIdx.x;
  if (!pwin[w]) return;
  const int a = prow[64 * w + l], b = prow[64 * w + 32 + l];
  const int ea = (a >= 0 && a < N) ? hrow[a] : 0;
  const int la = (a >= 0 && a < N) ? hrow[a + 1] - ea : 0;
  const int eb = (b >= 0 && b < N) ? hrow[b] : 0;
  const int lb = (b >= 0 && b < N) ? hrow[b + 1] - eb : 0;
  const int m = paoff[w + 1] - paoff[w];
  for (int t = 0; t < m; ++t) {
    const long long d = 32LL * (paoff[w] + t) + l;
    const int e = t < la ? ea + t : eb + (t - la);
    const bool live = t < la + lb;
    pacol[d] = live ? hcol[e] : 0;
    paval64[d] = live ? hval64[e] : 0.0;
    paval32[d] = live ? hval32[e] : 0.0f;
  }
}

template <class T>
void upload(DevBuf& b, const std::vector<T>& h, cudaStream_t st) {
  b.alloc(sizeof(T) * (h.size() ? h.size() : 1));
  if (!h.empty())
    QSW_CUDA_TRY(cudaMemcpyAsync(b.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
}

// cnt[0..n) -> rowptr[0..n] on the device.  The totals that size the
// following allocations are known on the host (see the callers), so the build
// issues its kernels without waiting for read-backs.
void scan_counts(DevBuf& cnt, DevBuf& rowptr, int n, cudaStream_t st) {
  rowptr.alloc(sizeof(int) * (n + 1));
  QSW_LAUNCH scan_small_kernel<<<1, 1024, 0, st>>>(cnt.as<int>(), rowptr.as<int>(), n);
  QSW_CUDA_TRY(cudaGetLastError());
}

// Off-diagonal entries of G^u = max(G, G^T) (union_count_kernel's total):
// rows of G and of its transpose merged, counting distinct columns.  O(nnz).
int undirected_offdiag(int N, const std::vector<int>& rowptr, const std::vector<int>& col,
                       std::vector<int>& rowlen) {
  std::vector<int> tr(N + 1, 0), tc(col.size());
  for (int c : col) ++tr[c + 1];
  for (int i = 0; i < N; ++i) tr[i + 1] += tr[i];
  std::vector<int> fill(tr.begin(), tr.end() - 1);
  for (int i = 0; i < N; ++i)
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) tc[fill[col[e]]++] = i;   // rows in order
  long long total = 0;
  rowlen.assign(N, 0);
  for (int i = 0; i < N; ++i) {
    int a = rowptr[i], b = tr[i];
    while (a < rowptr[i + 1] || b < tr[i + 1]) {
      const int ca = a < rowptr[i + 1] ? col[a] : INT_MAX;
      const int cb = b < tr[i + 1] ? tc[b] : INT_MAX;
      if (ca <= cb) ++a;
      if (cb <= ca) ++b;
      ++total;
      ++rowlen[i];
    }
  }
  return (int)total;
}

}  // namespace

void build_graph(Op& op) {
  cudaStream_t st = op.ctx->stream;
  GraphDev& g = op.g;
  g.N = op.N;
  g.Nt = op.Nt;
  g.nnz_g = (int)op.g_col.size();
  g.n_src = (int)op.src_v.size();
  g.n_snk = (int)op.snk_v.size();
  const int N = g.N;
  upload(g.g_rowptr, op.g_rowptr, st);
  upload(g.g_col, op.g_col, st);
  upload(g.g_w, op.g_w, st);
  upload(g.src_v, op.src_v, st);
  upload(g.src_r, op.src_r, st);
  upload(g.snk_v, op.snk_v, st);
  upload(g.snk_r, op.snk_r, st);

  // G^T: count per column, scan, scatter, sort segments.
  g.scratch.alloc(sizeof(int) * (g.Nt + 1));
  QSW_CUDA_TRY(cudaMemsetAsync(g.scratch.p, 0, sizeof(int) * (N + 1), st));
  if (g.nnz_g)
    QSW_LAUNCH count_cols_kernel<<<grid_for(g.nnz_g, 256, 4096), 256, 0, st>>>(g.nnz_g, g.g_col.as<int>(),
                                                                     g.scratch.as<int>());
  scan_counts(g.scratch, g.gt_rowptr, N, st);   // total: nnz(G)
  g.gt_col.alloc(sizeof(int) * (g.nnz_g + 1));
  g.gt_w.alloc(sizeof(double) * (g.nnz_g + 1));
  QSW_CUDA_TRY(cudaMemcpyAsync(g.scratch.p, g.gt_rowptr.p, sizeof(int) * N,
                               cudaMemcpyDeviceToDevice, st));
  QSW_LAUNCH scatter_transpose_kernel<<<grid_for(N, 128, 4096), 128, 0, st>>>(
      N, g.g_rowptr.as<int>(), g.g_col.as<int>(), g.g_w.as<double>(), g.scratch.as<int>(),
      g.gt_col.as<int>(), g.gt_w.as<double>());
  QSW_LAUNCH sort_segments_kernel<<<grid_for(N, 128, 4096), 128, 0, st>>>(N, g.gt_rowptr.as<int>(),
                                                               g.gt_col.as<int>(), g.gt_w.as<double>());
  QSW_CUDA_TRY(cudaGetLastError());

  // Hamiltonian.
  g.hdiag.alloc(sizeof(double) * g.Nt);
  QSW_CUDA_TRY(cudaMemsetAsync(g.hdiag.p, 0, sizeof(double) * g.Nt, st));
  if (!op.h_given) {
    QSW_LAUNCH union_count_kernel<<<grid_for(N, 128, 4096), 128, 0, st>>>(
        N, g.g_rowptr.as<int>(), g.g_col.as<int>(), g.gt_rowptr.as<int>(), g.gt_col.as<int>(),
        g.scratch.as<int>());
    scan_counts(g.scratch, g.hoff_rowptr, N, st);
    g.nnz_hoff = undirected_offdiag(N, op.g_rowptr, op.g_col, g.hlen);
    g.hoff_col.alloc(sizeof(int) * (g.nnz_hoff + 1));
    g.hoff_val.alloc(sizeof(double) * (g.nnz_hoff + 1));
    QSW_LAUNCH laplacian_fill_kernel<<<grid_for(N, 128, 4096), 128, 0, st>>>(
        N, g.g_rowptr.as<int>(), g.g_col.as<int>(), g.g_w.as<double>(), g.gt_rowptr.as<int>(),
        g.gt_col.as<int>(), g.gt_w.as<double>(), g.hoff_rowptr.as<int>(), g.hoff_col.as<int>(),
        g.hoff_val.as<double>(), g.hdiag.as<double>());
  } else {
    DevBuf hr, hc, hw;
    upload(hr, op.h_rowptr, st);
    upload(hc, op.h_col, st);
    upload(hw, op.h_w, st);
    QSW_LAUNCH h_offcount_kernel<<<grid_for(N, 128, 4096), 128, 0, st>>>(N, hr.as<int>(), hc.as<int>(),
                                                               g.scratch.as<int>());
    scan_counts(g.scratch, g.hoff_rowptr, N, st);
    g.nnz_hoff = 0;   // h_offcount_kernel's total: entries off the diagonal
    g.hlen.assign(N, 0);
    for (int i = 0; i < N; ++i)
      for (int e = op.h_rowptr[i]; e < op.h_rowptr[i + 1]; ++e)
        if (op.h_col[e] != i) {
          ++g.nnz_hoff;
          ++g.hlen[i];
        }
    g.hoff_col.alloc(sizeof(int) * (g.nnz_hoff + 1));
    g.hoff_val.alloc(sizeof(double) * (g.nnz_hoff + 1));
    QSW_LAUNCH h_split_kernel<<<grid_for(N, 128, 4096), 128, 0, st>>>(
        N, hr.as<int>(), hc.as<int>(), hw.as<double>(), g.hoff_rowptr.as<int>(),
        g.hoff_col.as<int>(), g.hoff_val.as<double>(), g.hdiag.as<double>());
    // hr/hc/hw are freed in stream order after h_split_kernel
  }
  QSW_CUDA_TRY(cudaGetLastError());
}

void build_jumps(Op& op) {
  cudaStream_t st = op.ctx->stream;
  GraphDev& g = op.g;
  const int Nt = g.Nt;
  const int graph_on = op.omega > 0.0;
  PortArgs pa{g.N, Nt, g.n_src, g.n_snk, g.src_v.as<int>(), g.src_r.as<double>(),
              g.snk_v.as<int>(), g.snk_r.as<double>()};
  // jump_count_kernel's total, either direction: one jump per arc when the
  // graph terms are on, plus one per port
  const int total = (graph_on ? g.nnz_g : 0) + g.n_src + g.n_snk;
  for (int adjoint = 0; adjoint < 2; ++adjoint) {
    DevBuf& rp = adjoint ? g.jt_rowptr : g.j_rowptr;
    DevBuf& cl = adjoint ? g.jt_col : g.j_col;
    DevBuf& vl = adjoint ? g.jt_val : g.j_val;
    const int* grow = adjoint ? g.gt_rowptr.as<int>() : g.g_rowptr.as<int>();
    const int* gcol = adjoint ? g.gt_col.as<int>() : g.g_col.as<int>();
    const double* gw = adjoint ? g.gt_w.as<double>() : g.g_w.as<double>();
    QSW_LAUNCH jump_count_kernel<<<grid_for(Nt, 128, 4096), 128, 0, st>>>(pa, graph_on, grow,
                                                               g.scratch.as<int>(), adjoint);
    QSW_CUDA_TRY(cudaGetLastError());
    scan_counts(g.scratch, rp, Nt, st);
    cl.alloc(sizeof(int) * (total + 1));
    vl.alloc(sizeof(double) * (total + 1));
    QSW_LAUNCH jump_fill_kernel<<<grid_for(Nt, 128, 4096), 128, 0, st>>>(pa, graph_on, op.omega, grow, gcol,
                                                              gw, rp.as<int>(), cl.as<int>(),
                                                              vl.as<double>(), adjoint);
    QSW_CUDA_TRY(cudaGetLastError());
  }
  g.n_jumps = total;
  g.dtot.alloc(sizeof(double) * Nt);
  QSW_LAUNCH row_sum_kernel<<<grid_for(Nt, 128, 4096), 128, 0, st>>>(Nt, g.jt_rowptr.as<int>(),
                                                          g.jt_val.as<double>(), g.dtot.as<double>());
  QSW_CUDA_TRY(cudaGetLastError());
}

void prep_matfree(Op& op) {
  cudaStream_t st = op.ctx->stream;
  GraphDev& g = op.g;
  MfData& m = op.mf;
  const int Nt = g.Nt, nh = std::max(1, g.nnz_hoff), nj = std::max(1, g.n_jumps);
  m.hval64.alloc(sizeof(double) * nh);
  m.hval32.alloc(sizeof(float) * nh);
  m.ad64.alloc(sizeof(double) * Nt);
  m.ad32.alloc(sizeof(float) * Nt);
  m.hw64.alloc(sizeof(double) * Nt);
  m.hw32.alloc(sizeof(float) * Nt);
  m.habs.alloc(sizeof(double) * Nt);
  m.jval32.alloc(sizeof(float) * nj);
  m.jtval32.alloc(sizeof(float) * nj);
  const double omw = 1.0 - op.omega;
  QSW_LAUNCH prep_mf_kernel<<<grid_for(std::max(g.nnz_hoff, Nt), 256, 1024), 256, 0, st>>>(
      g.N, Nt, omw, g.hoff_rowptr.as<int>(), g.hoff_val.as<double>(), g.nnz_hoff,
      m.hval64.as<double>(), m.hval32.as<float>(), g.hdiag.as<double>(), g.dtot.as<double>(),
      m.ad64.as<double>(), m.ad32.as<float>(), m.hw64.as<double>(), m.hw32.as<float>(),
      m.habs.as<double>(), g.j_val.as<double>(), m.jval32.as<float>(), g.n_jumps,
      g.jt_val.as<double>(), m.jtval32.as<float>(), g.n_jumps);
  QSW_CUDA_TRY(cudaGetLastError());
  const int nwin = (Nt + 63) / 64;
  m.prow.alloc(sizeof(int) * 64 * (size_t)nwin);
  m.pwin.alloc(sizeof(int) * (size_t)nwin);
  m.pmax.alloc(sizeof(int) * (size_t)nwin);
  const int nh_rows = op.omega < 1.0 ? g.N : 0;
  QSW_LAUNCH window_rows_kernel<<<nwin, 64, 0, st>>>(nh_rows, Nt, g.hoff_rowptr.as<int>(),
                                                     m.prow.as<int>(), m.pwin.as<int>(),
                                                     m.pmax.as<int>());
  QSW_CUDA_TRY(cudaGetLastError());
  m.pa_ready = false;   // the interleaved lists follow these values: built on first use
  // entries of the CSR form: diagonal + commutator stripes/blocks + one per jump
  const long long n = (long long)Nt * Nt;
  op.nnz_csr = n + (op.omega < 1.0 ? 2LL * Nt * g.nnz_hoff : 0LL) + g.n_jumps;
}

void ensure_pair_lists(Op& op) {
  MfData& m = op.mf;
  if (m.pa_ready) return;
  cudaStream_t st = op.ctx->stream;
  const GraphDev& g = op.g;
  const int nwin = (g.Nt + 63) / 64;
  const int nh_rows = op.omega < 1.0 ? g.N : 0;
  // offsets by a scan on the device; the storage is sized on the host,
  // without a read-back, by a bound: a window's longest merged list is at
  // most its two longest rows together
  m.paoff.alloc(sizeof(int) * ((size_t)nwin + 1));
  QSW_LAUNCH scan_small_kernel<<<1, 1024, 0, st>>>(m.pmax.as<int>(), m.paoff.as<int>(), nwin);
  QSW_CUDA_TRY(cudaGetLastError());
  long long bound = 0;
  QSW_CHECK_ARG((int)g.hlen.size() >= nh_rows, QSW_ERR_CUDA, "H row lengths missing on the host");
  for (int w = 0; w < nwin && nh_rows > 0; ++w) {
    int top1 = 0, top2 = 0;
    for (int i = 64 * w; i < std::min(64 * w + 64, nh_rows); ++i) {
      const int l = g.hlen[i];
      if (l > top1) {
        top2 = top1;
        top1 = l;
      } else if (l > top2) {
        top2 = l;
      }
    }
    bound += top1 + top2;
  }
  const size_t pe = 32 * (size_t)std::max(1LL, bound);
  m.pacol.alloc(sizeof(int) * pe);
  m.paval64.alloc(sizeof(double) * pe);
  m.paval32.alloc(sizeof(float) * pe);
  QSW_LAUNCH pair_lists_kernel<<<nwin, 32, 0, st>>>(
      nh_rows, g.hoff_rowptr.as<int>(), g.hoff_col.as<int>(), m.hval64.as<double>(),
      m.hval32.as<float>(), m.prow.as<int>(), m.pwin.as<int>(), m.paoff.as<int>(),
      m.pacol.as<int>(), m.paval64.as<double>(), m.paval32.as<float>());
  QSW_CUDA_TRY(cudaGetLastError());
  m.pa_ready = true;
}

}  // namespace qsw
