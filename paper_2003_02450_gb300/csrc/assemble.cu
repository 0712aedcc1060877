// Superoperator assembly into CSR (paper Section 3.3, Eq. condensed_lindblads:
// L~ is built row by row straight from H and the jump list, with no Kronecker
// intermediates).
//
// Row (i, j) of L~ (vec index k = i + N~ j, column-major) holds, in increasing
// column order:
//   column (m, j), m in offdiag(H, row i) : -i(1-omega) H_im        [I (x) H]
//   column (i, m), m in offdiag(H, row j) : +i(1-omega) H_mj        [-H^T (x) I]
//   column (i, j)                         : -i(1-omega)(H_ii - H_jj) - (dtot_i + dtot_j)/2
//   column (q, q) when i == j, for every jump |i><q| of rate r : r   [L_k^* (x) L_k]
// where dtot_v is the total rate of jumps leaving v (the anticommutator term
// -1/2 {sum_k L_k^dag L_k, rho}).  This follows from Eq. vec_mappings applied
// to Eq. qsw_ss with one jump operator per arc.
//
// The adjoint L~^H (needed by the 1-norm estimator) has the same shape with the
// imaginary parts negated and the jump list transposed (|q><i| read from J^T).
//
// Row pointers have a closed form, so no device-wide scan is needed: with
// o(v) = |offdiag(H, row v)| (0 when omega = 1), O(v) = sum_{v'<v} o(v') and
// c(v) the number of jumps in row v of J (or J^T),
//   rowptr(i, j) = B(j) + i (1 + o(j)) + O(i) + [i > j] c(j),
//   B(j) = sum_{j' < j} ( N~ (1 + o(j')) + O(N~) + c(j') ).
#include "op.h"

namespace qsw {
namespace {

template <class T>
__global__ void scan_small_t(const T* __restrict__ cnt, T* __restrict__ out, int n) {
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
    out[n] = (T)acc;
  }
  __syncthreads();
  long long acc = part[t];
  for (int i = lo; i < hi; ++i) {
    out[i] = (T)acc;
    acc += cnt[i];
  }
}

struct AsmArgs {
  int N, Nt;
  long long n;
  int comm_on;
  double one_minus_omega;
  double sigma;   // +1 for L, -1 for L^H
  const double* hdiag;
  const int* hoff_rowptr;
  const int* hoff_col;
  const double* hoff_val;
  const int* j_rowptr;
  const int* j_col;
  const double* j_val;
  const double* dtot;
  const long long* blockstart;  // [Nt + 1]
  const long long* prefoff;     // [Nt + 1]
  int* rowptr;
  int* col;
  double2* val;
};

__device__ __forceinline__ int off_count(const AsmArgs& a, int v) {
  return (a.comm_on && v < a.N) ? a.hoff_rowptr[v + 1] - a.hoff_rowptr[v] : 0;
}

__global__ void block_lengths_kernel(AsmArgs a, long long* __restrict__ offc,
                                     long long* __restrict__ blen) {
  // pass 1 (offc): o(v); pass 2 uses O(N~) from prefoff
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.Nt; v += gridDim.x * blockDim.x) {
    offc[v] = off_count(a, v);
    if (blen) {
      const long long total_off = a.prefoff[a.Nt];
      blen[v] = (long long)a.Nt * (1 + off_count(a, v)) + total_off +
                (a.j_rowptr[v + 1] - a.j_rowptr[v]);
    }
  }
}

__global__ void assemble_kernel(AsmArgs a) {
  const double cm = a.sigma * a.one_minus_omega;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < a.n;
       r += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(r % a.Nt);
    const int j = (int)(r / a.Nt);
    const int oj = off_count(a, j);
    const int jc = a.j_rowptr[j + 1] - a.j_rowptr[j];
    long long pos = a.blockstart[j] + (long long)i * (1 + oj) + a.prefoff[i] + (i > j ? jc : 0);
    a.rowptr[r] = (int)pos;
    if (r == a.n - 1) a.rowptr[a.n] = (int)a.blockstart[a.Nt];

    int sa = 0, se = 0;
    if (a.comm_on && j < a.N) { sa = a.hoff_rowptr[j]; se = a.hoff_rowptr[j + 1]; }
    int ja = 0, je = 0;
    if (i == j) { ja = a.j_rowptr[i]; je = a.j_rowptr[i + 1]; }
    bool block_done = false;
    while (true) {
      const int ms = sa < se ? a.hoff_col[sa] : INT_MAX;
      const int mq = ja < je ? a.j_col[ja] : INT_MAX;
      const int nxt = ms < mq ? ms : mq;
      if (!block_done && j < nxt) {
        // block j: columns (m, j) for m in offdiag(H, row i) plus the diagonal
        int ba = 0, be = 0;
        if (a.comm_on && i < a.N) { ba = a.hoff_rowptr[i]; be = a.hoff_rowptr[i + 1]; }
        bool diag_done = false;
        const long long base = (long long)a.Nt * j;
        for (int e = ba; e <= be; ++e) {
          const int m = e < be ? a.hoff_col[e] : INT_MAX;
          if (!diag_done && i < m) {
            a.col[pos] = (int)(base + i);
            a.val[pos] = make_double2(-0.5 * (a.dtot[i] + a.dtot[j]),
                                      -cm * (a.hdiag[i] - a.hdiag[j]));
            ++pos;
            diag_done = true;
          }
          if (e < be) {
            a.col[pos] = (int)(base + m);
            a.val[pos] = make_double2(0.0, -cm * a.hoff_val[e]);
            ++pos;
          }
        }
        block_done = true;
        continue;
      }
      if (nxt == INT_MAX) break;
      if (ms < mq || (ms == mq && i < ms)) {
        a.col[pos] = (int)(i + (long long)a.Nt * ms);
        a.val[pos] = make_double2(0.0, cm * a.hoff_val[sa]);
        ++sa;
      } else {
        a.col[pos] = (int)((long long)mq * (a.Nt + 1));
        a.val[pos] = make_double2(a.j_val[ja], 0.0);
        ++ja;
      }
      ++pos;
    }
  }
}

__global__ void narrow_kernel(long long nnz, const double2* __restrict__ in, float2* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[e];
    out[e] = make_float2((float)v.x, (float)v.y);
  }
}

}  // namespace

void assemble(Op& op, bool adjoint, Csr& out) {
  cudaStream_t st = op.ctx->stream;
  GraphDev& g = op.g;
  const int Nt = g.Nt;
  AsmArgs a{};
  a.N = g.N;
  a.Nt = Nt;
  a.n = (long long)Nt * Nt;
  a.comm_on = op.omega < 1.0;
  a.one_minus_omega = 1.0 - op.omega;
  a.sigma = adjoint ? -1.0 : 1.0;
  a.hdiag = g.hdiag.as<double>();
  a.hoff_rowptr = g.hoff_rowptr.as<int>();
  a.hoff_col = g.hoff_col.as<int>();
  a.hoff_val = g.hoff_val.as<double>();
  a.j_rowptr = adjoint ? g.jt_rowptr.as<int>() : g.j_rowptr.as<int>();
  a.j_col = adjoint ? g.jt_col.as<int>() : g.j_col.as<int>();
  a.j_val = adjoint ? g.jt_val.as<double>() : g.j_val.as<double>();
  a.dtot = g.dtot.as<double>();

  DevBuf offc, prefoff, blen, bstart;
  offc.alloc(sizeof(long long) * (Nt + 1));
  prefoff.alloc(sizeof(long long) * (Nt + 1));
  blen.alloc(sizeof(long long) * (Nt + 1));
  bstart.alloc(sizeof(long long) * (Nt + 1));
  QSW_LAUNCH block_lengths_kernel<<<grid_for(Nt, 128, 4096), 128, 0, st>>>(a, offc.as<long long>(), nullptr);
  QSW_LAUNCH scan_small_t<long long><<<1, 1024, 0, st>>>(offc.as<long long>(), prefoff.as<long long>(), Nt);
  a.prefoff = prefoff.as<long long>();
  QSW_LAUNCH block_lengths_kernel<<<grid_for(Nt, 128, 4096), 128, 0, st>>>(a, offc.as<long long>(),
                                                                blen.as<long long>());
  QSW_LAUNCH scan_small_t<long long><<<1, 1024, 0, st>>>(blen.as<long long>(), bstart.as<long long>(), Nt);
  QSW_CUDA_TRY(cudaGetLastError());
  long long nnz = 0;
  QSW_CUDA_TRY(cudaMemcpyAsync(&nnz, bstart.as<long long>() + Nt, sizeof(long long),
                               cudaMemcpyDeviceToHost, st));
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  QSW_CHECK_ARG(nnz < (1LL << 31) - 1, QSW_ERR_TOO_LARGE,
                "nnz(L) = " + std::to_string(nnz) + " does not fit 32-bit CSR indices");
  a.blockstart = bstart.as<long long>();
  out.nnz = nnz;
  out.fp32 = false;
  out.rowptr.alloc(sizeof(int) * (a.n + 1));
  out.col.alloc(sizeof(int) * (nnz + 1));
  out.val.alloc(sizeof(double2) * (nnz + 1));
  a.rowptr = out.rowptr.as<int>();
  a.col = out.col.as<int>();
  a.val = out.val.as<double2>();
  QSW_LAUNCH assemble_kernel<<<grid_for(a.n, 256, 152 * 64), 256, 0, st>>>(a);
  QSW_CUDA_TRY(cudaGetLastError());
  QSW_CUDA_TRY(cudaStreamSynchronize(st));   // scratch buffers die at scope exit
}

void to_fp32(Op& op, Csr& m) {
  if (m.fp32) return;
  cudaStream_t st = op.ctx->stream;
  DevBuf v32;
  v32.alloc(sizeof(float2) * (m.nnz + 1));
  QSW_LAUNCH narrow_kernel<<<grid_for(m.nnz, 256, 152 * 64), 256, 0, st>>>(m.nnz, m.val.as<double2>(),
                                                                 v32.as<float2>());
  QSW_CUDA_TRY(cudaGetLastError());
  QSW_CUDA_TRY(cudaStreamSynchronize(st));
  m.val = std::move(v32);
  m.fp32 = true;
}

}  // namespace qsw
